// layout.cu -- the intermediate step of Sec. 4.2 on the device.
//
// * Canonical component ids: components sorted by level descending, then
//   size descending (Sec. 4.2), ties by smallest vertex ascending.  Two
//   stable radix sorts (size, then level) over the component list, which is
//   built in ascending smallest-vertex order.
// * Permutation: vertices ordered by (component id, wave descending,
//   internal in-degree ascending, out-degree descending, vertex id).  Each
//   component is a contiguous range; inside a CAC the wave order is a
//   topological order (an edge v -> w inside a CAC has wave(v) > wave(w)),
//   so runs of equal wave ("sub-levels") can be solved one after the other
//   in a single pass, as the CAC BFS of Sec. 4.3.1 does.  Rows of similar
//   in-degree side by side give the 32 lanes of a warp rows of similar
//   length, and make the in-degree-class order of the grid-wide sweeps the
//   position order itself (their per-row reads and writes coalesce); among
//   equal in-degrees the out-degree key puts the entries of z that the sweeps
//   gather most often next to each other.
// * Per permuted vertex: internal in-edges (same component) and external
//   in-edges (from components of higher levels), both as permuted source
//   positions in CSC order; these are the edge lists "within each component"
//   and "between levels" of Sec. 4.2.
// * Per level: the components split by size class (grid-wide / one CTA /
//   one warp / 1-vertex collection; Sec. 4.2 groups the 1-vertex components
//   of a level together).
#include <algorithm>

#include "common.cuh"
#include "spmv.cuh"

namespace prgb {

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

static unsigned grid1(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  int64_t cap = (int64_t)num_sms() * 16;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}
static unsigned gridw(int64_t n) {
  int64_t g = (n * 32 + kBlock - 1) / kBlock;
  int64_t cap = (int64_t)num_sms() * 16;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

__global__ void csize_k(int32_t n, const int32_t* crep, const int32_t* level, int32_t* csize, uint8_t* isrep,
                        Ctl* ctl) {
  // lanes of the same component share one atomic; one level maximum per warp
  int lmax = -1;
  const int lane = threadIdx.x & 31;
  for (int64_t vb = gtid() - lane; vb < n; vb += gstride()) {
    const int64_t v = vb + lane;
    const int r = v < n ? crep[v] : -1;
    const unsigned same = __match_any_sync(0xffffffffu, r);
    if (r >= 0 && lane == __ffs(same) - 1) atomicAdd(&csize[r], __popc(same));
    if (v < n) {
      isrep[v] = r == (int32_t)v;
      lmax = max(lmax, level[v]);
    }
  }
  lmax = __reduce_max_sync(0xffffffffu, lmax);
  if (lane == 0 && lmax >= 0) atomicMax(&ctl->cnt[5], lmax);
}

__global__ void compact_reps_k(int32_t n, const uint8_t* isrep, const int32_t* ridx, const int32_t* csize,
                               uint32_t* keys, uint32_t* vals) {
  for (int64_t v = gtid(); v < n; v += gstride()) {
    if (isrep[v]) {
      const int k = ridx[v];
      vals[k] = (uint32_t)v;
      keys[k] = (uint32_t)(n - csize[v]);  // size descending
    }
  }
}

__global__ void level_keys_k(int32_t K, const uint32_t* vals, const int32_t* level, int32_t maxl, uint32_t* keys) {
  for (int64_t k = gtid(); k < K; k += gstride()) keys[k] = (uint32_t)(maxl - level[vals[k]]);
}

__global__ void comp_of_rep_k(int32_t K, const uint32_t* vals, int32_t* comp_of_rep) {
  for (int64_t k = gtid(); k < K; k += gstride()) comp_of_rep[vals[k]] = (int32_t)k;
}

// in-edges from the same final component, per vertex: a thread per vertex
// with at most kHeavy in-edges (the others start at zero)
__global__ void int_indeg_k(int32_t n, const int32_t* __restrict__ iptr, const int32_t* __restrict__ iidx,
                            const int32_t* __restrict__ crep, int32_t* icnt_v) {
  for (int64_t v = gtid(); v < n; v += gstride()) {
    const int e0 = iptr[v], e1 = iptr[v + 1];
    int in = 0;
    if (e1 - e0 <= kHeavy) {
      const int r = crep[v];
      for (int e = e0; e < e1; e++) in += crep[iidx[e]] == r;
    }
    icnt_v[v] = in;
  }
}

// the vertices with more: a warp per chunk of kChunkH in-edges, which also
// keeps its own count (chunk_in) for the order-preserving split below
__global__ void int_indeg_heavy_k(int32_t nchunks, const int32_t* __restrict__ rows,
                                  const int32_t* __restrict__ choff, const int32_t* __restrict__ chrow,
                                  const int32_t* __restrict__ iptr, const int32_t* __restrict__ iidx,
                                  const int32_t* __restrict__ crep, int32_t* icnt_v, int32_t* chunk_in) {
  const int lane = threadIdx.x & 31;
  for (int64_t c = gtid() >> 5; c < nchunks; c += gstride() >> 5) {
    const int h = chrow[c];
    const int v = rows[h];
    const int r = crep[v];
    const int e0 = iptr[v] + ((int)c - choff[h]) * kChunkH, e1 = min(iptr[v + 1], e0 + kChunkH);
    int in = 0;
    for (int e = e0 + lane; e < e1; e += 32) in += crep[iidx[e]] == r;
    in = __reduce_add_sync(0xffffffffu, in);
    if (lane == 0) {
      chunk_in[c] = in;
      atomicAdd(&icnt_v[v], in);
    }
  }
}

// Order key of a vertex inside its component: wave descending (a CAC's
// sub-levels in topological order; one wave for all members of an SCC),
// then internal in-degree ascending (ibits, capped), then out-degree
// descending (obits, capped).
__global__ void vertex_comp_k(int32_t n, const int32_t* crep, const int32_t* comp_of_rep, const int32_t* wave,
                              int32_t maxw, const int32_t* __restrict__ outdeg, const int32_t* __restrict__ icnt_v,
                              int ibits, int obits, int32_t* comp_id, uint32_t* keys, uint32_t* vals) {
  const uint32_t imax = (1u << ibits) - 1u, omax = (1u << obits) - 1u;
  for (int64_t v = gtid(); v < n; v += gstride()) {
    comp_id[v] = comp_of_rep[crep[v]];
    const uint32_t d = min((uint32_t)outdeg[v], omax);
    const uint32_t in = min((uint32_t)icnt_v[v], imax);
    keys[v] = ((((uint32_t)(maxw - wave[v]) << ibits) | in) << obits) | (omax - d);
    vals[v] = (uint32_t)v;
  }
}

__global__ void comp_keys_k(int32_t n, const uint32_t* vals, const int32_t* comp_id, uint32_t* keys) {
  for (int64_t i = gtid(); i < n; i += gstride()) keys[i] = (uint32_t)comp_id[vals[i]];
}

__global__ void perm_tables_k(int32_t n, const uint32_t* perm_u, const int32_t* comp_id, const int32_t* wave,
                              const int32_t* outdeg, const uint8_t* type, const int32_t* level, int32_t* perm,
                              int32_t* pos, int32_t* p_outdeg, int32_t* c_off, uint8_t* c_type, int32_t* c_level,
                              uint8_t* subflag) {
  for (int64_t p = gtid(); p < n; p += gstride()) {
    const int v = (int)perm_u[p];
    perm[p] = v;
    pos[v] = (int32_t)p;
    p_outdeg[p] = outdeg[v];
    const int c = comp_id[v];
    bool first = (p == 0) || comp_id[perm_u[p - 1]] != c;
    if (first) {
      c_off[c] = (int32_t)p;
      c_type[c] = type[v];
      c_level[c] = level[v];
    }
    subflag[p] = first || wave[perm_u[p - 1]] != wave[v];
  }
}

__global__ void sub_tables_k(int32_t n, int32_t K, const uint8_t* subflag, const int32_t* subidx,
                             const int32_t* c_off, int32_t* sub_ptr, int32_t* c_sub) {
  for (int64_t p = gtid(); p < n; p += gstride())
    if (subflag[p]) sub_ptr[subidx[p]] = (int32_t)p;
  for (int64_t c = gtid(); c < K; c += gstride()) c_sub[c] = subidx[c_off[c]];
}

// internal / external in-edge counts by position
__global__ void edge_count_k(int32_t n, const int32_t* perm, const int32_t* __restrict__ iptr,
                             const int32_t* __restrict__ icnt_v, int32_t* icnt, int32_t* ecnt) {
  for (int64_t p = gtid(); p < n; p += gstride()) {
    const int v = perm[p];
    const int in = icnt_v[v];
    icnt[p] = in;
    ecnt[p] = (iptr[v + 1] - iptr[v]) - in;
  }
}

// Order-preserving split of in-edges [b, e_end) of v into internal ones
// (written from int_idx + oi) and external ones (from ext_idx + oe), as
// positions; the warp's 32 lanes take 32 edges at a time.
__device__ __forceinline__ void split_edges(int b, int e_end, int cv, int oi, int oe, const int32_t* pos,
                                            const int32_t* iidx, const int32_t* comp_id, int32_t* int_idx,
                                            int32_t* ext_idx) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  for (int base = b; base < e_end; base += 32) {
    const int e = base + lane;
    const bool ok = e < e_end;
    int u = ok ? iidx[e] : 0;
    const bool in = ok && comp_id[u] == cv;
    const bool ex = ok && !in;
    const unsigned bi = __ballot_sync(0xffffffffu, in);
    const unsigned be = __ballot_sync(0xffffffffu, ex);
    if (in) int_idx[oi + __popc(bi & lt)] = pos[u];
    if (ex) ext_idx[oe + __popc(be & lt)] = pos[u];
    oi += __popc(bi);
    oe += __popc(be);
  }
}

// a warp per permuted vertex with at most kHeavy in-edges
__global__ void edge_fill_k(int32_t n, const int32_t* perm, const int32_t* pos, const int32_t* iptr,
                            const int32_t* iidx, const int32_t* comp_id, const int32_t* int_ptr,
                            const int32_t* ext_ptr, int32_t* int_idx, int32_t* ext_idx) {
  const int64_t w0 = gtid() >> 5, nw = gstride() >> 5;
  for (int64_t p = w0; p < n; p += nw) {
    const int v = perm[p];
    const int b = iptr[v], e_end = iptr[v + 1];
    if (e_end - b > kHeavy) continue;
    split_edges(b, e_end, comp_id[v], int_ptr[p], ext_ptr[p], pos, iidx, comp_id, int_idx, ext_idx);
  }
}

// the others, a warp per chunk of kChunkH in-edges: chunk_pre (exclusive
// prefix of the chunks' internal counts) places each chunk's edges after
// those of the vertex's earlier chunks
__global__ void edge_fill_heavy_k(int32_t nchunks, const int32_t* __restrict__ rows,
                                  const int32_t* __restrict__ choff, const int32_t* __restrict__ chrow,
                                  const int32_t* __restrict__ chunk_pre, const int32_t* pos, const int32_t* iptr,
                                  const int32_t* iidx, const int32_t* comp_id, const int32_t* int_ptr,
                                  const int32_t* ext_ptr, int32_t* int_idx, int32_t* ext_idx) {
  for (int64_t c = gtid() >> 5; c < nchunks; c += gstride() >> 5) {
    const int h = chrow[c];
    const int v = rows[h];
    const int c0 = choff[h];
    const int p = pos[v];
    const int in_before = chunk_pre[c] - chunk_pre[c0];
    const int e_before = ((int)c - c0) * kChunkH;
    const int b = iptr[v] + e_before, e_end = min(iptr[v + 1], b + kChunkH);
    split_edges(b, e_end, comp_id[v], int_ptr[p] + in_before, ext_ptr[p] + e_before - in_before, pos, iidx,
                comp_id, int_idx, ext_idx);
  }
}

__device__ __forceinline__ int size_class(int sz) {
  if (sz > kCluCompMax) return 0;
  if (sz > kCtaCompMax) return 1;
  if (sz > kWarpCompMax) return 2;
  if (sz > 1) return 3;
  return 4;
}

__global__ void level_begin_k(int32_t K, const int32_t* c_level, int32_t maxl, int32_t* lvl_cbeg) {
  for (int64_t c = gtid(); c < K; c += gstride())
    if (c == 0 || c_level[c - 1] != c_level[c]) lvl_cbeg[maxl - c_level[c]] = (int32_t)c;
}

__global__ void class_begin_k(int32_t K, const int32_t* c_level, const int32_t* c_off, int32_t maxl,
                              int32_t* cls /* [nlev][kNumClasses] */) {
  // Within a level the classes do not decrease (sizes descend), so class k
  // of a level begins at the first component whose class is >= k: that is
  // c for every k in (class of c's predecessor in the level, class of c].
  // Each slot is written once; slots of classes a level lacks at its end
  // keep their initial value.
  for (int64_t c = gtid(); c < K; c += gstride()) {
    const int li = maxl - c_level[c];
    const int cl = size_class(c_off[c + 1] - c_off[c]);
    const bool first = c == 0 || c_level[c - 1] != c_level[c];
    const int pcl = first ? 0 : size_class(c_off[c] - c_off[c - 1]);
    for (int k = pcl + 1; k <= cl; k++) cls[li * kNumClasses + k] = (int)c;
  }
}

__global__ void level_ranges_k(int32_t nlev, int32_t K, const int32_t* lvl_cbeg, const int32_t* cls,
                               const int32_t* c_off, LevelRange* out) {
  for (int64_t li = gtid(); li < nlev; li += gstride()) {
    LevelRange r;
    r.cbeg = lvl_cbeg[li];
    r.cend = lvl_cbeg[li + 1];
    r.clu = min(cls[li * kNumClasses + 1], r.cend);
    r.cta = min(cls[li * kNumClasses + 2], r.cend);
    r.warp = min(cls[li * kNumClasses + 3], r.cend);
    r.single = min(cls[li * kNumClasses + 4], r.cend);
    const bool ok = r.cbeg >= 0 && r.cbeg <= K && r.cend >= 0 && r.cend <= K && r.single >= 0 && r.clu >= 0;
    r.clu_max = (ok && r.cta > r.clu) ? c_off[r.clu + 1] - c_off[r.clu] : 0;
    // a missing level leaves -1 here; the host check rejects it
    r.vbeg = ok ? c_off[r.cbeg] : -1;
    r.vsingle = ok ? c_off[r.single] : -1;
    r.vend = ok ? c_off[r.cend] : -1;
    out[li] = r;
  }
}

__global__ void pos_comp_k(int32_t n, const int32_t* perm, const int32_t* comp_id, int32_t* pc) {
  for (int64_t p = gtid(); p < n; p += gstride()) pc[p] = comp_id[perm[p]];
}

__global__ void pos_level_k(int32_t n, const int32_t* perm, const int32_t* level, int32_t maxl, int32_t* pl) {
  for (int64_t p = gtid(); p < n; p += gstride()) pl[p] = maxl - level[perm[p]];
}

__global__ void large_flags_k(int32_t K, const int32_t* c_off, uint8_t* flag) {
  for (int64_t c = gtid(); c < K; c += gstride()) flag[c] = size_class(c_off[c + 1] - c_off[c]) == 0;
}

__global__ void large_fill_k(int32_t K, const uint8_t* flag, const int32_t* lidx, const int32_t* c_off,
                             const int32_t* c_sub, const uint8_t* c_type, const int32_t* c_level, int32_t maxl,
                             const int32_t* int_ptr, const int32_t* ext_ptr, LargeComp* out) {
  for (int64_t c = gtid(); c < K; c += gstride()) {
    if (!flag[c]) continue;
    LargeComp L;
    L.c = (int32_t)c;
    L.off = c_off[c];
    L.size = c_off[c + 1] - c_off[c];
    L.type = c_type[c];
    L.sub_begin = c_sub[c];
    L.sub_end = c_sub[c + 1];
    L.level_idx = maxl - c_level[c];
    L.m_int = int_ptr[c_off[c + 1]] - int_ptr[c_off[c]];
    L.m_ext = ext_ptr[c_off[c + 1]] - ext_ptr[c_off[c]];
    L.heavy_begin = L.heavy_end = L.chunk_begin = L.chunk_end = 0;
    out[lidx[c]] = L;
  }
}

__global__ void scc_count_k(int32_t K, const uint8_t* c_type, const int32_t* c_off, Ctl* ctl) {
  int cnt = 0, verts = 0;
  for (int64_t c = gtid(); c < K; c += gstride())
    if (c_type[c] == PR_TYPE_SCC) {
      cnt++;
      verts += c_off[c + 1] - c_off[c];
    }
  if (cnt) {
    atomicAdd(&ctl->cnt[3], cnt);
    atomicAdd(&ctl->cnt[4], verts);
  }
}

// ---- SELL-32 form of the light rows of the grid-wide SCCs -----------------
// Members are ordered by internal in-degree ascending, so a component's
// light rows are [off, off + nlight) and its heavy rows the rest; a slice's
// width is the in-degree of its last row.
__global__ void sell_width_k(const int32_t* __restrict__ int_ptr, int32_t off, int32_t nlight, int32_t nsl,
                             int32_t* w32, int32_t* cost) {
  for (int64_t sl = gtid(); sl < nsl; sl += gstride()) {
    const int last = off + (int)min((int64_t)nlight - 1, sl * 32 + 31);
    const int w = int_ptr[last + 1] - int_ptr[last];
    w32[sl] = 32 * w;
    cost[sl] = w + 2;
  }
}

// Every entry of every slice is written, including the lanes of the last
// slice that lie past the component's light rows (their loads happen too;
// they read the zero slot).  Each entry is a component-local index in
// [0, pad] (pad = size: the zero slot); an internal edge from outside the
// component would mean a broken layout and is recorded instead of stored.
__global__ void sell_fill_k(const int32_t* __restrict__ int_ptr, const int32_t* __restrict__ int_idx, int32_t off,
                            int32_t nlight, int32_t pad, const int32_t* __restrict__ sptr, int32_t* sell_idx,
                            Ctl* ctl) {
  const int64_t lanes = ((int64_t)nlight + 31) / 32 * 32;
  for (int64_t i = gtid(); i < lanes; i += gstride()) {
    const int r = off + (int)i;
    const int sl = (int)(i >> 5), lane = (int)(i & 31);
    const int b = sptr[sl] + lane, w = (sptr[sl + 1] - sptr[sl]) >> 5;
    const bool row = i < nlight;
    const int e0 = row ? int_ptr[r] : 0, d = row ? int_ptr[r + 1] - e0 : 0;
    for (int k = 0; k < w; k++) {
      int q = pad;
      if (k < d) {
        q = int_idx[e0 + k] - off;
        if ((unsigned)q >= (unsigned)pad) {
          set_err(ctl, PR_EINTERNAL, 230);
          q = pad;
        }
      }
      sell_idx[b + 32 * k] = q;
    }
  }
}

pr_status build_sell(pr_partition_s* P, const std::vector<int32_t>& hrows, Arena& tmp, Ctl* ctl) {
  cudaStream_t s = tmp.stream();
  Arena& keep = *P->keep;
  // slices per SCC whose heavy rows are exactly its last rows
  int32_t nsl_all = 0;
  for (LargeComp& L : P->large) {
    L.nlight = L.size - (L.heavy_end - L.heavy_begin);
    L.sell_begin = L.sell_end = nsl_all;
    bool tail = L.type == PR_TYPE_SCC && L.nlight > 0;
    for (int32_t h = L.heavy_begin; tail && h < L.heavy_end; h++)
      tail = hrows[h] == L.off + L.nlight + (h - L.heavy_begin);
    if (!tail) continue;
    L.sell_end = nsl_all + (L.nlight + 31) / 32;
    nsl_all = L.sell_end;
  }
  // a light row has at most kHeavy in-edges, so the padded slices fit int32
  // offsets whenever 32 * kHeavy * slices does; larger graphs keep the CSC
  // sweep
  if (nsl_all == 0 || (int64_t)32 * kHeavy * nsl_all >= ((int64_t)1 << 31)) {
    for (LargeComp& L : P->large) L.sell_begin = L.sell_end = 0;
    return PR_OK;
  }
  P->nsell = nsl_all;
  int32_t *w32, *cost;
  PRGB_TRY(tmp.alloc(&w32, (size_t)nsl_all + 1));
  PRGB_TRY(tmp.alloc(&cost, (size_t)nsl_all + 1));
  PRGB_TRY(keep.alloc(&P->sell_ptr, (size_t)nsl_all + 1));
  PRGB_TRY(keep.alloc(&P->sell_cpre, (size_t)nsl_all + 1));
  for (const LargeComp& L : P->large) {
    if (L.sell_end == L.sell_begin) continue;
    sell_width_k<<<grid1(L.sell_end - L.sell_begin), kBlock, 0, s>>>(P->int_ptr, L.off, L.nlight,
                                                                     L.sell_end - L.sell_begin, w32 + L.sell_begin,
                                                                     cost + L.sell_begin);
    PRGB_LAUNCH();
  }
  PRGB_TRY(scan_i32(w32, P->sell_ptr, nsl_all, tmp));
  PRGB_TRY(scan_i32(cost, P->sell_cpre, nsl_all, tmp));
  int32_t total = 0;
  PRGB_CUDA(cudaMemcpyAsync(&total, P->sell_ptr + nsl_all, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  PRGB_TRY(keep.alloc(&P->sell_idx, (size_t)(total > 0 ? total : 1)));
  for (const LargeComp& L : P->large) {
    if (L.sell_end == L.sell_begin) continue;
    sell_fill_k<<<grid1((int64_t)(L.sell_end - L.sell_begin) * 32), kBlock, 0, s>>>(P->int_ptr, P->int_idx, L.off,
                                                                                   L.nlight, L.size,
                                                    P->sell_ptr + L.sell_begin, P->sell_idx, ctl);
    PRGB_LAUNCH();
  }
  return PR_OK;
}

pr_status build_layout(pr_partition_s* P, const int32_t* crep, const int32_t* wave, int32_t max_wave, Arena& tmp,
                       Ctl* ctl) {
  cudaStream_t s = tmp.stream();
  Arena& keep = *P->keep;
  const DevGraph& g = P->g;
  const int32_t n = g.n;
  P->n_comp = 0;
  P->n_levels = 0;
  if (n == 0) return PR_OK;
  int32_t* csize;
  uint8_t* isrep;
  int32_t* ridx;
  PRGB_TRY(tmp.alloc(&csize, n));
  PRGB_TRY(tmp.alloc(&isrep, n));
  PRGB_TRY(tmp.alloc(&ridx, (size_t)n + 1));
  PRGB_CUDA(cudaMemsetAsync(csize, 0, (size_t)n * 4, s));
  PRGB_TRY(init_ctl(ctl, s));
  csize_k<<<grid1(n), kBlock, 0, s>>>(n, crep, P->level, csize, isrep, ctl);
  PRGB_LAUNCH();
  PRGB_TRY(scan_u8(isrep, ridx, n, tmp));
  int32_t hK = 0, hmaxl = 0;
  PRGB_CUDA(cudaMemcpyAsync(&hK, ridx + n, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaMemcpyAsync(&hmaxl, &ctl->cnt[5], 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  const int32_t K = hK, maxl = hmaxl, nlev = maxl + 1;
  P->n_comp = K;
  P->n_levels = nlev;
  uint32_t *ck, *cv, *ckt, *cvt;
  PRGB_TRY(tmp.alloc(&ck, K));
  PRGB_TRY(tmp.alloc(&cv, K));
  PRGB_TRY(tmp.alloc(&ckt, K));
  PRGB_TRY(tmp.alloc(&cvt, K));
  compact_reps_k<<<grid1(n), kBlock, 0, s>>>(n, isrep, ridx, csize, ck, cv);
  PRGB_LAUNCH();
  PRGB_TRY(radix_sort_pairs(ck, cv, ckt, cvt, K, bits_for((uint32_t)n), tmp));
  level_keys_k<<<grid1(K), kBlock, 0, s>>>(K, cv, P->level, maxl, ck);
  PRGB_LAUNCH();
  PRGB_TRY(radix_sort_pairs(ck, cv, ckt, cvt, K, bits_for((uint32_t)maxl), tmp));
  int32_t* comp_of_rep;
  PRGB_TRY(tmp.alloc(&comp_of_rep, n));
  comp_of_rep_k<<<grid1(K), kBlock, 0, s>>>(K, cv, comp_of_rep);
  PRGB_LAUNCH();
  // permutation by (component, wave desc, vertex)
  uint32_t *vk, *vv, *vkt, *vvt;
  PRGB_TRY(tmp.alloc(&vk, n));
  PRGB_TRY(tmp.alloc(&vv, n));
  PRGB_TRY(tmp.alloc(&vkt, n));
  PRGB_TRY(tmp.alloc(&vvt, n));
  // the out-degree key fills the wave key's last 8-bit radix pass (at least
  // 8 bits while the wave key leaves room)
  // internal in-degrees (from the final components) for the order key and
  // the internal / external split below
  int32_t* icnt_v;
  PRGB_TRY(tmp.alloc(&icnt_v, n));
  int32_t *chunk_in = nullptr, *chunk_pre = nullptr;
  PRGB_TRY(tmp.alloc(&chunk_in, (size_t)g.nchunks + 1));
  PRGB_TRY(tmp.alloc(&chunk_pre, (size_t)g.nchunks + 1));
  int_indeg_k<<<grid1(n), kBlock, 0, s>>>(n, g.iptr, g.iidx, crep, icnt_v);
  PRGB_LAUNCH();
  if (g.nchunks > 0) {
    int_indeg_heavy_k<<<gridw(g.nchunks), kBlock, 0, s>>>(g.nchunks, g.heavy_rows, g.heavy_choff, g.heavy_chrow,
                                                          g.iptr, g.iidx, crep, icnt_v, chunk_in);
    PRGB_LAUNCH();
  }
  PRGB_TRY(scan_i32(chunk_in, chunk_pre, g.nchunks, tmp));
  // the secondary keys fill the radix passes the wave key leaves: up to 8
  // bits of in-degree and 4 of out-degree
  const int wbits = bits_for((uint32_t)max_wave);
  const int vbits = std::min(32, (wbits + 12 + 7) / 8 * 8);
  const int ibits = std::min(8, vbits - wbits);
  const int obits = std::min(4, vbits - wbits - ibits);
  vertex_comp_k<<<grid1(n), kBlock, 0, s>>>(n, crep, comp_of_rep, wave, max_wave, g.outdeg, icnt_v, ibits, obits,
                                            P->comp_id, vk, vv);
  PRGB_LAUNCH();
  PRGB_TRY(radix_sort_pairs(vk, vv, vkt, vvt, n, vbits, tmp));
  comp_keys_k<<<grid1(n), kBlock, 0, s>>>(n, vv, P->comp_id, vk);
  PRGB_LAUNCH();
  PRGB_TRY(radix_sort_pairs(vk, vv, vkt, vvt, n, bits_for((uint32_t)(K - 1)), tmp));
  int32_t* pos;
  int32_t* c_level;
  uint8_t* subflag;
  int32_t* subidx;
  PRGB_TRY(keep.alloc(&P->perm, n));
  PRGB_TRY(keep.alloc(&P->p_outdeg, n));
  PRGB_TRY(keep.alloc(&P->c_off, (size_t)K + 1));
  PRGB_TRY(keep.alloc(&P->c_sub, (size_t)K + 1));
  PRGB_TRY(keep.alloc(&P->c_type, K));
  PRGB_TRY(tmp.alloc(&pos, n));
  PRGB_TRY(tmp.alloc(&c_level, K));
  PRGB_TRY(tmp.alloc(&subflag, n));
  PRGB_TRY(tmp.alloc(&subidx, (size_t)n + 1));
  perm_tables_k<<<grid1(n), kBlock, 0, s>>>(n, vv, P->comp_id, wave, g.outdeg, P->type, P->level, P->perm, pos,
                                            P->p_outdeg, P->c_off, P->c_type, c_level, subflag);
  PRGB_LAUNCH();
  PRGB_CUDA(cudaMemcpyAsync(P->c_off + K, &n, 4, cudaMemcpyHostToDevice, s));
  PRGB_TRY(scan_u8(subflag, subidx, n, tmp));
  int32_t S = 0;
  PRGB_CUDA(cudaMemcpyAsync(&S, subidx + n, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  P->n_sub = S;
  PRGB_TRY(keep.alloc(&P->sub_ptr, (size_t)S + 1));
  sub_tables_k<<<grid1(n), kBlock, 0, s>>>(n, K, subflag, subidx, P->c_off, P->sub_ptr, P->c_sub);
  PRGB_LAUNCH();
  PRGB_CUDA(cudaMemcpyAsync(P->sub_ptr + S, &n, 4, cudaMemcpyHostToDevice, s));
  PRGB_CUDA(cudaMemcpyAsync(P->c_sub + K, &S, 4, cudaMemcpyHostToDevice, s));
  // internal / external in-edges
  int32_t *icnt, *ecnt;
  PRGB_TRY(tmp.alloc(&icnt, n));
  PRGB_TRY(tmp.alloc(&ecnt, n));
  PRGB_TRY(build_inv(P->p_outdeg, n, keep, &P->p_inv, s));
  PRGB_TRY(keep.alloc(&P->int_ptr, (size_t)n + 1));
  PRGB_TRY(keep.alloc(&P->ext_ptr, (size_t)n + 1));
  edge_count_k<<<grid1(n), kBlock, 0, s>>>(n, P->perm, g.iptr, icnt_v, icnt, ecnt);
  PRGB_LAUNCH();
  PRGB_TRY(scan_i32(icnt, P->int_ptr, n, tmp));
  PRGB_TRY(scan_i32(ecnt, P->ext_ptr, n, tmp));
  int32_t mi = 0, me = 0;
  PRGB_CUDA(cudaMemcpyAsync(&mi, P->int_ptr + n, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaMemcpyAsync(&me, P->ext_ptr + n, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  P->m_int = mi;
  P->m_ext = me;
  PRGB_TRY(keep.alloc(&P->int_idx, (size_t)(mi > 0 ? mi : 1)));
  PRGB_TRY(keep.alloc(&P->ext_idx, (size_t)(me > 0 ? me : 1)));
  edge_fill_k<<<gridw(n), kBlock, 0, s>>>(n, P->perm, pos, g.iptr, g.iidx, P->comp_id, P->int_ptr, P->ext_ptr,
                                          P->int_idx, P->ext_idx);
  PRGB_LAUNCH();
  if (g.nchunks > 0) {
    edge_fill_heavy_k<<<gridw(g.nchunks), kBlock, 0, s>>>(g.nchunks, g.heavy_rows, g.heavy_choff, g.heavy_chrow,
                                                          chunk_pre, pos, g.iptr, g.iidx, P->comp_id, P->int_ptr,
                                                          P->ext_ptr, P->int_idx, P->ext_idx);
    PRGB_LAUNCH();
  }
  // level ranges and size classes
  int32_t *lvl_cbeg, *cls;
  LevelRange* dlev;
  PRGB_TRY(tmp.alloc(&lvl_cbeg, (size_t)nlev + 1));
  PRGB_TRY(tmp.alloc(&cls, (size_t)nlev * kNumClasses));
  PRGB_TRY(tmp.alloc(&dlev, nlev));
  PRGB_CUDA(cudaMemsetAsync(lvl_cbeg, 0xff, ((size_t)nlev + 1) * 4, s));
  level_begin_k<<<grid1(K), kBlock, 0, s>>>(K, c_level, maxl, lvl_cbeg);
  PRGB_LAUNCH();
  PRGB_CUDA(cudaMemcpyAsync(lvl_cbeg + nlev, &K, 4, cudaMemcpyHostToDevice, s));
  PRGB_CUDA(cudaMemsetAsync(cls, 0x7f, (size_t)nlev * kNumClasses * 4, s));
  class_begin_k<<<grid1(K), kBlock, 0, s>>>(K, c_level, P->c_off, maxl, cls);
  PRGB_LAUNCH();
  level_ranges_k<<<grid1(nlev), kBlock, 0, s>>>(nlev, K, lvl_cbeg, cls, P->c_off, dlev);
  PRGB_LAUNCH();
  uint8_t* lflag;
  int32_t* lidx;
  PRGB_TRY(tmp.alloc(&lflag, K));
  PRGB_TRY(tmp.alloc(&lidx, (size_t)K + 1));
  large_flags_k<<<grid1(K), kBlock, 0, s>>>(K, P->c_off, lflag);
  PRGB_LAUNCH();
  PRGB_TRY(scan_u8(lflag, lidx, K, tmp));
  int32_t nlarge = 0;
  PRGB_CUDA(cudaMemcpyAsync(&nlarge, lidx + K, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaMemsetAsync(&ctl->cnt[3], 0, 8, s));
  scc_count_k<<<grid1(K), kBlock, 0, s>>>(K, P->c_type, P->c_off, ctl);
  PRGB_LAUNCH();
  int32_t hs[2] = {0, 0};
  PRGB_CUDA(cudaMemcpyAsync(hs, &ctl->cnt[3], 8, cudaMemcpyDeviceToHost, s));
  P->levels.resize(nlev);
  PRGB_CUDA(cudaMemcpyAsync(P->levels.data(), dlev, sizeof(LevelRange) * nlev, cudaMemcpyDeviceToHost, s));
  P->h_c_off.resize((size_t)K + 1);
  PRGB_CUDA(cudaMemcpyAsync(P->h_c_off.data(), P->c_off, ((size_t)K + 1) * 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  P->n_scc = hs[0];
  P->n_scc_vertices = hs[1];
  P->large.resize(nlarge);
  P->max_large = 0;
  PRGB_TRY(keep.alloc(&P->p_comp, n));
  pos_comp_k<<<grid1(n), kBlock, 0, s>>>(n, P->perm, P->comp_id, P->p_comp);
  PRGB_LAUNCH();
  if (nlarge > 0) {
    LargeComp* dl;
    PRGB_TRY(tmp.alloc(&dl, nlarge));
    large_fill_k<<<grid1(K), kBlock, 0, s>>>(K, lflag, lidx, P->c_off, P->c_sub, P->c_type, c_level, maxl,
                                             P->int_ptr, P->ext_ptr, dl);
    PRGB_LAUNCH();
    PRGB_CUDA(cudaMemcpyAsync(P->large.data(), dl, sizeof(LargeComp) * nlarge, cudaMemcpyDeviceToHost, s));
    PRGB_CUDA(cudaStreamSynchronize(s));
    for (const LargeComp& L : P->large) P->max_large = L.size > P->max_large ? L.size : P->max_large;
    // heavy rows of the internal CSC, sliced per large component, and the
    // light rows of each component ordered by in-degree class
    PRGB_TRY(build_heavy(P->int_ptr, n, keep, tmp, &P->heavy_rows, &P->heavy_choff, &P->heavy_chrow, &P->nheavy,
                          &P->nchunks));
    int32_t* pc = P->p_comp;
    PRGB_TRY(build_lorder(P->int_ptr, n, pc, K - 1, keep, tmp, &P->lorder));
    PRGB_TRY(build_lpre(P->int_ptr, P->lorder, n, P->m_int, keep, tmp, &P->lpre));
    std::vector<int32_t> hrows(P->nheavy), hcho(P->nheavy + 1);
    if (P->nheavy > 0) {
      PRGB_CUDA(cudaMemcpyAsync(hrows.data(), P->heavy_rows, (size_t)P->nheavy * 4, cudaMemcpyDeviceToHost, s));
    }
    PRGB_CUDA(cudaMemcpyAsync(hcho.data(), P->heavy_choff, ((size_t)P->nheavy + 1) * 4, cudaMemcpyDeviceToHost, s));
    PRGB_CUDA(cudaStreamSynchronize(s));
    for (LargeComp& L : P->large) {
      L.heavy_begin = (int32_t)(std::lower_bound(hrows.begin(), hrows.end(), L.off) - hrows.begin());
      L.heavy_end = (int32_t)(std::lower_bound(hrows.begin(), hrows.end(), L.off + L.size) - hrows.begin());
      L.chunk_begin = hcho[L.heavy_begin];
      L.chunk_end = hcho[L.heavy_end];
      P->max_heavy = std::max(P->max_heavy, L.heavy_end - L.heavy_begin);
      P->max_chunks = std::max(P->max_chunks, L.chunk_end - L.chunk_begin);
    }
    PRGB_TRY(build_sell(P, hrows, tmp, ctl));
  }
  PRGB_TRY(build_fx_sched(P, tmp, ctl));
  // rows with many external in-edges (the inflow gather of Eq. PR:levels)
  // and the light rows of each level ordered by external in-degree class
  {
    PRGB_TRY(build_heavy(P->ext_ptr, n, keep, tmp, &P->xheavy_rows, &P->xheavy_choff, &P->xheavy_chrow,
                         &P->nxheavy, &P->nxchunks));
    int32_t* pl;
    PRGB_TRY(tmp.alloc(&pl, n));
    pos_level_k<<<grid1(n), kBlock, 0, s>>>(n, P->perm, P->level, maxl, pl);
    PRGB_LAUNCH();
    PRGB_TRY(build_lorder(P->ext_ptr, n, pl, nlev - 1, keep, tmp, &P->xlorder));
    std::vector<int32_t> xrows(P->nxheavy), xcho(P->nxheavy + 1);
    if (P->nxheavy > 0)
      PRGB_CUDA(cudaMemcpyAsync(xrows.data(), P->xheavy_rows, (size_t)P->nxheavy * 4, cudaMemcpyDeviceToHost, s));
    PRGB_CUDA(cudaMemcpyAsync(xcho.data(), P->xheavy_choff, ((size_t)P->nxheavy + 1) * 4, cudaMemcpyDeviceToHost, s));
    PRGB_CUDA(cudaStreamSynchronize(s));
    for (LevelRange& r : P->levels) {
      r.xh_begin = (int32_t)(std::lower_bound(xrows.begin(), xrows.end(), r.vbeg) - xrows.begin());
      r.xh_end = (int32_t)(std::lower_bound(xrows.begin(), xrows.end(), r.vend) - xrows.begin());
      r.xc_begin = xcho[r.xh_begin];
      r.xc_end = xcho[r.xh_end];
      P->max_xheavy = std::max(P->max_xheavy, r.xh_end - r.xh_begin);
      P->max_xchunks = std::max(P->max_xchunks, r.xc_end - r.xc_begin);
    }
  }
  // host-side consistency checks of everything the solver will index with
  int32_t prev_end = 0, prev_vend = 0;
  for (int32_t li = 0; li < nlev; li++) {
    const LevelRange& r = P->levels[li];
    const bool ok = r.cbeg == prev_end && r.cbeg <= r.clu && r.clu <= r.cta && r.cta <= r.warp && r.warp <= r.single &&
                    r.clu_max >= 0 && r.clu_max <= kCluCompMax &&
                    r.single <= r.cend && r.cend <= K && r.cend > r.cbeg && r.vbeg == prev_vend &&
                    r.vbeg <= r.vsingle && r.vsingle <= r.vend && r.vend <= n && r.vend - r.vsingle == r.cend - r.single;
    if (!ok) return PR_EINTERNAL;
    prev_end = r.cend;
    prev_vend = r.vend;
  }
  if (prev_end != K || prev_vend != n) return PR_EINTERNAL;
  int32_t prev_li = 0;
  for (const LargeComp& L : P->large) {
    if (L.c < 0 || L.c >= K || L.off < 0 || L.size <= kCluCompMax || (int64_t)L.off + L.size > n ||
        L.sub_begin < 0 || L.sub_begin >= L.sub_end || L.sub_end > S || L.level_idx < prev_li ||
        L.level_idx >= nlev)
      return PR_EINTERNAL;
    const LevelRange& r = P->levels[L.level_idx];
    if (L.c < r.cbeg || L.c >= r.clu) return PR_EINTERNAL;
    prev_li = L.level_idx;
  }
  return PR_OK;
}

}  // namespace prgb
