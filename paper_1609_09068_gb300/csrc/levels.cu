// levels.cu -- levels (Def. 3.3) and the CAC merges of Theorem 3.1 on the
// device.
//
// The DFS of Sec. 4.1 finishes a vertex after all its successors, and then:
//   * an SCC (size >= 2) gets level 0 without external out-edges, else
//     1 + the largest level among the components it points to;
//   * a 1-vertex component v gets L = 1 + the largest level among the
//     components it points to (0 for none).  If L > 0 and no component it
//     points to at level L-1 is an SCC, v merges with all the CACs it points
//     to at level L-1 and takes level L-1; otherwise it stays at level L.
// A node's result depends only on its successors' final results, so the
// same rule runs here in Kahn order on the condensation (sinks first), one
// wave per longest-path step.  The successors' information is folded into
// one integer per node with atomicMax: 2*level + (successor is an SCC).
// The merges themselves are unions of v with its merge partners, done
// afterwards with a lock-free union-find (hook the larger root under the
// smaller), so a CAC's root is its smallest vertex.
#include "common.cuh"
#include "spmv.cuh"
#include "waves.cuh"

namespace prgb {

constexpr int kChunk = 32;  // in-edge entries per work item: one 32-lane pass of a warp

__device__ __forceinline__ int gwarp_l() { return (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); }
__device__ __forceinline__ int nwarps_l() { return (int)(((int64_t)gridDim.x * blockDim.x) >> 5); }

__global__ void count_nodes_k(const int32_t* __restrict__ optr, const int32_t* __restrict__ oidx, int32_t n,
                              const int32_t* __restrict__ rep, int32_t* nsize, int32_t* smin, int32_t* pending,
                              int32_t* cin_cnt) {
  const int lane = threadIdx.x & 31;
  // node sizes and smallest members: one thread per vertex, lanes of the
  // same node combined first (a giant SCC would otherwise take one atomic
  // per member on a single address)
  for (int64_t vb = (int64_t)gwarp_l() * 32; vb < n; vb += (int64_t)nwarps_l() * 32) {
    const int64_t v = vb + lane;
    const int U = v < n ? rep[v] : -1;
    const unsigned same = __match_any_sync(0xffffffffu, U);
    const int lead = __ffs(same) - 1;
    const int mn = __reduce_min_sync(same, (int)v);
    if (U >= 0 && lane == lead) {
      atomicAdd(&nsize[U], __popc(same));
      atomicMin(&smin[U], mn);
    }
  }
  // external out-edges: a thread per vertex with at most kHeavy out-edges
  // (the rest: count_nodes_heavy_k).  Lanes that update the same node add
  // their counts in one atomic: the giant SCC's node alone is the target of
  // about a tenth of all external edges and the source of a quarter, and
  // one atomic per edge would queue them all at one address.
  for (int64_t ub = (int64_t)gwarp_l() * 32; ub < n; ub += (int64_t)nwarps_l() * 32) {
    const int64_t u = ub + lane;
    int e0 = 0, e1 = 0, U = -1;
    if (u < n) {
      e0 = optr[u];
      e1 = optr[u + 1];
      if (e1 - e0 > kHeavy) e1 = e0;
      else U = rep[u];
    }
    int ext = 0;
    for (int e = e0; e < e1; e++) {
      const int W = rep[oidx[e]];
      const bool x = W != U;
      ext += x;
      const unsigned am = __activemask();
      const unsigned same = __match_any_sync(am, x ? W : -1);
      if (x && lane == __ffs(same) - 1) atomicAdd(&cin_cnt[W], __popc(same));
    }
    const unsigned same = __match_any_sync(0xffffffffu, ext ? U : -1);
    const int tot = __reduce_add_sync(same, ext);
    if (ext && lane == __ffs(same) - 1) atomicAdd(&pending[U], tot);
  }
}

// Edges [*e0, *e1) of chunk c of the out-heavy vertices (kChunkH edges
// each, the last one of a vertex shorter); returns the vertex.
__device__ __forceinline__ int out_chunk(const int32_t* optr, const int32_t* list, const int32_t* choff,
                                         const int32_t* chrow, int c, int* e0, int* e1) {
  const int h = chrow[c];
  const int u = list[h];
  *e0 = optr[u] + (c - choff[h]) * kChunkH;
  *e1 = min(optr[u + 1], *e0 + kChunkH);
  return u;
}

// the same for the vertices with more than kHeavy out-edges, a warp per
// chunk of kChunkH out-edges (a hub's edges spread over many warps)
__global__ void count_nodes_heavy_k(const int32_t* __restrict__ optr, const int32_t* __restrict__ oidx,
                                    const int32_t* __restrict__ list, const int32_t* __restrict__ choff,
                                    const int32_t* __restrict__ chrow, int32_t nchunks,
                                    const int32_t* __restrict__ rep, int32_t* pending, int32_t* cin_cnt) {
  const int lane = threadIdx.x & 31;
  for (int64_t c = gwarp_l(); c < nchunks; c += nwarps_l()) {
    int e0, e1;
    const int u = out_chunk(optr, list, choff, chrow, (int)c, &e0, &e1);
    const int U = rep[u];
    int ext = 0;
    for (int e = e0 + lane; e < e1; e += 32) {
      const int W = rep[oidx[e]];
      if (W != U) {
        ext++;
        atomicAdd(&cin_cnt[W], 1);
      }
    }
    ext = __reduce_add_sync(0xffffffffu, ext);
    if (lane == 0 && ext) atomicAdd(&pending[U], ext);
  }
}

// list == nullptr: a thread per vertex with at most kHeavy out-edges;
// otherwise a warp per chunk of the listed vertices' out-edges (n chunks)
__global__ void fill_cin_k(const int32_t* __restrict__ optr, const int32_t* __restrict__ oidx, int32_t n,
                           const int32_t* __restrict__ list, const int32_t* __restrict__ choff,
                           const int32_t* __restrict__ chrow, const int32_t* __restrict__ rep, int32_t* cursor,
                           int32_t* cin_src) {
  const int lane = threadIdx.x & 31;
  // lanes appending to the same node's list take their slots with one atomic
  auto append = [&](bool x, int W, int U) {
    const unsigned am = __activemask();
    const unsigned same = __match_any_sync(am, x ? W : -1);
    const int leader = __ffs(same) - 1;
    int base = 0;
    if (x && lane == leader) base = atomicAdd(&cursor[W], __popc(same));
    base = __shfl_sync(same, base, leader);
    if (x) cin_src[base + __popc(same & lanemask_lt())] = U;
  };
  if (!list) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
      const int e0 = optr[u], e1 = optr[u + 1];
      if (e1 - e0 > kHeavy) continue;
      const int U = rep[u];
      for (int e = e0; e < e1; e++) {
        const int W = rep[oidx[e]];
        append(W != U, W, U);
      }
    }
    return;
  }
  for (int64_t c = gwarp_l(); c < n; c += nwarps_l()) {
    int e0, e1;
    const int u = out_chunk(optr, list, choff, chrow, (int)c, &e0, &e1);
    const int U = rep[u];
    for (int e = e0 + lane; e < e1; e += 32) {
      const int W = rep[oidx[e]];
      append(W != U, W, U);
    }
  }
}

// finalize node X: read the folded successor key, decide level and merge.
// Returns the number of in-edge chunks to queue for the next wave.
__device__ int finalize_node(int X, int wave, const int32_t* nsize, int32_t* key, int32_t* level_node,
                             int32_t* wave_node, uint8_t* merged, const int32_t* cin_ptr) {
  const int k = atomicAdd(&key[X], 0);
  const bool scc = nsize[X] >= 2;
  int lvl = 0, m = 0;
  if (k >= 0) {
    const int L = (k >> 1) + 1;
    if (scc || (k & 1)) {
      lvl = L;
    } else {
      lvl = L - 1;
      m = 1;
    }
  }
  level_node[X] = lvl;
  wave_node[X] = wave;
  merged[X] = (uint8_t)m;
  const int len = cin_ptr[X + 1] - cin_ptr[X];
  return (len + kChunk - 1) / kChunk;
}

// fetch-and-add with acquire-release ordering at device scope: the last
// decrement of a node's pending count then sees every successor's key update
__device__ __forceinline__ int atomic_add_acq_rel(int* p, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

struct KahnK {
  const int32_t* nsize;
  int32_t *pending, *key, *level_node, *wave_node;
  uint8_t* merged;
  const int32_t *cin_ptr, *cin_src;
  __device__ void range(int X, int j, int* e0, int* e1) const {
    *e0 = cin_ptr[X] + j * kChunk;
    *e1 = min(cin_ptr[X + 1], *e0 + kChunk);
  }
  __device__ int4 pre(int X, int, bool) const {
    return make_int4(2 * level_node[X] + (nsize[X] >= 2 ? 1 : 0), 0, 0, 0);
  }
  // Lanes whose edges leave the same node U fold their keys and their
  // decrements into one atomicMax and one decrement by the group's size,
  // issued by the group's first lane; it finalizes U when the count reaches
  // zero (a node like the giant SCC has hundreds of thousands of successors,
  // and one pair of atomics per edge would queue at its two words).
  __device__ bool edge(int e, int4 p, int wave, int* w, int* nch) const {
    const int lane = threadIdx.x & 31;
    const int U = cin_src[e];
    *w = U;
    const unsigned am = __activemask();
    const unsigned same = __match_any_sync(am, U);
    const int kmax = __reduce_max_sync(same, p.x);
    const int cnt = __popc(same);
    if (lane != __ffs(same) - 1) return false;
    atomicMax(&key[U], kmax);
    if (atomic_add_acq_rel(&pending[U], -cnt) != cnt) return false;
    *nch = finalize_node(U, wave + 1, nsize, key, level_node, wave_node, merged, cin_ptr);
    return *nch > 0;
  }
};

__global__ void kahn_k(int32_t n, const int32_t* __restrict__ rep, const int32_t* __restrict__ nsize,
                       int32_t* pending, int32_t* key, int32_t* level_node, int32_t* wave_node, uint8_t* merged,
                       const int32_t* __restrict__ cin_ptr, const int32_t* __restrict__ cin_src, int* fa_node,
                       int* fa_chunk, int* fb_node, int* fb_chunk, int cap, Ctl* ctl) {
  const int lane = threadIdx.x & 31;
  const int gw = gwarp_l(), nw = nwarps_l();
  for (int64_t vb = (int64_t)gw * 32; vb < n; vb += (int64_t)nw * 32) {
    const int64_t v = vb + lane;
    int nch = 0;
    if (v < n && rep[v] == (int32_t)v && pending[v] == 0)
      nch = finalize_node((int)v, 0, nsize, key, level_node, wave_node, merged, cin_ptr);
    warp_push(nch > 0, (int)v, nch, fa_node, fa_chunk, &ctl->cnt[0], cap, ctl);
  }
  const Frontier f{fa_node, fa_chunk, fb_node, fb_chunk, cap};
  KahnK k{nsize, pending, key, level_node, wave_node, merged, cin_ptr, cin_src};
  run_waves(ctl, f, 211, kWaveKahn, k);
}

// lock-free union-find with parent[x] <= x (roots are the smallest ids)
__device__ __forceinline__ int uf_find(int* par, int v) {
  int cur = par[v];
  if (cur != v) {
    int next, prev = v;
    while (cur > (next = par[cur])) {
      par[prev] = next;
      prev = cur;
      cur = next;
    }
  }
  return cur;
}

__device__ __forceinline__ void uf_union(int* par, int a, int b) {
  int ra = uf_find(par, a), rb = uf_find(par, b);
  for (int guard = 0; ra != rb && guard < (1 << 22); guard++) {
    if (ra < rb) {
      const int ret = atomicCAS(&par[rb], rb, ra);
      if (ret == rb) break;
      rb = ret;
    } else {
      const int ret = atomicCAS(&par[ra], ra, rb);
      if (ret == ra) break;
      ra = ret;
    }
  }
}

__device__ __forceinline__ bool merges(int v, const int32_t* rep, const int32_t* nsize, const uint8_t* merged) {
  return merged[v] && rep[v] == v && nsize[v] == 1;
}

// unions of v with the 1-vertex components of its level among the targets
// of out-edges [e0, e1), in parallel lanes
__device__ __forceinline__ void merge_range(int v, int e0, int e1, const int32_t* oidx, const int32_t* rep,
                                            const int32_t* nsize, const int32_t* level_node, int* par) {
  const int lv = level_node[v];
  for (int e = e0 + (threadIdx.x & 31); e < e1; e += 32) {
    const int w = oidx[e];
    const int W = rep[w];
    if (nsize[W] == 1 && level_node[W] == lv) uf_union(par, v, w);
  }
}

// a thread per vertex finds the merging ones with at most kHeavy out-edges;
// the warp then takes each in turn
__global__ void merge_unions_k(const int32_t* __restrict__ optr, const int32_t* __restrict__ oidx, int32_t n,
                               const int32_t* __restrict__ rep, const int32_t* __restrict__ nsize,
                               const int32_t* __restrict__ level_node, const uint8_t* __restrict__ merged,
                               int* par) {
  const int lane = threadIdx.x & 31;
  for (int64_t vb = (int64_t)gwarp_l() * 32; vb < n; vb += (int64_t)nwarps_l() * 32) {
    const int64_t vl = vb + lane;
    const bool mine = vl < n && optr[vl + 1] - optr[vl] <= kHeavy && merges((int)vl, rep, nsize, merged);
    for (unsigned todo = __ballot_sync(0xffffffffu, mine); todo; todo &= todo - 1) {
      const int v = (int)vb + __ffs(todo) - 1;
      merge_range(v, optr[v], optr[v + 1], oidx, rep, nsize, level_node, par);
    }
  }
}

// the merging vertices with more out-edges: a warp per chunk of kChunkH
__global__ void merge_unions_heavy_k(const int32_t* __restrict__ optr, const int32_t* __restrict__ oidx,
                                     const int32_t* __restrict__ list, const int32_t* __restrict__ choff,
                                     const int32_t* __restrict__ chrow, int32_t nchunks,
                                     const int32_t* __restrict__ rep, const int32_t* __restrict__ nsize,
                                     const int32_t* __restrict__ level_node, const uint8_t* __restrict__ merged,
                                     int* par) {
  for (int64_t c = gwarp_l(); c < nchunks; c += nwarps_l()) {
    int e0, e1;
    const int u = out_chunk(optr, list, choff, chrow, (int)c, &e0, &e1);
    if (merges(u, rep, nsize, merged)) merge_range(u, e0, e1, oidx, rep, nsize, level_node, par);
  }
}

__global__ void finish_vertices_k(int32_t n, const int32_t* __restrict__ rep, const int32_t* __restrict__ nsize,
                                  const int32_t* __restrict__ smin, const int32_t* __restrict__ level_node,
                                  const int32_t* __restrict__ wave_node, int* par, int32_t* crep,
                                  int32_t* level, uint8_t* type, int32_t* wave, Ctl* ctl) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int X = rep[v];
    const bool scc = nsize[X] >= 2;
    crep[v] = scc ? smin[X] : uf_find(par, (int)v);
    const int lv = level_node[X];
    if (lv < 0) set_err(ctl, PR_EINTERNAL, 220);  // a node was never finalised
    level[v] = lv;
    type[v] = scc ? PR_TYPE_SCC : PR_TYPE_CAC;
    wave[v] = wave_node[X];
    atomicMax(&ctl->cnt[6], wave_node[X]);
  }
}

__global__ void iota_i32_k(int* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int)i;
}

static unsigned grid_w(int64_t n) {  // one warp per item
  int64_t g = (n * 32 + kBlock - 1) / kBlock;
  int64_t cap = (int64_t)num_sms() * 16;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}
static unsigned grid_t(int64_t n) {  // one thread per item
  int64_t g = (n + kBlock - 1) / kBlock;
  int64_t cap = (int64_t)num_sms() * 16;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

pr_status levels_and_merge(const DevGraph& g, const int32_t* rep, int32_t* crep, int32_t* level, uint8_t* type,
                           int32_t* wave, int32_t* max_wave, Arena& tmp, Ctl* ctl) {
  cudaStream_t s = tmp.stream();
  const int32_t n = g.n;
  *max_wave = 0;
  if (n == 0) return PR_OK;
  int32_t *nsize, *smin, *pending, *cin_cnt, *cin_ptr, *cursor, *cin_src, *key, *level_node, *wave_node, *par;
  uint8_t* merged;
  PRGB_TRY(tmp.alloc(&nsize, n));
  PRGB_TRY(tmp.alloc(&smin, n));
  PRGB_TRY(tmp.alloc(&pending, n));
  PRGB_TRY(tmp.alloc(&cin_cnt, n));
  PRGB_TRY(tmp.alloc(&cin_ptr, (size_t)n + 1));
  PRGB_TRY(tmp.alloc(&cursor, (size_t)n + 1));
  PRGB_TRY(tmp.alloc(&key, n));
  PRGB_TRY(tmp.alloc(&level_node, n));
  PRGB_TRY(tmp.alloc(&wave_node, n));
  PRGB_TRY(tmp.alloc(&par, n));
  PRGB_TRY(tmp.alloc(&merged, n));
  PRGB_CUDA(cudaMemsetAsync(nsize, 0, (size_t)n * 4, s));
  PRGB_CUDA(cudaMemsetAsync(smin, 0x7f, (size_t)n * 4, s));
  PRGB_CUDA(cudaMemsetAsync(pending, 0, (size_t)n * 4, s));
  PRGB_CUDA(cudaMemsetAsync(cin_cnt, 0, (size_t)n * 4, s));
  PRGB_CUDA(cudaMemsetAsync(key, 0xff, (size_t)n * 4, s));
  PRGB_CUDA(cudaMemsetAsync(level_node, 0xff, (size_t)n * 4, s));
  PRGB_CUDA(cudaMemsetAsync(wave_node, 0xff, (size_t)n * 4, s));
  PRGB_CUDA(cudaMemsetAsync(merged, 0, (size_t)n, s));
  count_nodes_k<<<grid_w(n), kBlock, 0, s>>>(g.optr, g.oidx, n, rep, nsize, smin, pending, cin_cnt);
  PRGB_LAUNCH();
  if (g.nochunks > 0) {
    count_nodes_heavy_k<<<grid_w(g.nochunks), kBlock, 0, s>>>(g.optr, g.oidx, g.oheavy, g.ochoff, g.ochrow,
                                                              g.nochunks, rep, pending, cin_cnt);
    PRGB_LAUNCH();
  }
  PRGB_TRY(scan_i32(cin_cnt, cin_ptr, n, tmp));
  // the condensation's edges number at most the graph's: sized by that
  // bound, the lists need no round trip for their exact count
  const int64_t m_ext = g.m;
  PRGB_TRY(tmp.alloc(&cin_src, (size_t)(m_ext > 0 ? m_ext : 1)));
  PRGB_CUDA(cudaMemcpyAsync(cursor, cin_ptr, ((size_t)n + 1) * 4, cudaMemcpyDeviceToDevice, s));
  fill_cin_k<<<grid_t(n), kBlock, 0, s>>>(g.optr, g.oidx, n, nullptr, nullptr, nullptr, rep, cursor, cin_src);
  PRGB_LAUNCH();
  if (g.nochunks > 0) {
    fill_cin_k<<<grid_w(g.nochunks), kBlock, 0, s>>>(g.optr, g.oidx, g.nochunks, g.oheavy, g.ochoff, g.ochrow, rep,
                                                     cursor, cin_src);
    PRGB_LAUNCH();
  }
  // frontier capacity: every node is queued once, in ceil(len/kChunk) items
  const int cap = (int)((int64_t)n + (int64_t)m_ext / kChunk + 1);
  int *fa_node, *fa_chunk, *fb_node, *fb_chunk;
  PRGB_TRY(tmp.alloc(&fa_node, cap));
  PRGB_TRY(tmp.alloc(&fa_chunk, cap));
  PRGB_TRY(tmp.alloc(&fb_node, cap));
  PRGB_TRY(tmp.alloc(&fb_chunk, cap));
  PRGB_TRY(init_ctl(ctl, s));
  {
    int32_t nn = n;
    int cp = cap;
    void* args[] = {&nn, &rep, &nsize, &pending, &key, &level_node, &wave_node, &merged, &cin_ptr, &cin_src,
                    &fa_node, &fa_chunk, &fb_node, &fb_chunk, &cp, &ctl};
    PRGB_TRY(launch_coop((const void*)kahn_k, kWaveBlock, 0, s, args, kWavePerSm, nullptr));
  }
  iota_i32_k<<<grid_t(n), kBlock, 0, s>>>(par, n);
  PRGB_LAUNCH();
  merge_unions_k<<<grid_t(n), kBlock, 0, s>>>(g.optr, g.oidx, n, rep, nsize, level_node, merged, par);
  PRGB_LAUNCH();
  if (g.nochunks > 0) {
    merge_unions_heavy_k<<<grid_w(g.nochunks), kBlock, 0, s>>>(g.optr, g.oidx, g.oheavy, g.ochoff, g.ochrow,
                                                               g.nochunks, rep, nsize, level_node, merged, par);
    PRGB_LAUNCH();
  }
  PRGB_CUDA(cudaMemsetAsync(&ctl->cnt[6], 0, sizeof(int), s));
  finish_vertices_k<<<grid_t(n), kBlock, 0, s>>>(n, rep, nsize, smin, level_node, wave_node, par, crep, level,
                                                 type, wave, ctl);
  PRGB_LAUNCH();
  int h[2] = {0, 0};
  PRGB_CUDA(cudaMemcpyAsync(&h[0], &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaMemcpyAsync(&h[1], &ctl->cnt[6], sizeof(int), cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  if (h[0]) return (pr_status)h[0];
  *max_wave = h[1];
  return PR_OK;
}

}  // namespace prgb
