// fx_sched.cu -- conflict-free slices for the fixed-point series of the level
// kernel (SCCs of 33..kFxMax vertices), built once per partition.
//
// The series gathers z[v] (16 bytes a vertex) for every in-edge of a row,
// one row per lane.  A 16-byte shared-memory load of a warp runs as four
// phases of eight consecutive lanes, and a phase takes one pass only when
// its eight addresses fall in distinct groups of four banks -- for z, when
// the eight indices differ modulo 8.  Random sources make that rare (about
// ten passes a load where four would do).  A row's fixed-point sum is exact
// in any order, so each group of eight rows is laid out here column by
// column such that no column holds two entries with the same index mod 8:
// a first-fit colouring of the bipartite multigraph (rows x index classes
// mod 8), each column a matching.  Rows that have no entry in a column read
// one of eight zero slots z[sz..sz+7], chosen among the classes the column
// leaves free, so every load of the series is conflict-free.
//
// Layout (words of four 16-bit local indices, as the level kernel reads
// them): warp w of a component (its rows 32w..32w+31) owns wcnt words a
// lane; lane l's j-th word is at slice_w + 32 j + l, slice_w the prefix of
// 32 * wcnt over the component's earlier warps, from fxs_ptr[c].
#include "common.cuh"
#include "solve.cuh"

namespace prgb {

namespace {
__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }
unsigned grid1(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  const int64_t cap = (int64_t)num_sms() * 16;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}
}  // namespace

constexpr int kSchedCols = 64;  // columns a group of eight rows may use
static_assert(kSchedCols == 8 * sizeof(unsigned long long), "one bit a column in the masks");

__device__ __forceinline__ bool fxs_component(const int32_t* c_off, const uint8_t* c_type, int c) {
  const int sz = c_off[c + 1] - c_off[c];
  return c_type[c] == PR_TYPE_SCC && sz > kWarpCompMax && sz <= kFxMax;
}

// First fit of the in-edges of the group's rows g0..g0+7 (local; rows at or
// past sz are empty).  qm[q] marks the columns holding an index of class q,
// rm[l] the columns of row l.  emit(l, col, v) sees every placement.
// Returns the number of columns, or -1 (more than kSchedCols needed, or a
// source outside the component: the layout is broken).
template <class Emit>
__device__ int fxs_greedy(const int32_t* __restrict__ int_ptr, const int32_t* __restrict__ int_idx, int off, int sz,
                          int g0, unsigned long long* qm, unsigned long long* rm, Emit emit) {
  for (int q = 0; q < 8; q++) qm[q] = 0ull;
  int ncol = 0;
  for (int l = 0; l < 8; l++) {
    rm[l] = 0ull;
    const int r = g0 + l;
    if (r >= sz) continue;
    const int p = off + r;
    for (int e = int_ptr[p]; e < int_ptr[p + 1]; e++) {
      const int v = int_idx[e] - off;
      if ((unsigned)v >= (unsigned)sz) return -1;
      const int q = v & 7;
      const unsigned long long fr = ~(rm[l] | qm[q]);
      if (fr == 0ull) return -1;
      const int col = __ffsll((long long)fr) - 1;
      rm[l] |= 1ull << col;
      qm[q] |= 1ull << col;
      ncol = max(ncol, col + 1);
      emit(l, col, v);
    }
  }
  return ncol;
}

// component of global group gid: the last c with gpre[c] <= gid
__device__ __forceinline__ int fxs_comp_of(const int32_t* gpre, int K, int gid) {
  int lo = 0, hi = K;  // gpre[lo] <= gid < gpre[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (gpre[mid] <= gid) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void fxs_groups_k(int32_t K, const int32_t* __restrict__ c_off, const uint8_t* __restrict__ c_type,
                             int32_t* __restrict__ ngroup) {
  for (int64_t c = gtid(); c < K; c += gstride()) {
    const int sz = c_off[c + 1] - c_off[c];
    ngroup[c] = fxs_component(c_off, c_type, (int)c) ? (sz + 31) / 32 * 4 : 0;
  }
}

// columns of every group (255: no schedule)
__global__ void fxs_count_k(int32_t K, int32_t G, const int32_t* __restrict__ gpre, const int32_t* __restrict__ c_off,
                            const int32_t* __restrict__ int_ptr, const int32_t* __restrict__ int_idx,
                            uint8_t* __restrict__ gcol) {
  for (int64_t gid = gtid(); gid < G; gid += gstride()) {
    const int c = fxs_comp_of(gpre, K, (int)gid);
    const int lg = (int)gid - gpre[c];
    const int off = c_off[c], sz = c_off[c + 1] - off;
    unsigned long long qm[8], rm[8];
    const int nc = fxs_greedy(int_ptr, int_idx, off, sz, 32 * (lg >> 2) + 8 * (lg & 3), qm, rm,
                              [](int, int, int) {});
    gcol[gid] = nc < 0 ? 255 : (uint8_t)nc;
  }
}

// per component: the words per lane of each warp (max over its four
// groups, in words of four columns) and the component's words, 0 when a
// group has no schedule
__global__ void fxs_comp_k(int32_t K, const int32_t* __restrict__ gpre, const uint8_t* __restrict__ gcol,
                           uint8_t* __restrict__ wcnt, int32_t* __restrict__ cwords, uint8_t* __restrict__ cok) {
  for (int64_t c = gtid(); c < K; c += gstride()) {
    const int g0 = gpre[c], ng = gpre[c + 1] - g0;
    bool ok = ng > 0;
    int words = 0;
    for (int w = 0; w < ng / 4; w++) {
      int cols = 0;
      for (int g = 0; g < 4; g++) {
        const int v = gcol[g0 + 4 * w + g];
        ok = ok && v != 255;
        cols = max(cols, v == 255 ? 0 : v);
      }
      const int wc = (cols + 3) / 4;
      wcnt[g0 / 4 + w] = (uint8_t)wc;
      words += 32 * wc;
    }
    cok[c] = ok;
    cwords[c] = ok ? words : 0;
  }
}

__global__ void fxs_ptr_k(int32_t K, const uint8_t* __restrict__ cok, const int32_t* __restrict__ cpre,
                          const int32_t* __restrict__ gpre, int32_t* __restrict__ fxs_ptr,
                          int32_t* __restrict__ fxs_wbase) {
  for (int64_t c = gtid(); c < K; c += gstride()) {
    fxs_ptr[c] = cok[c] ? cpre[c] : -1;
    fxs_wbase[c] = gpre[c] / 4;
  }
}

// the words: each group's thread places its rows' indices (lanes 8g..8g+7
// of its warp) and the zero slots of the columns' free classes
__global__ void fxs_fill_k(int32_t K, int32_t G, const int32_t* __restrict__ gpre, const int32_t* __restrict__ c_off,
                           const int32_t* __restrict__ int_ptr, const int32_t* __restrict__ int_idx,
                           const uint8_t* __restrict__ cok, const int32_t* __restrict__ cpre,
                           const uint8_t* __restrict__ wcnt, uint16_t* __restrict__ words, Ctl* ctl) {
  for (int64_t gid = gtid(); gid < G; gid += gstride()) {
    const int c = fxs_comp_of(gpre, K, (int)gid);
    if (!cok[c]) continue;
    const int lg = (int)gid - gpre[c], w = lg >> 2, g = lg & 3;
    const int off = c_off[c], sz = c_off[c + 1] - off;
    const int wb = gpre[c] / 4;
    int64_t slice = cpre[c];
    for (int v = 0; v < w; v++) slice += 32 * (int64_t)wcnt[wb + v];
    const int ncol = 4 * wcnt[wb + w];
    auto at = [&](int l, int col) -> uint16_t& {
      return words[(slice + 32 * (int64_t)(col >> 2) + 8 * g + l) * 4 + (col & 3)];
    };
    unsigned long long qm[8], rm[8];
    const int nc = fxs_greedy(int_ptr, int_idx, off, sz, 32 * w + 8 * g, qm, rm,
                              [&](int l, int col, int v) {
                                if (col < ncol) at(l, col) = (uint16_t)v;
                              });
    if (nc < 0 || nc > ncol) {  // the count pass said otherwise: the layout changed under us
      set_err(ctl, PR_EINTERNAL, 520);
      continue;
    }
    for (int col = 0; col < ncol; col++) {
      unsigned used = 0;
      for (int q = 0; q < 8; q++) used |= (unsigned)((qm[q] >> col) & 1ull) << q;
      for (int l = 0; l < 8; l++) {
        if ((rm[l] >> col) & 1ull) continue;
        const int qf = __ffs(~used & 0xffu) - 1;  // a free class: one per row without an entry
        used |= 1u << qf;
        at(l, col) = (uint16_t)(sz + ((qf - sz) & 7));
      }
    }
  }
}

pr_status build_fx_sched(pr_partition_s* P, Arena& tmp, Ctl* ctl) {
  cudaStream_t s = tmp.stream();
  Arena& keep = *P->keep;
  const int32_t K = P->n_comp;
  P->fxs_ptr = nullptr;
  P->fxs_wbase = nullptr;
  P->fxs_wcnt = nullptr;
  P->fxs_words = nullptr;
  if (K == 0) return PR_OK;
  int32_t *ngroup, *gpre, *cwords, *cpre;
  uint8_t *gcol, *cok;
  PRGB_TRY(tmp.alloc(&ngroup, (size_t)K + 1));
  PRGB_TRY(tmp.alloc(&gpre, (size_t)K + 1));
  fxs_groups_k<<<grid1(K), kBlock, 0, s>>>(K, P->c_off, P->c_type, ngroup);
  PRGB_LAUNCH();
  PRGB_TRY(scan_i32(ngroup, gpre, K, tmp));
  int32_t G = 0;
  PRGB_CUDA(cudaMemcpyAsync(&G, gpre + K, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  if (G == 0) return PR_OK;
  PRGB_TRY(tmp.alloc(&gcol, (size_t)G));
  PRGB_TRY(tmp.alloc(&cwords, (size_t)K + 1));
  PRGB_TRY(tmp.alloc(&cpre, (size_t)K + 1));
  PRGB_TRY(tmp.alloc(&cok, (size_t)K));
  PRGB_TRY(keep.alloc(&P->fxs_wcnt, (size_t)G / 4 + 1));
  fxs_count_k<<<grid1(G), kBlock, 0, s>>>(K, G, gpre, P->c_off, P->int_ptr, P->int_idx, gcol);
  PRGB_LAUNCH();
  fxs_comp_k<<<grid1(K), kBlock, 0, s>>>(K, gpre, gcol, P->fxs_wcnt, cwords, cok);
  PRGB_LAUNCH();
  PRGB_TRY(scan_i32(cwords, cpre, K, tmp));
  int32_t total = 0;
  PRGB_CUDA(cudaMemcpyAsync(&total, cpre + K, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  if (total <= 0) return PR_OK;  // no component has a schedule: the kernel builds slices itself
  PRGB_TRY(keep.alloc(&P->fxs_ptr, (size_t)K));
  PRGB_TRY(keep.alloc(&P->fxs_wbase, (size_t)K));
  PRGB_TRY(keep.alloc(&P->fxs_words, (size_t)total));
  fxs_ptr_k<<<grid1(K), kBlock, 0, s>>>(K, cok, cpre, gpre, P->fxs_ptr, P->fxs_wbase);
  PRGB_LAUNCH();
  fxs_fill_k<<<grid1(G), kBlock, 0, s>>>(K, G, gpre, P->c_off, P->int_ptr, P->int_idx, cok, cpre, P->fxs_wcnt,
                                         reinterpret_cast<uint16_t*>(P->fxs_words), ctl);
  PRGB_LAUNCH();
  return PR_OK;
}

}  // namespace prgb
