// spmv.cuh -- one balanced pull sweep acc_i = sum_{j -> i} val(j) over a set
// of rows, used by the grid-wide power-series kernels (large SCCs and the
// global baseline) and by the residual.
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so the sweep is
// organised to issue as few FP64 warp instructions as possible:
//   * light rows (in-degree <= kHeavy) are summed one row per thread; the
//     rows are pre-sorted into in-degree classes (powers of two), so the 32
//     rows of a warp have similar lengths and few lanes idle;
//   * heavy rows are split into chunks of kChunkH edges, one warp per chunk;
//     the warp that finishes a row's last chunk (atomic arrival counter)
//     adds the chunk partials in chunk order, so the result does not depend
//     on scheduling;
//   * the finished heavy rows' results are folded in a fixed two-level tree
//     (groups of 256 rows, then the groups) by whichever warp finishes last,
//     giving one deterministic total per sweep.
// No thread ever waits on another.
#pragma once

#include "common.cuh"

namespace prgb {

constexpr int kHeavy = 64;     // rows above this in-degree are chunked
constexpr int kChunkH = 256;   // edges per heavy chunk (8 per lane)
constexpr int kHGroup = 256;   // heavy rows per first-level fold

// In-degree class used to order light rows: 0 for no in-edge, else
// 1 + ceil(log2(d)) for d <= kHeavy; heavy rows get the last class.
__host__ __device__ __forceinline__ int deg_class(int d) {
  if (d > kHeavy) return 15;
  if (d == 0) return 0;
  int c = 1;
  while ((1 << (c - 1)) < d) c++;
  return c;
}

// heavy rows of a row set: row ids and their chunk offsets.  The arrays may
// be a slice of a longer list: chunk ids in choff and chrow are absolute,
// cbase / hbase are the slice's first chunk / first heavy row.
struct HeavyRows {
  const int32_t* rows = nullptr;   // [nheavy]
  const int32_t* choff = nullptr;  // [nheavy+1]
  const int32_t* chrow = nullptr;  // [all chunks] heavy-row index of each chunk
  int32_t nheavy = 0;
  int32_t nchunks = 0;
  int32_t cbase = 0;
  int32_t hbase = 0;
};

// scratch of the heavy rows; counters are zero at launch and left zero
struct HeavyScratch {
  double* part = nullptr;   // [nchunks] chunk partials
  int32_t* cnt = nullptr;   // [nheavy] chunk arrivals per row
  double* pn = nullptr;     // [nheavy] finished row values
  int32_t* gcnt = nullptr;  // [ngroups] finished rows per group
  double* gsum = nullptr;   // [ngroups] group folds
  int32_t* tcnt = nullptr;  // [1] finished groups
  double* total = nullptr;  // [2] fold of all heavy rows, by sweep parity
};

// allocate the heavy-row scratch (counters zeroed) on the arena's stream
inline pr_status alloc_heavy_scratch(HeavyScratch* hs, int nheavy, int nchunks, Arena& tmp) {
  const int ng = (nheavy + kHGroup - 1) / kHGroup;
  PRGB_TRY(tmp.alloc(&hs->part, (size_t)nchunks + 1));
  PRGB_TRY(tmp.alloc(&hs->cnt, (size_t)nheavy + 1));
  PRGB_TRY(tmp.alloc(&hs->pn, (size_t)nheavy + 1));
  PRGB_TRY(tmp.alloc(&hs->gcnt, (size_t)ng + 1));
  PRGB_TRY(tmp.alloc(&hs->gsum, (size_t)ng + 1));
  PRGB_TRY(tmp.alloc(&hs->tcnt, 1));
  PRGB_TRY(tmp.alloc(&hs->total, 2));
  PRGB_CUDA(cudaMemsetAsync(hs->cnt, 0, ((size_t)nheavy + 1) * 4, tmp.stream()));
  PRGB_CUDA(cudaMemsetAsync(hs->gcnt, 0, ((size_t)ng + 1) * 4, tmp.stream()));
  PRGB_CUDA(cudaMemsetAsync(hs->tcnt, 0, 4, tmp.stream()));
  PRGB_CUDA(cudaMemsetAsync(hs->total, 0, 16, tmp.stream()));
  return PR_OK;
}

__device__ __forceinline__ double fold2(double a, double b, bool l1) { return l1 ? a + b : fmax(a, b); }

// One sweep.  lorder[0, nlight) are the light rows (class-sorted).  For each
// row, fin(row, acc, heavy) is called exactly once and returns the value to
// fold into the sweep's norm; light rows fold it themselves (in the caller's
// per-thread accumulator), heavy rows are folded here into hs.total[parity].
// The edge sums are accumulated in the type val returns (double, or float
// for the FP32 sweeps of the mixed-precision solve); chunk partials and the
// heavy-row folds are kept in FP64.
// The warp's share of the light rows when the sweep is balanced by cost:
// rows [*r0, *r1) of lorder[0, nlight), whose costs (lpre, a prefix over the
// same rows, lpre[0] its base) add up to about 1/(number of warps) of the
// total.  Binary searches, once per launch.
__device__ __forceinline__ void warp_row_range(const int32_t* __restrict__ lpre, int nlight, int* r0, int* r1) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t base = lpre[0], total = (int64_t)lpre[nlight] - base;
  auto lower = [&](int64_t t) {
    int lo = 0, hi = nlight;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((int64_t)lpre[mid] - base < t) lo = mid + 1;
      else hi = mid;
    }
    return lo;
  };
  *r0 = lower(total * gw / nw);
  *r1 = lower(total * (gw + 1) / nw);
}

template <class Fin, class Val>
__device__ __forceinline__ void balanced_sweep(const int32_t* __restrict__ ptr, const int32_t* __restrict__ lorder,
                                               int nlight, const HeavyRows& hv, const HeavyScratch& hs, int parity,
                                               bool l1, Fin fin, Val val, int r0 = -1, int r1 = -1) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  using T = decltype(val(0));
  const int ngroups = (hv.nheavy + kHGroup - 1) / kHGroup;
  // heavy chunks first, so that the long rows start early
  for (int64_t ch = gw; ch < hv.nchunks; ch += nw) {
    const int cha = (int)ch + hv.cbase;
    const int h = hv.chrow[cha] - hv.hbase;
    const int row = hv.rows[h];
    const int j = cha - hv.choff[h];
    const int e0 = ptr[row] + j * kChunkH;
    const int e1 = min(ptr[row + 1], e0 + kChunkH);
    T acc = 0;
#pragma unroll
    for (int k = 0; k < kChunkH / 32; k++) {
      const int e = e0 + k * 32 + lane;
      if (e < e1) acc += val(e);
    }
    acc = group_sum<32>(acc);
    const int nch = hv.choff[h + 1] - hv.choff[h];
    int last = 0;
    if (lane == 0) {
      hs.part[ch] = (double)acc;
      __threadfence();
      last = atomicAdd(&hs.cnt[h], 1) == nch - 1;
    }
    if (!__shfl_sync(0xffffffffu, last, 0)) continue;
    // this warp finishes row h: partials in chunk order
    __threadfence();
    const int pb = hv.choff[h] - hv.cbase;
    double t = 0.0;
    for (int q = lane; q < nch; q += 32) t += __ldcg(&hs.part[pb + q]);
    t = group_sum<32>(t);
    int glast = 0;
    if (lane == 0) {
      hs.cnt[h] = 0;
      hs.pn[h] = fin(row, (T)t, true);
      __threadfence();
      const int g = h / kHGroup;
      const int gsz = min(kHGroup, hv.nheavy - g * kHGroup);
      glast = atomicAdd(&hs.gcnt[g], 1) == gsz - 1;
    }
    if (!__shfl_sync(0xffffffffu, glast, 0)) continue;
    // ... and the last row of its group: fold the group in row order
    __threadfence();
    const int g = h / kHGroup;
    const int h0 = g * kHGroup, h1 = min(hv.nheavy, h0 + kHGroup);
    double gs = 0.0;
    for (int q = h0 + lane; q < h1; q += 32) gs = fold2(gs, __ldcg(&hs.pn[q]), l1);
    gs = l1 ? group_sum<32>(gs) : group_max<32>(gs);
    int tlast = 0;
    if (lane == 0) {
      hs.gcnt[g] = 0;
      hs.gsum[g] = gs;
      __threadfence();
      tlast = atomicAdd(hs.tcnt, 1) == ngroups - 1;
    }
    if (!__shfl_sync(0xffffffffu, tlast, 0)) continue;
    // ... and the last group: fold the groups in order
    __threadfence();
    double ts = 0.0;
    for (int q = lane; q < ngroups; q += 32) ts = fold2(ts, __ldcg(&hs.gsum[q]), l1);
    ts = l1 ? group_sum<32>(ts) : group_max<32>(ts);
    if (lane == 0) {
      *hs.tcnt = 0;
      hs.total[parity] = ts;
    }
  }
  // light rows: one per thread; with a range, the warp's contiguous share
  // (rows of similar length, by their class order), else strided groups
  const bool ranged = r0 >= 0;
  const int64_t lb = ranged ? r0 : gw * 32, le = ranged ? r1 : nlight, ls = ranged ? 32 : nw * 32;
  for (int64_t base = lb; base < le; base += ls) {
    const int64_t i = base + lane;
    if (i < le) {
      const int row = lorder[i];
      const int b = ptr[row], e = ptr[row + 1];
      T acc = 0;
#pragma unroll 4
      for (int q = b; q < e; q++) acc += val(q);
      fin(row, acc, false);
    }
  }
}

// The warp's share of slices [0, nsl) when each slice costs cpre[s+1] -
// cpre[s] (cpre[0] is the base of the component's part of the prefix).
__device__ __forceinline__ void warp_slice_range(const int32_t* __restrict__ cpre, int nsl, int* s0, int* s1) {
  warp_row_range(cpre, nsl, s0, s1);
}

// Light rows in SELL-32 form (one warp per 32-row slice, the k-th in-edges
// of the slice's rows side by side): slice s covers rows r0 + 32 s + lane,
// the first nrows of them exist.  The index loads of a warp are one
// contiguous 128-byte line and its per-row reads and writes (fin) are
// consecutive; padding entries point at a z slot that holds 0.
template <class Fin, class Val>
__device__ __forceinline__ void sell_rows(const int32_t* __restrict__ sptr, const int32_t* __restrict__ sidx, int s0,
                                          int s1, int r0, int nrows, Val val, Fin fin) {
  const int lane = threadIdx.x & 31;
  using T = decltype(val(0));
  for (int s = s0; s < s1; s++) {
    const int b = sptr[s], w = (sptr[s + 1] - b) >> 5;
    const int32_t* p = sidx + b + lane;
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    int k = 0;
    for (; k + 3 < w; k += 4) {
      a0 += val(p[32 * k]);
      a1 += val(p[32 * (k + 1)]);
      a2 += val(p[32 * (k + 2)]);
      a3 += val(p[32 * (k + 3)]);
    }
    for (; k < w; k++) a0 += val(p[32 * k]);
    const int i = 32 * s + lane;
    if (i < nrows) fin(r0 + i, (a0 + a1) + (a2 + a3), false);
  }
}

}  // namespace prgb
