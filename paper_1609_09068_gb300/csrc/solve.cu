// solve.cu -- the PageRank step of Sec. 4.3 on the permuted layout.
//
// Levels run from the highest down (Sec. 4.3 steps 1-4).  Inside a level all
// components are independent and run concurrently (Sec. 4.3 last paragraph):
//   * 1-vertex components (Sec. 4.3 item 1, loops ignored): R = W;
//   * CACs (item 2, Sec. 4.3.1): one pass in topological order, sub-level by
//     sub-level: R_v = W_v + c * sum_{j->v inside} R_j / outdeg(j);
//   * SCCs (item 4, Sec. 4.3.2): power series P_0 = W, P_{k+1} = c A^T P_k,
//     R = sum_k P_k, stopping after adding P with ||P||_1 <= tol*|C|/n (or the
//     paper's max(P) < tol).
// The weight update of Eq. (PR:levels) is done as a pull: every vertex of a
// level gathers W_v = u_v + c * sum over external in-edges of R_j/outdeg(j)
// from levels already solved, fused into the kernel that solves it.
//
// Kernel classes by component size: one warp (<= 32 vertices, one vertex per
// lane, z in shared memory), one CTA (<= 2048 vertices, z in shared memory),
// and grid-wide cooperative kernels with bounded grid barriers for the rest.
// z = R/outdeg (or P/outdeg during the series) is the only per-vertex vector
// gathered: A_ij = 1/outdeg(i) depends on the source only, so no edge values
// are stored.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "solve.cuh"
#include "spmv.cuh"

namespace cg = cooperative_groups;

namespace prgb {

// z = x / outdeg as x * (1/outdeg): the reciprocal is precomputed once per
// vertex, because FP64 division is expensive on this part.

__device__ __forceinline__ bool keep_going(double s, double tau, int norm) {
  return norm == PR_NORM_LINF ? (s >= tau) : (s > tau);
}

// The warp and CTA kernels reduce the stopping norm in FP32: FP64 shuffles
// and adds cost more than the rows themselves on this part.  The FP32 sum
// of n non-negative terms is within n * 2^-24 of the FP64 one, so a relative
// margin of 1e-4 on the test keeps the FP64 norm at or below the threshold
// whenever the series stops (it may run one iteration longer than an exact
// test would).
constexpr double kNormMargin = 1.0 + 1e-4;
__device__ __forceinline__ bool keep_going32(float s, double tau, int norm) {
  const double sd = (double)s * kNormMargin;
  return norm == PR_NORM_LINF ? (sd >= tau) : (sd > tau);
}

// A local index outside [0, sz) would mean a broken layout: record it and
// read slot 0 instead of touching memory out of bounds.
__device__ __forceinline__ int local_or_err(const SolveArgs& a, int q, int sz) {
  if ((unsigned)q >= (unsigned)sz) {
    set_err(a.ctl, PR_EINTERNAL, 301);
    return 0;
  }
  return q;
}

__device__ __forceinline__ double check_u(const SolveArgs& a, double uu) {
  if (!(uu >= 0.0) || !isfinite(uu)) set_err(a.ctl, PR_EINVAL, 300);
  return uu;
}

// ---------------------------------------------------------------------------
// one warp per component of 2..32 vertices, one vertex per lane.  The
// component's internal in-edges (at most 32*31) are staged in shared memory
// as 8-bit local indices, so each series iteration reads shared memory only.
// ---------------------------------------------------------------------------
constexpr int kWarpEdges = kWarpCompMax * (kWarpCompMax - 1);
constexpr int kWarpBlock = 64;  // two components per block, spread over many SMs

__global__ void __launch_bounds__(kWarpBlock) solve_warp_k(SolveArgs a, int32_t cbeg, int32_t cend) {
  __shared__ double zsh[kWarpBlock / 32][32];
  __shared__ uint8_t ish[kWarpBlock / 32][kWarpEdges];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int c = cbeg + (int)blockIdx.x * (kWarpBlock / 32) + wib;
  if (c >= cend) return;  // warp-uniform
  double* z = zsh[wib];
  uint8_t* ix = ish[wib];
  const int off = a.c_off[c], sz = a.c_off[c + 1] - off;
  const bool act = lane < sz;
  const int p = off + lane;
  const double inv = act ? a.p_inv[p] : 0.0;
  const int ib0 = a.int_ptr[off];
  const int m = a.int_ptr[off + sz] - ib0;
  for (int e = lane; e < m && e < kWarpEdges; e += 32) ix[e] = (uint8_t)local_or_err(a, a.int_idx[ib0 + e] - off, sz);
  if (m > kWarpEdges) set_err(a.ctl, PR_EINTERNAL, 302);
  const double W = act ? a.W[p] : 0.0;
  const int ib = act ? a.int_ptr[p] - ib0 : 0, ie = act ? min(a.int_ptr[p + 1] - ib0, kWarpEdges) : 0;
  __syncwarp();
  double R = W;
  int k = 0;
  if (a.c_type[c] == PR_TYPE_CAC) {
    const int sb = a.c_sub[c], se = a.c_sub[c + 1];
    for (int s = sb; s < se; s++) {
      const int lo = a.sub_ptr[s], hi = a.sub_ptr[s + 1];
      if (act && p >= lo && p < hi) {
        double acc = 0.0;
        for (int e = ib; e < ie; e++) acc += z[ix[e]];
        R = W + a.c * acc;
        z[lane] = R * inv;
      }
      __syncwarp();
    }
  } else {
    const double tau = a.norm == PR_NORM_L1 ? a.tol * (double)sz / (double)a.n : a.tol;
    const int fixed = a.replay ? a.replay[c] : -1;
    if (act) z[lane] = W * inv;
    __syncwarp();
    for (;;) {
      // two partial sums halve the chain of dependent FP64 adds
      double acc0 = 0.0, acc1 = 0.0;
      int e = ib;
      for (; e + 1 < ie; e += 2) {
        acc0 += z[ix[e]];
        acc1 += z[ix[e + 1]];
      }
      if (e < ie) acc0 += z[ix[e]];
      const double pn = a.c * (acc0 + acc1);
      __syncwarp();
      if (act) {
        z[lane] = pn * inv;
        R += pn;
      }
      __syncwarp();
      k++;
      if (fixed >= 0) {
        if (k >= fixed) break;
        continue;
      }
      const float pf = (float)pn;
      const float s = a.norm == PR_NORM_L1 ? group_sumf<32>(pf) : group_maxf<32>(pf);
      if (!keep_going32(s, tau, a.norm)) break;
      if (k >= a.max_iter) {
        if (lane == 0) atomicOr(&a.ctl->flags[0], 1);
        break;
      }
    }
  }
  if (act) {
    a.R[p] = R;
    a.zr[p] = R * inv;
  }
  if (lane == 0) a.iters[c] = k;
}

// ---------------------------------------------------------------------------
// one CTA of 256 threads per component of 33..kCtaCompMax vertices, one row
// per thread.  The component's internal in-edges are staged in
// shared memory as 16-bit local indices with local row offsets, next to R
// and the double-buffered z, so the series runs from shared memory only.  A
// component with more internal edges than the staging area reads its
// indices from global memory instead.
// ---------------------------------------------------------------------------
constexpr int kCtaThreads = 256;
constexpr int kCtaEdgeCap = 8192;
constexpr int kCtaRows = kCtaCompMax / kCtaThreads;
constexpr size_t kCtaSmem = (size_t)kCtaCompMax * (3 * sizeof(double) + sizeof(int)) + sizeof(int) +
                            (size_t)kCtaEdgeCap * sizeof(uint16_t);

__global__ void __launch_bounds__(kCtaThreads) solve_cta_k(SolveArgs a, int32_t cbeg) {
  extern __shared__ double sm[];
  double* Rs = sm;
  double* z = sm + kCtaCompMax;
  double* iv = sm + 2 * kCtaCompMax;
  int* ip = reinterpret_cast<int*>(sm + 3 * kCtaCompMax);  // [sz+1] local edge offsets
  uint16_t* ix = reinterpret_cast<uint16_t*>(ip + kCtaCompMax + 1);
  __shared__ float red[kCtaThreads / 32];
  const int c = cbeg + (int)blockIdx.x;
  const int off = a.c_off[c], sz = a.c_off[c + 1] - off;
  const int ib = a.int_ptr[off];
  const int m = a.int_ptr[off + sz] - ib;
  const bool staged = m <= kCtaEdgeCap;
  const bool scc = a.c_type[c] == PR_TYPE_SCC;
  for (int i = threadIdx.x; i <= sz; i += blockDim.x) ip[i] = a.int_ptr[off + i] - ib;
  if (staged)
    for (int e = threadIdx.x; e < m; e += blockDim.x) ix[e] = (uint16_t)local_or_err(a, a.int_idx[ib + e] - off, sz);
  // inflow-adjusted weights from the level's gather
  for (int i = threadIdx.x; i < sz; i += blockDim.x) {
    const int p = off + i;
    const double inv = a.p_inv[p];
    const double W = a.W[p];
    iv[i] = inv;
    Rs[i] = W;
    z[i] = W * inv;
  }
  __syncthreads();
  auto row_sum = [&](int i) -> double {
    double acc = 0.0;
    const int e0 = ip[i], e1 = ip[i + 1];
    if (staged) {
#pragma unroll 4
      for (int e = e0; e < e1; e++) acc += z[ix[e]];
    } else {
      for (int e = e0; e < e1; e++) acc += z[local_or_err(a, a.int_idx[ib + e] - off, sz)];
    }
    return acc;
  };
  int k = 0;
  if (!scc) {
    // CAC: one pass, sub-level by sub-level (topological order)
    const int sb = a.c_sub[c], se = a.c_sub[c + 1];
    for (int s2 = sb; s2 < se; s2++) {
      const int lo = a.sub_ptr[s2] - off, hi = a.sub_ptr[s2 + 1] - off;
      for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double Rv = Rs[i] + a.c * row_sum(i);
        Rs[i] = Rv;
        z[i] = Rv * iv[i];
      }
      __syncthreads();
    }
  } else {
    const double tau = a.norm == PR_NORM_L1 ? a.tol * (double)sz / (double)a.n : a.tol;
    const int fixed = a.replay ? a.replay[c] : -1;
    for (;;) {
      double pn[kCtaRows];
      double local = 0.0;
#pragma unroll
      for (int r = 0; r < kCtaRows; r++) {
        const int i = threadIdx.x + r * kCtaThreads;
        pn[r] = i < sz ? a.c * row_sum(i) : 0.0;
      }
      __syncthreads();  // every row has read z before it is overwritten
#pragma unroll
      for (int r = 0; r < kCtaRows; r++) {
        const int i = threadIdx.x + r * kCtaThreads;
        if (i < sz) {
          Rs[i] += pn[r];
          z[i] = pn[r] * iv[i];
          local = a.norm == PR_NORM_L1 ? local + pn[r] : fmax(local, pn[r]);
        }
      }
      // the reduction ends with __syncthreads, which also publishes z
      const float s2 = block_sumf((float)local, red, a.norm != PR_NORM_L1);
      k++;
      if (fixed >= 0) {
        if (k >= fixed) break;
        continue;
      }
      if (!keep_going32(s2, tau, a.norm)) break;
      if (k >= a.max_iter) {
        if (threadIdx.x == 0) atomicOr(&a.ctl->flags[0], 1);
        break;
      }
    }
  }
  for (int i = threadIdx.x; i < sz; i += blockDim.x) {
    a.R[off + i] = Rs[i];
    a.zr[off + i] = Rs[i] * iv[i];
  }
  if (threadIdx.x == 0) a.iters[c] = k;
}

// ---------------------------------------------------------------------------
// one cluster of kClu CTAs (on kClu SMs) per component of
// kCtaCompMax+1..kCluCompMax vertices.  Rank r owns the component-local rows
// [r*chunk, (r+1)*chunk) with chunk a power of two; z lives in distributed
// shared memory (each rank holds its rows' z, double-buffered), a row reads
// the z of any rank through the cluster's shared-memory window, and one
// hardware cluster barrier per iteration publishes the new z and the rank
// partials of the stopping norm.  This spreads a component's FP64 work over
// kClu SMs instead of one.
// ---------------------------------------------------------------------------
constexpr int kClu = 8;
constexpr int kCluThreads = 256;
constexpr int kCluEdgesPerRow = 8;  // staged edges per row (more are read from global memory)

__host__ __device__ __forceinline__ int clu_shift(int sz) {
  int sh = 0;
  while ((kClu << sh) < sz) sh++;
  return sh;
}

__host__ __device__ __forceinline__ size_t clu_smem(int chunk) {
  return (size_t)chunk * (4 * sizeof(double) + sizeof(int)) + 2 * sizeof(int) + 2 * sizeof(float) +
         (size_t)chunk * kCluEdgesPerRow * sizeof(uint16_t);
}

__global__ void __cluster_dims__(kClu, 1, 1) __launch_bounds__(kCluThreads)
    solve_clu_k(SolveArgs a, int32_t cbeg, int32_t chunk_max) {
  extern __shared__ double cs[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  double* zA = cs;
  double* zB = cs + chunk_max;
  double* Rs = cs + 2 * chunk_max;
  double* iv = cs + 3 * chunk_max;
  int* ip = reinterpret_cast<int*>(cs + 4 * chunk_max);         // [chunk_max + 1]
  float* part = reinterpret_cast<float*>(ip + chunk_max + 2);   // [2]
  uint16_t* ix = reinterpret_cast<uint16_t*>(part + 2);         // [chunk_max * kCluEdgesPerRow]
  __shared__ float red[kCluThreads / 32];
  __shared__ double* remA[kClu];
  __shared__ double* remB[kClu];
  __shared__ float* remP[kClu];
  const int c = cbeg + (int)(blockIdx.x / kClu);
  const int off = a.c_off[c], sz = a.c_off[c + 1] - off;
  const int sh = clu_shift(sz);
  const int chunk = 1 << sh;
  const int r0 = rank * chunk;
  const int nr = max(0, min(sz, r0 + chunk) - r0);
  if (threadIdx.x < kClu) {
    remA[threadIdx.x] = cl.map_shared_rank(zA, (int)threadIdx.x);
    remB[threadIdx.x] = cl.map_shared_rank(zB, (int)threadIdx.x);
    remP[threadIdx.x] = cl.map_shared_rank(part, (int)threadIdx.x);
  }
  // stage this rank's rows: local edge offsets and component-local indices
  const int ib = a.int_ptr[off + r0];
  const int m = nr > 0 ? a.int_ptr[off + r0 + nr] - ib : 0;
  const bool staged = m <= chunk_max * kCluEdgesPerRow;
  for (int i = threadIdx.x; i <= nr; i += blockDim.x) ip[i] = a.int_ptr[off + r0 + i] - ib;
  if (staged)
    for (int e = threadIdx.x; e < m; e += blockDim.x) ix[e] = (uint16_t)local_or_err(a, a.int_idx[ib + e] - off, sz);
  // inflow-adjusted weights of this rank's rows
  for (int i = threadIdx.x; i < nr; i += blockDim.x) {
    const int p = off + r0 + i;
    const double inv = a.p_inv[p];
    const double W = a.W[p];
    iv[i] = inv;
    Rs[i] = W;
    zA[i] = W * inv;
  }
  cl.sync();
  const int mask = chunk - 1;
  auto row_sum = [&](double* const* rem, int i) -> double {
    double acc0 = 0.0, acc1 = 0.0;
    const int e0 = ip[i], e1 = ip[i + 1];
    int e = e0;
    if (staged) {
      for (; e + 1 < e1; e += 2) {
        const int q0 = ix[e], q1 = ix[e + 1];
        acc0 += rem[q0 >> sh][q0 & mask];
        acc1 += rem[q1 >> sh][q1 & mask];
      }
      if (e < e1) {
        const int q = ix[e];
        acc0 += rem[q >> sh][q & mask];
      }
    } else {
      for (; e < e1; e++) {
        const int q = local_or_err(a, a.int_idx[ib + e] - off, sz);
        acc0 += rem[q >> sh][q & mask];
      }
    }
    return acc0 + acc1;
  };
  int k = 0;
  if (a.c_type[c] != PR_TYPE_SCC) {
    // CAC: one pass, sub-level by sub-level, one cluster barrier each
    const int sb = a.c_sub[c], se = a.c_sub[c + 1];
    for (int s2 = sb; s2 < se; s2++) {
      const int lo = max(a.sub_ptr[s2] - off - r0, 0), hi = min(a.sub_ptr[s2 + 1] - off - r0, nr);
      for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double Rv = Rs[i] + a.c * row_sum(remA, i);
        Rs[i] = Rv;
        zA[i] = Rv * iv[i];
      }
      cl.sync();
    }
  } else {
    const double tau = a.norm == PR_NORM_L1 ? a.tol * (double)sz / (double)a.n : a.tol;
    const int fixed = a.replay ? a.replay[c] : -1;
    const bool is_max = a.norm != PR_NORM_L1;
    for (;;) {
      double* const* rem = (k & 1) ? remB : remA;
      double* nxt = (k & 1) ? zA : zB;
      float local = 0.0f;
      for (int i = threadIdx.x; i < nr; i += blockDim.x) {
        const double pn = a.c * row_sum(rem, i);
        Rs[i] += pn;
        nxt[i] = pn * iv[i];
        local = is_max ? fmaxf(local, (float)pn) : local + (float)pn;
      }
      const float bs = block_sumf(local, red, is_max);
      if (threadIdx.x == 0) part[k & 1] = bs;
      cl.sync();  // publishes nxt and the rank partials
      float s2 = 0.0f;
      for (int r = 0; r < kClu; r++) s2 = is_max ? fmaxf(s2, remP[r][k & 1]) : s2 + remP[r][k & 1];
      k++;
      if (fixed >= 0) {
        if (k >= fixed) break;
        continue;
      }
      if (!keep_going32(s2, tau, a.norm)) break;
      if (k >= a.max_iter) {
        if (rank == 0 && threadIdx.x == 0) atomicOr(&a.ctl->flags[0], 1);
        break;
      }
    }
  }
  for (int i = threadIdx.x; i < nr; i += blockDim.x) {
    a.R[off + r0 + i] = Rs[i];
    a.zr[off + r0 + i] = Rs[i] * iv[i];
  }
  if (rank == 0 && threadIdx.x == 0) a.iters[c] = k;
  cl.sync();  // no rank leaves while another may still read its shared memory
}

// ---------------------------------------------------------------------------
// inflow gather of one level (Eq. PR:levels as a pull): for every vertex of
// the level, W = u + c * sum over external in-edges of R_j / outdeg(j), with
// the balanced sweep (hubs receive tens of thousands of external edges).
// The level's 1-vertex components are finished here (R = W, Sec. 4.3 item 1).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) gather_level_k(SolveArgs a, LevelRange r, HeavyRows hv,
                                                         HeavyScratch hs) {
  auto fin = [&](int row, double acc, bool) -> double {
    const double W = check_u(a, a.u[a.perm[row]]) + a.c * acc;
    a.W[row] = W;
    if (row >= r.vsingle) {
      a.R[row] = W;
      a.zr[row] = W * a.p_inv[row];
    }
    return 0.0;
  };
  auto val = [&](int e) -> double { return a.zr[a.ext_idx[e]]; };
  const int nlight = (r.vend - r.vbeg) - (r.xh_end - r.xh_begin);
  balanced_sweep(a.ext_ptr, a.xlorder + r.vbeg, nlight, hv, hs, 0, true, fin, val);
}

// ---------------------------------------------------------------------------
// grid-wide kernels for large components (cooperative launch)
// ---------------------------------------------------------------------------
constexpr int kG = 8;  // lanes per row

// R[p] = W[p] and z0[p - off] = W/outdeg for the rows of a component
__device__ __forceinline__ void load_rows(const SolveArgs& a, int off, int sz, double* z0) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sz; i += (int64_t)gridDim.x * blockDim.x) {
    const int p = off + (int)i;
    const double W = a.W[p];
    a.R[p] = W;
    if (z0) z0[i] = W * a.p_inv[p];
  }
}

__global__ void __launch_bounds__(kBlock) solve_large_scc_k(SolveArgs a, LargeComp L, double* zA, double* zB,
                                                            double* part, HeavyRows hv, HeavyScratch hs) {
  __shared__ double red[kBlock / 32];
  const int off = L.off, sz = L.size;
  const int nlight = sz - hv.nheavy;
  const int* lorder = a.lorder + off;
  load_rows(a, off, sz, zA);
  if (!grid_sync(a.ctl, 310)) return;
  const double tau = a.norm == PR_NORM_L1 ? a.tol * (double)sz / (double)a.n : a.tol;
  const int fixed = a.replay ? a.replay[L.c] : -1;
  const bool l1 = a.norm == PR_NORM_L1;
  int k = 0;
  for (;;) {
    const double* cur = (k & 1) ? zB : zA;
    double* nxt = (k & 1) ? zA : zB;
    double local = 0.0;
    auto fin = [&](int row, double acc, bool heavy) -> double {
      const double pn = a.c * acc;
      a.R[row] += pn;
      nxt[row - off] = pn * a.p_inv[row];
      if (!heavy) local = fold2(local, pn, l1);
      return pn;
    };
    auto val = [&](int e) -> double { return cur[local_or_err(a, a.int_idx[e] - off, sz)]; };
    balanced_sweep(a.int_ptr, lorder, nlight, hv, hs, k & 1, l1, fin, val);
    const double bs = l1 ? block_sum(local, red) : block_max(local, red);
    double* slot = part + (size_t)(k & 1) * gridDim.x;
    if (threadIdx.x == 0) slot[blockIdx.x] = bs;
    if (!grid_sync(a.ctl, 311)) return;
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t = fold2(t, __ldcg(&slot[b]), l1);
    double s = l1 ? block_sum(t, red) : block_max(t, red);
    if (hv.nheavy > 0) s = fold2(s, __ldcg(&hs.total[k & 1]), l1);
    k++;
    if (fixed >= 0) {
      if (k >= fixed) break;
      continue;
    }
    if (!keep_going(s, tau, a.norm)) break;
    if (k >= a.max_iter) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctl->flags[0], 1);
      break;
    }
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sz; i += (int64_t)gridDim.x * blockDim.x)
    a.zr[off + i] = a.R[off + i] * a.p_inv[off + i];
  if (blockIdx.x == 0 && threadIdx.x == 0) a.iters[L.c] = k;
}

__global__ void __launch_bounds__(kBlock) solve_large_cac_k(SolveArgs a, LargeComp L) {
  load_rows(a, L.off, L.size, nullptr);  // R[p] = W
  if (!grid_sync(a.ctl, 320)) return;
  const int lane = threadIdx.x & (kG - 1);
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kG;
  const int64_t ng = ((int64_t)gridDim.x * blockDim.x) / kG;
  const int64_t wb = g0 - ((threadIdx.x & 31) / kG);
  for (int s = L.sub_begin; s < L.sub_end; s++) {
    const int lo = a.sub_ptr[s], hi = a.sub_ptr[s + 1];
    for (int64_t base = wb; base < hi - lo; base += ng) {
      const int64_t i = base + ((threadIdx.x & 31) / kG);
      const int p = lo + (int)i;
      double acc = 0.0;
      if (p < hi)
        for (int e = a.int_ptr[p] + lane; e < a.int_ptr[p + 1]; e += kG) acc += a.zr[a.int_idx[e]];
      acc = group_sum<kG>(acc);
      if (p < hi && lane == 0) {
        const double Rv = a.R[p] + a.c * acc;
        a.R[p] = Rv;
        a.zr[p] = Rv * a.p_inv[p];
      }
    }
    if (!grid_sync(a.ctl, 321)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.iters[L.c] = 0;
}

__global__ void scatter_out_k(int32_t n, const int32_t* perm, const double* Rp, double* R) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    R[perm[p]] = Rp[p];
}

// edge reads of the solve: ext edges once, CAC internal edges once, SCC
// internal edges once per iteration
__global__ void edge_visits_k(int32_t K, const int32_t* c_off, const uint8_t* c_type, const int32_t* int_ptr,
                              const int32_t* ext_ptr, const int32_t* iters, unsigned long long* out) {
  unsigned long long loc = 0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < K; c += (int64_t)gridDim.x * blockDim.x) {
    const int b = c_off[c], e = c_off[c + 1];
    const long long mi = int_ptr[e] - int_ptr[b], me = ext_ptr[e] - ext_ptr[b];
    loc += (unsigned long long)(me + (c_type[c] == PR_TYPE_SCC ? mi * (long long)iters[c] : mi));
  }
  atomicAdd(out, loc);
}

}  // namespace prgb

namespace prgb {

// three non-blocking side streams and the fork / join events of a solve
struct SideStreams {
  cudaStream_t st[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[3] = {nullptr, nullptr, nullptr};
  pr_status create() {
    for (int q = 0; q < 3; q++) {
      PRGB_CUDA(cudaStreamCreateWithFlags(&st[q], cudaStreamNonBlocking));
      PRGB_CUDA(cudaEventCreateWithFlags(&join[q], cudaEventDisableTiming));
    }
    PRGB_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    return PR_OK;
  }
  ~SideStreams() {
    for (int q = 0; q < 3; q++) {
      if (st[q]) cudaStreamDestroy(st[q]);
      if (join[q]) cudaEventDestroy(join[q]);
    }
    if (fork) cudaEventDestroy(fork);
  }
};

static unsigned grid_cap(int64_t blocks) {
  int64_t cap = (int64_t)num_sms() * 32;
  return (unsigned)(blocks < 1 ? 1 : (blocks > cap ? cap : blocks));
}

pr_status run_solve(const pr_partition_s* P, double c, const double* u, double tol, int norm, int max_iter,
                    const int32_t* replay, double* R, int32_t* iters_dev, Arena& tmp, Ctl* ctl,
                    int64_t* launches, KernelTiming* timing) {
  cudaStream_t s = tmp.stream();
  const int32_t n = P->g.n;
  int64_t nl = 0;
  if (n == 0) {
    *launches = 0;
    return PR_OK;
  }
  SolveArgs a;
  a.n = n;
  a.c = c;
  a.tol = tol;
  a.norm = norm;
  a.max_iter = max_iter;
  a.u = u;
  a.perm = P->perm;
  a.p_outdeg = P->p_outdeg;
  a.p_inv = P->p_inv;
  a.lorder = P->lorder;
  a.int_ptr = P->int_ptr;
  a.int_idx = P->int_idx;
  a.ext_ptr = P->ext_ptr;
  a.ext_idx = P->ext_idx;
  a.c_off = P->c_off;
  a.c_sub = P->c_sub;
  a.sub_ptr = P->sub_ptr;
  a.c_type = P->c_type;
  a.replay = replay;
  a.iters = iters_dev;
  a.ctl = ctl;
  a.xlorder = P->xlorder;
  PRGB_TRY(tmp.alloc(&a.R, n));
  PRGB_TRY(tmp.alloc(&a.zr, n));
  PRGB_TRY(tmp.alloc(&a.W, n));
  double *zA = nullptr, *zB = nullptr, *part = nullptr;
  HeavyScratch hs;  // shared by the level gathers and the grid-wide series (left zeroed after each)
  PRGB_TRY(alloc_heavy_scratch(&hs, std::max(P->max_heavy, P->max_xheavy), std::max(P->max_chunks, P->max_xchunks),
                               tmp));
  if (P->max_large > 0) {
    PRGB_TRY(tmp.alloc(&zA, P->max_large));
    PRGB_TRY(tmp.alloc(&zB, P->max_large));
    PRGB_TRY(tmp.alloc(&part, (size_t)2 * num_sms() * 8));
  }
  static bool cta_attr = false;
  static size_t clu_attr = 48 * 1024;
  // The cluster, CTA and warp kernels of a level are independent: they run on
  // three side streams, forked after the level's gather and joined before
  // the next level, so one kernel's tail overlaps the others.
  SideStreams side;
  PRGB_TRY(side.create());
  if (!cta_attr) {
    PRGB_CUDA(cudaFuncSetAttribute(solve_cta_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCtaSmem));
    cta_attr = true;
  }
  size_t li_large = 0;
  for (size_t li = 0; li < P->levels.size(); li++) {
    const LevelRange& r = P->levels[li];
    {
      HeavyRows xv;
      xv.rows = P->xheavy_rows + r.xh_begin;
      xv.choff = P->xheavy_choff + r.xh_begin;
      xv.chrow = P->xheavy_chrow;
      xv.nheavy = r.xh_end - r.xh_begin;
      xv.nchunks = r.xc_end - r.xc_begin;
      xv.cbase = r.xc_begin;
      xv.hbase = r.xh_begin;
      const int64_t work = (int64_t)(r.vend - r.vbeg) + (int64_t)xv.nchunks * 32;
      gather_level_k<<<grid_cap((work + kBlock - 1) / kBlock), kBlock, 0, s>>>(a, r, xv, hs);
      PRGB_LAUNCH();
      nl++;
    }
    while (li_large < P->large.size() && P->large[li_large].level_idx == (int)li) {
      LargeComp L = P->large[li_large++];
      PRGB_TRY(reset_ctl(ctl, s));
      if (L.type == PR_TYPE_SCC) {
        HeavyRows hv;
        hv.rows = P->heavy_rows + L.heavy_begin;
        hv.choff = P->heavy_choff + L.heavy_begin;
        hv.chrow = P->heavy_chrow;
        hv.nheavy = L.heavy_end - L.heavy_begin;
        hv.nchunks = L.chunk_end - L.chunk_begin;
        hv.cbase = L.chunk_begin;
        hv.hbase = L.heavy_begin;
        void* args[] = {&a, &L, &zA, &zB, &part, &hv, &hs};
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (timing) {
          PRGB_CUDA(cudaEventCreate(&e0));
          timing->start.push_back(e0);
          PRGB_CUDA(cudaEventCreate(&e1));
          timing->stop.push_back(e1);
          timing->comps.push_back(L);
          PRGB_CUDA(cudaEventRecord(e0, s));
        }
        PRGB_TRY(launch_coop((const void*)solve_large_scc_k, kBlock, 0, s, args, 4, nullptr));
        if (timing) PRGB_CUDA(cudaEventRecord(e1, s));
      } else {
        void* args[] = {&a, &L};
        PRGB_TRY(launch_coop((const void*)solve_large_cac_k, kBlock, 0, s, args, 4, nullptr));
      }
      nl++;
    }
    PRGB_CUDA(cudaEventRecord(side.fork, s));
    bool joined[3] = {false, false, false};
    if (r.cta > r.clu) {
      PRGB_CUDA(cudaStreamWaitEvent(side.st[0], side.fork, 0));
      joined[0] = true;
      const int chunk = 1 << clu_shift(r.clu_max);
      const size_t smem = clu_smem(chunk);
      if (smem > clu_attr) {
        PRGB_CUDA(cudaFuncSetAttribute(solve_clu_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        clu_attr = smem;
      }
      solve_clu_k<<<(r.cta - r.clu) * kClu, kCluThreads, smem, side.st[0]>>>(a, r.clu, chunk);
      PRGB_LAUNCH();
      nl++;
    }
    if (r.warp > r.cta) {
      PRGB_CUDA(cudaStreamWaitEvent(side.st[1], side.fork, 0));
      joined[1] = true;
      solve_cta_k<<<r.warp - r.cta, kCtaThreads, kCtaSmem, side.st[1]>>>(a, r.cta);
      PRGB_LAUNCH();
      nl++;
    }
    if (r.single > r.warp) {
      const int nw = r.single - r.warp;
      PRGB_CUDA(cudaStreamWaitEvent(side.st[2], side.fork, 0));
      joined[2] = true;
      solve_warp_k<<<(nw + kWarpBlock / 32 - 1) / (kWarpBlock / 32), kWarpBlock, 0, side.st[2]>>>(a, r.warp,
                                                                                                  r.single);
      PRGB_LAUNCH();
      nl++;
    }
    for (int q = 0; q < 3; q++) {
      if (!joined[q]) continue;
      PRGB_CUDA(cudaEventRecord(side.join[q], side.st[q]));
      PRGB_CUDA(cudaStreamWaitEvent(s, side.join[q], 0));
    }
  }
  scatter_out_k<<<grid_cap((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, P->perm, a.R, R);
  PRGB_LAUNCH();
  nl++;
  *launches = nl;
  return PR_OK;
}

pr_status solve_edge_visits(const pr_partition_s* P, const int32_t* iters_dev, int64_t* out, Arena& tmp) {
  cudaStream_t s = tmp.stream();
  *out = 0;
  if (P->n_comp == 0) return PR_OK;
  unsigned long long* d = nullptr;
  PRGB_TRY(tmp.alloc(&d, 1));
  PRGB_CUDA(cudaMemsetAsync(d, 0, 8, s));
  edge_visits_k<<<grid_cap((P->n_comp + kBlock - 1) / kBlock), kBlock, 0, s>>>(
      P->n_comp, P->c_off, P->c_type, P->int_ptr, P->ext_ptr, iters_dev, d);
  PRGB_LAUNCH();
  unsigned long long h = 0;
  PRGB_CUDA(cudaMemcpyAsync(&h, d, 8, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  *out = (int64_t)h;
  return PR_OK;
}

}  // namespace prgb
