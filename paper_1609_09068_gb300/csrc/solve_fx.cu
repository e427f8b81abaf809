// solve_fx.cu -- the power series of Sec. 4.3.2 for SCCs of 33..kFxMax
// vertices, one CTA per component, with exact fixed-point row sums.
//
// P_0 = W, P_{k+1} = c A^T P_k, R = sum_k P_k, per component, stopping by
// the same rule as the other kernels (L1: after adding P with
// ||P||_1 <= tol |C| / n; L-inf: the paper's max(P) < tol).  The gathered
// vector is z = c P / outdeg, so a row's in-edge sum is the next term.
//
// All of a component's state stays in shared memory and registers.  What
// differs from the FP64 kernels is the arithmetic of the sums: z is stored
// as 128-bit fixed point (fx128.cuh) with a binary point chosen once per
// component from ||W_C||_1, a row's sum of z over its in-edges is an exact
// integer sum, and R accumulates the terms exactly.  Per row and sweep one
// FP64 multiply remains (z = P * c/outdeg, with P rounded to a double);
// everything else runs on the integer pipes, which GB300 has at many times
// its FP64 rate.  The only roundings are that product and the conversions,
// so every term is within a few units in the last place of the FP64 series'
// term and sums lose nothing (the FP64 kernels round once per edge).
//
// CACs in the same size range are solved in FP64 by one pass over their
// topological sub-levels (Sec. 4.3.1), exactly as in the other kernels.
#include <algorithm>

#include "common.cuh"
#include "fx128.cuh"
#include "solve.cuh"

namespace prgb {

// sum of z over the in-edges [e0, e1) (local indices staged in ix, or read
// from the global layout), two independent carry chains
template <bool kStaged>
__device__ __forceinline__ fx128 fx_row(const SolveArgs& a, const fx128* __restrict__ z,
                                        const uint16_t* __restrict__ ix, int ib, int off, int sz, int e0, int e1) {
  fx128 s0 = 0, s1 = 0;
  int e = e0;
  for (; e + 1 < e1; e += 2) {
    const int q0 = kStaged ? (int)ix[e] : local_or_err(a, a.int_idx[ib + e] - off, sz);
    const int q1 = kStaged ? (int)ix[e + 1] : local_or_err(a, a.int_idx[ib + e + 1] - off, sz);
    s0 += z[q0];
    s1 += z[q1];
  }
  if (e < e1) s0 += z[kStaged ? (int)ix[e] : local_or_err(a, a.int_idx[ib + e] - off, sz)];
  return s0 + s1;
}

template <int T>
__device__ __forceinline__ float block_norm(float part, float (*red)[T / 32], int parity, bool is_max) {
  // warp partials, one barrier, then every warp folds the same partials in
  // the same order (deterministic, no second barrier)
  constexpr int kNW = T / 32;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  part = is_max ? group_maxf<32>(part) : group_sumf<32>(part);
  if (lane == 0) red[parity][wib] = part;
  __syncthreads();
  float t = lane < kNW ? red[parity][lane] : 0.0f;
  return is_max ? group_maxf<32>(t) : group_sumf<32>(t);
}

template <int T, bool kStaged>
__device__ void fx_series(const SolveArgs& a, int c, int off, int sz, int ib, fx128* zA, fx128* zB,
                          const int* ip, const uint16_t* ix, float (*red)[T / 32], double* red64) {
  constexpr int kR = T == kFxBigThreads ? kFxMax / kFxBigThreads : 1;  // rows per thread
  const bool l1 = a.norm == PR_NORM_L1;
  const double tau = l1 ? a.tol * (double)sz / (double)a.n : a.tol;
  const int fixed = a.replay ? a.replay[c] : -1;
  double civ[kR];
  fx128 Rf[kR];
  int e0[kR], e1[kR];
  double wl = 0.0;
#pragma unroll
  for (int r = 0; r < kR; r++) {
    const int i = threadIdx.x + r * T;
    civ[r] = 0.0;
    e0[r] = e1[r] = 0;
    if (i < sz) {
      civ[r] = a.c * a.p_inv[off + i];
      e0[r] = ip[i];
      e1[r] = ip[i + 1];
      wl += fabs(a.W[off + i]);
    }
  }
  const int F = fx_point(block_sum(wl, red64));
  int k = 0;
  fx128* cur = zA;
  fx128* nxt = zB;
  if (a.R0) {
    // warm start: R = R0 + r with the residual r = W + c A^T(R0/outdeg) - R0
    // (signed), from which the series continues
#pragma unroll
    for (int r = 0; r < kR; r++) {
      const int i = threadIdx.x + r * T;
      if (i < sz) {
        const double g0 = a.R0[off + i];
        Rf[r] = to_fx(g0, F);
        zA[i] = to_fx(g0 * civ[r], F);
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kR; r++) {
      const int i = threadIdx.x + r * T;
      if (i < sz) {
        const fx128 res = to_fx(a.W[off + i], F) + fx_row<kStaged>(a, zA, ix, ib, off, sz, e0[r], e1[r]) - Rf[r];
        Rf[r] += res;
        zB[i] = to_fx(from_fx(res, F) * civ[r], F);
      }
    }
    cur = zB;
    nxt = zA;
    k = 1;
  } else {
#pragma unroll
    for (int r = 0; r < kR; r++) {
      const int i = threadIdx.x + r * T;
      if (i < sz) {
        const double W = a.W[off + i];
        Rf[r] = to_fx(W, F);
        zA[i] = to_fx(W * civ[r], F);
      }
    }
  }
  __syncthreads();
  for (;;) {
    float part = 0.0f;
#pragma unroll
    for (int r = 0; r < kR; r++) {
      const int i = threadIdx.x + r * T;
      if (i < sz) {
        const fx128 p = fx_row<kStaged>(a, cur, ix, ib, off, sz, e0[r], e1[r]);  // the next term, exact
        Rf[r] += p;
        const double pd = from_fx(p, F);
        nxt[i] = to_fx(pd * civ[r], F);
        const float pf = abs_to_float(pd);
        part = l1 ? part + pf : fmaxf(part, pf);
      }
    }
    const float s2 = block_norm<T>(part, red, k & 1, !l1);  // also publishes nxt
    fx128* t = cur;
    cur = nxt;
    nxt = t;
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
#pragma unroll
  for (int r = 0; r < kR; r++) {
    const int i = threadIdx.x + r * T;
    if (i < sz) {
      const double R = from_fx(Rf[r], F);
      a.R[off + i] = R;
      a.zr[off + i] = R * a.p_inv[off + i];
    }
  }
  if (threadIdx.x == 0) a.iters[c] = k;
}

// one CTA of T threads per component of [cbeg, cbeg + gridDim.x); cap: the
// largest component of the launch (rows of the z buffers), ecap: staged
// edge capacity (a component with more internal edges reads its indices
// from global memory)
template <int T>
__global__ void __launch_bounds__(T, 1) solve_fx_k(SolveArgs a, int32_t cbeg, int32_t cap, int32_t ecap) {
  extern __shared__ __align__(16) unsigned char fx_sm[];
  fx128* zA = reinterpret_cast<fx128*>(fx_sm);
  fx128* zB = zA + cap;
  int* ip = reinterpret_cast<int*>(zB + cap);             // [cap + 1] local edge offsets
  uint16_t* ix = reinterpret_cast<uint16_t*>(ip + cap + 1);  // [ecap] local source indices
  __shared__ float red[2][T / 32];
  __shared__ double red64[T / 32];
  constexpr int kR = T == kFxBigThreads ? kFxMax / kFxBigThreads : 1;
  const int c = cbeg + (int)blockIdx.x;
  const int off = a.c_off[c], sz = a.c_off[c + 1] - off;
  const bool scc = a.c_type[c] == PR_TYPE_SCC;
  if (scc && sz < a.lu_threshold) return;  // solved by solve_lu_k (block-uniform)
  if (sz > cap || sz > kR * T) {           // launch does not match the layout
    if (threadIdx.x == 0) set_err(a.ctl, PR_EINTERNAL, 340);
    return;
  }
  const int ib = a.int_ptr[off];
  const int m = a.int_ptr[off + sz] - ib;
  const bool staged = m <= ecap;
  for (int i = threadIdx.x; i <= sz; i += T) ip[i] = a.int_ptr[off + i] - ib;
  if (staged)
    for (int e = threadIdx.x; e < m; e += T) ix[e] = (uint16_t)local_or_err(a, a.int_idx[ib + e] - off, sz);
  __syncthreads();
  if (scc) {
    if (staged) fx_series<T, true>(a, c, off, sz, ib, zA, zB, ip, ix, red, red64);
    else fx_series<T, false>(a, c, off, sz, ib, zA, zB, ip, ix, red, red64);
    return;
  }
  // CAC: one FP64 pass, sub-level by sub-level (topological order); z and R
  // in the space of the fixed-point buffers
  double* z = reinterpret_cast<double*>(zA);
  double* Rs = z + cap;
  for (int i = threadIdx.x; i < sz; i += T) {
    const double W = a.W[off + i];
    Rs[i] = W;
    z[i] = W * a.p_inv[off + i];
  }
  __syncthreads();
  const int sb = a.c_sub[c], se = a.c_sub[c + 1];
  for (int s2 = sb; s2 < se; s2++) {
    const int lo = a.sub_ptr[s2] - off, hi = a.sub_ptr[s2 + 1] - off;
    for (int i = lo + (int)threadIdx.x; i < hi; i += T) {
      double acc = 0.0;
      for (int e = ip[i]; e < ip[i + 1]; e++)
        acc += z[staged ? (int)ix[e] : local_or_err(a, a.int_idx[ib + e] - off, sz)];
      const double Rv = Rs[i] + a.c * acc;
      Rs[i] = Rv;
      z[i] = Rv * a.p_inv[off + i];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < sz; i += T) {
    a.R[off + i] = Rs[i];
    a.zr[off + i] = Rs[i] * a.p_inv[off + i];
  }
  if (threadIdx.x == 0) a.iters[c] = 0;
}

// dynamic shared memory of a launch (z pair, offsets, staged indices)
static size_t fx_smem(int cap, int ecap) {
  const size_t b = (size_t)2 * cap * sizeof(fx128) + ((size_t)cap + 1) * sizeof(int) + (size_t)ecap * sizeof(uint16_t);
  return (b + 15) / 16 * 16;
}

// shared memory budget per CTA: the 1024-thread launches take one SM each;
// the 256-thread ones stay small enough for several per SM
constexpr size_t kFxBigSmem = 200 * 1024;
constexpr int kFxEdgeCap = 8192;

pr_status set_fx_attrs() {
  static bool done = false;
  if (done) return PR_OK;
  PRGB_CUDA(cudaFuncSetAttribute(solve_fx_k<kFxBigThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kFxBigSmem));
  PRGB_CUDA(cudaFuncSetAttribute(solve_fx_k<kFxThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fx_smem(kCtaCompMax, kFxEdgeCap)));
  done = true;
  return PR_OK;
}

pr_status launch_fx(const SolveArgs& a, int32_t cbeg, int32_t cend, int32_t max_size, bool big, cudaStream_t s) {
  if (cend <= cbeg) return PR_OK;
  PRGB_TRY(set_fx_attrs());
  const unsigned nb = (unsigned)(cend - cbeg);
  if (big) {
    const int cap = max_size;
    if (cap > kFxMax) return PR_EINTERNAL;
    const size_t base = fx_smem(cap, 0);
    const int ecap = (int)std::min<size_t>((kFxBigSmem - base) / sizeof(uint16_t), (size_t)1 << 20);
    solve_fx_k<kFxBigThreads><<<nb, kFxBigThreads, fx_smem(cap, ecap), s>>>(a, cbeg, cap, ecap);
  } else {
    const int cap = std::min<int>(max_size, kCtaCompMax);
    if (max_size > kFxThreads) return PR_EINTERNAL;
    solve_fx_k<kFxThreads><<<nb, kFxThreads, fx_smem(cap, kFxEdgeCap), s>>>(a, cbeg, cap, kFxEdgeCap);
  }
  PRGB_LAUNCH();
  return PR_OK;
}

}  // namespace prgb
