// warp_solve.cuh -- one warp per component of 2..32 vertices (Sec. 4.3:
// CACs in one topological pass, SCCs by the power series of Sec. 4.3.2),
// the warp items of the persistent level kernel.
#pragma once

#include "common.cuh"
#include "fx128.cuh"
#include "mpnn.cuh"
#include "solve.cuh"

namespace prgb {

// Mixed precision (the SCC series of the cluster class; the gather, CACs
// and 1-vertex components stay FP64, and the other SCCs run the exact
// fixed-point series in either mode).  Per SCC C with budget
// tau = tol*|C|/n:
//   1. the series P_0 = W, P_{k+1} = c A^T P_k, F = sum P_k in FP32 values
//      and FP32 accumulation, until the FP32 norm of P falls to
//      max(tau, kMixKappa * ||W||_1): below that FP32 rounding of F
//      dominates what further terms would add;
//   2. R += F in FP64 and the FP64 residual r = W + c A^T (R/outdeg) - R,
//      its L1 norm rho; done when rho <= tau;
//   3. otherwise solve (I - c A^T) D = r by the same series in FP32 from
//      P_0 = r (signed), until the FP32 norm of P falls to
//      max(tau/2, kMixKappa * rho); F = D, back to 2.
// Each FP32 pass gains about six digits, so one or two rounds of 2-3 meet
// any budget above ~1e-13 ||R||_1; after kMixRounds residuals above tau the
// component is reported as not converged (PR_ENOCONV).  The final per-SCC
// residual check is FP64, so the L1 residual budget holds as in FP64 mode.
constexpr float kMixKappa = 8.0f * 5.9604645e-8f;  // 8 * 2^-24
constexpr int kMixRounds = 6;


// ---------------------------------------------------------------------------
// one warp per component of 2..32 vertices, one vertex per lane.  The
// component's internal in-edges (at most 32*31) are staged in shared memory
// as 8-bit local indices, so each series iteration reads shared memory only.
// ---------------------------------------------------------------------------
constexpr int kWarpEdges = kWarpCompMax * (kWarpCompMax - 1);
// the warp's z space: 32 fixed-point entries (an SCC's series) or 32 doubles
// (a CAC's pass); 16-byte aligned
constexpr int kWarpZBytes = 32 * 16;

// Warm start of a warp's fixed-point series from the network's guess
// R0 = W + exp(clamp(yhat)) mean_C(W): R = R0 + r, the series continuing from
// the residual r = W + c A^T(R0/outdeg) - R0 (signed), written to zx as
// r c/outdeg with *Rf = R0 + r -- if the guess pays: a residual of at least
// c ||W_C||_1 (the cold series' next term is at most that) returns false,
// the caller then starts from W (*Rf = W is left as it was).  Run once per
// component, outside the sweep loop's registers.
static __device__ __noinline__ bool warp_fx_warm(const SolveArgs& a, int p, bool act, double W, double mean, int F,
                                                 FxMul mul, const uint8_t* ix, int ib, int ie, fx128* zx, fx128* Rf) {
  const int lane = threadIdx.x & 31;
  const fx128 r0 =
      act ? to_fx(W + (double)expf(fminf(fmaxf(a.yhat[p], kMpYMin), kMpYMax)) * mean, F) : (fx128)0;
  if (act) zx[lane] = fx_scale(r0, mul);
  __syncwarp();
  fx128 acc = 0;
  for (int e = ib; e < ie; e++) acc += zx[ix[e]];
  const fx128 res = act ? *Rf + acc - r0 : (fx128)0;
  __syncwarp();
  const double wsum = mean * (double)__popc(__ballot_sync(0xffffffffu, act));
  if (!((double)group_sumf<32>(fx_abs_float(res, F)) < a.c * wsum)) return false;
  *Rf = r0 + res;
  if (act) zx[lane] = fx_scale(res, mul);
  return true;
}

// One warp solves component c in its own shared memory: zbuf (kWarpZBytes,
// 16-byte aligned) and ix (kWarpEdges bytes).  FP64 mode runs the SCC
// series in exact 128-bit fixed point (fx128.cuh, as for the larger
// components): a row's in-edge sum and R are exact integer sums, z' = P
// c/outdeg the exact product rounded once, and a sweep has no floating-point
// arithmetic.  CACs take one FP64 pass over their sub-levels.
static __device__ void warp_component(const SolveArgs& a, int c, unsigned char* zbuf, uint8_t* ix) {
  const int lane = threadIdx.x & 31;
  const int off = a.c_off[c], sz = a.c_off[c + 1] - off;
  if (sz < a.lu_threshold && a.c_type[c] == PR_TYPE_SCC) return;  // solved by solve_lu_k (warp-uniform)
  double* z = reinterpret_cast<double*>(zbuf);
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
    const float thr = stop_thr32(tau);
    const int fixed = a.replay ? a.replay[c] : -1;
    // z holds c P / outdeg in fixed point, so that the in-edge sum is the
    // next term itself
    fx128* zx = reinterpret_cast<fx128*>(zbuf);
    const double wsum = group_sum<32>(W);  // W >= 0
    const int F = fx_point(wsum);
    const FxMul mul = fx_mul_of(a.c * inv);
    fx128 Rf = act ? to_fx(W, F) : (fx128)0;
    const bool cold = !(a.yhat && warp_fx_warm(a, p, act, W, wsum / (double)sz, F, mul, ix, ib, ie, zx, &Rf));
    if (cold && act) zx[lane] = fx_scale(Rf, mul);
    if (!cold) k = 1;
    const float qscale = norm_q_scale(thr);
    __syncwarp();
    for (;;) {
      // two carry chains of exact adds
      fx128 s0 = 0, s1 = 0;
      int e = ib;
      for (; e + 1 < ie; e += 2) {
        s0 += zx[ix[e]];
        s1 += zx[ix[e + 1]];
      }
      if (e < ie) s0 += zx[ix[e]];
      const fx128 pn = s0 + s1;  // the next term, exact
      __syncwarp();
      if (act) {
        zx[lane] = fx_scale(pn, mul);
        Rf += pn;
      }
      __syncwarp();
      k++;
      if (fixed >= 0) {
        if (k >= fixed) break;
        continue;
      }
      const unsigned q = norm_q(fx_abs_float(pn, F), qscale);  // terms are signed after a warm start
      const unsigned s = a.norm == PR_NORM_L1 ? __reduce_add_sync(0xffffffffu, q) : __reduce_max_sync(0xffffffffu, q);
      if (!keep_going_q(s, a.norm)) break;
      if (k >= a.max_iter) {
        if (lane == 0) atomicOr(&a.ctl->flags[0], 1);
        break;
      }
    }
    R = act ? from_fx(Rf, F) : 0.0;
  }
  if (act) {
    a.R[p] = R;
    a.zr[p] = R * inv;
  }
  if (lane == 0) a.iters[c] = k;
}

}  // namespace prgb
