// giant_fx.cu -- the power series of Sec. 4.3.2 for an SCC too large for a
// CTA cluster, swept by the whole grid (one cooperative launch, a grid
// barrier per sweep), in exact 128-bit fixed point (fx128.cuh).
//
// The FP64 form of this sweep spends about half of its time in the FP64
// pipe, which GB300 keeps small: every edge is one FP64 add.  Here the
// terms are integers at a binary point F fixed per component, so a row's
// in-edge sum is a chain of 128-bit integer adds (exact, in any order),
// z' = P c/outdeg is the exact product rounded once (fx_scale), and R is an
// exact running sum; a sweep issues no floating-point instruction but the
// stopping norm's FP32 conversion.  The results equal the real-number
// series up to one rounding of each z (and, where z is gathered as FP64
// values, its rounding to the nearest double) and of the final R.
//
// The stopping norm is reduced on integers too: each row contributes
// q = ceil(|P_i| 2^32 / thr) (thr = tau / (1 + 1e-4) rounded down to FP32
// once, |P_i| truncated to FP32 -- the margin of stop_thr32), capped at 2^33;
// a block adds its rows' q in shared memory and one 64-bit atomic per block
// (capped at 2^40) folds it into the sweep's slot.  Integer sums do not
// depend on the order of the atomics, so the sweep count is deterministic;
// the rounding up of q makes the test conservative (at most |C| 2^-32 thr
// of overestimate).
#include "common.cuh"
#include "fx128.cuh"
#include "solve.cuh"
#include "spmv.cuh"

namespace prgb {

constexpr unsigned long long kGNormOne = 1ULL << 32;  // thr in q units
constexpr float kGNormOneF = 4294967296.0f;
constexpr float kGNormMaxF = 8589934592.0f;           // 2^33: one row at twice thr
constexpr unsigned long long kGBlockCap = 1ULL << 40; // a block this far above thr decides alone

__device__ __forceinline__ unsigned long long gnorm_q(float pf, float scale) {
  if (!(pf > 0.0f)) return 0ULL;
  return scale > 0.0f ? __float2ull_ru(fminf(__fmul_ru(pf, scale), kGNormMaxF))
                      : (unsigned long long)kGNormMaxF;
}

__device__ __forceinline__ unsigned long long warp_fold_u64(unsigned long long v, bool l1) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
    v = l1 ? v + t : (t > v ? t : v);
  }
  return v;
}

__device__ __forceinline__ fx128 warp_sum_fx(fx128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)((ufx128)v >> 64);
    const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o), h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    v += (fx128)(((ufx128)h2 << 64) | (ufx128)l2);
  }
  return v;
}

// a 16-byte fixed-point value written by another block (L2, not L1)
__device__ __forceinline__ fx128 ld_cg_fx(const fx128* p) {
  const int4 v = __ldcg(reinterpret_cast<const int4*>(p));
  const ufx128 lo = (ufx128)(((unsigned long long)(unsigned)v.y << 32) | (unsigned)v.x);
  const ufx128 hi = (ufx128)(((unsigned long long)(unsigned)v.w << 32) | (unsigned)v.z);
  return (fx128)((hi << 64) | lo);
}

// The gathered vector z = P c/outdeg: 16-byte fixed-point words (ZT =
// fx128) when the sweep fits in L2, else FP64 values (ZT = double, half the
// bytes of every gather that misses L2), each the fixed-point product
// rounded to the nearest double and decoded exactly into the row's
// fixed-point sum.
template <class ZT>
__device__ __forceinline__ fx128 z_load(const ZT* z, int q, int F) {
  if constexpr (sizeof(ZT) == 16) return z[q];
  else return to_fx(z[q], F);
}
template <class ZT>
__device__ __forceinline__ ZT z_value(fx128 p, FxMul mul, int F) {
  if constexpr (sizeof(ZT) == 16) return fx_scale(p, mul);
  else return from_fx(fx_scale(p, mul), F);
}

template <class ZT>
__device__ __forceinline__ void giant_fx_body(const SolveArgs& a, const LargeComp& L, const GiantFxBufs& g,
                                              const HeavyRows& hv) {
  __shared__ unsigned long long sh_acc, sh_val;
  ZT* const zA = reinterpret_cast<ZT*>(g.zA);
  ZT* const zB = reinterpret_cast<ZT*>(g.zB);
  const int lane = threadIdx.x & 31;
  const int off = L.off, sz = L.size;
  const int nlight = sz - hv.nheavy;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int64_t gw = tid >> 5, nw = nth >> 5;
  const bool l1 = a.norm == PR_NORM_L1;
  // binary point from a bound of ||W_C||_1 that does not depend on the
  // order of a sum: |C| max_i W_i (W >= 0, so the bit patterns order as the
  // values do)
  unsigned long long wb = 0;
  for (int64_t i = tid; i < sz; i += nth) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(a.W[off + i]);
    wb = b > wb ? b : wb;
  }
  wb = warp_fold_u64(wb, false);
  if (lane == 0 && wb) atomicMax(&g.acc[3], wb);
  if (!grid_sync(a.ctl, 320)) return;
  const double wmax = __longlong_as_double((long long)__ldcg(&g.acc[3]));
  const int F = fx_point(wmax * (double)sz);
  // R = W (cold) or the guess R0 (warm), z = R c/outdeg; slot sz of both z
  // buffers holds the 0 that SELL padding reads
  const bool warm0 = a.R0 != nullptr;
  for (int64_t i = tid; i < sz; i += nth) {
    const int p = off + (int)i;
    const fx128 R = to_fx(warm0 ? a.R0[p] : a.W[p], F);
    g.R[i] = R;
    zA[i] = z_value<ZT>(R, fx_mul_of(a.civ[p]), F);
  }
  if (tid == 0) {
    zA[sz] = 0;
    zB[sz] = 0;
  }
  const bool sell = L.sell_end > L.sell_begin;
  int ls0 = 0, ls1 = 0, lr0 = -1, lr1 = -1;
  if (sell) warp_slice_range(a.sell_cpre + L.sell_begin, L.sell_end - L.sell_begin, &ls0, &ls1);
  else if (a.lpre) warp_row_range(a.lpre + off, nlight, &lr0, &lr1);
  const int* lorder = a.lorder + off;
  if (!grid_sync(a.ctl, 321)) return;
  const double tau = l1 ? a.tol * (double)sz / (double)a.n : a.tol;
  const float thr = stop_thr32(tau);
  const float qs = thr > 0.0f ? kGNormOneF / thr : 0.0f;
  const int fixed = a.replay ? a.replay[L.c] : -1;
  int k = 0;
  for (;;) {
    // the first sweep of a warm start forms the residual
    // r = W + c A^T(R0/outdeg) - R0 (signed) and continues from it
    const bool warm = warm0 && k == 0;
    const ZT* cur = (k & 1) ? zB : zA;
    ZT* nxt = (k & 1) ? zA : zB;
    unsigned long long local = 0;
    if (threadIdx.x == 0) {
      sh_acc = 0;
      // the slot of sweep k + 1 was last read after barrier k - 2
      if (blockIdx.x == 0) g.acc[(k + 1) % 3] = 0;
    }
    __syncthreads();
    auto fin = [&](int row, fx128 acc) -> unsigned long long {
      const int i = row - off;
      fx128 R = g.R[i];
      const fx128 pn = warm ? to_fx(a.W[row], F) + acc - R : acc;
      g.R[i] = R + pn;
      nxt[i] = z_value<ZT>(pn, fx_mul_of(a.civ[row]), F);
      return gnorm_q(fx_abs_float(pn, F), qs);
    };
    // heavy rows: a warp per chunk of kChunkH edges; the warp that brings a
    // row's last chunk adds the partials (exact, in any order)
    for (int64_t ch = gw; ch < hv.nchunks; ch += nw) {
      const int cha = (int)ch + hv.cbase;
      const int h = hv.chrow[cha] - hv.hbase;
      const int row = hv.rows[h];
      const int j = cha - hv.choff[h];
      const int e0 = a.int_ptr[row] + j * kChunkH;
      const int e1 = min(a.int_ptr[row + 1], e0 + kChunkH);
      fx128 acc = 0;
#pragma unroll
      for (int kk = 0; kk < kChunkH / 32; kk++) {
        const int e = e0 + kk * 32 + lane;
        if (e < e1) acc += z_load(cur, local_or_err(a, a.int_idx[e] - off, sz), F);
      }
      acc = warp_sum_fx(acc);
      const int nch = hv.choff[h + 1] - hv.choff[h];
      if (nch == 1) {
        if (lane == 0) {
          const unsigned long long q = fin(row, acc);
          local = l1 ? local + q : (q > local ? q : local);
        }
        continue;
      }
      int last = 0;
      if (lane == 0) {
        g.part[ch] = acc;
        __threadfence();
        last = atomicAdd(&g.cnt[h], 1) == nch - 1;
      }
      if (!__shfl_sync(0xffffffffu, last, 0)) continue;
      __threadfence();
      const int pb = hv.choff[h] - hv.cbase;
      fx128 t = 0;
      for (int q = lane; q < nch; q += 32) t += ld_cg_fx(&g.part[pb + q]);
      t = warp_sum_fx(t);
      if (lane == 0) {
        g.cnt[h] = 0;
        const unsigned long long q = fin(row, t);
        local = l1 ? local + q : (q > local ? q : local);
      }
    }
    // light rows
    if (sell) {
      const int32_t* sptr = a.sell_ptr + L.sell_begin;
      for (int s = ls0; s < ls1; s++) {
        const int b = sptr[s], w = (sptr[s + 1] - b) >> 5;
        const int32_t* pp = a.sell_idx + b + lane;  // entries <= sz by construction of the slices
        fx128 a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        int kk = 0;
        for (; kk + 3 < w; kk += 4) {
          a0 += z_load(cur, pp[32 * kk], F);
          a1 += z_load(cur, pp[32 * (kk + 1)], F);
          a2 += z_load(cur, pp[32 * (kk + 2)], F);
          a3 += z_load(cur, pp[32 * (kk + 3)], F);
        }
        for (; kk < w; kk++) a0 += z_load(cur, pp[32 * kk], F);
        const int i = 32 * s + lane;
        if (i < L.nlight) {
          const unsigned long long q = fin(off + i, (a0 + a1) + (a2 + a3));
          local = l1 ? local + q : (q > local ? q : local);
        }
      }
    } else {
      const bool ranged = lr0 >= 0;
      const int64_t lb = ranged ? lr0 : gw * 32, le = ranged ? lr1 : nlight, ls = ranged ? 32 : nw * 32;
      for (int64_t base = lb; base < le; base += ls) {
        const int64_t i = base + lane;
        if (i < le) {
          const int row = lorder[i];
          fx128 acc = 0;
          for (int e = a.int_ptr[row]; e < a.int_ptr[row + 1]; e++)
            acc += z_load(cur, local_or_err(a, a.int_idx[e] - off, sz), F);
          const unsigned long long q = fin(row, acc);
          local = l1 ? local + q : (q > local ? q : local);
        }
      }
    }
    // the sweep's norm: warp, block (shared), grid (one atomic per block)
    local = warp_fold_u64(local, l1);
    if (lane == 0 && local) {
      if (l1) atomicAdd(&sh_acc, local);
      else atomicMax(&sh_acc, local);
    }
    __syncthreads();
    if (threadIdx.x == 0 && sh_acc) {
      const unsigned long long v = sh_acc < kGBlockCap ? sh_acc : kGBlockCap;
      if (l1) atomicAdd(&g.acc[k % 3], v);
      else atomicMax(&g.acc[k % 3], v);
    }
    if (!grid_sync(a.ctl, 322)) return;
    if (threadIdx.x == 0) sh_val = __ldcg(&g.acc[k % 3]);
    __syncthreads();
    const unsigned long long s = sh_val;
    k++;
    if (fixed >= 0) {
      if (k >= fixed) break;
      continue;
    }
    if (!(l1 ? s > kGNormOne : s >= kGNormOne)) break;
    if (k >= a.max_iter) {
      if (tid == 0) atomicOr(&a.ctl->flags[0], 1);
      break;
    }
  }
  for (int64_t i = tid; i < sz; i += nth) {
    const int p = off + (int)i;
    const double R = from_fx(g.R[i], F);
    a.R[p] = R;
    a.zr[p] = R * a.p_inv[p];
  }
  if (tid == 0) a.iters[L.c] = k;
}

__global__ void __launch_bounds__(kBlock) solve_large_scc_fx_k(SolveArgs a, LargeComp L, GiantFxBufs g,
                                                               HeavyRows hv) {
  giant_fx_body<fx128>(a, L, g, hv);
}

__global__ void __launch_bounds__(kBlock) solve_large_scc_fxd_k(SolveArgs a, LargeComp L, GiantFxBufs g,
                                                                HeavyRows hv) {
  giant_fx_body<double>(a, L, g, hv);
}

}  // namespace prgb
