// solve_fx.cu -- the power series of Sec. 4.3.2 for SCCs of 33..kFxMax
// vertices, one CTA per component, with exact fixed-point row sums.
//
// P_0 = W, P_{k+1} = c A^T P_k, R = sum_k P_k, per component, stopping by
// the same rule as the other kernels (L1: after adding P with
// ||P||_1 <= tol |C| / n; L-inf: the paper's max(P) < tol).  The gathered
// vector is z = c P / outdeg, so a row's in-edge sum is the next term.
//
// All of a component's state stays in shared memory and registers.  What
// differs from the FP64 kernels is the arithmetic: z is stored as 128-bit
// fixed point (fx128.cuh) with a binary point chosen once per component from
// ||W_C||_1, a row's sum of z over its in-edges is an exact integer sum, R
// accumulates the terms exactly, and z' = P c/outdeg is the exact product of
// the fixed-point P and the double c/outdeg, rounded once to the quantum.
// A sweep has no floating-point arithmetic at all: GB300 has many times its
// FP64 rate on the integer pipes.  The only roundings are the conversions
// (W in, R out) and the one per product, each far below an FP64 unit in
// the last place of the value, so every term is at least as accurate as the
// FP64 series' term and sums lose nothing (the FP64 kernels round once per
// edge).

// CACs in the same size range are solved in FP64 by one pass over their
// topological sub-levels (Sec. 4.3.1), exactly as in the other kernels.
//
// The persistent level kernel (solve_level_k) takes every component of a
// level with at most kFxMax vertices in one launch: CTAs of 1024 threads
// pull work, largest first, from three size buckets -- components above
// cta_max vertices (one whole CTA each), up to cta_max (one 256-thread
// quarter each, with a named barrier of its own) and up to 32 (one warp
// each) -- so the components of very uneven sizes of a level share the GPU
// without one launch per size class (Sec. 4.3, last paragraph: the
// components of a level are independent).
#include <algorithm>

#include "common.cuh"
#include "fx128.cuh"
#include "mpnn.cuh"
#include "solve.cuh"
#include "warp_solve.cuh"

namespace prgb {

// A group of T threads that solves one component: a whole CTA of T threads
// (barrier 0) or one quarter of a 1024-thread CTA (named barrier 1 + q).
template <int T>
struct Grp {
  int tid;  // thread index in the group
  int bar;  // barrier id
  __device__ __forceinline__ void sync() const {
    if (bar == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(T) : "memory");
  }
};

// Shared memory of one group (its part of the CTA's, `bytes` long): the
// scratch (reduction partials and the per-warp slice widths), the z pair of
// cap + kFxZeros entries each (entries sz .. sz + 7 are the zeros that
// padded slice entries read, one per bank group), then the staged in-edges.
constexpr int kFxScratch = 768;
constexpr int kFxZeros = 8;
__host__ __device__ constexpr size_t fx_group_fixed(int cap) {
  return kFxScratch + (size_t)2 * (cap + kFxZeros) * sizeof(fx128);
}

// deterministic sum over the group (fixed tree)
template <int T>
__device__ __forceinline__ double grp_sum(const Grp<T>& g, double v, double* red64) {
  const int lane = g.tid & 31, wib = g.tid >> 5;
  v = group_sum<32>(v);
  g.sync();
  if (lane == 0) red64[wib] = v;
  g.sync();
  return group_sum<32>(lane < T / 32 ? red64[lane] : 0.0);
}

// sum of z over the in-edges [e0, e1) read from the global layout (the
// components whose edges do not fit the shared memory), two carry chains
__device__ __forceinline__ fx128 fx_row_global(const SolveArgs& a, const fx128* __restrict__ z, int ib, int off,
                                               int sz, int e0, int e1) {
  fx128 s0 = 0, s1 = 0;
  int e = e0;
  for (; e + 1 < e1; e += 2) {
    const int q0 = local_or_err(a, a.int_idx[ib + e] - off, sz);
    const int q1 = local_or_err(a, a.int_idx[ib + e + 1] - off, sz);
    s0 += z[q0];
    s1 += z[q1];
  }
  if (e < e1) s0 += z[local_or_err(a, a.int_idx[ib + e] - off, sz)];
  return s0 + s1;
}

// warp partials, one barrier, then every warp folds the same partials in
// the same order (deterministic, no second barrier)
template <int T>
__device__ __forceinline__ float grp_norm(const Grp<T>& g, float part, float* red, int parity, bool is_max) {
  constexpr int kNW = T / 32;
  const int lane = g.tid & 31, wib = g.tid >> 5;
  part = is_max ? group_maxf<32>(part) : group_sumf<32>(part);
  if (lane == 0) red[parity * kNW + wib] = part;
  g.sync();
  const float t = lane < kNW ? red[parity * kNW + lane] : 0.0f;
  return is_max ? group_maxf<32>(t) : group_sumf<32>(t);
}

// the same over the integer norm (norm_q): one redux.sync a warp, one
// barrier, one redux.sync over the warps' partials
template <int T>
__device__ __forceinline__ unsigned grp_norm_q(const Grp<T>& g, unsigned q, unsigned* red, int parity,
                                               bool is_max) {
  constexpr int kNW = T / 32;
  const int lane = g.tid & 31, wib = g.tid >> 5;
  q = is_max ? __reduce_max_sync(0xffffffffu, q) : __reduce_add_sync(0xffffffffu, q);
  if (lane == 0) red[parity * kNW + wib] = q;
  g.sync();
  const unsigned t = lane < kNW ? red[parity * kNW + lane] : 0u;
  return is_max ? __reduce_max_sync(0xffffffffu, t) : __reduce_add_sync(0xffffffffu, t);
}

// The series of SCC c, one row per thread (sz <= T).
//
// The in-edges are staged as one slice per warp (SELL-32, Sec. 4.3.2's
// sweep is a gather over them): lane l of warp w holds its row's local
// source indices, 16 bits each, four to an 8-byte word, word j at
// slice_w + 32 j + l, and each word load is one coalesced access for the
// warp.  Where the partition holds the component's conflict-free slices
// (fx_sched.cu: every column's eight lanes of a phase read distinct bank
// groups of z), they are copied in; otherwise they are built here from the
// CSR, every row of the warp padded to the warp's longest (rounded up to 4)
// with index sz, whose z entry is zero (the layout order puts rows of
// similar in-degree next to each other, so the padding is small).
//
// Per sweep and row: the exact fixed-point sum of z over the in-edges (the
// next term p), R += p, z' = p c/outdeg as the exact product rounded once to
// the fixed-point quantum, and |p| as a float for the stopping norm: no
// floating-point arithmetic.
template <int T>
__device__ void fx_series(const SolveArgs& a, const Grp<T>& g, int c, int off, int sz, int ib, int m,
                          unsigned char* base, size_t bytes, int cap) {
  constexpr int kNW = T / 32;
  float* red = reinterpret_cast<float*>(base);                 // [2][kNW]
  double* red64 = reinterpret_cast<double*>(base + 256);       // [kNW]
  int* wcnt = reinterpret_cast<int*>(base + 512);              // [kNW] words per lane of each slice
  fx128* zA = reinterpret_cast<fx128*>(base + kFxScratch);
  fx128* zB = zA + cap + kFxZeros;
  unsigned char* tail = reinterpret_cast<unsigned char*>(zB + cap + kFxZeros);
  const size_t room = bytes - (size_t)(tail - base);
  const int i = g.tid, lane = i & 31, wib = i >> 5;
  const bool act = i < sz;
  const bool l1 = a.norm == PR_NORM_L1;
  const double tau = l1 ? a.tol * (double)sz / (double)a.n : a.tol;
  const float thr = stop_thr32(tau);
  const int fixed = a.replay ? a.replay[c] : -1;
  const FxMul mul = fx_mul_of(act ? a.c * a.p_inv[off + i] : 0.0);
  const int e0 = act ? a.int_ptr[off + i] - ib : 0, e1 = act ? a.int_ptr[off + i + 1] - ib : 0;
  const bool pre = a.fxs_ptr != nullptr && a.fxs_ptr[c] >= 0;
  int words;
  if (pre) words = wib < (sz + 31) / 32 ? (int)a.fxs_wcnt[a.fxs_wbase[c] + wib] : 0;
  else words = (int)((__reduce_max_sync(0xffffffffu, (unsigned)(e1 - e0)) + 3) >> 2);
  if (lane == 0) wcnt[wib] = words;
  if (i < kFxZeros) {
    zA[sz + i] = 0;
    zB[sz + i] = 0;
  }
  g.sync();
  int slice = 0, total = 0;  // this warp's first word, all slices' words
  for (int w = 0; w < kNW; w++) {
    const int u = wcnt[w] * 32;
    slice += w < wib ? u : 0;
    total += u;
  }
  // sliced: the rows read slices (else each row reads its CSR from global)
  bool sliced;
  const uint2* ell;
  if (pre) {
    // the partition's slices: copied in when they fit, else read in place
    const uint2* src = a.fxs_words + a.fxs_ptr[c];
    const bool fits = (size_t)total * 8 <= room;
    if (fits)
      for (int t = i; t < total; t += T) reinterpret_cast<uint2*>(tail)[t] = src[t];
    ell = (fits ? reinterpret_cast<const uint2*>(tail) : src) + slice + lane;
    sliced = true;
  } else {
    // the slices, built from a staged copy of the CSR at the end of the space
    sliced = (size_t)total * 8 + (size_t)m * 2 <= room;
    ell = reinterpret_cast<const uint2*>(tail) + slice + lane;
    if (sliced) {
      uint16_t* csr = reinterpret_cast<uint16_t*>(base + bytes) - m;
      for (int e = i; e < m; e += T) csr[e] = (uint16_t)local_or_err(a, a.int_idx[ib + e] - off, sz);
      g.sync();
      uint2* dst = reinterpret_cast<uint2*>(tail) + slice + lane;
      const unsigned pad = (unsigned)sz;
      for (int j = 0; j < words; j++) {
        const int e = e0 + 4 * j;
        const unsigned q0 = e < e1 ? csr[e] : pad, q1 = e + 1 < e1 ? csr[e + 1] : pad;
        const unsigned q2 = e + 2 < e1 ? csr[e + 2] : pad, q3 = e + 3 < e1 ? csr[e + 3] : pad;
        dst[32 * j] = make_uint2(q0 | (q1 << 16), q2 | (q3 << 16));
      }
    }
  }
  const double wsum = grp_sum(g, act ? fabs(a.W[off + i]) : 0.0, red64);  // its barriers publish the slices
  const int F = fx_point(wsum);
  auto row = [&](const fx128* __restrict__ z) -> fx128 {
    if (!sliced) return act ? fx_row_global(a, z, ib, off, sz, e0, e1) : (fx128)0;
    fx128 s0 = 0, s1 = 0;
#pragma unroll 1
    for (int j = 0; j < words; j++) {
      const uint2 v = ell[32 * j];
      const fx128 a0 = z[v.x & 0xffffu], a1 = z[v.x >> 16], a2 = z[v.y & 0xffffu], a3 = z[v.y >> 16];
      s0 += a0;
      s1 += a1;
      s0 += a2;
      s1 += a3;
    }
    return s0 + s1;
  };
  fx128 Rf = 0;
  int k = 0;
  fx128* cur = zA;
  fx128* nxt = zB;
  bool cold = true;
  if (a.yhat) {
    // warm start from the network's guess R0 = W + exp(clamp(yhat)) mean_C(W):
    // R = R0 + r with the residual r = W + c A^T(R0/outdeg) - R0 (signed),
    // from which the series continues -- if the guess pays: the cold
    // series' next term is at most c ||W_C||_1, so a residual at least that
    // large means starting from W instead (one sweep lost at most)
    if (act) {
      const float y = fminf(fmaxf(a.yhat[off + i], kMpYMin), kMpYMax);
      Rf = to_fx(a.W[off + i] + (double)expf(y) * (wsum / (double)sz), F);
      zA[i] = fx_scale(Rf, mul);
    }
    g.sync();
    const fx128 s = row(zA);
    fx128 res = 0;
    if (act) res = to_fx(a.W[off + i], F) + s - Rf;
    const float rn = grp_norm(g, act ? fx_abs_float(res, F) : 0.0f, red, 0, false);  // after every read of zA
    cold = !((double)rn < a.c * wsum);
    if (!cold) {
      if (act) {
        Rf += res;
        zB[i] = fx_scale(res, mul);
      }
      cur = zB;
      nxt = zA;
      k = 1;
    }
  }
  if (cold && act) {
    Rf = to_fx(a.W[off + i], F);
    zA[i] = fx_scale(Rf, mul);
  }
  g.sync();
  const float qscale = norm_q_scale(thr);
  for (;;) {
    const fx128 p = row(cur);  // the next term, exact
    unsigned q = 0u;
    if (act) {
      Rf += p;
      nxt[i] = fx_scale(p, mul);
      q = norm_q(fx_abs_float(p, F), qscale);
    }
    const unsigned s2 = grp_norm_q(g, q, reinterpret_cast<unsigned*>(red), k & 1, !l1);  // also publishes nxt
    fx128* t = cur;
    cur = nxt;
    nxt = t;
    k++;
    if (fixed >= 0) {
      if (k >= fixed) break;
      continue;
    }
    if (!keep_going_q(s2, a.norm)) break;
    if (k >= a.max_iter) {
      if (g.tid == 0) atomicOr(&a.ctl->flags[0], 1);
      break;
    }
  }
  if (act) {
    const double R = from_fx(Rf, F);
    a.R[off + i] = R;
    a.zr[off + i] = R * a.p_inv[off + i];
  }
  if (g.tid == 0) a.iters[c] = k;
}

// Component c (at most cap <= T vertices) by a group of T threads in the
// `bytes` of shared memory at base.
template <int T>
__device__ void fx_component(const SolveArgs& a, const Grp<T>& g, int c, unsigned char* base, size_t bytes, int cap) {
  const int off = a.c_off[c], sz = a.c_off[c + 1] - off;
  const bool scc = a.c_type[c] == PR_TYPE_SCC;
  if (scc && sz < a.lu_threshold) return;  // solved by solve_lu_k (group-uniform)
  if (sz > cap || sz > T) {                // the work does not match the layout
    if (g.tid == 0) set_err(a.ctl, PR_EINTERNAL, 340);
    return;
  }
  g.sync();  // the group's previous component is done with this memory
  const int ib = a.int_ptr[off];
  const int m = a.int_ptr[off + sz] - ib;
  if (scc) {
    fx_series(a, g, c, off, sz, ib, m, base, bytes, cap);
    return;
  }
  // CAC: one FP64 pass, sub-level by sub-level (topological order); z and R
  // in the space of the fixed-point buffers, the CSR staged after them
  double* z = reinterpret_cast<double*>(base + kFxScratch);
  double* Rs = z + cap;
  int* ip = reinterpret_cast<int*>(base + fx_group_fixed(cap));  // [cap + 1] local edge offsets
  uint16_t* ix = reinterpret_cast<uint16_t*>(ip + cap + 1);      // local source indices
  const bool staged = (size_t)m * sizeof(uint16_t) <= bytes - (size_t)(reinterpret_cast<unsigned char*>(ix) - base);
  for (int i = g.tid; i <= sz; i += T) ip[i] = a.int_ptr[off + i] - ib;
  if (staged)
    for (int e = g.tid; e < m; e += T) ix[e] = (uint16_t)local_or_err(a, a.int_idx[ib + e] - off, sz);
  for (int i = g.tid; i < sz; i += T) {
    const double W = a.W[off + i];
    Rs[i] = W;
    z[i] = W * a.p_inv[off + i];
  }
  g.sync();
  const int sb = a.c_sub[c], se = a.c_sub[c + 1];
  for (int s2 = sb; s2 < se; s2++) {
    const int lo = a.sub_ptr[s2] - off, hi = a.sub_ptr[s2 + 1] - off;
    for (int i = lo + g.tid; i < hi; i += T) {
      double acc = 0.0;
      for (int e = ip[i]; e < ip[i + 1]; e++)
        acc += z[staged ? (int)ix[e] : local_or_err(a, a.int_idx[ib + e] - off, sz)];
      const double Rv = Rs[i] + a.c * acc;
      Rs[i] = Rv;
      z[i] = Rv * a.p_inv[off + i];
    }
    g.sync();
  }
  for (int i = g.tid; i < sz; i += T) {
    a.R[off + i] = Rs[i];
    a.zr[off + i] = Rs[i] * a.p_inv[off + i];
  }
  if (g.tid == 0) a.iters[c] = 0;
}

// ---------------------------------------------------------------------------
// the persistent level kernel
// ---------------------------------------------------------------------------
constexpr int kLevelThreads = 1024;
constexpr int kQuarter = 256;
constexpr size_t kLevelSmem = 200 * 1024;  // one CTA per SM
constexpr size_t kQuarterBytes = kLevelSmem / 4;
constexpr size_t kWarpBytes = kWarpZBytes + kWarpEdges;
static_assert(kWarpBytes % 16 == 0, "every warp's z space stays 16-byte aligned");
static_assert(kLevelThreads / kQuarter == 4, "four quarters per CTA");
static_assert(kCtaCompMax <= kQuarter, "a quarter holds one row per thread");

// The three buckets of one level: [big0, big1) whole-CTA items (largest
// component big_max vertices), [mid0, mid1) quarter items, [small0, small1)
// warp items; ctr: the level's three claim counters (zero at launch).
struct LevelWork {
  int32_t big0, big1, mid0, mid1, small0, small1;
  int32_t big_max;
};

// Claims.  The first round is static, so that the largest items land on
// distinct SMs: CTA b < nb = min(#whole-CTA items, G) takes whole-CTA item b,
// quarter q of CTA b >= nb takes quarter item q (G - nb) + b - nb (the CTAs
// busy with a whole-CTA item get no quarter item in the first round), and
// warp j of the r-th quarter left without a quarter item (quarters counted
// layer by layer, q = 0 first) takes warp item d F + r with d = (j - q) mod 8,
// F such quarters in all (so the first warp items of a CTA's quarters sit on
// different SM sub-partitions, warp j running on sub-partition j mod 4).
// Later claims come from the counters, offset past the static indices.
__global__ void __launch_bounds__(kLevelThreads, 1) solve_level_k(SolveArgs a, LevelWork w, int32_t* ctr) {
  extern __shared__ __align__(16) unsigned char lv_sm[];
  __shared__ int claim[5];
  const int G = (int)gridDim.x, b = (int)blockIdx.x;
  const int nb = min(w.big1 - w.big0, G);
  // whole-CTA items, largest first
  const Grp<kLevelThreads> g{(int)threadIdx.x, 0};
  for (bool first = true;; first = false) {
    __syncthreads();
    if (threadIdx.x == 0) claim[0] = first && b < nb ? b : nb + atomicAdd(&ctr[0], 1);
    __syncthreads();
    const int c = w.big0 + claim[0];
    if (c >= w.big1) break;
    fx_component(a, g, c, lv_sm, kLevelSmem, w.big_max);
  }
  // quarter items, each quarter on its own part of the shared memory
  const int q = (int)threadIdx.x / kQuarter;
  const Grp<kQuarter> gq{(int)threadIdx.x % kQuarter, 1 + q};
  unsigned char* qbase = lv_sm + (size_t)q * kQuarterBytes;
  const int free_ctas = G - nb;
  for (bool first = b >= nb;; first = false) {
    gq.sync();
    if (gq.tid == 0) claim[1 + q] = first ? q * free_ctas + (b - nb) : 4 * free_ctas + atomicAdd(&ctr[1], 1);
    gq.sync();
    const int c = w.mid0 + claim[1 + q];
    if (c >= w.mid1) break;
    fx_component(a, gq, c, qbase, kQuarterBytes, kCtaCompMax);
  }
  // warp items in the quarter's memory, once its last quarter item is done
  const int lane = threadIdx.x & 31, wq = gq.tid >> 5;
  const int nmid = w.mid1 - w.mid0;
  int nfree = 0, rank = -1;  // quarters without a first-round quarter item; this one's rank among them
  for (int l = 0; l < kLevelThreads / kQuarter; l++) {
    const int lo = nb + min(max(nmid - l * free_ctas, 0), free_ctas);  // layer l is free on CTAs [lo, G)
    if (l == q && b >= lo) rank = nfree + (b - lo);
    nfree += G - lo;
  }
  unsigned char* wb = qbase + (size_t)wq * kWarpBytes;
  uint8_t* ix = wb + kWarpZBytes;
  for (bool first = rank >= 0;; first = false) {
    int i = 0;
    const int d = (wq - q + kQuarter / 32) % (kQuarter / 32);
    if (lane == 0) i = first ? d * nfree + rank : (kQuarter / 32) * nfree + atomicAdd(&ctr[2], 1);
    i = __shfl_sync(0xffffffffu, i, 0);
    const int c = w.small0 + i;
    if (c >= w.small1) break;
    warp_component(a, c, wb, ix);
    __syncwarp();
  }
}

static_assert(fx_group_fixed(kCtaCompMax) + (kCtaCompMax + 1) * sizeof(int) + 4096 <= kQuarterBytes,
              "a quarter item fits its part");
static_assert(fx_group_fixed(kFxMax) + (kFxMax + 1) * sizeof(int) + 16384 <= kLevelSmem, "a CTA item fits");
static_assert(8 * kWarpBytes <= kQuarterBytes, "a quarter's warps fit its part");

pr_status set_fx_attrs() {
  static bool done = false;
  if (done) return PR_OK;
  PRGB_CUDA(cudaFuncSetAttribute(solve_level_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLevelSmem));
  done = true;
  return PR_OK;
}

pr_status launch_level(const SolveArgs& a, const LevelRange& r, int32_t* ctr, cudaStream_t s) {
  LevelWork w;
  w.big0 = r.big;
  w.big1 = r.cta;
  w.mid0 = r.cta;
  w.mid1 = r.warp;
  w.small0 = r.warp;
  w.small1 = r.single;
  w.big_max = r.big_max;
  if (w.big_max > kFxMax) return PR_EINTERNAL;
  // an SM per item while there are SMs (the first round spreads the items
  // over them, largest first)
  const int64_t units = (int64_t)(w.big1 - w.big0) + (w.mid1 - w.mid0) + (w.small1 - w.small0);
  if (units <= 0) return PR_OK;
  PRGB_TRY(set_fx_attrs());
  const unsigned grid = (unsigned)std::min<int64_t>(units, num_sms());
  solve_level_k<<<grid, kLevelThreads, kLevelSmem, s>>>(a, w, ctr);
  PRGB_LAUNCH();
  return PR_OK;
}

}  // namespace prgb
