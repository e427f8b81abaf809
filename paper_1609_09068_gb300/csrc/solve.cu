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
#include <type_traits>

#include <mutex>
#include <vector>

#include "common.cuh"
#include "mpnn.cuh"
#include "solve.cuh"
#include "spmv.cuh"
#include "warp_solve.cuh"

namespace cg = cooperative_groups;

namespace prgb {

// z = x / outdeg as x * (1/outdeg): the reciprocal is precomputed once per
// vertex, because FP64 division is expensive on this part.


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

// Shared memory of one rank for rows [0, chunk): doubles first (zA, zB, R,
// 1/outdeg, two FP64 partials), then ints (local edge offsets), floats (two
// FP32 partials; with mixed precision the FP32 z pair, F and 1/outdeg), and
// the 16-bit staged indices.
struct CluSmem {
  double *zA, *zB, *Rs, *iv, *dpart;
  int* ip;
  float *part, *fA, *fB, *F, *ivf;
  uint16_t* ix;
};

// z vectors: with push, every rank holds the whole component's z (kClu *
// chunk entries) and writes its rows into every rank's copy; without, a rank
// holds its own slice and reads the others' through the cluster window.
__host__ __device__ __forceinline__ size_t clu_smem(int chunk, bool mixed, bool push) {
  const size_t zlen = push ? (size_t)chunk * kClu : (size_t)chunk;
  return (2 * zlen + 2 * (size_t)chunk + 2) * sizeof(double) + ((size_t)chunk + 2) * sizeof(int) +
         (2 + (mixed ? 2 * zlen + 2 * (size_t)chunk : 0)) * sizeof(float) +
         (size_t)chunk * kCluEdgesPerRow * sizeof(uint16_t);
}

__device__ __forceinline__ CluSmem clu_carve(double* base, int chunk, bool mixed, bool push) {
  const int zlen = push ? chunk * kClu : chunk;
  CluSmem m;
  m.zA = base;
  m.zB = base + zlen;
  m.Rs = base + 2 * zlen;
  m.iv = m.Rs + chunk;
  m.dpart = m.iv + chunk;
  m.ip = reinterpret_cast<int*>(m.dpart + 2);
  m.part = reinterpret_cast<float*>(m.ip + chunk + 2);
  float* f = m.part + 2;
  m.fA = mixed ? f : nullptr;
  m.fB = mixed ? f + zlen : nullptr;
  m.F = mixed ? f + 2 * zlen : nullptr;
  m.ivf = mixed ? f + 2 * zlen + chunk : nullptr;
  m.ix = reinterpret_cast<uint16_t*>(f + (mixed ? 2 * zlen + 2 * chunk : 0));
  return m;
}

// largest component (vertices) a cluster solves in push mode
constexpr int kCluPushMax = 4096;

template <bool kMixed, bool kPush>
__global__ void __cluster_dims__(kClu, 1, 1) __launch_bounds__(kCluThreads)
    solve_clu_k(SolveArgs a, int32_t cbeg, int32_t chunk_max) {
  extern __shared__ double cs[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const CluSmem sm = clu_carve(cs, chunk_max, kMixed, kPush);
  double* zA = sm.zA;
  double* zB = sm.zB;
  double* Rs = sm.Rs;
  double* iv = sm.iv;
  int* ip = sm.ip;
  float* part = sm.part;
  uint16_t* ix = sm.ix;
  __shared__ float red[kCluThreads / 32];
  __shared__ double red64[kCluThreads / 32];
  __shared__ double* remA[kClu];
  __shared__ double* remB[kClu];
  __shared__ double* remD[kClu];
  __shared__ float* remFA[kClu];
  __shared__ float* remFB[kClu];
  // every warp's norm partial of a sweep, gathered in every rank: slot
  // (parity, rank * 8 + warp)
  constexpr int kCluWarps = kCluThreads / 32;
  __shared__ float pw[2 * kClu * kCluWarps];
  __shared__ float* remPW[kClu];
  const int c = cbeg + (int)(blockIdx.x / kClu);
  const int off = a.c_off[c], sz = a.c_off[c + 1] - off;
  const int sh = clu_shift(sz);
  const int chunk = 1 << sh;
  const int r0 = rank * chunk;
  const int nr = max(0, min(sz, r0 + chunk) - r0);
  if (threadIdx.x < kClu) {
    // this rank's own buffers by their plain shared-memory address
    const int t = (int)threadIdx.x;
    const bool own = t == rank;
    remA[t] = own ? zA : cl.map_shared_rank(zA, t);
    remB[t] = own ? zB : cl.map_shared_rank(zB, t);
    remD[t] = own ? sm.dpart : cl.map_shared_rank(sm.dpart, t);
    remPW[t] = own ? pw : cl.map_shared_rank(pw, t);
    if (kMixed) {
      remFA[t] = own ? sm.fA : cl.map_shared_rank(sm.fA, t);
      remFB[t] = own ? sm.fB : cl.map_shared_rank(sm.fB, t);
    }
  }
  __syncthreads();
  // with push the staging below already writes other ranks' shared memory:
  // every block of the cluster must be running first
  if (kPush) cl.sync();
  // The norm of a sweep: each warp reduces its rows' terms and stores the
  // result into every rank's pw; after the cluster barrier every thread
  // folds the same kClu * 8 values in the same order.
  auto norm_put = [&](float local, int parity, bool is_max) {
    const float w = is_max ? group_maxf<32>(local) : group_sumf<32>(local);
    if ((threadIdx.x & 31) == 0) {
      const int slot = parity * kClu * kCluWarps + rank * kCluWarps + (int)(threadIdx.x >> 5);
#pragma unroll
      for (int rk = 0; rk < kClu; rk++) remPW[rk][slot] = w;
    }
  };
  auto norm_get = [&](int parity, bool is_max) {
    float s = 0.0f;
    const float* b = pw + parity * kClu * kCluWarps;
#pragma unroll 8
    for (int j = 0; j < kClu * kCluWarps; j++) s = is_max ? fmaxf(s, b[j]) : s + b[j];
    return s;
  };
  // z of this rank's row i into buffer X: every rank's copy (push) or the
  // own slice (pull)
  auto zput = [&](auto* const* remX, int i, auto v) {
    if (kPush) {
#pragma unroll
      for (int rk = 0; rk < kClu; rk++) remX[rk][r0 + i] = v;
    } else {
      remX[rank][i] = v;
    }
  };
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
    zput(remA, i, W * inv);
  }
  cl.sync();
  const int mask = chunk - 1;
  // z of component-local vertex q: from this rank's full copy (push) or
  // from the owner rank's slice (pull)
  auto zat = [&](auto const* rem, int q) {
    if (kPush) return rem[rank][q];
    return rem[q >> sh][q & mask];
  };
  // sum of z over row i's in-edges
  auto row_sum = [&](auto const* rem, int i) {
    using T = typename std::remove_pointer<typename std::remove_const<
        typename std::remove_pointer<decltype(rem)>::type>::type>::type;
    // four independent partial sums: four loads in flight at once
    T acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
    const int e0 = ip[i], e1 = ip[i + 1];
    int e = e0;
    if (staged) {
      for (; e + 3 < e1; e += 4) {
        acc0 += zat(rem, ix[e]);
        acc1 += zat(rem, ix[e + 1]);
        acc2 += zat(rem, ix[e + 2]);
        acc3 += zat(rem, ix[e + 3]);
      }
      for (; e < e1; e++) acc0 += zat(rem, ix[e]);
    } else {
      for (; e < e1; e++) acc0 += zat(rem, local_or_err(a, a.int_idx[ib + e] - off, sz));
    }
    return (acc0 + acc1) + (acc2 + acc3);
  };
  int k = 0, k64 = 0;
  if (a.c_type[c] != PR_TYPE_SCC) {
    // CAC: one pass, sub-level by sub-level, one cluster barrier each
    const int sb = a.c_sub[c], se = a.c_sub[c + 1];
    for (int s2 = sb; s2 < se; s2++) {
      const int lo = max(a.sub_ptr[s2] - off - r0, 0), hi = min(a.sub_ptr[s2 + 1] - off - r0, nr);
      for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double Rv = Rs[i] + a.c * row_sum(remA, i);
        Rs[i] = Rv;
        zput(remA, i, Rv * iv[i]);
      }
      cl.sync();
    }
  } else if (kMixed) {
    // FP32 series with FP64 residual refinement (see kMixKappa).  F holds
    // the FP32 sum of the current pass, Rs the FP64 result so far.
    const double tau = a.tol * (double)sz / (double)a.n;
    const float cf = (float)a.c;
    float* F = sm.F;
    float* ivf = sm.ivf;
    double wl = 0.0;
    const bool warm = a.R0 != nullptr;  // start from the guess's residual
    for (int i = threadIdx.x; i < nr; i += blockDim.x) {
      const double W = Rs[i];
      F[i] = warm ? 0.0f : (float)W;
      zput(remFA, i, (float)(W * iv[i]));
      ivf[i] = (float)iv[i];
      Rs[i] = warm ? a.R0[off + r0 + i] : 0.0;
      wl += W;
    }
    const double wb = block_sum(wl, red64);
    if (threadIdx.x == 0) sm.dpart[0] = wb;
    cl.sync();  // publishes fA and the partials
    double wsum = 0.0;
    for (int r = 0; r < kClu; r++) wsum += remD[r][0];
    float thr = (float)fmax(tau, (double)kMixKappa * wsum);
    int zc = 0, dq = 1, rounds = 0;
    bool skip = warm;
    for (;;) {
      bool stop = false;
      for (; !skip;) {
        float* const* rem = zc ? remFB : remFA;
        float* const* nxt = zc ? remFA : remFB;
        float local = 0.0f;
        for (int i = threadIdx.x; i < nr; i += blockDim.x) {
          const float pn = cf * row_sum(rem, i);
          F[i] += pn;
          zput(nxt, i, pn * ivf[i]);
          local += fabsf(pn);
        }
        norm_put(local, k & 1, false);
        cl.sync();  // publishes nxt and the partials
        const float s2 = norm_get(k & 1, false);
        k++;
        zc ^= 1;
        if (s2 <= thr) break;
        if (k >= a.max_iter) {
          if (rank == 0 && threadIdx.x == 0) atomicOr(&a.ctl->flags[0], 1);
          stop = true;
          break;
        }
      }
      skip = false;
      for (int i = threadIdx.x; i < nr; i += blockDim.x) {
        const double R = Rs[i] + (double)F[i];
        Rs[i] = R;
        zput(remA, i, R * iv[i]);
      }
      if (stop) break;
      cl.sync();  // publishes zA
      // FP64 residual; r becomes the start of the next correction pass
      float* const* cur = zc ? remFB : remFA;
      double rl = 0.0;
      for (int i = threadIdx.x; i < nr; i += blockDim.x) {
        const double r = a.W[off + r0 + i] + a.c * row_sum(remA, i) - Rs[i];
        F[i] = (float)r;
        zput(cur, i, (float)(r * iv[i]));
        rl += fabs(r);
      }
      const double rb = block_sum(rl, red64);
      if (threadIdx.x == 0) sm.dpart[dq] = rb;
      cl.sync();  // publishes cur and the partials
      double rho = 0.0;
      for (int r = 0; r < kClu; r++) rho += remD[r][dq];
      dq ^= 1;
      k++;
      k64++;
      if (rho <= tau) break;
      if (++rounds >= kMixRounds || k >= a.max_iter) {
        if (rank == 0 && threadIdx.x == 0) atomicOr(&a.ctl->flags[0], 1);
        break;
      }
      thr = fmaxf(0.5f * (float)tau, kMixKappa * (float)rho);
    }
  } else {
    const double tau = a.norm == PR_NORM_L1 ? a.tol * (double)sz / (double)a.n : a.tol;
    const float thr = stop_thr32(tau);
    const int fixed = a.replay ? a.replay[c] : -1;
    const bool is_max = a.norm != PR_NORM_L1;
    // iv holds c / outdeg during the series (z = c P / outdeg: the in-edge
    // sum is the next term itself); 1/outdeg is restored for the result
    for (int i = threadIdx.x; i < nr; i += blockDim.x) iv[i] *= a.c;
    if (a.R0) {
      // warm start: R = R0 + r; the series continues from r (in zB, k = 1)
      for (int i = threadIdx.x; i < nr; i += blockDim.x) zput(remA, i, a.R0[off + r0 + i] * iv[i]);
      cl.sync();
      for (int i = threadIdx.x; i < nr; i += blockDim.x) {
        const double g0 = a.R0[off + r0 + i];
        const double r = Rs[i] + row_sum(remA, i) - g0;
        Rs[i] = g0 + r;
        zput(remB, i, r * iv[i]);
      }
      k = 1;
    } else {
      for (int i = threadIdx.x; i < nr; i += blockDim.x) zput(remA, i, Rs[i] * iv[i]);  // Rs holds W
    }
    cl.sync();
    for (;;) {
      double* const* rem = (k & 1) ? remB : remA;
      double* const* nxt = (k & 1) ? remA : remB;
      float local = 0.0f;
      for (int i = threadIdx.x; i < nr; i += blockDim.x) {
        const double pn = row_sum(rem, i);
        Rs[i] += pn;
        zput(nxt, i, pn * iv[i]);
        const float pf = abs_to_float(pn);
        local = is_max ? fmaxf(local, pf) : local + pf;
      }
      norm_put(local, k & 1, is_max);
      cl.sync();  // publishes nxt and the partials
      const float s2 = norm_get(k & 1, is_max);
      k++;
      if (fixed >= 0) {
        if (k >= fixed) break;
        continue;
      }
      if (!keep_going32(s2, thr, a.norm)) break;
      if (k >= a.max_iter) {
        if (rank == 0 && threadIdx.x == 0) atomicOr(&a.ctl->flags[0], 1);
        break;
      }
    }
    for (int i = threadIdx.x; i < nr; i += blockDim.x) iv[i] = a.p_inv[off + r0 + i];
  }
  for (int i = threadIdx.x; i < nr; i += blockDim.x) {
    a.R[off + r0 + i] = Rs[i];
    a.zr[off + r0 + i] = Rs[i] * iv[i];
  }
  if (rank == 0 && threadIdx.x == 0) {
    a.iters[c] = k;
    if (kMixed && a.c_type[c] == PR_TYPE_SCC) a.iters64[c] = k64;
  }
  cl.sync();  // no rank leaves while another may still read its shared memory
}

// ---------------------------------------------------------------------------
// Sec. 4.3 item 3: an SCC of fewer than lu_threshold (<= kLuMax + 1)
// vertices is solved directly, (I - c A_C^T) R_C = W_C, by Gaussian
// elimination in shared memory, one CTA per component.  The matrix is
// column diagonally dominant (each column's off-diagonal entries sum to
// c * internal outdeg / outdeg <= c < 1) and stays so under elimination, so
// no pivoting is needed and every pivot is at least 1 - c.
// ---------------------------------------------------------------------------
constexpr int kLuMax = 128;
constexpr int kLuThreads = 256;
constexpr size_t kLuSmem = ((size_t)kLuMax * kLuMax + 3 * kLuMax) * sizeof(double);

__global__ void __launch_bounds__(kLuThreads) solve_lu_k(SolveArgs a, int32_t cbeg) {
  extern __shared__ double lm[];
  const int c = cbeg + (int)blockIdx.x;
  const int off = a.c_off[c], sz = a.c_off[c + 1] - off;
  if (a.c_type[c] != PR_TYPE_SCC || sz >= a.lu_threshold || sz > kLuMax) return;  // block-uniform
  double* M = lm;                      // [sz][sz], row i = equation of vertex i
  double* b = lm + kLuMax * kLuMax;    // [sz] right-hand side, then the solution
  double* l = b + kLuMax;              // [sz] multipliers of one step
  double* iv = l + kLuMax;             // [sz] 1/outdeg
  for (int t = threadIdx.x; t < sz * sz; t += blockDim.x) M[t] = (t / sz == t % sz) ? 1.0 : 0.0;
  for (int i = threadIdx.x; i < sz; i += blockDim.x) {
    b[i] = a.W[off + i];
    iv[i] = a.p_inv[off + i];
  }
  __syncthreads();
  // row i: -c / outdeg(j) for each internal edge j -> i
  for (int i = threadIdx.x; i < sz; i += blockDim.x)
    for (int e = a.int_ptr[off + i]; e < a.int_ptr[off + i + 1]; e++) {
      const int j = local_or_err(a, a.int_idx[e] - off, sz);
      M[i * sz + j] -= a.c * a.p_inv[off + j];
    }
  __syncthreads();
  for (int k = 0; k + 1 < sz; k++) {
    const double ip = 1.0 / M[k * sz + k];
    for (int i = k + 1 + threadIdx.x; i < sz; i += blockDim.x) l[i] = M[i * sz + k] * ip;
    __syncthreads();
    const int w = sz - k - 1;  // rows k+1.., columns k+1..
    for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
      const int i = k + 1 + t / w, j = k + 1 + t % w;
      M[i * sz + j] -= l[i] * M[k * sz + j];
    }
    for (int i = k + 1 + threadIdx.x; i < sz; i += blockDim.x) b[i] -= l[i] * b[k];
    __syncthreads();
  }
  // back substitution, column by column
  for (int i = sz - 1; i >= 0; i--) {
    if (threadIdx.x == 0) b[i] = b[i] / M[i * sz + i];
    __syncthreads();
    for (int r = threadIdx.x; r < i; r += blockDim.x) b[r] -= M[r * sz + i] * b[i];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < sz; i += blockDim.x) {
    a.R[off + i] = b[i];
    a.zr[off + i] = b[i] * iv[i];
  }
  if (threadIdx.x == 0) a.iters[c] = 0;
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

// R[p] = W[p], and z0[p - off] = W * scale[p] when z0 is given, for the
// rows of a component
__device__ __forceinline__ void load_rows(const SolveArgs& a, int off, int sz, double* z0, const double* scale) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sz; i += (int64_t)gridDim.x * blockDim.x) {
    const int p = off + (int)i;
    const double W = a.W[p];
    a.R[p] = W;
    if (z0) z0[i] = W * scale[p];
  }
}

__global__ void __launch_bounds__(kBlock) solve_large_cac_k(SolveArgs a, LargeComp L) {
  load_rows(a, L.off, L.size, nullptr, nullptr);  // R[p] = W
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
                              const int32_t* ext_ptr, const int32_t* iters, const int32_t* iters64,
                              unsigned long long* out) {
  unsigned long long loc = 0, loc64 = 0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < K; c += (int64_t)gridDim.x * blockDim.x) {
    const int b = c_off[c], e = c_off[c + 1];
    const long long mi = int_ptr[e] - int_ptr[b], me = ext_ptr[e] - ext_ptr[b];
    const bool scc = c_type[c] == PR_TYPE_SCC;
    loc += (unsigned long long)(me + (scc ? mi * (long long)iters[c] : mi));
    if (iters64 && scc) loc64 += (unsigned long long)(mi * (long long)iters64[c]);
  }
  atomicAdd(out, loc);
  if (iters64) atomicAdd(out + 1, loc64);
}

}  // namespace prgb

namespace prgb {

static unsigned grid_cap(int64_t blocks) {
  int64_t cap = (int64_t)num_sms() * 32;
  return (unsigned)(blocks < 1 ? 1 : (blocks > cap ? cap : blocks));
}

__global__ void scale_k(int32_t n, double c, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = c * x[i];
}

// Process-wide pools of non-blocking streams and timing-free events, per
// device: a partition's first solve and every replayed-count solve would
// otherwise create (and later destroy) about ten of each.  Never freed (it
// must outlive the handles' last use at process exit).
namespace {
struct HandlePool {
  std::mutex mu;
  std::vector<cudaStream_t> streams[64];
  std::vector<cudaEvent_t> events[64];
};
HandlePool& handle_pool() {
  static HandlePool* p = new HandlePool;
  return *p;
}
int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d >= 0 && d < 64 ? d : 0;
}
}  // namespace

cudaError_t pool_stream(int dev, cudaStream_t* out) {
  HandlePool& p = handle_pool();
  {
    std::lock_guard<std::mutex> lock(p.mu);
    if (!p.streams[dev].empty()) {
      *out = p.streams[dev].back();
      p.streams[dev].pop_back();
      return cudaSuccess;
    }
  }
  return cudaStreamCreateWithFlags(out, cudaStreamNonBlocking);
}
cudaError_t pool_event(int dev, cudaEvent_t* out) {
  HandlePool& p = handle_pool();
  {
    std::lock_guard<std::mutex> lock(p.mu);
    if (!p.events[dev].empty()) {
      *out = p.events[dev].back();
      p.events[dev].pop_back();
      return cudaSuccess;
    }
  }
  return cudaEventCreateWithFlags(out, cudaEventDisableTiming);
}
void pool_release(int dev, cudaStream_t st, cudaEvent_t ev) {
  HandlePool& p = handle_pool();
  std::lock_guard<std::mutex> lock(p.mu);
  if (st) p.streams[dev].push_back(st);
  if (ev) p.events[dev].push_back(ev);
}

pr_status SideStreams::create() {
  dev = current_device();
  for (int q = 0; q < kSideStreams; q++) {
    PRGB_CUDA(pool_stream(dev, &st[q]));
    PRGB_CUDA(pool_event(dev, &join[q]));
  }
  PRGB_CUDA(pool_event(dev, &fork));
  return PR_OK;
}

SideStreams::~SideStreams() {
  for (int q = 0; q < kSideStreams; q++) pool_release(dev, st[q], join[q]);
  pool_release(dev, nullptr, fork);
}

pr_status KernelTiming::ensure(const pr_partition_s* P) {
  size_t k = 0;
  for (const LargeComp& L : P->large) k += L.type == PR_TYPE_SCC;
  comps.clear();
  for (const LargeComp& L : P->large)
    if (L.type == PR_TYPE_SCC) comps.push_back(L);
  while (start.size() < k) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PRGB_CUDA(cudaEventCreate(&e0));
    start.push_back(e0);
    PRGB_CUDA(cudaEventCreate(&e1));
    stop.push_back(e1);
  }
  while (levels && level.size() < P->levels.size() + 1) {
    cudaEvent_t e = nullptr;
    PRGB_CUDA(cudaEventCreate(&e));
    level.push_back(e);
  }
  return PR_OK;
}

KernelTiming::~KernelTiming() {
  for (cudaEvent_t e : start) cudaEventDestroy(e);
  for (cudaEvent_t e : stop) cudaEventDestroy(e);
  for (cudaEvent_t e : level) cudaEventDestroy(e);
}

pr_status set_solve_attrs(const pr_partition_s* P, bool mixed);

// Work buffers of a solve (all by permuted position), allocated from `a`;
// also sets the kernels' shared-memory limits for this partition, so that
// nothing but launches and memsets is left for the level loop.
pr_status alloc_solve_bufs(const pr_partition_s* P, bool mixed, Arena& a, SolveBufs* b, int64_t* nl) {
  cudaStream_t s = a.stream();
  const int32_t n = P->g.n;
  PRGB_TRY(a.alloc(&b->R, n));
  PRGB_TRY(a.alloc(&b->zr, n));
  PRGB_TRY(a.alloc(&b->W, n));
  PRGB_TRY(a.alloc(&b->lvl_ctr, 4 * P->levels.size() + 4));
  // shared by the level gathers and the grid-wide series (left zeroed after each)
  PRGB_TRY(alloc_heavy_scratch(&b->hs, std::max(P->max_heavy, P->max_xheavy), std::max(P->max_chunks, P->max_xchunks),
                               a));
  if (P->max_large > 0) {
    PRGB_TRY(a.alloc(&b->civ, (size_t)n + 1));
    {
      // one z slot more: the zero that padded SELL entries read
      GiantFxBufs& g = b->gfx;
      PRGB_TRY(a.alloc(&g.zA, (size_t)P->max_large + 1));
      PRGB_TRY(a.alloc(&g.zB, (size_t)P->max_large + 1));
      PRGB_TRY(a.alloc(&g.R, (size_t)P->max_large + 1));
      PRGB_TRY(a.alloc(&g.part, (size_t)P->max_chunks + 1));
      PRGB_TRY(a.alloc(&g.cnt, (size_t)P->max_heavy + 1));
      PRGB_TRY(a.alloc(&g.acc, 4));
      PRGB_CUDA(cudaMemsetAsync(g.cnt, 0, ((size_t)P->max_heavy + 1) * 4, s));
    }
  }
  return set_solve_attrs(P, mixed);
}

// dynamic shared memory limits of the solve kernels for this partition's
// largest cluster-class component (raised, never lowered)
pr_status set_solve_attrs(const pr_partition_s* P, bool mixed) {
  static bool cta_attr = false;
  static size_t clu_attr[4] = {48 * 1024, 48 * 1024, 48 * 1024, 48 * 1024};
  if (!cta_attr) {
    PRGB_TRY(set_fx_attrs());
    PRGB_CUDA(cudaFuncSetAttribute(solve_lu_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLuSmem));
    cta_attr = true;
  }
  // the largest cluster-class component of any level, with and without push
  int clu_max = 0, push_max = 0;
  for (const LevelRange& r : P->levels) {
    const int m = r.cta > r.clu ? r.clu_max : 0;
    clu_max = std::max(clu_max, m);
    if (m <= kCluPushMax) push_max = std::max(push_max, m);
  }
  for (int push = 0; push < 2; push++) {
    const int m = push ? push_max : clu_max;
    const size_t smem = clu_smem(1 << clu_shift(m), mixed, push != 0);
    const int slot = (mixed ? 2 : 0) + push;
    if (m > 0 && smem > clu_attr[slot]) {
      const void* f = mixed ? (push ? (const void*)solve_clu_k<true, true> : (const void*)solve_clu_k<true, false>)
                            : (push ? (const void*)solve_clu_k<false, true> : (const void*)solve_clu_k<false, false>);
      PRGB_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      clu_attr[slot] = smem;
    }
  }
  return PR_OK;
}

SolveArgs make_solve_args(const pr_partition_s* P, double c, const double* u, double tol, int norm, int max_iter,
                          const int32_t* replay, const SolveBufs& b, int32_t* iters, int32_t* iters64, Ctl* ctl) {
  SolveArgs a;
  a.n = P->g.n;
  a.c = c;
  a.tol = tol;
  a.norm = norm;
  a.max_iter = max_iter;
  a.u = u;
  a.perm = P->perm;
  a.p_outdeg = P->p_outdeg;
  a.p_inv = P->p_inv;
  a.lorder = P->lorder;
  a.lpre = P->balance ? P->lpre : nullptr;
  a.int_ptr = P->int_ptr;
  a.int_idx = P->int_idx;
  a.ext_ptr = P->ext_ptr;
  a.ext_idx = P->ext_idx;
  a.c_off = P->c_off;
  a.c_sub = P->c_sub;
  a.sub_ptr = P->sub_ptr;
  a.c_type = P->c_type;
  a.replay = replay;
  a.xlorder = P->xlorder;
  a.civ = b.civ;
  a.sell_ptr = P->sell_ptr;
  a.sell_idx = P->sell_idx;
  a.sell_cpre = P->sell_cpre;
  a.fxs_ptr = P->fxs_ptr;
  a.fxs_wbase = P->fxs_wbase;
  a.fxs_wcnt = P->fxs_wcnt;
  a.fxs_words = P->fxs_words;
  a.R0 = nullptr;
  a.yhat = nullptr;
  a.lu_threshold = 0;
  a.iters64 = iters64;
  a.W = b.W;
  a.R = b.R;
  a.zr = b.zr;
  a.iters = iters;
  a.ctl = ctl;
  return a;
}

// The level loop (Sec. 4.3): per level, the inflow gather and 1-vertex
// components on s, the grid-wide components on s, then the cluster, CTA and
// warp classes on the three side streams, joined back into s before the
// next level.  Only launches, memsets and event records: it can be
// captured into a CUDA graph.
bool giant_fits_l2(const LargeComp& L) { return (int64_t)L.size * kGiantFxRowBytes <= l2_bytes() / 2; }

// A timing event: inside a stream capture an external record, which becomes
// an event-record node so that the event times each replay; a plain record
// otherwise.
static cudaError_t record_timing(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t q = cudaStreamIsCapturing(s, &cs);
  if (q != cudaSuccess) return q;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                             : cudaEventRecord(e, s);
}

pr_status enqueue_levels(const pr_partition_s* P, SolveArgs a, const SolveBufs& b, bool mixed, SideStreams& side,
                         cudaStream_t s, KernelTiming* timing, int64_t* nl, const float* yhat = nullptr) {
  Ctl* ctl = a.ctl;
  HeavyScratch hs = b.hs;
  size_t li_large = 0, ti = 0;
  PRGB_CUDA(cudaMemsetAsync(b.lvl_ctr, 0, (4 * P->levels.size() + 4) * sizeof(int32_t), s));
  if (b.civ && P->g.n > 0) {
    // c / outdeg for the grid-wide series of this solve's c
    scale_k<<<grid_cap((P->g.n + kBlock - 1) / kBlock), kBlock, 0, s>>>(P->g.n, a.c, P->p_inv, b.civ);
    PRGB_LAUNCH();
    ++*nl;
  }
  for (size_t li = 0; li < P->levels.size(); li++) {
    const LevelRange& r = P->levels[li];
    NvtxRange nvtx_level("prgb level", (int)li);
    // external records: inside a captured graph they become event-record
    // nodes, so the events time each replay
    if (timing && timing->levels) PRGB_CUDA(record_timing(timing->level[li], s));
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
      ++*nl;
    }
    // learned warm start: the guess R0 of the level's SCCs that the level
    // kernel does not take (all of them in mixed precision), from the
    // weights W the gather has just formed; the level kernel forms its own
    if (yhat && a.R0) {
      PRGB_TRY(mpnn_level_r0(P, r.cbeg, r.big, a.W, yhat, const_cast<double*>(a.R0), s, nl));
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
        // external records: inside a captured graph they become event-record
        // nodes, so the events time each replay
        if (timing) PRGB_CUDA(record_timing(timing->start[ti], s));
        // the exact fixed-point series in both precision modes: on GB300 it
        // beat the FP32 series with FP64 refinement at every size measured
        // (web_like's 400k-vertex giant 1.9 against 3.0 ms, the 50M graph's
        // 25M-vertex one 243 against 261 ms per solve)
        GiantFxBufs gfx = b.gfx;
        void* argsfx[] = {&a, &L, &gfx, &hv};
        PRGB_CUDA(cudaMemsetAsync(gfx.acc, 0, 4 * sizeof(unsigned long long), s));
        const void* kfx = giant_fits_l2(L) ? (const void*)solve_large_scc_fx_k : (const void*)solve_large_scc_fxd_k;
        PRGB_TRY(launch_coop(kfx, kBlock, 0, s, argsfx, P->coop_blocks, nullptr));
        if (timing) PRGB_CUDA(record_timing(timing->stop[ti], s));
        ti++;
      } else {
        void* args[] = {&a, &L};
        PRGB_TRY(launch_coop((const void*)solve_large_cac_k, kBlock, 0, s, args, P->coop_blocks, nullptr));
      }
      ++*nl;
    }
    PRGB_CUDA(cudaEventRecord(side.fork, s));
    bool joined[kSideStreams] = {false, false, false, false};
    // the cluster class keeps the components above kFxMax vertices; the
    // smaller ones go to the level kernel below
    const int32_t clu_end = r.big;
    if (clu_end > r.clu) {
      PRGB_CUDA(cudaStreamWaitEvent(side.st[0], side.fork, 0));
      joined[0] = true;
      const int chunk = 1 << clu_shift(r.clu_max);
      const bool push = r.clu_max <= kCluPushMax;
      const size_t smem = clu_smem(chunk, mixed, push);
      const unsigned nb = (unsigned)(clu_end - r.clu) * kClu;
      if (mixed && push) solve_clu_k<true, true><<<nb, kCluThreads, smem, side.st[0]>>>(a, r.clu, chunk);
      else if (mixed) solve_clu_k<true, false><<<nb, kCluThreads, smem, side.st[0]>>>(a, r.clu, chunk);
      else if (push) solve_clu_k<false, true><<<nb, kCluThreads, smem, side.st[0]>>>(a, r.clu, chunk);
      else solve_clu_k<false, false><<<nb, kCluThreads, smem, side.st[0]>>>(a, r.clu, chunk);
      PRGB_LAUNCH();
      ++*nl;
    }
    if (a.lu_threshold > 0) {
      // the level's components below the threshold form a suffix of
      // [cbeg, single) (sizes descend); the kernel skips the CACs among them
      int lo = std::max(r.cta, r.cbeg), hi = r.single;
      while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (P->h_c_off[mid + 1] - P->h_c_off[mid] < a.lu_threshold) hi = mid;
        else lo = mid + 1;
      }
      if (r.single > lo) {
        if (!joined[1]) PRGB_CUDA(cudaStreamWaitEvent(side.st[1], side.fork, 0));
        joined[1] = true;
        solve_lu_k<<<r.single - lo, kLuThreads, kLuSmem, side.st[1]>>>(a, lo);
        PRGB_LAUNCH();
        ++*nl;
      }
    }
    if (r.single > r.big) {
      // every component of at most kFxMax vertices: one persistent launch
      PRGB_TRY(launch_level(a, r, b.lvl_ctr + 4 * li, s));
      ++*nl;
    }
    for (int q = 0; q < kSideStreams; q++) {
      if (!joined[q]) continue;
      PRGB_CUDA(cudaEventRecord(side.join[q], side.st[q]));
      PRGB_CUDA(cudaStreamWaitEvent(s, side.join[q], 0));
    }
  }
  if (timing && timing->levels && !P->levels.empty())
    PRGB_CUDA(record_timing(timing->level[P->levels.size()], s));
  return PR_OK;
}

pr_status scatter_out(const pr_partition_s* P, const double* Rp, double* R, cudaStream_t s, int64_t* nl) {
  const int32_t n = P->g.n;
  if (n == 0) return PR_OK;
  scatter_out_k<<<grid_cap((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, P->perm, Rp, R);
  PRGB_LAUNCH();
  ++*nl;
  return PR_OK;
}

pr_status run_solve(const pr_partition_s* P, double c, const double* u, double tol, int norm, int max_iter,
                    const int32_t* replay, bool mixed, int lu_threshold, double* R, int32_t* iters_dev,
                    int32_t* iters64_dev, Arena& tmp, Ctl* ctl, int64_t* launches, KernelTiming* timing) {
  cudaStream_t s = tmp.stream();
  int64_t nl = 0;
  *launches = 0;
  if (P->g.n == 0) return PR_OK;
  SolveBufs b;
  PRGB_TRY(alloc_solve_bufs(P, mixed, tmp, &b, &nl));
  SolveArgs a = make_solve_args(P, c, u, tol, norm, max_iter, replay, b, iters_dev, iters64_dev, ctl);
  a.lu_threshold = lu_threshold;
  SideStreams side;
  PRGB_TRY(side.create());
  if (timing) PRGB_TRY(timing->ensure(P));
  PRGB_TRY(enqueue_levels(P, a, b, mixed, side, s, timing, &nl));
  PRGB_TRY(scatter_out(P, b.R, R, s, &nl));
  *launches = nl;
  return PR_OK;
}

// ---------------------------------------------------------------------------
// per-partition CUDA graph of the level loop
// ---------------------------------------------------------------------------
SolvePlan::~SolvePlan() {
  for (PlanGraph& e : graphs) {
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.graph) cudaGraphDestroy(e.graph);
  }
  pool_release(dev, cs, done);
  delete keep;
}

// The cached graph for these parameters, or null.  The graphs of the last
// kPlanGraphs parameter sets are kept (a caller alternating, say, FP64 and
// mixed solves does not re-capture each time).
static PlanGraph* plan_find(SolvePlan* pl, double c, double tol, int norm, int max_iter, bool mixed, int timing,
                            const pr_mpnn_s* warm, int lu) {
  for (PlanGraph& e : pl->graphs)
    if (e.c == c && e.tol == tol && e.norm == norm && e.max_iter == max_iter && e.mixed == mixed &&
        e.timing == timing && e.warm_uid == (warm ? warm->uid : 0) && e.lu == lu && e.wait_us == wait_limit_us()) {
      e.last_use = ++pl->uses;
      return &e;
    }
  return nullptr;
}

// The plan's buffers and streams, allocated on first use (and the mixed,
// warm-start and timing extras when first asked for).
static pr_status plan_setup(pr_partition_s* P, SolvePlan* pl, bool mixed, int timing, const pr_mpnn_s* warm) {
  const int32_t n = P->g.n;
  const int32_t K = P->n_comp;
  if (!pl->keep) {
    pl->keep = new (std::nothrow) Arena(P->stream);
    if (!pl->keep) return PR_ENOMEM;
    pl->dev = current_device();
    PRGB_CUDA(pool_stream(pl->dev, &pl->cs));
    PRGB_CUDA(pool_event(pl->dev, &pl->done));
    PRGB_TRY(pl->side.create());
    PRGB_TRY(pl->cap_side.create());
    PRGB_TRY(pl->keep->alloc(&pl->ctl, 1));
    PRGB_TRY(pl->keep->alloc(&pl->iters, (size_t)K + 1));
    PRGB_TRY(pl->keep->alloc(&pl->iters64, (size_t)K + 1));
    PRGB_TRY(pl->keep->alloc(&pl->u, (size_t)n + 1));
    PRGB_TRY(pl->keep->alloc(&pl->Rout, (size_t)n + 1));
    int64_t nl = 0;
    PRGB_TRY(alloc_solve_bufs(P, false, *pl->keep, &pl->b, &nl));
    PRGB_CUDA(cudaStreamSynchronize(P->stream));
  }
  if (warm) PRGB_TRY(mpnn_prepare());
  if (warm && !pl->R0) {
    // the guess by position, the network's output and its activations
    PRGB_TRY(pl->keep->alloc(&pl->R0, (size_t)n + 1));
    PRGB_TRY(pl->keep->alloc(&pl->yhat, (size_t)n + 1));
    PRGB_TRY(pl->keep->alloc(&pl->inf.X, (size_t)n * kMpF0 + 4));
    PRGB_TRY(pl->keep->alloc(&pl->inf.H1, (size_t)n * kMpH + 4));
    PRGB_TRY(pl->keep->alloc(&pl->inf.dout, (size_t)n + 1));
    pl->yhat_uid = 0;
  }
  pl->kt.levels = timing >= 2;
  if (timing) PRGB_TRY(pl->kt.ensure(P));
  return set_solve_attrs(P, mixed);
}

static SolveArgs plan_args(pr_partition_s* P, SolvePlan* pl, double c, double tol, int norm, int max_iter,
                           bool mixed, const pr_mpnn_s* warm, int lu) {
  SolveArgs a = make_solve_args(P, c, pl->u, tol, norm, max_iter, nullptr, pl->b, pl->iters,
                                mixed ? pl->iters64 : nullptr, pl->ctl);
  if (warm) {
    a.R0 = pl->R0;
    a.yhat = pl->yhat;
  }
  a.lu_threshold = lu;
  return a;
}

// The start of every solve of the plan: its control word and counters.
static pr_status plan_head(SolvePlan* pl, int32_t K, cudaStream_t s, int64_t* nl) {
  PRGB_TRY(init_ctl(pl->ctl, s));
  PRGB_CUDA(cudaMemsetAsync(pl->iters, 0, ((size_t)K + 1) * 4, s));
  PRGB_CUDA(cudaMemsetAsync(pl->iters64, 0, ((size_t)K + 1) * 4, s));
  if (wait_limit_us()) ++*nl;  // the kernel that sets the wait limit
  return PR_OK;
}

// Capture the level loop for these parameters into a CUDA graph (on the
// plan's own capture stream and side streams, so that it can run while the
// device still executes work the call enqueued on the others) and cache it,
// evicting the least recently used graph beyond kPlanGraphs.
static pr_status plan_capture(pr_partition_s* P, SolvePlan* pl, double c, double tol, int norm, int max_iter,
                              bool mixed, int timing, const pr_mpnn_s* warm, int lu) {
  if (pl->graphs.size() >= (size_t)kPlanGraphs) {
    size_t old = 0;
    for (size_t i = 1; i < pl->graphs.size(); i++)
      if (pl->graphs[i].last_use < pl->graphs[old].last_use) old = i;
    if (pl->graphs[old].exec) cudaGraphExecDestroy(pl->graphs[old].exec);
    if (pl->graphs[old].graph) cudaGraphDestroy(pl->graphs[old].graph);
    pl->graphs.erase(pl->graphs.begin() + old);
  }
  const SolveArgs a = plan_args(P, pl, c, tol, norm, max_iter, mixed, warm, lu);
  const long long before = launch_count();
  int64_t nl = 0;
  PRGB_CUDA(cudaStreamBeginCapture(pl->cs, cudaStreamCaptureModeThreadLocal));
  pr_status st = plan_head(pl, P->n_comp, pl->cs, &nl);
  if (st == PR_OK)
    st = enqueue_levels(P, a, pl->b, mixed, pl->cap_side, pl->cs, timing ? &pl->kt : nullptr, &nl,
                        warm ? pl->yhat : nullptr);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(pl->cs, &g);
  add_launches(before - launch_count());  // captured, not launched
  if (st != PR_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  PRGB_CUDA(ec);
  PlanGraph e;
  e.graph = g;
  if (cudaGraphInstantiate(&e.exec, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    PRGB_CUDA(cudaGetLastError());
    return PR_ECUDA;
  }
  e.nodes = nl;
  e.c = c;
  e.tol = tol;
  e.norm = norm;
  e.max_iter = max_iter;
  e.mixed = mixed;
  e.timing = timing;
  e.warm_uid = warm ? warm->uid : 0;
  e.lu = lu;
  e.wait_us = wait_limit_us();
  e.last_use = ++pl->uses;
  pl->graphs.push_back(e);
  return PR_OK;
}

pr_status plan_solve(pr_partition_s* P, double c, const double* u, bool u_on_host, double tol, int norm,
                     int max_iter, bool mixed, int timing, const pr_mpnn_s* warm, int lu, double* R,
                     bool R_on_host, cudaStream_t s, SolvePlan** out, int64_t* launches) {
  if (!P->plan) {
    P->plan = new (std::nothrow) SolvePlan;
    if (!P->plan) return PR_ENOMEM;
  }
  SolvePlan* pl = P->plan;
  *out = pl;
  const int32_t n = P->g.n;
  PRGB_TRY(plan_setup(P, pl, mixed, timing, warm));
  PlanGraph* ge = plan_find(pl, c, tol, norm, max_iter, mixed, timing, warm, lu);
  // the plan's buffers are reused: order this call after the previous one
  PRGB_CUDA(cudaStreamWaitEvent(s, pl->done, 0));
  if (n > 0)
    PRGB_COPY(cudaMemcpyAsync(pl->u, u, (size_t)n * 8, u_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                              s));
  int64_t nl = 0;
  if (warm && (pl->yhat_uid != warm->uid || pl->yhat_ver != warm->version)) {
    // the network's output depends on the graph and the weights only: once
    // per partition and model version, before the level loop
    const long long before = launch_count();
    PRGB_TRY(mpnn_guess(warm, P, pl->yhat, pl->inf, nullptr, s));
    nl += launch_count() - before;
    pl->yhat_uid = warm->uid;
    pl->yhat_ver = warm->version;
  }
  if (ge) {
    PRGB_CUDA(cudaGraphLaunch(ge->exec, s));
    add_launches(ge->nodes);
    nl += ge->nodes;
  } else {
    // first solve with these parameters: the level loop launched directly
    // (the device starts at once), then captured for the next calls while
    // the device runs this one
    const SolveArgs a = plan_args(P, pl, c, tol, norm, max_iter, mixed, warm, lu);
    PRGB_TRY(plan_head(pl, P->n_comp, s, &nl));
    PRGB_TRY(enqueue_levels(P, a, pl->b, mixed, pl->side, s, timing ? &pl->kt : nullptr, &nl,
                            warm ? pl->yhat : nullptr));
  }
  if (R_on_host) {
    PRGB_TRY(scatter_out(P, pl->b.R, pl->Rout, s, &nl));
    if (n > 0) PRGB_COPY(cudaMemcpyAsync(R, pl->Rout, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
  } else {
    PRGB_TRY(scatter_out(P, pl->b.R, R, s, &nl));
  }
  PRGB_CUDA(cudaEventRecord(pl->done, s));
  *launches = nl;
  if (!ge) PRGB_TRY(plan_capture(P, pl, c, tol, norm, max_iter, mixed, timing, warm, lu));
  return PR_OK;
}

static int32_t g_tuned_cta = kCtaCompMax;
static int32_t g_tuned_blocks = 4;
static int32_t g_tuned_balance = 1;

void tuned_defaults(int32_t* cta_max, int32_t* coop_blocks, int32_t* balance) {
  *cta_max = g_tuned_cta;
  *coop_blocks = g_tuned_blocks;
  *balance = g_tuned_balance;
}

void split_fx_ranges(pr_partition_s* P) {
  const std::vector<int32_t>& co = P->h_c_off;
  auto size = [&](int c) { return co[c + 1] - co[c]; };
  for (LevelRange& r : P->levels) {
    // sizes descend: [big, cta) are the cluster-class components of at most
    // kFxMax vertices
    int lo = r.clu, hi = r.cta;
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      if (size(mid) <= kFxMax) hi = mid;
      else lo = mid + 1;
    }
    r.big = lo;
    r.big_max = r.cta > r.big ? size(r.big) : 0;
  }
}

void retune_levels(pr_partition_s* P, int32_t cta_max, int32_t coop_blocks, int32_t balance) {
  P->cta_max = cta_max;
  P->coop_blocks = coop_blocks;
  P->balance = balance;
  const std::vector<int32_t>& co = P->h_c_off;
  auto size = [&](int c) { return co[c + 1] - co[c]; };
  for (LevelRange& r : P->levels) {
    // sizes descend inside a level: the CTA class starts at the first
    // component in [clu, warp) with at most cta_max vertices
    int lo = r.clu, hi = r.warp;
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      if (size(mid) <= cta_max) hi = mid;
      else lo = mid + 1;
    }
    r.cta = lo;
    r.clu_max = r.cta > r.clu ? size(r.clu) : 0;
  }
  split_fx_ranges(P);
  if (P->plan) {
    for (PlanGraph& e : P->plan->graphs) {
      if (e.exec) cudaGraphExecDestroy(e.exec);
      if (e.graph) cudaGraphDestroy(e.graph);
    }
    P->plan->graphs.clear();
  }
}

pr_status tune_partition(pr_partition_s* P, double c, const double* u, double tol, cudaStream_t s,
                         int32_t* cta_max, int32_t* coop_blocks, int32_t* balance, float* best_ms) {
  // the class boundary x grid shape with cost-balanced sweeps, then the best
  // of those without balancing
  struct Cand {
    int32_t cta, blocks, bal;
  };
  std::vector<Cand> cands;
  for (int32_t cm : {64, 128, kCtaCompMax})
    for (int32_t b : {3, 4}) cands.push_back({cm, b, 1});
  float best = -1.0f;
  Cand bc{P->cta_max, P->coop_blocks, P->balance};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PRGB_CUDA(cudaEventCreate(&e0));
  PRGB_CUDA(cudaEventCreate(&e1));
  pr_status st = PR_OK;
  double* R = nullptr;
  Arena tmp(s);
  st = tmp.alloc(&R, (size_t)P->g.n + 1);
  for (size_t ci = 0; ci <= cands.size() && st == PR_OK; ci++) {
    // the last round tries the best so far without balancing
    const Cand cd = ci < cands.size() ? cands[ci] : Cand{bc.cta, bc.blocks, 0};
    retune_levels(P, cd.cta, cd.blocks, cd.bal);
    SolvePlan* pl = nullptr;
    int64_t nl = 0;
    float t = 1e30f;
    for (int rep = 0; rep < 3 && st == PR_OK; rep++) {  // the first runs directly and captures the graph
      if (cudaEventRecord(e0, s) != cudaSuccess) st = PR_ECUDA;
      if (st == PR_OK)
        st = plan_solve(P, c, u, false, tol, PR_NORM_L1, 10000, false, false, nullptr, 0, R, false, s, &pl, &nl);
      if (st == PR_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
        st = PR_ECUDA;
      float ms = 0.0f;
      if (st == PR_OK && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) t = std::min(t, ms);
    }
    if (st == PR_OK && pl) {
      int err = 0;
      if (cudaMemcpyAsync(&err, &pl->ctl->err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        st = PR_ECUDA;
      else if (err)
        st = (pr_status)err;
    }
    if (st == PR_OK && (best < 0.0f || t < best)) {
      best = t;
      bc = cd;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  retune_levels(P, bc.cta, bc.blocks, bc.bal);
  if (st != PR_OK) return st;
  g_tuned_cta = bc.cta;
  g_tuned_blocks = bc.blocks;
  g_tuned_balance = bc.bal;
  if (cta_max) *cta_max = bc.cta;
  if (coop_blocks) *coop_blocks = bc.blocks;
  if (balance) *balance = bc.bal;
  if (best_ms) *best_ms = best;
  return PR_OK;
}

pr_status solve_edge_visits(const pr_partition_s* P, const int32_t* iters_dev, const int32_t* iters64_dev,
                            int64_t* out, int64_t* out64, Arena& tmp) {
  cudaStream_t s = tmp.stream();
  *out = 0;
  if (out64) *out64 = 0;
  if (P->n_comp == 0) return PR_OK;
  unsigned long long* d = nullptr;
  PRGB_TRY(tmp.alloc(&d, 2));
  PRGB_CUDA(cudaMemsetAsync(d, 0, 16, s));
  edge_visits_k<<<grid_cap((P->n_comp + kBlock - 1) / kBlock), kBlock, 0, s>>>(
      P->n_comp, P->c_off, P->c_type, P->int_ptr, P->ext_ptr, iters_dev, iters64_dev, d);
  PRGB_LAUNCH();
  unsigned long long h[2] = {0, 0};
  PRGB_CUDA(cudaMemcpyAsync(h, d, 16, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  *out = (int64_t)h[0];
  if (out64) *out64 = (int64_t)h[1];
  return PR_OK;
}

}  // namespace prgb
