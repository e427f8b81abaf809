// global.cu -- the baseline method (Sec. 4.3.2: the same power series on the
// whole graph; Sec. 5.2 method 1) and the residual of the defining system
// (I - cA^T) R = u (Def. 3.5).
#include <algorithm>

#include "common.cuh"
#include "global.cuh"
#include "spmv.cuh"

namespace prgb {


__device__ __forceinline__ double gdiv(double x, int deg) { return deg > 0 ? x / (double)deg : 0.0; }

// P_0 = u, R = u; repeat P <- c A^T P, R += P; stop after adding P with
// ||P||_1 <= tol (L1) or when max(P) < tol (the paper's rule).  One
// cooperative launch; the stopping sum is reduced deterministically (block
// partials summed in block order by every block, heavy rows by the fixed
// tree of spmv.cuh).
__global__ void __launch_bounds__(kBlock) global_power_k(GlobalArgs a) {
  __shared__ double red[kBlock / 32];
  const int n = a.n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double uu = a.u[i];
    if (!(uu >= 0.0) || !isfinite(uu)) set_err(a.ctl, PR_EINVAL, 400);
    a.R[i] = uu;
    a.zA[i] = uu * a.civ[i];
  }
  if (!grid_sync(a.ctl, 401)) return;
  const bool l1 = a.norm == PR_NORM_L1;
  const int nlight = n - a.hv.nheavy;
  int lr0 = -1, lr1 = -1;  // this warp's light rows, balanced by cost
  if (a.lpre) warp_row_range(a.lpre, nlight, &lr0, &lr1);
  int k = 0;
  for (;;) {
    const double* cur = (k & 1) ? a.zB : a.zA;
    double* nxt = (k & 1) ? a.zA : a.zB;
    double local = 0.0;
    // z holds c P / outdeg (civ = c / outdeg): the in-edge sum is the next
    // term itself
    auto fin = [&](int row, double acc, bool heavy) -> double {
      const double pn = acc;
      a.R[row] += pn;
      nxt[row] = pn * a.civ[row];
      if (!heavy) local = fold2(local, pn, l1);
      return pn;
    };
    auto val = [&](int e) -> double { return cur[a.iidx[e]]; };
    balanced_sweep(a.iptr, a.lorder, nlight, a.hv, a.hs, k & 1, l1, fin, val, lr0, lr1);
    const double bs = l1 ? block_sum(local, red) : block_max(local, red);
    double* slot = a.part + (size_t)(k & 1) * gridDim.x;
    if (threadIdx.x == 0) slot[blockIdx.x] = bs;
    if (!grid_sync(a.ctl, 402)) return;
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t = fold2(t, __ldcg(&slot[b]), l1);
    double s = l1 ? block_sum(t, red) : block_max(t, red);
    if (a.hv.nheavy > 0) s = fold2(s, __ldcg(&a.hs.total[k & 1]), l1);
    k++;
    if (a.fixed >= 0) {
      if (k >= a.fixed) break;
      continue;
    }
    if (!(a.norm == PR_NORM_LINF ? (s >= a.tol) : (s > a.tol))) break;
    if (k >= a.max_iter) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctl->flags[0], 1);
      break;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->cnt[7] = k;
}

// sum_i |u_i + c * sum_{j -> i} R_j / outdeg(j) - R_i| with the division
// written out per edge (the defining expression), block partials plus the
// heavy rows' fold in hs.total[0]
__global__ void __launch_bounds__(kBlock) residual_k(int32_t n, const int32_t* __restrict__ iptr,
                                                     const int32_t* __restrict__ iidx,
                                                     const int32_t* __restrict__ outdeg,
                                                     const int32_t* __restrict__ lorder, HeavyRows hv,
                                                     HeavyScratch hs, double c, const double* __restrict__ u,
                                                     const double* __restrict__ R, double* __restrict__ part) {
  __shared__ double red[kBlock / 32];
  double local = 0.0;
  auto fin = [&](int row, double acc, bool heavy) -> double {
    const double r = fabs(u[row] + c * acc - R[row]);
    if (!heavy) local += r;
    return r;
  };
  auto val = [&](int e) -> double {
    const int j = iidx[e];
    return R[j] / (double)outdeg[j];
  };
  balanced_sweep(iptr, lorder, n - hv.nheavy, hv, hs, 0, true, fin, val);
  const double bs = block_sum(local, red);
  if (threadIdx.x == 0) part[blockIdx.x] = bs;
}

__global__ void __launch_bounds__(kBlock) sum_parts_k(const double* __restrict__ part, int np,
                                                      const double* __restrict__ heavy_total, double* out) {
  __shared__ double red[kBlock / 32];
  double t = 0.0;
  for (int b = threadIdx.x; b < np; b += blockDim.x) t += part[b];
  t = block_sum(t, red);
  if (threadIdx.x == 0) *out = heavy_total ? t + *heavy_total : t;
}

int residual_grid() { return num_sms() * 4; }

__global__ void civ_k(int32_t n, double c, const double* __restrict__ inv, double* __restrict__ civ) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    civ[i] = c * inv[i];
}

pr_status run_global(const DevGraph& g, double c, const double* u, double tol, int norm, int max_iter, int fixed,
                     double* R, int* iters, Arena& tmp, Ctl* ctl, float* kernel_ms) {
  cudaStream_t s = tmp.stream();
  *iters = 0;
  if (kernel_ms) *kernel_ms = 0.0f;
  if (g.n == 0) return PR_OK;
  GlobalArgs a;
  a.n = g.n;
  a.iptr = g.iptr;
  a.iidx = g.iidx;
  a.outdeg = g.outdeg;
  a.u = u;
  a.c = c;
  a.tol = tol;
  a.norm = norm;
  a.max_iter = max_iter;
  a.fixed = fixed;
  a.R = R;
  a.ctl = ctl;
  PRGB_TRY(tmp.alloc(&a.zA, g.n));
  PRGB_TRY(tmp.alloc(&a.zB, g.n));
  PRGB_TRY(tmp.alloc(&a.part, (size_t)2 * num_sms() * 8));
  a.hv.rows = g.heavy_rows;
  a.hv.choff = g.heavy_choff;
  a.hv.nheavy = g.nheavy;
  a.hv.nchunks = g.nchunks;
  a.hv.chrow = g.heavy_chrow;
  a.hv.cbase = 0;
  a.hv.hbase = 0;
  a.lorder = g.lorder;
  a.lpre = g.lpre;
  a.inv = g.inv;
  double* civ = nullptr;
  PRGB_TRY(tmp.alloc(&civ, g.n));
  civ_k<<<(unsigned)std::min<int64_t>(((int64_t)g.n + kBlock - 1) / kBlock, (int64_t)num_sms() * 16), kBlock, 0, s>>>(
      g.n, c, g.inv, civ);
  PRGB_LAUNCH();
  a.civ = civ;
  PRGB_TRY(alloc_heavy_scratch(&a.hs, g.nheavy, g.nchunks, tmp));
  PRGB_TRY(reset_ctl(ctl, s));
  void* args[] = {&a};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (kernel_ms) {
    PRGB_CUDA(cudaEventCreate(&e0));
    PRGB_CUDA(cudaEventCreate(&e1));
    PRGB_CUDA(cudaEventRecord(e0, s));
  }
  pr_status ls = launch_coop((const void*)global_power_k, kBlock, 0, s, args, 4, nullptr);
  if (kernel_ms && ls == PR_OK) cudaEventRecord(e1, s);
  int h[3] = {0, 0, 0};
  PRGB_CUDA(cudaMemcpyAsync(&h[0], &ctl->err, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaMemcpyAsync(&h[1], &ctl->flags[0], 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaMemcpyAsync(&h[2], &ctl->cnt[7], 4, cudaMemcpyDeviceToHost, s));
  cudaError_t se = cudaStreamSynchronize(s);
  if (kernel_ms && ls == PR_OK && se == cudaSuccess) cudaEventElapsedTime(kernel_ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (ls != PR_OK) return ls;
  PRGB_CUDA(se);
  *iters = h[2];
  if (h[0]) return (pr_status)h[0];
  if (h[1]) return PR_ENOCONV;
  return PR_OK;
}

pr_status run_residual(const DevGraph& g, double c, const double* u, const double* R, double* part, double* out_dev,
                       Arena& tmp) {
  cudaStream_t s = tmp.stream();
  const int np = residual_grid();
  HeavyRows hv;
  hv.rows = g.heavy_rows;
  hv.choff = g.heavy_choff;
  hv.chrow = g.heavy_chrow;
  hv.nheavy = g.nheavy;
  hv.nchunks = g.nchunks;
  HeavyScratch hs;
  PRGB_TRY(alloc_heavy_scratch(&hs, g.nheavy, g.nchunks, tmp));
  residual_k<<<np, kBlock, 0, s>>>(g.n, g.iptr, g.iidx, g.outdeg, g.lorder, hv, hs, c, u, R, part);
  PRGB_LAUNCH();
  sum_parts_k<<<1, kBlock, 0, s>>>(part, np, g.nheavy > 0 ? hs.total : nullptr, out_dev);
  PRGB_LAUNCH();
  return PR_OK;
}

}  // namespace prgb
