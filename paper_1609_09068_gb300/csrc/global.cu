// global.cu -- the baseline method (Sec. 4.3.2: the same power series on the
// whole graph; Sec. 5.2 method 1) and the residual of the defining system
// (I - cA^T) R = u (Def. 3.5).
#include "common.cuh"
#include "global.cuh"

namespace prgb {

constexpr int kGG = 8;  // lanes per row

__device__ __forceinline__ double gdiv(double x, int deg) { return deg > 0 ? x / (double)deg : 0.0; }

// P_0 = u, R = u; repeat P <- c A^T P, R += P; stop after adding P with
// ||P||_1 <= tol (L1) or when max(P) < tol (the paper's rule).  One
// cooperative launch; the stopping sum is reduced deterministically (block
// partials summed in block order by every block).
__global__ void __launch_bounds__(kBlock) global_power_k(GlobalArgs a) {
  __shared__ double red[kBlock / 32];
  const int n = a.n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double uu = a.u[i];
    if (!(uu >= 0.0) || !isfinite(uu)) set_err(a.ctl, PR_EINVAL, 400);
    a.R[i] = uu;
    a.zA[i] = gdiv(uu, a.outdeg[i]);
  }
  if (!grid_sync(a.ctl, 401)) return;
  const int lane = threadIdx.x & (kGG - 1);
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kGG;
  const int64_t ng = ((int64_t)gridDim.x * blockDim.x) / kGG;
  const int64_t wb = g0 - ((threadIdx.x & 31) / kGG);
  int k = 0;
  for (;;) {
    const double* cur = (k & 1) ? a.zB : a.zA;
    double* nxt = (k & 1) ? a.zA : a.zB;
    double local = 0.0;
    for (int64_t base = wb; base < n; base += ng) {
      const int64_t i = base + ((threadIdx.x & 31) / kGG);
      double acc = 0.0;
      if (i < n)
        for (int e = a.iptr[i] + lane; e < a.iptr[i + 1]; e += kGG) acc += cur[a.iidx[e]];
      acc = group_sum<kGG>(acc);
      if (i < n && lane == 0) {
        const double pn = a.c * acc;
        a.R[i] += pn;
        nxt[i] = gdiv(pn, a.outdeg[i]);
        local = a.norm == PR_NORM_L1 ? local + pn : fmax(local, pn);
      }
    }
    const double bs = a.norm == PR_NORM_L1 ? block_sum(local, red) : block_max(local, red);
    double* slot = a.part + (size_t)(k & 1) * gridDim.x;
    if (threadIdx.x == 0) slot[blockIdx.x] = bs;
    if (!grid_sync(a.ctl, 402)) return;
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      t = a.norm == PR_NORM_L1 ? t + slot[b] : fmax(t, slot[b]);
    const double s = a.norm == PR_NORM_L1 ? block_sum(t, red) : block_max(t, red);
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

// sum_i |u_i + c * sum_{j -> i} R_j / outdeg(j) - R_i|, block partials
__global__ void __launch_bounds__(kBlock) residual_k(int32_t n, const int32_t* __restrict__ iptr,
                                                     const int32_t* __restrict__ iidx,
                                                     const int32_t* __restrict__ outdeg, double c,
                                                     const double* __restrict__ u, const double* __restrict__ R,
                                                     double* __restrict__ part) {
  __shared__ double red[kBlock / 32];
  const int lane = threadIdx.x & (kGG - 1);
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kGG;
  const int64_t ng = ((int64_t)gridDim.x * blockDim.x) / kGG;
  const int64_t wb = g0 - ((threadIdx.x & 31) / kGG);
  double local = 0.0;
  for (int64_t base = wb; base < n; base += ng) {
    const int64_t i = base + ((threadIdx.x & 31) / kGG);
    double acc = 0.0;
    if (i < n)
      for (int e = iptr[i] + lane; e < iptr[i + 1]; e += kGG) {
        const int j = iidx[e];
        acc += R[j] / (double)outdeg[j];
      }
    acc = group_sum<kGG>(acc);
    if (i < n && lane == 0) local += fabs(u[i] + c * acc - R[i]);
  }
  const double bs = block_sum(local, red);
  if (threadIdx.x == 0) part[blockIdx.x] = bs;
}

__global__ void __launch_bounds__(kBlock) sum_parts_k(const double* __restrict__ part, int np, double* out) {
  __shared__ double red[kBlock / 32];
  double t = 0.0;
  for (int b = threadIdx.x; b < np; b += blockDim.x) t += part[b];
  t = block_sum(t, red);
  if (threadIdx.x == 0) *out = t;
}

int residual_grid() { return num_sms() * 4; }

pr_status run_global(const DevGraph& g, double c, const double* u, double tol, int norm, int max_iter, int fixed,
                     double* R, int* iters, Arena& tmp, Ctl* ctl) {
  cudaStream_t s = tmp.stream();
  *iters = 0;
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
  PRGB_TRY(reset_ctl(ctl, s));
  void* args[] = {&a};
  PRGB_TRY(launch_coop((const void*)global_power_k, kBlock, 0, s, args, 4, nullptr));
  int h[3] = {0, 0, 0};
  PRGB_CUDA(cudaMemcpyAsync(&h[0], &ctl->err, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaMemcpyAsync(&h[1], &ctl->flags[0], 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaMemcpyAsync(&h[2], &ctl->cnt[7], 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  *iters = h[2];
  if (h[0]) return (pr_status)h[0];
  if (h[1]) return PR_ENOCONV;
  return PR_OK;
}

pr_status run_residual(const DevGraph& g, double c, const double* u, const double* R, double* part, double* out_dev,
                       cudaStream_t s) {
  const int np = residual_grid();
  residual_k<<<np, kBlock, 0, s>>>(g.n, g.iptr, g.iidx, g.outdeg, c, u, R, part);
  PRGB_LAUNCH();
  sum_parts_k<<<1, kBlock, 0, s>>>(part, np, out_dev);
  PRGB_LAUNCH();
  return PR_OK;
}

}  // namespace prgb
