// noalloc.cu -- pr_residual_l1_static: the L1 residual without any device
// allocation.
//
// Some callers cannot allocate device memory: code that runs inside another
// framework's memory manager (which owns every device byte and rejects side
// allocations), or code on a latency-critical path where cudaMalloc and
// cudaFree would synchronise the device.  This entry point serves them: it
// reads the caller's CSR, u and R and writes the residual to host memory,
// using only the fixed scratch below, which lives in the library's own
// device data segment.  Every GPU that loads the library holds that scratch
// (about 8 MiB) until the process exits.
#include <mutex>

#include "common.cuh"

namespace prgb {

constexpr int kStaticBlocks = 1024;  // block partials of the final sum

// One accumulator per vertex (in-flow c * sum R_j / outdeg_j), the block
// partials, the result slot and an error flag.  Shared by every call on the
// device: each call clears the accumulators it uses, and calls that overlap
// on the GPU race on them.
static __device__ __align__(256) double g_static_acc[PR_STATIC_MAX_N];
static __device__ __align__(256) double g_static_part[kStaticBlocks + 1];
static __device__ __align__(256) int g_static_err[2];

struct StaticScratch {
  double* acc = nullptr;
  double* part = nullptr;
  int* err = nullptr;
};

// Host code cannot use the symbols above as device addresses: each device's
// addresses are looked up once, with that device current.
static pr_status static_scratch(StaticScratch* out) {
  static std::mutex mu;
  static bool ready[64] = {false};
  static StaticScratch cache[64];
  int dev = 0;
  PRGB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return PR_EINTERNAL;
  std::lock_guard<std::mutex> lock(mu);
  if (!ready[dev]) {
    StaticScratch s;
    PRGB_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&s.acc), g_static_acc));
    PRGB_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&s.part), g_static_part));
    PRGB_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&s.err), g_static_err));
    cache[dev] = s;
    ready[dev] = true;
  }
  *out = cache[dev];
  return PR_OK;
}

__global__ void static_clear_k(int32_t n, double* acc, int* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc[i] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) err[0] = 0;
}

// one warp per row i: push c * R_i / outdeg(i) to every out-neighbour j != i
// (self-loops are ignored); malformed rows (bad offsets, columns out of
// range, unsorted or repeated) are flagged and skipped
__global__ void static_push_k(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int32_t n,
                              int64_t nnz, double c, const double* __restrict__ R, double* acc, int* err) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < n; i += nw) {
    const int64_t s = rowptr[i], e = rowptr[i + 1];
    if (s < 0 || e < s || e > nnz || (i == 0 && s != 0) || (i == n - 1 && e != nnz)) {
      if (lane == 0) atomicExch(err, 1);
      continue;
    }
    // the graph model is a simple digraph with sorted rows, as pr_graph_create
    // requires: a repeated or out-of-order column is rejected, not counted
    bool bad = false;
    for (int64_t k = s + 1 + lane; k < e; k += 32) bad |= col[k - 1] >= col[k];
    if (__any_sync(0xffffffffu, bad)) {
      if (lane == 0) atomicExch(err, 1);
      continue;
    }
    int loops = 0;
    for (int64_t k = s + lane; k < e; k += 32) loops += col[k] == (int32_t)i;
    loops = __reduce_add_sync(0xffffffffu, loops);
    const int64_t deg = (e - s) - loops;
    if (deg <= 0) continue;
    const double v = c * (R[i] / (double)deg);
    for (int64_t k = s + lane; k < e; k += 32) {
      const int32_t j = col[k];
      if (j < 0 || j >= n) {
        atomicExch(err, 1);
        continue;
      }
      if (j != (int32_t)i) atomicAdd(&acc[j], v);
    }
  }
}

__global__ void static_resid_k(int32_t n, const double* __restrict__ u, const double* __restrict__ R,
                               const double* __restrict__ acc, double* part) {
  __shared__ double red[kBlock / 32];
  double t = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    t += fabs(u[i] + acc[i] - R[i]);
  t = block_sum(t, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void static_final_k(int nparts, double* part) {
  __shared__ double red[kBlock / 32];
  double t = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) t += part[b];
  t = block_sum(t, red);
  if (threadIdx.x == 0) part[kStaticBlocks] = t;
}

}  // namespace prgb

using namespace prgb;

static pr_status pr_residual_l1_static_body(const pr_csr* g, double c, const double* u, const double* R,
                                           double* out_host, void* stream) {
  if (!g || !out_host || g->on_host) return PR_EINVAL;
  if (g->n < 0 || g->n > PR_STATIC_MAX_N || g->nnz < 0 || g->nnz >= ((int64_t)1 << 31)) return PR_EINVAL;
  const int32_t n = g->n;
  if (n > 0 && (!g->rowptr || (g->nnz > 0 && !g->col) || !u || !R)) return PR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  StaticScratch sc;
  PRGB_TRY(static_scratch(&sc));
  const int nb = (int)((n + kBlock - 1) / kBlock) < kStaticBlocks ? (int)((n + kBlock - 1) / kBlock) : kStaticBlocks;
  const int grid = nb < 1 ? 1 : nb;
  static_clear_k<<<grid, kBlock, 0, s>>>(n, sc.acc, sc.err);
  PRGB_LAUNCH();
  if (n > 0) {
    static_push_k<<<kStaticBlocks, kBlock, 0, s>>>(g->rowptr, g->col, n, g->nnz, c, R, sc.acc, sc.err);
    PRGB_LAUNCH();
  }
  static_resid_k<<<grid, kBlock, 0, s>>>(n, u, R, sc.acc, sc.part);
  PRGB_LAUNCH();
  static_final_k<<<1, kBlock, 0, s>>>(grid, sc.part);
  PRGB_LAUNCH();
  int err = 0;
  PRGB_CUDA(cudaMemcpyAsync(out_host, sc.part + kStaticBlocks, sizeof(double), cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaMemcpyAsync(&err, sc.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  return err ? PR_EINVAL : PR_OK;
}

extern "C" pr_status pr_residual_l1_static(const pr_csr* g, double c, const double* u, const double* R,
                                           double* out_host, void* stream) {
  return prgb::note_status(pr_residual_l1_static_body(g, c, u, R, out_host, stream));
}
