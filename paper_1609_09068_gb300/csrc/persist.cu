// persist.cu -- the device side of pr_partition_save / pr_partition_load.
//
// A partition file keeps what the search of Sec. 4.1 finds (per vertex: its
// component, the component's type of Def. 3.1-3.2 and level of Def. 3.3,
// and the sub-level wave that orders a CAC topologically).  Everything else
// of a partition is the layout of Sec. 4.2, which build_layout derives from
// those arrays and the graph alone.  The file is tied to its graph by a
// digest of the loop-free edge set; the arrays carry a digest of their own,
// and the loader checks their ranges before the layout indexes with them.
#include <stdint.h>

#include "common.cuh"

namespace prgb {

namespace {

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

unsigned grid1(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  int64_t cap = (int64_t)num_sms() * 16;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

// The SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014): a bijection of 64-bit words
// whose outputs are well spread, so that the sum of mix(item) over a set is
// an order-independent digest of the set.
__device__ __forceinline__ uint64_t mix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// a warp's sum modulo 2^64, then one atomic per warp
__device__ __forceinline__ void warp_add_u64(uint64_t h, unsigned long long* out) {
  for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, (unsigned long long)h);
}

// sum over the in-edges (w -> v) of mix(w, v): the rows are walked by
// threads, whole warps stay in the loop so that the shuffles see all lanes
__global__ void edge_digest_k(int32_t n, const int32_t* __restrict__ iptr, const int32_t* __restrict__ iidx,
                              unsigned long long* out) {
  uint64_t h = 0;
  const int lane = threadIdx.x & 31;
  for (int64_t vb = gtid() - lane; vb < n; vb += gstride()) {
    const int64_t v = vb + lane;
    if (v < n) {
      for (int e = iptr[v]; e < iptr[v + 1]; e++) h += mix(((uint64_t)(uint32_t)iidx[e] << 32) | (uint64_t)v);
    }
  }
  warp_add_u64(h, out);
}

// sum over the vertices of a digest of (v, comp, level, wave, type); with
// check set, a value outside its range sets PR_EINVAL
__global__ void part_digest_k(int32_t n, const int32_t* __restrict__ comp, const uint8_t* __restrict__ type,
                              const int32_t* __restrict__ level, const int32_t* __restrict__ wave, int32_t n_comp,
                              int32_t n_levels, int32_t max_wave, int check, unsigned long long* out, Ctl* ctl) {
  uint64_t h = 0;
  const int lane = threadIdx.x & 31;
  for (int64_t vb = gtid() - lane; vb < n; vb += gstride()) {
    const int64_t v = vb + lane;
    if (v < n) {
      const int32_t c = comp[v], l = level[v], w = wave[v];
      const uint8_t t = type[v];
      if (check && (c < 0 || c >= n_comp || l < 0 || l >= n_levels || w < 0 || w > max_wave || t > 1))
        set_err(ctl, PR_EINVAL, 60);
      uint64_t x = mix(((uint64_t)v << 32) | (uint32_t)c);
      x = mix(x ^ (((uint64_t)(uint32_t)l << 32) | (uint32_t)w));
      h += mix(x ^ t);
    }
  }
  warp_add_u64(h, out);
}

__global__ void comp_min_k(int32_t n, const int32_t* __restrict__ comp, int32_t* cmin) {
  for (int64_t v = gtid(); v < n; v += gstride()) atomicMin(&cmin[comp[v]], (int32_t)v);
}

__global__ void crep_of_k(int32_t n, const int32_t* __restrict__ comp, const int32_t* __restrict__ cmin,
                          int32_t* crep) {
  for (int64_t v = gtid(); v < n; v += gstride()) crep[v] = cmin[comp[v]];
}

__global__ void same_ids_k(int32_t n, const int32_t* __restrict__ a, const int32_t* __restrict__ b, Ctl* ctl) {
  for (int64_t v = gtid(); v < n; v += gstride())
    if (a[v] != b[v]) set_err(ctl, PR_EINVAL, 61);
}

pr_status read_u64(const unsigned long long* d, uint64_t* out, cudaStream_t s) {
  unsigned long long h = 0;
  PRGB_CUDA(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  *out = (uint64_t)h;
  return PR_OK;
}

}  // namespace

pr_status graph_digest(const DevGraph& g, Arena& tmp, uint64_t* out) {
  cudaStream_t s = tmp.stream();
  unsigned long long* d;
  PRGB_TRY(tmp.alloc(&d, 1));
  PRGB_CUDA(cudaMemsetAsync(d, 0, sizeof(*d), s));
  if (g.n > 0) {
    edge_digest_k<<<grid1(g.n), kBlock, 0, s>>>(g.n, g.iptr, g.iidx, d);
    PRGB_LAUNCH();
  }
  return read_u64(d, out, s);
}

pr_status partition_digest(int32_t n, const int32_t* comp, const uint8_t* type, const int32_t* level,
                           const int32_t* wave, int32_t n_comp, int32_t n_levels, int32_t max_wave, bool check,
                           Arena& tmp, Ctl* ctl, uint64_t* out) {
  cudaStream_t s = tmp.stream();
  unsigned long long* d;
  PRGB_TRY(tmp.alloc(&d, 1));
  PRGB_CUDA(cudaMemsetAsync(d, 0, sizeof(*d), s));
  if (n > 0) {
    part_digest_k<<<grid1(n), kBlock, 0, s>>>(n, comp, type, level, wave, n_comp, n_levels, max_wave, check ? 1 : 0,
                                              d, ctl);
    PRGB_LAUNCH();
  }
  return read_u64(d, out, s);
}

pr_status smallest_members(int32_t n, int32_t n_comp, const int32_t* comp, int32_t* crep, Arena& tmp) {
  cudaStream_t s = tmp.stream();
  if (n == 0) return PR_OK;
  int32_t* cmin;
  PRGB_TRY(tmp.alloc(&cmin, (size_t)n_comp));
  PRGB_CUDA(cudaMemsetAsync(cmin, 0x7f, (size_t)n_comp * 4, s));
  comp_min_k<<<grid1(n), kBlock, 0, s>>>(n, comp, cmin);
  PRGB_LAUNCH();
  crep_of_k<<<grid1(n), kBlock, 0, s>>>(n, comp, cmin, crep);
  PRGB_LAUNCH();
  return PR_OK;
}

pr_status check_same_ids(int32_t n, const int32_t* a, const int32_t* b, Ctl* ctl, cudaStream_t s) {
  if (n == 0) return PR_OK;
  same_ids_k<<<grid1(n), kBlock, 0, s>>>(n, a, b, ctl);
  PRGB_LAUNCH();
  return PR_OK;
}

}  // namespace prgb
