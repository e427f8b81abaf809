// prims.cu -- scan, stable radix sort and launch helpers used by the
// partitioner and the layout step (Sec. 4.2 notes that sorting by level and
// size can be done without comparisons; a radix sort is that kind of sort).
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>

#include <stddef.h>

#include "common.cuh"
#include "spmv.cuh"

namespace prgb {

static thread_local int g_last_cuda_error = 0;
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void add_launches(long long d) { g_launches.fetch_add(d, std::memory_order_relaxed); }
void set_last_cuda_error(cudaError_t e) { g_last_cuda_error = static_cast<int>(e); }

static thread_local int g_last_status = 0;

pr_status note_status(pr_status s) {
  if (s != PR_OK) g_last_status = static_cast<int>(s);
  return s;
}

pr_status take_last_status() {
  const int s = g_last_status;
  g_last_status = 0;
  return static_cast<pr_status>(s);
}
int last_cuda_error() { return g_last_cuda_error; }

// PRGB_FAULT: the spec as last seen, and the events counted since
static std::mutex g_fault_mu;
static std::string g_fault_spec;
static long long g_fault_seen[4] = {0, 0, 0, 0};

bool fault_hit(FaultKind k) {
  const char* env = getenv("PRGB_FAULT");
  if (!env || !*env) {
    if (!g_fault_spec.empty()) {
      std::lock_guard<std::mutex> lock(g_fault_mu);
      g_fault_spec.clear();
    }
    return false;
  }
  std::lock_guard<std::mutex> lock(g_fault_mu);
  if (g_fault_spec != env) {
    g_fault_spec = env;
    for (long long& c : g_fault_seen) c = 0;
  }
  static const char* const names[4] = {"alloc", "launch", "copy", "noconv"};
  const size_t len = strlen(names[k]);
  if (g_fault_spec.compare(0, len, names[k]) != 0 ||
      (g_fault_spec.size() > len && g_fault_spec[len] != ':'))
    return false;
  if (k == kFaultNoconv) return true;
  long long nth = 1;
  if (g_fault_spec.size() > len + 1) nth = atoll(g_fault_spec.c_str() + len + 1);
  return ++g_fault_seen[k] == (nth > 0 ? nth : 1);
}

static std::atomic<unsigned int> g_wait_us{0};
unsigned int wait_limit_us() { return g_wait_us.load(std::memory_order_relaxed); }
void set_wait_limit_us(unsigned int us) { g_wait_us.store(us, std::memory_order_relaxed); }

__global__ void set_wait_k(Ctl* ctl, unsigned int us) { ctl->wait_us = us; }

pr_status init_ctl(Ctl* ctl, cudaStream_t s) {
  // the wave counters are left alone: they add up over a whole partition
  PRGB_CUDA(cudaMemsetAsync(ctl, 0, offsetof(Ctl, waves), s));
  const unsigned int us = wait_limit_us();
  if (us) {
    set_wait_k<<<1, 1, 0, s>>>(ctl, us);
    PRGB_LAUNCH();
  }
  return PR_OK;
}

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

int64_t l2_bytes() {
  static int64_t cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

pr_status launch_coop(const void* kernel, int block, size_t smem, cudaStream_t s, void** args,
                      int max_per_sm, int* grid_out) {
  int per_sm = 0;
  PRGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem));
  if (per_sm <= 0) return PR_EINTERNAL;
  if (max_per_sm > 0 && per_sm > max_per_sm) per_sm = max_per_sm;
  const int grid = per_sm * num_sms();
  if (grid_out) *grid_out = grid;
  if (fault_hit(kFaultLaunch)) return PR_ECUDA;
  PRGB_CUDA(cudaLaunchCooperativeKernel(kernel, dim3(grid), dim3(block), args, smem, s));
  count_launch();
  return PR_OK;
}

int bits_for(uint32_t max_value) {
  int b = 0;
  while (b < 32 && (max_value >> b) != 0) b++;
  return b;
}

// ---------------------------------------------------------------------------
// exclusive scan (out has n+1 entries): tile reduce, scan of tile sums,
// tile scan with the tile offset.
// ---------------------------------------------------------------------------
constexpr int kScanItems = 16;
constexpr int kScanTile = kBlock * kScanItems;  // 4096
constexpr int64_t kScanFold = 2048;             // tiles up to which blocks fold the prefix themselves

// sum of v over the block (every thread gets it), on the integer pipes
__device__ __forceinline__ int32_t block_sum_i32(int32_t v, int32_t* sh) {
  v = (int32_t)__reduce_add_sync(0xffffffffu, (unsigned)v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  const int32_t t = (threadIdx.x & 31) < (int)(blockDim.x >> 5) ? sh[threadIdx.x & 31] : 0;
  const int32_t r = (int32_t)__reduce_add_sync(0xffffffffu, (unsigned)t);
  __syncthreads();  // sh may be reused
  return r;
}

template <typename T>
__global__ void scan_reduce_k(const T* __restrict__ in, int64_t n, int32_t* __restrict__ tile_sums) {
  __shared__ int32_t sh[kBlock / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    int64_t i = base + (int64_t)k * kBlock + threadIdx.x;
    if (i < n) s += (int32_t)in[i];
  }
  const int32_t t = block_sum_i32(s, sh);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = t;
}

// single block: exclusive scan of tile sums in place
__global__ void scan_tiles_k(int32_t* __restrict__ sums, int64_t ntiles) {
  __shared__ int32_t sh[kBlock];
  int32_t carry = 0;
  for (int64_t b = 0; b < ntiles; b += kBlock) {
    int64_t i = b + threadIdx.x;
    int32_t v = (i < ntiles) ? sums[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kBlock; o <<= 1) {
      int32_t t = (threadIdx.x >= o) ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    int32_t incl = sh[threadIdx.x];
    if (i < ntiles) sums[i] = carry + incl - v;
    int32_t tot = sh[kBlock - 1];
    __syncthreads();
    carry += tot;
  }
}

// tile_off: the exclusive prefix of the tile sums, or (fold) the tile sums
// themselves, whose prefix this block adds up first (few tiles: it saves
// the single-block scan launch between the two passes)
template <typename T>
__global__ void scan_tile_k(const T* __restrict__ in, int64_t n, const int32_t* __restrict__ tile_off, bool fold,
                            int32_t* __restrict__ out) {
  __shared__ int32_t sh[kBlock];
  __shared__ int32_t shr[kBlock / 32];
  int32_t toff;
  if (fold) {
    int32_t a = 0;
    for (int64_t t = threadIdx.x; t < (int64_t)blockIdx.x; t += blockDim.x) a += tile_off[t];
    toff = block_sum_i32(a, shr);
  } else {
    toff = tile_off[blockIdx.x];
  }
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  int32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    int64_t i = base + k;
    v[k] = (i < n) ? (int32_t)in[i] : 0;
    s += v[k];
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < kBlock; o <<= 1) {
    int32_t t = (threadIdx.x >= o) ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  int32_t run = toff + sh[threadIdx.x] - s;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    int64_t i = base + k;
    run += v[k];
    if (i < n) out[i + 1] = run;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

template <typename T>
static pr_status scan_impl(const T* in, int32_t* out, int64_t n, Arena& a) {
  cudaStream_t s = a.stream();
  if (n <= 0) {
    PRGB_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), s));
    return PR_OK;
  }
  const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
  int32_t* sums = nullptr;
  PRGB_TRY(a.alloc(&sums, (size_t)ntiles));
  scan_reduce_k<T><<<(unsigned)ntiles, kBlock, 0, s>>>(in, n, sums);
  PRGB_LAUNCH();
  // up to kScanFold tiles each block adds its predecessors' sums itself
  const bool fold = ntiles <= kScanFold;
  if (!fold) {
    scan_tiles_k<<<1, kBlock, 0, s>>>(sums, ntiles);
    PRGB_LAUNCH();
  }
  scan_tile_k<T><<<(unsigned)ntiles, kBlock, 0, s>>>(in, n, sums, fold, out);
  PRGB_LAUNCH();
  return PR_OK;
}

pr_status scan_i32(const int32_t* in, int32_t* out, int64_t n, Arena& a) { return scan_impl(in, out, n, a); }
pr_status scan_u8(const uint8_t* in, int32_t* out, int64_t n, Arena& a) { return scan_impl(in, out, n, a); }

__global__ void iota_k(uint32_t* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (uint32_t)i;
}

static unsigned grid_for(int64_t n, int block = kBlock) {
  int64_t g = (n + block - 1) / block;
  int64_t cap = (int64_t)num_sms() * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

pr_status iota_u32(uint32_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return PR_OK;
  iota_k<<<grid_for(n), kBlock, 0, s>>>(out, n);
  PRGB_LAUNCH();
  return PR_OK;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 8 bits per pass.  A tile is 8 warps x 256 items;
// warp w owns items [w*256, w*256+256) of the tile, processed in 8 rounds of
// 32 consecutive items, so (warp, round, lane) is the input order and the
// local rank below preserves it.
// ---------------------------------------------------------------------------
constexpr int kRadixWarps = 8;
constexpr int kRadixRounds = 8;
constexpr int kRadixTile = kRadixWarps * kRadixRounds * 32;  // 2048

__global__ void radix_hist_k(const uint32_t* __restrict__ keys, int64_t n, int shift, int ntiles,
                             int32_t* __restrict__ hist) {
  __shared__ int32_t h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  for (int k = threadIdx.x; k < kRadixTile; k += blockDim.x) {
    int64_t i = base + k;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

__global__ void radix_scatter_k(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
                                int shift, int ntiles, const int32_t* __restrict__ offs) {
  __shared__ int32_t wcnt[kRadixWarps][256];
  __shared__ int32_t base[256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kRadixWarps * 256; i += blockDim.x) (&wcnt[0][0])[i] = 0;
  for (int d = threadIdx.x; d < 256; d += blockDim.x) base[d] = offs[(int64_t)d * ntiles + blockIdx.x];
  __syncthreads();
  const int64_t w0 = (int64_t)blockIdx.x * kRadixTile + warp * (kRadixRounds * 32);
  uint32_t k[kRadixRounds], v[kRadixRounds];
  int d[kRadixRounds];
#pragma unroll
  for (int r = 0; r < kRadixRounds; r++) {
    const int64_t i = w0 + r * 32 + lane;
    const bool ok = i < n;
    k[r] = ok ? kin[i] : 0u;
    v[r] = ok ? vin[i] : 0u;
    d[r] = ok ? (int)((k[r] >> shift) & 255u) : 256 + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, d[r]);
    if (ok && lane == __ffs(peers) - 1) wcnt[warp][d[r]] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  for (int dd = threadIdx.x; dd < 256; dd += blockDim.x) {
    int run = 0;
    for (int w = 0; w < kRadixWarps; w++) {
      int c = wcnt[w][dd];
      wcnt[w][dd] = run;
      run += c;
    }
  }
  __syncthreads();
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int r = 0; r < kRadixRounds; r++) {
    const bool ok = d[r] < 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d[r]);
    if (ok) {
      const int pos = base[d[r]] + wcnt[warp][d[r]] + __popc(peers & lt);
      kout[pos] = k[r];
      vout[pos] = v[r];
    }
    __syncwarp();
    if (ok && lane == __ffs(peers) - 1) wcnt[warp][d[r]] += __popc(peers);
    __syncwarp();
  }
}

pr_status radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                           int64_t n, int key_bits, Arena& a) {
  if (n <= 1 || key_bits <= 0) return PR_OK;
  if (n >= (int64_t)1 << 31) return PR_EINVAL;
  cudaStream_t s = a.stream();
  const int ntiles = (int)((n + kRadixTile - 1) / kRadixTile);
  int32_t *hist = nullptr, *offs = nullptr;
  PRGB_TRY(a.alloc(&hist, (size_t)ntiles * 256));
  PRGB_TRY(a.alloc(&offs, (size_t)ntiles * 256 + 1));
  uint32_t *ka = keys, *va = vals, *kb = keys_tmp, *vb = vals_tmp;
  for (int shift = 0; shift < key_bits; shift += 8) {
    radix_hist_k<<<ntiles, kBlock, 0, s>>>(ka, n, shift, ntiles, hist);
    PRGB_LAUNCH();
    PRGB_TRY(scan_i32(hist, offs, (int64_t)ntiles * 256, a));
    radix_scatter_k<<<ntiles, kRadixWarps * 32, 0, s>>>(ka, va, kb, vb, n, shift, ntiles, offs);
    PRGB_LAUNCH();
    uint32_t* t;
    t = ka; ka = kb; kb = t;
    t = va; va = vb; vb = t;
  }
  if (ka != keys) {
    PRGB_CUDA(cudaMemcpyAsync(keys, ka, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    PRGB_CUDA(cudaMemcpyAsync(vals, va, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
  }
  return PR_OK;
}

}  // namespace prgb

namespace prgb {

__global__ void heavy_flags_k(const int32_t* __restrict__ ptr, int32_t nrows, uint8_t* flag, int32_t* nch) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x) {
    const int d = ptr[i + 1] - ptr[i];
    const bool h = d > kHeavy;
    flag[i] = h;
    nch[i] = h ? (d + kChunkH - 1) / kChunkH : 0;
  }
}

__global__ void heavy_fill_k(int32_t nrows, const uint8_t* flag, const int32_t* hidx, const int32_t* cho_all,
                             int32_t* rows, int32_t* choff) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x) {
    if (flag[i]) {
      rows[hidx[i]] = (int32_t)i;
      choff[hidx[i]] = cho_all[i];
    }
  }
}

__global__ void heavy_chrow_k(int32_t nheavy, const int32_t* choff, int32_t* chrow) {
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nheavy; h += (int64_t)gridDim.x * blockDim.x)
    for (int c = choff[h]; c < choff[h + 1]; c++) chrow[c] = (int32_t)h;
}

pr_status build_heavy(const int32_t* ptr, int32_t nrows, Arena& keep, Arena& tmp, int32_t** rows,
                      int32_t** choff, int32_t** chrow, int32_t* nheavy, int32_t* nchunks) {
  cudaStream_t s = tmp.stream();
  *nheavy = 0;
  *nchunks = 0;
  uint8_t* flag;
  int32_t *nch, *hidx, *cho_all;
  PRGB_TRY(tmp.alloc(&flag, (size_t)nrows + 1));
  PRGB_TRY(tmp.alloc(&nch, (size_t)nrows + 1));
  PRGB_TRY(tmp.alloc(&hidx, (size_t)nrows + 1));
  PRGB_TRY(tmp.alloc(&cho_all, (size_t)nrows + 1));
  if (nrows > 0) {
    heavy_flags_k<<<grid_for(nrows), kBlock, 0, s>>>(ptr, nrows, flag, nch);
    PRGB_LAUNCH();
  }
  PRGB_TRY(scan_u8(flag, hidx, nrows, tmp));
  PRGB_TRY(scan_i32(nch, cho_all, nrows, tmp));
  int32_t h[2] = {0, 0};
  PRGB_CUDA(cudaMemcpyAsync(&h[0], hidx + nrows, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaMemcpyAsync(&h[1], cho_all + nrows, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  *nheavy = h[0];
  *nchunks = h[1];
  PRGB_TRY(keep.alloc(rows, (size_t)h[0] + 1));
  PRGB_TRY(keep.alloc(choff, (size_t)h[0] + 1));
  if (h[0] > 0) {
    heavy_fill_k<<<grid_for(nrows), kBlock, 0, s>>>(nrows, flag, hidx, cho_all, *rows, *choff);
    PRGB_LAUNCH();
  }
  // a copy from pageable host memory has read its source when the call
  // returns, so h may go out of scope without a synchronisation
  PRGB_CUDA(cudaMemcpyAsync(*choff + h[0], &h[1], 4, cudaMemcpyHostToDevice, s));
  PRGB_TRY(keep.alloc(chrow, (size_t)h[1] + 1));
  if (h[0] > 0) {
    heavy_chrow_k<<<grid_for(h[0]), kBlock, 0, s>>>(h[0], *choff, *chrow);
    PRGB_LAUNCH();
  }
  return PR_OK;
}

}  // namespace prgb

namespace prgb {

__global__ void lorder_keys_k(const int32_t* __restrict__ ptr, int32_t nrows, const int32_t* __restrict__ group,
                              uint32_t* keys, uint32_t* vals) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t g = group ? (uint32_t)group[i] : 0u;
    keys[i] = (g << 4) | (uint32_t)deg_class(ptr[i + 1] - ptr[i]);
    vals[i] = (uint32_t)i;
  }
}

pr_status build_lorder(const int32_t* ptr, int32_t nrows, const int32_t* group, int32_t group_max, Arena& keep,
                       Arena& tmp, int32_t** lorder) {
  cudaStream_t s = tmp.stream();
  const int gbits = group ? bits_for((uint32_t)group_max) : 0;
  if (gbits + 4 > 32) return PR_EINVAL;
  uint32_t *k, *kt, *vt;
  PRGB_TRY(tmp.alloc(&k, (size_t)nrows + 1));
  PRGB_TRY(tmp.alloc(&kt, (size_t)nrows + 1));
  PRGB_TRY(tmp.alloc(&vt, (size_t)nrows + 1));
  PRGB_TRY(keep.alloc(lorder, (size_t)nrows + 1));
  if (nrows == 0) return PR_OK;
  lorder_keys_k<<<grid_for(nrows), kBlock, 0, s>>>(ptr, nrows, group, k, reinterpret_cast<uint32_t*>(*lorder));
  PRGB_LAUNCH();
  return radix_sort_pairs(k, reinterpret_cast<uint32_t*>(*lorder), kt, vt, nrows, gbits + 4, tmp);
}

__global__ void row_cost_k(const int32_t* __restrict__ ptr, const int32_t* __restrict__ lorder, int32_t n,
                           int32_t* __restrict__ cost) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int r = lorder[i];
    cost[i] = ptr[r + 1] - ptr[r] + kRowCost;
  }
}

pr_status build_lpre(const int32_t* ptr, const int32_t* lorder, int32_t n, int64_t m, Arena& keep, Arena& tmp,
                     int32_t** lpre) {
  *lpre = nullptr;
  if (n == 0 || m + (int64_t)kRowCost * n >= ((int64_t)1 << 31)) return PR_OK;  // ranges off: prefix too large
  cudaStream_t s = tmp.stream();
  int32_t* cost;
  PRGB_TRY(tmp.alloc(&cost, (size_t)n + 1));
  PRGB_TRY(keep.alloc(lpre, (size_t)n + 1));
  row_cost_k<<<grid_for(n), kBlock, 0, s>>>(ptr, lorder, n, cost);
  PRGB_LAUNCH();
  return scan_i32(cost, *lpre, n, tmp);
}

__global__ void inv_deg_k(const int32_t* __restrict__ deg, int32_t n, double* inv) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    inv[i] = deg[i] > 0 ? 1.0 / (double)deg[i] : 0.0;
}

pr_status build_inv(const int32_t* deg, int32_t n, Arena& keep, double** inv, cudaStream_t s) {
  PRGB_TRY(keep.alloc(inv, (size_t)n + 1));
  if (n == 0) return PR_OK;
  inv_deg_k<<<grid_for(n), kBlock, 0, s>>>(deg, n, *inv);
  PRGB_LAUNCH();
  return PR_OK;
}

}  // namespace prgb
