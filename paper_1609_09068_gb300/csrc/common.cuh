// common.cuh -- internal definitions shared by the CUDA translation units of
// the componentwise PageRank library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>
#include <vector>

#include "prgb.h"

namespace prgb {

constexpr int kWarp = 32;
constexpr int kBlock = 256;                 // threads per block for most kernels
constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded device waits: 2 s

// ---------------------------------------------------------------------------
// status plumbing
// ---------------------------------------------------------------------------
void set_last_cuda_error(cudaError_t e);
// records a non-OK status of a public call (read and cleared by
// pr_last_device_error); returns s
pr_status note_status(pr_status s);
pr_status take_last_status();

#define PRGB_TRY(expr)                                   \
  do {                                                   \
    pr_status st_ = (expr);                              \
    if (st_ != PR_OK) return st_;                        \
  } while (0)

#define PRGB_CUDA(expr)                                  \
  do {                                                   \
    cudaError_t e_ = (expr);                             \
    if (e_ != cudaSuccess) {                             \
      ::prgb::set_last_cuda_error(e_);                   \
      return e_ == cudaErrorMemoryAllocation ? PR_ENOMEM : PR_ECUDA; \
    }                                                    \
  } while (0)

// Host-side fault injection for tests of the failure paths (no GPU fault
// is involved): PRGB_FAULT=alloc[:N], launch[:N] or copy[:N] makes the N-th
// device allocation, kernel launch or host<->device copy (N = 1 by default,
// counted from the moment the variable took its current value) report
// failure -- PR_ENOMEM, PR_ECUDA, PR_ECUDA.  An allocation, a copy or a
// cooperative launch is then not made; an ordinary kernel launch is reported
// failed right after it is enqueued, as a launch error would be (the call's
// buffers are released in stream order behind it).  PRGB_FAULT=noconv caps
// the series at one sweep (PR_ENOCONV).
enum FaultKind { kFaultAlloc = 0, kFaultLaunch = 1, kFaultCopy = 2, kFaultNoconv = 3 };
bool fault_hit(FaultKind k);

void count_launch();
long long launch_count();
void add_launches(long long d);  // kernels launched by a graph replay (or removed: captured, not run)
#define PRGB_LAUNCH()                                               \
  do {                                                              \
    if (::prgb::fault_hit(::prgb::kFaultLaunch)) return PR_ECUDA;   \
    ::prgb::count_launch();                                         \
    PRGB_CUDA(cudaGetLastError());                                  \
  } while (0)
// a host<->device copy of the caller's data
#define PRGB_COPY(expr)                                             \
  do {                                                              \
    if (::prgb::fault_hit(::prgb::kFaultCopy)) return PR_ECUDA;     \
    PRGB_CUDA(expr);                                                \
  } while (0)

// A named range on the host timeline of a profiler (NVTX): the phases of a
// call and each level of a solve.  It brackets what the call enqueues; for a
// solve replayed from its CUDA graph the level ranges mark the capture.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  NvtxRange(const char* name, int k) {
    char buf[64];
    snprintf(buf, sizeof buf, "%s %d", name, k);
    nvtxRangePushA(buf);
  }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------
// device control block: error word and grid-barrier state.  One per call
// site that needs it, zeroed before each persistent launch.
// ---------------------------------------------------------------------------
// The words that different blocks hammer at the same time sit on separate
// 128-byte lines, so barrier arrivals, barrier polls and frontier pushes do
// not queue behind each other at one L2 slice.
struct Ctl {
  alignas(128) int err;  // pr_status written by kernels (first error wins)
  int where;             // diagnostic: which wait expired
  unsigned int wait_us;  // limit of each bounded wait in microseconds (0: kWaitNs)
  alignas(128) unsigned int bar_count;  // grid barrier arrivals
  alignas(128) unsigned int bar_gen;    // grid barrier releases (polled)
  alignas(128) int cnt[8];  // frontier counters (rotating)
  alignas(128) int flags[8];  // misc flags (e.g. not-converged)
  double dsum[4];
  // waves run by the partitioner's wave kernels, per WaveKind: [0] by the
  // whole grid (a grid barrier each), [1] by block 0 alone; counted by
  // block 0's thread 0.  init_ctl leaves them alone (they add up over the
  // phases of a partition): the partition zeroes them once.
  alignas(128) int waves[8][2];
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int vload(const int* p) { return *(volatile const int*)p; }
__device__ __forceinline__ unsigned int vloadu(const unsigned int* p) {
  return *(volatile const unsigned int*)p;
}

// the time a bounded wait may take before it gives up
__device__ __forceinline__ unsigned long long wait_limit_ns(const Ctl* ctl) {
  const unsigned int us = *(volatile const unsigned int*)&ctl->wait_us;
  return us ? (unsigned long long)us * 1000ull : kWaitNs;
}

__device__ __forceinline__ void set_err(Ctl* ctl, int code, int where) {
  if (atomicCAS(&ctl->err, 0, code) == 0) ctl->where = where;
}

// Arrival at the grid barrier: one fetch-add with acquire-release ordering
// at device scope (the block's earlier writes are visible to every block that
// sees the arrival, and this block sees theirs).
__device__ __forceinline__ unsigned int arrive_acq_rel(unsigned int* p) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
  return old;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 of a block arrives at the grid barrier and waits for the others,
// with a bounded wait.  The last block to arrive resets the count and
// releases the generation word, which the others poll with acquire loads;
// the count is thus 0 after every barrier (and must be when the kernel
// starts).  After wait_limit_ns a waiting block records PR_ETIMEOUT and
// leaves.
__device__ __forceinline__ void grid_arrive_wait(Ctl* ctl, int where) {
  // the generation cannot move before this block arrives, and it is at
  // least the one this block saw released at its previous barrier
  const unsigned int gen = ld_acquire_u32(&ctl->bar_gen);
  if (arrive_acq_rel(&ctl->bar_count) == gridDim.x - 1) {
    // the reset is ordered before the release of the generation, which
    // every block sees before it arrives again
    asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(&ctl->bar_count) : "memory");
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctl->bar_gen) : "memory");
    return;
  }
  const unsigned long long t0 = globaltimer_ns(), lim = wait_limit_ns(ctl);
  for (;;) {
    // both words in flight together: one round trip per poll
    const unsigned int g = ld_acquire_u32(&ctl->bar_gen);
    const int e = vload(&ctl->err);
    if (g != gen || e != 0) return;
    __nanosleep(32);
    if (globaltimer_ns() - t0 > lim) {
      set_err(ctl, PR_ETIMEOUT, where);
      return;
    }
  }
}

// Grid-wide barrier for cooperative launches.  Returns false when any block
// has recorded an error, so that callers can return early.
__device__ __forceinline__ bool grid_sync(Ctl* ctl, int where) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    grid_arrive_wait(ctl, where);
    ok = vload(&ctl->err) == 0;  // one read per block, not per thread
  }
  __syncthreads();
  return ok != 0;
}

// ---------------------------------------------------------------------------
// warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <int G>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int G>
__device__ __forceinline__ double group_max(double v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// FP32 overload: a float argument must not be widened to the FP64 version
template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int G>
__device__ __forceinline__ float group_sumf(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int G>
__device__ __forceinline__ float group_maxf(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide FP32 sum / max (fixed tree); scratch: blockDim/32 floats.
__device__ __forceinline__ float block_sumf(float v, float* scratch, bool is_max) {
  v = is_max ? group_maxf<32>(v) : group_sumf<32>(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  float t = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0f;
  if (w == 0) t = is_max ? group_maxf<32>(t) : group_sumf<32>(t);
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  const float r = scratch[0];
  __syncthreads();
  return r;
}

// Block-wide sum with a fixed reduction tree (deterministic for a fixed
// blockDim).  scratch: at least blockDim/32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  v = group_sum<32>(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  double t = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0;
  if (w == 0) t = group_sum<32>(t);
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  double r = scratch[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double block_max(double v, double* scratch) {
  v = group_max<32>(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  double t = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0;
  if (w == 0) t = group_max<32>(t);
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  double r = scratch[0];
  __syncthreads();
  return r;
}

// Warp-aggregated frontier push.  All 32 lanes must call it; a lane with
// want set appends nch items (v, 0), ..., (v, nch-1).  One atomic per warp.
__device__ __forceinline__ void warp_push(bool want, int v, int nch, int* fv, int* fc, int* counter, int cap,
                                          Ctl* ctl) {
  const int lane = threadIdx.x & 31;
  const int cnt = want ? nch : 0;
  int inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  const int total = __shfl_sync(0xffffffffu, inc, 31);
  if (total == 0) return;
  int base = 0;
  if (lane == 31) base = atomicAdd(counter, total);
  base = __shfl_sync(0xffffffffu, base, 31);
  if (base + total > cap) {
    if (lane == 0) set_err(ctl, PR_EINTERNAL, 50);
    return;
  }
  const int pos = base + inc - cnt;
  for (int j = 0; j < cnt; j++) {
    fv[pos + j] = v;
    fc[pos + j] = j;
  }
}

// ---------------------------------------------------------------------------
// stream-ordered device buffers
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

class Arena {
 public:
  explicit Arena(cudaStream_t s) : s_(s) {}
  ~Arena() { release(); }
  template <typename T>
  pr_status alloc(T** out, size_t count) {
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    if (fault_hit(kFaultAlloc)) {
      *out = nullptr;
      return PR_ENOMEM;
    }
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, s_);
    if (e != cudaSuccess) {
      set_last_cuda_error(e);
      *out = nullptr;
      return PR_ENOMEM;
    }
    bufs_.push_back(p);
    *out = static_cast<T*>(p);
    return PR_OK;
  }
  void release() {
    for (void* p : bufs_) cudaFreeAsync(p, s_);
    bufs_.clear();
  }
  cudaStream_t stream() const { return s_; }

 private:
  cudaStream_t s_;
  std::vector<void*> bufs_;
};

// Zero a control block and set the wait limit of this process
// (pr_set_wait_limit) in it; only launches and memsets, so it can be captured.
pr_status init_ctl(Ctl* ctl, cudaStream_t s);
// the limit of pr_set_wait_limit in microseconds (0: the default kWaitNs)
unsigned int wait_limit_us();

// zero the barrier counter and the frontier counters (not the error word)
// before a persistent launch
inline pr_status reset_ctl(Ctl* ctl, cudaStream_t s) {
  PRGB_CUDA(cudaMemsetAsync(&ctl->bar_count, 0, sizeof(unsigned int), s));
  PRGB_CUDA(cudaMemsetAsync(ctl->cnt, 0, sizeof(ctl->cnt), s));
  return PR_OK;
}

// number of SMs of the current device (cached per device)
int num_sms();
// L2 cache size of the current device in bytes (cached per device)
int64_t l2_bytes();

// cooperative launch with as many co-resident blocks as fit (capped per SM)
pr_status launch_coop(const void* kernel, int block, size_t smem, cudaStream_t s, void** args,
                      int max_per_sm, int* grid_out);

// ---------------------------------------------------------------------------
// primitives (prims.cu)
// ---------------------------------------------------------------------------
// out[0] = 0, out[i+1] = in[0] + ... + in[i]  (out has n+1 entries)
pr_status scan_i32(const int32_t* in, int32_t* out, int64_t n, Arena& a);
pr_status scan_u8(const uint8_t* in, int32_t* out, int64_t n, Arena& a);
// Stable LSD radix sort of (key, val) pairs on the low key_bits bits of key.
// Result is left in keys/vals; keys_tmp/vals_tmp are scratch of n entries.
pr_status radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                           int64_t n, int key_bits, Arena& a);
int bits_for(uint32_t max_value);
pr_status iota_u32(uint32_t* out, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------------------
// loop-free device graph
// ---------------------------------------------------------------------------
struct DevGraph {
  int32_t n = 0;
  int64_t m = 0;            // loop-free edges
  int32_t* optr = nullptr;  // [n+1] out-edges, targets ascending
  int32_t* oidx = nullptr;  // [m]
  int32_t* iptr = nullptr;  // [n+1] in-edges, sources ascending
  int32_t* iidx = nullptr;  // [m]
  int32_t* outdeg = nullptr;  // [n]
  // rows of the CSC with more in-edges than the SpMV chunk (see spmv.cuh)
  int32_t* heavy_rows = nullptr;
  int32_t* heavy_choff = nullptr;
  int32_t* heavy_chrow = nullptr;
  int32_t nheavy = 0, nchunks = 0;
  int32_t* lorder = nullptr;  // [n] rows ordered by in-degree class (heavy last)
  int32_t* lpre = nullptr;    // [n+1] row-cost prefix over lorder (see build_lpre), or null
  int32_t* oheavy = nullptr;  // vertices with more than kHeavy out-edges (ascending)
  int32_t* ochoff = nullptr;  // their kChunkH-edge chunks: first chunk per listed vertex
  int32_t* ochrow = nullptr;  // per chunk, its index in oheavy
  int32_t noheavy = 0, nochunks = 0;
  double* inv = nullptr;      // [n] 1/outdeg, 0 for dangling vertices
};

// Rows [0, nrows) of ptr ordered by (group[row], in-degree class), stable
// (group may be null).  Used to give the 32 rows of a warp similar lengths.
pr_status build_lorder(const int32_t* ptr, int32_t nrows, const int32_t* group, int32_t group_max, Arena& keep,
                       Arena& tmp, int32_t** lorder);
// Prefix of the row costs (in-degree + kRowCost) in lorder order:
// lpre[i] = cost of rows lorder[0..i).  Used to give each warp of a sweep
// an equal share of edges.  Left null when it would not fit in int32.
constexpr int kRowCost = 8;
pr_status build_lpre(const int32_t* ptr, const int32_t* lorder, int32_t n, int64_t m, Arena& keep, Arena& tmp,
                     int32_t** lpre);
// inv[i] = 1/deg[i] (0 where deg is 0)
pr_status build_inv(const int32_t* deg, int32_t n, Arena& keep, double** inv, cudaStream_t s);

// List the rows r in [0, nrows) of ptr with ptr[r+1]-ptr[r] > kHeavy
// (ascending), their chunk offsets (exclusive prefix of ceil(deg/kChunkH))
// and, per chunk, its heavy-row index; reads the two counts back
// (synchronises).
pr_status build_heavy(const int32_t* ptr, int32_t nrows, Arena& keep, Arena& tmp, int32_t** rows,
                      int32_t** choff, int32_t** chrow, int32_t* nheavy, int32_t* nchunks);

// fx_sched.cu: the conflict-free slices of the fixed-point series (after
// the layout).
pr_status build_fx_sched(pr_partition_s* P, Arena& tmp, Ctl* ctl);

// ingest.cu: validate the CSR, drop loops, build out- and in-adjacency.
// Buffers of g are allocated from `keep`; scratch from `tmp`.
pr_status ingest(const pr_csr* csr, uint32_t flags, DevGraph* g, Arena& keep, Arena& tmp, Ctl* ctl);

// scc.cu: rep[v] = representative (largest vertex id) of v's SCC.
// ev (may be null): events recorded after the trim and after the giant SCC's
// forward-backward search; *rounds (may be null): colouring rounds run
pr_status scc_detect(const DevGraph& g, int32_t* rep, Arena& tmp, Ctl* ctl, cudaEvent_t* ev = nullptr,
                     int32_t* rounds = nullptr);

// levels.cu: levels, merge flags and CAC grouping (Theorem 3.1 restated
// per condensation node).  Outputs per vertex: crep (smallest vertex of the
// final component), level, type (PR_TYPE_*), wave (longest path to a sink
// in the condensation, counted in nodes).
pr_status levels_and_merge(const DevGraph& g, const int32_t* rep, int32_t* crep, int32_t* level,
                           uint8_t* type, int32_t* wave, int32_t* max_wave, Arena& tmp, Ctl* ctl);

// large components: solved by grid-wide cooperative kernels
struct LargeComp {
  int32_t c;       // canonical component id
  int32_t off;     // first permuted vertex
  int32_t size;
  int32_t type;
  int32_t sub_begin, sub_end;  // sub-level range (CAC topological waves)
  int32_t level_idx;           // processing index of its level (0 = highest)
  int32_t m_int;               // internal in-edges
  int32_t m_ext;               // external in-edges
  int32_t heavy_begin, heavy_end;  // slice of the partition's heavy-row list
  int32_t chunk_begin, chunk_end;  // its chunk range
  // SCCs: the light rows [off, off + nlight) (the heavy ones follow) as
  // 32-row slices [sell_begin, sell_end) of the partition's SELL layout;
  // sell_end == sell_begin when the component has none
  int32_t nlight, sell_begin, sell_end;
};

// per level (in processing order): component ranges by class
//   [cbeg, clu) grid-wide, [clu, cta) one cluster of CTAs each, [cta, warp)
//   one CTA each, [warp, single) one warp each, [single, cend) 1-vertex
struct LevelRange {
  int32_t cbeg, clu, cta, warp, single, cend;
  int32_t clu_max;              // vertices of the largest cluster-class component
  // FP64 solves split the cluster class: [clu, big) stays on clusters,
  // [big, cta) (at most kFxMax vertices) goes to one 1024-thread CTA each;
  // big_max is the largest component of [big, cta) (host-side, set by
  // split_fx_ranges)
  int32_t big, big_max;
  int32_t vbeg, vsingle, vend;  // permuted vertex range of the level / its singletons
  // rows of the level with more than kHeavy external in-edges: a slice of
  // the partition's external heavy-row list, and its chunk range
  int32_t xh_begin, xh_end, xc_begin, xc_end;
};

constexpr int kWarpCompMax = 32;     // components of <= 32 vertices: one warp
constexpr int kCtaCompMax = 256;     // <= 256 vertices: one CTA
constexpr int kCluCompMax = 16384;   // <= 16384 vertices: one cluster of 8 CTAs
constexpr int kNumClasses = 5;       // grid-wide, cluster, CTA, warp, 1-vertex

struct SolvePlan;  // solve.cuh

}  // namespace prgb

// The opaque handles of the C ABI.
struct pr_graph_s {
  cudaStream_t stream = nullptr;
  prgb::Arena* keep = nullptr;  // owns the buffers of g
  prgb::DevGraph g;
};

struct pr_partition_s {
  cudaStream_t stream = nullptr;
  prgb::Arena* keep = nullptr;   // owns every device buffer below
  prgb::DevGraph g;
  int32_t n_comp = 0, n_levels = 0, n_scc = 0, n_scc_vertices = 0;
  // per original vertex
  int32_t* comp_id = nullptr;
  uint8_t* type = nullptr;
  int32_t* level = nullptr;
  // permuted layout (p = permuted position)
  int32_t* perm = nullptr;     // [n] p -> v
  int32_t* p_outdeg = nullptr; // [n]
  int32_t* int_ptr = nullptr;  // [n+1] internal in-edges (same component)
  int32_t* int_idx = nullptr;  //       permuted source positions
  int32_t* ext_ptr = nullptr;  // [n+1] external in-edges (higher levels)
  int32_t* ext_idx = nullptr;
  int32_t* c_off = nullptr;    // [K+1] component -> first permuted vertex
  int32_t* c_sub = nullptr;    // [K+1] component -> first sub-level
  int32_t* sub_ptr = nullptr;  // [S+1] sub-level -> first permuted vertex
  uint8_t* c_type = nullptr;   // [K]
  int32_t n_sub = 0;
  int64_t m_int = 0, m_ext = 0;
  int32_t max_large = 0;       // largest vertex count among large components
  int32_t* heavy_rows = nullptr;   // permuted rows with > kHeavy internal in-edges
  int32_t* heavy_choff = nullptr;
  int32_t* heavy_chrow = nullptr;
  int32_t* lorder = nullptr;       // [n] positions by (component, internal in-degree class)
  int32_t* lpre = nullptr;         // [n+1] row-cost prefix over lorder (internal in-degrees), or null
  double* p_inv = nullptr;         // [n] 1/outdeg by position
  int32_t* p_comp = nullptr;       // [n] component of each position
  int32_t* xheavy_rows = nullptr;  // positions with > kHeavy external in-edges
  int32_t* xheavy_choff = nullptr;
  int32_t* xheavy_chrow = nullptr;
  int32_t nxheavy = 0, nxchunks = 0;
  int32_t max_xheavy = 0, max_xchunks = 0;  // largest slice over the levels
  int32_t* xlorder = nullptr;      // [n] positions by (level, external in-degree class)
  int32_t nheavy = 0, nchunks = 0;
  int32_t max_heavy = 0, max_chunks = 0;  // largest slice over the large components
  // light rows of the grid-wide SCCs in SELL-32 form: slice s holds 32
  // consecutive rows, its k-th in-edges side by side at
  // sell_idx[sell_ptr[s] + 32 k + lane] (component-local sources; short rows
  // padded with the component's size, a slot that holds 0); sell_cpre is a
  // prefix of the slices' costs (width + 2) for balanced shares
  int32_t* sell_ptr = nullptr;
  int32_t* sell_idx = nullptr;
  int32_t* sell_cpre = nullptr;
  int32_t nsell = 0;
  // conflict-free slices of the SCCs of the fixed-point level kernel
  // (fx_sched.cu): per component the word offset of its slices in fxs_words
  // (-1: none, the kernel builds them), the index of its first warp in
  // fxs_wcnt; per warp its words a lane.  Null when no component has one.
  int32_t* fxs_ptr = nullptr;
  int32_t* fxs_wbase = nullptr;
  uint8_t* fxs_wcnt = nullptr;
  uint2* fxs_words = nullptr;
  // the sub-level wave of every vertex (longest path to a sink in the
  // condensation) and its maximum: with comp_id, type and level, all that
  // pr_partition_save writes
  int32_t* wave = nullptr;
  int32_t max_wave = 0;
  // PR_PARTITION_TIMING: phase times (pr_partition_timing order) and counts
  bool timed = false;
  float phase_ms[6] = {0, 0, 0, 0, 0, 0};
  int32_t colour_rounds = 0;
  int32_t waves[5][2] = {};
  std::vector<prgb::LevelRange> levels;  // host, processing order
  std::vector<int32_t> h_c_off;          // host copy of c_off [K+1]
  int32_t cta_max = prgb::kCtaCompMax;   // largest component of the one-CTA class (tunable)
  int32_t coop_blocks = 4;               // blocks per SM of the grid-wide solve kernels (tunable)
  int32_t balance = 1;                   // grid-wide sweeps share light rows by cost (tunable)
  std::vector<prgb::LargeComp> large;    // host
  prgb::SolvePlan* plan = nullptr;       // cached solve (graph), built on first use
  std::mutex plan_mu;                    // one call at a time uses the plan
};
