// waves.cuh -- frontier waves inside one cooperative launch, shared by the
// partitioner's kernels (trim, reachability, label propagation, Kahn order).
//
// A frontier item is (vertex, chunk of its adjacency).  A large frontier is
// processed by the whole grid, one bounded grid barrier per wave.  Once the
// frontier holds fewer than kSmallFrontier items, block 0 runs the next
// waves alone with block barriers while the other blocks wait at the grid
// barrier; it joins them again when the frontier grows, empties, or after
// kLocalWaves waves (well inside the barrier's time limit).  Long chains of
// tiny waves -- the common tail -- then cost a block barrier each instead of
// a grid barrier.
#pragma once

#include "common.cuh"

namespace prgb {

constexpr int kWaveBlock = 256;      // threads per block of the wave kernels
constexpr int kWavePerSm = 4;        // their co-resident blocks per SM (2 and 8: slower)
constexpr int kSmallFrontier = 64;
constexpr int kLocalWaves = 4096;

// which kernel runs the waves (the slot of Ctl::waves)
enum WaveKind { kWaveTrim = 0, kWaveProp = 1, kWaveReach = 2, kWaveRoot = 3, kWaveKahn = 4 };

struct Frontier {
  int* av;
  int* ac;
  int* bv;
  int* bc;
  int cap;
};

// Appends (w, 0..nch-1) to the next frontier; all 32 lanes call it.
struct Pusher {
  int* v;
  int* c;
  int* counter;
  int cap;
  Ctl* ctl;
  __device__ __forceinline__ void operator()(bool want, int w, int nch) const {
    warp_push(want, w, nch, v, c, counter, cap, ctl);
  }
};

// One wave.  Each warp takes `per` items, per = ceil(items / warps) capped
// at 32, so that every warp has work however small the frontier; they are
// strided by the number of warps, so that the consecutive chunks of a hub
// go to different warps.  A warp lays its items' edge ranges end to end
// (a prefix sum over the run, one item per lane) and walks the concatenation
// 32 edges at a time; each lane finds the item of its edge by a binary
// search over the prefix sums.  A warp thus keeps 32 edges' loads in flight
// whether its items have one edge each or hundreds.  The kernel supplies
//   K::range(v, j, &e0, &e1)      edges of item (v, j)
//   K::pre(v, j, first) -> int4   per-item data; called once per item with
//                                 first = true
//   K::edge(e, pre, wave, &w, &nch) -> bool   visit edge e; true pushes w
//                                 (with nch chunks) into the next frontier
template <class K>
__device__ __forceinline__ void one_wave(Ctl* ctl, const Frontier& f, int wave, int cnt, int w0, int nws,
                                         const K& k) {
  const int lane = threadIdx.x & 31;
  const int* cv = (wave & 1) ? f.bv : f.av;
  const int* cc = (wave & 1) ? f.bc : f.ac;
  Pusher push{(wave & 1) ? f.av : f.bv, (wave & 1) ? f.ac : f.bc, &ctl->cnt[(wave + 1) % 3], f.cap, ctl};
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->cnt[(wave + 2) % 3] = 0;
  const int per = min(32, max(1, (int)(((int64_t)cnt + nws - 1) / nws)));
  for (int64_t r0 = 0; r0 < cnt; r0 += (int64_t)nws * per) {
    const int64_t i = r0 + w0 + (int64_t)lane * nws;  // this lane's item
    int e0 = 0, d = 0;
    int4 pre = make_int4(0, 0, 0, 0);
    if (lane < per && i < cnt) {
      const int v = cv[i], j = cc[i];
      int e1 = 0;
      k.range(v, j, &e0, &e1);
      d = e1 - e0;
      pre = k.pre(v, j, true);
    }
    int incl = d;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int base = 0; base < total; base += 32) {
      const int q = base + lane;
      // it = number of items whose edges end at or before q
      int it = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1)
        if (__shfl_sync(0xffffffffu, incl, it + step - 1) <= q) it += step;
      const int ie0 = __shfl_sync(0xffffffffu, e0, it);
      const int ibeg = __shfl_sync(0xffffffffu, incl - d, it);
      const int4 ip = make_int4(__shfl_sync(0xffffffffu, pre.x, it), __shfl_sync(0xffffffffu, pre.y, it),
                                __shfl_sync(0xffffffffu, pre.z, it), __shfl_sync(0xffffffffu, pre.w, it));
      bool want = false;
      int w = 0, nch = 0;
      if (q < total) want = k.edge(ie0 + (q - ibeg), ip, wave, &w, &nch);
      push(want, w, want ? nch : 0);
    }
  }
}

// Grid barrier of the wave kernels (grid_arrive_wait), after which each
// block reads the next wave (next, or the wave block 0 left in flags[7] when
// next < 0) and its frontier size: the three frontier counters rotate, so the
// one read here is not written again before every block has passed the next
// barrier.
struct WaveState {
  int wave;
  int cnt;
};

__device__ __forceinline__ bool wave_barrier(Ctl* ctl, int where, int next, WaveState* out) {
  __shared__ int sh[3];
  __syncthreads();
  if (threadIdx.x == 0) {
    grid_arrive_wait(ctl, where);
    const int w = next >= 0 ? next : vload(&ctl->flags[7]);
    sh[0] = w;
    sh[1] = vload(&ctl->cnt[w % 3]);
    sh[2] = vload(&ctl->err);
  }
  __syncthreads();
  out->wave = sh[0];
  out->cnt = sh[1];
  return sh[2] == 0;
}

// Runs waves until the frontier is empty.  The caller has filled the first
// frontier (wave 0) into (av, ac), counting it in ctl->cnt[0]; this starts
// with the barrier that publishes it.  Returns false when a barrier failed.
template <class K>
__device__ bool run_waves(Ctl* ctl, const Frontier& f, int where, WaveKind kind, const K& item) {
  const int gw = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
  const int lw0 = threadIdx.x >> 5, lnw = blockDim.x >> 5;
  WaveState st;
  if (!wave_barrier(ctl, where, 0, &st)) return false;
  for (;;) {
    if (st.cnt == 0) return true;
    if (st.cnt >= kSmallFrontier) {
      if (blockIdx.x == 0 && threadIdx.x == 0) ctl->waves[kind][0]++;
      one_wave(ctl, f, st.wave, st.cnt, gw, nw, item);
      if (!wave_barrier(ctl, where, st.wave + 1, &st)) return false;
      continue;
    }
    // small frontier: block 0 alone, block barriers; the others wait below
    if (blockIdx.x == 0) {
      __shared__ int shc;
      int wave = st.wave, c = st.cnt;
      for (int k = 0; k < kLocalWaves; k++) {
        one_wave(ctl, f, wave, c, lw0, lnw, item);
        __syncthreads();
        wave++;
        if (threadIdx.x == 0) shc = atomicAdd(&ctl->cnt[wave % 3], 0);
        __syncthreads();
        c = shc;
        if (c == 0 || c >= kSmallFrontier) break;
      }
      if (threadIdx.x == 0) {
        ctl->waves[kind][1] += wave - st.wave;
        ctl->flags[7] = wave;
        __threadfence();
      }
    }
    if (!wave_barrier(ctl, where + 1, -1, &st)) return false;
  }
}

}  // namespace prgb
