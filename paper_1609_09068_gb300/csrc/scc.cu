// scc.cu -- strongly connected components (Def. 3.1) on the device.
//
// The paper finds SCCs with a Tarjan DFS (Sec. 4.1), which is sequential.
// Here: (1) trim -- repeatedly remove vertices with no remaining in- or
// out-edge; each is a 1-vertex SCC (it lies on no cycle, Sec. 3 remark on
// 1-vertex SCCs); (2) forward-backward reachability from the best-connected
// vertex, which takes out the giant SCC; (3) colouring rounds on what is
// left: every vertex gets colour(v) = largest id that reaches it inside its
// piece.  A vertex r with colour(r) == r is a root: the vertices of colour r
// from which r is reachable (a backward search from every root at once,
// staying inside the root's colour) are exactly r's SCC, and r is its
// largest id.  Two vertices of one SCC have the same ancestors, hence the
// same colour, so the colours become the pieces of the next round.  Every
// round settles at least the SCC of each piece's largest vertex.
//
// Result: rep[v] = largest vertex id of v's SCC.
#include "common.cuh"
#include "waves.cuh"

namespace prgb {

__device__ __forceinline__ int gwarp() { return (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); }
__device__ __forceinline__ int nwarps() { return (int)(((int64_t)gridDim.x * blockDim.x) >> 5); }

constexpr int kChunkE = 32;  // edges per frontier item: one 32-lane pass of a warp

__device__ __forceinline__ int nchunks_of(int d) { return (d + kChunkE - 1) / kChunkE; }

// ---- trim: Kahn peeling in both directions, one persistent launch ---------
// Items are (vertex, chunk): chunks [0, co) cover the out-edges and
// [co, co + ci) the in-edges, kChunkE edges each.
__device__ __forceinline__ int trim_chunks(const int32_t* optr, const int32_t* iptr, int v) {
  const int n = nchunks_of(optr[v + 1] - optr[v]) + nchunks_of(iptr[v + 1] - iptr[v]);
  return n > 0 ? n : 1;
}

struct TrimK {
  const int32_t *optr, *oidx, *iptr, *iidx;
  int32_t *rem_out, *rem_in, *state, *rep;
  __device__ void range(int v, int j, int* e0, int* e1) const {
    const int co = nchunks_of(optr[v + 1] - optr[v]);
    if (j < co) {
      *e0 = optr[v] + j * kChunkE;
      *e1 = min(optr[v + 1], *e0 + kChunkE);
    } else {
      *e0 = iptr[v] + (j - co) * kChunkE;
      *e1 = min(iptr[v + 1], *e0 + kChunkE);
    }
  }
  __device__ int4 pre(int v, int j, bool first) const {
    if (j == 0 && first) rep[v] = v;
    return make_int4(j < nchunks_of(optr[v + 1] - optr[v]) ? 1 : 0, 0, 0, 0);
  }
  __device__ bool edge(int e, int4 p, int, int* w, int* nch) const {
    const bool out = p.x != 0;
    *w = out ? oidx[e] : iidx[e];
    int32_t* rem = out ? rem_in : rem_out;
    if (atomicSub(&rem[*w], 1) == 1 && atomicCAS(&state[*w], 0, 1) == 0) {
      *nch = trim_chunks(optr, iptr, *w);
      return true;
    }
    return false;
  }
};

__global__ void trim_k(const int32_t* __restrict__ optr, const int32_t* __restrict__ oidx,
                       const int32_t* __restrict__ iptr, const int32_t* __restrict__ iidx, int32_t n,
                       int32_t* rem_out, int32_t* rem_in, int32_t* state, int32_t* rep, int* fav, int* fac,
                       int* fbv, int* fbc, int cap, Ctl* ctl) {
  const int lane = threadIdx.x & 31;
  const int gw = gwarp(), nw = nwarps();
  for (int64_t vb = (int64_t)gw * 32; vb < n; vb += (int64_t)nw * 32) {
    const int64_t v = vb + lane;
    bool want = false;
    if (v < n) {
      const int ro = optr[v + 1] - optr[v], ri = iptr[v + 1] - iptr[v];
      rem_out[v] = ro;
      rem_in[v] = ri;
      rep[v] = -1;
      want = (ro == 0 || ri == 0);
      state[v] = want ? 1 : 0;
    }
    warp_push(want, (int)v, want ? trim_chunks(optr, iptr, (int)v) : 0, fav, fac, &ctl->cnt[0], cap, ctl);
  }
  const Frontier f{fav, fac, fbv, fbc, cap};
  TrimK k{optr, oidx, iptr, iidx, rem_out, rem_in, state, rep};
  run_waves(ctl, f, 101, kWaveTrim, k);
}

// ---- max-label propagation inside the pieces, frontier driven ---------------
// Along out-edges: sig(v) = largest id that reaches v through unsettled
// vertices of v's piece (piece: pin, the colour of the round before, -2 / -1
// for the giant's forward set / the rest in the first round, kSettled once
// the vertex's SCC is known).  Frontier items are (vertex, chunk of kChunkE
// edges), so the adjacency of a hub is spread over many warps.
constexpr int32_t kSettled = INT32_MIN;

struct PropK {
  const int32_t *ptr, *idx, *pin;
  int32_t *sig, *stamp;
  __device__ void range(int u, int j, int* e0, int* e1) const {
    *e0 = ptr[u] + j * kChunkE;
    *e1 = min(ptr[u + 1], *e0 + kChunkE);
  }
  __device__ int4 pre(int u, int, bool) const { return make_int4(vload(&sig[u]), pin[u], 0, 0); }
  __device__ bool edge(int e, int4 p, int wave, int* w, int* nch) const {
    *w = idx[e];
    const int x = *w;
    // both loads in flight at once (a short-circuit test would serialise
    // them); a settled target's piece is kSettled, never a live one's
    const int px = pin[x], sx = vload(&sig[x]);
    if ((px != p.y) | (sx >= p.x)) return false;
    const int old = atomicMax(&sig[x], p.x);
    if (old < p.x && atomicExch(&stamp[x], wave) != wave) {
      *nch = nchunks_of(ptr[x + 1] - ptr[x]);
      return *nch > 0;
    }
    return false;
  }
};

// first frontier of a propagation: every live vertex with out-edges, its
// own id as its label
__device__ __forceinline__ void prop_init(const int32_t* __restrict__ ptr, int32_t n, const int32_t* __restrict__ rep,
                                          int32_t* sig, int32_t* stamp, int* fav, int* fac, int cap, Ctl* ctl) {
  const int lane = threadIdx.x & 31;
  const int gw = gwarp(), nw = nwarps();
  for (int64_t vb = (int64_t)gw * 32; vb < n; vb += (int64_t)nw * 32) {
    const int64_t v = vb + lane;
    bool want = false;
    int nch = 0;
    if (v < n) {
      stamp[v] = -1;
      // a settled vertex's colour is -1: it matches no root in the search
      const bool live = rep[v] < 0;
      sig[v] = live ? (int32_t)v : -1;
      if (live) {
        nch = nchunks_of(ptr[v + 1] - ptr[v]);
        want = nch > 0;
      }
    }
    warp_push(want, (int)v, nch, fav, fac, &ctl->cnt[0], cap, ctl);
  }
}

// ---- backward search from every colour root --------------------------------
// From each root r (colour(r) == r) along in-edges, entering only unsettled
// vertices of the same colour (a settled vertex's colour is -1): they reach r
// and r reaches them.
struct RootBfsK {
  const int32_t *ptr, *idx, *color;
  int32_t* mark;
  int tag;
  __device__ void range(int u, int j, int* e0, int* e1) const {
    *e0 = ptr[u] + j * kChunkE;
    *e1 = min(ptr[u + 1], *e0 + kChunkE);
  }
  __device__ int4 pre(int v, int, bool) const { return make_int4(color[v], 0, 0, 0); }
  __device__ bool edge(int e, int4 p, int, int* w, int* nch) const {
    *w = idx[e];
    const int x = *w;
    const int cx = color[x], mx = vload(&mark[x]);
    if ((cx != p.x) | (mx == tag) || atomicExch(&mark[x], tag) == tag) return false;
    *nch = nchunks_of(ptr[x + 1] - ptr[x]);
    return *nch > 0;
  }
};

// first frontier of the backward search: the roots (colour(r) == r)
__device__ __forceinline__ void root_init(const int32_t* __restrict__ ptr, int32_t n, const int32_t* __restrict__ rep,
                                          const int32_t* __restrict__ color, int32_t* mark, int tag, int* fav,
                                          int* fac, int cap, Ctl* ctl) {
  const int lane = threadIdx.x & 31;
  const int gw = gwarp(), nw = nwarps();
  for (int64_t vb = (int64_t)gw * 32; vb < n; vb += (int64_t)nw * 32) {
    const int64_t v = vb + lane;
    bool want = false;
    int nch = 0;
    if (v < n && rep[v] < 0 && color[v] == (int32_t)v) {
      mark[v] = tag;
      nch = nchunks_of(ptr[v + 1] - ptr[v]);
      want = nch > 0;
    }
    warp_push(want, (int)v, nch, fav, fac, &ctl->cnt[0], cap, ctl);
  }
}

// settle what the search reached (its colour's largest id is the SCC's
// representative); the colours become the next pieces; the vertices left
// are counted into *left
__device__ __forceinline__ void assign_color(int32_t n, int32_t* rep, int32_t* pin, const int32_t* color,
                                             const int32_t* mark, int tag, int* left_ctr) {
  int left = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (rep[v] >= 0) continue;
    if (mark[v] == tag) {
      rep[v] = color[v];
      pin[v] = kSettled;
    } else {
      pin[v] = color[v];
      left++;
    }
  }
  left = __reduce_add_sync(0xffffffffu, left);
  if ((threadIdx.x & 31) == 0 && left) atomicAdd(left_ctr, left);
}

// Between two phases of the fused colouring kernel: every block has left
// the previous phase's waves before block 0 clears the frontier counters
// (and the vertex counter of the next round), and the next phase pushes
// only after that.
__device__ __forceinline__ bool phase_reset(Ctl* ctl, int where, int next_left) {
  if (!grid_sync(ctl, where)) return false;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->cnt[0] = 0;
    ctl->cnt[1] = 0;
    ctl->cnt[2] = 0;
    if (next_left >= 0) ctl->cnt[next_left] = 0;
  }
  return grid_sync(ctl, where + 1);
}

// All colouring rounds in one cooperative launch: per round the forward
// label propagation, the backward search from the roots and the settling
// pass, separated by grid barriers instead of host round trips.  Round r
// counts the vertices still unsettled into cnt[6 + (r & 1)] (the other slot
// is cleared for the next round after every block has read it); the
// number of rounds run goes to cnt[5].
__global__ void colour_k(const int32_t* __restrict__ optr, const int32_t* __restrict__ oidx,
                         const int32_t* __restrict__ iptr, const int32_t* __restrict__ iidx, int32_t n, int32_t* rep,
                         int32_t* pin, int32_t* sig, int32_t* stamp, int32_t* mark, int* fav, int* fac, int* fbv,
                         int* fbc, int cap, Ctl* ctl) {
  const Frontier f{fav, fac, fbv, fbc, cap};
  for (int round = 0; round < 20000; round++) {
    const int tag = round + 1;
    const int slot = 6 + (round & 1);
    prop_init(optr, n, rep, sig, stamp, fav, fac, cap, ctl);
    if (!run_waves(ctl, f, 111, kWaveProp, PropK{optr, oidx, pin, sig, stamp})) return;
    if (!phase_reset(ctl, 141, 6 + ((round + 1) & 1))) return;
    root_init(iptr, n, rep, sig, mark, tag, fav, fac, cap, ctl);
    if (!run_waves(ctl, f, 131, kWaveRoot, RootBfsK{iptr, iidx, sig, mark, tag})) return;
    assign_color(n, rep, pin, sig, mark, tag, &ctl->cnt[slot]);
    if (!phase_reset(ctl, 151, -1)) return;
    if (vload(&ctl->cnt[slot]) == 0) {
      if (blockIdx.x == 0 && threadIdx.x == 0) ctl->cnt[5] = round + 1;
      return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) set_err(ctl, PR_EINTERNAL, 160);
}

// ---- FW-BW for the largest SCC ---------------------------------------------
// pivot: the unassigned vertex with the largest in-degree x out-degree
__global__ void pivot_k(const int32_t* __restrict__ optr, const int32_t* __restrict__ iptr, int32_t n,
                        const int32_t* __restrict__ rep, unsigned long long* best) {
  unsigned long long loc = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (rep[v] >= 0) continue;
    const long long p = (long long)(optr[v + 1] - optr[v]) * (long long)(iptr[v + 1] - iptr[v]);
    const unsigned long long key = ((unsigned long long)(p > 0x7fffffffLL ? 0x7fffffffLL : p) << 32) |
                                   (unsigned long long)(uint32_t)v;
    loc = key > loc ? key : loc;
  }
  // one atomic per warp: a grid of single-address atomics would serialise
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, loc, o);
    loc = t > loc ? t : loc;
  }
  if ((threadIdx.x & 31) == 0 && loc) atomicMax(best, loc);
}

struct ReachK {
  const int32_t *ptr, *idx, *rep;
  int32_t* mark;
  int tag;
  const int32_t* need;
  int tag_need;
  __device__ void range(int u, int j, int* e0, int* e1) const {
    *e0 = ptr[u] + j * kChunkE;
    *e1 = min(ptr[u + 1], *e0 + kChunkE);
  }
  __device__ int4 pre(int, int, bool) const { return make_int4(0, 0, 0, 0); }
  __device__ bool edge(int e, int4, int, int* w, int* nch) const {
    *w = idx[e];
    const int x = *w;
    const int rx = rep[x], nx = need != nullptr ? need[x] : tag_need, mx = vload(&mark[x]);
    if ((rx >= 0) | (nx != tag_need) | (mx == tag) || atomicExch(&mark[x], tag) == tag) return false;
    *nch = nchunks_of(ptr[x + 1] - ptr[x]);
    return *nch > 0;
  }
};

// Reachability from pivot among unassigned vertices: mark[v] = tag for every
// vertex reached along (ptr, idx); when need is set, only vertices with
// need[v] == tag_need are entered (the backward pass stays inside the
// forward set).
__global__ void reach_k(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx, int32_t n,
                        const unsigned long long* __restrict__ best,
                        const int32_t* __restrict__ rep, int32_t* mark, int tag, const int32_t* __restrict__ need,
                        int tag_need, int* fav, int* fac, int* fbv, int* fbc, int cap, Ctl* ctl) {
  const int lane = threadIdx.x & 31;
  const int gw = gwarp(), nw = nwarps();
  // the pivot (pivot_k's key: its low word; none when the key is 0)
  const unsigned long long key = *best;
  const int pivot = (int)(uint32_t)(key & 0xffffffffu);
  if (gw == 0 && key != 0 && pivot < n) {
    const int nch = nchunks_of(ptr[pivot + 1] - ptr[pivot]);
    if (lane == 0) mark[pivot] = tag;
    warp_push(lane == 0 && nch > 0, pivot, nch, fav, fac, &ctl->cnt[0], cap, ctl);
  }
  const Frontier f{fav, fac, fbv, fbc, cap};
  ReachK k{ptr, idx, rep, mark, tag, need, tag_need};
  run_waves(ctl, f, 121, kWaveReach, k);
}

// the SCC of the pivot is F and B: find its largest id, then assign it and
// split the rest into "in F" / "not in F" pieces for the signature rounds
__global__ void fwbw_max_k(int32_t n, const int32_t* fw, const int32_t* bw, int* best) {
  int loc = -1;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (fw[v] == 1 && bw[v] == 2) loc = (int)v;
  loc = __reduce_max_sync(0xffffffffu, loc);
  if ((threadIdx.x & 31) == 0 && loc >= 0) atomicMax(best, loc);
}

// also gives every vertex settled so far (trimmed or in the giant) the
// piece kSettled
__global__ void fwbw_assign_k(int32_t n, const int32_t* fw, const int32_t* bw, const int* best, int32_t* rep,
                              int32_t* pin) {
  const int r = *best;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (rep[v] >= 0) {
      pin[v] = kSettled;
    } else if (fw[v] == 1 && bw[v] == 2) {
      rep[v] = r;
      pin[v] = kSettled;
    } else {
      pin[v] = fw[v] == 1 ? -2 : -1;
    }
  }
}

static unsigned grid_n(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  int64_t cap = (int64_t)num_sms() * 16;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

pr_status scc_detect(const DevGraph& g, int32_t* rep, Arena& tmp, Ctl* ctl, cudaEvent_t* ev, int32_t* rounds) {
  cudaStream_t s = tmp.stream();
  const int32_t n = g.n;
  if (n == 0) return PR_OK;
  int32_t *rem_out, *rem_in, *state, *sin, *pin, *stamp;
  int *fav, *fac, *fbv, *fbc;
  const int cap = (int)(2 * (int64_t)n + 2 * g.m / kChunkE + 2);
  PRGB_TRY(tmp.alloc(&fav, cap));
  PRGB_TRY(tmp.alloc(&fac, cap));
  PRGB_TRY(tmp.alloc(&fbv, cap));
  PRGB_TRY(tmp.alloc(&fbc, cap));
  PRGB_TRY(tmp.alloc(&rem_out, n));
  PRGB_TRY(tmp.alloc(&rem_in, n));
  PRGB_TRY(tmp.alloc(&state, n));
  PRGB_TRY(tmp.alloc(&sin, n));
  PRGB_TRY(tmp.alloc(&pin, n));
  PRGB_TRY(tmp.alloc(&stamp, n));
  PRGB_CUDA(cudaMemsetAsync(pin, 0xff, (size_t)n * 4, s));
  PRGB_TRY(init_ctl(ctl, s));
  {
    DevGraph gg = g;
    int32_t nn = n;
    int cp = cap;
    void* args[] = {&gg.optr, &gg.oidx, &gg.iptr, &gg.iidx, &nn, &rem_out, &rem_in, &state, &rep,
                    &fav, &fac, &fbv, &fbc, &cp, &ctl};
    PRGB_TRY(launch_coop((const void*)trim_k, kWaveBlock, 0, s, args, kWavePerSm, nullptr));
  }
  if (ev) PRGB_CUDA(cudaEventRecord(ev[0], s));
  // FW-BW from the best-connected unassigned vertex takes out the giant SCC
  {
    unsigned long long* best;
    int* bmax;
    int32_t *fw, *bw;
    PRGB_TRY(tmp.alloc(&best, 1));
    PRGB_TRY(tmp.alloc(&bmax, 1));
    PRGB_TRY(tmp.alloc(&fw, n));
    PRGB_TRY(tmp.alloc(&bw, n));
    PRGB_CUDA(cudaMemsetAsync(best, 0, 8, s));
    PRGB_CUDA(cudaMemsetAsync(bmax, 0xff, 4, s));
    PRGB_CUDA(cudaMemsetAsync(fw, 0, (size_t)n * 4, s));
    PRGB_CUDA(cudaMemsetAsync(bw, 0, (size_t)n * 4, s));
    pivot_k<<<grid_n(n), kBlock, 0, s>>>(g.optr, g.iptr, n, rep, best);
    PRGB_LAUNCH();
    // the searches read the pivot on the device (none: they visit nothing
    // and every vertex keeps its piece), so no round trip is needed
    {
      int32_t nn = n;
      int cp = cap;
      for (int dir = 0; dir < 2; dir++) {
        PRGB_TRY(reset_ctl(ctl, s));
        const int32_t* ptr = dir == 0 ? g.optr : g.iptr;
        const int32_t* idx = dir == 0 ? g.oidx : g.iidx;
        int32_t* mark = dir == 0 ? fw : bw;
        int tag = dir == 0 ? 1 : 2;
        const int32_t* need = dir == 0 ? nullptr : fw;
        int tag_need = 1;
        void* args[] = {&ptr, &idx, &nn, &best, &rep, &mark, &tag, &need, &tag_need, &fav, &fac, &fbv, &fbc, &cp,
                        &ctl};
        PRGB_TRY(launch_coop((const void*)reach_k, kWaveBlock, 0, s, args, kWavePerSm, nullptr));
      }
      fwbw_max_k<<<grid_n(n), kBlock, 0, s>>>(n, fw, bw, bmax);
      PRGB_LAUNCH();
      fwbw_assign_k<<<grid_n(n), kBlock, 0, s>>>(n, fw, bw, bmax, rep, pin);
      PRGB_LAUNCH();
    }
  }
  if (ev) PRGB_CUDA(cudaEventRecord(ev[1], s));
  int32_t* mark;
  PRGB_TRY(tmp.alloc(&mark, n));
  PRGB_CUDA(cudaMemsetAsync(mark, 0, (size_t)n * 4, s));
  {
    PRGB_TRY(reset_ctl(ctl, s));
    int32_t nn = n;
    int cp = cap;
    DevGraph gg = g;
    void* args[] = {&gg.optr, &gg.oidx, &gg.iptr, &gg.iidx, &nn, &rep, &pin, &sin, &stamp, &mark,
                    &fav, &fac, &fbv, &fbc, &cp, &ctl};
    PRGB_TRY(launch_coop((const void*)colour_k, kWaveBlock, 0, s, args, kWavePerSm, nullptr));
  }
  int h[2] = {0, 0};
  PRGB_CUDA(cudaMemcpyAsync(&h[0], &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaMemcpyAsync(&h[1], &ctl->cnt[5], sizeof(int), cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  if (rounds) *rounds = h[1];
  return (pr_status)h[0];
}

}  // namespace prgb
