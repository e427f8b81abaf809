// solve.cuh -- arguments of the level solver kernels (solve.cu).
#pragma once

#include "common.cuh"
#include "fx128.cuh"
#include "mpnn.cuh"
#include "spmv.cuh"

namespace prgb {

struct SolveArgs {
  int32_t n;
  double c;
  double tol;
  int norm;
  int max_iter;
  const double* u;          // [n] original vertex order
  const int32_t* perm;      // [n] permuted position -> vertex
  const int32_t* p_outdeg;  // [n] loop-free out-degree by position
  const double* p_inv;      // [n] 1/outdeg by position (0 for dangling)
  const int32_t* lorder;    // [n] positions by (component, in-degree class)
  const int32_t* lpre;      // [n+1] row-cost prefix over lorder, or nullptr
  const int32_t* int_ptr;
  const int32_t* int_idx;
  const int32_t* ext_ptr;
  const int32_t* ext_idx;
  const int32_t* c_off;
  const int32_t* c_sub;
  const int32_t* sub_ptr;
  const uint8_t* c_type;
  const int32_t* replay;    // [K] fixed iteration counts, or nullptr
  const int32_t* xlorder;   // [n] positions by (level, external in-degree class)
  const double* R0;         // [n] warm-start guess by position for SCC rows, or nullptr
  const float* yhat;        // [n] the network's log-amplification by position: the level kernel forms its
                            //   own guess from it (FP64 warm start), or nullptr
  const double* civ;        // [n] c / outdeg by position (grid-wide series), or nullptr
  const int32_t* fxs_ptr;   // conflict-free slices of the fixed-point series (see pr_partition_s), or nullptr
  const int32_t* fxs_wbase;
  const uint8_t* fxs_wcnt;
  const uint2* fxs_words;
  const int32_t* sell_ptr;  // SELL-32 slices of the grid-wide SCCs' light rows (see pr_partition_s)
  const int32_t* sell_idx;
  const int32_t* sell_cpre;
  int lu_threshold;         // SCCs with fewer vertices are solved by dense elimination
  int32_t* iters64;         // [K] FP64 residual sweeps per SCC (mixed only)
  double* W;                // [n] inflow-adjusted weights by position
  double* R;                // [n] by position
  double* zr;               // [n] R/outdeg by position
  int32_t* iters;           // [K]
  Ctl* ctl;
};

// ---------------------------------------------------------------------------
// device helpers shared by the solve kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool keep_going(double s, double tau, int norm) {
  return norm == PR_NORM_LINF ? (s >= tau) : (s > tau);
}

// The warp and CTA kernels reduce the stopping norm in FP32: FP64 shuffles
// and adds cost more than the rows themselves on this part.  The FP32 sum
// of n non-negative terms is within n * 2^-24 of the FP64 one, so a relative
// margin of 1e-4 on the test keeps the FP64 norm at or below the threshold
// whenever the series stops (it may run one iteration longer than an exact
// test would).
// The test runs in FP32 against thr = tau / margin rounded down to a float
// (stop_thr32, once per component), so stopping still implies
// s * margin <= tau, and a sweep pays no FP64 instruction for it (GB300's
// FP64 pipe takes ~76 cycles to issue one warp instruction per
// sub-partition).
constexpr double kNormMargin = 1.0 + 1e-4;
__device__ __forceinline__ float stop_thr32(double tau) { return __double2float_rd(tau / kNormMargin); }
__device__ __forceinline__ bool keep_going32(float s, float thr, int norm) {
  return norm == PR_NORM_LINF ? (s >= thr) : (s > thr);
}

// The same test on integers, so that a warp reduces the norm with one
// redux.sync instead of a chain of shuffles: each lane's |term| becomes
// q = ceil(|term| * 2^20 / thr), capped at 2^21 (a lane at twice the
// threshold keeps the series going on its own).  Rounding up makes the sum
// of q an upper bound of the scaled FP32 norm, so stopping still implies
// norm <= thr; it may add one sweep when the norm ends within 2^-10 of
// thr.  At most 1,024 lanes of 2^21 sum below 2^32.
constexpr float kNormQOne = 1048576.0f;  // 2^20: thr in q units
constexpr float kNormQMax = 2097152.0f;  // 2^21
__device__ __forceinline__ float norm_q_scale(float thr) { return thr > 0.0f ? kNormQOne / thr : 0.0f; }
__device__ __forceinline__ unsigned norm_q(float pf, float scale) {
  if (!(pf > 0.0f)) return 0u;
  return scale > 0.0f ? __float2uint_ru(fminf(__fmul_ru(pf, scale), kNormQMax)) : (unsigned)kNormQMax;
}
__device__ __forceinline__ bool keep_going_q(unsigned s, int norm) {
  return norm == PR_NORM_LINF ? (s >= (unsigned)kNormQOne) : (s > (unsigned)kNormQOne);
}

// |x| as a float, from the bit pattern of the double: the sign dropped, the
// exponent rebiased from 1023 to 127 and the mantissa cut to 23 bits
// (rounding toward zero, relative error below 2^-23); magnitudes under the
// float range give 0, over it the largest float.  Integer operations only,
// so the stopping norm costs nothing on the FP64 pipe.
__device__ __forceinline__ float abs_to_float(double x) {
  const long long b = __double_as_longlong(x) & 0x7fffffffffffffffLL;
  const long long f = (b >> 29) - ((long long)(1023 - 127) << 23);
  if (f <= 0) return 0.0f;
  if (f >= 0x7f800000LL) return 3.4028235e38f;
  return __int_as_float((int)f);
}

// A local index outside [0, sz) would mean a broken layout: record it and
// read slot 0 instead of touching memory out of bounds.
__device__ __forceinline__ int local_or_err(const SolveArgs& a, int q, int sz) {
  if ((unsigned)q >= (unsigned)sz) {
    set_err(a.ctl, PR_EINTERNAL, 301);
    return 0;
  }
  return q;
}

__device__ __forceinline__ double check_u(const SolveArgs& a, double uu) {
  if (!(uu >= 0.0) || !isfinite(uu)) set_err(a.ctl, PR_EINVAL, 300);
  return uu;
}

// CUDA events around the grid-wide power-series launches (opt-in timing):
// one pair per large SCC of the partition, created before any capture
struct KernelTiming {
  std::vector<cudaEvent_t> start, stop;
  std::vector<LargeComp> comps;
  std::vector<cudaEvent_t> level;  // [n_levels + 1]: each level's start, then the end of the last
  bool levels = false;             // record the level events too (they cost a few microseconds a level);
                                   // ensure() creates them only then
  pr_status ensure(const pr_partition_s* P);
  ~KernelTiming();
};

// four non-blocking side streams and the fork / join events of a solve
constexpr int kSideStreams = 4;
struct SideStreams {
  cudaStream_t st[kSideStreams] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kSideStreams] = {nullptr, nullptr, nullptr, nullptr};
  int dev = 0;  // the device of the pooled handles
  pr_status create();
  ~SideStreams();
};

// scratch of the grid-wide fixed-point series (giant_fx.cu), sized for the
// partition's largest grid-wide SCC
struct GiantFxBufs {
  fx128* zA = nullptr;   // [max_large + 1] z = P c/outdeg, two sweeps alternating
  fx128* zB = nullptr;
  fx128* R = nullptr;    // [max_large] the running sum
  fx128* part = nullptr; // [max_chunks] heavy-row chunk partials
  int32_t* cnt = nullptr;  // [max_heavy] chunk arrivals, zero between launches
  unsigned long long* acc = nullptr;  // [4] norm slots of sweeps k % 3, then max W's bits; zeroed per launch
};

// work buffers of a solve, by permuted position
struct SolveBufs {
  double* R = nullptr;
  double* zr = nullptr;
  double* W = nullptr;
  HeavyScratch hs;
  double* civ = nullptr;  // c / outdeg (when there are grid-wide components)
  int32_t* lvl_ctr = nullptr;  // [4 * levels] claim counters of the level kernels
  GiantFxBufs gfx;             // FP64 mode's grid-wide SCC series (when there are grid-wide SCCs)
};

// one captured level loop and the parameters it was captured for
struct PlanGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t nodes = 0;  // kernels per replay
  double c = 0.0, tol = 0.0;
  int norm = 0, max_iter = 0;
  bool mixed = false;
  int timing = 0;  // 0 none, 1 the grid-wide kernels, 2 also the levels
  uint64_t warm_uid = 0;  // the warm-start network's id (0: none)
  int lu = 0;
  unsigned int wait_us = 0;  // the wait limit captured in the graph
  uint64_t last_use = 0;
};
constexpr int kPlanGraphs = 4;

// A partition's cached solve: its own buffers and the level loop captured
// as CUDA graphs, one per recent set of (c, tol, norm, max_iter, precision,
// timing, warm start).  Calls that use it are ordered on the device
// through `done`.
struct SolvePlan {
  Arena* keep = nullptr;
  SolveBufs b;
  SideStreams side;      // the directly launched solves
  SideStreams cap_side;  // the captures
  KernelTiming kt;
  cudaStream_t cs = nullptr;
  cudaEvent_t done = nullptr;
  int dev = 0;  // the device of the pooled cs and done
  std::vector<PlanGraph> graphs;
  uint64_t uses = 0;
  Ctl* ctl = nullptr;
  int32_t* iters = nullptr;
  int32_t* iters64 = nullptr;
  double* u = nullptr;
  double* Rout = nullptr;
  double* R0 = nullptr;             // [n] the warm-start guess by position (classes outside the level kernel)
  float* yhat = nullptr;            // [n] the network's output for this partition, by position
  uint64_t yhat_uid = 0, yhat_ver = 0;  // the model (and its weights' version) yhat was computed with
  MpnnInfer inf;
  ~SolvePlan();
};

// The exact fixed-point series of one grid-wide SCC (giant_fx.cu); a
// cooperative launch of kBlock-thread blocks.  g.acc must be zero at launch.
// Its sweep touches about kGiantFxRowBytes per row (z twice, R, z gathered).
constexpr int64_t kGiantFxRowBytes = 48;
// Whether its fixed-point sweep fits in half the L2 (else z is gathered as
// FP64 values)
bool giant_fits_l2(const LargeComp& L);
__global__ void solve_large_scc_fx_k(SolveArgs a, LargeComp L, GiantFxBufs g, HeavyRows hv);
// the same with z gathered as FP64 values (for an SCC whose 16-byte sweep
// does not fit in L2)
__global__ void solve_large_scc_fxd_k(SolveArgs a, LargeComp L, GiantFxBufs g, HeavyRows hv);

// Every component of a level with at most kFxMax vertices (SCCs by the
// exact fixed-point series, CACs by one FP64 pass) in one persistent launch
// of solve_fx.cu (solve_level_k), in FP64 and mixed precision alike; larger
// ones keep the cluster and grid-wide kernels.
constexpr int kFxMax = 1024;  // above it the 8-CTA clusters are faster (measured)
pr_status set_fx_attrs();
// the level's components [big, single) in one launch on s; ctr: three claim
// counters of this level, zero when the launch starts
pr_status launch_level(const SolveArgs& a, const LevelRange& r, int32_t* ctr, cudaStream_t s);
// host: every level's split of its cluster class at kFxMax (big, big_max)
void split_fx_ranges(pr_partition_s* P);

// Level-by-level solve of a partition with buffers of its own (used for
// replayed iteration counts).  u and R are device pointers in the original
// vertex order; replay (device, [K]) may be null; timing may be null.
// mixed: SCC series in FP32 with FP64 residual refinement (iters64 then
// receives the FP64 sweeps per component; it may be null otherwise).
// lu_threshold: SCCs of fewer vertices (at most 128) are solved by dense
// elimination (Sec. 4.3 item 3); 0 turns it off.
pr_status run_solve(const pr_partition_s* P, double c, const double* u, double tol, int norm, int max_iter,
                    const int32_t* replay, bool mixed, int lu_threshold, double* R, int32_t* iters_dev,
                    int32_t* iters64_dev, Arena& tmp, Ctl* ctl, int64_t* launches, KernelTiming* timing);

// The same through the partition's cached graph: copies u in, replays the
// graph, scatters R out (host or device pointers); *plan receives the plan,
// whose ctl / iters / iters64 / kt hold the call's results once the stream
// has reached them.  warm (may be null): the network that guesses each
// SCC's start, evaluated per level inside the graph.
pr_status plan_solve(pr_partition_s* P, double c, const double* u, bool u_on_host, double tol, int norm,
                     int max_iter, bool mixed, int timing, const pr_mpnn_s* warm, int lu, double* R,
                     bool R_on_host, cudaStream_t s, SolvePlan** plan, int64_t* launches);

// Autotuner (f-1): move the boundary between the one-CTA and the cluster
// classes of every level to cta_max (33..kCtaCompMax) and set the grid-wide
// kernels' blocks per SM; drops the partition's captured graphs.
// balance: 1 = the grid-wide sweeps share their light rows among warps by
// cost, 0 = in strided groups.
void retune_levels(pr_partition_s* P, int32_t cta_max, int32_t coop_blocks, int32_t balance);
// Times the captured solve for each candidate and keeps the fastest; the
// choice also becomes the default of partitions created later in the process.
pr_status tune_partition(pr_partition_s* P, double c, const double* u, double tol, cudaStream_t s,
                         int32_t* cta_max, int32_t* coop_blocks, int32_t* balance, float* best_ms);
// the process-wide tuned defaults (kCtaCompMax / 4 / 1 until a tuning ran)
void tuned_defaults(int32_t* cta_max, int32_t* coop_blocks, int32_t* balance);

// edges read by the solve; with iters64 (may be null), also the edges read
// by FP64 residual sweeps
pr_status solve_edge_visits(const pr_partition_s* P, const int32_t* iters_dev, const int32_t* iters64_dev,
                            int64_t* out, int64_t* out64, Arena& tmp);

}  // namespace prgb
