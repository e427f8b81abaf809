// solve.cuh -- arguments of the level solver kernels (solve.cu).
#pragma once

#include "common.cuh"

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
  const float* p_invf;      // [n] 1/outdeg in FP32 (mixed precision only)
  int32_t* iters64;         // [K] FP64 residual sweeps per SCC (mixed only)
  double* W;                // [n] inflow-adjusted weights by position
  double* R;                // [n] by position
  double* zr;               // [n] R/outdeg by position
  int32_t* iters;           // [K]
  Ctl* ctl;
};

// CUDA events around the grid-wide power-series launches (opt-in timing)
struct KernelTiming {
  std::vector<cudaEvent_t> start, stop;
  std::vector<LargeComp> comps;
  ~KernelTiming() {
    for (cudaEvent_t e : start) cudaEventDestroy(e);
    for (cudaEvent_t e : stop) cudaEventDestroy(e);
  }
};

// Level-by-level solve of a partition.  u and R are device pointers in the
// original vertex order; replay (device, [K]) may be null; timing may be null.
// mixed: SCC series in FP32 with FP64 residual refinement (iters64 then
// receives the FP64 sweeps per component; it may be null otherwise).
pr_status run_solve(const pr_partition_s* P, double c, const double* u, double tol, int norm, int max_iter,
                    const int32_t* replay, bool mixed, double* R, int32_t* iters_dev, int32_t* iters64_dev,
                    Arena& tmp, Ctl* ctl, int64_t* launches, KernelTiming* timing);

// edges read by the solve; with iters64 (may be null), also the edges read
// by FP64 residual sweeps
pr_status solve_edge_visits(const pr_partition_s* P, const int32_t* iters_dev, const int32_t* iters64_dev,
                            int64_t* out, int64_t* out64, Arena& tmp);

}  // namespace prgb
