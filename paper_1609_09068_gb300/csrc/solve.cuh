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
pr_status run_solve(const pr_partition_s* P, double c, const double* u, double tol, int norm, int max_iter,
                    const int32_t* replay, double* R, int32_t* iters_dev, Arena& tmp, Ctl* ctl,
                    int64_t* launches, KernelTiming* timing);

pr_status solve_edge_visits(const pr_partition_s* P, const int32_t* iters_dev, int64_t* out, Arena& tmp);

}  // namespace prgb
