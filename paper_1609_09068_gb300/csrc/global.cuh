// global.cuh -- global power series and residual (global.cu).
#pragma once

#include "common.cuh"
#include "spmv.cuh"

namespace prgb {

struct GlobalArgs {
  int32_t n;
  const int32_t* iptr;
  const int32_t* iidx;
  const int32_t* outdeg;
  const int32_t* lorder;
  const int32_t* lpre;  // row-cost prefix over lorder, or nullptr
  const double* inv;
  const double* civ;  // c / outdeg
  const double* u;
  double c, tol;
  int norm, max_iter, fixed;
  double* R;
  double* zA;
  double* zB;
  double* part;
  HeavyRows hv;
  HeavyScratch hs;
  Ctl* ctl;
};

// kernel_ms (nullable): device time of the power-series kernel (CUDA events)
pr_status run_global(const DevGraph& g, double c, const double* u, double tol, int norm, int max_iter, int fixed,
                     double* R, int* iters, Arena& tmp, Ctl* ctl, float* kernel_ms);

// number of block partials the residual kernel writes
int residual_grid();

// residual into out_dev (device double), using part[residual_grid()] and
// heavy-row scratch from tmp
pr_status run_residual(const DevGraph& g, double c, const double* u, const double* R, double* part, double* out_dev,
                       Arena& tmp);

}  // namespace prgb
