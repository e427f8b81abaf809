// global.cuh -- global power series and residual (global.cu).
#pragma once

#include "common.cuh"

namespace prgb {

struct GlobalArgs {
  int32_t n;
  const int32_t* iptr;
  const int32_t* iidx;
  const int32_t* outdeg;
  const double* u;
  double c, tol;
  int norm, max_iter, fixed;
  double* R;
  double* zA;
  double* zB;
  double* part;
  Ctl* ctl;
};

pr_status run_global(const DevGraph& g, double c, const double* u, double tol, int norm, int max_iter, int fixed,
                     double* R, int* iters, Arena& tmp, Ctl* ctl);

// number of block partials the residual kernel writes
int residual_grid();

// residual into out_dev (device double), using part[residual_grid()] scratch
pr_status run_residual(const DevGraph& g, double c, const double* u, const double* R, double* part, double* out_dev,
                       cudaStream_t s);

}  // namespace prgb
