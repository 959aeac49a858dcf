// One precision's instantiations of the standalone likelihood kernel,
// compiled once per precision with -DSHARPY_LL_PREC so they build in parallel.
#include "loglike_kernel.cuh"

#ifndef SHARPY_LL_PREC
#error "compile with -DSHARPY_LL_PREC=<0|1|2>"
#endif

namespace sharpy {

#define SHARPY_LL_CAT2(a, b) a##b
#define SHARPY_LL_CAT(a, b) SHARPY_LL_CAT2(a, b)
cudaError_t SHARPY_LL_CAT(launch_ll_p, SHARPY_LL_PREC)(sharpy_ctx* c, bool grad, int split, int64_t n,
                                                       const double* th, double* lnl, double* g, cudaStream_t s) {
  return grad ? launch_ll_det<SHARPY_LL_PREC, true>(c, split, n, th, lnl, g, s)
              : launch_ll_det<SHARPY_LL_PREC, false>(c, split, n, th, lnl, g, s);
}

}  // namespace sharpy
