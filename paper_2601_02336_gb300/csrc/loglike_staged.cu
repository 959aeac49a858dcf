// The staged likelihood kernel's instantiations (mixed path, with and without
// the gradient, 1-3 detectors), compiled as a unit of their own so they build
// in parallel with the other kernels.
#include "loglike_kernel.cuh"

namespace sharpy {

cudaError_t launch_ll_staged_unit(sharpy_ctx* c, bool grad, int ndet, int64_t n, const double* th, double* lnl,
                                  double* g, cudaStream_t s) {
  switch (ndet) {
    case 1:
      return grad ? launch_ll_staged<true, 1, false>(c, n, th, lnl, g, s)
                  : launch_ll_staged<false, 1, false>(c, n, th, lnl, g, s);
    case 2:
      return grad ? launch_ll_staged<true, 2, false>(c, n, th, lnl, g, s)
                  : launch_ll_staged<false, 2, false>(c, n, th, lnl, g, s);
    default:
      return grad ? launch_ll_staged<true, 3, false>(c, n, th, lnl, g, s)
                  : launch_ll_staged<false, 3, false>(c, n, th, lnl, g, s);
  }
}

}  // namespace sharpy
