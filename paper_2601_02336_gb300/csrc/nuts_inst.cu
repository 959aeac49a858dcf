// One (precision, detector count) instantiation of the persistent NUTS kernel,
// compiled once per combination with -DSHARPY_NUTS_PREC and -DSHARPY_NUTS_NDET
// so the variants build in parallel.
#include "nuts_kernel.cuh"

#ifndef SHARPY_NUTS_PREC
#error "compile with -DSHARPY_NUTS_PREC=<0|1> -DSHARPY_NUTS_NDET=<1|2|3>"
#endif

namespace sharpy {

#define SHARPY_CAT2(a, b, c) a##b##_##c
#define SHARPY_CAT(a, b, c) SHARPY_CAT2(a, b, c)
int SHARPY_CAT(launch_nuts_p, SHARPY_NUTS_PREC, SHARPY_NUTS_NDET)(int slots, const NutsArgs& A, unsigned grid, cudaStream_t s) {
  return launch_nuts_impl<SHARPY_NUTS_PREC, SHARPY_NUTS_NDET>(slots, A, grid, s);
}

}  // namespace sharpy
