// Autotuners. The standalone likelihood kernel's split factor (warps per
// particle, sharing its bins by streams) is timed the same way on the
// caller's own call; its results do not depend on the split either.
//
// Autotuner for the persistent NUTS launch: the slot count (particles per
// CTA, i.e. the CTA's tile of particles) trades the FP64 cost of the per-
// particle phases, which warp 0 runs with one lane per slot, against the
// number of CTAs that fill the SMs. Which one wins depends on N, the segment
// lengths and the tree depths, so it is measured: each candidate runs the
// same trial mutation on copies of the caller's particles, timed with CUDA
// events on the launching stream. A NUTS result does not depend on the slot
// count, so tuning never changes what a run computes.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace sharpy {

constexpr int kSlotChoices[] = {4, 8, 16, 32};
constexpr int kNumSlotChoices = 4;
// Warps that share one particle's sweep in the standalone likelihood kernel
// (plus the staged kernel, choice 16, on long segments of the mixed path).
constexpr int kSplitChoices[] = {1, 2, 4, 8};
constexpr int kNumSplitChoices = 4;

struct TuneCandidate {
  int slots;
  float ms;
};

// trial(slots, stream) enqueues one trial launch. Each candidate runs once
// untimed (module loading and first-touch costs) and once timed.
template <class Trial>
int tune_slots(TuneCandidate* c, int nc, Trial&& trial, cudaStream_t s, int* best) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return SHARPY_ECUDA;
  }
  int rc = SHARPY_OK;
  int bi = 0;
  for (int i = 0; i < nc && !rc; ++i) {
    rc = trial(c[i].slots, s);
    if (!rc && cudaEventRecord(e0, s) != cudaSuccess) rc = SHARPY_ECUDA;
    if (!rc) rc = trial(c[i].slots, s);
    if (!rc && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&c[i].ms, e0, e1) != cudaSuccess))
      rc = SHARPY_ECUDA;
    if (!rc && c[i].ms < c[bi].ms) bi = i;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!rc) *best = c[bi].slots;
  return rc;
}

}  // namespace sharpy
