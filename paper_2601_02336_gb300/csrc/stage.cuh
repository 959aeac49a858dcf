// SMC stage kernels shared by the single-event calls and the batched driver:
// tempering root + weights + evidence (one thread-block cluster per event),
// weighted covariance, integer systematic resampling and gather.
#pragma once
#include "context.cuh"

namespace sharpy {

constexpr int kRwCluster = 8;    // CTAs per event in the reweight kernel (one cluster)
constexpr int kRwThreads = 256;  // threads per CTA
constexpr int64_t kMaxParticles = (int64_t)1 << 20;

// One event's stage: particles, scratch, outputs and (batched driver only)
// control words.
struct StageArgs {
  int64_t n;
  int D;
  double* theta;                // [n][D] particles (resampled in place)
  double* lnl;                  // [n]
  double* grad;                 // [n][D] or null
  const double* beta_prev_ptr;  // device beta, or null: beta_prev
  double beta_prev;
  double alpha;
  double* w;                    // [n] out: W_i = e^{db (lnL_i - max)}; FP32 scratch during the root search
  unsigned long long* csum;     // [n] out: inclusive prefix sums of floor(W_i 2^32)
  int32_t* anc;                 // [n] out: ancestors
  double* th0;                  // [n][D], [n][D], [n]: copies the gather reads from
  double* g0;
  double* l0;
  double* beta_next;            // device scalars out
  double* dlnz;
  double* ess;
  double* sum_w;                // sum of W (for the covariance)
  double* cov;                  // [D][D] out, or null
  double* lnz_acc;              // [2] ln Z and stage count, or null
  double* beta_state;           // set to beta_next, or null
  int* status;
  // batched driver only (null otherwise): the event runs a stage while
  // *active != 0; *stage counts its stages and names their random numbers
  int* active;
  int* stage;
  int max_stages;
  uint64_t key;
};

// Enqueue the kernels of one stage: tempering root, weights and evidence
// increment; the weighted covariance (if one.cov / the events' cov is set and
// cov is true); the resampling and the gather (if gather). `batch` null: one
// event described by `one`, resampled with the uniform U / 2^32. Otherwise
// `batch` is a device array of n_events descriptors (max_n: the largest n,
// max_d: the largest D) whose uniforms come from (key, stage) on the device;
// events that are not active are skipped.
int enqueue_stage_kernels(const StageArgs& one, const StageArgs* batch, int n_events, int64_t max_n, int max_d,
                          bool cov, bool gather, unsigned long long U, cudaStream_t s);

}  // namespace sharpy
