// The context structure and host-side helpers shared by the translation units.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

// Key of the likelihood call's tuned split factor.
struct LoglikeTuneKey {
  int64_t n_bins;
  int n_det;
  int64_t n;
  int precision, grad;
  bool operator==(const LoglikeTuneKey& o) const {
    return n_bins == o.n_bins && n_det == o.n_det && n == o.n && precision == o.precision && grad == o.grad;
  }
};
struct LoglikeTuned {
  LoglikeTuneKey key;
  int split;
};

struct sharpy_ctx {
  int device = 0;
  sharpy::DevModel model{};
  sharpy::DevEvent ev{};
  bool has_data = false;
  // event tables (device)
  double* d_f = nullptr;
  double* d_b64 = nullptr;
  float* d_b32 = nullptr;
  float* d_b32lo = nullptr;
  double2* d_e64 = nullptr;
  float2* d_e32 = nullptr;
  unsigned char* d_stage = nullptr;  // staged records of a long segment
  double* d_pref = nullptr;
  // status word and evidence accumulator (device)
  int* d_status = nullptr;
  double* d_lnz = nullptr;   // [0] ln Z, [1] number of stages (as double)
  // scratch (grown on demand)
  void* d_scratch = nullptr;
  size_t scratch_bytes = 0;
  // pinned host staging for small readbacks
  double* h_pinned = nullptr;
  cudaStream_t last_stream = nullptr;
  // host copies for the Fisher-information prefix tables (built on first use)
  std::vector<double> h_wamp2;  // [n_det][K] w f^-7/3
  std::vector<double> h_basis;  // [kNBasis][K]
  std::vector<double> h_amp;    // [K] f^-7/6 (grid table kept for the next event on the same grid)
  double* d_p1 = nullptr;       // [n_det][kNBasis][K] prefix sums of w f^-7/3 B_m
  double* d_p2 = nullptr;       // [n_det][kNBasis (kNBasis + 1) / 2][K] prefix sums of w f^-7/3 B_m B_n
  // NUTS slot count picked by the autotuner, per precision and metric kind
  // (shared / per-particle), for tuned_n[p][l] particles (0: not tuned)
  int64_t nuts_tick_limit = 0;  // > 0: lowered NUTS tick bound (sharpy_set_nuts_tick_limit)
  int64_t first_id = 0;         // ensemble index of row 0 of the particle arrays (sharpy_set_shard)
  // staged likelihood kernel, failure-detection tests (sharpy_set_stage_test_hooks): the block whose bulk copy
  // is left out (-1: none) and the mbarrier wait bound in polls (0: the default)
  int stage_skip_block = -1;
  int stage_wait_polls = 0;
  int tuned_slots[3][2] = {};
  // likelihood kernel: warps per particle picked per call shape (loglike.cu)
  std::vector<LoglikeTuned> ll_tuned;
  int ll_split_forced = 0;  // > 0: every likelihood call uses this split (sharpy_set_loglike_split)
  int nuts_slots_forced = 0;  // > 0: NUTS launches of this context use this slot count (sharpy_set_nuts_slots)
  int64_t tuned_n[3][2] = {{-1, -1}, {-1, -1}, {-1, -1}};
};

namespace sharpy {
// Make sure the context's scratch holds at least `bytes`; stream-ordered users
// only (a grow synchronises the device first).
int ensure_scratch(sharpy_ctx* ctx, size_t bytes);
int check_ctx(sharpy_ctx* ctx, bool need_data);
}  // namespace sharpy
