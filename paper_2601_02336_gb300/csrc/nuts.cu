// sharpy_nuts_mutate: host side of the persistent NUTS kernel (nuts_kernel.cuh).
#include "nuts_kernel.cuh"

using namespace sharpy;

namespace sharpy {

// Defined by the six compilations of nuts_inst.cu.
int launch_nuts_p0_1(int slots, const NutsArgs& A, unsigned grid, cudaStream_t s);
int launch_nuts_p0_2(int slots, const NutsArgs& A, unsigned grid, cudaStream_t s);
int launch_nuts_p0_3(int slots, const NutsArgs& A, unsigned grid, cudaStream_t s);
int launch_nuts_p1_1(int slots, const NutsArgs& A, unsigned grid, cudaStream_t s);
int launch_nuts_p1_2(int slots, const NutsArgs& A, unsigned grid, cudaStream_t s);
int launch_nuts_p1_3(int slots, const NutsArgs& A, unsigned grid, cudaStream_t s);
int launch_nuts_p2_1(int slots, const NutsArgs& A, unsigned grid, cudaStream_t s);
int launch_nuts_p2_2(int slots, const NutsArgs& A, unsigned grid, cudaStream_t s);
int launch_nuts_p2_3(int slots, const NutsArgs& A, unsigned grid, cudaStream_t s);

int launch_nuts(int precision, int ndet, int slots, const NutsArgs& A, unsigned grid, cudaStream_t s) {
  if (precision == SHARPY_FP64) {
    if (ndet == 1) return launch_nuts_p0_1(slots, A, grid, s);
    if (ndet == 2) return launch_nuts_p0_2(slots, A, grid, s);
    return launch_nuts_p0_3(slots, A, grid, s);
  }
  if (precision == SHARPY_MIXED) {
    if (ndet == 1) return launch_nuts_p1_1(slots, A, grid, s);
    if (ndet == 2) return launch_nuts_p1_2(slots, A, grid, s);
    return launch_nuts_p1_3(slots, A, grid, s);
  }
  if (ndet == 1) return launch_nuts_p2_1(slots, A, grid, s);
  if (ndet == 2) return launch_nuts_p2_2(slots, A, grid, s);
  return launch_nuts_p2_3(slots, A, grid, s);
}
// Segments of at least this many bins (the 128 s BNS workload) spread each
// long sweep's streams over the warps of a NUTS tick.
constexpr int64_t kLongSignalBins = 65536;

// slots: particles per CTA; 0 picks the autotuned count for (n, precision) if
// the context has one, else the widest count that still gives about two CTAs
// per SM.
int enqueue_nuts(sharpy_ctx* c, int64_t n, const double* beta_ptr, double beta, double* theta, double* lnl,
                 double* grad, const double* inv_mass, const double* cov_step, double step, int max_depth,
                 int n_steps, uint64_t key, uint32_t ctr, int precision, sharpy_nuts_stats* stats, cudaStream_t s,
                 int slots, const double* pminv, const double* pchol) {
  NutsArgs A;
  A.m = c->model;
  A.ev = c->ev;
  A.n = n;
  A.theta = theta;
  A.lnl = lnl;
  A.grad = grad;
  A.beta_ptr = beta_ptr;
  A.beta = beta;
  A.minv = inv_mass;
  A.cov_step = cov_step;
  A.step = step;
  A.max_depth = max_depth;
  A.n_steps = n_steps;
  A.key = key;
  A.ctr = ctr;
  A.stats = stats;
  A.status = c->d_status;
  A.tick_limit = c->nuts_tick_limit;
  A.id_offset = c->first_id;
  A.stream_part = nullptr;
  const int lm = pminv ? 1 : 0;
  if (!slots && c->nuts_slots_forced) slots = c->nuts_slots_forced;
  if (!slots && c->tuned_slots[precision][lm] && c->tuned_n[precision][lm] == n) slots = c->tuned_slots[precision][lm];
  if (!slots) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    slots = n >= (int64_t)16 * 2 * sms * 3 / 4 ? 16 : 8;
  }
  const int nd = c->model.model == SHARPY_MODEL_TAYLORF2 ? c->ev.n_det : 1;
  if (c->model.model == SHARPY_MODEL_TAYLORF2 && c->ev.n_bins >= kLongSignalBins) {
    // long signals: the sweeps' streams spread over the warps of a tick
    const int64_t rows = (n + slots - 1) / slots * slots;
    const int rc = ensure_scratch(c, (size_t)rows * kStreams * 64 * sizeof(double));
    if (rc) return rc;
    A.stream_part = (double*)c->d_scratch;
  }
  A.pminv = pminv;
  A.pchol = pchol;
  A.local_metric = pminv ? 1 : 0;
  A.batch = nullptr;
  A.cta_map = nullptr;
  A.active = nullptr;
  A.stage = nullptr;
  return launch_nuts(precision, nd, slots, A, 0u, s);
}
}  // namespace sharpy

extern "C" int sharpy_nuts_mutate(sharpy_ctx* c, int64_t n, double beta, double* theta, double* lnl, double* grad,
                                  const double* inv_mass, double step, int max_depth, int n_steps, uint64_t key,
                                  uint64_t ctr, int precision, sharpy_nuts_stats* stats, sharpy_stream stream) {
  int rc = check_ctx(c, true);
  if (rc) return rc;
  if (n < 0 || n > ((int64_t)1 << 31) - 1) return SHARPY_EINVAL;
  if (n == 0) return SHARPY_OK;
  if (!theta || !lnl || !grad || !(step > 0.0) || !isfinite(step) || max_depth < 0 || max_depth > kMaxDepth ||
      n_steps < 0 || !(beta >= 0.0 && beta <= 1.0))
    return SHARPY_EINVAL;
  if (precision != SHARPY_FP64 && precision != SHARPY_MIXED && precision != SHARPY_MIXED_SPLIT)
    return SHARPY_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return enqueue_nuts(c, n, nullptr, beta, theta, lnl, grad, inv_mass, nullptr, step, max_depth, n_steps, key,
                      (uint32_t)ctr, precision, stats, s, 0, nullptr, nullptr);
}

extern "C" int sharpy_nuts_mutate_local(sharpy_ctx* c, int64_t n, double beta, double* theta, double* lnl,
                                        double* grad, const double* inv_mass, const double* chol, double step,
                                        int max_depth, int n_steps, uint64_t key, uint64_t ctr, int precision,
                                        sharpy_nuts_stats* stats, sharpy_stream stream) {
  int rc = check_ctx(c, true);
  if (rc) return rc;
  if (n < 0 || n > ((int64_t)1 << 31) - 1) return SHARPY_EINVAL;
  if (n == 0) return SHARPY_OK;
  if (!theta || !lnl || !grad || !inv_mass || !chol || !(step > 0.0) || !isfinite(step) || max_depth < 0 ||
      max_depth > kMaxDepth || n_steps < 0 || !(beta >= 0.0 && beta <= 1.0))
    return SHARPY_EINVAL;
  if (precision != SHARPY_FP64 && precision != SHARPY_MIXED && precision != SHARPY_MIXED_SPLIT)
    return SHARPY_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return enqueue_nuts(c, n, nullptr, beta, theta, lnl, grad, nullptr, nullptr, step, max_depth, n_steps, key,
                      (uint32_t)ctr, precision, stats, s, 0, inv_mass, chol);
}

extern "C" int sharpy_nuts_mutate_cov_step(sharpy_ctx* c, int64_t n, double beta, double* theta, double* lnl,
                                           double* grad, const double* cov, double eps_scale, int max_depth,
                                           int n_steps, uint64_t key, uint64_t ctr, int precision,
                                           sharpy_nuts_stats* stats, sharpy_stream stream) {
  int rc = check_ctx(c, true);
  if (rc) return rc;
  if (n < 0 || n > ((int64_t)1 << 31) - 1) return SHARPY_EINVAL;
  if (n == 0) return SHARPY_OK;
  if (!theta || !lnl || !grad || !cov || !(eps_scale > 0.0) || !isfinite(eps_scale) || max_depth < 0 ||
      max_depth > kMaxDepth || n_steps < 0 || !(beta >= 0.0 && beta <= 1.0))
    return SHARPY_EINVAL;
  if (precision != SHARPY_FP64 && precision != SHARPY_MIXED && precision != SHARPY_MIXED_SPLIT)
    return SHARPY_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return enqueue_nuts(c, n, nullptr, beta, theta, lnl, grad, nullptr, cov, eps_scale, max_depth, n_steps, key,
                      (uint32_t)ctr, precision, stats, s, 0, nullptr, nullptr);
}

extern "C" int sharpy_set_nuts_tick_limit(sharpy_ctx* c, int64_t max_ticks) {
  int rc = check_ctx(c, false);
  if (rc) return rc;
  if (max_ticks < 0) return SHARPY_EINVAL;
  c->nuts_tick_limit = max_ticks;
  return SHARPY_OK;
}

extern "C" int sharpy_set_nuts_slots(sharpy_ctx* c, int slots) {
  int rc = check_ctx(c, false);
  if (rc) return rc;
  if (slots != 0 && slots != 4 && slots != 8 && slots != 16 && slots != 32) return SHARPY_EINVAL;
  c->nuts_slots_forced = slots;
  return SHARPY_OK;
}

extern "C" int sharpy_set_shard(sharpy_ctx* c, int64_t first_id) {
  int rc = check_ctx(c, false);
  if (rc) return rc;
  if (first_id < 0 || first_id > ((int64_t)1 << 31) - 1) return SHARPY_EINVAL;
  c->first_id = first_id;
  return SHARPY_OK;
}
