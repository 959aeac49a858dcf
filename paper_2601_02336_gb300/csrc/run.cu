// sharpy_smc_run: the full SMC loop (Sec. 3) driven from the host, with all
// per-stage state (beta, ln Z, particles, metric) kept on the device.
#include <cmath>

#include <nvtx3/nvToolsExt.h>

#include "context.cuh"
#include "tune.cuh"

using namespace sharpy;

namespace sharpy {
int enqueue_stage(sharpy_ctx* c, int64_t n, double* theta, double* lnl, double* grad, const double* beta_prev_ptr,
                  double beta_prev, double alpha, double u, double* beta_next, double* dlnz, double* ess,
                  int32_t* anc_out, double* cov, double* beta_state, cudaStream_t s);
int enqueue_nuts(sharpy_ctx* c, int64_t n, const double* beta_ptr, double beta, double* theta, double* lnl,
                 double* grad, const double* inv_mass, const double* cov_step, double step, int max_depth,
                 int n_steps, uint64_t key, uint32_t ctr, int precision, sharpy_nuts_stats* stats, cudaStream_t s,
                 int slots, const double* pminv, const double* pchol);
int enqueue_local_metric(sharpy_ctx* c, int64_t n, const double* theta, const double* beta_ptr, double beta,
                         double* mass, double* minv, double* chol, cudaStream_t s);

// Per-stage record: [beta, ess, dlnz, eps, accept_sum, depth_sum, n_leapfrog, n_divergent, active_bins, ln Z]
constexpr int kRec = 10;
// Stage on which a context without a tuned slot count times the candidates
// (a mid-run state; on the first stage every tree reaches the depth limit).
constexpr int kTuneStage = 3;

__global__ void stage_record_kernel(int64_t n, int D, const sharpy_nuts_stats* __restrict__ st,
                                    const double* beta, const double* ess, const double* dlnz, const double* cov,
                                    int metric, double eps_scale, const double* lnz_acc, double* rec) {
  __shared__ double red[5][32];
  double a[5] = {0, 0, 0, 0, 0};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    a[0] += st[i].accept_sum;
    a[1] += st[i].depth_sum;
    a[2] += st[i].n_leapfrog;
    a[3] += st[i].n_divergent;
    a[4] += st[i].active_bins;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 5; ++k) {
    double v = warp_sum(a[k]);
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 5; ++k) {
      double s = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[k][w];
      rec[4 + k] = s;
    }
    rec[0] = *beta;
    rec[1] = *ess;
    rec[2] = *dlnz;
    double eps = eps_scale;
    if (metric == 0) {
      double smin = INFINITY;
      for (int j = 0; j < D; ++j) smin = fmin(smin, sqrt(cov[j * D + j]));
      eps = eps_scale * smin;
    }
    rec[3] = eps;
    rec[9] = lnz_acc[0];
  }
}
}  // namespace sharpy

extern "C" int sharpy_smc_run(sharpy_ctx* c, const sharpy_smc_options* o, uint64_t key, double* lnz, int* n_stages,
                              double* theta_out, double* lnl_out, sharpy_stage* stages, sharpy_stream stream) {
  int rc = check_ctx(c, true);
  if (rc) return rc;
  if (!o || !lnz || o->n_particles < 1 || o->n_particles > ((int64_t)1 << 20) || !(o->alpha > 0.0 && o->alpha <= 1.0) ||
      o->n_mut < 0 || o->max_depth < 0 || o->max_depth > SHARPY_MAX_DEPTH || o->max_stages < 1 ||
      !(o->eps_scale > 0.0) || (o->metric != 0 && o->metric != 1 && o->metric != 2) ||
      (o->precision != SHARPY_FP64 && o->precision != SHARPY_MIXED && o->precision != SHARPY_MIXED_SPLIT))
    return SHARPY_EINVAL;
  const int64_t n = o->n_particles;
  const int D = c->model.n_dim;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  // run buffers: theta, grad [N][D], lnl [N], stats [N], scalars, cov, record;
  // copies of theta, grad, lnl for the autotuner's trials when it has to run
  const bool local = o->metric == 2;  // per-particle metric: [N][D][D] inverse and Cholesky factor
  const bool tune = !c->nuts_slots_forced && !(c->tuned_slots[o->precision][local] && c->tuned_n[o->precision][local] == n);
  size_t bytes = (size_t)n * (2 * D + 1) * sizeof(double) * (tune ? 2 : 1) + (size_t)n * sizeof(sharpy_nuts_stats) +
                 (8 + D * D + kRec) * sizeof(double) + (local ? 2 * (size_t)n * D * D * sizeof(double) : 0);
  char* buf = nullptr;
  SHARPY_CUDA_TRY(cudaMallocAsync((void**)&buf, bytes, s));
  double* th = (double*)buf;
  double* gr = th + n * D;
  double* ll = gr + n * D;
  sharpy_nuts_stats* st = (sharpy_nuts_stats*)(ll + n);
  double* sc = (double*)(st + n);
  double* beta_state = sc + 0;
  double* beta_next = sc + 1;
  double* dlnz = sc + 2;
  double* ess = sc + 3;
  double* cov = sc + 8;
  double* rec = cov + D * D;
  double* trial = rec + kRec;  // [N][D] theta, [N][D] grad, [N] lnl (autotuner)
  double* pminv = trial + (tune ? (size_t)n * (2 * D + 1) : 0);
  double* pchol = pminv + (size_t)n * D * D;
  int out = SHARPY_OK;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evr = nullptr;
  auto fail = [&](int code) {
    cudaFreeAsync(buf, s);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (evr) cudaEventDestroy(evr);
    return code;
  };
  if (cudaMemsetAsync(beta_state, 0, sizeof(double), s) != cudaSuccess) return fail(SHARPY_ECUDA);
  if ((rc = sharpy_reset_evidence(c, stream))) return fail(rc);
  if ((rc = sharpy_prior_sample(c, n, th, key, 0, stream))) return fail(rc);
  if ((rc = sharpy_loglike_grad(c, n, th, ll, gr, o->precision, stream))) return fail(rc);
  if (o->timing && (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess ||
                    cudaEventCreate(&evr) != cudaSuccess))
    return fail(SHARPY_ECUDA);
  double beta = 0.0;
  int t = 0;
  nvtxRangePushA("sharpy_smc_run");
  struct RangeEnd {
    ~RangeEnd() { nvtxRangePop(); }
  } range_end;
  while (beta < 1.0 && t < o->max_stages) {
    ++t;
    nvtxRangePushA("stage");
    struct StageEnd {
      ~StageEnd() { nvtxRangePop(); }
    } stage_end;
    double u0, u1;
    uniform2(key, 0u, (uint32_t)t, RNG_RESAMPLE, 0u, &u0, &u1);
    if (o->timing) cudaEventRecord(evr, s);
    rc = enqueue_stage(c, n, th, ll, gr, beta_state, 0.0, o->alpha, u0, beta_next, dlnz, ess, nullptr, cov,
                       beta_state, s);
    if (rc) return fail(rc);
    const double* minv = o->metric == 1 ? cov : nullptr;
    const double* cov_step = o->metric == 0 ? cov : nullptr;
    if (local && (rc = enqueue_local_metric(c, n, th, beta_state, 0.0, nullptr, pminv, pchol, s))) return fail(rc);
    const double* pm = local ? pminv : nullptr;
    const double* pc = local ? pchol : nullptr;
    if (t == kTuneStage && tune) {
      // pick the slot count on this stage: its full mutation on copies of the particles
      auto go = [&](int slots, cudaStream_t ts) -> int {
        SHARPY_CUDA_TRY(cudaMemcpyAsync(trial, th, (size_t)n * (2 * D + 1) * sizeof(double),
                                        cudaMemcpyDeviceToDevice, ts));
        return enqueue_nuts(c, n, beta_state, 0.0, trial, trial + 2 * n * D, trial + n * D, minv, cov_step,
                            o->eps_scale, o->max_depth, o->n_mut, key, (uint32_t)t << 8, o->precision, st, ts,
                            slots, pm,
                            pc);
      };
      TuneCandidate cands[kNumSlotChoices];
      for (int i = 0; i < kNumSlotChoices; ++i) cands[i].slots = kSlotChoices[i];
      int best = 0;
      if ((rc = tune_slots(cands, kNumSlotChoices, go, s, &best))) return fail(rc);
      c->tuned_slots[o->precision][local] = best;
      c->tuned_n[o->precision][local] = n;
    }
    if (o->timing) cudaEventRecord(ev0, s);
    rc = enqueue_nuts(c, n, beta_state, 0.0, th, ll, gr, minv, cov_step, o->eps_scale, o->max_depth, o->n_mut, key,
                      (uint32_t)t << 8, o->precision, st, s, 0, pm, pc);
    if (rc) return fail(rc);
    if (o->timing) cudaEventRecord(ev1, s);
    if (o->pool_theta && o->pool_lnl && (int64_t)t * n <= o->pool_cap) {
      const int64_t row = (int64_t)(t - 1) * n;
      if (cudaMemcpyAsync(o->pool_theta + row * D, th, n * D * sizeof(double), cudaMemcpyDeviceToDevice, s) !=
              cudaSuccess ||
          cudaMemcpyAsync(o->pool_lnl + row, ll, n * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fail(SHARPY_ECUDA);
    }
    stage_record_kernel<<<1, 1024, 0, s>>>(n, D, st, beta_next, ess, dlnz, cov, o->metric, o->eps_scale, c->d_lnz,
                                           rec);
    if (cudaGetLastError() != cudaSuccess) return fail(SHARPY_ECUDA);
    if (cudaMemcpyAsync(c->h_pinned, rec, kRec * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(SHARPY_ECUDA);
    const double* r = c->h_pinned;
    if (stages) {
      sharpy_stage& g = stages[t - 1];
      g.beta = r[0];
      g.dbeta = r[0] - beta;
      g.ess = r[1];
      g.dlnz = r[2];
      g.eps = r[3];
      g.accept_mean = r[4] / (double)(n * (o->n_mut > 0 ? o->n_mut : 1));
      g.depth_mean = r[5] / (double)(n * (o->n_mut > 0 ? o->n_mut : 1));
      g.n_leapfrog = (int64_t)r[6];
      g.n_divergent = (int)r[7];
      g.pad = 0;
      g.active_bins = r[8];
      float ms = 0.0f, rms = 0.0f;
      if (o->timing) {
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventElapsedTime(&rms, evr, ev0);
      }
      g.nuts_ms = ms;
      g.reweight_ms = rms;
      g.lnz = r[9];
    }
    beta = r[0];
    if (!std::isfinite(beta)) return fail(SHARPY_ENONFINITE);
  }
  if (theta_out && cudaMemcpyAsync(theta_out, th, n * D * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return fail(SHARPY_ECUDA);
  if (lnl_out && cudaMemcpyAsync(lnl_out, ll, n * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return fail(SHARPY_ECUDA);
  cudaFreeAsync(buf, s);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (evr) cudaEventDestroy(evr);
  int ns = 0;
  if ((rc = sharpy_log_evidence(c, lnz, &ns))) return rc;
  if (n_stages) *n_stages = ns;
  if (beta < 1.0) out = SHARPY_ETIMEOUT;
  return out;
}
