// sharpy_loglike_grad, sharpy_waveform, sharpy_prior_* : kernels and entry points.
//
// The likelihood kernel itself is in loglike_kernel.cuh.
#include <cstdio>

#include "loglike_kernel.cuh"
#include "tune.cuh"

using namespace sharpy;

namespace sharpy {

__global__ void gaussmix_kernel(DevModel m, int64_t n, const double* __restrict__ theta, double* __restrict__ lnl,
                                double* __restrict__ grad) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int D = m.n_dim;
  double x[kMaxDim], g[kMaxDim];
  for (int i = 0; i < D; ++i) x[i] = theta[p * D + i];
  double l;
  gaussmix(m, x, &l, grad ? g : nullptr);
  lnl[p] = l;
  if (grad)
    for (int i = 0; i < D; ++i) grad[p * D + i] = g[i];
}

// One CTA per (particle, block of 256 bins): FP64 strain of every detector.
__global__ void waveform_kernel(DevModel m, DevEvent ev, int64_t n, const double* __restrict__ theta,
                                double* __restrict__ h) {
  __shared__ SweepCoef sc;
  __shared__ EpiCoef<double> ec;
  const int64_t p = blockIdx.y;
  if (threadIdx.x == 0) {
    double th[kMaxDim];
    for (int i = 0; i < m.n_dim; ++i) th[i] = theta[p * m.n_dim + i];
    prologue<double, false>(m, ev, th, sc, ec);
  }
  __syncthreads();
  const int64_t K = ev.n_bins;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  for (int a = 0; a < ev.n_det; ++a) {
    double hr = 0.0, hi = 0.0;
    if (sc.ok && k <= sc.kisco) {
      double S = sc.c0;
      for (int j = 0; j < kNPn; ++j) S = fma(sc.alpha[j], ev.b64[(int64_t)j * K + k], S);
      double f = ev.f[k];
      double P = fma(f, sc.tau[a], S);
      double r = P - rint(P);
      double sn, cs;
      sincospi(2.0 * r, &sn, &cs);
      double amp = ec.A0 * pow(f, -7.0 / 6.0);
      hr = amp * (ec.cre[a] * cs + ec.cim[a] * sn);
      hi = amp * (ec.cim[a] * cs - ec.cre[a] * sn);
    }
    int64_t o = ((p * ev.n_det + a) * K + k) * 2;
    h[o] = hr;
    h[o + 1] = hi;
  }
}

__global__ void prior_sample_kernel(DevModel m, int64_t n, double* __restrict__ theta, uint64_t key, uint32_t ctr,
                                    int64_t first) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  for (int i = 0; i < m.n_dim; ++i) {
    double u0, u1;
    uniform2(key, (uint32_t)(p + first), ctr, RNG_PRIOR, (uint32_t)i, &u0, &u1);
    double lo = m.lo[i], hi = m.hi[i], x;
    if (m.prior[i] == SHARPY_PRIOR_POWER2)
      x = cbrt(lo * lo * lo + u0 * (hi * hi * hi - lo * lo * lo));
    else
      x = lo + u0 * (hi - lo);
    theta[p * m.n_dim + i] = x;
  }
}

__global__ void prior_logpdf_kernel(DevModel m, int64_t n, const double* __restrict__ theta, double* __restrict__ lp,
                                    double* __restrict__ glp) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double x[kMaxDim], g[kMaxDim];
  for (int i = 0; i < m.n_dim; ++i) x[i] = theta[p * m.n_dim + i];
  lp[p] = prior_logpdf(m, x, glp ? g : nullptr);
  if (glp)
    for (int i = 0; i < m.n_dim; ++i) glp[p * m.n_dim + i] = g[i];
}

// The split factor for this call: the context's tuned choice for (bins,
// detectors, particles, precision, gradient), else every candidate is timed
// on this call (one untimed and one timed launch each; the outputs are the
// same for every candidate) and the fastest is kept.
template <int PREC, bool GRAD>
static cudaError_t launch_ll_prec(sharpy_ctx* c, int split, int64_t n, const double* th, double* lnl, double* grad,
                                 cudaStream_t s) {
  if (PREC == SHARPY_FP64) return launch_ll_p0(c, GRAD, split, n, th, lnl, grad, s);
  if (PREC == SHARPY_MIXED) return launch_ll_p1(c, GRAD, split, n, th, lnl, grad, s);
  return launch_ll_p2(c, GRAD, split, n, th, lnl, grad, s);
}

template <int PREC, bool GRAD>
static int launch_ll(sharpy_ctx* c, int64_t n, const double* th, double* lnl, double* grad, cudaStream_t s) {
  if (c->ll_split_forced > 0)
    return launch_ll_prec<PREC, GRAD>(c, c->ll_split_forced, n, th, lnl, grad, s) == cudaSuccess ? SHARPY_OK
                                                                                              : SHARPY_ECUDA;
  const LoglikeTuneKey key{c->ev.n_bins, c->ev.n_det, n, PREC, GRAD ? 1 : 0};
  for (const auto& e : c->ll_tuned)
    if (e.key == key) return launch_ll_prec<PREC, GRAD>(c, e.split, n, th, lnl, grad, s) == cudaSuccess
                                 ? SHARPY_OK : SHARPY_ECUDA;
  // 1, 2, 4, 8 warps per vector, and the staged kernel where it applies
  TuneCandidate cands[kNumSplitChoices + 1];
  int nc = 0;
  for (int i = 0; i < kNumSplitChoices; ++i) cands[nc++].slots = kSplitChoices[i];
  if (PREC != SHARPY_FP64 && c->ev.stage) cands[nc++].slots = kSplitStaged;
  auto trial = [&](int split, cudaStream_t ts) -> int {
    return launch_ll_prec<PREC, GRAD>(c, split, n, th, lnl, grad, ts) == cudaSuccess ? SHARPY_OK : SHARPY_ECUDA;
  };
  int best = 1;
  const int rc = tune_slots(cands, nc, trial, s, &best);
  if (rc) return rc;
  c->ll_tuned.push_back({key, best});
  return SHARPY_OK;
}

}  // namespace sharpy

extern "C" {

int sharpy_loglike_grad(sharpy_ctx* c, int64_t n, const double* theta, double* lnl, double* grad, int precision,
                        sharpy_stream stream) {
  int rc = check_ctx(c, true);
  if (rc) return rc;
  if (n < 0 || (n > 0 && (!theta || !lnl))) return SHARPY_EINVAL;
  if (precision != SHARPY_FP64 && precision != SHARPY_MIXED && precision != SHARPY_MIXED_SPLIT)
    return SHARPY_EINVAL;
  if (n == 0) return SHARPY_OK;
  if (n > ((int64_t)1 << 31) - 1) return SHARPY_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  cudaError_t e;
  if (c->model.model == SHARPY_MODEL_GAUSSMIX) {
    gaussmix_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(c->model, n, theta, lnl, grad);
    e = cudaGetLastError();
  } else if (precision == SHARPY_FP64) {
    return grad ? launch_ll<SHARPY_FP64, true>(c, n, theta, lnl, grad, s) : launch_ll<SHARPY_FP64, false>(c, n, theta, lnl, grad, s);
  } else if (precision == SHARPY_MIXED) {
    return grad ? launch_ll<SHARPY_MIXED, true>(c, n, theta, lnl, grad, s)
                : launch_ll<SHARPY_MIXED, false>(c, n, theta, lnl, grad, s);
  } else {
    return grad ? launch_ll<SHARPY_MIXED_SPLIT, true>(c, n, theta, lnl, grad, s)
                : launch_ll<SHARPY_MIXED_SPLIT, false>(c, n, theta, lnl, grad, s);
  }
  return e == cudaSuccess ? SHARPY_OK : SHARPY_ECUDA;
}

int sharpy_set_loglike_split(sharpy_ctx* c, int split) {
  int rc = check_ctx(c, false);
  if (rc) return rc;
  if (split != 0 && split != 1 && split != 2 && split != 4 && split != 8 && split != kSplitStaged)
    return SHARPY_EINVAL;
  c->ll_split_forced = split;
  return SHARPY_OK;
}

int sharpy_set_stage_test_hooks(sharpy_ctx* c, int skip_block, int wait_polls) {
  int rc = check_ctx(c, false);
  if (rc) return rc;
  if (skip_block < -1 || wait_polls < 0) return SHARPY_EINVAL;
  c->stage_skip_block = skip_block;
  c->stage_wait_polls = wait_polls;
  return SHARPY_OK;
}

int sharpy_loglike_split(sharpy_ctx* c, int64_t n, int precision, int with_grad) {
  int rc = check_ctx(c, true);
  if (rc) return rc;
  const LoglikeTuneKey key{c->ev.n_bins, c->ev.n_det, n, precision, with_grad ? 1 : 0};
  for (const auto& e : c->ll_tuned)
    if (e.key == key) return e.split;
  return 0;
}

int sharpy_waveform(sharpy_ctx* c, int64_t n, const double* theta, double* h, sharpy_stream stream) {
  int rc = check_ctx(c, true);
  if (rc) return rc;
  if (c->model.model != SHARPY_MODEL_TAYLORF2) return SHARPY_EINVAL;
  if (n < 0 || n > 65535 || (n > 0 && (!theta || !h))) return SHARPY_EINVAL;
  if (n == 0) return SHARPY_OK;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  dim3 grid((unsigned)((c->ev.n_bins + 255) / 256), (unsigned)n);
  waveform_kernel<<<grid, 256, 0, s>>>(c->model, c->ev, n, theta, h);
  return cudaGetLastError() == cudaSuccess ? SHARPY_OK : SHARPY_ECUDA;
}

int sharpy_prior_sample(sharpy_ctx* c, int64_t n, double* theta, uint64_t key, uint64_t ctr, sharpy_stream stream) {
  int rc = check_ctx(c, false);
  if (rc) return rc;
  if (n < 0 || n > ((int64_t)1 << 31) - 1 || (n > 0 && !theta)) return SHARPY_EINVAL;
  if (n == 0) return SHARPY_OK;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  prior_sample_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(c->model, n, theta, key, (uint32_t)ctr,
                                                                   c->first_id);
  return cudaGetLastError() == cudaSuccess ? SHARPY_OK : SHARPY_ECUDA;
}

int sharpy_prior_logpdf_grad(sharpy_ctx* c, int64_t n, const double* theta, double* lp, double* glp,
                             sharpy_stream stream) {
  int rc = check_ctx(c, false);
  if (rc) return rc;
  if (n < 0 || n > ((int64_t)1 << 31) - 1 || (n > 0 && (!theta || !lp))) return SHARPY_EINVAL;
  if (n == 0) return SHARPY_OK;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  prior_logpdf_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(c->model, n, theta, lp, glp);
  return cudaGetLastError() == cudaSuccess ? SHARPY_OK : SHARPY_ECUDA;
}

}  // extern "C"
