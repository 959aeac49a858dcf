// Context lifetime, event staging, status word and evidence accumulator.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "context.cuh"
#include "split_stage.cuh"

using namespace sharpy;

namespace sharpy {

int ensure_scratch(sharpy_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->scratch_bytes) return SHARPY_OK;
  SHARPY_CUDA_TRY(cudaDeviceSynchronize());
  if (ctx->d_scratch) cudaFree(ctx->d_scratch);
  ctx->d_scratch = nullptr;
  ctx->scratch_bytes = 0;
  size_t want = bytes + bytes / 4;
  if (cudaMalloc(&ctx->d_scratch, want) != cudaSuccess) return SHARPY_ENOMEM;
  ctx->scratch_bytes = want;
  return SHARPY_OK;
}

int check_ctx(sharpy_ctx* ctx, bool need_data) {
  if (!ctx) return SHARPY_EINVAL;
  if (need_data && ctx->model.model == SHARPY_MODEL_TAYLORF2 && !ctx->has_data) return SHARPY_ESTATE;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return SHARPY_ECUDA;
  return SHARPY_OK;
}

// One CTA per staged record: thread i copies bin g kStageBins + i of every
// table the mixed sweep reads into record g of the mixed set, and of every
// table the split sweep reads into record g of the split set (zeros past the
// last bin).
__global__ void stage_tables_kernel(DevEvent ev, int nb, unsigned char* out) {
  const int g = blockIdx.x, i = threadIdx.x;
  const int64_t K = ev.n_bins, k = (int64_t)g * kStageBins + i;
  const bool in = k < K;
  unsigned char* rec = out + (size_t)g * stage_rec_bytes(ev.n_det);
  float* b32 = reinterpret_cast<float*>(rec);
  float* lo = reinterpret_cast<float*>(rec + stage_off_lo());
  double* b64 = reinterpret_cast<double*>(rec + stage_off_b64());
  float2* e32 = reinterpret_cast<float2*>(rec + stage_off_e32());
  for (int j = 0; j < kNBasis; ++j) b32[j * kStageBins + i] = in ? ev.b32[j * K + k] : 0.0f;
  constexpr int lo_j[5] = {3, 5, 6, 7, 8};
  for (int r = 0; r < 5; ++r) lo[r * kStageBins + i] = in ? ev.b32lo[lo_j[r] * K + k] : 0.0f;
  constexpr int b64_j[4] = {0, 1, 2, 4};
  for (int r = 0; r < 4; ++r) b64[r * kStageBins + i] = in ? ev.b64[b64_j[r] * K + k] : 0.0;
  for (int a = 0; a < ev.n_det; ++a) e32[a * kStageBins + i] = in ? ev.e32[a * K + k] : make_float2(0.0f, 0.0f);
  unsigned char* srec = out + split_set_offset(nb, ev.n_det) + (size_t)g * split_rec_bytes(ev.n_det);
  float* sb32 = reinterpret_cast<float*>(srec);
  float* slo = reinterpret_cast<float*>(srec + split_off_lo());
  float2* se32 = reinterpret_cast<float2*>(srec + split_off_e32());
  for (int j = 0; j < kNBasis; ++j) {
    sb32[j * kStageBins + i] = in ? ev.b32[j * K + k] : 0.0f;
    slo[j * kStageBins + i] = in ? ev.b32lo[j * K + k] : 0.0f;
  }
  for (int a = 0; a < ev.n_det; ++a) se32[a * kStageBins + i] = in ? ev.e32[a * K + k] : make_float2(0.0f, 0.0f);
}

}  // namespace sharpy

static void free_event(sharpy_ctx* c) {
  cudaFree(c->d_f);
  cudaFree(c->d_b64);
  cudaFree(c->d_b32);
  cudaFree(c->d_b32lo);
  cudaFree(c->d_e64);
  cudaFree(c->d_e32);
  cudaFree(c->d_pref);
  cudaFree(c->d_p1);
  cudaFree(c->d_p2);
  cudaFree(c->d_stage);
  c->d_stage = nullptr;
  c->ev.stage = nullptr;
  c->ev.stage_blocks = 0;
  c->d_p1 = c->d_p2 = nullptr;
  c->ev.p1 = c->ev.p2 = nullptr;
  c->d_f = c->d_b64 = c->d_pref = nullptr;
  c->d_b32 = nullptr;
  c->d_b32lo = nullptr;
  c->d_e64 = nullptr;
  c->d_e32 = nullptr;
  c->has_data = false;
}

// Detector tensor and position of an L-shaped detector on a spherical Earth.
static void detector_geometry(const sharpy_detector& in, DevDetector& out) {
  out.fixed_response = in.fixed_response;
  out.fplus = in.fplus;
  out.fcross = in.fcross;
  out.delay = in.delay;
  double sl = std::sin(in.lat), cl = std::cos(in.lat), so = std::sin(in.lon), co = std::cos(in.lon);
  double east[3] = {-so, co, 0.0};
  double north[3] = {-sl * co, -sl * so, cl};
  double ca = std::cos(in.azimuth), sa = std::sin(in.azimuth);
  double x[3], y[3];
  for (int i = 0; i < 3; ++i) {
    x[i] = ca * north[i] + sa * east[i];
    y[i] = -sa * north[i] + ca * east[i];
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      out.D[i][j] = 0.5 * (x[i] * x[j] - y[i] * y[j]);
      out.Df[i][j] = (float)out.D[i][j];
    }
  out.r[0] = kEarthR * cl * co;
  out.r[1] = kEarthR * cl * so;
  out.r[2] = kEarthR * sl;
  for (int i = 0; i < 3; ++i) {
    out.rcd[i] = out.r[i] / kClight;
    out.rcf[i] = (float)out.rcd[i];
  }
}

extern "C" {

int sharpy_create(sharpy_ctx** out, const sharpy_config* cfg, int device) {
  if (!out || !cfg) return SHARPY_EINVAL;
  *out = nullptr;
  if (cfg->n_dim < 1 || cfg->n_dim > SHARPY_MAX_DIM) return SHARPY_EINVAL;
  if (cfg->model != SHARPY_MODEL_TAYLORF2 && cfg->model != SHARPY_MODEL_GAUSSMIX) return SHARPY_EINVAL;
  for (int i = 0; i < cfg->n_dim; ++i) {
    if (!(cfg->lo[i] < cfg->hi[i]) || !std::isfinite(cfg->lo[i]) || !std::isfinite(cfg->hi[i])) return SHARPY_EINVAL;
    if (cfg->model == SHARPY_MODEL_TAYLORF2 && (cfg->phys[i] < 0 || cfg->phys[i] >= SHARPY_NPHYS)) return SHARPY_EINVAL;
    if (cfg->prior[i] == SHARPY_PRIOR_POWER2 && !(cfg->lo[i] > 0.0)) return SHARPY_EINVAL;
    if (cfg->prior[i] != SHARPY_PRIOR_UNIFORM && cfg->prior[i] != SHARPY_PRIOR_POWER2) return SHARPY_EINVAL;
    if (cfg->boundary[i] != SHARPY_BOUND_REFLECT && cfg->boundary[i] != SHARPY_BOUND_PERIODIC) return SHARPY_EINVAL;
  }
  if (cfg->model == SHARPY_MODEL_GAUSSMIX) {
    if (cfg->n_comp < 1 || cfg->n_comp > SHARPY_MAX_COMP) return SHARPY_EINVAL;
    for (int c = 0; c < cfg->n_comp; ++c)
      for (int i = 0; i < cfg->n_dim; ++i)
        if (!(cfg->mix_sigma[c][i] > 0.0)) return SHARPY_EINVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return SHARPY_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return SHARPY_ECUDA;
  sharpy_ctx* c = new (std::nothrow) sharpy_ctx();
  if (!c) return SHARPY_ENOMEM;
  c->device = device;
  DevModel& m = c->model;
  m.model = cfg->model;
  m.n_dim = cfg->n_dim;
  for (int i = 0; i < SHARPY_MAX_DIM; ++i) {
    m.phys[i] = cfg->phys[i];
    m.lo[i] = cfg->lo[i];
    m.hi[i] = cfg->hi[i];
    m.prior[i] = cfg->prior[i];
    m.boundary[i] = cfg->boundary[i];
  }
  for (int i = 0; i < SHARPY_NPHYS; ++i) m.fixed[i] = cfg->fixed[i];
  m.n_comp = cfg->n_comp;
  for (int k = 0; k < SHARPY_MAX_COMP; ++k) {
    m.mix_logw[k] = cfg->mix_logw[k];
    for (int i = 0; i < SHARPY_MAX_DIM; ++i) {
      m.mix_mu[k][i] = cfg->mix_mu[k][i];
      m.mix_sigma[k][i] = cfg->mix_sigma[k][i];
    }
  }
  bool ok = cudaMalloc(&c->d_status, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&c->d_lnz, 2 * sizeof(double)) == cudaSuccess &&
            cudaMallocHost(&c->h_pinned, 64 * sizeof(double)) == cudaSuccess &&
            cudaMemset(c->d_status, 0, sizeof(int)) == cudaSuccess &&
            cudaMemset(c->d_lnz, 0, 2 * sizeof(double)) == cudaSuccess &&
            cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    sharpy_destroy(c);
    return SHARPY_ENOMEM;
  }
  *out = c;
  return SHARPY_OK;
}

void sharpy_destroy(sharpy_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  free_event(c);
  cudaFree(c->d_status);
  cudaFree(c->d_lnz);
  cudaFree(c->d_scratch);
  cudaFreeHost(c->h_pinned);
  delete c;
}

int sharpy_set_data(sharpy_ctx* c, int n_det, int64_t n_bins, double f_min, double df, const double* d,
                    const double* psd, const sharpy_detector* det) {
  if (!c || !d || !psd || !det) return SHARPY_EINVAL;
  if (c->model.model != SHARPY_MODEL_TAYLORF2) return SHARPY_EINVAL;
  if (n_det < 1 || n_det > SHARPY_MAX_DET || n_bins < 1 || n_bins > (int64_t)1 << 30) return SHARPY_EINVAL;
  if (!(f_min > 0.0) || !(df > 0.0) || !std::isfinite(f_min) || !std::isfinite(df)) return SHARPY_EINVAL;
  if (n_det != 1 && n_det != 2 && n_det != 3) return SHARPY_EINVAL;  // kernels are instantiated for 1-3
  int64_t K = n_bins;
  for (int64_t i = 0; i < (int64_t)n_det * K; ++i) {
    if (!std::isfinite(psd[i]) || !(psd[i] > 0.0)) return SHARPY_ENONFINITE;
    if (!std::isfinite(d[2 * i]) || !std::isfinite(d[2 * i + 1])) return SHARPY_ENONFINITE;
  }
  int rc = check_ctx(c, false);
  if (rc) return rc;

  // The frequency-grid tables (f, basis functions, f^-7/6) depend only on
  // (K, f_min, df): a new event on the same grid and detector count keeps
  // them and the device buffers, and only the data-dependent tables are
  // rebuilt and copied.
  const bool same_grid = c->has_data && c->ev.n_det == n_det && c->ev.n_bins == K && c->ev.f_min == f_min &&
                         c->ev.df == df && (int64_t)c->h_amp.size() == K;
  if (!same_grid) {
    std::vector<double> f(K), b64(kNBasis * K), amp(K);
    std::vector<float> b32(kNBasis * K), b32lo(kNBasis * K);
    for (int64_t k = 0; k < K; ++k) {
      double fk = f_min + (double)k * df;
      f[k] = fk;
      double x = std::cbrt(1.0 / fk), y = std::cbrt(fk), l = std::log(fk);
      double x2 = x * x;
      double B[kNBasis] = {x2 * x2 * x, x2 * x, x2, x, l, y, y * l, y * y, fk};
      for (int j = 0; j < kNBasis; ++j) {
        b64[j * K + k] = B[j];
        b32[j * K + k] = (float)B[j];
        b32lo[j * K + k] = (float)(B[j] - (double)b32[j * K + k]);
      }
      amp[k] = std::pow(fk, -7.0 / 6.0);
    }
    free_event(c);
    bool ok = cudaMalloc(&c->d_f, K * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&c->d_b64, kNBasis * K * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&c->d_b32, kNBasis * K * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&c->d_b32lo, kNBasis * K * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&c->d_e64, n_det * K * sizeof(double2)) == cudaSuccess &&
              cudaMalloc(&c->d_e32, n_det * K * sizeof(float2)) == cudaSuccess &&
              cudaMalloc(&c->d_pref, n_det * K * sizeof(double)) == cudaSuccess;
    if (!ok) {
      free_event(c);
      return SHARPY_ENOMEM;
    }
    ok = cudaMemcpy(c->d_f, f.data(), K * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(c->d_b64, b64.data(), b64.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(c->d_b32, b32.data(), b32.size() * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(c->d_b32lo, b32lo.data(), b32lo.size() * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
      free_event(c);
      return SHARPY_ECUDA;
    }
    c->h_basis.swap(b64);
    c->h_amp.swap(amp);
    c->h_wamp2.clear();
  } else if (cudaDeviceSynchronize() != cudaSuccess) {
    // the previous event's tables may still be read by queued work
    return SHARPY_ECUDA;
  }
  const std::vector<double>& amp = c->h_amp;
  std::vector<double> e64(2 * n_det * K), pref(n_det * K), wamp2(n_det * K);
  std::vector<float> e32(2 * n_det * K);
  // <d|d> with a compensated sum; P_a prefix sums of w f^-7/3 (compensated).
  double dd = 0.0, ddc = 0.0;
  for (int a = 0; a < n_det; ++a) {
    double s = 0.0, cmp = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      int64_t i = a * K + k;
      double w = 4.0 * df / psd[i];
      double dr = d[2 * i], di = d[2 * i + 1];
      // E = w conj(d) f^-7/6
      e64[2 * i] = w * dr * amp[k];
      e64[2 * i + 1] = -w * di * amp[k];
      e32[2 * i] = (float)e64[2 * i];
      e32[2 * i + 1] = (float)e64[2 * i + 1];
      double term = w * amp[k] * amp[k];
      wamp2[i] = term;
      double t = s + term;
      cmp += std::fabs(s) >= std::fabs(term) ? (s - t) + term : (term - t) + s;
      s = t;
      pref[i] = s + cmp;
      double dt = w * (dr * dr + di * di);
      double u = dd + dt;
      ddc += std::fabs(dd) >= std::fabs(dt) ? (dd - u) + dt : (dt - u) + dd;
      dd = u;
    }
  }
  const bool ok = cudaMemcpy(c->d_e64, e64.data(), e64.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(c->d_e32, e32.data(), e32.size() * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(c->d_pref, pref.data(), pref.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    free_event(c);
    return SHARPY_ECUDA;
  }
  // the Fisher prefix tables depend on w f^-7/3 only: kept while it is unchanged
  if (wamp2 != c->h_wamp2) {
    cudaFree(c->d_p1);
    cudaFree(c->d_p2);
    c->d_p1 = c->d_p2 = nullptr;
    c->h_wamp2.swap(wamp2);
  }
  DevEvent& ev = c->ev;
  ev.n_det = n_det;
  ev.n_bins = K;
  ev.f_min = f_min;
  ev.df = df;
  ev.inv_df = 1.0 / df;
  ev.dd = dd + ddc;
  {
    const double h = -0.5 * ev.dd;  // the epilogue's starting sum, as a double-float
    ev.ddh_hi = (float)h;
    ev.ddh_lo = (float)(h - (double)ev.ddh_hi);
  }
  ev.f = c->d_f;
  ev.b64 = c->d_b64;
  ev.b32 = c->d_b32;
  ev.b32lo = c->d_b32lo;
  ev.e64 = c->d_e64;
  ev.e32 = c->d_e32;
  ev.pref = c->d_pref;
  ev.p1 = c->d_p1;
  ev.p2 = c->d_p2;
  for (int a = 0; a < n_det; ++a) detector_geometry(det[a], ev.det[a]);
  // staged records of a long segment (rebuilt with every data set: they hold E)
  if (c->model.model == SHARPY_MODEL_TAYLORF2 && K >= kStageMinBins) {
    const int nb = (int)((K + kStageBins - 1) / kStageBins);
    const size_t bytes = split_set_offset(nb, n_det) + (size_t)nb * split_rec_bytes(n_det);
    if (!c->d_stage && cudaMalloc(&c->d_stage, bytes) != cudaSuccess) {
      c->d_stage = nullptr;
      free_event(c);
      return SHARPY_ENOMEM;
    }
    stage_tables_kernel<<<nb, kStageBins>>>(ev, nb, c->d_stage);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
      free_event(c);
      return SHARPY_ECUDA;
    }
    ev.stage = c->d_stage;
    ev.stage_blocks = nb;
  } else {
    ev.stage = nullptr;
    ev.stage_blocks = 0;
  }
  c->has_data = true;
  return SHARPY_OK;
}

int sharpy_reset_evidence(sharpy_ctx* c, sharpy_stream stream) {
  int rc = check_ctx(c, false);
  if (rc) return rc;
  SHARPY_CUDA_TRY(cudaMemsetAsync(c->d_lnz, 0, 2 * sizeof(double), (cudaStream_t)stream));
  c->last_stream = (cudaStream_t)stream;
  return SHARPY_OK;
}

int sharpy_set_evidence(sharpy_ctx* c, double lnz, int n_stages, sharpy_stream stream) {
  int rc = check_ctx(c, false);
  if (rc) return rc;
  if (!std::isfinite(lnz) || n_stages < 0) return SHARPY_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // through the pinned staging buffer, after the stream's earlier work has read it
  SHARPY_CUDA_TRY(cudaStreamSynchronize(s));
  c->h_pinned[0] = lnz;
  c->h_pinned[1] = (double)n_stages;
  SHARPY_CUDA_TRY(cudaMemcpyAsync(c->d_lnz, c->h_pinned, 2 * sizeof(double), cudaMemcpyHostToDevice, s));
  SHARPY_CUDA_TRY(cudaStreamSynchronize(s));
  c->last_stream = s;
  return SHARPY_OK;
}

int sharpy_log_evidence(sharpy_ctx* c, double* lnz, int* n_stages) {
  int rc = check_ctx(c, false);
  if (rc) return rc;
  if (!lnz) return SHARPY_EINVAL;
  SHARPY_CUDA_TRY(cudaMemcpyAsync(c->h_pinned, c->d_lnz, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                  c->last_stream));
  SHARPY_CUDA_TRY(cudaStreamSynchronize(c->last_stream));
  *lnz = c->h_pinned[0];
  if (n_stages) *n_stages = (int)c->h_pinned[1];
  return SHARPY_OK;
}

int sharpy_get_status(sharpy_ctx* c) {
  int rc = check_ctx(c, false);
  if (rc) return rc;
  int s = 0;
  SHARPY_CUDA_TRY(cudaDeviceSynchronize());
  SHARPY_CUDA_TRY(cudaMemcpy(&s, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  return s;
}

int sharpy_clear_status(sharpy_ctx* c) {
  int rc = check_ctx(c, false);
  if (rc) return rc;
  SHARPY_CUDA_TRY(cudaDeviceSynchronize());
  SHARPY_CUDA_TRY(cudaMemset(c->d_status, 0, sizeof(int)));
  SHARPY_CUDA_TRY(cudaDeviceSynchronize());
  return SHARPY_OK;
}

const char* sharpy_error_string(int code) {
  switch (code) {
    case SHARPY_OK: return "ok";
    case SHARPY_EINVAL: return "invalid argument";
    case SHARPY_ECUDA: return "CUDA runtime error";
    case SHARPY_ENOMEM: return "out of memory";
    case SHARPY_ENONFINITE: return "non-finite value";
    case SHARPY_ETIMEOUT: return "device loop bound reached";
    case SHARPY_EBOUNDS: return "index out of bounds";
    case SHARPY_ESTATE: return "call out of order";
    default: return "unknown error";
  }
}

}  // extern "C"

extern "C" void sharpy_uniform2(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double* u) {
  if (u) sharpy::uniform2(key, c0, c1, c2, c3, u, u + 1);
}
