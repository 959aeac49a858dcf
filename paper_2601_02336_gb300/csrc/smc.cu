// SMC stage kernels (Sec. 3): adaptive tempering, weights, ESS, evidence
// increment, weighted covariance, integer systematic resampling and gather.
#include <cmath>

#include "context.cuh"

using namespace sharpy;

namespace sharpy {

constexpr int kSmcThreads = 1024;
constexpr int64_t kMaxParticles = (int64_t)1 << 20;

// Block-wide sum (fixed tree order: deterministic).
template <class T>
__device__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T r = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r += red[w];
  return r;
}

static __device__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
  return r;
}

struct EssSums {
  double s1, s2, s1x, s2x;
};

// S1 = sum e^{db x}, S2 = sum e^{2 db x} and their db-derivatives / x-weighted sums.
static __device__ EssSums ess_sums(const double* lnl, int64_t n, double mx, double db, double* red) {
  double s1 = 0, s2 = 0, s1x = 0, s2x = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double l = lnl[i];
    if (!isfinite(l)) continue;
    double x = l - mx;
    double w = exp(db * x);
    double w2 = w * w;
    s1 += w;
    s2 += w2;
    s1x += w * x;
    s2x += w2 * x;
  }
  EssSums r;
  r.s1 = block_sum(s1, red);
  r.s2 = block_sum(s2, red);
  r.s1x = block_sum(s1x, red);
  r.s2x = block_sum(s2x, red);
  return r;
}

// Single-CTA stage kernel. Solves ESS(db) = alpha N for the tempering
// increment (Eq. 6). ESS decreases with db and S2(db) = S1(2 db), so one FP32
// pass over the geometric grid db_m = hi 2^-m (m = -1..kGrid-2) brackets the
// root within a factor of two; a Newton iteration on g(db) = 2 ln S1 - ln S2 -
// ln(alpha N) in FP64, safeguarded by that bracket, then locates the root to
// ~1e-13 relative and keeps the largest evaluated db with ESS >= alpha N. Writes W = e^{db (lnL - max)}, the integer prefix sums C of
// floor(W 2^32), the ESS, dlnz, beta_next, the covariance, and updates ln Z.
constexpr int kGrid = 54;
constexpr int kGridChunk = 9;

__global__ void __launch_bounds__(kSmcThreads)
reweight_kernel(int64_t n, const double* __restrict__ lnl, const double* __restrict__ theta, int D,
                const double* beta_prev_ptr, double beta_prev_val, double alpha, double* __restrict__ w_out,
                unsigned long long* __restrict__ csum, double* beta_next, double* dlnz, double* ess_out,
                double* cov, double* lnz_acc, double* beta_state, int* status) {
  __shared__ double red[32];
  __shared__ float redf[kGridChunk][32];
  __shared__ float s1grid[kGrid];
  __shared__ double sh_db;
  __shared__ unsigned long long carry[kSmcThreads];
  const double beta_prev = beta_prev_ptr ? *beta_prev_ptr : beta_prev_val;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  double mx = -INFINITY;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
    if (isfinite(lnl[i])) mx = fmax(mx, lnl[i]);
  mx = block_max(mx, red);
  if (!isfinite(mx)) {
    if (threadIdx.x == 0) set_status(status, SHARPY_ENONFINITE);
    return;
  }
  const double target = alpha * (double)n;
  const double lt = log(target);
  double hi = 1.0 - beta_prev;
  if (threadIdx.x == 0) sh_db = 0.0;
  if (hi > 0.0) {
    EssSums e = ess_sums(lnl, n, mx, hi, red);
    double ess_hi = e.s1 * e.s1 / e.s2;
    if (ess_hi >= target) {
      if (threadIdx.x == 0) sh_db = hi;
    } else {
      // FP32 grid: s1grid[m] = S1(hi 2^(1-m)), so g(hi 2^-m) uses s1grid[m+1] and s1grid[m]
      for (int c0 = 0; c0 < kGrid; c0 += kGridChunk) {
        float acc[kGridChunk];
#pragma unroll
        for (int c = 0; c < kGridChunk; ++c) acc[c] = 0.0f;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
          double l = lnl[i];
          if (!isfinite(l)) continue;
          const float x = (float)((l - mx) * hi * 1.4426950408889634);  // log2(e) * db0 * x
#pragma unroll
          for (int c = 0; c < kGridChunk; ++c) acc[c] += exp2f(ldexpf(x, 1 - (c0 + c)));
        }
#pragma unroll
        for (int c = 0; c < kGridChunk; ++c) {
          float v = warp_sum(acc[c]);
          if (lane == 0) redf[c][warp] = v;
        }
        __syncthreads();
        if (threadIdx.x < kGridChunk) {
          float t = 0.0f;
          for (int w = 0; w < nwarp; ++w) t += redf[threadIdx.x][w];
          s1grid[c0 + threadIdx.x] = t;
        }
        __syncthreads();
      }
      // largest grid point with ESS >= target: bracket [hi 2^-m, hi 2^(1-m)]
      int m = 1;
      while (m < kGrid - 1 && 2.0f * logf(s1grid[m + 1]) - logf(s1grid[m]) < (float)lt) ++m;
      double lo = (m < kGrid - 1) ? ldexp(hi, -m) : 0.0;
      double up = ldexp(hi, 1 - m);
      // the FP32 bracket may be one cell off near the crossing: widen until FP64 agrees
      for (int k = 0; k < 4 && lo > 0.0; ++k) {
        EssSums a = ess_sums(lnl, n, mx, lo, red);
        if (2.0 * log(a.s1) - log(a.s2) - lt >= 0.0) break;
        up = lo;
        lo = (k == 3) ? 0.0 : 0.5 * lo;
      }
      double x = lo > 0.0 ? sqrt(lo * up) : 0.5 * up;
      // Newton on g inside [lo, up] until the step falls below 1e-13 relative:
      // g itself is only known to ~1e-15 (logs of large sums), so closer than
      // that the iteration would wander inside rounding noise. The result is the
      // root to ~1e-13 relative (the oracle bisects to adjacent doubles).
      for (int it = 0; it < 60; ++it) {
        EssSums sm = ess_sums(lnl, n, mx, x, red);
        double g = 2.0 * log(sm.s1) - log(sm.s2) - lt;
        if (g >= 0.0)
          lo = x;
        else
          up = x;
        double gp = 2.0 * (sm.s1x / sm.s1 - sm.s2x / sm.s2);
        double xn = x - g / gp;
        if (!(xn > lo && xn < up)) xn = 0.5 * (lo + up);
        if (fabs(xn - x) <= 1e-13 * x || !(up - lo > 1e-13 * up)) {
          // converged; if Newton approached from above, lo may still be far below:
          // evaluate just under the lowest point known to be above the root
          const double xb = up * (1.0 - 2e-13);
          if (xb > lo && up - lo > 2e-13 * up) {
            EssSums sb = ess_sums(lnl, n, mx, xb, red);
            if (2.0 * log(sb.s1) - log(sb.s2) - lt >= 0.0) lo = xb;
          }
          break;
        }
        x = xn;
      }
      if (threadIdx.x == 0) sh_db = lo;
    }
  }
  __syncthreads();
  const double db = sh_db;
  // weights, ESS and evidence increment
  double s1 = 0, s2 = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double l = lnl[i];
    double w = isfinite(l) ? exp(db * (l - mx)) : 0.0;
    w_out[i] = w;
    s1 += w;
    s2 += w * w;
  }
  s1 = block_sum(s1, red);
  s2 = block_sum(s2, red);
  // inclusive prefix sums of q_i = floor(W_i 2^32): contiguous chunk per thread
  const int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
  const int64_t b0 = threadIdx.x * chunk;
  const int64_t b1 = b0 + chunk < n ? b0 + chunk : n;
  unsigned long long loc = 0;
  for (int64_t i = b0; i < b1; ++i) loc += (unsigned long long)floor(w_out[i] * 4294967296.0);
  carry[threadIdx.x] = loc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long run = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      unsigned long long v = carry[t];
      carry[t] = run;
      run += v;
    }
  }
  __syncthreads();
  unsigned long long run = carry[threadIdx.x];
  for (int64_t i = b0; i < b1; ++i) {
    run += (unsigned long long)floor(w_out[i] * 4294967296.0);
    csum[i] = run;
  }
  if (threadIdx.x == 0) {
    double bn = (db >= 1.0 - beta_prev) ? 1.0 : beta_prev + db;
    double dl = db * mx + log(s1) - log((double)n);
    *beta_next = bn;
    *dlnz = dl;
    *ess_out = s1 * s1 / s2;
    if (lnz_acc) {
      lnz_acc[0] += dl;
      lnz_acc[1] += 1.0;
    }
    if (beta_state) *beta_state = bn;
  }
  // weighted covariance of theta under W (mean-centred, two passes)
  if (cov) {
    double mu[kMaxDim];
    for (int a = 0; a < D; ++a) {
      double s = 0;
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += w_out[i] * theta[i * D + a];
      mu[a] = block_sum(s, red) / s1;
    }
    for (int a = 0; a < D; ++a)
      for (int b = a; b < D; ++b) {
        double s = 0;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
          s += w_out[i] * (theta[i * D + a] - mu[a]) * (theta[i * D + b] - mu[b]);
        s = block_sum(s, red) / s1;
        if (threadIdx.x == 0) {
          cov[a * D + b] = s;
          cov[b * D + a] = s;
        }
      }
  }
}

// p_m = floor((m 2^32 + U) C / (N 2^32)); ancestor = min{ j : C_j > p_m }.
__global__ void systematic_kernel(int64_t n, const unsigned long long* __restrict__ csum, unsigned long long U,
                                  int32_t* __restrict__ anc_out) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  unsigned long long total = csum[n - 1];
  if (total == 0) {
    anc_out[m] = -1;
    return;
  }
  unsigned __int128 x = ((unsigned __int128)(unsigned long long)m << 32) + U;
  unsigned __int128 den = (unsigned __int128)(unsigned long long)n << 32;
  unsigned long long p = (unsigned long long)((x * total) / den);
  int64_t lo = 0, hi = n - 1;  // csum[hi] = total > p
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (csum[mid] > p)
      hi = mid;
    else
      lo = mid + 1;
  }
  anc_out[m] = (int32_t)lo;
}

// Quantise W, build the prefix sums (single CTA).
__global__ void __launch_bounds__(kSmcThreads)
prefix_kernel(int64_t n, const double* __restrict__ w, unsigned long long* __restrict__ csum, int* bad) {
  __shared__ unsigned long long carry[kSmcThreads];
  const int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
  const int64_t b0 = threadIdx.x * chunk;
  const int64_t b1 = b0 + chunk < n ? b0 + chunk : n;
  unsigned long long loc = 0;
  int badw = 0;
  for (int64_t i = b0; i < b1; ++i) {
    double v = w[i];
    if (!(v >= 0.0 && v <= 1.0)) {
      badw = 1;
      v = 0.0;
    }
    loc += (unsigned long long)floor(v * 4294967296.0);
  }
  if (badw) atomicExch(bad, 1);
  carry[threadIdx.x] = loc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long run = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      unsigned long long v = carry[t];
      carry[t] = run;
      run += v;
    }
  }
  __syncthreads();
  unsigned long long run = carry[threadIdx.x];
  for (int64_t i = b0; i < b1; ++i) {
    double v = w[i];
    if (!(v >= 0.0 && v <= 1.0)) v = 0.0;
    run += (unsigned long long)floor(v * 4294967296.0);
    csum[i] = run;
  }
}

// Gather theta, lnl, grad from saved copies by ancestor index.
__global__ void gather_kernel(int64_t n, int D, const int32_t* __restrict__ anc, const double* __restrict__ th0,
                              const double* __restrict__ l0, const double* __restrict__ g0, double* __restrict__ th,
                              double* __restrict__ l, double* __restrict__ g) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  int64_t a = anc[m];
  if (a < 0) a = m;
  for (int i = 0; i < D; ++i) th[m * D + i] = th0[a * D + i];
  if (g)
    for (int i = 0; i < D; ++i) g[m * D + i] = g0[a * D + i];
  l[m] = l0[a];
}

}  // namespace sharpy

// Scratch layout of one reweight/resample call (bytes).
static size_t stage_scratch_bytes(int64_t n, int D) {
  return n * sizeof(double)                   // W
         + n * sizeof(unsigned long long)     // C
         + n * sizeof(int32_t) + 16           // ancestors
         + n * sizeof(double) * (2 * D + 1);  // saved theta, grad, lnl
}

namespace sharpy {
// Enqueue one stage (used by the public call and the run driver).
int enqueue_stage(sharpy_ctx* c, int64_t n, double* theta, double* lnl, double* grad, const double* beta_prev_ptr,
                  double beta_prev, double alpha, double u, double* beta_next, double* dlnz, double* ess,
                  int32_t* anc_out, double* cov, double* beta_state, cudaStream_t s) {
  const int D = c->model.n_dim;
  int rc = ensure_scratch(c, stage_scratch_bytes(n, D));
  if (rc) return rc;
  char* p = (char*)c->d_scratch;
  double* W = (double*)p;
  p += n * sizeof(double);
  unsigned long long* C = (unsigned long long*)p;
  p += n * sizeof(unsigned long long);
  int32_t* anc = (int32_t*)p;
  p += ((n * sizeof(int32_t) + 15) / 16) * 16;
  double* th0 = (double*)p;
  double* g0 = th0 + n * D;
  double* l0 = g0 + n * D;
  reweight_kernel<<<1, kSmcThreads, 0, s>>>(n, lnl, theta, D, beta_prev_ptr, beta_prev, alpha, W, C, beta_next,
                                            dlnz, ess, cov, c->d_lnz, beta_state, c->d_status);
  SHARPY_CUDA_TRY(cudaGetLastError());
  unsigned long long U = (unsigned long long)floor(u * 4294967296.0);
  int32_t* a = anc_out ? anc_out : anc;
  unsigned blocks = (unsigned)((n + 255) / 256);
  systematic_kernel<<<blocks, 256, 0, s>>>(n, C, U, a);
  SHARPY_CUDA_TRY(cudaGetLastError());
  SHARPY_CUDA_TRY(cudaMemcpyAsync(th0, theta, n * D * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (grad) SHARPY_CUDA_TRY(cudaMemcpyAsync(g0, grad, n * D * sizeof(double), cudaMemcpyDeviceToDevice, s));
  SHARPY_CUDA_TRY(cudaMemcpyAsync(l0, lnl, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  gather_kernel<<<blocks, 256, 0, s>>>(n, D, a, th0, l0, g0, theta, lnl, grad);
  SHARPY_CUDA_TRY(cudaGetLastError());
  return SHARPY_OK;
}
}  // namespace sharpy

extern "C" {

int sharpy_smc_reweight_resample(sharpy_ctx* c, int64_t n, double* theta, double* lnl, double* grad,
                                 double beta_prev, double alpha, double u, double* beta_next, double* dlnz,
                                 double* ess, int32_t* ancestors, double* cov, sharpy_stream stream) {
  int rc = check_ctx(c, false);
  if (rc) return rc;
  if (n < 1 || n > kMaxParticles || !theta || !lnl || !beta_next || !dlnz || !ess) return SHARPY_EINVAL;
  if (!(u >= 0.0 && u < 1.0) || !(alpha > 0.0 && alpha <= 1.0) || !(beta_prev >= 0.0 && beta_prev <= 1.0))
    return SHARPY_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return enqueue_stage(c, n, theta, lnl, grad, nullptr, beta_prev, alpha, u, beta_next, dlnz, ess, ancestors, cov,
                       nullptr, s);
}

int sharpy_systematic_resample(int64_t n, const double* w, double u, int32_t* anc, sharpy_stream stream) {
  if (n < 1 || n > kMaxParticles || !w || !anc || !(u >= 0.0 && u < 1.0)) return SHARPY_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* C = nullptr;
  int* bad = nullptr;
  if (cudaMallocAsync((void**)&C, n * sizeof(unsigned long long) + 16, s) != cudaSuccess) return SHARPY_ENOMEM;
  bad = (int*)(C + n);
  SHARPY_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
  prefix_kernel<<<1, kSmcThreads, 0, s>>>(n, w, C, bad);
  unsigned long long U = (unsigned long long)floor(u * 4294967296.0);
  systematic_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, C, U, anc);
  cudaError_t e = cudaGetLastError();
  int hbad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(C, s);
  if (e != cudaSuccess) return SHARPY_ECUDA;
  return hbad ? SHARPY_EINVAL : SHARPY_OK;
}

}  // extern "C"

// ------------------------------------------------ allocation-free variant
// Systematic resampling for callers that must not allocate device memory once
// they are running. Its scratch (the prefix sums and an invalid-weight flag)
// is a file-scope device array of fixed size; every device that loads the
// library keeps it until the process exits.
#include <mutex>

namespace sharpy {
constexpr int64_t kStaticResampleMax = (int64_t)1 << 18;  // 262144 particles (2 MiB of scratch)
static __device__ __align__(256) unsigned long long g_resample_scratch[kStaticResampleMax + 32];
constexpr int kStaticMaxDevices = 64;
static unsigned long long* g_resample_scratch_addr[kStaticMaxDevices];
static std::mutex g_resample_scratch_mu;
}  // namespace sharpy

extern "C" int sharpy_systematic_resample_static(int64_t n, const double* w, double u, int32_t* anc,
                                                 sharpy_stream stream) {
  using namespace sharpy;
  if (n < 1 || n > kStaticResampleMax || !w || !anc || !(u >= 0.0 && u < 1.0)) return SHARPY_EINVAL;
  int dev = 0;
  SHARPY_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticMaxDevices) return SHARPY_EINVAL;
  unsigned long long* base = nullptr;
  {
    // One-time set-up per device (the current one): the host-side name of the
    // array is only a stand-in, so fetch its device address.
    std::lock_guard<std::mutex> lock(g_resample_scratch_mu);
    if (!g_resample_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_resample_scratch) != cudaSuccess || !p) return SHARPY_ECUDA;
      g_resample_scratch_addr[dev] = (unsigned long long*)p;
    }
    base = g_resample_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* C = base;
  int* bad = (int*)(base + kStaticResampleMax);
  // the flag must start at zero; the prefix sums are fully rewritten below
  SHARPY_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
  prefix_kernel<<<1, kSmcThreads, 0, s>>>(n, w, C, bad);
  unsigned long long U = (unsigned long long)floor(u * 4294967296.0);
  systematic_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, C, U, anc);
  cudaError_t e = cudaGetLastError();
  int hbad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return SHARPY_ECUDA;
  return hbad ? SHARPY_EINVAL : SHARPY_OK;
}
