// Sample recycling (Sec. 5, "Samples recycling"): the particles of every
// stage t = 1..T form a pool drawn from the mixture (1/T) sum_t p_t,
// p_t = L^beta_t pi / Z_t. Each pooled particle gets its importance weight for
// the final target p_T = L pi / Z_T,
//   ln w_i = ln L_i - ln Z_T - ln[(1/T) sum_t exp(beta_t ln L_i - ln Z_t)],
// and a rejection step (keep i when u_i < w_i / max_j w_j) turns the pool into
// i.i.d. draws of the target, kept in pool order.
#include <cmath>

#include "context.cuh"

using namespace sharpy;

namespace sharpy {

constexpr int kRecThreads = 1024;
constexpr int kRecMaxStages = 1 << 14;
constexpr uint32_t kRngRecycle = 7;  // Philox purpose of the rejection uniforms

// ln w of one pooled particle per thread (FP64; the largest term of the
// mixture sum is factored out).
__global__ void recycle_weights_kernel(int64_t m, int t, const double* __restrict__ lnl,
                                       const double* __restrict__ beta, const double* __restrict__ lnz_t,
                                       double* __restrict__ log_w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double l = lnl[i];
  double mx = -INFINITY;
  for (int s = 0; s < t; ++s) mx = fmax(mx, beta[s] * l - lnz_t[s]);
  double acc = 0.0;
  for (int s = 0; s < t; ++s) acc += exp(beta[s] * l - lnz_t[s] - mx);
  const double ln_mix = mx + log(acc) - log((double)t);
  log_w[i] = l - lnz_t[t - 1] - ln_mix;
}

// Largest ln w, keep flags and their exclusive prefix sums (one CTA: each
// thread owns a contiguous piece of the pool).
__global__ void __launch_bounds__(kRecThreads)
    recycle_keep_kernel(int64_t m, const double* __restrict__ log_w, uint64_t key, int64_t* __restrict__ pos,
                        int64_t* __restrict__ n_keep, double* __restrict__ log_w_max) {
  __shared__ double redd[kRecThreads / 32];
  __shared__ long long redi[kRecThreads / 32];
  __shared__ double s_mx;
  __shared__ long long s_off[kRecThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kRecThreads / 32;
  double mx = -INFINITY;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) mx = fmax(mx, log_w[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) redd[warp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = redd[0];
    for (int w = 1; w < nw; ++w) r = fmax(r, redd[w]);
    s_mx = r;
    *log_w_max = r;
  }
  __syncthreads();
  mx = s_mx;
  const int64_t chunk = (m + kRecThreads - 1) / kRecThreads;
  const int64_t b0 = (int64_t)threadIdx.x * chunk < m ? (int64_t)threadIdx.x * chunk : m;
  const int64_t b1 = b0 + chunk < m ? b0 + chunk : m;
  long long cnt = 0;
  for (int64_t i = b0; i < b1; ++i) {
    double u0, u1;
    uniform2(key, (uint32_t)i, (uint32_t)((uint64_t)i >> 32), kRngRecycle, 0u, &u0, &u1);
    const int k = u0 < exp(log_w[i] - mx) ? 1 : 0;
    pos[i] = k ? 1 : 0;  // flag for now; replaced by the output position below
    cnt += k;
  }
  // exclusive scan of the per-thread counts
  long long inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) redi[warp] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long run = 0;
    for (int w = 0; w < nw; ++w) {
      s_off[w] = run;
      run += redi[w];
    }
    *n_keep = run;
  }
  __syncthreads();
  long long p = s_off[warp] + inc - cnt;
  for (int64_t i = b0; i < b1; ++i) {
    const int64_t k = pos[i];
    pos[i] = k ? p : -1;
    p += k;
  }
}

__global__ void recycle_gather_kernel(int64_t m, int d, const int64_t* __restrict__ pos,
                                      const double* __restrict__ theta, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t p = pos[i];
  if (p < 0) return;
  for (int j = 0; j < d; ++j) out[p * d + j] = theta[i * d + j];
}

}  // namespace sharpy

extern "C" int sharpy_recycle(int64_t m, int d, int t, const double* theta, const double* lnl, const double* beta,
                              const double* lnz_t, uint64_t key, double* log_w, double* out_theta, int64_t* n_out,
                              sharpy_stream stream) {
  if (m < 1 || m > ((int64_t)1 << 31) || d < 1 || d > SHARPY_MAX_DIM || t < 1 || t > kRecMaxStages || !lnl ||
      !beta || !lnz_t || !n_out || (out_theta && !theta))
    return SHARPY_EINVAL;
  for (int s = 0; s < t; ++s)
    if (!std::isfinite(beta[s]) || !std::isfinite(lnz_t[s])) return SHARPY_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // scratch: beta, ln Z_t, ln w (if the caller passes none), positions, count, max
  const size_t bytes = 2 * (size_t)t * sizeof(double) + (size_t)m * sizeof(double) + (size_t)m * sizeof(int64_t) +
                       2 * sizeof(int64_t) + sizeof(double);
  char* buf = nullptr;
  if (cudaMallocAsync((void**)&buf, bytes, s) != cudaSuccess) return SHARPY_ENOMEM;
  double* d_beta = (double*)buf;
  double* d_lnz = d_beta + t;
  double* d_lw = log_w ? log_w : d_lnz + t;
  int64_t* d_pos = (int64_t*)(d_lnz + t + m);
  int64_t* d_n = d_pos + m;
  double* d_mx = (double*)(d_n + 2);
  int64_t h_n = 0;
  cudaError_t e = cudaMemcpyAsync(d_beta, beta, t * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_lnz, lnz_t, t * sizeof(double), cudaMemcpyHostToDevice, s);
  const unsigned blocks = (unsigned)((m + 255) / 256);
  if (e == cudaSuccess) {
    recycle_weights_kernel<<<blocks, 256, 0, s>>>(m, t, lnl, d_beta, d_lnz, d_lw);
    recycle_keep_kernel<<<1, kRecThreads, 0, s>>>(m, d_lw, key, d_pos, d_n, d_mx);
    if (out_theta) recycle_gather_kernel<<<blocks, 256, 0, s>>>(m, d, d_pos, theta, out_theta);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_n, d_n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(buf, s);
  if (e != cudaSuccess) return SHARPY_ECUDA;
  *n_out = h_n;
  return SHARPY_OK;
}
