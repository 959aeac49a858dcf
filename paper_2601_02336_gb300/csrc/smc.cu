// SMC stage kernels (Sec. 3): adaptive tempering (Eq. 6), weights (Eq. 4),
// ESS (Eq. 5), evidence increment (Sec. 3.1, Eqs. 7-8), weighted covariance,
// integer systematic resampling and gather.
//
// The tempering root is found by one thread-block cluster of kRwCluster CTAs
// per event: FP64 runs at 1/64 of the FP32 rate on this GPU, so the FP64 work
// is spread over the cluster's SMs and cut to a few passes. An FP32 geometric
// grid brackets the root, an FP32 Newton iteration refines it, and an FP64
// Newton iteration finishes on a point verified in FP64. Partial sums meet in
// distributed shared memory in rank order, so every CTA of the cluster holds the
// same totals and takes the same decisions.
#include <cooperative_groups.h>

#include <cmath>

#include "stage.cuh"

namespace cg = cooperative_groups;
using namespace sharpy;

namespace sharpy {

constexpr int kSmcThreads = 1024;  // single-CTA prefix kernel of the plain resampling calls
constexpr int kRwWarps = kRwThreads / 32;
constexpr int kGrid = 54;          // FP32 grid db_m = hi 2^-m
constexpr int kGridChunk = 9;      // grid points per pass
constexpr int kNewton32 = 8;       // FP32 Newton passes at most
constexpr int kCovThreads = 256;

struct RwShared {
  double red[4][kRwWarps];
  double part[4];
  double tot[4];
  float redf[kGridChunk][kRwWarps];
  float partf[kGridChunk];
  float totf[kGridChunk];
  float s1grid[kGrid];
  unsigned long long wtot[kRwWarps];
  unsigned long long ctot;
};

__device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

struct SumOp {
  template <class T>
  __device__ T operator()(T a, T b) const { return a + b; }
};
struct MaxOp {
  __device__ double operator()(double a, double b) const { return fmax(a, b); }
};

// Cluster-wide reduction of K values: warp trees, then the CTA's warps in
// order, then the cluster's CTAs in rank order. Every thread of every CTA gets
// the same totals.
template <int K, class T, class Op>
__device__ __forceinline__ void cluster_reduce(T (&v)[K], T (*red)[kRwWarps], T* part, T* tot, Op op) {
  cg::cluster_group cl = cg::this_cluster();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    T x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = op(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) red[k][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    T r = red[threadIdx.x][0];
    for (int w = 1; w < kRwWarps; ++w) r = op(r, red[threadIdx.x][w]);
    part[threadIdx.x] = r;
  }
  cl.sync();
  if (threadIdx.x < K) {
    T r = *cl.map_shared_rank(&part[threadIdx.x], 0);
    for (int q = 1; q < kRwCluster; ++q) r = op(r, *cl.map_shared_rank(&part[threadIdx.x], q));
    tot[threadIdx.x] = r;
  }
  cl.sync();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = tot[k];
}

// FP32 sums at db over x_i = lnL_i - max (FP32, -inf where lnL is not finite):
// S1 = sum e^{db x}, S2 = sum e^{2 db x}, S1x = sum x e^{db x}, S2x = sum x e^{2 db x}.
__device__ void sums32(const float* xf, int64_t n, int64_t i0, int64_t step, float db, float (&s)[4], RwShared& sh) {
  const float c = db * 1.44269504f;  // log2(e)
  float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int64_t i = i0; i < n; i += step) {
    const float x = xf[i];
    if (!(x > -INFINITY)) continue;
    const float w = exp2f(x * c);
    const float w2 = w * w;
    a[0] += w;
    a[1] += w2;
    a[2] += w * x;
    a[3] += w2 * x;
  }
  cluster_reduce<4, float>(a, sh.redf, sh.partf, sh.totf, SumOp());
#pragma unroll
  for (int k = 0; k < 4; ++k) s[k] = a[k];
}

// The same sums in FP64 from lnL.
__device__ void sums64(const double* lnl, int64_t n, int64_t i0, int64_t step, double mx, double db,
                       double (&s)[4], RwShared& sh) {
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = i0; i < n; i += step) {
    const double l = lnl[i];
    if (!isfinite(l)) continue;
    const double x = l - mx;
    const double w = exp(db * x);
    const double w2 = w * w;
    a[0] += w;
    a[1] += w2;
    a[2] += w * x;
    a[3] += w2 * x;
  }
  cluster_reduce<4, double>(a, sh.red, sh.part, sh.tot, SumOp());
#pragma unroll
  for (int k = 0; k < 4; ++k) s[k] = a[k];
}

// Tempering root, weights, ESS, evidence increment and the integer prefix sums
// of one event (one cluster). Solves ESS(db) = alpha N (Eq. 6) with
// ESS = S1^2 / S2, i.e. g(db) = 2 ln S1 - ln S2 - ln(alpha N) = 0; g decreases
// with db and S2(db) = S1(2 db). Keeps the largest FP64-evaluated db with
// g >= 0 (within 1e-12 of the root); db = 1 - beta_prev when that already
// satisfies ESS >= alpha N.
__global__ void __cluster_dims__(kRwCluster, 1, 1) __launch_bounds__(kRwThreads)
    reweight_cluster_kernel(StageArgs one, const StageArgs* batch) {
  __shared__ RwShared sh;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const StageArgs A = batch ? batch[blockIdx.x / kRwCluster] : one;
  const bool lead = rank == 0 && threadIdx.x == 0;
  // batched driver: every CTA of the cluster reads the same control words and
  // leaves together (clearing `active` only makes the others leave too)
  if (A.active) {
    if (*A.active == 0) return;
    if (*A.beta_prev_ptr >= 1.0 || *A.stage >= A.max_stages) {
      if (lead) *A.active = 0;
      return;
    }
  }
  const double beta_prev = A.beta_prev_ptr ? *A.beta_prev_ptr : A.beta_prev;
  const int64_t n = A.n;
  const int64_t i0 = (int64_t)rank * kRwThreads + threadIdx.x;
  const int64_t step = (int64_t)kRwCluster * kRwThreads;
  double mx = -INFINITY;
  for (int64_t i = i0; i < n; i += step) {
    const double l = A.lnl[i];
    if (isfinite(l)) mx = fmax(mx, l);
  }
  {
    double v[1] = {mx};
    cluster_reduce<1, double>(v, sh.red, sh.part, sh.tot, MaxOp());
    mx = v[0];
  }
  if (!isfinite(mx)) {
    if (lead) {
      set_status(A.status, SHARPY_ENONFINITE);
      if (A.active) *A.active = 0;
    }
    return;
  }
  const double target = A.alpha * (double)n;
  const double lt = log(target);
  const double hi = 1.0 - beta_prev;
  double db = 0.0;
  if (hi > 0.0) {
    float* xf = reinterpret_cast<float*>(A.w);  // FP32 scratch, overwritten by the weights below
    for (int64_t i = i0; i < n; i += step) {
      const double l = A.lnl[i];
      xf[i] = isfinite(l) ? (float)(l - mx) : -INFINITY;
    }
    // FP32 geometric grid: s1grid[m] = S1(hi 2^(1-m)), so
    // g(hi 2^-m) = 2 ln s1grid[m+1] - ln s1grid[m] - ln(alpha N)
    const float c = (float)(hi * 1.4426950408889634);
    for (int c0 = 0; c0 < kGrid; c0 += kGridChunk) {
      float acc[kGridChunk];
#pragma unroll
      for (int k = 0; k < kGridChunk; ++k) acc[k] = 0.0f;
      for (int64_t i = i0; i < n; i += step) {
        const float x = xf[i];
        if (!(x > -INFINITY)) continue;
        const float y = x * c;
#pragma unroll
        for (int k = 0; k < kGridChunk; ++k) acc[k] += exp2f(ldexpf(y, 1 - (c0 + k)));
      }
      cluster_reduce<kGridChunk, float>(acc, sh.redf, sh.partf, sh.totf, SumOp());
      if (threadIdx.x < kGridChunk) sh.s1grid[c0 + threadIdx.x] = acc[threadIdx.x];
    }
    __syncthreads();
    const float ltf = (float)lt;
    const float g_hi = 2.0f * logf(sh.s1grid[1]) - logf(sh.s1grid[0]) - ltf;
    bool all_in = g_hi > 1e-3f;
    if (!all_in && g_hi > -1e-3f) {  // too close to call in FP32
      double sd[4];
      sums64(A.lnl, n, i0, step, mx, hi, sd, sh);
      all_in = 2.0 * log(sd[0]) - log(sd[1]) - lt >= 0.0;
    }
    if (all_in) {
      db = hi;
    } else {
      // bracket [glo, gup]: the largest grid point with ESS >= alpha N and the one above
      int m = 1;
      while (m < kGrid - 1 && 2.0f * logf(sh.s1grid[m + 1]) - logf(sh.s1grid[m]) < ltf) ++m;
      const double glo = (m < kGrid - 1) ? ldexp(hi, -m) : 0.0;
      const double gup = ldexp(hi, 1 - m);
      // FP32 Newton inside the bracket, on t = ln db (g is smooth in t across
      // the decades db spans); FP32 sums carry ~1e-6 relative noise, so a few
      // steps to ~1e-5 are all FP32 can give: the FP64 steps below finish
      float flo = (float)glo, fup = (float)gup;
      float x = glo > 0.0 ? sqrtf(flo * fup) : 0.5f * fup;
      for (int it = 0; it < kNewton32; ++it) {
        float sf[4];
        sums32(xf, n, i0, step, x, sf, sh);
        const float g = 2.0f * logf(sf[0]) - logf(sf[1]) - ltf;
        if (g >= 0.0f)
          flo = x;
        else
          fup = x;
        const float gt = 2.0f * (sf[2] / sf[0] - sf[3] / sf[1]) * x;  // dg / d ln db
        float xn = x * expf(-g / gt);
        if (!(xn > flo && xn < fup)) xn = flo > 0.0f ? sqrtf(flo * fup) : 0.5f * fup;
        const bool done = fabsf(xn - x) <= 1e-5f * x || !(fup - flo > 1e-5f * fup);
        x = xn;
        if (done) break;
      }
      // FP64 Newton from the FP32 root, bracketed by [lo, up] (g(0) >= 0 > g(hi)).
      // Converged (Newton step within 2e-12, or g at its rounding noise): a point
      // with g >= 0 is the answer; from above, step 1e-12 below the root's
      // estimate and evaluate there. Typically 2-3 passes.
      double lo = 0.0, up = hi;
      double xd = (double)x;
      if (!(xd > 0.0 && xd < hi)) xd = glo > 0.0 ? sqrt(glo * gup) : 0.5 * gup;
      for (int it = 0; it < 60; ++it) {
        double sd[4];
        sums64(A.lnl, n, i0, step, mx, xd, sd, sh);
        const double g = 2.0 * log(sd[0]) - log(sd[1]) - lt;
        if (g >= 0.0)
          lo = fmax(lo, xd);
        else
          up = fmin(up, xd);
        const double gp = 2.0 * (sd[2] / sd[0] - sd[3] / sd[1]);
        const double xr = xd - g / gp;  // Newton's estimate of the root
        const bool conv = fabs(xr - xd) <= 2e-12 * xd || fabs(g) <= 1e-13;
        if (conv && g >= 0.0) break;
        double xn = conv ? xr * (1.0 - 1e-12) : xr;
        if (!(xn > lo && xn < up)) xn = lo > 0.0 ? 0.5 * (lo + up) : 0.5 * fmin(xd, up);
        if (!(up - lo > 1e-12 * up)) break;
        xd = xn;
      }
      db = lo;
    }
  }
  // weights, ESS and evidence increment (FP64); every CTA has finished with
  // the FP32 scratch (the last reduction above ended on a cluster barrier)
  double s[2] = {0.0, 0.0};
  for (int64_t i = i0; i < n; i += step) {
    const double l = A.lnl[i];
    const double w = isfinite(l) ? exp(db * (l - mx)) : 0.0;
    A.w[i] = w;
    s[0] += w;
    s[1] += w * w;
  }
  cluster_reduce<2, double>(s, sh.red, sh.part, sh.tot, SumOp());
  // inclusive prefix sums of q_i = floor(W_i 2^32) (exact integers): rank r
  // owns a contiguous block, each thread a contiguous piece of it
  const int64_t cn = (n + kRwCluster - 1) / kRwCluster;
  const int64_t r0 = imin64(n, (int64_t)rank * cn), r1 = imin64(n, r0 + cn);
  const int64_t tn = (r1 - r0 + kRwThreads - 1) / kRwThreads;
  const int64_t b0 = imin64(r1, r0 + (int64_t)threadIdx.x * tn), b1 = imin64(r1, b0 + tn);
  unsigned long long loc = 0;
  for (int64_t i = b0; i < b1; ++i) loc += (unsigned long long)floor(A.w[i] * 4294967296.0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long inc = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sh.wtot[warp] = inc;
  __syncthreads();
  unsigned long long woff = 0, ctot = 0;
  for (int w = 0; w < kRwWarps; ++w) {
    if (w < warp) woff += sh.wtot[w];
    ctot += sh.wtot[w];
  }
  if (threadIdx.x == 0) sh.ctot = ctot;
  cl.sync();
  unsigned long long run = 0;
  for (int q = 0; q < rank; ++q) run += *cl.map_shared_rank(&sh.ctot, q);
  cl.sync();  // no CTA leaves while another may still read its shared memory
  run += woff + inc - loc;
  for (int64_t i = b0; i < b1; ++i) {
    run += (unsigned long long)floor(A.w[i] * 4294967296.0);
    A.csum[i] = run;
  }
  if (lead) {
    const double bn = (db >= hi) ? 1.0 : beta_prev + db;
    const double dl = db * mx + log(s[0]) - log((double)n);
    *A.beta_next = bn;
    *A.dlnz = dl;
    *A.ess = s[0] * s[0] / s[1];
    if (A.sum_w) *A.sum_w = s[0];
    if (A.lnz_acc) {
      A.lnz_acc[0] += dl;
      A.lnz_acc[1] += 1.0;
    }
    if (A.beta_state) *A.beta_state = bn;
    if (A.stage) *A.stage += 1;
  }
}

// Block-wide FP64 sum (warp trees, then the warps in order; 256 threads).
__device__ __forceinline__ double block_sum256(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = red[0];
#pragma unroll
  for (int w = 1; w < kCovThreads / 32; ++w) r += red[w];
  return r;
}

// Weighted covariance of theta under W (before resampling), mean-centred:
// one CTA per entry (a, b), a <= b; blockIdx.y = event.
__global__ void __launch_bounds__(kCovThreads) cov_kernel(StageArgs one, const StageArgs* batch) {
  __shared__ double red[kCovThreads / 32];
  const StageArgs A = batch ? batch[blockIdx.y] : one;
  if (A.active && *A.active == 0) return;
  if (!A.cov) return;
  const int D = A.D;
  int a = 0, p = (int)blockIdx.x;
  while (a < D && p >= D - a) {
    p -= D - a;
    ++a;
  }
  if (a >= D) return;
  const int b = a + p;
  const int64_t n = A.n;
  const double sw = *A.sum_w;
  double sa = 0.0, sb = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double w = A.w[i];
    sa += w * A.theta[i * D + a];
    sb += w * A.theta[i * D + b];
  }
  const double mua = block_sum256(sa, red) / sw;
  const double mub = block_sum256(sb, red) / sw;
  double sc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
    sc += A.w[i] * (A.theta[i * D + a] - mua) * (A.theta[i * D + b] - mub);
  const double c = block_sum256(sc, red) / sw;
  if (threadIdx.x == 0) {
    A.cov[a * D + b] = c;
    A.cov[b * D + a] = c;
  }
}

// Systematic resampling on the integer prefix sums (see systematic_kernel);
// blockIdx.y = event. The batched driver draws the uniform on the device from
// (key, stage), as the single-event run does on the host.
__global__ void systematic_stage_kernel(StageArgs one, const StageArgs* batch, unsigned long long U) {
  const StageArgs A = batch ? batch[blockIdx.y] : one;
  if (A.active && *A.active == 0) return;
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = A.n;
  if (m >= n) return;
  if (A.stage) {
    double u0, u1;
    uniform2(A.key, 0u, (uint32_t)*A.stage, RNG_RESAMPLE, 0u, &u0, &u1);
    U = (unsigned long long)floor(u0 * 4294967296.0);
  }
  const unsigned long long total = A.csum[n - 1];
  if (total == 0) {
    A.anc[m] = -1;
    return;
  }
  const unsigned __int128 x = ((unsigned __int128)(unsigned long long)m << 32) + U;
  const unsigned __int128 den = (unsigned __int128)(unsigned long long)n << 32;
  const unsigned long long pm = (unsigned long long)((x * total) / den);
  int64_t lo = 0, hi = n - 1;  // csum[hi] = total > pm
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (A.csum[mid] > pm)
      hi = mid;
    else
      lo = mid + 1;
  }
  A.anc[m] = (int32_t)lo;
}

// Copy theta, grad, lnL to the gather sources; blockIdx.y = event.
__global__ void save_stage_kernel(StageArgs one, const StageArgs* batch) {
  const StageArgs A = batch ? batch[blockIdx.y] : one;
  if (A.active && *A.active == 0) return;
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= A.n) return;
  const int D = A.D;
  for (int i = 0; i < D; ++i) A.th0[m * D + i] = A.theta[m * D + i];
  if (A.grad)
    for (int i = 0; i < D; ++i) A.g0[m * D + i] = A.grad[m * D + i];
  A.l0[m] = A.lnl[m];
}

// Gather theta, lnL, grad by ancestor; blockIdx.y = event.
__global__ void gather_stage_kernel(StageArgs one, const StageArgs* batch) {
  const StageArgs A = batch ? batch[blockIdx.y] : one;
  if (A.active && *A.active == 0) return;
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= A.n) return;
  const int D = A.D;
  int64_t a = A.anc[m];
  if (a < 0) a = m;
  for (int i = 0; i < D; ++i) A.theta[m * D + i] = A.th0[a * D + i];
  if (A.grad)
    for (int i = 0; i < D; ++i) A.grad[m * D + i] = A.g0[a * D + i];
  A.lnl[m] = A.l0[a];
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


int enqueue_stage_kernels(const StageArgs& one, const StageArgs* batch, int n_events, int64_t max_n, int max_d,
                          bool cov, bool gather, unsigned long long U, cudaStream_t s) {
  const unsigned ne = batch ? (unsigned)n_events : 1u;
  reweight_cluster_kernel<<<ne * kRwCluster, kRwThreads, 0, s>>>(one, batch);
  SHARPY_CUDA_TRY(cudaGetLastError());
  if (cov) {
    dim3 g((unsigned)(max_d * (max_d + 1) / 2), ne);
    cov_kernel<<<g, kCovThreads, 0, s>>>(one, batch);
    SHARPY_CUDA_TRY(cudaGetLastError());
  }
  if (gather) {
    dim3 g((unsigned)((max_n + 255) / 256), ne);
    systematic_stage_kernel<<<g, 256, 0, s>>>(one, batch, U);
    SHARPY_CUDA_TRY(cudaGetLastError());
    save_stage_kernel<<<g, 256, 0, s>>>(one, batch);
    SHARPY_CUDA_TRY(cudaGetLastError());
    gather_stage_kernel<<<g, 256, 0, s>>>(one, batch);
    SHARPY_CUDA_TRY(cudaGetLastError());
  }
  return SHARPY_OK;
}

}  // namespace sharpy

// Scratch layout of one single-event stage (bytes): W, C, ancestors, saved
// theta, grad, lnL, sum of W.
static size_t stage_scratch_bytes(int64_t n, int D) {
  return n * sizeof(double) + n * sizeof(unsigned long long) + ((n * sizeof(int32_t) + 15) / 16) * 16 +
         n * sizeof(double) * (2 * D + 1) + 16;
}

namespace sharpy {
// Enqueue one stage of one event (used by the public call and the run driver).
int enqueue_stage(sharpy_ctx* c, int64_t n, double* theta, double* lnl, double* grad, const double* beta_prev_ptr,
                  double beta_prev, double alpha, double u, double* beta_next, double* dlnz, double* ess,
                  int32_t* anc_out, double* cov, double* beta_state, cudaStream_t s) {
  const int D = c->model.n_dim;
  int rc = ensure_scratch(c, stage_scratch_bytes(n, D));
  if (rc) return rc;
  char* p = (char*)c->d_scratch;
  StageArgs A{};
  A.n = n;
  A.D = D;
  A.theta = theta;
  A.lnl = lnl;
  A.grad = grad;
  A.beta_prev_ptr = beta_prev_ptr;
  A.beta_prev = beta_prev;
  A.alpha = alpha;
  A.w = (double*)p;
  p += n * sizeof(double);
  A.csum = (unsigned long long*)p;
  p += n * sizeof(unsigned long long);
  A.anc = anc_out ? anc_out : (int32_t*)p;
  p += ((n * sizeof(int32_t) + 15) / 16) * 16;
  A.th0 = (double*)p;
  A.g0 = A.th0 + n * D;
  A.l0 = A.g0 + n * D;
  A.sum_w = A.l0 + n;
  A.beta_next = beta_next;
  A.dlnz = dlnz;
  A.ess = ess;
  A.cov = cov;
  A.lnz_acc = c->d_lnz;
  A.beta_state = beta_state;
  A.status = c->d_status;
  const unsigned long long U = (unsigned long long)floor(u * 4294967296.0);
  return enqueue_stage_kernels(A, nullptr, 1, n, D, cov != nullptr, true, U, s);
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
  if (cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess) {
    cudaFreeAsync(C, s);
    return SHARPY_ECUDA;
  }
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
namespace sharpy {
constexpr int64_t kStaticResampleMax = (int64_t)1 << 18;  // 262144 particles (2 MiB of scratch)
static __device__ __align__(256) unsigned long long g_resample_scratch[kStaticResampleMax + 32];
}  // namespace sharpy

extern "C" int sharpy_systematic_resample_static(int64_t n, const double* w, double u, int32_t* anc,
                                                 sharpy_stream stream) {
  using namespace sharpy;
  if (n < 1 || n > kStaticResampleMax || !w || !anc || !(u >= 0.0 && u < 1.0)) return SHARPY_EINVAL;
  // The host-side name of the array is only a stand-in: fetch its device
  // address on the current device, on every call (a lookup, no allocation),
  // so that the address stays right after a device reset or in another
  // context.
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_resample_scratch) != cudaSuccess || !p) return SHARPY_ECUDA;
  unsigned long long* base = (unsigned long long*)p;
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
