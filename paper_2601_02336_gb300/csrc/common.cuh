// Internal definitions shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sharpy.h"

namespace sharpy {

constexpr double kPi = 3.141592653589793238;
constexpr double kTwoPi = 6.283185307179586477;
constexpr double kTsun = 4.925491025543576e-6;               // G Msun / c^3 [s]
constexpr double kMpcSec = 3.085677581491367e22 / 299792458.0;  // 1 Mpc / c [s]
constexpr double kEarthR = 6.371e6;                          // [m]
constexpr double kClight = 299792458.0;                      // [m/s]
constexpr double kEulerGamma = 0.57721566490153286061;
// Phase accumulator offset: for |Psi| < 2^19 turns, Psi + kTurnOffset lies in
// [2^20, 2^21), where the low 32 bits of the FP64 mantissa are the fractional
// turn in units of 2^-32 (wrapping mod 1 turn for free).
constexpr double kTurnOffset = 1572864.0;                    // 1.5 * 2^20
constexpr int kMaxDim = SHARPY_MAX_DIM;
constexpr int kMaxDet = SHARPY_MAX_DET;
constexpr int kNBasis = 9;  // x^5, x^3, x^2, x, ln f, y, y ln f, y^2, f  (x = f^-1/3, y = f^1/3)
constexpr int kNPn = 8;     // the first eight: post-Newtonian phase basis
// The mixed sweep's split of the post-Newtonian basis: terms accumulated in
// FP64 (x^5, x^3, x^2, ln f) and terms formed in FP32 pairs (x, y, y ln f, y^2).
__host__ __device__ constexpr int large_pn(int i) { return i < 3 ? i : 4; }
__host__ __device__ constexpr int small_pn(int i) { return i == 0 ? 3 : i + 4; }
__host__ __device__ constexpr bool is_large_pn(int j) { return j < 3 || j == 4; }

// Staged tables of a long segment (K >= kStageMinBins): one contiguous record
// per block of kStageBins bins, so that one bulk copy brings a block's tables
// into shared memory. Record layout (bins g kStageBins + i, i < kStageBins;
// zeros past the last bin):
//   float  b32[9][kStageBins]       basis functions, FP32 hi parts
//   float  lo[5][kStageBins]        FP32 lo parts of x, y, y ln f, y^2 and f
//   double b64[4][kStageBins]       x^5, x^3, x^2, ln f in FP64
//   float2 e32[n_det][kStageBins]   pre-whitened data
// Every offset and the record size are multiples of 16 bytes.
constexpr int kStageBins = 256;
constexpr int64_t kStageMinBins = 65536;
__host__ __device__ constexpr int stage_off_lo() { return kNBasis * kStageBins * 4; }
__host__ __device__ constexpr int stage_off_b64() { return stage_off_lo() + 5 * kStageBins * 4; }
__host__ __device__ constexpr int stage_off_e32() { return stage_off_b64() + 4 * kStageBins * 8; }
__host__ __device__ constexpr int stage_rec_bytes(int n_det) { return stage_off_e32() + n_det * kStageBins * 8; }
// row of basis function j among the staged lo parts (j = 3, 5, 6, 7, 8) and FP64 rows (j = 0, 1, 2, 4)
__host__ __device__ constexpr int stage_lo_row(int j) { return j == 3 ? 0 : j == 5 ? 1 : j == 6 ? 2 : j == 7 ? 3 : 4; }
__host__ __device__ constexpr int stage_b64_row(int j) { return j == 4 ? 3 : j; }
static_assert(stage_off_lo() % 16 == 0 && stage_off_b64() % 16 == 0 && stage_off_e32() % 16 == 0 &&
                  stage_rec_bytes(1) % 16 == 0,
              "bulk copies move multiples of 16 bytes between 16-byte aligned addresses");

// Model configuration as passed to kernels (by value).
struct DevModel {
  int model;
  int n_dim;
  int phys[kMaxDim];
  double lo[kMaxDim], hi[kMaxDim];
  int prior[kMaxDim];
  int boundary[kMaxDim];
  double fixed[SHARPY_NPHYS];
  int n_comp;
  double mix_logw[SHARPY_MAX_COMP];
  double mix_mu[SHARPY_MAX_COMP][kMaxDim];
  double mix_sigma[SHARPY_MAX_COMP][kMaxDim];
};

struct DevDetector {
  int fixed_response;
  double fplus, fcross, delay;
  double D[3][3];  // detector tensor (x x^T - y y^T)/2
  float Df[3][3];  // the same in FP32 (antenna patterns of the mixed path)
  double r[3];     // position [m]
  double rcd[3];   // position / c [s]
  float rcf[3];    // the same in FP32 (delays of the mixed path)
};

// Staged event tables (device pointers, SoA), built by sharpy_set_data.
struct DevEvent {
  int n_det;
  int64_t n_bins;
  double f_min, df;
  double inv_df;             // 1 / df (k_ISCO guess; the table decides)
  double dd;                 // <d|d> over all bins and detectors
  float ddh_hi, ddh_lo;      // -<d|d>/2 as a double-float: hi = (float)x, lo = (float)(x - hi)
  const double* f;           // [K] f_k
  const double* b64;         // [kNBasis][K] basis functions (FP64)
  const float* b32;          // [kNBasis][K] basis functions (FP32, = hi part)
  const float* b32lo;        // [kNBasis][K] B - (double)hi (FP32 lo part)
  const double2* e64;        // [n_det][K] E = w conj(d) f^-7/6 (FP64)
  const float2* e32;         // [n_det][K] same, FP32
  const double* pref;        // [n_det][K] prefix sums of w f^-7/3
  const double* p1;          // [n_det][kNBasis][K] prefix sums of w f^-7/3 B_m (Fisher), or null
  const double* p2;          // [n_det][kNBasis (kNBasis + 1) / 2][K] ... B_m B_n, m <= n, or null
  const unsigned char* stage;  // staged records (see stage_rec_bytes), or null for K < kStageMinBins
  int stage_blocks;            // records: ceil(K / kStageBins)
  DevDetector det[kMaxDet];
};

// Sticky status word: the first error recorded wins.
__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__host__ __device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                       uint32_t k0, uint32_t k1, uint32_t out[4]) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// Random-number purposes (third counter word).
enum { RNG_PRIOR = 1, RNG_MOMENTUM = 2, RNG_DIRECTION = 3, RNG_LEAF = 4, RNG_TOP = 5, RNG_RESAMPLE = 6 };

// Uniform in (0,1) with 53 random bits from two 32-bit words.
__host__ __device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  uint64_t m = ((uint64_t)a << 21) | (uint64_t)(b >> 11);
  return ((double)m + 0.5) * 1.1102230246251565404e-16;  // 2^-53
}

__host__ __device__ __forceinline__ void uniform2(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2,
                                                  uint32_t c3, double* u0, double* u1) {
  uint32_t x[4];
  philox4x32_10(c0, c1, c2, c3, (uint32_t)key, (uint32_t)(key >> 32), x);
  *u0 = u53(x[0], x[1]);
  *u1 = u53(x[2], x[3]);
}

// ----------------------------------------------------------- warp helpers
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace sharpy

// Host-side error plumbing.
#define SHARPY_CUDA_TRY(expr)                  \
  do {                                         \
    cudaError_t _e = (expr);                   \
    if (_e != cudaSuccess) return SHARPY_ECUDA; \
  } while (0)
