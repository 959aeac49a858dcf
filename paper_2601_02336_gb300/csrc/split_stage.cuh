// Staged records of a long segment for the split sweep (SHARPY_MIXED_SPLIT),
// which forms every phase term from FP32 hi/lo pairs and so reads the lo
// parts of all nine basis functions and no FP64 table. They follow the mixed
// sweep's records (common.cuh) in the same allocation: record g of the split
// set starts at stage_blocks * stage_rec_bytes(n_det) + g * split_rec_bytes(n_det).
// Layout (bins g kStageBins + i, i < kStageBins; zeros past the last bin):
//   float  b32[9][kStageBins]       basis functions, FP32 hi parts
//   float  lo[9][kStageBins]        their FP32 lo parts
//   float2 e32[n_det][kStageBins]   pre-whitened data
#pragma once
#include "common.cuh"

namespace sharpy {

__host__ __device__ constexpr int split_off_lo() { return kNBasis * kStageBins * 4; }
__host__ __device__ constexpr int split_off_e32() { return 2 * kNBasis * kStageBins * 4; }
__host__ __device__ constexpr int split_rec_bytes(int n_det) { return split_off_e32() + n_det * kStageBins * 8; }
__host__ __device__ constexpr size_t split_set_offset(int stage_blocks, int n_det) {
  return (size_t)stage_blocks * stage_rec_bytes(n_det);
}
static_assert(split_off_lo() % 16 == 0 && split_off_e32() % 16 == 0 && split_rec_bytes(1) % 16 == 0,
              "bulk copies need 16-byte multiples");

// The split sweep's table values of bin i of a split record in shared memory:
// the values GlobalBin reads from the SoA tables, so the same sums.
struct StagedSplitBin {
  const unsigned char* rec;
  int i;
  __device__ __forceinline__ float b32(int j) const { return reinterpret_cast<const float*>(rec)[j * kStageBins + i]; }
  __device__ __forceinline__ float b32lo(int j) const {
    return reinterpret_cast<const float*>(rec + split_off_lo())[j * kStageBins + i];
  }
  // not read by the split sweep (its phase has no FP64 term); hi + lo for completeness
  __device__ __forceinline__ double b64(int j) const { return (double)b32(j) + (double)b32lo(j); }
  __device__ __forceinline__ float2 e32(int a) const {
    return reinterpret_cast<const float2*>(rec + split_off_e32())[a * kStageBins + i];
  }
};

}  // namespace sharpy
