// sharpy_probe_peaks: FP32 / FP64 FMA and SFU sin+cos throughput of the current
// device, measured with register-only kernels (the roofline denominators of the
// ALU-bound sweep).
#include "context.cuh"

namespace sharpy {

constexpr int kProbeIters = 1024;

__global__ void probe_f32(float* out, float a, float b) {
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = threadIdx.x + j;
  for (int i = 0; i < kProbeIters; ++i)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = fmaf(x[j], a, b);
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_f64(double* out, double a, double b) {
  double x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = threadIdx.x + j;
  for (int i = 0; i < kProbeIters / 16; ++i)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_sfu(float* out, float a) {
  float x[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) x[j] = threadIdx.x * 1e-3f + 0.1f * j;
  for (int i = 0; i < kProbeIters / 4; ++i)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      x[0] = __sinf(x[0]) + a;
      x[1] = __cosf(x[1]) + a;
      x[2] = __sinf(x[2]) + a;
      x[3] = __cosf(x[3]) + a;
    }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] + x[1] + x[2] + x[3];
}

}  // namespace sharpy

extern "C" int sharpy_probe_peaks(int device, double* out) {
  using namespace sharpy;
  if (!out) return SHARPY_EINVAL;
  SHARPY_CUDA_TRY(cudaSetDevice(device));
  cudaDeviceProp p;
  SHARPY_CUDA_TRY(cudaGetDeviceProperties(&p, device));
  const int blocks = p.multiProcessorCount * 8, threads = 256;
  const double n = (double)blocks * threads;
  void* buf = nullptr;
  SHARPY_CUDA_TRY(cudaMalloc(&buf, (size_t)blocks * threads * sizeof(double)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best[3] = {0, 0, 0};
  for (int rep = 0; rep < 3; ++rep) {
    float ms;
    cudaEventRecord(e0);
    probe_f32<<<blocks, threads>>>((float*)buf, 0.999f, 0.001f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    best[0] = fmax(best[0], n * kProbeIters * 32 * 2 / (ms * 1e-3) / 1e12);
    cudaEventRecord(e0);
    probe_f64<<<blocks, threads>>>((double*)buf, 0.999, 0.001);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    best[1] = fmax(best[1], n * (kProbeIters / 16) * 32 * 2 / (ms * 1e-3) / 1e12);
    cudaEventRecord(e0);
    probe_sfu<<<blocks, threads>>>((float*)buf, 0.5f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    best[2] = fmax(best[2], n * (kProbeIters / 4) * 16 / (ms * 1e-3) / 1e9);
  }
  cudaError_t e = cudaDeviceSynchronize();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) return SHARPY_ECUDA;
  out[0] = best[0];
  out[1] = best[1];
  out[2] = best[2];
  return SHARPY_OK;
}
