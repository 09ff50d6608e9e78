// alu_peak.cu -- measured FP32 and FP64 CUDA-core throughput of this GPU.
//
// The sweep kernels are bound by instruction issue and arithmetic, not by
// memory traffic alone, so their reports need the arithmetic roof beside
// the HBM roof.  This is a plain measurement: every thread runs independent
// chains of dependent fused multiply-adds (enough chains and resident warps
// to hide the pipe latency), timed with CUDA events on the caller's stream.
// One fused multiply-add counts as two floating-point operations.
#include <cuda_runtime.h>

#include "../../include/shasta.h"

namespace {

constexpr int kChains = 8;    // independent chains per thread
constexpr int kUnroll = 16;   // multiply-adds per chain per loop trip
constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) {
  return __fmaf_rn(a, b, c);
}
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) {
  return __fma_rn(a, b, c);
}

// a <- a*b + c converges to c / (1 - b) for 0 < b < 1: the values stay
// finite and normal however long the chain runs.
template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chains(T* out, int trips, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + 1 + k) * (T)1e-3;
  for (int t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma_t<T>(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  // never true for the arguments below; the store keeps the chains live
  if (s < (T)0) out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
shasta_status measure(int device, void* stream, double* flops, double* seconds) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return SHASTA_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int blocks = sms * 8;  // 2048 threads per SM: 16 warps per scheduler
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * kThreads) != cudaSuccess) return SHASTA_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  shasta_status rc = SHASTA_OK;
  float ms = 0.f;
  int trips = 64;
  const T b = (T)0.999, c = (T)1e-4;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = SHASTA_ECUDA;
    goto done;
  }
  // grow the trip count until one launch takes at least 20 ms
  for (int attempt = 0; attempt < 24; ++attempt) {
    fma_chains<T><<<blocks, kThreads, 0, st>>>(out, trips, b, c);  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r) fma_chains<T><<<blocks, kThreads, 0, st>>>(out, trips, b, c);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      rc = SHASTA_ECUDA;
      goto done;
    }
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms / 3.f >= 20.f || trips >= (1 << 26)) break;
    trips *= 2;
  }
  {
    const double fmas = 3.0 * (double)blocks * kThreads * kChains * kUnroll * (double)trips;
    *flops = 2.0 * fmas / (ms * 1e-3);
    if (seconds) *seconds = ms * 1e-3 / 3.0;
  }
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}

}  // namespace

extern "C" shasta_status shasta_alu_peak(int kind, int device, void* stream, double* flops_per_s,
                                         double* seconds_per_launch) {
  if (!flops_per_s || (kind != SHASTA_ALU_FP32 && kind != SHASTA_ALU_FP64)) return SHASTA_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess)
    return SHASTA_ECUDA;
  shasta_status rc = kind == SHASTA_ALU_FP32
                         ? measure<float>(device, stream, flops_per_s, seconds_per_launch)
                         : measure<double>(device, stream, flops_per_s, seconds_per_launch);
  cudaSetDevice(prev);
  return rc;
}
