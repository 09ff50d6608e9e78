// sweep_mixed.cu -- MIXED: state, transport and limiter in float; the recovery's E^2 - |M|^2 in double-float.
#include "kernels.h"
#include "sweep_fast.cuh"

namespace shasta {

namespace {

constexpr int kWarps = 4, kRing = 8, kDist = 3;

template <int EOS, int AXIS, int MINB>
cudaError_t go2(const SweepParams& P, cudaStream_t s) {
  auto k = fast::sweep_fast_kernel<EOS, AXIS, true, kWarps, kRing, kDist, MINB>;
  const size_t smem = (size_t)kWarps * fast::Smem<AXIS, kRing>::per_warp * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // one wave of resident warps loops over the (line group, segment) items
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWarps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const long long items = ((P.plane + 31) / 32) * P.nseg;
  long long blocks = (items + kWarps - 1) / kWarps;
  const long long wave = (long long)sms * per_sm;
  if (blocks > wave) blocks = wave;
  k<<<(unsigned)blocks, kWarps * 32, smem, s>>>(P);
  return cudaGetLastError();
}

// variant 0: registers capped for 3 CTAs (12 warps) per SM; 1: uncapped.
template <int EOS, int AXIS>
cudaError_t go(const SweepParams& P, cudaStream_t s) {
  return P.variant == 1 ? go2<EOS, AXIS, 1>(P, s) : go2<EOS, AXIS, 3>(P, s);
}

template <int AXIS>
int resident_warps_per_sm(int variant) {
  auto k0 = fast::sweep_fast_kernel<EOS_IDEAL, AXIS, true, kWarps, kRing, kDist, 3>;
  auto k1 = fast::sweep_fast_kernel<EOS_IDEAL, AXIS, true, kWarps, kRing, kDist, 1>;
  const size_t smem = (size_t)kWarps * fast::Smem<AXIS, kRing>::per_warp * sizeof(float);
  int per_sm = 0;
  if (variant == 1) {
    cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k1, kWarps * 32, smem);
  } else {
    cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k0, kWarps * 32, smem);
  }
  return per_sm * kWarps;
}

}  // namespace

int sweep_warps_per_sm_mixed(int axis, int variant) {
  return axis == 0 ? resident_warps_per_sm<0>(variant)
                   : (axis == 1 ? resident_warps_per_sm<1>(variant) : resident_warps_per_sm<2>(variant));
}

cudaError_t launch_sweep_mixed(const SweepParams& P, int axis, int eos, cudaStream_t s) {
  if (P.plane <= 0) return cudaSuccess;
  switch (eos * 3 + axis) {
    case 0: return go<EOS_IDEAL, 0>(P, s);
    case 1: return go<EOS_IDEAL, 1>(P, s);
    case 2: return go<EOS_IDEAL, 2>(P, s);
    case 3: return go<EOS_BAG, 0>(P, s);
    case 4: return go<EOS_BAG, 1>(P, s);
    case 5: return go<EOS_BAG, 2>(P, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace shasta
