// sweep_mixed.cu -- MIXED: state, transport and limiter in float; the recovery's E^2 - |M|^2 in double-float.
#include <mutex>

#include "kernels.h"
#include "sweep_fast.cuh"

namespace shasta {

namespace {

constexpr int kWarps = 4, kRing = 8, kDist = 3;

template <int EOS, int AXIS, int MINB>
void* kfun() {
  return (void*)fast::sweep_fast_kernel<EOS, AXIS, true, kWarps, kRing, kDist, MINB>;
}

template <int AXIS>
size_t smem_bytes() {
  return (size_t)kWarps * fast::Smem<AXIS, kRing>::per_warp * sizeof(float);
}

// kernel of (eos, axis, variant); variant 0: registers capped for 3 CTAs
// (12 warps) per SM, 1: uncapped
void* kernel_of(int eos, int axis, int variant) {
  static void* const table[2][3][2] = {
      {{kfun<EOS_IDEAL, 0, 3>(), kfun<EOS_IDEAL, 0, 1>()},
       {kfun<EOS_IDEAL, 1, 3>(), kfun<EOS_IDEAL, 1, 1>()},
       {kfun<EOS_IDEAL, 2, 3>(), kfun<EOS_IDEAL, 2, 1>()}},
      {{kfun<EOS_BAG, 0, 3>(), kfun<EOS_BAG, 0, 1>()},
       {kfun<EOS_BAG, 1, 3>(), kfun<EOS_BAG, 1, 1>()},
       {kfun<EOS_BAG, 2, 3>(), kfun<EOS_BAG, 2, 1>()}}};
  return table[eos][axis][variant];
}

size_t smem_of(int axis) { return axis == 0 ? smem_bytes<0>() : (axis == 1 ? smem_bytes<1>() : smem_bytes<2>()); }

}  // namespace

cudaError_t prepare_sweep_mixed(int occupancy[2][3][2]) {
  for (int eos = 0; eos < 2; ++eos)
    for (int axis = 0; axis < 3; ++axis)
      for (int var = 0; var < 2; ++var) {
        const void* k = kernel_of(eos, axis, var);
        const size_t smem = smem_of(axis);
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWarps * 32, smem);
        if (e != cudaSuccess) return e;
        occupancy[eos][axis][var] = per_sm * kWarps;
      }
  return cudaSuccess;
}

cudaError_t launch_sweep_mixed(const SweepParams& P, int axis, int eos, cudaStream_t s) {
  if (P.plane <= 0) return cudaSuccess;
  if (axis < 0 || axis > 2 || eos < 0 || eos > 1 || P.variant < 0 || P.variant > 1 || P.blocks < 1)
    return cudaErrorInvalidValue;
  void* args[] = {const_cast<SweepParams*>(&P)};
  return cudaLaunchKernel(kernel_of(eos, axis, P.variant), dim3((unsigned)P.blocks), dim3(kWarps * 32),
                          args, smem_of(axis), s);
}

int sweep_warps_per_block_mixed() { return kWarps; }

}  // namespace shasta
