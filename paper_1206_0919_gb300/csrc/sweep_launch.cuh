// sweep_launch.cuh -- kernel tables and launchers of the streaming FP32 /
// MIXED sweeps (sweep_fast.cuh), one instantiation per including unit.
#pragma once

#include "kernels.h"
#include "sweep_fast.cuh"

namespace shasta {
namespace launch {

constexpr int kWarps = 4, kRing = 8, kDist = 3;

// Kernel families: one event, a batch, one event without antidiffusion
// (FP32 only).
enum Kind { SINGLE = 0, BATCH = 1, NOAF = 2 };

// Tabulated EoS: single-event FP32 kernels only (MIXED's double-float
// applies to the closed forms; batches take closed-form EoS).
template <int REC, int KIND, int EOS, int AXIS, int MINB>
void* kfun() {
  if constexpr (EOS == EOS_TABLE && (REC != fast::REC_F32 || KIND != SINGLE))
    return nullptr;
  else if constexpr (KIND == BATCH)
    return (void*)fast::sweep_batch_kernel<EOS, AXIS, REC, kWarps, kRing, kDist, MINB>;
  else if constexpr (KIND == NOAF)
    return (void*)fast::sweep_noaf_kernel<EOS, AXIS, kWarps, kRing, kDist, MINB>;
  else
    return (void*)fast::sweep_fast_kernel<EOS, AXIS, REC, kWarps, kRing, kDist, MINB>;
}

template <int AXIS>
size_t smem_bytes() {
  return (size_t)kWarps * fast::Smem<AXIS, kRing>::per_warp * sizeof(float);
}

inline size_t smem_of(int axis) {
  return axis == 0 ? smem_bytes<0>() : (axis == 1 ? smem_bytes<1>() : smem_bytes<2>());
}

// Kernel of (eos, axis, variant); variant 0: registers capped for 3 CTAs
// (12 warps) per SM, 1: uncapped.  Null where the family has no such EoS.
template <int REC, int KIND>
void* kernel_of(int eos, int axis, int variant) {
  static void* const table[3][3][2] = {
      {{kfun<REC, KIND, EOS_IDEAL, 0, 3>(), kfun<REC, KIND, EOS_IDEAL, 0, 1>()},
       {kfun<REC, KIND, EOS_IDEAL, 1, 3>(), kfun<REC, KIND, EOS_IDEAL, 1, 1>()},
       {kfun<REC, KIND, EOS_IDEAL, 2, 3>(), kfun<REC, KIND, EOS_IDEAL, 2, 1>()}},
      {{kfun<REC, KIND, EOS_BAG, 0, 3>(), kfun<REC, KIND, EOS_BAG, 0, 1>()},
       {kfun<REC, KIND, EOS_BAG, 1, 3>(), kfun<REC, KIND, EOS_BAG, 1, 1>()},
       {kfun<REC, KIND, EOS_BAG, 2, 3>(), kfun<REC, KIND, EOS_BAG, 2, 1>()}},
      {{kfun<REC, KIND, EOS_TABLE, 0, 3>(), kfun<REC, KIND, EOS_TABLE, 0, 1>()},
       {kfun<REC, KIND, EOS_TABLE, 1, 3>(), kfun<REC, KIND, EOS_TABLE, 1, 1>()},
       {kfun<REC, KIND, EOS_TABLE, 2, 3>(), kfun<REC, KIND, EOS_TABLE, 2, 1>()}}};
  return table[eos][axis][variant];
}

// Sets the shared-memory attribute of every kernel of the table and reports
// resident warps per SM [eos][axis][variant] (0 where there is no kernel).
template <int REC, int KIND>
cudaError_t prepare(int occupancy[3][3][2]) {
  for (int eos = 0; eos < 3; ++eos)
    for (int axis = 0; axis < 3; ++axis)
      for (int var = 0; var < 2; ++var) {
        const void* k = kernel_of<REC, KIND>(eos, axis, var);
        occupancy[eos][axis][var] = 0;
        if (!k) continue;
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

inline bool bad_choice(const SweepParams& P, int axis, int eos) {
  return axis < 0 || axis > 2 || eos < 0 || eos > 2 || P.variant < 0 || P.variant > 1 ||
         P.blocks < 1;
}

template <int REC, int KIND = SINGLE>
cudaError_t launch_single(const SweepParams& P, int axis, int eos, cudaStream_t s) {
  if (P.plane <= 0) return cudaSuccess;
  if (bad_choice(P, axis, eos)) return cudaErrorInvalidValue;
  void* args[] = {const_cast<SweepParams*>(&P)};
  void* k = kernel_of<REC, KIND>(eos, axis, P.variant);
  if (!k) return cudaErrorInvalidValue;
  return cudaLaunchKernel(k, dim3((unsigned)P.blocks),
                          dim3(kWarps * 32), args, smem_of(axis), s);
}

template <int REC>
cudaError_t launch_batch(const SweepParams& P, const BatchList& L, int axis, int eos,
                         cudaStream_t s) {
  if (L.nlist <= 0) return cudaSuccess;
  if (bad_choice(P, axis, eos) || !L.ev || !L.idx || !L.prefix) return cudaErrorInvalidValue;
  void* args[] = {const_cast<SweepParams*>(&P), const_cast<BatchList*>(&L)};
  void* k = kernel_of<REC, BATCH>(eos, axis, P.variant);
  if (!k) return cudaErrorInvalidValue;
  return cudaLaunchKernel(k, dim3((unsigned)P.blocks),
                          dim3(kWarps * 32), args, smem_of(axis), s);
}

}  // namespace launch
}  // namespace shasta
