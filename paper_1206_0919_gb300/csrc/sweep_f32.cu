// sweep_f32.cu -- FP32: state, transport, limiter and recovery in float.
#include "kernels.h"

namespace shasta {

template <int EOS, int AXIS>
static cudaError_t go(const SweepParams& P, cudaStream_t s) {
  const int threads = 128;
  long long blocks = (P.plane + threads - 1) / threads;
  sweep_kernel<float, float, EOS, AXIS, true><<<(unsigned)blocks, threads, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_sweep_f32(const SweepParams& P, int axis, int eos, cudaStream_t s) {
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
