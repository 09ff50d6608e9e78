// sweep_f32.cu -- FP32: state, transport, limiter and recovery in float.
#include "sweep_launch.cuh"

namespace shasta {

cudaError_t prepare_sweep_f32(int occupancy[3][3][2]) {
  return launch::prepare<fast::REC_F32, launch::SINGLE>(occupancy);
}

cudaError_t launch_sweep_f32(const SweepParams& P, int axis, int eos, cudaStream_t s) {
  return launch::launch_single<fast::REC_F32>(P, axis, eos, s);
}

int sweep_warps_per_block_f32() { return launch::kWarps; }

}  // namespace shasta
