// sweep_mixed64.cu -- MIXED_FP64: state, transport and limiter in float;
// the recovery (D = E^2 - |M|^2, the root, p and the velocity along the
// sweep) in double from the float state.
#include "sweep_launch.cuh"

namespace shasta {

cudaError_t prepare_sweep_mixed64(int occupancy[3][3][2]) {
  return launch::prepare<fast::REC_F64, launch::SINGLE>(occupancy);
}

cudaError_t launch_sweep_mixed64(const SweepParams& P, int axis, int eos, cudaStream_t s) {
  return launch::launch_single<fast::REC_F64>(P, axis, eos, s);
}

int sweep_warps_per_block_mixed64() { return launch::kWarps; }

}  // namespace shasta
