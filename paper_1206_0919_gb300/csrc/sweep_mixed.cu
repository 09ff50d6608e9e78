// sweep_mixed.cu -- MIXED: state, transport and limiter in float; the
// recovery's E^2 - |M|^2 in double-float.
#include "sweep_launch.cuh"

namespace shasta {

cudaError_t prepare_sweep_mixed(int occupancy[3][3][2]) {
  return launch::prepare<fast::REC_DF, launch::SINGLE>(occupancy);
}

cudaError_t launch_sweep_mixed(const SweepParams& P, int axis, int eos, cudaStream_t s) {
  return launch::launch_single<fast::REC_DF>(P, axis, eos, s);
}

int sweep_warps_per_block_mixed() { return launch::kWarps; }

}  // namespace shasta
