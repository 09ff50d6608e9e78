// batch_mixed.cu -- batched MIXED sweeps: one launch over the work list of
// many events.
#include "sweep_launch.cuh"

namespace shasta {

cudaError_t prepare_batch_mixed(int occupancy[3][3][2]) {
  return launch::prepare<fast::REC_DF, launch::BATCH>(occupancy);
}

cudaError_t launch_batch_mixed(const SweepParams& P, const BatchList& L, int axis, int eos,
                               cudaStream_t s) {
  return launch::launch_batch<fast::REC_DF>(P, L, axis, eos, s);
}

}  // namespace shasta
