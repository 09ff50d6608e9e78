// batch_f32.cu -- batched FP32 sweeps: one launch over the work list of many
// events.
#include "sweep_launch.cuh"

namespace shasta {

cudaError_t prepare_batch_f32(int occupancy[3][3][2]) {
  return launch::prepare<fast::REC_F32, launch::BATCH>(occupancy);
}

cudaError_t launch_batch_f32(const SweepParams& P, const BatchList& L, int axis, int eos,
                             cudaStream_t s) {
  return launch::launch_batch<fast::REC_F32>(P, L, axis, eos, s);
}

}  // namespace shasta
