// sweep_f32_noaf.cu -- FP32 sweeps without the antidiffusion stage (the
// transport alone, A = 0): an ablation measuring what antidiffusion and
// flux limiter cost (Sec. 4, the with / without anti-flux comparison).
#include "sweep_launch.cuh"

namespace shasta {

cudaError_t prepare_sweep_f32_noaf(int occupancy[3][3][2]) {
  return launch::prepare<fast::REC_F32, launch::NOAF>(occupancy);
}

cudaError_t launch_sweep_f32_noaf(const SweepParams& P, int axis, int eos, cudaStream_t s) {
  return launch::launch_single<fast::REC_F32, launch::NOAF>(P, axis, eos, s);
}

}  // namespace shasta
