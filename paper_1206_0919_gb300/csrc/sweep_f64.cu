// sweep_f64.cu -- FP64 instances of the fused sweep.  Built with
// -fmad=false and IEEE division / square root so that the arithmetic is the
// plain double-precision evaluation of each expression in source order.
#include "kernels.h"

namespace shasta {

template <int EOS, int AXIS>
static cudaError_t go(const SweepParams& P, cudaStream_t s) {
  const int threads = 128;
  const int L = P.range_len > 0 && P.range_len < P.n ? (int)P.range_len : P.n;
  const long long work = P.plane * ((P.n + L - 1) / L);
  long long blocks = (work + threads - 1) / threads;
  sweep_kernel<double, double, EOS, AXIS, false><<<(unsigned)blocks, threads, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_sweep_f64(const SweepParams& P, int axis, int eos, cudaStream_t s) {
  if (P.plane <= 0) return cudaSuccess;
  switch (eos * 3 + axis) {
    case 0: return go<EOS_IDEAL, 0>(P, s);
    case 1: return go<EOS_IDEAL, 1>(P, s);
    case 2: return go<EOS_IDEAL, 2>(P, s);
    case 3: return go<EOS_BAG, 0>(P, s);
    case 4: return go<EOS_BAG, 1>(P, s);
    case 5: return go<EOS_BAG, 2>(P, s);
    case 6: return go<EOS_TABLE, 0>(P, s);
    case 7: return go<EOS_TABLE, 1>(P, s);
    case 8: return go<EOS_TABLE, 2>(P, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace shasta
