// noalloc.cu -- grid totals of caller-owned fields without any allocation.
//
// Some callers cannot allocate device memory at the point where they want
// the conserved totals: code that runs inside another framework's memory
// pool or allocator (where a cudaMalloc would bypass its accounting, or
// synchronise the device), and code that must not allocate after start-up
// at all.  For them shasta_totals_noalloc computes the same five sums as
// shasta_totals, but its per-block partial sums live in the fixed array
// below, which the CUDA runtime creates when it loads this library's device
// code on a GPU and keeps until the process exits.  Nothing here calls
// cudaMalloc, cudaFree or any routine that allocates device memory.
#include <cuda_runtime.h>

#include "../../include/shasta.h"
#include "kernels.h"

using namespace shasta;

namespace {

// One partial sum per block and field.  Each block sums a fixed run of cells,
// so the array bounds the number of cells one call can take.
constexpr size_t kCellsPerBlock = SHASTA_TOTALS_NOALLOC_CELLS_PER_BLOCK;
constexpr int kMaxBlocks = (int)(SHASTA_TOTALS_NOALLOC_MAX_CELLS / kCellsPerBlock);
static_assert((size_t)kMaxBlocks * kCellsPerBlock == SHASTA_TOTALS_NOALLOC_MAX_CELLS,
              "the cell limit is a whole number of blocks");

static __device__ __align__(256) double g_totals_scratch[5 * kMaxBlocks];

// Device address of g_totals_scratch on the current device.  It is looked up
// on every call rather than cached: after a device reset (or any teardown of
// the primary context) the runtime loads this module again, possibly at
// another address, and a cached pointer would then be stale.  The lookup is
// a table search in the runtime and allocates nothing.
shasta_status scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SHASTA_ECUDA;
  double* p = nullptr;
  if (cudaGetSymbolAddress((void**)&p, g_totals_scratch) != cudaSuccess || !p)
    return SHASTA_ECUDA;
  *out = p;
  return SHASTA_OK;
}

}  // namespace

extern "C" shasta_status shasta_totals_noalloc(const double* E, const double* Mx, const double* My,
                                               const double* Mz, const double* R, size_t n,
                                               double* out, void* stream) {
  if (!out) return SHASTA_EINVAL;
  if (n > SHASTA_TOTALS_NOALLOC_MAX_CELLS) return SHASTA_EINVAL;
  if (n && (!E || !Mx || !My || !Mz || !R)) return SHASTA_EINVAL;
  double* scratch = nullptr;
  shasta_status st = scratch_for_current_device(&scratch);
  if (st != SHASTA_OK) return st;
  FieldView f{};
  const double* in[5] = {E, Mx, My, Mz, R};
  for (int k = 0; k < 5; ++k) {
    f.p[k] = const_cast<double*>(in[k]);
    f.s[k] = 1;
  }
  // Every partial the final pass reads is written by the first pass of the
  // same call, so nothing left in the array by an earlier call is used.
  int nb = (int)((n + kCellsPerBlock - 1) / kCellsPerBlock);
  cudaError_t e = launch_totals_chunked(f, n, 0, kCellsPerBlock, nb, scratch, out,
                                        static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SHASTA_OK : SHASTA_ECUDA;
}
