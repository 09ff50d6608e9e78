// kernels.h -- launchers shared between the host API and the kernel units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "sweep.cuh"

namespace shasta {

// Fused sweep launchers, one per precision (sweep_f64.cu, sweep_f32.cu,
// sweep_mixed.cu, sweep_mixed64.cu).  Return the launch error.
cudaError_t launch_sweep_f64(const SweepParams& P, int axis, int eos, cudaStream_t s);
cudaError_t launch_sweep_f32(const SweepParams& P, int axis, int eos, cudaStream_t s);
cudaError_t launch_sweep_mixed(const SweepParams& P, int axis, int eos, cudaStream_t s);
cudaError_t launch_sweep_mixed64(const SweepParams& P, int axis, int eos, cudaStream_t s);
// Sets the shared-memory attribute of every FP32 / mixed sweep kernel and
// reports resident warps per SM as [eos][axis][variant].  Call once per
// device before the first launch (and before any stream capture).
cudaError_t prepare_sweep_f32(int occupancy[3][3][2]);
cudaError_t prepare_sweep_mixed(int occupancy[3][3][2]);
cudaError_t prepare_sweep_mixed64(int occupancy[3][3][2]);
int sweep_warps_per_block_f32();
// FP32 sweeps without the antidiffusion stage (sweep_f32_noaf.cu), same
// launch parameters and occupancy layout as the fused FP32 sweeps.
cudaError_t prepare_sweep_f32_noaf(int occupancy[3][3][2]);
cudaError_t launch_sweep_f32_noaf(const SweepParams& P, int axis, int eos, cudaStream_t s);
// The split scheme (sweep_split.cu): one FP32 sweep as recovery, transport
// and antidiffusion kernels with intermediates in device memory.  half_q /
// half_r hold the half-step state (the layout of P.qin / P.rin); scratch
// holds split_scratch_floats(nx, ny, nz) floats.
size_t split_scratch_floats(int nx, int ny, int nz);
cudaError_t launch_sweep_split(const SweepParams& P, int axis, int eos, float* scratch,
                               float* half_q, float* half_r, cudaStream_t s);
int sweep_warps_per_block_mixed();
// The first two sweeps of a step in one launch (sweep_fuse2.cu; FP32,
// reflecting or periodic walls, ideal or bag EoS): along axis_a, then
// axis_b, from P.qin/P.rin to P.qout/P.rout.  prepare_fuse2 sets the
// kernels' shared-memory attribute (once per device, before any capture).
cudaError_t prepare_fuse2();
cudaError_t launch_fuse2(const SweepParams& P, int nx, int ny, int nz, int axis_a, int axis_b,
                         int eos, int sm_count, cudaStream_t s);
int sweep_warps_per_block_mixed64();
// Batched FP32 / MIXED sweeps (one launch over the work list L, all along
// `axis`); prepare_* as above for the batched kernels.
cudaError_t prepare_batch_f32(int occupancy[3][3][2]);
cudaError_t prepare_batch_mixed(int occupancy[3][3][2]);
cudaError_t launch_batch_f32(const SweepParams& P, const BatchList& L, int axis, int eos,
                             cudaStream_t s);
cudaError_t launch_batch_mixed(const SweepParams& P, const BatchList& L, int axis, int eos,
                               cudaStream_t s);

// Where the five fields of a state live: element i of field k is at
// p[k] + i * s[k] (in elements of the storage type).  FP64 states are five
// dense arrays (s = 1); FP32 states keep (E, Mx, My, Mz) as one 16-byte quad
// per cell (p[k] = quad + k, s = 4) and R as a dense array.
struct FieldView {
  void* p[5];
  long long s[5];
};

// Physics constants handed to the auxiliary kernels.
struct EosParams {
  int kind;
  double B, ec;
  double omd;    // 1 - delta
  EosTable tab;  // EOS_TABLE
};

// Auxiliary kernels (aux.cu).  `is32` selects float (1) or double (0) storage.
cudaError_t launch_from_f64(const double* src, void* dst, long long dstride, size_t n, int is32,
                            cudaStream_t s);
cudaError_t launch_to_f64(const void* src, long long sstride, double* dst, size_t n, int is32,
                          cudaStream_t s);
cudaError_t launch_prim2cons(const double* const prim[5], const FieldView& cons, size_t n,
                             int is32, EosParams eos, cudaStream_t s);
cudaError_t launch_recover(const FieldView& cons, double* const prim[6], size_t n, int is32,
                           EosParams eos, cudaStream_t s);
// Counts cells with non-finite values, E < 0 or |M| >= E (cons) or e < 0,
// n < 0, |v| >= 1 (prims) into *count (device).
cudaError_t launch_check_cons(const double* const f[5], size_t n, unsigned long long* count,
                              cudaStream_t s);
cudaError_t launch_check_prims(const double* const f[5], size_t n, unsigned long long* count,
                               cudaStream_t s);
// Totals: per-block partial sums into `partials` (5 * nblocks doubles, device
// scratch), then one block sums them in fixed order into out[5] (device).
int totals_blocks(size_t n);
cudaError_t launch_totals(const FieldView& f, size_t n, int is32, double* partials, double* out,
                          cudaStream_t s);
// The same two-pass totals with an explicit chunk per block and block count
// nb (partials: 5 * nb doubles of scratch).
cudaError_t launch_totals_chunked(const FieldView& f, size_t n, int is32, size_t chunk, int nb,
                                  double* partials, double* out, cudaStream_t s);
// Frozen ghost store: for each axis a block [side][layer][field][plane].
size_t frozen_elems(int nx, int ny, int nz);
size_t frozen_axis_offset(int nx, int ny, int nz, int axis);
cudaError_t launch_frozen_capture(const FieldView& f, void* frozen, int nx, int ny, int nz,
                                  int is32, cudaStream_t s);

}  // namespace shasta
