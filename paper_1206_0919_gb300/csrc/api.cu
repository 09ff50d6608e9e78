// api.cu -- the C ABI of include/shasta.h: contexts, state transfer and the
// step loop.  Every numerical step runs in the kernels of this library.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/shasta.h"
#include "kernels.h"
#include "work_ranges.h"

using namespace shasta;

namespace {

thread_local std::string g_create_error;

const char* kVersion = "shasta-gb300 0.1 (sm_103a)";

// Fixed permutation of the sweep axes, Sec. 3.1.4.
const int kAxisTable[18] = {0, 1, 2, 0, 2, 1, 2, 0, 1, 2, 1, 0, 1, 2, 0, 1, 0, 2};

// Work-range cost model of the FP32 / MIXED sweeps (measured per warp on
// 200^3 and 256^3 hot spots): a piece costs its positions plus 13 of lead-in
// and lag, plus about 11 for each line end it touches (ghost positions); the
// three CTAs resident on an SM, in launch order, ran 8% faster / on par / 9%
// slower than the mean with equal shares.
constexpr double kEdgeCost = 11.0;
constexpr double kRankSkew = 0.04;
// Rank skews the autotuner times (with equal shares, the last CTA of an SM
// finished up to 9% after the mean; measured optimum 0.04-0.08 for one range
// per warp: 0.8-1.3% off the 200^3 / 256^3 step, larger skews slower).
const double kSkewCands[] = {0.0, 0.04, 0.08};

}  // namespace

struct shasta_ctx {
  int device = 0;
  shasta_grid g{};
  double dx = 1, lambda = 0.4;
  shasta_eos eos{};
  shasta_opts o{};
  int is32 = 1;
  size_t ncell = 0, esize = 4;
  void* state_mem = nullptr;  // both buffers
  void* split_mem = nullptr;  // SPLIT scheme: the half-step state and the intermediates
  float* split_q = nullptr;   // half-step state (quads, R)
  float* split_r = nullptr;
  float* split_scratch = nullptr;
  void* tab_mem = nullptr;    // tabulated EoS: the table in double, then in float
  EosTable tab{};
  FieldView view[2] = {};     // where the fields of each buffer live
  float* quad[2] = {};        // FP32 / MIXED: (E, Mx, My, Mz) per cell
  float* rf[2] = {};          // FP32 / MIXED: R
  int cur = 0;
  bool state_set = false;
  void* frozen = nullptr;
  double* staging = nullptr;  // 6 * ncell doubles, allocated on first host transfer
  double* partials = nullptr;
  double* d_tot = nullptr;
  unsigned long long* d_count = nullptr;  // [0] clamp count, [1] check scratch
  unsigned long long* d_chk = nullptr;    // checked builds: refused accesses [count, code, index]
  double* h_small = nullptr;              // pinned: 5 totals + counters
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // set / get: copies and format conversions run on a stream of the lowest
  // priority, ordered after the context stream's earlier work and before its
  // later work by two events, so that a caller's higher-priority compute
  // streams keep the SMs while they overlap
  cudaStream_t xfer = nullptr;
  cudaEvent_t ev_main = nullptr, ev_xfer = nullptr;
  int64_t steps = 0;
  int sm_count = 152;
  int occ[3][3][2] = {};  // FP32 / MIXED: resident warps per SM [eos][axis][variant]
  int wpb = 4;            // warps per block of the FP32 / MIXED kernels
  long long force_range = 0;  // nonzero: positions per work range (environment override)
  int force_variant = -1; // >= 0: launch variant (environment override)
  bool tuned = false;     // autotuned launch choice below is valid
  int tune_var[3] = {0, 0, 0};
  long long tune_range[3] = {0, 0, 0};
  // FP32 / MIXED: per axis, the bounds of balanced work ranges (device), built
  // for one range length; off with SHASTA_BALANCE=0 or a forced range length
  bool balance = true;
  int* d_ranges[3] = {};
  long long ranges_cap[3] = {};  // capacity in bounds
  long long ranges_len[3] = {};  // range length the table was built for (0: none)
  int ranges_var[3] = {};        // launch variant the table was built for
  long long ranges_n[3] = {};    // ranges in the table
  // work shares of the CTAs resident on one SM, by launch order: the first
  // CTA takes 1 + skew times the mean work, the last 1 - skew (the warp
  // schedulers favour older CTAs, so equal shares finish staggered)
  double rank_skew[3] = {kRankSkew, kRankSkew, kRankSkew};  // per axis
  bool force_skew = false;  // rank skew set by the environment (not tuned)
  double ranges_skew[3] = {};  // rank skew the table was built for
  double edge_cost = kEdgeCost;  // streaming cost of a line end a piece touches, in positions
  cudaGraphExec_t graph = nullptr;  // six steps from phase 0, buffer 0
  std::string err;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int now = -1;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
  }
};

shasta_status fail(shasta_ctx* c, shasta_status s, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    g_create_error = msg;
  return s;
}

shasta_status cuda_fail(shasta_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(c, e == cudaErrorMemoryAllocation ? SHASTA_ENOMEM : SHASTA_ECUDA, m);
}

#define CK(call, where)                                    \
  do {                                                     \
    cudaError_t _e = (call);                               \
    if (_e != cudaSuccess) return cuda_fail(c, _e, where); \
  } while (0)

EosParams eos_params(const shasta_ctx* c) {
  EosParams q;
  q.kind = c->eos.kind;
  q.B = c->eos.B;
  q.ec = c->eos.e_c;
  q.omd = 1.0 - c->o.delta;
  q.tab = c->tab;
  return q;
}

shasta_status ensure_staging(shasta_ctx* c) {
  if (c->staging) return SHASTA_OK;
  CK(cudaMalloc((void**)&c->staging, 6 * c->ncell * sizeof(double)), "cudaMalloc staging");
  return SHASTA_OK;
}

// Copies five caller arrays into device doubles: returns device pointers
// (the caller's own for DEVICE memory, the staging area for HOST memory).
shasta_status stage_in(shasta_ctx* c, const double* const src[5], int mem, const double* out[5],
                       cudaStream_t st) {
  if (mem == SHASTA_MEM_DEVICE) {
    for (int k = 0; k < 5; ++k) out[k] = src[k];
    return SHASTA_OK;
  }
  shasta_status s = ensure_staging(c);
  if (s != SHASTA_OK) return s;
  for (int k = 0; k < 5; ++k) {
    double* d = c->staging + (size_t)k * c->ncell;
    CK(cudaMemcpyAsync(d, src[k], c->ncell * sizeof(double), cudaMemcpyHostToDevice, st),
       "cudaMemcpyAsync H2D");
    out[k] = d;
  }
  return SHASTA_OK;
}

shasta_status check_count(shasta_ctx* c, bool prims, const double* const f[5], cudaStream_t st) {
  CK(cudaMemsetAsync(c->d_count + 1, 0, sizeof(unsigned long long), st), "memset");
  if (prims)
    CK(launch_check_prims(f, c->ncell, c->d_count + 1, st), "check_prims");
  else
    CK(launch_check_cons(f, c->ncell, c->d_count + 1, st), "check_cons");
  unsigned long long* h = reinterpret_cast<unsigned long long*>(c->h_small + 8);
  CK(cudaMemcpyAsync(h, c->d_count + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st),
     "memcpy count");
  CK(cudaStreamSynchronize(st), "sync");
  if (*h) {
    char m[160];
    snprintf(m, sizeof m, "%llu cells are not physical (non-finite, %s)", *h,
             prims ? "e < 0, n < 0 or |v| >= 1" : "E < 0 or |M| >= E");
    return fail(c, SHASTA_EUNPHYSICAL, m);
  }
  return SHASTA_OK;
}

// The transfer stream starts after the work enqueued so far on the context
// stream (a set must not overwrite a state still being swept; a get reads the
// state the steps leave) ...
shasta_status xfer_begin(shasta_ctx* c) {
  CK(cudaEventRecord(c->ev_main, c->stream), "event record");
  CK(cudaStreamWaitEvent(c->xfer, c->ev_main, 0), "stream wait");
  return SHASTA_OK;
}

// ... and the context stream's later work waits for what it enqueued.
shasta_status xfer_end(shasta_ctx* c) {
  CK(cudaEventRecord(c->ev_xfer, c->xfer), "event record");
  CK(cudaStreamWaitEvent(c->stream, c->ev_xfer, 0), "stream wait");
  return SHASTA_OK;
}

shasta_status after_set(shasta_ctx* c) {
  if (c->g.bc == SHASTA_BC_FROZEN) {
    CK(launch_frozen_capture(c->view[c->cur], c->frozen, c->g.nx, c->g.ny, c->g.nz, c->is32,
                             c->stream),
       "frozen_capture");
  }
  CK(cudaMemsetAsync(c->d_count, 0, sizeof(unsigned long long), c->stream), "memset");
  c->state_set = true;
  c->steps = 0;
  return SHASTA_OK;
}

// Positions (line group x position pairs) of a sweep along `axis`.
long long work_positions(const shasta_ctx* c, int axis) {
  const long long nx = c->g.nx, ny = c->g.ny, nz = c->g.nz;
  const long long n = axis == 0 ? nx : (axis == 1 ? ny : nz);
  const long long plane = axis == 0 ? ny * nz : (axis == 1 ? nx * nz : nx * ny);
  return (plane + 31) / 32 * n;
}

// Range length giving every resident warp of one wave `share` ranges (at
// least 24 positions: each piece pays a 13-position halo and lag).
long long range_for(long long total, long long warps, double share) {
  const double want = (double)warps * share;
  long long len = (long long)((double)total / (want > 1.0 ? want : 1.0)) + 1;
  return len < 24 ? 24 : len;
}

void drop_graph(shasta_ctx* c);

// Makes the device table of balanced ranges of an axis match range length
// `len` (as many ranges as uniform ranges of len would give); synchronous,
// so never called while a graph is being captured.
shasta_status ensure_ranges(shasta_ctx* c, int axis, long long len, int variant) {
  if (c->o.precision == SHASTA_FP64 || !c->balance || c->force_range > 0 || len < 1) return SHASTA_OK;
  if (c->ranges_len[axis] == len && c->ranges_var[axis] == variant &&
      c->ranges_skew[axis] == c->rank_skew[axis])
    return SHASTA_OK;
  const long long n = axis == 0 ? c->g.nx : (axis == 1 ? c->g.ny : c->g.nz);
  const long long total = work_positions(c, axis);
  const long long R = (total + len - 1) / len;
  const int wpsm = c->occ[c->eos.kind][axis][variant];
  const long long K = wpsm > 0 ? wpsm / c->wpb : 1;  // CTAs per SM
  const double skew = c->rank_skew[axis];
  auto weight = [&](long long r) { return rank_weight(r, c->sm_count, K, c->wpb, skew); };
  const std::vector<int> b = balanced_bounds(total, n, R, axis == 0 ? 8 : 1, 13.0, c->edge_cost, weight);
  drop_graph(c);  // a captured graph holds the old table and its size
  c->ranges_len[axis] = 0;
  if ((long long)b.size() > c->ranges_cap[axis]) {
    CK(cudaStreamSynchronize(c->stream), "ranges");  // no launch still reads the old table
    cudaFree(c->d_ranges[axis]);
    c->d_ranges[axis] = nullptr;
    c->ranges_cap[axis] = 0;
    CK(cudaMalloc(&c->d_ranges[axis], b.size() * sizeof(int)), "cudaMalloc ranges");
    c->ranges_cap[axis] = (long long)b.size();
  }
  CK(cudaMemcpyAsync(c->d_ranges[axis], b.data(), b.size() * sizeof(int), cudaMemcpyHostToDevice,
                     c->stream),
     "upload ranges");
  CK(cudaStreamSynchronize(c->stream), "upload ranges");
  c->ranges_len[axis] = len;
  c->ranges_var[axis] = variant;
  c->ranges_skew[axis] = c->rank_skew[axis];
  c->ranges_n[axis] = (long long)b.size() - 1;
  return SHASTA_OK;
}

SweepParams sweep_params(shasta_ctx* c, int axis, int from, int variant, long long range) {
  SweepParams P;
  memset(&P, 0, sizeof P);
  long long nx = c->g.nx, ny = c->g.ny, nz = c->g.nz;
  for (int k = 0; k < NF; ++k) {
    P.in[k] = c->view[from].p[k];
    P.out[k] = c->view[from ^ 1].p[k];
  }
  P.qin = c->quad[from];
  P.rin = c->rf[from];
  P.qout = c->quad[from ^ 1];
  P.rout = c->rf[from ^ 1];
  if (axis == 0) {
    P.n = (int)nx;
    P.stride = 1;
    P.plane = ny * nz;
    P.nb = (int)ny;
    P.sb = nx;
    P.sc = nx * ny;
  } else if (axis == 1) {
    P.n = (int)ny;
    P.stride = nx;
    P.plane = nx * nz;
    P.nb = (int)nx;
    P.sb = 1;
    P.sc = nx * ny;
  } else {
    P.n = (int)nz;
    P.stride = nx * ny;
    P.plane = nx * ny;
    P.nb = (int)nx;
    P.sb = 1;
    P.sc = nx;
  }
  P.bc = c->g.bc;
  P.frozen = c->frozen ? (const char*)c->frozen +
                             frozen_axis_offset((int)nx, (int)ny, (int)nz, axis) * c->esize
                       : nullptr;
  P.tau_h = 0.5 * c->lambda;
  P.tau_f = c->lambda;
  P.htau_h = 0.5 * P.tau_h;
  P.htau_f = 0.5 * P.tau_f;
  // NO_ANTIFLUX: the FP32 kernels leave the stage out; the others compute
  // it with eta = 0, which gives A = 0
  P.eta = c->o.scheme == SHASTA_SCHEME_NO_ANTIFLUX ? 0.0 : c->o.eta;
  P.omd = 1.0 - c->o.delta;
  P.bag_B = c->eos.B;
  P.bag_ec = c->eos.e_c;
  P.clamp_count = c->d_count;
  P.tab = c->tab;
  set_float_scalars(P);
  P.ncap = (long long)c->ncell;
  P.chk = c->d_chk;  // null unless this is a checked build
#ifdef SHASTA_CHECKED
  // test aid of checked builds: a smaller bound on the state arrays (the
  // accesses above it are then refused, which shows that the checks work)
  if (const char* v = getenv("SHASTA_CHECKED_NCAP"))
    if (atoll(v) > 0 && atoll(v) < P.ncap) P.ncap = atoll(v);
#endif
  P.range_len = range < 1 ? 1 : range;  // FP64: cells per line segment
  P.variant = variant;
  if (c->o.precision != SHASTA_FP64) {
    // the balanced table built for this range length, if any
    if (c->balance && c->force_range == 0 && c->ranges_len[axis] == P.range_len &&
        c->ranges_var[axis] == variant && c->ranges_skew[axis] == c->rank_skew[axis]) {
      P.ranges = c->d_ranges[axis];
      P.nranges = c->ranges_n[axis];
    }
    // at most one wave of resident warps loops over the ranges
    const long long total = work_positions(c, axis);
    const long long ranges = P.ranges ? P.nranges : (total + P.range_len - 1) / P.range_len;
    long long blocks = (ranges + c->wpb - 1) / c->wpb;
    const int wpsm = c->occ[c->eos.kind][axis][variant];
    const long long wave = (long long)c->sm_count * (wpsm > 0 ? wpsm / c->wpb : 1);
    P.blocks = blocks < wave ? blocks : (wave > 0 ? wave : 1);
  }
  return P;
}

// FP64 kernel: one thread per line segment; default segment length for
// about 1024 threads per SM, segments of at least 16 cells (each re-runs a
// 6-cell halo per side).
long long fp64_segment(const shasta_ctx* c, int axis) {
  const long long n = axis == 0 ? c->g.nx : (axis == 1 ? c->g.ny : c->g.nz);
  const long long plane = (long long)c->g.nx * c->g.ny * c->g.nz / (n > 0 ? n : 1);
  const long long want = (long long)c->sm_count * 1024;
  long long nseg = (want + plane - 1) / (plane > 0 ? plane : 1);
  const long long cap = n / 16 > 1 ? n / 16 : 1;
  nseg = nseg < 1 ? 1 : (nseg > cap ? cap : nseg);
  return (n + nseg - 1) / nseg;
}

// Launch choice for an axis: environment overrides, else the autotuned
// choice, else variant 0 and one range per resident warp (FP32 / MIXED) or
// the default segment length (FP64).
void launch_choice(const shasta_ctx* c, int axis, int& variant, long long& range) {
  if (c->o.precision == SHASTA_FP64) {
    variant = 0;
    range = c->tuned && c->tune_range[axis] > 0 ? c->tune_range[axis] : fp64_segment(c, axis);
    if (c->force_range > 0) range = c->force_range;
    return;
  }
  variant = c->tuned ? c->tune_var[axis] : 0;
  if (c->force_variant >= 0) variant = c->force_variant;
  const long long warps = (long long)c->sm_count * c->occ[c->eos.kind][axis][variant];
  range = c->tuned ? c->tune_range[axis] : range_for(work_positions(c, axis), warps, 1.0);
  if (c->force_range > 0) range = c->force_range;
}

// Balanced range tables for the current launch choice of every axis (before
// launches or a capture).
shasta_status prepare_ranges(shasta_ctx* c) {
  for (int axis = 0; axis < 3; ++axis) {
    int v;
    long long r;
    launch_choice(c, axis, v, r);
    const shasta_status st = ensure_ranges(c, axis, r, v);
    if (st != SHASTA_OK) return st;
  }
  return SHASTA_OK;
}

cudaError_t launch_params(shasta_ctx* c, int axis, const SweepParams& P) {
  if (c->o.precision == SHASTA_FP64) return launch_sweep_f64(P, axis, c->eos.kind, c->stream);
  if (c->o.precision == SHASTA_MIXED) return launch_sweep_mixed(P, axis, c->eos.kind, c->stream);
  if (c->o.precision == SHASTA_MIXED_FP64)
    return launch_sweep_mixed64(P, axis, c->eos.kind, c->stream);
  if (c->o.scheme == SHASTA_SCHEME_NO_ANTIFLUX)
    return launch_sweep_f32_noaf(P, axis, c->eos.kind, c->stream);
  if (c->o.scheme == SHASTA_SCHEME_SPLIT)
    return launch_sweep_split(P, axis, c->eos.kind, c->split_scratch, c->split_q, c->split_r,
                              c->stream);
  return launch_sweep_f32(P, axis, c->eos.kind, c->stream);
}

cudaError_t launch_sweep(shasta_ctx* c, int axis) {
  int variant;
  long long range;
  launch_choice(c, axis, variant, range);
  cudaError_t e = launch_params(c, axis, sweep_params(c, axis, c->cur, variant, range));
  if (e == cudaSuccess) c->cur ^= 1;
  return e;
}

// The three sweeps of step phase ph (TWO_SWEEPS: the first two in one
// launch, from the current buffer into the other).
cudaError_t launch_step(shasta_ctx* c, int ph) {
  const int* ax = kAxisTable + 3 * ph;
  if (c->o.scheme == SHASTA_SCHEME_TWO_SWEEPS) {
    SweepParams P = sweep_params(c, ax[0], c->cur, 0, 1);
    cudaError_t e = launch_fuse2(P, c->g.nx, c->g.ny, c->g.nz, ax[0], ax[1], c->eos.kind,
                                 c->sm_count, c->stream);
    if (e != cudaSuccess) return e;
    c->cur ^= 1;
    return launch_sweep(c, ax[2]);
  }
  for (int sub = 0; sub < 3; ++sub) {
    cudaError_t e = launch_sweep(c, ax[sub]);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void drop_graph(shasta_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
}

// Mean time of `reps` sweeps of axis with parameters P (after `warm`
// untimed ones), from the current buffer into the other one.
cudaError_t time_choice(shasta_ctx* c, int axis, const SweepParams& P, int warm, int reps,
                        cudaEvent_t e0, cudaEvent_t e1, float& ms) {
  cudaError_t ce = cudaSuccess;
  for (int r = 0; r < warm && ce == cudaSuccess; ++r) ce = launch_params(c, axis, P);
  if (ce == cudaSuccess) ce = cudaEventRecord(e0, c->stream);
  for (int r = 0; r < reps && ce == cudaSuccess; ++r) ce = launch_params(c, axis, P);
  if (ce == cudaSuccess) ce = cudaEventRecord(e1, c->stream);
  if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
  if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
  return ce;
}

// Times candidate launch choices per axis with repeated sweeps from the
// current buffer into the other one (the state itself is not changed) and
// keeps the fastest.  FP32 / MIXED: the register variant, and ranges of one
// line group (no line is cut) or of 1/4 .. 3 ranges per resident warp.
// FP64: the line segment length (the default one, 24 .. 128 cells, whole
// lines).  The choice does not change results.
shasta_status autotune(shasta_ctx* c) {
  if (c->o.scheme == SHASTA_SCHEME_SPLIT) {
    c->tuned = true;
    return SHASTA_OK;
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "cudaEventCreate");
  CK(cudaEventCreate(&e1), "cudaEventCreate");
  shasta_status st = SHASTA_OK;
  const bool f64 = c->o.precision == SHASTA_FP64;
  static const double shares[] = {0.25, 0.5, 1.0, 2.0, 3.0};
  static const long long segments[] = {24, 32, 48, 64, 100, 128};
  for (int axis = 0; axis < 3 && st == SHASTA_OK; ++axis) {
    const int n = axis == 0 ? c->g.nx : (axis == 1 ? c->g.ny : c->g.nz);
    const long long total = work_positions(c, axis);
    float best = 1e30f;
    int bv = 0;
    long long br = f64 ? fp64_segment(c, axis) : n;
    for (int var = 0; var < (f64 ? 1 : 2); ++var) {
      long long cands[8];
      int nc = 0;
      auto add = [&](long long r) {
        bool dup = false;
        for (int i = 0; i < nc; ++i) dup = dup || cands[i] == r;
        if (!dup) cands[nc++] = r;
      };
      if (f64) {
        add(fp64_segment(c, axis));
        for (long long r : segments)
          if (r < n) add(r);
        add(n);
      } else {
        const long long warps = (long long)c->sm_count * c->occ[c->eos.kind][axis][var];
        add(n);
        for (double sh : shares) {
          const long long r = range_for(total, warps, sh);
          if (r < total) add(r);
        }
      }
      for (int ci = 0; ci < nc && st == SHASTA_OK; ++ci) {
        st = ensure_ranges(c, axis, cands[ci], var);
        if (st != SHASTA_OK) break;
        float ms = 0;
        const cudaError_t ce = time_choice(c, axis, sweep_params(c, axis, c->cur, var, cands[ci]),
                                           f64 ? 1 : 2, f64 ? 2 : 4, e0, e1, ms);
        if (ce != cudaSuccess) {
          st = cuda_fail(c, ce, "autotune");
          break;
        }
        if (ms < best) {
          best = ms;
          bv = var;
          br = cands[ci];
        }
      }
    }
    c->tune_var[axis] = bv;
    c->tune_range[axis] = br;
    // FP32 / MIXED: the work shares of the CTAs of an SM for that choice
    if (!f64 && st == SHASTA_OK && c->balance && c->force_range == 0 && !c->force_skew) {
      const double keep = c->rank_skew[axis];
      double bs = keep;
      float bms = 1e30f;
      for (double sk : kSkewCands) {
        c->rank_skew[axis] = sk;
        st = ensure_ranges(c, axis, br, bv);
        if (st != SHASTA_OK) break;
        float ms = 0;
        const cudaError_t ce = time_choice(c, axis, sweep_params(c, axis, c->cur, bv, br), 2, 4, e0, e1, ms);
        if (ce != cudaSuccess) {
          st = cuda_fail(c, ce, "autotune");
          break;
        }
        if (ms < bms) {
          bms = ms;
          bs = sk;
        }
      }
      c->rank_skew[axis] = st == SHASTA_OK ? bs : keep;
    }
    if (st == SHASTA_OK) st = ensure_ranges(c, axis, br, bv);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == SHASTA_OK) {
    c->tuned = true;
    drop_graph(c);
  }
  return st;
}

void release(shasta_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->xfer) cudaStreamSynchronize(c->xfer);
  cudaFree(c->state_mem);
  cudaFree(c->split_mem);
  cudaFree(c->tab_mem);
  cudaFree(c->frozen);
  cudaFree(c->staging);
  cudaFree(c->partials);
  cudaFree(c->d_tot);
  cudaFree(c->d_count);
  cudaFree(c->d_chk);
  for (int a = 0; a < 3; ++a) cudaFree(c->d_ranges[a]);
  cudaFreeHost(c->h_small);
  drop_graph(c);
  if (c->xfer) cudaStreamDestroy(c->xfer);
  if (c->ev_main) cudaEventDestroy(c->ev_main);
  if (c->ev_xfer) cudaEventDestroy(c->ev_xfer);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // namespace

extern "C" {

void shasta_default_opts(shasta_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->precision = SHASTA_FP32;
  o->eta = 0.125;
  o->delta = 0.0;
  o->stream = nullptr;
  o->device = 0;
  o->check_input = 1;
  o->autotune = 1;
  o->use_graphs = 1;
  o->scheme = SHASTA_SCHEME_FUSED;
}

shasta_status shasta_create(const shasta_grid* g, double dx, double lambda, const shasta_eos* eos,
                            const shasta_opts* o, shasta_ctx** out) {
  g_create_error.clear();
  if (!out) return fail(nullptr, SHASTA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!g) return fail(nullptr, SHASTA_EINVAL, "grid is NULL");
  if (g->nx < 1 || g->ny < 1 || g->nz < 1)
    return fail(nullptr, SHASTA_EINVAL, "grid sizes must be >= 1");
  if ((long long)g->nx * g->ny > (1LL << 31) || (long long)g->ny * g->nz > (1LL << 31) ||
      (long long)g->nx * g->nz > (1LL << 31))
    return fail(nullptr, SHASTA_EINVAL, "grid plane too large");
  if (g->bc < SHASTA_BC_REFLECT || g->bc > SHASTA_BC_FROZEN)
    return fail(nullptr, SHASTA_EINVAL, "unknown boundary rule");
  if (!(dx > 0) || !isfinite(dx)) return fail(nullptr, SHASTA_EINVAL, "dx must be > 0");
  if (!(lambda > 0.0 && lambda <= 0.5)) return fail(nullptr, SHASTA_EINVAL, "need 0 < lambda <= 0.5");
  shasta_opts opts;
  if (o)
    opts = *o;
  else
    shasta_default_opts(&opts);
  if (opts.precision < SHASTA_FP64 || opts.precision > SHASTA_MIXED_FP64)
    return fail(nullptr, SHASTA_EINVAL, "unknown precision");
  if (opts.precision != SHASTA_FP64 && (long long)g->nx * g->ny * g->nz >= (1LL << 32))
    return fail(nullptr, SHASTA_EINVAL, "FP32 / MIXED grids hold fewer than 2^32 cells");
  const bool mixed = opts.precision == SHASTA_MIXED || opts.precision == SHASTA_MIXED_FP64;
  if (!(opts.eta >= 0.0 && opts.eta <= 0.5)) return fail(nullptr, SHASTA_EINVAL, "need 0 <= eta <= 0.5");
  if (!(opts.delta >= 0.0 && opts.delta < 0.5)) return fail(nullptr, SHASTA_EINVAL, "need 0 <= delta < 0.5");
  if (opts.scheme != SHASTA_SCHEME_FUSED && opts.scheme != SHASTA_SCHEME_NO_ANTIFLUX &&
      opts.scheme != SHASTA_SCHEME_SPLIT && opts.scheme != SHASTA_SCHEME_TWO_SWEEPS)
    return fail(nullptr, SHASTA_EINVAL, "unknown scheme");
  if (opts.scheme == SHASTA_SCHEME_TWO_SWEEPS) {
    if (opts.precision != SHASTA_FP32)
      return fail(nullptr, SHASTA_EINVAL, "the two-sweep scheme is FP32 only");
    if (g->bc == SHASTA_BC_FROZEN)
      return fail(nullptr, SHASTA_EINVAL, "the two-sweep scheme takes reflecting or periodic walls");
    if (eos && eos->kind == SHASTA_EOS_TABLE)
      return fail(nullptr, SHASTA_EINVAL, "the two-sweep scheme takes the closed-form EoS");
  }
  if (opts.scheme == SHASTA_SCHEME_SPLIT && opts.precision != SHASTA_FP32)
    return fail(nullptr, SHASTA_EINVAL, "the split scheme is FP32 only");
  if (opts.delta == 0.0) opts.delta = opts.precision == SHASTA_FP64 ? 1e-10 : 1e-6;
  shasta_eos e;
  if (eos)
    e = *eos;
  else {
    e.kind = SHASTA_EOS_IDEAL;
    e.B = 0.0;
    e.e_c = 0.0;
  }
  if (e.kind != SHASTA_EOS_IDEAL && e.kind != SHASTA_EOS_BAG && e.kind != SHASTA_EOS_TABLE)
    return fail(nullptr, SHASTA_EINVAL, "unknown EoS");
  if (e.kind == SHASTA_EOS_BAG && !(e.B >= 0.0 && 4.0 * e.B <= e.e_c))
    return fail(nullptr, SHASTA_EINVAL, "bag EoS needs 0 <= 4B <= e_c");
  if (e.kind == SHASTA_EOS_TABLE) {
    if (mixed) return fail(nullptr, SHASTA_EINVAL, "a tabulated EoS runs in FP64 or FP32");
    if (opts.scheme == SHASTA_SCHEME_NO_ANTIFLUX && opts.precision == SHASTA_FP32)
      return fail(nullptr, SHASTA_EINVAL, "no FP32 transport-only kernels for a tabulated EoS");
    if (!e.table || e.table_n < 2 || e.table_n > (1 << 26) || !(e.table_de > 0.0) ||
        !isfinite(e.table_de))
      return fail(nullptr, SHASTA_EINVAL, "table EoS needs a table of >= 2 values and table_de > 0");
    for (int k = 0; k < e.table_n; ++k) {
      const double pk = e.table[k];
      if (!isfinite(pk) || pk < 0.0) return fail(nullptr, SHASTA_EINVAL, "table values must be finite and >= 0");
      if (k > 0) {
        const double slope = (pk - e.table[k - 1]) / e.table_de;
        if (!(slope >= 0.0 && slope < 1.0))
          return fail(nullptr, SHASTA_EINVAL, "table slopes dp/de must lie in [0, 1)");
      }
    }
  } else {
    e.table = nullptr;
    e.table_n = 0;
    e.table_de = 0.0;
  }
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev < 1)
    return fail(nullptr, SHASTA_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(ce));
  if (opts.device < 0 || opts.device >= ndev) return fail(nullptr, SHASTA_EINVAL, "bad device ordinal");

  shasta_ctx* c = new (std::nothrow) shasta_ctx();
  if (!c) return fail(nullptr, SHASTA_ENOMEM, "host allocation failed");
  c->device = opts.device;
  DeviceGuard dg(c->device);
  c->g = *g;
  c->dx = dx;
  c->lambda = lambda;
  c->eos = e;
  c->o = opts;
  c->is32 = opts.precision != SHASTA_FP64;
  c->esize = c->is32 ? 4 : 8;
  c->ncell = (size_t)g->nx * g->ny * g->nz;
  {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) == cudaSuccess && sms > 0)
      c->sm_count = sms;
    const char* v = getenv("SHASTA_RANGE");
    if (v && atoll(v) > 0) c->force_range = atoll(v);
    v = getenv("SHASTA_BALANCE");
    if (v && atoi(v) == 0) c->balance = false;
    v = getenv("SHASTA_VARIANT");
    if (v && atoi(v) >= 0 && atoi(v) <= 1) c->force_variant = atoi(v);
    v = getenv("SHASTA_RANK_SKEW");
    if (v && atof(v) >= 0.0 && atof(v) < 0.5) {
      c->rank_skew[0] = c->rank_skew[1] = c->rank_skew[2] = atof(v);
      c->force_skew = true;
    }
    v = getenv("SHASTA_EDGE_COST");
    if (v && atof(v) >= 0.0 && atof(v) <= 64.0) c->edge_cost = atof(v);
  }
  auto bail = [&](cudaError_t err, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(err);
    release(c);
    return fail(nullptr, err == cudaErrorMemoryAllocation ? SHASTA_ENOMEM : SHASTA_ECUDA, m);
  };
  // FP64: five dense fields per buffer.  FP32 / MIXED: a quad array of
  // (E, Mx, My, Mz) per cell and a dense R array per buffer.  Every array
  // starts on a 256-byte boundary.
  size_t field_bytes = ((c->ncell * c->esize + 255) / 256) * 256;
  cudaError_t err = cudaMalloc(&c->state_mem, 2 * NF * field_bytes);
  if (err != cudaSuccess) return bail(err, "cudaMalloc state");
  for (int b = 0; b < 2; ++b) {
    char* bb = (char*)c->state_mem + (size_t)b * NF * field_bytes;
    if (c->is32) {
      c->quad[b] = (float*)bb;
      c->rf[b] = (float*)(bb + 4 * field_bytes);
      for (int k = 0; k < 4; ++k) {
        c->view[b].p[k] = c->quad[b] + k;
        c->view[b].s[k] = 4;
      }
      c->view[b].p[4] = c->rf[b];
      c->view[b].s[4] = 1;
    } else {
      for (int k = 0; k < NF; ++k) {
        c->view[b].p[k] = bb + (size_t)k * field_bytes;
        c->view[b].s[k] = 1;
      }
    }
  }
  if (e.kind == SHASTA_EOS_TABLE) {
    const size_t n = (size_t)e.table_n;
    const size_t b64 = ((n * sizeof(double) + 255) / 256) * 256;
    err = cudaMalloc(&c->tab_mem, b64 + n * sizeof(float));
    if (err != cudaSuccess) return bail(err, "cudaMalloc EoS table");
    std::vector<float> t32(e.table, e.table + n);
    err = cudaMemcpy(c->tab_mem, e.table, n * sizeof(double), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
      err = cudaMemcpy((char*)c->tab_mem + b64, t32.data(), n * sizeof(float), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return bail(err, "copy EoS table");
    c->tab.p64 = (const double*)c->tab_mem;
    c->tab.p32 = (const float*)((char*)c->tab_mem + b64);
    c->tab.n = e.table_n;
    c->tab.de = e.table_de;
    c->tab.inv_de32 = (float)(1.0 / e.table_de);
    c->eos.table = nullptr;  // the caller's memory is not kept
  }
  if (opts.scheme == SHASTA_SCHEME_SPLIT) {
    const size_t half = ((c->ncell * 20 + 255) / 256) * 256;
    const size_t scratch = split_scratch_floats(g->nx, g->ny, g->nz) * sizeof(float);
    err = cudaMalloc(&c->split_mem, half + scratch);
    if (err != cudaSuccess) return bail(err, "cudaMalloc split-scheme buffers");
    c->split_q = (float*)c->split_mem;
    c->split_r = c->split_q + 4 * c->ncell;
    c->split_scratch = (float*)((char*)c->split_mem + half);
  }
  if (g->bc == SHASTA_BC_FROZEN) {
    err = cudaMalloc(&c->frozen, frozen_elems(g->nx, g->ny, g->nz) * c->esize);
    if (err != cudaSuccess) return bail(err, "cudaMalloc frozen");
  }
  err = cudaMalloc((void**)&c->partials, 5 * 1024 * sizeof(double));
  if (err != cudaSuccess) return bail(err, "cudaMalloc partials");
  err = cudaMalloc((void**)&c->d_tot, 8 * sizeof(double));
  if (err != cudaSuccess) return bail(err, "cudaMalloc totals");
  err = cudaMalloc((void**)&c->d_count, 4 * sizeof(unsigned long long));
  if (err != cudaSuccess) return bail(err, "cudaMalloc counters");
  err = cudaMemset(c->d_count, 0, 4 * sizeof(unsigned long long));
  if (err != cudaSuccess) return bail(err, "cudaMemset counters");
#ifdef SHASTA_CHECKED
  err = cudaMalloc((void**)&c->d_chk, 4 * sizeof(unsigned long long));
  if (err == cudaSuccess) err = cudaMemset(c->d_chk, 0, 4 * sizeof(unsigned long long));
  if (err != cudaSuccess) return bail(err, "check record");
#endif
  err = cudaMallocHost((void**)&c->h_small, 16 * sizeof(double));
  if (err != cudaSuccess) return bail(err, "cudaMallocHost");
  if (opts.precision != SHASTA_FP64) {
    err = opts.precision == SHASTA_MIXED                 ? prepare_sweep_mixed(c->occ)
          : opts.precision == SHASTA_MIXED_FP64          ? prepare_sweep_mixed64(c->occ)
          : opts.scheme == SHASTA_SCHEME_NO_ANTIFLUX ? prepare_sweep_f32_noaf(c->occ)
                                                     : prepare_sweep_f32(c->occ);
    if (err != cudaSuccess) return bail(err, "prepare sweep kernels");
    if (opts.scheme == SHASTA_SCHEME_TWO_SWEEPS) {
      err = prepare_fuse2();
      if (err != cudaSuccess) return bail(err, "prepare two-sweep kernels");
    }
    c->wpb = opts.precision == SHASTA_MIXED        ? sweep_warps_per_block_mixed()
             : opts.precision == SHASTA_MIXED_FP64 ? sweep_warps_per_block_mixed64()
                                                   : sweep_warps_per_block_f32();
  }
  if (opts.stream) {
    c->stream = (cudaStream_t)opts.stream;
  } else {
    err = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (err != cudaSuccess) return bail(err, "cudaStreamCreate");
    c->own_stream = true;
  }
  {
    int least = 0, greatest = 0;
    err = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (err == cudaSuccess) err = cudaStreamCreateWithPriority(&c->xfer, cudaStreamNonBlocking, least);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&c->ev_main, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&c->ev_xfer, cudaEventDisableTiming);
    if (err != cudaSuccess) return bail(err, "transfer stream");
  }
  *out = c;
  return SHASTA_OK;
}

shasta_status shasta_destroy(shasta_ctx* c) {
  if (!c) return SHASTA_OK;
  DeviceGuard dg(c->device);
  release(c);
  return SHASTA_OK;
}

shasta_status shasta_set_conserved(shasta_ctx* c, const double* E, const double* Mx,
                                   const double* My, const double* Mz, const double* R, int mem) {
  if (!c) return SHASTA_EINVAL;
  if (!E || !Mx || !My || !Mz || !R) return fail(c, SHASTA_EINVAL, "NULL field pointer");
  if (mem != SHASTA_MEM_HOST && mem != SHASTA_MEM_DEVICE) return fail(c, SHASTA_EINVAL, "bad mem");
  DeviceGuard dg(c->device);
  const double* src[5] = {E, Mx, My, Mz, R};
  const double* d[5];
  shasta_status s = xfer_begin(c);
  if (s == SHASTA_OK) s = stage_in(c, src, mem, d, c->xfer);
  if (s != SHASTA_OK) return s;
  if (c->o.check_input) {
    s = check_count(c, false, d, c->xfer);
    if (s != SHASTA_OK) return s;
  }
  c->cur = 0;
  for (int k = 0; k < 5; ++k)
    CK(launch_from_f64(d[k], c->view[0].p[k], c->view[0].s[k], c->ncell, c->is32, c->xfer),
       "convert in");
  s = xfer_end(c);
  return s == SHASTA_OK ? after_set(c) : s;
}

shasta_status shasta_set_primitives(shasta_ctx* c, const double* e, const double* vx,
                                    const double* vy, const double* vz, const double* n, int mem) {
  if (!c) return SHASTA_EINVAL;
  if (!e || !vx || !vy || !vz || !n) return fail(c, SHASTA_EINVAL, "NULL field pointer");
  if (mem != SHASTA_MEM_HOST && mem != SHASTA_MEM_DEVICE) return fail(c, SHASTA_EINVAL, "bad mem");
  DeviceGuard dg(c->device);
  const double* src[5] = {e, vx, vy, vz, n};
  const double* d[5];
  shasta_status s = xfer_begin(c);
  if (s == SHASTA_OK) s = stage_in(c, src, mem, d, c->xfer);
  if (s != SHASTA_OK) return s;
  if (c->o.check_input) {
    s = check_count(c, true, d, c->xfer);
    if (s != SHASTA_OK) return s;
  }
  c->cur = 0;
  CK(launch_prim2cons(d, c->view[0], c->ncell, c->is32, eos_params(c), c->xfer), "prim2cons");
  s = xfer_end(c);
  return s == SHASTA_OK ? after_set(c) : s;
}

shasta_status shasta_step(shasta_ctx* c, int nsteps) {
  if (!c) return SHASTA_EINVAL;
  if (nsteps < 0) return fail(c, SHASTA_EINVAL, "nsteps < 0");
  if (!c->state_set) return fail(c, SHASTA_EINVAL, "state not set");
  DeviceGuard dg(c->device);
  if (!c->tuned && c->o.autotune && nsteps > 0) {
    shasta_status st = autotune(c);
    if (st != SHASTA_OK) return st;
  }
  if (nsteps > 0) {
    const shasta_status st = prepare_ranges(c);
    if (st != SHASTA_OK) return st;
  }
  while (nsteps > 0) {
    if (c->o.use_graphs && nsteps >= 6 && c->steps % 6 == 0 && c->cur == 0) {
      // six steps (18 sweeps) bring phase and buffer back: one graph
      if (!c->graph) {
        cudaGraph_t gr = nullptr;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t ce = cudaSuccess;
        for (int s = 0; s < 6 && ce == cudaSuccess; ++s) ce = launch_step(c, s);
        cudaError_t ce2 = cudaStreamEndCapture(c->stream, &gr);
        c->cur = 0;
        if (ce != cudaSuccess || ce2 != cudaSuccess) {
          if (gr) cudaGraphDestroy(gr);
          return cuda_fail(c, ce != cudaSuccess ? ce : ce2, "capture six steps");
        }
        ce = cudaGraphInstantiate(&c->graph, gr, 0);
        cudaGraphDestroy(gr);
        if (ce != cudaSuccess) {
          c->graph = nullptr;
          return cuda_fail(c, ce, "cudaGraphInstantiate");
        }
      }
      CK(cudaGraphLaunch(c->graph, c->stream), "cudaGraphLaunch");
      c->steps += 6;
      nsteps -= 6;
      continue;
    }
    CK(launch_step(c, (int)(c->steps % 6)), "sweep launch");
    ++c->steps;
    --nsteps;
  }
  return SHASTA_OK;
}

shasta_status shasta_autotune(shasta_ctx* c) {
  if (!c) return SHASTA_EINVAL;
  if (!c->state_set) return fail(c, SHASTA_EINVAL, "state not set");
  DeviceGuard dg(c->device);
  return autotune(c);
}

shasta_status shasta_get_tuning(const shasta_ctx* c, int out[6]) {
  if (!c || !out) return SHASTA_EINVAL;
  for (int a = 0; a < 3; ++a) {
    int v;
    long long r;
    launch_choice(c, a, v, r);
    out[2 * a] = v;
    out[2 * a + 1] = (int)(r < 2147483647LL ? r : 2147483647LL);
  }
  return SHASTA_OK;
}

shasta_status shasta_sweep(shasta_ctx* c, int axis) {
  if (!c) return SHASTA_EINVAL;
  if (axis < 0 || axis > 2) return fail(c, SHASTA_EINVAL, "axis must be 0, 1 or 2");
  if (!c->state_set) return fail(c, SHASTA_EINVAL, "state not set");
  DeviceGuard dg(c->device);
  const shasta_status st = prepare_ranges(c);
  if (st != SHASTA_OK) return st;
  CK(launch_sweep(c, axis), "sweep launch");
  return SHASTA_OK;
}

shasta_status shasta_sync(shasta_ctx* c) {
  if (!c) return SHASTA_EINVAL;
  DeviceGuard dg(c->device);
  CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  return SHASTA_OK;
}

shasta_status shasta_get_conserved(shasta_ctx* c, double* E, double* Mx, double* My, double* Mz,
                                   double* R, int mem) {
  if (!c) return SHASTA_EINVAL;
  if (mem != SHASTA_MEM_HOST && mem != SHASTA_MEM_DEVICE) return fail(c, SHASTA_EINVAL, "bad mem");
  if (!c->state_set) return fail(c, SHASTA_EINVAL, "state not set");
  DeviceGuard dg(c->device);
  double* dst[5] = {E, Mx, My, Mz, R};
  if (mem == SHASTA_MEM_HOST) {
    shasta_status s = ensure_staging(c);
    if (s != SHASTA_OK) return s;
  }
  shasta_status s = xfer_begin(c);
  if (s != SHASTA_OK) return s;
  for (int k = 0; k < 5; ++k) {
    if (!dst[k]) continue;
    double* d = mem == SHASTA_MEM_DEVICE ? dst[k] : c->staging + (size_t)k * c->ncell;
    CK(launch_to_f64(c->view[c->cur].p[k], c->view[c->cur].s[k], d, c->ncell, c->is32,
                     c->xfer),
       "convert out");
    if (mem == SHASTA_MEM_HOST)
      CK(cudaMemcpyAsync(dst[k], d, c->ncell * sizeof(double), cudaMemcpyDeviceToHost, c->xfer),
         "cudaMemcpyAsync D2H");
  }
  CK(cudaStreamSynchronize(c->xfer), "sync");
  return SHASTA_OK;
}

shasta_status shasta_get_primitives(shasta_ctx* c, double* e, double* vx, double* vy, double* vz,
                                    double* n, double* p, int mem) {
  if (!c) return SHASTA_EINVAL;
  if (mem != SHASTA_MEM_HOST && mem != SHASTA_MEM_DEVICE) return fail(c, SHASTA_EINVAL, "bad mem");
  if (!c->state_set) return fail(c, SHASTA_EINVAL, "state not set");
  DeviceGuard dg(c->device);
  double* dst[6] = {e, vx, vy, vz, n, p};
  double* d[6];
  if (mem == SHASTA_MEM_HOST) {
    shasta_status s = ensure_staging(c);
    if (s != SHASTA_OK) return s;
  }
  for (int k = 0; k < 6; ++k)
    d[k] = !dst[k] ? nullptr : (mem == SHASTA_MEM_DEVICE ? dst[k] : c->staging + (size_t)k * c->ncell);
  shasta_status s = xfer_begin(c);
  if (s != SHASTA_OK) return s;
  CK(launch_recover(c->view[c->cur], d, c->ncell, c->is32, eos_params(c), c->xfer), "recover");
  if (mem == SHASTA_MEM_HOST)
    for (int k = 0; k < 6; ++k)
      if (dst[k])
        CK(cudaMemcpyAsync(dst[k], d[k], c->ncell * sizeof(double), cudaMemcpyDeviceToHost,
                           c->xfer),
           "cudaMemcpyAsync D2H");
  CK(cudaStreamSynchronize(c->xfer), "sync");
  return SHASTA_OK;
}

shasta_status shasta_totals(shasta_ctx* c, double out[5]) {
  if (!c || !out) return SHASTA_EINVAL;
  if (!c->state_set) return fail(c, SHASTA_EINVAL, "state not set");
  DeviceGuard dg(c->device);
  CK(launch_totals(c->view[c->cur], c->ncell, c->is32, c->partials, c->d_tot, c->stream),
     "totals");
  CK(cudaMemcpyAsync(c->h_small, c->d_tot, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
     "memcpy totals");
  CK(cudaStreamSynchronize(c->stream), "sync");
  for (int k = 0; k < 5; ++k) out[k] = c->h_small[k];
  return SHASTA_OK;
}

int64_t shasta_steps_done(const shasta_ctx* c) { return c ? c->steps : -1; }

shasta_status shasta_set_step_counter(shasta_ctx* c, int64_t steps) {
  if (!c) return SHASTA_EINVAL;
  if (steps < 0) return fail(c, SHASTA_EINVAL, "negative step counter");
  c->steps = steps;
  return SHASTA_OK;
}

shasta_status shasta_checked_report(shasta_ctx* c, unsigned long long out[3]) {
  if (!c || !out) return SHASTA_EINVAL;
#ifdef SHASTA_CHECKED
  DeviceGuard dg(c->device);
  unsigned long long h[4] = {};
  CK(cudaStreamSynchronize(c->stream), "sync");
  CK(cudaMemcpy(h, c->d_chk, sizeof h, cudaMemcpyDeviceToHost), "read the record");
  CK(cudaMemset(c->d_chk, 0, sizeof h), "clear the record");
  for (int k = 0; k < 3; ++k) out[k] = h[k];
  return SHASTA_OK;
#else
  return fail(c, SHASTA_EINVAL, "not a checked build (built without SHASTA_CHECKED)");
#endif
}

shasta_status shasta_counters(shasta_ctx* c, int64_t out[1]) {
  if (!c || !out) return SHASTA_EINVAL;
  DeviceGuard dg(c->device);
  unsigned long long* h = reinterpret_cast<unsigned long long*>(c->h_small + 9);
  CK(cudaMemcpyAsync(h, c->d_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream),
     "memcpy counters");
  CK(cudaStreamSynchronize(c->stream), "sync");
  out[0] = (int64_t)*h;
  return SHASTA_OK;
}

void* shasta_stream(const shasta_ctx* c) { return c ? (void*)c->stream : nullptr; }

const char* shasta_last_error(const shasta_ctx* c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

const char* shasta_status_string(shasta_status s) {
  switch (s) {
    case SHASTA_OK: return "SHASTA_OK";
    case SHASTA_EINVAL: return "SHASTA_EINVAL";
    case SHASTA_ENOMEM: return "SHASTA_ENOMEM";
    case SHASTA_EAGAIN: return "SHASTA_EAGAIN";
    case SHASTA_EUNPHYSICAL: return "SHASTA_EUNPHYSICAL";
    case SHASTA_ETIMEOUT: return "SHASTA_ETIMEOUT";
    case SHASTA_ECUDA: return "SHASTA_ECUDA";
    case SHASTA_ENOTFOUND: return "SHASTA_ENOTFOUND";
  }
  return "SHASTA_UNKNOWN";
}

const char* shasta_version(void) { return kVersion; }

}  // extern "C"
