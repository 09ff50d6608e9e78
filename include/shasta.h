/*
 * shasta.h -- C ABI of a GB300-native relativistic SHASTA solver.
 *
 * The solver advances the conserved energy E, momentum (Mx, My, Mz) and
 * baryon density R of ideal relativistic hydrodynamics on a Cartesian grid
 * (J. Gerhard, V. Lindenstruth, M. Bleicher, "Relativistic Hydrodynamics on
 * Graphic Cards", arXiv:1206.0919).  Sec. 2 defines the system: the
 * conservation laws of T^{mu nu} and of the baryon current, with
 *   R = n gamma, M = (e + p) gamma^2 v, E = (e + p v^2) gamma^2.
 * Sec. 3 defines one time step: dimensionally split sweeps, each a half step
 * and a full step of geometric transport with pressure sources, phoenical
 * antidiffusion and the flux limiter, followed by the recovery of the
 * primitive variables (e, v, n, p) through the equation of state.
 *
 * Conventions shared by every call:
 *  - Arrays are dense nx*ny*nz grids with x fastest, element (i, j, k) at
 *    index i + nx*(j + ny*k).  They are always double precision at the ABI,
 *    whatever the precision the solver keeps its state in.
 *  - mem = SHASTA_MEM_HOST: ordinary host pointers (pinned memory makes the
 *    copies asynchronous-capable and faster).  SHASTA_MEM_DEVICE: device
 *    pointers on the context's device.  Arrays passed in are copied; the
 *    caller keeps ownership of every pointer it passes.
 *  - Every call returns a shasta_status.  No call throws or aborts; after an
 *    error, shasta_last_error(ctx) holds a one-line message.  A context may
 *    be used by one host thread at a time.
 *  - The library owns its device state.  Work is enqueued on the context's
 *    stream; calls that return data to the host synchronise that stream.
 */
#ifndef SHASTA_H
#define SHASTA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum shasta_status {
  SHASTA_OK = 0,
  SHASTA_EINVAL = 1,      /* bad argument (sizes, pointers, parameters) */
  SHASTA_ENOMEM = 2,      /* device or host allocation failed */
  SHASTA_EAGAIN = 3,      /* try again later (queue full, result not ready) */
  SHASTA_EUNPHYSICAL = 4, /* input state with non-finite values, E < 0 or |M| >= E */
  SHASTA_ETIMEOUT = 5,    /* a bounded wait ran out */
  SHASTA_ECUDA = 6,       /* a CUDA runtime call failed (message in last_error) */
  SHASTA_ENOTFOUND = 7    /* unknown ticket or handle */
} shasta_status;

/* Boundary rule at the six faces (Sec. 3.1.3 keeps halo cells around the
 * grid).  REFLECT: mirror image through the wall, the momentum normal to it
 * negated.  PERIODIC: wrap.  FROZEN: three ghost layers per face hold the
 * edge cell of the state given to the last set call and never change (the
 * paper's halo cells copied through unchanged). */
enum { SHASTA_BC_REFLECT = 0, SHASTA_BC_PERIODIC = 1, SHASTA_BC_FROZEN = 2 };

/* Equation of state.  IDEAL: p = e/3 (Sec. 2).  BAG: p = e/3 for e <= e_c and
 * p = (e - 4B)/3 above (not in the paper; requires 0 <= 4B <= e_c).  TABLE:
 * a tabulated p(e) (Sec. 2 allows tabulated equations of state), recovered
 * by the fixed-point iteration of Sec. 3; single contexts, FP64 and FP32. */
enum { SHASTA_EOS_IDEAL = 0, SHASTA_EOS_BAG = 1, SHASTA_EOS_TABLE = 2 };

/* Precision of the device state and arithmetic (Sec. 4-5: single precision
 * throughout, or double precision for the parts that lose accuracy as
 * v -> 1, where 1 - v^2 cancels).  FP64: everything in double.  FP32:
 * state, transport, limiter and recovery in float.  MIXED: state,
 * transport, limiter and most of the recovery in float; only the cancelling
 * difference D = E^2 - |M|^2 of the recovery is formed at about double
 * accuracy, as a compensated double-float evaluation on the FP32 pipe
 * (error-free products and sums).  MIXED_FP64: state, transport and
 * limiter in float; the whole recovery at every sweep position (D, the
 * closed-form root, p and the velocity along the sweep) in IEEE double from
 * the float state, rounded to float for the transport; single contexts
 * with the ideal or bag EoS.  The primitive output (shasta_get_primitives)
 * and the totals are computed in double for every precision. */
enum { SHASTA_FP64 = 0, SHASTA_FP32 = 1, SHASTA_MIXED = 2, SHASTA_MIXED_FP64 = 3 };

enum { SHASTA_MEM_HOST = 0, SHASTA_MEM_DEVICE = 1 };

typedef struct shasta_grid {
  int nx, ny, nz; /* interior cells per axis, each >= 1 */
  int bc;         /* SHASTA_BC_* */
} shasta_grid;

typedef struct shasta_eos {
  int kind;   /* SHASTA_EOS_* */
  double B;   /* bag constant (BAG only) */
  double e_c; /* branch point of the bag EoS (BAG only) */
  /* TABLE only: p at e = k * table_de, k = 0 .. table_n-1 (host memory,
   * copied by shasta_create), linear in between, the last interval
   * continued above the table.  Must be finite with p >= 0 and
   * 0 <= (p[k+1] - p[k]) / table_de < 1 (monotone and causal: the recovery
   * iteration then contracts).  Recovery: the root of
   * |v| = M/(E + p(E - M |v|)) from |v| = M/(E + p(E)): FP64 iterates that
   * map until |v| changes by at most 1e-14, FP32 takes Newton steps on it
   * to a change of 1e-7; e = E - M |v|. */
  const double* table;
  int table_n;
  double table_de;
} shasta_eos;

typedef struct shasta_opts {
  int precision; /* SHASTA_FP64 / SHASTA_FP32 / SHASTA_MIXED / SHASTA_MIXED_FP64 */
  double eta;    /* outer antidiffusion coefficient; Sec. 3 uses 1/8 */
  double delta;  /* recovery clamps |M| to (1 - delta) E; 0 selects 1e-10 (FP64)
                    or 1e-6 (FP32, MIXED, MIXED_FP64) */
  void* stream;  /* cudaStream_t to enqueue on; NULL: the context makes its own */
  int device;    /* CUDA device ordinal */
  int check_input; /* nonzero: set calls scan the state and return
                      SHASTA_EUNPHYSICAL for non-finite values, E < 0 or |M| >= E */
  int autotune;    /* nonzero: the first shasta_step times launch choices (work
                      range length, register variant) per axis and keeps the fastest;
                      results do not depend on the choice */
  int use_graphs;  /* nonzero: runs of six steps starting at phase 0 replay one
                      captured CUDA graph of 18 sweeps */
  int scheme;      /* SHASTA_SCHEME_*: how a sweep is computed (below) */
} shasta_opts;

/* Sweep schemes.  FUSED (the default) is the method of Sec. 3 in one fused
 * kernel per sweep.  NO_ANTIFLUX leaves antidiffusion and flux limiter out
 * (A = 0 in Eq. shasta-n: the transport alone, the same result as eta = 0);
 * with FP32 it runs kernels without that stage, so that its cost can be
 * measured (the with / without anti-flux comparison of Sec. 4); FP64 and
 * MIXED run the fused kernels with eta = 0 (same result, same cost).  SPLIT
 * (FP32 only) is the alternative decomposition of Sec. 3.1: each pass as
 * separate recovery, transport and antidiffusion kernels whose intermediate
 * results go through device memory (about 50 extra bytes of device memory
 * per cell); the method is the same, the rounding of a few differences is
 * not.  TWO_SWEEPS (FP32; reflecting or periodic walls; ideal or bag EoS)
 * blocks the first two sweeps of every step in time (the recompute-for-
 * traffic trade of Sec. 3.1.4): one launch sweeps tiles of the plane of
 * their two axes, with a 6-cell halo per side held in shared memory, along
 * the first axis and then the second, so the state crosses device memory
 * once for the two; the third sweep is the fused kernel.  Results are
 * bitwise those of FUSED; single sweeps (shasta_sweep) use FUSED. */
enum {
  SHASTA_SCHEME_FUSED = 0,
  SHASTA_SCHEME_NO_ANTIFLUX = 1,
  SHASTA_SCHEME_SPLIT = 2,
  SHASTA_SCHEME_TWO_SWEEPS = 3
};

typedef struct shasta_ctx shasta_ctx;

/* Fills *o with the defaults: FP32, eta = 1/8, delta = 0, stream NULL,
 * device 0, check_input 1, autotune 1, use_graphs 1, scheme FUSED. */
void shasta_default_opts(shasta_opts* o);

/* Creates a solver for one event.  dx is the cell size, lambda = dt/dx the
 * CFL number of Sec. 3 (0 < lambda <= 0.5); the time step is dt = lambda*dx.
 * eos may be NULL (ideal gas), o may be NULL (defaults).  Allocates two
 * copies of the five conserved fields on the device (double buffering,
 * Sec. 3.1.3).  Errors: EINVAL (sizes < 1, bad lambda/eta/eos/scheme, NULL out,
 * FP32 / MIXED grids of 2^32 cells or more), ENOMEM, ECUDA.  On error *out is NULL and shasta_last_error(NULL) holds
 * the message. */
shasta_status shasta_create(const shasta_grid* g, double dx, double lambda,
                            const shasta_eos* eos, const shasta_opts* o, shasta_ctx** out);

/* Releases every resource of ctx (NULL is accepted).  Synchronises first. */
shasta_status shasta_destroy(shasta_ctx* ctx);

/* Sets the conserved state (Sec. 2, Eqs. cf-density, cf-momentum,
 * cf-energy).  Five arrays of nx*ny*nz doubles in memory space mem.  Resets
 * the step counter to 0.  The copy, input check and conversion run on the
 * context's own transfer stream, created at the lowest stream priority: they
 * start after the work already enqueued on the context's stream, and work
 * enqueued there afterwards waits for them (a caller whose compute streams
 * have a higher priority keeps the SMs for them while transfers overlap).
 * Errors: EINVAL (NULL pointer or bad mem), EUNPHYSICAL (check_input set and
 * the state is not physical; the state is left as it was), ECUDA. */
shasta_status shasta_set_conserved(shasta_ctx* ctx, const double* E, const double* Mx,
                                   const double* My, const double* Mz, const double* R,
                                   int mem);

/* Sets the state from primitives: rest-frame energy density e, velocity v,
 * baryon density n (Sec. 2 map to E, M, R, computed on the device).  Same
 * layout, ownership and errors as shasta_set_conserved (|v| >= 1 or e < 0
 * gives EUNPHYSICAL when check_input is set). */
shasta_status shasta_set_primitives(shasta_ctx* ctx, const double* e, const double* vx,
                                    const double* vy, const double* vz, const double* n,
                                    int mem);

/* Enqueues nsteps full split steps (nsteps >= 0) and returns without
 * waiting.  Step k sweeps the axes in the order of entries 3(k mod 6) ..
 * 3(k mod 6)+2 of the permutation table of Sec. 3.1.4
 * {x,y,z, x,z,y, z,x,y, z,y,x, y,z,x, y,x,z}.  Each sweep is one fused
 * kernel: recovery at level n, half step (lambda/2), recovery at n+1/2,
 * full step from the old state (Sec. 3).  Errors: EINVAL (state never set,
 * nsteps < 0), ECUDA. */
shasta_status shasta_step(shasta_ctx* ctx, int nsteps);

/* Enqueues ONE sweep along axis (0 = x, 1 = y, 2 = z): the fused kernel of
 * shasta_step for a single axis.  Does not change the step counter; used to
 * time or study one sweep.  Errors: EINVAL (bad axis, state never set), ECUDA. */
shasta_status shasta_sweep(shasta_ctx* ctx, int axis);

/* Times the launch choices of the sweep kernels for this grid and keeps the
 * fastest per axis.  FP32 / MIXED: work range length and register variant (a
 * sweep's positions, line groups of 32 lines x positions along the axis, are
 * cut into as many ranges as that length gives, handed to the resident warps;
 * the cuts balance each range's streaming cost, its cells plus a 13-position
 * halo per line it touches and about 11 per line end, unless the environment
 * sets SHASTA_BALANCE=0), and the share of work of the CTAs resident on one
 * SM by launch order (1 + s for the first, 1 - s for the last, s timed among
 * 0, 0.04 and 0.08 unless SHASTA_RANK_SKEW sets it).  FP64: the length of the
 * line segments streamed one per thread.  No choice changes results.
 * Runs sweeps from the current state into the spare buffer only, so the
 * state is unchanged; synchronous.  Errors: EINVAL (state not set), ECUDA. */
shasta_status shasta_autotune(shasta_ctx* ctx);

/* Current launch choice per axis: out[2a] = register variant (FP64: 0),
 * out[2a+1] = positions per work range (FP64: cells per line segment). */
shasta_status shasta_get_tuning(const shasta_ctx* ctx, int out[6]);

/* Waits until all work enqueued on the context's stream has finished. */
shasta_status shasta_sync(shasta_ctx* ctx);

/* Copies the conserved state out (five arrays, any may be NULL to skip).
 * Synchronous with respect to the context's stream: it waits for the work
 * enqueued there, then converts and copies on the transfer stream (see
 * shasta_set_conserved) and returns when the arrays are filled. */
shasta_status shasta_get_conserved(shasta_ctx* ctx, double* E, double* Mx, double* My,
                                   double* Mz, double* R, int mem);

/* Recovers and copies out the primitives e, vx, vy, vz, n, p of the current
 * state (Sec. 3 phases 3-4; any pointer may be NULL to skip).  Synchronous,
 * on the transfer stream as shasta_get_conserved. */
shasta_status shasta_get_primitives(shasta_ctx* ctx, double* e, double* vx, double* vy,
                                    double* vz, double* n, double* p, int mem);

/* Sums of E, Mx, My, Mz, R over the grid, accumulated in double on the
 * device with a fixed reduction order (deterministic).  out: 5 host doubles.
 * Synchronous. */
shasta_status shasta_totals(shasta_ctx* ctx, double out[5]);

/* Totals without allocation (the paper has no counterpart: this is a
 * service for callers that cannot allocate device memory).
 *
 * Some callers cannot call cudaMalloc where they need the totals: code that
 * runs under another framework's device-memory pool, where a raw allocation
 * would escape its accounting or synchronise the device, and code that is
 * forbidden to allocate once it has started.  This call sums caller-owned
 * fields and allocates nothing; its per-block partial sums live in a fixed
 * array of 5 * SHASTA_TOTALS_NOALLOC_MAX_CELLS /
 * SHASTA_TOTALS_NOALLOC_CELLS_PER_BLOCK doubles (320 KiB) inside the
 * library's device code, which every GPU that loads the library holds until
 * the process exits.
 *
 * E, Mx, My, Mz, R: device pointers to n doubles each on the calling
 * thread's current device (any layout, summed as flat arrays).  out: device
 * pointer to 5 doubles, written with the sums of E, Mx, My, Mz, R in a fixed
 * reduction order (deterministic for a given n; the order differs from
 * shasta_totals', so the two agree to rounding).  stream: a cudaStream_t of
 * that device, NULL for the legacy default stream.  The work is enqueued and
 * the call returns without waiting; out is ready when the stream reaches it.
 * The caller keeps ownership of every pointer.
 *
 * Every call looks up the address of the fixed array on the current device
 * (a runtime table search, no allocation; looking it up each time keeps it
 * right after a device reset, which may reload the library's device code at
 * another address).  The first call on a device may load the library's
 * device code there; make that first call before any stream capture on the
 * device.  All calls on a device
 * share the array, which keeps the last call's partials: each call writes
 * every partial it reads, so nothing needs clearing, but calls whose work
 * overlaps on the GPU (two streams, or two threads) race on the array and
 * must be ordered by the caller.
 *
 * Errors: EINVAL (out NULL, a field NULL with n > 0, n larger than
 * SHASTA_TOTALS_NOALLOC_MAX_CELLS),
 * ECUDA (no current device, the address lookup or a launch failed).  No
 * message is kept: the status is the whole report. */
#define SHASTA_TOTALS_NOALLOC_MAX_CELLS 67108864ull /* 2^26 cells, e.g. 406^3 */
#define SHASTA_TOTALS_NOALLOC_CELLS_PER_BLOCK 8192ull
shasta_status shasta_totals_noalloc(const double* E, const double* Mx, const double* My,
                                    const double* Mz, const double* R, size_t n, double* out,
                                    void* stream);

/* Measured CUDA-core throughput of a device (the paper has no counterpart:
 * this is the arithmetic roof that the benchmark reports beside the HBM
 * roof, since the sweeps are bound by instruction issue).
 *
 * kind: SHASTA_ALU_FP32 or SHASTA_ALU_FP64.  Runs independent chains of
 * dependent fused multiply-adds on every SM of `device` on `stream` (a
 * cudaStream_t of that device, NULL for the legacy default stream), growing
 * the chain length until one launch takes at least 20 ms, and times three
 * launches with CUDA events.  Writes the rate in floating-point operations
 * per second (one fused multiply-add = 2) to *flops_per_s and, when
 * seconds_per_launch is not NULL, the time of one launch.  Synchronous.
 * Allocates and frees a small output buffer; changes no device setting.
 * Errors: EINVAL (bad kind, flops_per_s NULL), ENOMEM, ECUDA. */
#define SHASTA_ALU_FP32 0
#define SHASTA_ALU_FP64 1
shasta_status shasta_alu_peak(int kind, int device, void* stream, double* flops_per_s,
                              double* seconds_per_launch);


/* Number of full steps taken since the state was last set (the permutation
 * phase is this mod 6). */
int64_t shasta_steps_done(const shasta_ctx* ctx);

/* Sets the step counter, e.g. to resume from a checkpoint taken with
 * shasta_get_conserved + shasta_steps_done.  Errors: EINVAL (negative). */
shasta_status shasta_set_step_counter(shasta_ctx* ctx, int64_t steps);

/* Device counters since the state was last set: out[0] = recoveries of the
 * level-n state (each cell once per sweep) in which |M| was clamped or
 * E <= 0 (the solver's vacuum/clamp reading).  Synchronous. */
shasta_status shasta_counters(shasta_ctx* ctx, int64_t out[1]);

/* Checked builds only (the library built with SHASTA_CHECKED, a test aid
 * with no counterpart in the paper): the sweep kernels test every global
 * access (and the FP32 / MIXED ones every shared-memory access) at a
 * computed index against the bounds of its buffer and skip it if it falls
 * outside; out[0] = accesses
 * refused since the last report, out[1] / out[2] = code (1 state load,
 * 2 frozen-ghost load, 3 state store, 4 shared-memory ring, 5 range table)
 * and index of the first.  Clears the record.  Synchronous.  Errors: EINVAL
 * (NULL arguments, or a library built without the checks), ECUDA. */
shasta_status shasta_checked_report(shasta_ctx* ctx, unsigned long long out[3]);

/* The context's stream (cudaStream_t as void*). */
void* shasta_stream(const shasta_ctx* ctx);

/* Last error message of ctx, or of the calling thread's last failed create
 * when ctx is NULL.  Never NULL; "" when there was no error. */
const char* shasta_last_error(const shasta_ctx* ctx);

/* Name of a status code. */
const char* shasta_status_string(shasta_status s);

/* Library version string. */
const char* shasta_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SHASTA_H */
