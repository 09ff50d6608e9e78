/*
 * shasta_batch.h -- many independent events advanced together (C ABI).
 *
 * A batch keeps the state of many events in one device pool and advances
 * every resident event with one launch per sweep axis over a work list of
 * its events (work units: whole line groups, or equal ranges of positions
 * that may cut lines), instead of one launch per event and sweep.  The paper weighs the size of a kernel's working set against the
 * cost of orchestrating many kernel calls from the host (Sec. 3.1.2) and
 * enqueues the sweeps of one grid from a host loop (Sec. 3.1.3); here the
 * work of all events of a sweep shares a launch, and six steps of launches
 * are replayed as one CUDA graph while the batch does not change.
 *
 * Every event is advanced exactly as a single context with the same grid,
 * boundary rule, EoS, lambda and options would advance it (shasta.h): the
 * same arithmetic in the same order, so the results agree bit for bit.  Each
 * event keeps its own step counter, so events added at different times run
 * their own phase of the axis permutation (Sec. 3.1.4); the events of one
 * launch may differ in everything but the precision, eta and delta, which
 * belong to the batch.
 *
 * Conventions are those of shasta.h (arrays FP64, x fastest, host or device
 * memory, copied in and out, status codes, one host thread per batch).
 */
#ifndef SHASTA_BATCH_H
#define SHASTA_BATCH_H

#include "shasta.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct shasta_batch shasta_batch;

/* Kind of the five arrays handed to shasta_batch_add. */
enum { SHASTA_STATE_CONSERVED = 0, SHASTA_STATE_PRIMITIVE = 1 };

typedef struct shasta_batch_opts {
  int precision;          /* SHASTA_FP32 or SHASTA_MIXED (FP64 events use shasta.h) */
  double eta;             /* antidiffusion coefficient, default 1/8 */
  double delta;           /* |M| <= (1 - delta) E; 0 selects 1e-6 */
  void* stream;           /* cudaStream_t to use, or NULL for a stream of the batch's own */
  int device;             /* CUDA device ordinal */
  int check_input;        /* nonzero: reject unphysical input arrays (default 1) */
  int autotune;           /* nonzero: time launch choices when the batch has changed (default 1) */
  int use_graphs;         /* nonzero: replay six steps as one CUDA graph (default 1) */
  int max_events;         /* resident events at most, 1..65536 (default 1024) */
  int64_t capacity_cells; /* cells of state the pool holds (sum over resident events); required */
} shasta_batch_opts;

/* Fills *o with the defaults above (capacity_cells = 0: must be set). */
void shasta_batch_default_opts(shasta_batch_opts* o);

/* Creates a batch and allocates its pool: 40 bytes per cell of capacity
 * (two buffers of an (E, Mx, My, Mz) float quad and an R float) plus small
 * tables.  Errors: EINVAL (options), ENOMEM, ECUDA; the message is in
 * shasta_batch_last_error(NULL). */
shasta_status shasta_batch_create(const shasta_batch_opts* o, shasta_batch** out);

/* Waits for the batch's work and frees everything it holds. */
shasta_status shasta_batch_destroy(shasta_batch* b);

/* Adds an event: grid, dx, lambda and EoS as for shasta_create, initial
 * state in five arrays (E, Mx, My, Mz, R) or (e, vx, vy, vz, n) by `kind`,
 * in host or device memory by `mem`.  The arrays are copied; the event's
 * step counter starts at 0.  *id receives the event's handle (>= 0), valid
 * until shasta_batch_remove.  Synchronous.  Errors: EINVAL (arguments),
 * EUNPHYSICAL (check_input and bad cells), EAGAIN (no free slot, or no
 * contiguous room for the grid in the pool: remove events first), ENOMEM,
 * ECUDA. */
shasta_status shasta_batch_add(shasta_batch* b, const shasta_grid* g, double dx, double lambda,
                               const shasta_eos* eos, const double* const fields[5], int kind,
                               int mem, int* id);

/* Removes an event and frees its room in the pool (after the work already
 * enqueued has finished with it).  Errors: ENOTFOUND. */
shasta_status shasta_batch_remove(shasta_batch* b, int id);

/* Enqueues nsteps full split steps of every resident event and returns.
 * Errors: EINVAL (nsteps < 0), ECUDA. */
shasta_status shasta_batch_step(shasta_batch* b, int nsteps);

/* Waits until the batch's enqueued work has finished. */
shasta_status shasta_batch_sync(shasta_batch* b);

/* Times launch choices (register variant, segment length) per axis on the
 * resident events without changing their state and keeps the fastest.
 * shasta_batch_step does this by itself when autotune is set and the set of
 * events has changed since the last tuning. */
shasta_status shasta_batch_autotune(shasta_batch* b);

/* Copies an event's conserved state (E, Mx, My, Mz, R; a NULL entry skips
 * that field) or its primitives (e, vx, vy, vz, n, p) out.  Synchronous.
 * Errors: ENOTFOUND, EINVAL. */
shasta_status shasta_batch_get_conserved(shasta_batch* b, int id, double* const out[5], int mem);
shasta_status shasta_batch_get_primitives(shasta_batch* b, int id, double* const out[6], int mem);

/* Sums of E, Mx, My, Mz, R of one event (as shasta_totals).  Synchronous. */
shasta_status shasta_batch_totals(shasta_batch* b, int id, double out[5]);

/* Steps the event has taken since it was added, or -1 if id is unknown. */
int64_t shasta_batch_steps_done(const shasta_batch* b, int id);

/* Sets an event's step counter (the phase of the axis permutation is this
 * mod 6), e.g. to resume an event saved with shasta_batch_get_conserved and
 * shasta_batch_steps_done.  Errors: ENOTFOUND, EINVAL (negative). */
shasta_status shasta_batch_set_step_counter(shasta_batch* b, int id, int64_t steps);

/* Clamp / vacuum recoveries of the event since it was added (as
 * shasta_counters).  Synchronous. */
shasta_status shasta_batch_counters(shasta_batch* b, int id, int64_t out[1]);

/* Checked builds only: as shasta_checked_report, for the batched sweeps of
 * all events (waits for the whole device).  Errors: EINVAL (NULL arguments,
 * or a library built without the checks), ECUDA. */
shasta_status shasta_batch_checked_report(shasta_batch* b, unsigned long long out[3]);

/* out[0] resident events, out[1] cells in use, out[2] capacity in cells,
 * out[3] largest free run of cells, out[4] kernel launches per step of the
 * current work lists, out[5] work items per step, out[6] sweep kernel
 * launches issued since creation (those replayed in graphs included; the
 * autotuner's trial launches not). */
shasta_status shasta_batch_info(shasta_batch* b, int64_t out[7]);

/* The batch's stream (cudaStream_t as void*). */
void* shasta_batch_stream(const shasta_batch* b);

/* Last error message of the batch, or of the calling thread's last failed
 * shasta_batch_create when b is NULL.  Never NULL; "" if none. */
const char* shasta_batch_last_error(const shasta_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* SHASTA_BATCH_H */
