/*
 * shasta_serve.h -- a serving loop over the batched solver (C ABI).
 *
 * Events of different grid sizes arrive as they come (shasta_submit never
 * blocks).  A worker thread of the server admits them into one resident
 * batch (shasta_batch.h) at the boundaries of the resident events' six-step
 * axis cycle (Sec. 3.1.4), first come first served, as soon as a slot,
 * contiguous room in the state pool and staging memory are free and their
 * input has been copied in and scanned for unphysical values: admission is
 * by device-memory footprint (40 bytes per cell of state
 * plus 40 bytes per cell of input staging while it is copied in and 8 per
 * cell and output field, plus 8 for the clamp counter, while the results
 * are copied out; staging_bytes is
 * split evenly between input and output staging).  All resident events
 * advance together in the batched launches; an event leaves the batch after
 * its own number of steps, its results are copied into the caller's buffers
 * and its room goes to the next event in the queue.  Input copies of queued
 * events and output copies of finished ones run on copy streams while the
 * resident events compute; the worker only queues work on the device, at
 * most two rounds ahead of it.
 *
 * Each event advances exactly as it would alone (bit for bit: the batched
 * launch runs the single-event arithmetic), whatever else is resident.
 *
 * The paper has no serving loop: it runs one grid per device (Sec. 3.1);
 * this layer is for many independent events on one GPU.
 */
#ifndef SHASTA_SERVE_H
#define SHASTA_SERVE_H

#include "shasta_batch.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct shasta_server shasta_server;

typedef struct shasta_server_opts {
  int precision;            /* SHASTA_FP32 or SHASTA_MIXED */
  double eta;               /* antidiffusion coefficient, default 1/8 */
  double delta;             /* |M| <= (1 - delta) E; 0 selects 1e-6 */
  int device;               /* CUDA device ordinal */
  int64_t hbm_budget_bytes; /* device memory the server holds: state pool + staging (required) */
  int64_t staging_bytes;    /* the staging part of the budget (half input, half output); 0: an eighth */
  int max_resident;         /* events advanced together at most (default 256) */
  int max_queue;            /* submitted events not yet resident at most (default 4096) */
  int steps_per_round;      /* at most this many steps between admission checks
                               (default 6).  Events join only at phase 0 of the
                               resident events' six-step axis cycle, and rounds
                               end on those boundaries */
} shasta_server_opts;

/* One event.  fields: five host arrays (E, Mx, My, Mz, R) or (e, vx, vy,
 * vz, n) by kind, nx*ny*nz each, x fastest; copied by shasta_submit.
 * out_prims / out_cons: host buffers of nx*ny*nz doubles that receive the
 * primitives (e, vx, vy, vz, n, p) and the conserved fields (E, Mx, My, Mz,
 * R) after the last step (NULL entries are skipped); the caller keeps them
 * valid and untouched until shasta_poll reports the event finished. */
typedef struct shasta_event {
  shasta_grid grid;
  double dx, lambda;
  shasta_eos eos;
  const double* fields[5];
  int kind;   /* SHASTA_STATE_CONSERVED or SHASTA_STATE_PRIMITIVE */
  int nsteps; /* full split steps to run, >= 0 */
  double* out_prims[6];
  double* out_cons[5];
} shasta_event;

/* Timings of a finished event, in seconds on the server's clock
 * (shasta_server_clock): submitted, admitted into the batch, results in the
 * caller's buffers. */
typedef struct shasta_result {
  double t_submit, t_admit, t_done;
  int64_t steps;       /* steps taken */
  int64_t clamp_count; /* as shasta_counters */
} shasta_result;

/* Defaults of the options above (hbm_budget_bytes = 0: must be set). */
void shasta_server_default_opts(shasta_server_opts* o);

/* Creates the server, its state pool and staging memory, and starts its
 * worker thread.  Errors: EINVAL, ENOMEM, ECUDA (message in
 * shasta_server_last_error(NULL)). */
shasta_status shasta_server_create(const shasta_server_opts* o, shasta_server** out);

/* Stops the worker after its current round and frees everything; events
 * not finished by then are dropped (their buffers are not written later). */
shasta_status shasta_server_destroy(shasta_server* s);

/* Queues an event and returns at once with its ticket (> 0).  Errors:
 * EINVAL (arguments, or a grid that can never fit the pool or the staging
 * memory), EAGAIN (max_queue events are waiting), ENOMEM (host copy),
 * ECUDA (the server stopped after a device error). */
shasta_status shasta_submit(shasta_server* s, const shasta_event* ev, uint64_t* ticket);

/* State of a ticket: EAGAIN while the event is queued or running; OK once
 * its results are in the caller's buffers (*out filled, the ticket is then
 * forgotten); the event's own error (EUNPHYSICAL for bad input, ECUDA)
 * if it failed (also forgets the ticket); ENOTFOUND for unknown tickets. */
shasta_status shasta_poll(shasta_server* s, uint64_t ticket, shasta_result* out);

/* Waits until every submitted event has finished or failed, at most
 * timeout_s seconds.  Errors: ETIMEOUT, ECUDA. */
shasta_status shasta_server_drain(shasta_server* s, double timeout_s);

/* out[0] submitted, out[1] finished, out[2] failed, out[3] waiting in the
 * queue, out[4] resident or being copied in/out, out[5] most events ever
 * resident at once, out[6] batched steps run, out[7] state pool capacity
 * in cells, out[8] sweep kernel launches issued, out[9..15] seconds the
 * worker spent copying inputs in, admitting, harvesting results, enqueueing
 * steps, copying results out, waiting for the steps, and idle. */
shasta_status shasta_server_stats(shasta_server* s, double out[16]);

/* Seconds since the server was created (steady clock). */
double shasta_server_clock(const shasta_server* s);

/* Last error message of the server, or of the calling thread's last failed
 * create when s is NULL.  Never NULL. */
const char* shasta_server_last_error(const shasta_server* s);

#ifdef __cplusplus
}
#endif

#endif /* SHASTA_SERVE_H */
