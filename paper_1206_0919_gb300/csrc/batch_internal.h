// batch_internal.h -- enqueue-only batch calls for the serving loop
// (server.cu).  None of them waits for the device: they queue work on the
// batch stream in order with the steps already queued.
#pragma once

#include "../../include/shasta_batch.h"

namespace shasta {

// shasta_batch_add of device arrays without the input scan and without the
// final wait: the conversion into the pool is queued on the batch stream,
// and `fields` must stay untouched until the stream has passed it.
shasta_status batch_add_enqueue(shasta_batch* b, const shasta_grid* g, double dx, double lambda,
                                const shasta_eos* eos, const double* const fields[5], int kind,
                                int* id);

// shasta_batch_remove without the wait: the slot and its cells are free at
// once on the host, and reused only by work queued later on the batch stream.
shasta_status batch_remove_enqueue(shasta_batch* b, int id);

// Queues the event's primitives (prims[k] non-null), conserved fields
// (cons[k] non-null) into device arrays and its clamp counter into
// *counter (device memory, unsigned 64-bit).
shasta_status batch_extract_enqueue(shasta_batch* b, int id, double* const prims[6],
                                    double* const cons[5], unsigned long long* counter);

}  // namespace shasta
