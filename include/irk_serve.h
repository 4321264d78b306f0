/*
 * irk_serve.h -- serving runtime over the Gauss-IRK solver of irk.h.
 *
 * A server runs many independent IRK initial-value problems (each with its
 * own irk_config: grid, stage count, viscosity, ...) on one GPU with
 * continuous batching:
 *  - an HBM budget is reserved once; each request's solver arena is
 *    sub-allocated from it, and a request is admitted as soon as its arena
 *    (irk_config_device_bytes) fits in the free part of the budget;
 *  - up to `slots` admitted requests run at once, each on its own CUDA stream
 *    with its own worker thread, so their kernels overlap on the device; a
 *    slot that finishes admits the next waiting request immediately, while
 *    clients keep submitting;
 *  - a request's state and Krylov bases stay resident in its arena until it
 *    completes; per-step wall times give the p50/p99 step latency.
 * Results do not depend on the mix: each request computes exactly what the
 * same irk_create/irk_step sequence computes alone.
 *
 * Calls are thread-safe.  All buffers here are host memory owned by the
 * caller.  There is no counterpart in the paper; this is the serving form of
 * the method (independent requests, no communication between them).
 */
#ifndef IRK_SERVE_H
#define IRK_SERVE_H

#include <stddef.h>

#include "irk.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct irk_server irk_server;

typedef struct {
  long long submitted, completed, failed, steps;
  double wall_s;          /* first submission to last completion */
  double steps_per_s;     /* completed steps / wall_s */
  double p50_step_ms, p99_step_ms, max_step_ms;  /* wall time of one irk_step */
  double p50_request_ms, p99_request_ms;         /* submission to completion */
  double p50_queue_ms, p99_queue_ms;             /* submission to admission */
  int peak_active;        /* most requests resident at once */
  int slots;
  size_t budget_bytes, peak_bytes;               /* HBM budget and its peak use */
} irk_server_stats;

/* Start a server with `slots` (1..256) concurrent requests and an HBM budget
 * (bytes; 0 = half of the currently free device memory), reserved at once. */
irk_status irk_server_create(int slots, size_t budget_bytes, irk_server** out);

/* The batched form of the server (include/irk_batch.h): up to `capacity`
 * (1..64) resident requests are advanced together, one CUDA graph launch per
 * step covering all of them, by a single driver thread; a request is admitted
 * when a slot is free and its arena (irk_batch_instance_bytes) fits in the
 * free part of the budget, and leaves the batch when its steps are done.
 * Every request's step latency is the wall time of the batched step it took
 * part in.  With stream_slots > 0, requests of grid size n >= stream_min_n
 * are instead served as in irk_server_create by stream_slots worker threads,
 * each with its own stream, next to the batch (large grids fill the GPU on
 * their own and would hold every small request of the batch to their step
 * time).  Requests the batched path does not serve (see irk_batch.h) are
 * rejected at submission with IRK_ERR_INVALID.  A batched request's result is
 * bit for bit that of the same request alone in a batch. */
irk_status irk_server_create_batched(int capacity, int stream_slots, int stream_min_n,
                                    size_t budget_bytes, irk_server** out);

/* Queue one problem: cfg as for irk_create (not profiled), initial state u0
 * (host, ncomp*n^dim values; copied), start time t0, step dt, nsteps steps.
 * Returns its id.  IRK_ERR_NOMEM if its arena exceeds the whole budget. */
irk_status irk_server_submit(irk_server* s, const irk_config* cfg, const double* u0, double t0,
                             double dt, int nsteps, long long* id);

/* Block until request `id` is done; copy its final state to u_out (host,
 * may be NULL), its summed solver statistics to stats (may be NULL) and the
 * wall time of each of its steps to step_ms (nsteps values, may be NULL).
 * Returns the request's status.  Each id can be waited for once. */
irk_status irk_server_wait(irk_server* s, long long id, double* u_out, irk_stats* stats,
                           double* step_ms);

/* Throughput and latency statistics of the requests completed so far. */
irk_status irk_server_stats_get(irk_server* s, irk_server_stats* out);

/* Stop the workers after their running requests, drop queued ones, release
 * the budget.  NULL-safe. */
void irk_server_destroy(irk_server* s);

#ifdef __cplusplus
}
#endif

#endif /* IRK_SERVE_H */
