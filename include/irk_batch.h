/*
 * irk_batch.h -- many independent Gauss-IRK problems advanced in lock step,
 * each kernel launch covering all of them.
 *
 * A batch holds up to `capacity` resident instances of the 2D viscous Burgers
 * problem of irk.h (IRK_OP_BURGERS_2D), each with its own grid size n, stage
 * count s, viscosity nu, step dt and Newton/Krylov tolerances.  One call of
 * irk_batch_step advances every resident instance by one step of its own dt
 * (Algorithm 1 of Sec. 5 per instance: the Newton-like iteration with the
 * block-diagonal Jacobian of Sec. 3.2 (nonlinear_variant 2), flexible GMRES on
 * each diagonal block of the real Schur form, the preconditioner L_P of
 * Eq. Lprec with gamma* and one geometric-multigrid V-cycle per inner inverse),
 * as ONE CUDA graph:
 *  - each kernel is a persistent launch (a fixed grid) that walks a table of
 *    work chunks spanning every instance (or every block solve, or every
 *    multigrid row) taking part in that phase, so instances of different
 *    sizes share one launch;
 *  - the Newton loop and the FGMRES loop are conditional WHILE nodes that run
 *    while any instance (block solve) is still iterating; an instance (block)
 *    that has converged skips the work of the later iterations;
 *  - per-instance reductions are summed in a fixed order over that instance's
 *    own chunks, so an instance computes the same numbers bit for bit whatever
 *    else is in the batch.
 * The graph is captured again only when the launch structure changes (the
 * deepest V-cycle or the largest sweep count among the residents); otherwise
 * admitting or removing an instance only rewrites the chunk tables.
 *
 * Accepted configurations: op = IRK_OP_BURGERS_2D, mass identity, family
 * IRK_GAUSS or IRK_RADAU_IIA, basis IRK_BASIS_SCHUR, mg_precision FP64,
 * nonlinear_variant 2, no forcing, n a power of two in 32..2048,
 * krylov_restart <= 30.  Each V-cycle row must be shift dominated on its
 * coarsest level (sigma >= D/2 there, the depth rule of the single-instance
 * solver), which holds whenever dt nu is small against h^2 on some level of
 * the hierarchy; other configurations are rejected with IRK_ERR_INVALID.
 * Each FGMRES block solve runs one cycle of at most krylov_restart
 * iterations per Newton iteration (inexact Newton absorbs an early stop).
 *
 * Memory: each instance lives in one arena, either caller-owned (a memory
 * manager that owns the device pool; 256-byte aligned, at least
 * irk_batch_instance_bytes) or allocated by irk_batch_add (arena = NULL).
 * The batch itself allocates its tables once at irk_batch_create.
 * The paper has no counterpart: this is the batched serving form of the method.
 */
#ifndef IRK_BATCH_H
#define IRK_BATCH_H

#include <stddef.h>

#include "irk.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct irk_batch irk_batch;

/* A batch of up to `capacity` (1..64) instances on the current device; work
 * goes to cuda_stream (NULL: a stream the batch creates).  Every later call
 * on the batch makes that device current while it runs and gives the
 * caller's current device back on return. */
irk_status irk_batch_create(int capacity, void* cuda_stream, irk_batch** out);

/* Device bytes of one instance's arena for cfg (host-only); 0 if cfg is not
 * accepted (see above). */
size_t irk_batch_instance_bytes(const irk_config* cfg);

/* Admit one instance with state u0 (2 n^2 values, u then v; host or device
 * memory) and step dt into a free slot (*slot, 0..capacity-1).  arena: NULL
 * (the batch allocates) or caller-owned device memory of arena_bytes >=
 * irk_batch_instance_bytes(cfg).  The instance starts with zero stages. */
irk_status irk_batch_add(irk_batch* b, const irk_config* cfg, const double* u0, int u0_on_device,
                         double dt, void* arena, size_t arena_bytes, int* slot);

/* Advance every resident instance by one step of its own dt (one graph
 * launch; returns when done).  stats: NULL or an array of `capacity` entries;
 * entry k receives slot k's counters of this step (zeroed for free slots) and
 * status: NULL or `capacity` entries, IRK_OK or the Newton failure of slot
 * k.  A failed instance keeps its state of the previous step and restarts its
 * next step from zero stages.  Returns IRK_OK unless the launch failed. */
irk_status irk_batch_step(irk_batch* b, irk_stats* stats, irk_status* status);

/* State of slot k (2 n^2 values) to host or device memory. */
irk_status irk_batch_get_state(irk_batch* b, int slot, double* dst, int dst_on_device);

/* Stage vectors k_1..k_s of slot k's last accepted step (s 2 n^2 values). */
irk_status irk_batch_get_stages(irk_batch* b, int slot, double* dst, int dst_on_device);

/* Free slot k (its arena is released if the batch allocated it). */
irk_status irk_batch_remove(irk_batch* b, int slot);

/* Resident instances. */
int irk_batch_count(const irk_batch* b);

/* Text of the last failure on b (valid until the next call on b). */
const char* irk_batch_last_error(const irk_batch* b);

/* Release the batch and every arena it allocated.  NULL-safe. */
void irk_batch_destroy(irk_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* IRK_BATCH_H */
