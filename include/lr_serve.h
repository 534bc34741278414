/* lr_serve.h -- C ABI of the serving loop: simulations submitted at any
 * time are admitted into a running batch (include/lr_batch.h) as soon as
 * its pool has a free range of units for them and a member slot, advance
 * together with whatever else is resident (continuous batching: one batched
 * launch per kernel of the step for all resident requests), and are retired
 * with their results copied to host memory when they reach their step
 * count or end time.  A worker thread owned by the server drives the GPU;
 * the calls below only exchange requests and results with it and are safe
 * to make from any host thread.
 *
 * Scheduling.  Pending requests are admitted in arrival order; one that
 * does not fit yet may be passed by later ones that do, until it has been
 * passed over `max_bypass` times, after which nothing is admitted before
 * it.  Between two scheduling points the worker runs as many steps as the
 * closest step-count completion allows (at most max_chunk_steps).
 *
 * A request's result does not depend on what else was resident: every
 * member has its own CFL time step and no data is shared between members.
 */
#ifndef LR_SERVE_H
#define LR_SERVE_H

#include <stddef.h>
#include "lr.h"
#include "lr_batch.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lr_server lr_server;

typedef struct {
  lr_batch_config batch;   /* pool, precision, member slots (cuda_stream: NULL) */
  int max_chunk_steps;     /* most steps between scheduling points (default 64) */
  int max_bypass;          /* times a waiting request may be passed over (default 8) */
  int device;              /* CUDA device the worker uses (default 0) */
} lr_server_config;

/* Result fields kept for every request: LR_F_K, LR_F_RHO_MAT, LR_F_E_MAT,
 * LR_F_P, LR_F_UX, LR_F_UY (layouts as in lr.h). */

typedef struct {
  long submitted, admitted, completed, failed;
  long pending, resident;
  double cell_updates;     /* sum over completed requests of cells x steps */
  double busy_s;           /* worker time with at least one resident request */
  long steps_launched;     /* batch steps enqueued */
} lr_server_stats;

void lr_server_config_default(lr_server_config* cfg);
lr_status lr_server_create(const lr_server_config* cfg, lr_server** out);
/* Stops the worker after the batch step in flight; pending requests are dropped. */
void lr_server_destroy(lr_server* s);
const char* lr_server_last_error(const lr_server* s);

/* Submit a request (arguments as lr_batch_add; inputs are copied before the
 * call returns).  *id receives its id.  LR_ERR_ARG: invalid request;
 * LR_ERR_OOM: it can never fit this server's pool. */
lr_status lr_server_submit(lr_server* s, const lr_config* cfg, const lr_material* mats, const double* k,
                           const double* rho, const double* p, const double* ux, const double* uy, double t_end,
                           long max_steps, long* id);

/* Wait until request id has completed or failed, or timeout_s seconds
 * (< 0: no limit).  *state: 0 not finished, 1 done, -1 failed. */
lr_status lr_server_wait(lr_server* s, long id, double timeout_s, int* state);

/* Wait until every request submitted so far has completed or failed. */
lr_status lr_server_drain(lr_server* s, double timeout_s);

/* Timing of a request on the server clock (seconds since create): submit,
 * admission and completion (result on the host); its final t and steps.
 * Any pointer may be NULL. */
lr_status lr_server_info(lr_server* s, long id, double* submit_s, double* admit_s, double* done_s, double* t,
                         long* steps);

/* One kept result field of a completed request into host memory. */
size_t lr_server_result_size(lr_server* s, long id, int field);
lr_status lr_server_result(lr_server* s, long id, int field, double* out, size_t n);

/* Drop a finished request's stored result. */
lr_status lr_server_release(lr_server* s, long id);

lr_status lr_server_get_stats(lr_server* s, lr_server_stats* out);

/* Seconds on the server clock now. */
double lr_server_clock(const lr_server* s);

#ifdef __cplusplus
}
#endif
#endif
