/* lr_batch.h -- C ABI of the batched Lagrange-Remap step: many independent
 * 2D simulations of different sizes, each its own lr_config, advanced
 * together on one GPU with one launch per kernel of the step for the whole
 * batch (kernels grouped by material count), captured in a CUDA graph.
 *
 * Every member runs exactly the step of include/lr.h (staggered Lagrange
 * phase of section 1.2 with the multi-material closure of section 4.1,
 * DirectCF face and corner remap of section 2.3 with the VOF/PLIC material
 * split of section 4.4, dual-mesh momentum remap, CFL rule) with its own
 * time step: the CFL minimum is reduced per member on the device, so a
 * member's dt never depends on the other members (a member's result is the
 * same alone and in any mix).
 *
 * Memory.  The library owns one device pool of `capacity_units` units.  A
 * member on an nx x ny grid occupies (nx+2)(ny+2) consecutive units; every
 * per-cell, per-node, per-face and per-dual-cell array of the step lives in
 * the pool at the member's unit offset.  lr_batch_add admits a member only
 * when such a range is free (first fit), so the pool's HBM footprint is the
 * admission criterion; lr_batch_remove frees the range.
 *
 * Threading: one batch per host thread; every call is stream-ordered on the
 * batch's stream.  Errors: calls return lr_status; lr_batch_last_error
 * gives the message.  A numeric failure of one member (see lr_step) marks
 * that member failed (lr_batch_status) and stops it; the others continue.
 */
#ifndef LR_BATCH_H
#define LR_BATCH_H

#include <stddef.h>
#include "lr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lr_batch lr_batch;

typedef struct {
  int precision;           /* LR_FP64, LR_DF64 or LR_FP32, for every member */
  int nmat_max;            /* 1..3: material planes in the pool; members have nmat <= nmat_max */
  long capacity_units;     /* pool size in units (a member takes (nx+2)(ny+2)) */
  int capacity_members;    /* most members resident at once (>= 1) */
  long max_member_cells;   /* largest nx*ny a member may have (sizes the init staging) */
  void* cuda_stream;       /* cudaStream_t to run on; NULL = library-owned stream */
} lr_batch_config;

/* Defaults: FP64, nmat_max 3, 16 members, 2^20 units, 2^20 cells per member. */
void lr_batch_config_default(lr_batch_config* cfg);

/* Device bytes the pool and its bookkeeping take for this configuration. */
lr_status lr_batch_workspace_bytes(const lr_batch_config* cfg, size_t* bytes);

/* Bytes one unit of the pool costs (all arrays), for sizing the pool
 * from an HBM budget. */
lr_status lr_batch_unit_bytes(const lr_batch_config* cfg, size_t* bytes);

lr_status lr_batch_create(const lr_batch_config* cfg, lr_batch** out);
void lr_batch_destroy(lr_batch* b);
const char* lr_batch_last_error(const lr_batch* b);

/* Admit a member.  cfg: its grid and scheme options (cfg->precision must be
 * the batch's; cfg->cuda_stream is ignored; prescribed velocities are not
 * available in a batch).  mats: cfg->nmat materials.  k, rho, p, ux, uy: its
 * initial state as in lr_init (host arrays, copied before the call returns).
 * The member advances until t reaches t_end or it has taken max_steps steps
 * (max_steps <= 0: no step limit).  *member receives its id (>= 0).
 * Returns LR_ERR_OOM, with nothing changed, when no free range of units or
 * member slot is available now; LR_ERR_ARG for an invalid configuration or
 * state (then the state check of lr_init applies: *member is still set and
 * the member is marked failed). */
lr_status lr_batch_add(lr_batch* b, const lr_config* cfg, const lr_material* mats, const double* k,
                       const double* rho, const double* p, const double* ux, const double* uy, double t_end,
                       long max_steps, int* member);

/* Change a member's end time and step limit (max_steps <= 0: none); a
 * member that had stopped resumes when the new limits allow another step. */
lr_status lr_batch_set_limits(lr_batch* b, int member, double t_end, long max_steps);

/* Release a member and its units (its results are no longer readable). */
lr_status lr_batch_remove(lr_batch* b, int member);

/* Enqueue nsteps steps of every live member (asynchronous; idle members,
 * finished ones included, cost only an early exit).  The step sequence is
 * replayed from a CUDA graph that is re-captured when membership changes. */
lr_status lr_batch_step(lr_batch* b, int nsteps);

/* Wait for the batch's stream. */
lr_status lr_batch_sync(lr_batch* b);

/* Per-member progress (synchronises): t, steps taken, and state: 0 running,
 * 1 done (t_end or the step limit reached), -1 failed (numeric error, or an
 * invalid initial state).  Any pointer may be NULL. */
lr_status lr_batch_status(lr_batch* b, int member, double* t, long* steps, int* state);

/* Status of every slot at once (synchronises): state[s] as above, or -2
 * for an empty slot; steps[s] steps taken.  n >= capacity_members. */
lr_status lr_batch_status_all(lr_batch* b, int* state, long* steps, int n);

/* Field LR_F_* of a member (layout and size as lr_field_size would give for
 * its configuration); lr_batch_field_size gives the count. */
size_t lr_batch_field_size(const lr_batch* b, int member, int field);
lr_status lr_batch_get_fields(lr_batch* b, int member, int field, double* host_out, size_t n_elems);

/* Choose, per kernel, the tile shape (32x8, 64x4, 16x16, 128x2 threads) and
 * the number of persistent blocks, and the lanes per mixed cell, by timing
 * trial steps of the current members (trial_steps each, at least 1); then,
 * unless lr_batch_set_persistent was called, time whole steps of that
 * schedule against the persistent step and keep the faster.  The members'
 * state, time and step counts are restored afterwards. */
lr_status lr_batch_autotune(lr_batch* b, int trial_steps);

/* The schedule in use: for each of the nine step kernels (the order of
 * lr_kernel_times), its tile shape index (0..3 as above) and blocks per
 * SM (0 = one block per tile); lanes per mixed cell.  Arrays of 9. */
lr_status lr_batch_schedule(const lr_batch* b, int* tile_shape, int* blocks_per_sm, int* mixed_lanes);

/* Kernel launches the last step enqueued (all groups). */
int lr_batch_launches_per_step(const lr_batch* b);

/* Persistent step (on by default in LR_FP32 where the device can hold it
 * resident, off in LR_FP64 and LR_DF64; lr_batch_autotune picks between the
 * two paths unless this call has set one):
 * each step is one cooperative launch of co-resident blocks that walk every
 * member's 32 x 8 cell tiles and node tiles through the phases of the tiled
 * step (the Lagrange phase and remap geometry of section 1.2 and 2.3; the
 * interface lines and material fluxes of the mixed cells, section 4.4; the
 * material fluxes and cell update; the dual remap and node update of
 * section 2.1.1 with each member's own CFL time step), separated by grid-wide
 * barriers.  Every barrier wait has a limit (1 s); a wait that runs out
 * abandons the step, and lr_batch_sync then returns LR_ERR_TIMEOUT, as does
 * every later call that steps the batch (the batch has to be destroyed).
 * Off: one launch per kernel and material-count group, with the schedule
 * lr_batch_autotune picks (the autotuner times that path).
 * lr_batch_get_persistent returns 1 when the persistent step is in use. */
lr_status lr_batch_set_persistent(lr_batch* b, int on);
int lr_batch_get_persistent(const lr_batch* b);

/* Test hook of the persistent step's barrier: each barrier waits for
 * extra_arrivals arrivals that no block makes (0: none, the normal
 * setting), and gives up after limit_s seconds (default 1; at most 10). */
lr_status lr_batch_test_barrier(lr_batch* b, unsigned int extra_arrivals, double limit_s);

/* Per-kernel timing with CUDA events around every launch (profiling mode
 * launches without the graph); as lr_set_profiling / lr_kernel_times. */
lr_status lr_batch_set_profiling(lr_batch* b, int on);
int lr_batch_kernel_times(lr_batch* b, const char** names, long* launches, double* ms, int n);

#ifdef __cplusplus
}
#endif
#endif
