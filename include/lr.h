/*
 * lr.h -- C ABI of the GB300 (sm_103a) Lagrange-Remap library.
 *
 * One call of lr_step advances a 2D multi-material compressible-Euler state by
 * one time step of the scheme of Chaudet, "A scalable Lagrange-Remap scheme
 * for compressible multimaterial Euler equations with sharp interface
 * reconstruction" (arXiv 2208.13409):
 *   - the staggered-grid predictor-corrector (SGPC) Lagrange phase, section
 *     1.2 (eqs. "prediction" and "correction") in the iso-deformation
 *     multi-material form of section 4.1, with per-material EOS and Wilkins
 *     pseudo-viscosity;
 *   - the one-step "Direct with Corner Fluxes" remap of section 2.3, face and
 *     corner volume fluxes, limited linear reconstruction of section 2.1.1 at
 *     faces and the diagonal limited reconstruction of section 3.3 at corners;
 *   - VOF/PLIC material fluxes on the rectangular Lagrangian cell, section
 *     4.4, with Youngs normals (section 4.1, "interface positioning");
 *   - the dual-mesh momentum remap of sections 2.1.1 and 2.3;
 *   - the global CFL minimum (annex definition CFL = dt c / dx).
 *
 * Every phase runs in hand-written CUDA kernels on one GPU.  The library owns
 * its device state; the caller owns every host buffer it passes.
 *
 * Layout: cells (i,j), 0<=i<nx, 0<=j<ny, stored [j][i] (x fastest); nodes
 * (i,j), 0<=i<=nx, 0<=j<=ny, stored [(ny+1)][(nx+1)]; per-material fields
 * [nmat][ny][nx].  All values are IEEE double.
 *
 * Errors: every call returns an lr_status; lr_last_error() gives a message.
 * A numeric failure inside a step (non-positive volume, density or squared
 * sound speed, NaN, tangled flux geometry) is detected on the device and
 * reported by the next synchronising call; the context then stays in error
 * until lr_init.  Calls on one context are not thread-safe; distinct
 * contexts are independent.
 */
#ifndef LR_H
#define LR_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct lr_ctx lr_ctx;

typedef enum {
  LR_OK = 0,
  LR_ERR_ARG = -1,      /* invalid argument or configuration */
  LR_ERR_OOM = -2,      /* device allocation failed / workspace too small */
  LR_ERR_NUMERIC = -3,  /* numeric failure detected during a step */
  LR_ERR_TIMEOUT = -4,  /* reserved: a bounded device wait gave up */
  LR_ERR_STATE = -5,    /* call out of order (e.g. lr_step before lr_init) */
  LR_ERR_CUDA = -6      /* CUDA runtime error (message in lr_last_error) */
} lr_status;

enum { LR_BC_REFLECT = 0, LR_BC_PERIODIC = 1 };
enum { LR_EOS_IDEAL = 0, LR_EOS_STIFFENED = 1 };
/* Corner values of the remap (lr_config.corner_recon, section 3.3): upwind;
 * diagonal limited linear (default); diagonal average of donor and
 * receiver, clamped to the donor value; x-y limited linear; multidimensional
 * least-squares plane with a scalar limiter (also used for the face values
 * when face_order is 2).  The dual mesh uses the diagonal reconstruction for
 * every second-order choice. */
enum { LR_CORNER_UPWIND = 0, LR_CORNER_DIAG = 1, LR_CORNER_AVG = 2, LR_CORNER_XY = 3, LR_CORNER_LSQ = 4 };
/* Remap of the step (lr_config.remap):
 *   LR_REMAP_DIRECTCF  one step with face and corner fluxes (section 2.3; default);
 *   LR_REMAP_DIRECT    one step with face fluxes only, the faces moving with
 *                      their mean node velocity (section 2.2; multi-material:
 *                      one interface displaced along X for the X faces, one
 *                      along Y for the Y faces, section 4.3);
 *   LR_REMAP_AD        alternate directions (section 2.1): an X remap then a
 *                      Y remap, Y then X on every other step; multi-material
 *                      interfaces re-placed before each sweep (section 4.3).
 * The comparator remaps exist to compare against; they are not available in
 * a batch (include/lr_batch.h). */
enum { LR_REMAP_DIRECTCF = 0, LR_REMAP_DIRECT = 1, LR_REMAP_AD = 2 };
/* Arithmetic of the step (lr_config.precision):
 *   LR_FP64  native IEEE double (GB300 runs FP64 at 1/64 of its FP32 rate);
 *   LR_DF64  double-float: each value is an unevaluated sum of two floats
 *            (about 48 significand bits) computed on the FP32 pipe with
 *            error-free transformations; interface geometry stays in FP64;
 *   LR_FP32  single precision bulk (Lagrange phase and remap in float,
 *            interface geometry, flux clipping and conservation sums in
 *            FP64): the accuracy/throughput trade-off mode.
 * The state is stored in the step's type; lr_init and lr_get_fields
 * convert from and to double. */
enum { LR_FP64 = 0, LR_DF64 = 1, LR_FP32 = 2 };

/* Material EOS, section 5.2: p = (gamma - 1) rho e - pi; pi = 0 is the
 * perfect gas p = (gamma - 1) rho e of section 5.1.  gamma > 1, pi >= 0. */
typedef struct {
  int eos;       /* LR_EOS_IDEAL or LR_EOS_STIFFENED (informative; pi decides) */
  double gamma;
  double pi;
} lr_material;

typedef struct {
  int nx, ny;             /* cells, each >= 2; nx*ny <= 2^28 */
  double x0, x1, y0, y1;  /* domain, x1 > x0, y1 > y0 */
  int nmat;               /* 1..3 materials */
  double cfl;             /* CFL number of the time-step rule (0.25 default) */
  double a1, a2;          /* Wilkins linear / quadratic coefficients (0.5, 1.0) */
  int bc[4];              /* xlo, xhi, ylo, yhi: LR_BC_REFLECT | LR_BC_PERIODIC (a periodic
                             direction needs at least 3 cells);
                             xlo == xhi and ylo == yhi */
  int precision;          /* LR_FP64 (default), LR_DF64 or LR_FP32 */
  int face_order;         /* 1 upwind or 2 Van Leer limited linear (default 2) */
  int corner_recon;       /* LR_CORNER_* (default LR_CORNER_DIAG) */
  double dt_fixed;        /* > 0: use this dt instead of the CFL rule */
  int mixed_lanes;        /* threads per mixed cell in the interface kernel:
                             1, 2, 4 or 8; 0 (default) picks per precision */
  int remap;              /* LR_REMAP_DIRECTCF (default), LR_REMAP_DIRECT or LR_REMAP_AD */
  void* cuda_stream;      /* cudaStream_t to run on; NULL = library-owned stream */
} lr_config;

/* Fill *cfg with the defaults above (reflective walls, CFL 0.25, order 2,
 * diagonal corners, FP64, library stream).  nx, ny, domain and nmat still
 * have to be set. */
void lr_config_default(lr_config* cfg);

/* Bytes of device memory lr_create_in needs for this configuration. */
lr_status lr_workspace_bytes(const lr_config* cfg, size_t* bytes);

/* Create a context; the library allocates its device state with cudaMalloc.
 * *out receives the context (NULL on failure). */
lr_status lr_create(const lr_config* cfg, lr_ctx** out);

/* Create a context inside caller-owned device memory `dev_mem` (at least
 * lr_workspace_bytes bytes, 256-byte aligned, on the current device).  The
 * caller keeps ownership and must keep it alive until lr_destroy. */
lr_status lr_create_in(const lr_config* cfg, void* dev_mem, size_t bytes, lr_ctx** out);

/* Per-material EOS constants (section 5.2 form).  mats[nmat]. */
lr_status lr_set_materials(lr_ctx* ctx, int nmat, const lr_material* mats);

/* Upload an initial state from host memory (section 4.1 variables):
 *   k   [nmat][ny][nx] volume fractions in [0,1], summing to 1 per cell;
 *   rho [nmat][ny][nx] material densities (> 0 where k > 1e-12, else ignored);
 *   p   [nmat][ny][nx] material pressures (e is derived from the EOS);
 *   ux, uy [(ny+1)][(nx+1)] node velocities (wall-normal components are
 *   set to zero on reflective walls).
 * Materials with k <= 1e-12 are dropped and the others renormalised.  Sets
 * t = 0 and computes the first CFL time step.  Clears a sticky error. */
lr_status lr_init(lr_ctx* ctx, const double* k, const double* rho, const double* p,
                  const double* ux, const double* uy);

/* Checkpoint and resume: lr_checkpoint_save copies the context's current
 * state exactly (the state in the step's own arithmetic type, the cell
 * sound speeds of the CFL rule, the time, the step count and the time step
 * in flight) into the caller's host buffer of lr_checkpoint_bytes bytes
 * (synchronises; LR_ERR_STATE before lr_init, LR_ERR_ARG if the buffer is
 * too small; a sticky numeric error is returned instead of saving).
 * lr_checkpoint_load restores such a buffer into a context of the same grid,
 * material count, precision, remap and corner values (LR_ERR_ARG
 * otherwise; materials must be set), after which lr_step continues exactly
 * where the saved run would have: N steps, save, load (in this or a fresh
 * context), N steps equal 2N steps bit for bit.  The buffer belongs to the
 * caller; its layout is an 8-word header, the scalars, then the arrays. */
size_t lr_checkpoint_bytes(const lr_ctx* ctx);
lr_status lr_checkpoint_save(lr_ctx* ctx, void* host_buf, size_t bytes);
lr_status lr_checkpoint_load(lr_ctx* ctx, const void* host_buf, size_t bytes);

/* Prescribed node velocity (host arrays [(ny+1)][(nx+1)]), re-imposed every
 * step: the momentum equation and the dual remap are skipped and u^{n+1/2} =
 * u^{lag} = u^{n+1} = the given field (the imposed-velocity tests of section
 * 5.1).  NULL, NULL switches it off. */
lr_status lr_set_prescribed_velocity(lr_ctx* ctx, const double* ux, const double* uy);

/* One time step (section 1.2 Lagrange phase, then the section 2.3 remap):
 * dt = min(CFL rule, t_end - t).  When t >= t_end nothing changes and dt = 0.
 * With dt_taken == NULL the call only enqueues work on the stream (no host
 * synchronisation; errors surface at the next synchronising call); otherwise
 * it waits and stores the dt used. */
lr_status lr_step(lr_ctx* ctx, double t_end, double* dt_taken);

/* Up to max_steps steps towards t_end, enqueued as CUDA-graph launches with
 * the time step kept on the device; synchronises at the end.  steps_done and
 * t_now (either may be NULL) receive the steps that advanced time and the
 * final time. */
lr_status lr_run(lr_ctx* ctx, double t_end, long max_steps, long* steps_done, double* t_now);

/* Wait for queued work; return the sticky status. */
lr_status lr_sync(lr_ctx* ctx);

/* Field identifiers for lr_get_fields. */
enum {
  LR_F_K = 0,        /* [nmat][ny][nx] volume fractions */
  LR_F_RHO_MAT = 1,  /* [nmat][ny][nx] material densities (0 where absent) */
  LR_F_E_MAT = 2,    /* [nmat][ny][nx] material specific internal energies */
  LR_F_P = 3,        /* [ny][nx] mixture pressure sum_a k_a P_a */
  LR_F_RHO = 4,      /* [ny][nx] mixture density sum_a k_a rho_a */
  LR_F_E = 5,        /* [ny][nx] mixture specific internal energy */
  LR_F_UX = 6,       /* [(ny+1)][(nx+1)] node velocity x */
  LR_F_UY = 7,       /* [(ny+1)][(nx+1)] node velocity y */
  LR_F_CONS = 8,     /* [8] mass per material (3 slots), mass, momentum x, y,
                        internal energy, total energy (wall nodes weighted
                        1/2, corners 1/4) */
  LR_F_C = 9,        /* [ny][nx] cell sound speed used by the CFL rule */
  LR_F_UHX = 20,     /* [(ny+1)][(nx+1)] u^{n+1/2} of the last step */
  LR_F_UHY = 21,
  LR_F_VOL_LAGCF = 22, /* [ny][nx] flux-consistent Lagrangian volume, last step */
  LR_F_E_LAG = 23,   /* [nmat][ny][nx] e^{n+1,lag}, last step */
  LR_F_FX = 24,      /* [ny][nx+1] X-face volume flux (+ towards +x), last step */
  LR_F_FY = 25,      /* [ny+1][nx] Y-face volume flux (+ towards +y) */
  LR_F_FC = 26,      /* [(ny+1)][(nx+1)] corner volume flux |dx dy| */
  LR_F_MX = 27,      /* [ny][nx+1] X-face mass flux, signed */
  LR_F_MY = 28,      /* [ny+1][nx] Y-face mass flux, signed */
  LR_F_MC = 29,      /* [(ny+1)][(nx+1)] corner mass flux magnitude */
  LR_F_Q = 30,       /* [ny][nx] pseudo-viscosity Q^n of the last step */
  LR_F_DT = 31,      /* [1] dt of the last step */
  LR_F_CUTS = 32,    /* [6][ny][nx] interface lines of the last step's mixed cells
                        (n0x, n0y, d0, n1x, n1y, d1 in the cell's frame; 0 elsewhere) */
  LR_F_XA = 33,      /* [nmat][ny][nx+1] per-material X-face volume flux, signed */
  LR_F_YA = 34,      /* [nmat][ny+1][nx] per-material Y-face volume flux, signed */
  LR_F_CA = 35,      /* [nmat][(ny+1)][(nx+1)] per-material corner volume flux */
  LR_F_NMIXED = 36   /* [1] number of mixed cells (two or more materials) in the last step */
};

/* Number of doubles of a field, or 0 for an unknown field. */
size_t lr_field_size(const lr_ctx* ctx, int field);

/* Copy a field to host memory host_out[n_elems] (synchronises; n_elems must
 * be at least lr_field_size). */
lr_status lr_get_fields(lr_ctx* ctx, int field, double* host_out, size_t n_elems);

/* Same without synchronising: the copy is enqueued on the context's stream
 * and host_out must stay valid and unread until lr_sync returns.  Page-locked
 * (pinned) host memory is written by the device directly; pageable memory is
 * copied before the call returns.  LR_F_CONS is not available here.  Several
 * fields read this way cost one synchronisation. */
lr_status lr_get_fields_async(lr_ctx* ctx, int field, double* host_out, size_t n_elems);

/* Same, into caller-owned device memory on the context's stream (no host
 * synchronisation).  LR_F_CONS is not available here. */
lr_status lr_get_fields_device(lr_ctx* ctx, int field, double* dev_out, size_t n_elems);

/* Current simulation time and the CFL time step of the next step (synchronises). */
lr_status lr_time(lr_ctx* ctx, double* t, double* dt_next);

/* Kernel launches one lr_step issues (constant per configuration; lr_run
 * issues one fewer per step plus one per call). */
int lr_launches_per_step(const lr_ctx* ctx);

/* Per-kernel timing with CUDA events recorded on the context's stream around
 * every kernel launch of lr_step / lr_run (off by default; lr_run then runs
 * without graphs).  lr_kernel_times fills, for up to n kernels, the name,
 * number of launches and summed milliseconds since the last reset, and
 * returns the number of kernels. */
lr_status lr_set_profiling(lr_ctx* ctx, int on);
int lr_kernel_times(lr_ctx* ctx, const char** names, long* launches, double* ms, int n);

/* Tiled step (on = 1): kernel pairs of the step that otherwise exchange
 * their intermediate results through device memory run as one kernel over
 * tiles of the grid, each block staging its tile and a halo of inputs in
 * shared memory (the stencils of sections 2.1.1, 2.3 and 3.3 reach two cells
 * or nodes), with the boundary conditions applied once at staging.  The
 * arithmetic is the same; the rounding differs only in the order of a few
 * operations the compiler contracts.  Available for the DirectCF remap with
 * upwind or diagonal corner values (LR_ERR_ARG otherwise); on by default in
 * LR_FP32, off in LR_FP64 and LR_DF64.  Intermediate per-material flux
 * fields (LR_F_XA, LR_F_YA, LR_F_CA) of a tiled step hold only the objects
 * with a mixed donor.  Launches per step: 4 with one material, 6 with two;
 * with three the interface kernels run on the context's second stream
 * beside the cell tiles no mixed cell reaches, and the other tiles follow
 * them (7 launches).  lr_get_tiled returns the current setting. */
lr_status lr_set_tiled(lr_ctx* ctx, int on);
int lr_get_tiled(const lr_ctx* ctx);

void lr_destroy(lr_ctx* ctx);
const char* lr_last_error(const lr_ctx* ctx);

/* Allocation-free CFL time step.  The paper has no counterpart: this is a
 * service for callers that may not allocate device memory when they need a
 * time step (all device memory already reserved by another framework's
 * caching allocator, or a latency-critical loop that must not reach
 * cudaMalloc).  It computes the same rule as lr_step,
 * dt = cfl * min(dx,dy) / max_p (max over the node's cells of c_c + |u_p|),
 * from a state held in caller-owned device memory:
 *   k, rho, e  device [nmat][ny][nx] (volume fractions, densities, specific
 *              internal energies, as lr_get_fields_device returns them);
 *   ux, uy     device [(ny+1)][(nx+1)];
 *   dt_out     device pointer to one double that receives dt;
 * cfg supplies nx, ny, domain, nmat, cfl, bc and the stream
 * (cfg->cuda_stream, NULL = the legacy default stream); mats[nmat] the EOS.
 * The work is enqueued on that stream; nothing is synchronised.
 * Scratch is a fixed array inside the library (8 MiB on every GPU that loads
 * it, kept until the process exits): nx*ny above 2^20 is rejected with
 * LR_ERR_ARG.  No cudaMalloc/cudaFree or other allocating call is made.  The
 * first call on a device looks up the scratch address on that device (make
 * that first call before any stream capture).  All calls share the scratch,
 * so calls that overlap on the GPU (other streams, other host threads) race:
 * serialise them.  The scratch address is kept per device for the life of
 * the process: no call may follow a cudaDeviceReset of that device.
 * Validation follows lr_create's: LR_ERR_ARG for nx or ny < 2, nmat outside
 * 1..3, an empty domain, cfl outside (0, 1], a bc other than LR_BC_REFLECT
 * or LR_BC_PERIODIC, xlo != xhi or ylo != yhi, a periodic direction with
 * fewer than 3 cells, or a NULL pointer.  A state that is not finite (NaN
 * or infinite k, rho, e or u) or where a material of full weight has no
 * real sound speed (c^2 <= 0) gives *dt_out = NaN, so a caller can tell a
 * bad state from a quiet one (lr_step reports the same states through its
 * error flags). */
lr_status lr_cfl_dt_noalloc(const lr_config* cfg, const lr_material* mats, const double* k,
                            const double* rho, const double* e, const double* ux, const double* uy,
                            double* dt_out);

/* Arithmetic check: out[i] = a[i] op b[i], i < n, computed on the device by
 * the routine the FP64 step kernels use for that operation, so that a test
 * can compare it with IEEE 754 arithmetic.
 *   op LR_ARITH_DIV: the quotient a/b: the significand quotient to about
 *      2^-44 as a float pair (a float reciprocal seed, one Newton-Raphson
 *      step in double-float arithmetic, Dekker's exact product), then one
 *      Markstein correction with a fused multiply-add residual in double
 *      (P. W. Markstein, IBM J. Res. Dev. 34(1), 1990); correctly rounded
 *      except within about 2^-66 (relative) of a rounding midpoint, where it
 *      is one ulp off; a = +-0 gives the signed zero; b zero, subnormal,
 *      infinite, NaN or |b| >= 2^1020, a subnormal, infinite or NaN, and
 *      quotients outside the normal range take IEEE division.  The FP64 step
 *      uses it for every division and reciprocal.
 *   op LR_ARITH_SQRT: sqrt(a) (b unused, may equal a) the same way from a
 *      float reciprocal-square-root seed, correctly rounded except near
 *      midpoints as above; a zero, subnormal, negative, infinite, NaN or
 *      >= 2^1023 takes the IEEE square root.
 * a, b, out: device pointers to n doubles (out may alias a or b).
 * cuda_stream: cudaStream_t, NULL = the legacy default stream; the work is
 * enqueued, nothing is synchronised.  LR_ERR_ARG: unknown op, or n > 0 with
 * a NULL pointer; LR_ERR_CUDA: the launch failed. */
enum { LR_ARITH_DIV = 0, LR_ARITH_SQRT = 1 };

/* FP64 throughput probe (a measurement hook; the paper has no counterpart):
 * blocks x threads threads each run `iters` iterations of eight independent
 * fused multiply-add chains in double, 16 * iters flops per thread, and
 * store one double each to dev_out[blocks * threads] (device).  Timed by
 * the caller (CUDA events on cuda_stream, NULL = the legacy default
 * stream), it measures the FP64 rate the native-double step is bound by.
 * LR_ERR_ARG: NULL dev_out, blocks < 1, threads not a multiple of 32 in
 * [32, 1024], iters < 1; LR_ERR_CUDA: the launch failed. */
lr_status lr_fp64_fma_probe(double* dev_out, int blocks, int threads, int iters, void* cuda_stream);
lr_status lr_arith_check(int op, const double* a, const double* b, double* out, size_t n, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
