// lr_dev.cuh -- device-side data of the Lagrange-Remap step shared by the
// kernel and API translation units (no host types of torch or the oracle).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define LR_MAXM 3

// Error bits of the device error word.
enum {
  LR_DERR_VOLUME = 1,      // non-positive cell volume (tangled Lagrangian cell)
  LR_DERR_SOUND = 2,       // c^2 <= 0 for a material that counts in the CFL rule
  LR_DERR_MASS = 4,        // non-positive material or nodal mass after the remap
  LR_DERR_NAN = 8,         // NaN / Inf in an updated field
  LR_DERR_GEOM = 16        // face flux trapezoid with negative height
};

// Arithmetic of the step kernels (lr_config.precision).
enum { LR_MODE_FP64 = 0, LR_MODE_DF64 = 1, LR_MODE_FP32 = 2 };

// Constants of one simulation (host doubles; the kernels get them converted
// to their arithmetic type).
struct LrGrid {
  int nx, ny, M;
  int perx, pery;          // periodic flags (else reflective walls)
  int nxu, nyu;            // canonical node counts: nx (periodic) or nx+1
  int mode;                // LR_MODE_*
  double dx, dy, V, L, hmin, D;  // D = sqrt(dx^2+dy^2)
  double inv2dx, inv2dy, inv8dx, inv8dy, invV, invD;  // reciprocals of the constant divisors
  double cfl, a1, a2, dt_fixed;
  double gam[LR_MAXM], pin[LR_MAXM];
  int face_o2, corner_o2, presc;  // corner_o2: second-order dual corners
  int corner_kind;         // LR_CORNER_* of the primary mesh's corner values
  int mixed_lanes;         // lanes per mixed cell in lr_mixed: 1, 2, 4 or 8
  // Remap of the step (LR_REMAP_*) and, for the alternate-directions remap,
  // the sweep a launch belongs to: sweep 0 remaps with the full displacement,
  // 1 with its x part only (X faces), 2 with its y part only.  corners: the
  // remap has corner fluxes; lagrange: lr_cell_lag also computes Vol^{lag}
  // and e^{lag} (not in a second sweep); finalize: lr_node_update ends the
  // step (CFL rule, time advance).
  int remap, sweep, corners, lagrange, finalize;
  // Place of this simulation in arrays shared by a batch (all 0 for a lone
  // simulation): first cell, node and dual-cell index (face arrays use the
  // node offset, their per-instance slots being node-sized), its scalar
  // slot (scal[LR_NSCAL inst ..], red[LR_RED_INST + 2 inst ..], err[2 inst ..],
  // dtR[inst]), its mixed-cell counter red[mslot] with list start moff, and
  // the start of its initial-state staging.
  int coff, noff, doff, inst, mslot, moff;
  long long stoff;
};

// Scalars per simulation: [0] t, [1] dt from the CFL rule, [2] dt of the last
// step, [3] t_end, [4] steps taken, [5] dt of the step in flight (0: idle),
// [6] mixed cells in the last step, [7] step limit (0: none).
#define LR_NSCAL 8
// red[0..2]: mixed-cell counters (one per material-count group of a batch);
// red[LR_RED_INST + 2 s], red[LR_RED_INST + 2 s + 1]: CFL max key and tile
// counter of simulation slot s.
#define LR_RED_INST 4

// One tile of a batched launch: simulation slot, origin of the tile in that
// simulation's iteration domain, and the number of tiles the table holds for
// that simulation (the CFL reduction's completion count).
struct LrTile { int inst, i0, j0, n; };

// Real-valued device arrays, listed once so the generic (void*) and typed
// views stay in step.  Cell arrays have nx*ny entries ([j][i]); node arrays
// (nx+1)*(ny+1); X-face arrays (nx+1)*ny; Y-face arrays nx*(ny+1); dual
// arrays (nx+2)*(ny+2) indexed (i+1, j+1) for i in [-1, nx], j in [-1, ny].
#define LR_WORK_REALS(X)                                                      \
  X(pux) X(puy)                       /* prescribed velocity (nodes) */        \
  X(mc) X(Q) X(Pi) X(cc)              /* cell mass, Q, P+Q, sound speed */     \
  X(ox) X(oy) X(wx) X(wy) X(vcf)      /* Lagrangian rectangle, Vol^{lagCF} */  \
  X(uhx) X(uhy) X(ddx) X(ddy) X(ulx) X(uly)  /* node u^{n+1/2}, d, u^{lag} */  \
  X(fx) X(fxb) X(fxlo) X(fxhi)        /* X faces: flux and its rectangle */    \
  X(fy) X(fyb) X(fylo) X(fyhi)        /* Y faces */                            \
  X(MX) X(MY) X(Mpp) X(Mpm)           /* total mass fluxes */                  \
  X(dtR)                              /* [inst] dt of the step in flight */
#define LR_WORK_MAT_REALS(X)                                                  \
  X(elc)   /* (P_a^{n+1/2} + Q)/(rho_a dx dy): e^{lag} = e - elc (Vol^{lag} - V) */ \
  X(elag) X(rcf)                      /* e^{lag}, rho^{lagCF} */               \
  X(xAm) X(yAm) X(cAm)                /* material volumes of mixed donors */   \
  X(xA) X(xMm) X(xE) X(yA) X(yMm) X(yE) X(cA) X(cMm) X(cE)  /* final fluxes */

template <class R>
struct LrStateT {
  R* k[LR_MAXM];
  R* r[LR_MAXM];
  R* e[LR_MAXM];
  R* ux;
  R* uy;
};

template <class R>
struct LrWorkT {
  double* scal;            // LR_NSCAL per simulation (see above)
  unsigned long long* red; // mixed-cell counters, then CFL key and tile counter per simulation
  int* err;                // per simulation: [0] error bits, [1] first failing index
  int* mixed;              // work list of mixed cells (cell indices), red[mslot] entries
  int* minst;              // simulation slot of each list entry
  const LrGrid* gdev;      // lone simulation: its grid in device memory (the interface kernel reads it)
  unsigned char* mask;     // bit a set when material a is present in the cell at t^n
  unsigned int* tflag;     // tiled step: 1 for a cell tile with a mixed cell within one cell (else null)
  int* tlist;              // the flagged tiles, tcount[0] of them, each once
  unsigned int* tcount;    // [0] listed tiles, [1] blocks of the flagged-tile kernel that finished
  double* cut[6];          // interface lines of mixed cells (n0x, n0y, d0, n1x, n1y, d1)
  double* cutY[6];         // Direct remap: the lines that cut the Y faces (else null)
  double* stage;           // init staging: k, rho, p [3][nmat][nc] then ux, uy [2][nn]
#define LR_F1(n) R* n;
  LR_WORK_REALS(LR_F1)
#undef LR_F1
#define LR_F1(n) R* n[LR_MAXM];
  LR_WORK_MAT_REALS(LR_F1)
#undef LR_F1
  R* dX[3]; R* dY[3]; R* dPP[3]; R* dPM[3];  // dual objects: mass, x- and y-momentum
};

using LrState = LrStateT<void>;
using LrWork = LrWorkT<void>;

template <class R>
inline LrStateT<R> typed(const LrState& s) {
  LrStateT<R> t;
  for (int a = 0; a < LR_MAXM; ++a) {
    t.k[a] = static_cast<R*>(s.k[a]); t.r[a] = static_cast<R*>(s.r[a]); t.e[a] = static_cast<R*>(s.e[a]);
  }
  t.ux = static_cast<R*>(s.ux);
  t.uy = static_cast<R*>(s.uy);
  return t;
}
template <class R>
inline LrWorkT<R> typed(const LrWork& w) {
  LrWorkT<R> t;
  t.scal = w.scal; t.red = w.red; t.err = w.err; t.mixed = w.mixed; t.minst = w.minst; t.gdev = w.gdev;
  t.mask = w.mask;
  t.tflag = w.tflag; t.tlist = w.tlist; t.tcount = w.tcount;
  t.stage = w.stage;
  for (int q = 0; q < 6; ++q) { t.cut[q] = w.cut[q]; t.cutY[q] = w.cutY[q]; }
#define LR_F1(n) t.n = static_cast<R*>(w.n);
  LR_WORK_REALS(LR_F1)
#undef LR_F1
#define LR_F1(n) for (int a = 0; a < LR_MAXM; ++a) t.n[a] = static_cast<R*>(w.n[a]);
  LR_WORK_MAT_REALS(LR_F1)
#undef LR_F1
  for (int q = 0; q < 3; ++q) {
    t.dX[q] = static_cast<R*>(w.dX[q]); t.dY[q] = static_cast<R*>(w.dY[q]);
    t.dPP[q] = static_cast<R*>(w.dPP[q]); t.dPM[q] = static_cast<R*>(w.dPM[q]);
  }
  return t;
}

// Host-side launchers (lr_kernels.cu).  Each enqueues one kernel on `s`;
// the arithmetic follows g.mode.
enum LrKernelId {
  LRK_CELL_PRE = 0, LRK_NODE_HALF, LRK_CELL_LAG, LRK_CELL_CF, LRK_MIXED, LRK_MAT_FLUX,
  LRK_CELL_UPDATE, LRK_DUAL_FLUX, LRK_NODE_UPDATE, LRK_COUNT,
  LRK_PREPARE = 100,   // initial state from the staging area
  LRK_CFL_ONLY = 101,  // CFL rule from the current state
  LRK_SWEEP_PREP = 102, // alternate directions: the first sweep's result as the second's input
  LRK_MIXED_PLACE = 103, // interface lines of the mixed cells; LRK_MIXED then splits their fluxes
  // tiled step (lone simulations): fused kernel pairs over shared-memory tiles
  LRK_T_NODE_REMAP = 110,  // lr_dual_flux + lr_node_update
  LRK_T_CELL_REMAP = 111,  // lr_mat_flux + lr_cell_update
  LRK_T_LAGRANGE = 112,    // lr_cell_pre + lr_node_half + lr_cell_lag + lr_cell_cf
  LRK_T_CELL_CLEAN = 113,  // lr_t_cell_remap over the tiles no mixed cell reaches (beside the interface kernels)
  LRK_T_CELL_DIRTY = 114,  // lr_t_cell_flagged: the other tiles (after the interface kernels)
  LRK_MIXED_PLACE_PDL = 115,  // lb_mixed_place right after a kernel of the same stream (programmatic launch)
  LRK_MIXED_PDL = 116         // lb_mixed right after lb_mixed_place (programmatic launch)
};
// Interface-line placement spreads a short mixed-cell list over about this
// many warps (two per SM sub-partition of a 152-SM GPU), one lane per cell.
#ifndef LR_PLACE_SPREAD
#define LR_PLACE_SPREAD 1216
#endif
// Dynamic shared-memory limits of the tiled kernels (once per device, before
// their first launch).
cudaError_t lr_tiled_setup();

// Iteration domains of the kernels (tile tables of a batch are per domain).
enum { LR_DOM_CELLS = 0, LR_DOM_NODES, LR_DOM_DUAL, LR_DOM_NODES_ALL, LR_NDOM };
int lr_kernel_domain(int kid);
extern const char* const lr_kernel_names[LRK_COUNT];

cudaError_t lr_launch(int kid, const LrGrid& g, const LrState& cur, const LrState& nxt,
                      const LrWork& w, cudaStream_t s);
cudaError_t lr_launch_init(const LrGrid& g, const LrState& st, const LrWork& w, cudaStream_t s);
cudaError_t lr_launch_set_tend(const LrGrid& g, const LrWork& w, double t_end, cudaStream_t s);
// Zero the scalars, reduction words and error words of nsim simulations.
cudaError_t lr_launch_reset(int mode, const LrWork& w, int nsim, cudaStream_t s);

// One kernel of the step over a batch's tile table (kernels named lb_*).
struct LrBatchArgs {
  int mode;                // LR_MODE_* of every simulation
  int M;                   // material count of every simulation in the table
  const LrGrid* gs;        // device: grids by simulation slot
  const void* kcs;         // device: constants by slot, lr_kc_bytes(mode) each
  const LrTile* tiles;     // device: the tiles of this launch
  int ntiles;
  int bx, by;              // block = tile shape, bx * by == 256
  int grid;                // persistent blocks (lr_mixed: blocks of 128)
  int lanes, mslot, moff;  // lr_mixed: lanes per cell, counter slot, list start
};
cudaError_t lr_launch_batch(int kid, const LrBatchArgs& a, const LrState& cur, const LrState& nxt,
                            const LrWork& w, cudaStream_t s);
// Persistent batch step (lb_t_step): one cooperative launch of `grid`
// blocks per step over the cell tiles (32 x 8, every member) and the node
// tiles, with grid barriers between the phases (bar: count, generation,
// status; status LR_BAR_TIMEOUT after a wait of limit_ns).  groups: bit 2
// set when two-material members are present, bit 3 three-material ones; P
// the pool size (the three-material list starts at P).
struct LrGridBar { unsigned int count, gen; int status, pad; };
enum { LR_BAR_TIMEOUT = 1 };
struct LrPersistArgs {
  const LrGrid* gs;
  const void* kcs;
  const LrTile* ctiles;
  int nct;
  const LrTile* ntiles;
  int nnt;
  LrGridBar* bar;
  unsigned int extra;
  unsigned long long limit_ns;
  int groups, P, grid;
};
cudaError_t lr_launch_batch_persistent(int mode, const LrPersistArgs& p, const LrState& cur, const LrState& nxt,
                                       const LrWork& w, cudaStream_t s);
// Resident blocks of lb_t_step per SM (0 when it cannot run).
int lr_persistent_blocks_per_sm(int mode);
// Tile of the tiled step and of lb_t_step: cells (or nodes) per block.
void lr_tiled_tile_shape(int* tw, int* th);
size_t lr_kc_bytes(int mode);
void lr_make_kc(const LrGrid& g, void* out);
// Field views: convert a real array (element type from g.mode) to double,
// gathering with the boundary mapping: kind 0 plain copy of n values, 1 node
// array, 2 X-face array, 3 Y-face array.
cudaError_t lr_launch_view(const LrGrid& g, const void* src, double* dst, size_t n, int kind, cudaStream_t s);
cudaError_t lr_launch_mixture(const LrGrid& g, const LrState& st, double* dst, int which, cudaStream_t s);
cudaError_t lr_launch_cons(const LrGrid& g, const LrState& st, double* rows, double* dst, cudaStream_t s);
cudaError_t lr_launch_arith(int op, const double* a, const double* b, double* out, size_t n, cudaStream_t s);
cudaError_t lr_launch_dfma(double* out, int blocks, int threads, int iters, cudaStream_t s);
cudaError_t lr_launch_corner_debug(const LrGrid& g, const LrWork& w, double* fc_out, double* mc_out,
                                   cudaStream_t s);
cudaError_t lr_launch_cuts(const LrGrid& g, const LrState& prev, const LrWork& w, double* dst, cudaStream_t s);
cudaError_t lr_launch_from_double(const LrGrid& g, const double* src, void* dst, size_t n, cudaStream_t s);
size_t lr_real_size(int mode);
// Lanes per mixed cell in lr_mixed when the configuration leaves it open.
int lr_default_mixed_lanes(int mode);
