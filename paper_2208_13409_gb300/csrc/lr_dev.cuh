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

// Constants of one simulation (passed by value to every kernel).
struct LrGrid {
  int nx, ny, M;
  int perx, pery;          // periodic flags (else reflective walls)
  int nxu, nyu;            // canonical node counts: nx (periodic) or nx+1
  double dx, dy, V, L, hmin, D;  // D = sqrt(dx^2+dy^2)
  double inv2dx, inv2dy, inv8dx, inv8dy, invV, invD;  // reciprocals of the constant divisors
  double cfl, a1, a2, dt_fixed;
  double gam[LR_MAXM], pin[LR_MAXM];
  int face_o2, corner_o2, presc;
};

// Device arrays.  Cell arrays have nx*ny entries ([j][i]); node arrays
// (nx+1)*(ny+1); X-face arrays (nx+1)*ny; Y-face arrays nx*(ny+1); dual
// arrays (nx+2)*(ny+2) indexed (i+1, j+1) for i in [-1, nx], j in [-1, ny].
struct LrState {
  double* k[LR_MAXM];
  double* r[LR_MAXM];
  double* e[LR_MAXM];
  double* ux;
  double* uy;
};

struct LrWork {
  double* scal;            // [0] t, [1] dt from the CFL rule, [2] dt of the last step, [3] t_end,
                           // [4] steps taken, [5] dt of the step in flight (written by lr_cell_pre)
  unsigned long long* red; // [0] max(c+|u|) bits, [1] block counter, [2] mixed-cell count
  int* mixed;              // work list of mixed cells (cell indices), red[2] entries
  int* err;                // [0] error bits, [1] first failing index
  double* pux; double* puy;                  // prescribed velocity (nodes)
  // cells
  double* mc; double* Q; double* Pi; double* cc;
  double* elc[LR_MAXM];    // (P_a^{n+1/2} + Q) / (rho_a dx dy): e_a^{lag} = e_a - elc (Vol^{lag} - dx dy)
  double* elag[LR_MAXM]; double* rcf[LR_MAXM];
  unsigned char* mask;     // bit a set when material a is present in the cell at t^n
  double* ox; double* oy; double* wx; double* wy; double* vcf;
  double* cut[6];          // interface lines of mixed cells (n0x, n0y, d0, n1x, n1y, d1)
  // nodes
  double* uhx; double* uhy; double* ddx; double* ddy; double* ulx; double* uly;
  // X faces / Y faces: signed volume flux, rectangle (bar, lo, hi)
  double* fx; double* fxb; double* fxlo; double* fxhi;
  double* fy; double* fyb; double* fylo; double* fyhi;
  // per-material volumes of fluxes given by mixed donors
  double* xAm[LR_MAXM]; double* yAm[LR_MAXM]; double* cAm[LR_MAXM];
  // per-material final volume / mass / energy fluxes
  double* xA[LR_MAXM]; double* xMm[LR_MAXM]; double* xE[LR_MAXM];
  double* yA[LR_MAXM]; double* yMm[LR_MAXM]; double* yE[LR_MAXM];
  double* cA[LR_MAXM]; double* cMm[LR_MAXM]; double* cE[LR_MAXM];
  // total mass fluxes
  double* MX; double* MY; double* Mpp; double* Mpm;
  // dual objects: [0] mass, [1] x-momentum, [2] y-momentum
  double* dX[3]; double* dY[3]; double* dPP[3]; double* dPM[3];
};

// Host-side launchers (lr_kernels.cu).  Each enqueues one kernel on `s`.
enum LrKernelId {
  LRK_CELL_PRE = 0, LRK_NODE_HALF, LRK_CELL_LAG, LRK_CELL_CF, LRK_MIXED, LRK_MAT_FLUX,
  LRK_CELL_UPDATE, LRK_DUAL_FLUX, LRK_NODE_UPDATE, LRK_COUNT
};
extern const char* const lr_kernel_names[LRK_COUNT];

cudaError_t lr_launch(int kid, const LrGrid& g, const LrState& cur, const LrState& nxt,
                      const LrWork& w, cudaStream_t s);
cudaError_t lr_launch_init_cfl(const LrGrid& g, const LrState& cur, const LrWork& w, cudaStream_t s);
cudaError_t lr_launch_set_scalar(double* p, double v, cudaStream_t s);
cudaError_t lr_launch_reset(const LrWork& w, cudaStream_t s);
cudaError_t lr_launch_prepare_init(const LrGrid& g, const LrState& st, const LrWork& w, cudaStream_t s);
cudaError_t lr_launch_corner_debug(const LrGrid& g, const LrWork& w, double* fc_out, double* mc_out,
                                   cudaStream_t s);
