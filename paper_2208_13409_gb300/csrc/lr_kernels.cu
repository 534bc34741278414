// lr_kernels.cu -- sm_103a kernels of one Lagrange-Remap time step
// (Chaudet, arXiv 2208.13409): SGPC Lagrange phase (section 1.2, multi-material
// form of section 4.1), DirectCF face/corner fluxes (section 2.3), VOF/PLIC
// material split on the rectangular Lagrangian cell (section 4.4), limited
// reconstructions (sections 2.1.1 and 3.3), cell remap, dual-mesh momentum
// remap and the CFL minimum.
//
// Design: the step is FP64-pipe bound on GB300 (about 0.6e12 DFMA/s against
// ~7 TB/s of HBM), so every flux object -- X face, Y face, corner, dual face,
// dual corner -- is evaluated by exactly one thread and its result kept in HBM
// for the cells and nodes that share it; nothing is recomputed in halos.
// Boundary conditions are applied on read: an index outside the domain maps
// to its mirror image (reflective wall, with the sign of the mirrored vector
// component or flux flipped) or wraps (periodic).  Pure cells never enter
// the interface geometry; mixed cells do their PLIC work in the donor-owned
// kernel lr_cell_cf, which also writes the final material split of every
// flux they donate.
#include "lr_dev.cuh"
#include <math.h>

const char* const lr_kernel_names[LRK_COUNT] = {
  "lr_cell_pre", "lr_node_half", "lr_cell_lag", "lr_cell_cf", "lr_mixed", "lr_mat_flux",
  "lr_cell_update", "lr_dual_flux", "lr_node_update"};

namespace {

constexpr double EPS_K = 1e-12;  // material dropped when its volume <= EPS_K dx dy
constexpr double EPS_C = 1e-3;   // sound-speed weight min(1, k / EPS_C)
constexpr int BX = 32, BY = 8;

// ------------------------------------------------------------ index maps
__device__ __forceinline__ int map_cell(int i, int n, int per, int& flip) {
  flip = 0;
  if (i >= 0 && i < n) return i;
  if (per) return (i + n) % n;
  flip = 1;
  return i < 0 ? -1 - i : 2 * n - 1 - i;
}
__device__ __forceinline__ int map_node(int i, int n, int per, int& flip) {
  flip = 0;
  if (per) return (i + n) % n;
  if (i >= 0 && i <= n) return i;
  flip = 1;
  return i < 0 ? -i : 2 * n - i;
}
struct Ix { int idx, fx, fy; };
__device__ __forceinline__ Ix cix(const LrGrid& g, int i, int j) {
  Ix r;
  int mi = map_cell(i, g.nx, g.perx, r.fx), mj = map_cell(j, g.ny, g.pery, r.fy);
  r.idx = mj * g.nx + mi;
  return r;
}
__device__ __forceinline__ Ix nix(const LrGrid& g, int i, int j) {
  Ix r;
  int mi = map_node(i, g.nx, g.perx, r.fx), mj = map_node(j, g.ny, g.pery, r.fy);
  r.idx = mj * (g.nx + 1) + mi;
  return r;
}
// X face (i node-like, j cell-like) and Y face (i cell-like, j node-like)
__device__ __forceinline__ Ix xix(const LrGrid& g, int i, int j) {
  Ix r;
  int mi = map_node(i, g.nx, g.perx, r.fx), mj = map_cell(j, g.ny, g.pery, r.fy);
  r.idx = mj * (g.nx + 1) + mi;
  return r;
}
__device__ __forceinline__ Ix yix(const LrGrid& g, int i, int j) {
  Ix r;
  int mi = map_cell(i, g.nx, g.perx, r.fx), mj = map_node(j, g.ny, g.pery, r.fy);
  r.idx = mj * g.nx + mi;
  return r;
}
// dual objects: i, j in [-1, n]; periodic directions wrap into [0, n)
__device__ __forceinline__ int dix(const LrGrid& g, int i, int j) {
  if (g.perx) i = (i + g.nx) % g.nx;
  if (g.pery) j = (j + g.ny) % g.ny;
  return (j + 1) * (g.nx + 2) + (i + 1);
}
// mirrored node-vector reads
__device__ __forceinline__ double nodeX(const LrGrid& g, const double* a, int i, int j) {
  Ix q = nix(g, i, j);
  double v = a[q.idx];
  return q.fx ? -v : v;
}
__device__ __forceinline__ double nodeY(const LrGrid& g, const double* a, int i, int j) {
  Ix q = nix(g, i, j);
  double v = a[q.idx];
  return q.fy ? -v : v;
}
__device__ __forceinline__ double cellS(const LrGrid& g, const double* a, int i, int j) {
  return a[cix(g, i, j).idx];
}
__device__ __forceinline__ double cellOX(const LrGrid& g, const double* a, int i, int j) {
  Ix q = cix(g, i, j);
  return q.fx ? -a[q.idx] : a[q.idx];
}
__device__ __forceinline__ double cellOY(const LrGrid& g, const double* a, int i, int j) {
  Ix q = cix(g, i, j);
  return q.fy ? -a[q.idx] : a[q.idx];
}

__device__ __forceinline__ void set_err(const LrWork& w, int bit, int idx) {
  atomicOr(&w.err[0], bit);
  atomicCAS(&w.err[1], -1, idx);
}

// dt of the current step: CFL rule (or fixed), capped at t_end.  Evaluated
// by lr_cell_pre, which publishes it in scal[5] for the step's later kernels.
__device__ __forceinline__ double step_dt_eval(const LrGrid& g, const double* scal) {
  double t = scal[0], te = scal[3];
  double dt = g.dt_fixed > 0.0 ? g.dt_fixed : scal[1];
  if (te - t < dt) dt = te - t;
  return dt;
}
__device__ __forceinline__ double step_dt(const LrGrid&, const double* scal) { return scal[5]; }

// ---------------------------------------------------------------- EOS
// Stiffened gas of section 5.2: p = (gamma-1) rho e - pi; c^2 = (gamma p + pi)/rho.
__host__ __device__ __forceinline__ double eos_p(double ga, double pi, double rho, double e) {
  return (ga - 1.0) * rho * e - pi;
}
__host__ __device__ __forceinline__ double eos_c2(double ga, double pi, double rho, double p) {
  return (ga * p + pi) / rho;
}

// Cell volume F of section 1.2 (two triangles split along lr-ul), in
// coordinates local to the cell.
__host__ __device__ __forceinline__ double cell_F(double llx, double lly, double lrx, double lry,
                                         double ulx, double uly, double urx, double ury) {
  double lx = ulx - llx, ly = uly - lly, bx = lrx - llx, by = lry - lly;
  double rx = urx - lrx, ry = ury - lry, tx = urx - ulx, ty = ury - uly;
  return 0.5 * fabs(lx * by - ly * bx) + 0.5 * fabs(rx * ty - ry * tx);
}

// Van Leer limited slope (section 2.1.1) from the two one-sided differences
// dm = a_d - a_{d-1}, dp = a_{d+1} - a_d over the Lagrangian centre spacings
// hm, hp: the harmonic mean of dm/hm and dp/hp, written with one division.
__host__ __device__ __forceinline__ double vl_slope(double dm, double dp, double hm, double hp) {
  double pr = dm * dp;
  return pr > 0.0 ? 2.0 * pr / (dp * hm + dm * hp) : 0.0;
}

// --------------------------------------------------- half-plane geometry
// Area of the axis-aligned rectangle [x0,x1]x[y0,y1] on the side x.n <= d:
// with a <= b the extents of x.n along the two edge directions and s the
// distance of the line from the lowest corner, the area is s^2/(2|nx ny|)
// (triangle), W H (2s-a)/(2b) (trapezoid) or W H - (a+b-s)^2/(2|nx ny|).
__host__ __device__ double rect_half_area(double x0, double x1, double y0, double y1,
                                 double nx, double ny, double d) {
  double W = x1 - x0, H = y1 - y0;
  double ax = fabs(nx) * W, by = fabs(ny) * H;
  double a = fmin(ax, by), b = fmax(ax, by);
  double s = d - ((nx >= 0.0 ? x0 : x1) * nx + (ny >= 0.0 ? y0 : y1) * ny);
  double A = W * H;
  if (s <= 0.0) return 0.0;
  if (s >= a + b) return A;
  if (a <= 0.0) return A * (s / b);
  double pq = fabs(nx) * fabs(ny);
  if (s < a) return 0.5 * s * s / pq;
  if (s <= b) return A * (2.0 * s - a) / (2.0 * b);
  double r = a + b - s;
  return A - 0.5 * r * r / pq;
}
// Inverse of the above: the line constant d giving area fraction k (0<k<1).
__host__ __device__ double rect_plic(double x0, double x1, double y0, double y1, double nx, double ny,
                            double k) {
  double W = x1 - x0, H = y1 - y0;
  double ax = fabs(nx) * W, by = fabs(ny) * H;
  double a = fmin(ax, by), b = fmax(ax, by);
  double s0 = (nx >= 0.0 ? x0 : x1) * nx + (ny >= 0.0 ? y0 : y1) * ny;
  double s;
  if (a <= 0.0) s = k * b;
  else if (k <= 0.5 * a / b) s = sqrt(2.0 * a * b * k);
  else if (k <= 1.0 - 0.5 * a / b) s = k * b + 0.5 * a;
  else s = a + b - sqrt(2.0 * a * b * (1.0 - k));
  return s0 + s;
}

// Small convex polygons (three-material cells only).
struct Poly { int n; double x[8], y[8]; };
__host__ __device__ void poly_rect(Poly& p, double x0, double x1, double y0, double y1) {
  p.n = 4;
  p.x[0] = x0; p.y[0] = y0; p.x[1] = x1; p.y[1] = y0;
  p.x[2] = x1; p.y[2] = y1; p.x[3] = x0; p.y[3] = y1;
}
// keep the part with sgn * (x.n - d) <= 0
__host__ __device__ void poly_clip(const Poly& in, double nx, double ny, double d, double sgn, Poly& out) {
  out.n = 0;
  for (int a = 0; a < in.n; ++a) {
    int b = a + 1 == in.n ? 0 : a + 1;
    double fa = sgn * (in.x[a] * nx + in.y[a] * ny - d);
    double fb = sgn * (in.x[b] * nx + in.y[b] * ny - d);
    if (fa <= 0.0 && out.n < 8) { out.x[out.n] = in.x[a]; out.y[out.n] = in.y[a]; ++out.n; }
    if (((fa < 0.0 && fb > 0.0) || (fa > 0.0 && fb < 0.0)) && out.n < 8) {
      double t = fa / (fa - fb);
      out.x[out.n] = in.x[a] + t * (in.x[b] - in.x[a]);
      out.y[out.n] = in.y[a] + t * (in.y[b] - in.y[a]);
      ++out.n;
    }
  }
}
__host__ __device__ double poly_area(const Poly& p) {
  if (p.n < 3) return 0.0;
  double s = 0.0;
  for (int a = 0; a < p.n; ++a) {
    int b = a + 1 == p.n ? 0 : a + 1;
    s += p.x[a] * p.y[b] - p.x[b] * p.y[a];
  }
  return 0.5 * fabs(s);
}
__host__ __device__ double poly_half_area(const Poly& p, double nx, double ny, double d) {
  Poly q;
  poly_clip(p, nx, ny, d, 1.0, q);
  return poly_area(q);
}
// Line constant d with area(P & {x.n <= d}) = target, exactly: the area is
// a quadratic in d between consecutive vertex levels, so bracket the target
// by the vertex levels just below and just above it and solve the quadratic
// through the area at the two ends and the middle of that bracket.  (No
// local scratch array: every level is evaluated in place, n <= 8.)
__host__ __device__ __noinline__ double poly_plic(const Poly& p, double nx, double ny, double target) {
  int n = p.n;
  double lo = 1e300, hi = -1e300;
  for (int a = 0; a < n; ++a) {
    double v = p.x[a] * nx + p.y[a] * ny;
    lo = fmin(lo, v);
    hi = fmax(hi, v);
  }
  double alo = 0.0, ahi = poly_area(p);
  double blo = lo, bhi = hi;
  for (int a = 0; a < n; ++a) {
    double v = p.x[a] * nx + p.y[a] * ny;
    if (!(v > blo) || !(v < bhi)) continue;
    double av = poly_half_area(p, nx, ny, v);
    if (av < target) { blo = v; alo = av; }
    else { bhi = v; ahi = av; }
  }
  double h = bhi - blo;
  if (!(h > 0.0)) return blo;
  double amid = poly_half_area(p, nx, ny, blo + 0.5 * h);
  // A(blo + t h) = alo + c1 t + c2 t^2, t in [0,1]
  double c2 = 2.0 * (ahi + alo) - 4.0 * amid;
  double c1 = (ahi - alo) - c2;
  double T = target - alo;
  double t;
  if (fabs(c2) <= 1e-14 * fabs(c1)) {
    t = c1 != 0.0 ? T / c1 : 0.0;
  } else {
    double disc = c1 * c1 + 4.0 * c2 * T;
    disc = disc > 0.0 ? disc : 0.0;
    double sq = sqrt(disc);
    t = c1 >= 0.0 ? 2.0 * T / (c1 + sq) : (-c1 + sq) / (2.0 * c2);
  }
  t = fmin(fmax(t, 0.0), 1.0);
  return blo + t * h;
}

// Youngs normal n = -grad k / |grad k| (outward from the material), 9-point
// weights (1,2,1)/(8 dx), (1,2,1)/(8 dy) (section 4.1); n = (1,0) if grad k = 0.
__device__ void youngs(const LrGrid& g, const double* K, int i, int j, double& nxv, double& nyv) {
  double kpp = cellS(g, K, i + 1, j + 1), kp0 = cellS(g, K, i + 1, j), kpm = cellS(g, K, i + 1, j - 1);
  double kmp = cellS(g, K, i - 1, j + 1), km0 = cellS(g, K, i - 1, j), kmm = cellS(g, K, i - 1, j - 1);
  double k0p = cellS(g, K, i, j + 1), k0m = cellS(g, K, i, j - 1);
  double gx = ((kpp + 2.0 * kp0 + kpm) - (kmp + 2.0 * km0 + kmm)) * g.inv8dx;
  double gy = ((kpp + 2.0 * k0p + kmp) - (kpm + 2.0 * k0m + kmm)) * g.inv8dy;
  double gn = sqrt(gx * gx + gy * gy);
  if (gn > 0.0) { nxv = -gx / gn; nyv = -gy / gn; } else { nxv = 1.0; nyv = 0.0; }
}

// Corner donor table (section 3.3): returns 0 when the corner carries no flux.
__device__ __forceinline__ int corner_cells(double ddx, double ddy, int i, int j, int& di, int& dj,
                                            int& ri, int& rj) {
  if (ddx > 0.0 && ddy > 0.0) { di = i - 1; dj = j - 1; ri = i; rj = j; return 1; }
  if (ddx < 0.0 && ddy < 0.0) { di = i; dj = j; ri = i - 1; rj = j - 1; return 1; }
  if (ddx > 0.0 && ddy < 0.0) { di = i - 1; dj = j; ri = i; rj = j - 1; return 1; }
  if (ddx < 0.0 && ddy > 0.0) { di = i; dj = j - 1; ri = i - 1; rj = j; return 1; }
  return 0;
}

// ============================================================== kernels
// K1: pseudo-viscosity Q^n and the predictor thermodynamics (section 1.2,
// section 4.1): Vol^{n+1/2} = F(x^n + dt/2 u^n); rho_a^{n+1/2} =
// rho_a V / Vol^{n+1/2}; e_a^{n+1/2} = e_a - (P_a + Q)(1/rho_a^{n+1/2} -
// 1/rho_a); P^{n+1/2} = sum_a k_a EOS_a.  Q = rho (a1 L c |div u| + a2 L^2
// div u^2) for div u < 0 (quadratic term read with rho so Q is a pressure).
template <int M>
__global__ void __launch_bounds__(256) lr_cell_pre(LrGrid g, LrState cur, LrWork w) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  double dt = step_dt_eval(g, w.scal);
  if (i == 0 && j == 0) w.scal[5] = dt > 0.0 ? dt : 0.0;
  if (i >= g.nx || j >= g.ny) return;
  if (!(dt > 0.0)) return;
  int c = j * g.nx + i;
  int nn = g.nx + 1;
  int i1 = (g.perx && i + 1 == g.nx) ? 0 : i + 1;
  int j1 = (g.pery && j + 1 == g.ny) ? 0 : j + 1;
  int ll = j * nn + i, lr = j * nn + i1, ul = j1 * nn + i, ur = j1 * nn + i1;
  double uxll = cur.ux[ll], uxlr = cur.ux[lr], uxul = cur.ux[ul], uxur = cur.ux[ur];
  double uyll = cur.uy[ll], uylr = cur.uy[lr], uyul = cur.uy[ul], uyur = cur.uy[ur];
  double kk[M], rr[M], ee[M], pa[M], ir[M];
  double m = 0.0, cmax = 0.0;
  unsigned msk = 0u;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    kk[a] = cur.k[a][c];
    rr[a] = 0.0; ee[a] = 0.0; pa[a] = 0.0; ir[a] = 0.0;
    if (kk[a] > 0.0) {
      msk |= 1u << a;
      rr[a] = cur.r[a][c];
      ee[a] = cur.e[a][c];
      ir[a] = 1.0 / rr[a];
      pa[a] = eos_p(g.gam[a], g.pin[a], rr[a], ee[a]);
      double c2 = (g.gam[a] * pa[a] + g.pin[a]) * ir[a];
      double wgt = kk[a] * (1.0 / EPS_C) < 1.0 ? kk[a] * (1.0 / EPS_C) : 1.0;
      if (wgt >= 1.0 && !(c2 > 0.0)) set_err(w, LR_DERR_SOUND, c);
      double ca = sqrt(c2 > 0.0 ? c2 : 0.0);
      if (wgt * ca > cmax) cmax = wgt * ca;
      m += rr[a] * kk[a] * g.V;
    }
  }
  double div = ((uxlr + uxur) - (uxll + uxul)) * g.inv2dx + ((uyul + uyur) - (uyll + uylr)) * g.inv2dy;
  double rc = m * g.invV;
  double Q = div < 0.0 ? rc * (g.a1 * g.L * cmax * fabs(div) + g.a2 * g.L * g.L * div * div) : 0.0;
  double h = 0.5 * dt;
  double vol = cell_F(h * uxll, h * uyll, g.dx + h * uxlr, h * uylr, h * uxul, g.dy + h * uyul,
                      g.dx + h * uxur, g.dy + h * uyur);
  if (!(vol > 0.0)) set_err(w, LR_DERR_VOLUME, c);
  double dv = vol - g.V;
  double vV = g.V / vol;
  double P = 0.0;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    double cl = 0.0;
    if (msk & (1u << a)) {
      double rh = rr[a] * vV;
      double iv = ir[a] * g.invV;
      double eh = ee[a] - (pa[a] + Q) * (dv * iv);
      double ph = eos_p(g.gam[a], g.pin[a], rh, eh);
      P += kk[a] * ph;
      cl = (ph + Q) * iv;
    }
    w.elc[a][c] = cl;
  }
  w.mc[c] = m;
  w.Q[c] = Q;
  w.Pi[c] = P + Q;
  w.mask[c] = (unsigned char)msk;
  if (msk & (msk - 1u)) {  // two or more materials: interface work list
    unsigned long long slot = atomicAdd(&w.red[2], 1ull);
    w.mixed[slot] = c;
  }
}

// K2: node velocity at t^{n+1/2} (section 1.2): u^{n+1/2} = u^n - dt/2
// grad(P+Q)_p / rho_p with the four-cell gradient over 2dx, 2dy and
// rho_p = (1/4 sum m_c)/(dx dy); u^{lag} = 2 u^{n+1/2} - u^n; node
// displacement d = dt u^{n+1/2}.  Wall-normal components vanish.
__global__ void __launch_bounds__(256) lr_node_half(LrGrid g, LrState cur, LrWork w) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  if (i >= g.nxu || j >= g.nyu) return;
  double dt = step_dt(g, w.scal);
  if (!(dt > 0.0)) return;
  int n = j * (g.nx + 1) + i;
  double hx, hy, lx, ly;
  if (g.presc) {
    hx = w.pux[n]; hy = w.puy[n]; lx = hx; ly = hy;
  } else {
    int A = cix(g, i - 1, j - 1).idx, B = cix(g, i, j - 1).idx;
    int C = cix(g, i - 1, j).idx, D = cix(g, i, j).idx;
    double gx = ((w.Pi[B] + w.Pi[D]) - (w.Pi[A] + w.Pi[C])) * g.inv2dx;
    double gy = ((w.Pi[C] + w.Pi[D]) - (w.Pi[A] + w.Pi[B])) * g.inv2dy;
    double mp = 0.25 * (w.mc[A] + w.mc[B] + w.mc[C] + w.mc[D]);
    double f = 0.5 * dt * g.V / mp;  // dt/2 / rho_p
    double u0x = cur.ux[n], u0y = cur.uy[n];
    hx = u0x - f * gx;
    hy = u0y - f * gy;
    if (!g.perx && (i == 0 || i == g.nx)) hx = 0.0;
    if (!g.pery && (j == 0 || j == g.ny)) hy = 0.0;
    lx = 2.0 * hx - u0x;
    ly = 2.0 * hy - u0y;
  }
  if (!g.perx && (i == 0 || i == g.nx)) { hx = 0.0; lx = 0.0; }
  if (!g.pery && (j == 0 || j == g.ny)) { hy = 0.0; ly = 0.0; }
  w.uhx[n] = hx; w.uhy[n] = hy;
  w.ulx[n] = lx; w.uly[n] = ly;
  w.ddx[n] = dt * hx; w.ddy[n] = dt * hy;
}

// K3: corrector (section 1.2): Vol^{lag} = F(x^n + dt u^{n+1/2}),
// e_a^{lag} = e_a - (P_a^{n+1/2} + Q)(1/rho_a^{lag} - 1/rho_a); the
// rectangular Lagrangian cell through the four Lagrangian face midpoints
// (section 4.4): centre offset (ox, oy) and widths (wx, wy); and the face
// volume fluxes of section 2.3: for X face (i,j) with end nodes p- = (i,j),
// p+ = (i,j+1): y- = max(0, dy_{p-}), y+ = Dy + min(0, dy_{p+}), the
// straight Lagrangian face line x(y) through (dx_{p-}, dy_{p-}) and
// (dx_{p+}, Dy + dy_{p+}), dVol = 1/2 (x(y-) + x(y+)) (y+ - y-); the flux
// region is the rectangle [0, xbar] x [y-, y+].  Y faces swap the axes.
template <int M>
__global__ void __launch_bounds__(256) lr_cell_lag(LrGrid g, LrState cur, LrWork w) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  if (i >= g.nxu || j >= g.nyu) return;
  double dt = step_dt(g, w.scal);
  if (!(dt > 0.0)) return;
  int nn = g.nx + 1;
  int i1 = (g.perx && i + 1 == g.nx) ? 0 : i + 1;
  int j1 = (g.pery && j + 1 == g.ny) ? 0 : j + 1;
  if (i < g.nx && j < g.ny) {
    int c = j * g.nx + i;
    int ll = j * nn + i, lr = j * nn + i1, ul = j1 * nn + i, ur = j1 * nn + i1;
    double dxll = w.ddx[ll], dxlr = w.ddx[lr], dxul = w.ddx[ul], dxur = w.ddx[ur];
    double dyll = w.ddy[ll], dylr = w.ddy[lr], dyul = w.ddy[ul], dyur = w.ddy[ur];
    double vol = cell_F(dxll, dyll, g.dx + dxlr, dylr, dxul, g.dy + dyul, g.dx + dxur, g.dy + dyur);
    if (!(vol > 0.0)) set_err(w, LR_DERR_VOLUME, c);
    double dv = vol - g.V;
    unsigned msk = w.mask[c];
#pragma unroll
    for (int a = 0; a < M; ++a) {
      double el = 0.0;
      if (msk & (1u << a)) el = cur.e[a][c] - w.elc[a][c] * dv;
      w.elag[a][c] = el;
    }
    double xl = 0.5 * (dxll + dxul), xr = g.dx + 0.5 * (dxlr + dxur);
    double yb = 0.5 * (dyll + dylr), yt = g.dy + 0.5 * (dyul + dyur);
    w.ox[c] = 0.5 * (xl + xr) - 0.5 * g.dx;
    w.oy[c] = 0.5 * (yb + yt) - 0.5 * g.dy;
    w.wx[c] = xr - xl;
    w.wy[c] = yt - yb;
  }
  if (j < g.ny) {  // X face (i, j), canonical i
    int pm = j * nn + i, pp = j1 * nn + i;
    double ax = w.ddx[pm], ay = w.ddy[pm], bx = w.ddx[pp], by = g.dy + w.ddy[pp];
    double ylo = ay > 0.0 ? ay : 0.0;
    double dyp = w.ddy[pp];
    double yhi = g.dy + (dyp < 0.0 ? dyp : 0.0);
    if (!(yhi > ylo)) set_err(w, LR_DERR_GEOM, pm);
    double sl = (bx - ax) / (by - ay);
    double xlo = ax + sl * (ylo - ay), xhi = ax + sl * (yhi - ay);
    double xb = 0.5 * (xlo + xhi);
    int f = j * nn + i;
    w.fx[f] = xb * (yhi - ylo);
    w.fxb[f] = xb; w.fxlo[f] = ylo; w.fxhi[f] = yhi;
  }
  if (i < g.nx) {  // Y face (i, j), canonical j
    int pm = j * nn + i, pp = j * nn + i1;
    double ax = w.ddx[pm], ay = w.ddy[pm], bx = g.dx + w.ddx[pp], by = w.ddy[pp];
    double xlo = ax > 0.0 ? ax : 0.0;
    double dxp = w.ddx[pp];
    double xhi = g.dx + (dxp < 0.0 ? dxp : 0.0);
    if (!(xhi > xlo)) set_err(w, LR_DERR_GEOM, pm);
    double sl = (by - ay) / (bx - ax);
    double ylo = ay + sl * (xlo - ax), yhi = ay + sl * (xhi - ax);
    double yb = 0.5 * (ylo + yhi);
    int f = j * g.nx + i;
    w.fy[f] = yb * (xhi - xlo);
    w.fyb[f] = yb; w.fylo[f] = xlo; w.fyhi[f] = xhi;
  }
}

// Flux regions in the donor's frame (origin at its Eulerian lower-left node).
__device__ __forceinline__ void corner_region(const LrGrid& g, double ddx, double ddy, double* r) {
  double px = ddx > 0.0 ? g.dx : 0.0, py = ddy > 0.0 ? g.dy : 0.0;
  if (ddx > 0.0) { r[0] = px; r[1] = px + ddx; } else { r[0] = px + ddx; r[1] = px; }
  if (ddy > 0.0) { r[2] = py; r[3] = py + ddy; } else { r[2] = py + ddy; r[3] = py; }
}

// Material split of one flux region by the donor's interface lines.
template <int M>
__device__ void split_region(int ncut, const int* order, const double (*cut)[3], const double* r,
                             double vol, double* A) {
#pragma unroll
  for (int a = 0; a < M; ++a) A[a] = 0.0;
  int a0 = order[0];
  double p0 = rect_half_area(r[0], r[1], r[2], r[3], cut[0][0], cut[0][1], cut[0][2]);
  A[a0] = p0;
  double used = p0;
  if (ncut == 2) {
    int a1 = order[1];
    Poly q, rest;
    poly_rect(q, r[0], r[1], r[2], r[3]);
    poly_clip(q, cut[0][0], cut[0][1], cut[0][2], -1.0, rest);
    double p1 = poly_half_area(rest, cut[1][0], cut[1][1], cut[1][2]);
    A[a1] = p1;
    used += p1;
  }
  double left = vol - used;
  A[order[ncut]] = left > 0.0 ? left : 0.0;
}

// K4: flux-consistent Lagrangian volume (section 2.3; each flux has one donor
// and one receiver, Vol^{lagCF} = dx dy - received + donated), rho_a^{lagCF}
// = rho_a V / Vol^{lagCF}, and for mixed cells the interface (section 4.1
// Youngs normal, PLIC on the rectangular Lagrangian cell of section 4.4;
// three materials by nested cuts in material order), the split of every flux
// this cell donates, and the clipping of a material's outgoing volume to
// what it holds (excess to the dominant material).
template <int M>
__global__ void __launch_bounds__(256) lr_cell_cf(LrGrid g, LrState cur, LrWork w) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  double dt = step_dt(g, w.scal);
  if (!(dt > 0.0)) return;
  int c = j * g.nx + i;
  int fl = xix(g, i, j).idx, fr = xix(g, i + 1, j).idx;
  int fb = yix(g, i, j).idx, ft = yix(g, i, j + 1).idx;
  double vL = w.fx[fl], vR = w.fx[fr], vB = w.fy[fb], vT = w.fy[ft];
  double v = g.V + vR - vL + vT - vB;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int a = q & 1, b = q >> 1;
    int n = nix(g, i + a, j + b).idx;
    double cx = w.ddx[n], cy = w.ddy[n];
    int di, dj, ri, rj;
    if (!corner_cells(cx, cy, i + a, j + b, di, dj, ri, rj)) continue;
    double f = fabs(cx * cy);
    if (di == i && dj == j) v += f;
    if (ri == i && rj == j) v -= f;
  }
  if (!(v > 0.0)) set_err(w, LR_DERR_VOLUME, c);
  w.vcf[c] = v;
  unsigned msk = w.mask[c];
  double vV = g.V / v;
#pragma unroll
  for (int a = 0; a < M; ++a) w.rcf[a][c] = (msk & (1u << a)) ? cur.r[a][c] * vV : 0.0;
}

// K4b: the interface work of mixed cells only (the list built by lr_cell_pre):
// Youngs normals and PLIC lines in the rectangular Lagrangian cell (sections
// 4.1 and 4.4; three materials by nested cuts in material order), the split
// of every flux the cell donates, and the clipping of a material's outgoing
// volume to what it holds (excess to the dominant material).
template <int M>
__global__ void __launch_bounds__(128) lr_mixed(LrGrid g, LrState cur, LrWork w) {
  double dt = step_dt(g, w.scal);
  if (!(dt > 0.0)) return;
  int count = (int)w.red[2];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
    int c = w.mixed[t];
    int i = c % g.nx, j = c / g.nx;
    double v = w.vcf[c];
    int fl = xix(g, i, j).idx, fr = xix(g, i + 1, j).idx;
    int fb = yix(g, i, j).idx, ft = yix(g, i, j + 1).idx;
    double vL = w.fx[fl], vR = w.fx[fr], vB = w.fy[fb], vT = w.fy[ft];
    int nidx[4];
    double cdx[4], cdy[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int n = nix(g, i + (q & 1), j + (q >> 1)).idx;
      nidx[q] = n;
      cdx[q] = w.ddx[n];
      cdy[q] = w.ddy[n];
    }
    double kk[M];
    int np = 0, order[LR_MAXM] = {0, 0, 0}, dom = 0;
    unsigned msk = w.mask[c];
#pragma unroll
    for (int a = 0; a < M; ++a) {
      kk[a] = (msk & (1u << a)) ? cur.k[a][c] : 0.0;
      if (msk & (1u << a)) order[np++] = a;
      if (kk[a] > kk[dom]) dom = a;
    }
    // ---- mixed cell: interface lines in the rectangular Lagrangian cell
    double wxc = w.wx[c], wyc = w.wy[c];
    double xl = 0.5 * g.dx - 0.5 * wxc + w.ox[c], xr = xl + wxc;
    double yb = 0.5 * g.dy - 0.5 * wyc + w.oy[c], yt = yb + wyc;
    int ncut = np - 1;
    double cut[2][3];
    {
      double nxv, nyv;
      youngs(g, cur.k[order[0]], i, j, nxv, nyv);
      cut[0][0] = nxv; cut[0][1] = nyv;
      cut[0][2] = rect_plic(xl, xr, yb, yt, nxv, nyv, kk[order[0]]);
    }
    if (ncut == 2) {
      double nxv, nyv;
      youngs(g, cur.k[order[1]], i, j, nxv, nyv);
      Poly rect, rest;
      poly_rect(rect, xl, xr, yb, yt);
      poly_clip(rect, cut[0][0], cut[0][1], cut[0][2], -1.0, rest);
      double target = kk[order[1]] * (wxc * wyc);
      double ra = poly_area(rest);
      if (target > ra) target = ra;
      cut[1][0] = nxv; cut[1][1] = nyv;
      cut[1][2] = poly_plic(rest, nxv, nyv, target);
    }
    w.cut[0][c] = cut[0][0]; w.cut[1][c] = cut[0][1]; w.cut[2][c] = cut[0][2];
    if (ncut == 2) { w.cut[3][c] = cut[1][0]; w.cut[4][c] = cut[1][1]; w.cut[5][c] = cut[1][2]; }
    // ---- outgoing fluxes: 0 left, 1 right, 2 bottom, 3 top, 4..7 corners
    double A[8][M];
    int kind[8], fidx[8];
    int nf = 0;
    double r[4];
    double out[M];
  #pragma unroll
    for (int a = 0; a < M; ++a) out[a] = 0.0;
    if (vL < 0.0) {
      r[0] = w.fxb[fl]; r[1] = 0.0; r[2] = w.fxlo[fl]; r[3] = w.fxhi[fl];
      split_region<M>(ncut, order, cut, r, -vL, A[nf]); kind[nf] = 0; fidx[nf] = fl; ++nf;
    }
    if (vR > 0.0) {
      r[0] = g.dx; r[1] = g.dx + w.fxb[fr]; r[2] = w.fxlo[fr]; r[3] = w.fxhi[fr];
      split_region<M>(ncut, order, cut, r, vR, A[nf]); kind[nf] = 0; fidx[nf] = fr; ++nf;
    }
    if (vB < 0.0) {
      r[0] = w.fylo[fb]; r[1] = w.fyhi[fb]; r[2] = w.fyb[fb]; r[3] = 0.0;
      split_region<M>(ncut, order, cut, r, -vB, A[nf]); kind[nf] = 1; fidx[nf] = fb; ++nf;
    }
    if (vT > 0.0) {
      r[0] = w.fylo[ft]; r[1] = w.fyhi[ft]; r[2] = g.dy; r[3] = g.dy + w.fyb[ft];
      split_region<M>(ncut, order, cut, r, vT, A[nf]); kind[nf] = 1; fidx[nf] = ft; ++nf;
    }
    for (int q = 0; q < 4; ++q) {
      int a = q & 1, b = q >> 1;
      int di, dj, ri, rj;
      if (!corner_cells(cdx[q], cdy[q], i + a, j + b, di, dj, ri, rj)) continue;
      if (di != i || dj != j) continue;
      corner_region(g, cdx[q], cdy[q], r);
      split_region<M>(ncut, order, cut, r, fabs(cdx[q] * cdy[q]), A[nf]);
      kind[nf] = 2; fidx[nf] = nidx[q]; ++nf;
    }
    for (int f = 0; f < nf; ++f)
  #pragma unroll
      for (int a = 0; a < M; ++a) out[a] += A[f][a];
    double sc[M];
  #pragma unroll
    for (int a = 0; a < M; ++a) {
      sc[a] = 1.0;
      if (a == dom) continue;
      double avail = kk[a] * v;
      if (out[a] > avail) sc[a] = avail / out[a];
    }
    for (int f = 0; f < nf; ++f) {
      double moved = 0.0;
  #pragma unroll
      for (int a = 0; a < M; ++a) {
        if (sc[a] < 1.0) { moved += (1.0 - sc[a]) * A[f][a]; A[f][a] *= sc[a]; }
      }
      A[f][dom] += moved;
  #pragma unroll
      for (int a = 0; a < M; ++a) {
        double* dst = kind[f] == 0 ? w.xAm[a] : kind[f] == 1 ? w.yAm[a] : w.cAm[a];
        dst[fidx[f]] = A[f][a];
      }
    }
  }
}

// Purity from the material bitmask: the cell holds material a only.
__device__ __forceinline__ bool pure_in(const LrGrid& g, const unsigned char* mask, int i, int j, unsigned bit) {
  return mask[cix(g, i, j).idx] == bit;
}

// Face value (section 2.1.1): a_d + slope/2 (sgn(dVol) wx_d - dt u_f).
__device__ __forceinline__ double recon_face_x(const LrGrid& g, const double* q, const double* ox,
                                               const double* wx, int di, int dj, double sg,
                                               double fdisp, bool xdir) {
  int c = cix(g, di, dj).idx;
  double a0 = q[c];
  double am, ap, om, op;
  if (xdir) {
    am = cellS(g, q, di - 1, dj); ap = cellS(g, q, di + 1, dj);
    om = cellOX(g, ox, di - 1, dj); op = cellOX(g, ox, di + 1, dj);
  } else {
    am = cellS(g, q, di, dj - 1); ap = cellS(g, q, di, dj + 1);
    om = cellOY(g, ox, di, dj - 1); op = cellOY(g, ox, di, dj + 1);
  }
  double o0 = ox[c];
  double h = xdir ? g.dx : g.dy;
  double sl = vl_slope(a0 - am, ap - a0, h + o0 - om, h + op - o0);
  return a0 + 0.5 * sl * (sg * wx[c] - fdisp);
}
// Corner value, diagonal limited reconstruction (section 3.3): along v (or
// v_perp when dx dy < 0), slope over the diagonal neighbours' Lagrangian
// centres, evaluated at 1/2 (sgn(dx) (wx, +-wy) - (dx, dy)) . v from the
// donor's centre.
__device__ __forceinline__ double recon_corner(const LrGrid& g, const double* q, const LrWork& w,
                                               int di, int dj, double ddx, double ddy) {
  double sy = (ddx * ddy > 0.0) ? 1.0 : -1.0;
  int sj = sy > 0.0 ? 1 : -1;
  int c = cix(g, di, dj).idx;
  double a0 = q[c], ox0 = w.ox[c], oy0 = w.oy[c];
  double ap = cellS(g, q, di + 1, dj + sj), am = cellS(g, q, di - 1, dj - sj);
  double oxp = cellOX(g, w.ox, di + 1, dj + sj), oyp = cellOY(g, w.oy, di + 1, dj + sj);
  double oxm = cellOX(g, w.ox, di - 1, dj - sj), oym = cellOY(g, w.oy, di - 1, dj - sj);
  double sdy = sy * g.dy;
  double hp = ((g.dx + oxp - ox0) * g.dx + (sdy + oyp - oy0) * sdy) * g.invD;
  double hm = ((g.dx + ox0 - oxm) * g.dx + (sdy + oy0 - oym) * sdy) * g.invD;
  double sl = vl_slope(a0 - am, ap - a0, hm, hp);
  double sgx = ddx > 0.0 ? 1.0 : -1.0;
  double off = 0.5 * (sgx * (w.wx[c] * g.dx + w.wy[c] * g.dy) - (ddx * g.dx + sy * ddy * g.dy)) * g.invD;
  return a0 + sl * off;
}

// K5: per flux object (X face, Y face, corner): final material volumes (the
// pure donor gives its single material the whole flux; mixed donors' splits
// come from K4), reconstructed rho_a^{lagCF} and e_a^{lag} (order 2 only
// where the donor and its two neighbours along the direction are pure in
// that material -- section 4.2 remark), mass and energy fluxes, and the
// total mass fluxes the dual remap needs.
template <int M>
__global__ void __launch_bounds__(256) lr_mat_flux(LrGrid g, LrState cur, LrWork w) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  if (i >= g.nxu || j >= g.nyu) return;
  double dt = step_dt(g, w.scal);
  if (!(dt > 0.0)) return;
  int nn = g.nx + 1;
  int j1 = (g.pery && j + 1 == g.ny) ? 0 : j + 1;
  int i1 = (g.perx && i + 1 == g.nx) ? 0 : i + 1;
  // ---- X face (i, j)
  if (j < g.ny) {
    int f = j * nn + i;
    double v = w.fx[f];
    double mt = 0.0;
    unsigned dm = 0u;
    int di = 0, dc = 0;
    double sg = 1.0, fd = 0.0;
    if (v != 0.0) {
      bool left = v > 0.0;
      sg = left ? 1.0 : -1.0;
      di = left ? i - 1 : i;
      dc = cix(g, di, j).idx;
      dm = w.mask[dc];
      fd = 0.5 * (w.ddx[j * nn + i] + w.ddx[j1 * nn + i]);
    }
    bool mixed = (dm & (dm - 1u)) != 0u;
#pragma unroll
    for (int a = 0; a < M; ++a) {
      unsigned bit = 1u << a;
      if (!(dm & bit)) { w.xA[a][f] = 0.0; w.xMm[a][f] = 0.0; w.xE[a][f] = 0.0; continue; }
      double Aa = mixed ? w.xAm[a][f] : fabs(v);
      double Ma = 0.0, Ea = 0.0;
      if (!mixed || Aa > 0.0) {
        double rf = w.rcf[a][dc], ef = w.elag[a][dc];
        if (!mixed && g.face_o2 && pure_in(g, w.mask, di - 1, j, bit) && pure_in(g, w.mask, di + 1, j, bit)) {
          rf = recon_face_x(g, w.rcf[a], w.ox, w.wx, di, j, sg, fd, true);
          ef = recon_face_x(g, w.elag[a], w.ox, w.wx, di, j, sg, fd, true);
        }
        Ma = rf * Aa;
        Ea = Ma * ef;
      } else {
        Aa = 0.0;
      }
      w.xA[a][f] = sg * Aa; w.xMm[a][f] = sg * Ma; w.xE[a][f] = sg * Ea;
      mt += sg * Ma;
    }
    w.MX[f] = mt;
  }
  // ---- Y face (i, j)
  if (i < g.nx) {
    int f = j * g.nx + i;
    double v = w.fy[f];
    double mt = 0.0;
    unsigned dm = 0u;
    int dj = 0, dc = 0;
    double sg = 1.0, fd = 0.0;
    if (v != 0.0) {
      bool below = v > 0.0;
      sg = below ? 1.0 : -1.0;
      dj = below ? j - 1 : j;
      dc = cix(g, i, dj).idx;
      dm = w.mask[dc];
      fd = 0.5 * (w.ddy[j * nn + i] + w.ddy[j * nn + i1]);
    }
    bool mixed = (dm & (dm - 1u)) != 0u;
#pragma unroll
    for (int a = 0; a < M; ++a) {
      unsigned bit = 1u << a;
      if (!(dm & bit)) { w.yA[a][f] = 0.0; w.yMm[a][f] = 0.0; w.yE[a][f] = 0.0; continue; }
      double Aa = mixed ? w.yAm[a][f] : fabs(v);
      double Ma = 0.0, Ea = 0.0;
      if (!mixed || Aa > 0.0) {
        double rf = w.rcf[a][dc], ef = w.elag[a][dc];
        if (!mixed && g.face_o2 && pure_in(g, w.mask, i, dj - 1, bit) && pure_in(g, w.mask, i, dj + 1, bit)) {
          rf = recon_face_x(g, w.rcf[a], w.oy, w.wy, i, dj, sg, fd, false);
          ef = recon_face_x(g, w.elag[a], w.oy, w.wy, i, dj, sg, fd, false);
        }
        Ma = rf * Aa;
        Ea = Ma * ef;
      } else {
        Aa = 0.0;
      }
      w.yA[a][f] = sg * Aa; w.yMm[a][f] = sg * Ma; w.yE[a][f] = sg * Ea;
      mt += sg * Ma;
    }
    w.MY[f] = mt;
  }
  // ---- corner at node (i, j)
  {
    int n = j * nn + i;
    double ddx = w.ddx[n], ddy = w.ddy[n];
    double mt = 0.0;
    int di = 0, dj = 0, ri, rj, dc = 0, sj = 1;
    unsigned dm = 0u;
    double fv = 0.0;
    if (corner_cells(ddx, ddy, i, j, di, dj, ri, rj)) {
      fv = fabs(ddx * ddy);
      dc = cix(g, di, dj).idx;
      dm = w.mask[dc];
      sj = ddx * ddy > 0.0 ? 1 : -1;
    }
    bool mixed = (dm & (dm - 1u)) != 0u;
#pragma unroll
    for (int a = 0; a < M; ++a) {
      unsigned bit = 1u << a;
      if (!(dm & bit)) { w.cA[a][n] = 0.0; w.cMm[a][n] = 0.0; w.cE[a][n] = 0.0; continue; }
      double Aa = mixed ? w.cAm[a][n] : fv;
      double Ma = 0.0, Ea = 0.0;
      if (!mixed || Aa > 0.0) {
        double rf = w.rcf[a][dc], ef = w.elag[a][dc];
        if (!mixed && g.corner_o2 && pure_in(g, w.mask, di - 1, dj - sj, bit) &&
            pure_in(g, w.mask, di + 1, dj + sj, bit)) {
          rf = recon_corner(g, w.rcf[a], w, di, dj, ddx, ddy);
          ef = recon_corner(g, w.elag[a], w, di, dj, ddx, ddy);
        }
        Ma = rf * Aa;
        Ea = Ma * ef;
      } else {
        Aa = 0.0;
      }
      w.cA[a][n] = Aa; w.cMm[a][n] = Ma; w.cE[a][n] = Ea;
      mt += Ma;
    }
    double sgm = ddx > 0.0 ? mt : -mt;  // signed along +x
    bool pp = ddx * ddy > 0.0;
    w.Mpp[n] = pp ? sgm : 0.0;
    w.Mpm[n] = (!pp && dm) ? sgm : 0.0;
  }
}

// K6: cell remap (sections 2.3, 4.4): Vol_a, m_a and (m e)_a from the four
// faces and four corners; materials with Vol_a <= EPS_K dx dy are dropped
// (mass and energy to the largest remaining material); k_a = Vol_a / sum
// Vol; rho_a = m_a/(k_a dx dy); e_a = (m e)_a / m_a; the sound speed for the
// CFL rule of the next step.
template <int M>
__global__ void __launch_bounds__(256) lr_cell_update(LrGrid g, LrState cur, LrState nxt, LrWork w) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  int c = j * g.nx + i;
  double dt = step_dt(g, w.scal);
  if (!(dt > 0.0)) {
#pragma unroll
    for (int a = 0; a < M; ++a) { nxt.k[a][c] = cur.k[a][c]; nxt.r[a][c] = cur.r[a][c]; nxt.e[a][c] = cur.e[a][c]; }
    return;
  }
  // materials that can be in this cell after the remap: its own and those of
  // every cell that can donate to it (the 3x3 neighbourhood)
  unsigned own = w.mask[c], nb = own;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    if (q == 4) continue;
    nb |= w.mask[cix(g, i + q % 3 - 1, j + q / 3 - 1).idx];
  }
  int fl = xix(g, i, j).idx, fr = xix(g, i + 1, j).idx;
  int fb = yix(g, i, j).idx, ft = yix(g, i, j + 1).idx;
  int cn[4], cs[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int a = q & 1, b = q >> 1;
    int n = nix(g, i + a, j + b).idx;
    cn[q] = n;
    int di, dj, ri, rj;
    cs[q] = 0;
    if (corner_cells(w.ddx[n], w.ddy[n], i + a, j + b, di, dj, ri, rj)) {
      if (ri == i && rj == j) cs[q] = 1;
      if (di == i && dj == j) cs[q] = -1;
    }
  }
  double vcf = w.vcf[c];
  double vol[M], mas[M], ene[M];
#pragma unroll
  for (int a = 0; a < M; ++a) {
    vol[a] = 0.0; mas[a] = 0.0; ene[a] = 0.0;
    if (!(nb & (1u << a))) continue;
    double vv = 0.0, mm = 0.0, ee = 0.0;
    if (own & (1u << a)) {
      double ka = cur.k[a][c];
      mm = cur.r[a][c] * ka * g.V;
      vv = ka * vcf;
      ee = mm * w.elag[a][c];
    }
    vv += w.xA[a][fl] - w.xA[a][fr] + w.yA[a][fb] - w.yA[a][ft];
    mm += w.xMm[a][fl] - w.xMm[a][fr] + w.yMm[a][fb] - w.yMm[a][ft];
    ee += w.xE[a][fl] - w.xE[a][fr] + w.yE[a][fb] - w.yE[a][ft];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (cs[q] == 1) { vv += w.cA[a][cn[q]]; mm += w.cMm[a][cn[q]]; ee += w.cE[a][cn[q]]; }
      if (cs[q] == -1) { vv -= w.cA[a][cn[q]]; mm -= w.cMm[a][cn[q]]; ee -= w.cE[a][cn[q]]; }
    }
    vol[a] = vv; mas[a] = mm; ene[a] = ee;
  }
  bool keep[M];
  int big = -1, nkeep = 0;
  double tot = 0.0, lm = 0.0, le = 0.0;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    keep[a] = (nb & (1u << a)) && vol[a] > EPS_K * g.V;
    if (keep[a]) { tot += vol[a]; ++nkeep; if (big < 0 || vol[a] > vol[big]) big = a; }
    else { lm += mas[a]; le += ene[a]; }
  }
  if (big < 0) { set_err(w, LR_DERR_VOLUME, c); big = 0; tot = 1.0; }
#pragma unroll
  for (int a = 0; a < M; ++a) {
    if (a == big) { mas[a] += lm; ene[a] += le; }
  }
  double cmax = 0.0;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    double ka = 0.0, ra = 0.0, ea = 0.0;
    if (keep[a]) {
      ka = nkeep == 1 ? 1.0 : vol[a] / tot;
      if (!(mas[a] > 0.0)) set_err(w, LR_DERR_MASS, c);
      double im = 1.0 / mas[a];
      double kV = ka * g.V;
      ra = nkeep == 1 ? mas[a] * g.invV : mas[a] / kV;
      ea = ene[a] * im;
      double pa = eos_p(g.gam[a], g.pin[a], ra, ea);
      double c2 = (g.gam[a] * pa + g.pin[a]) * (kV * im);
      double wgt = ka * (1.0 / EPS_C) < 1.0 ? ka * (1.0 / EPS_C) : 1.0;
      if (wgt >= 1.0 && !(c2 > 0.0)) set_err(w, LR_DERR_SOUND, c);
      double ca = sqrt(c2 > 0.0 ? c2 : 0.0);
      if (wgt * ca > cmax) cmax = wgt * ca;
      if (!isfinite(ra) || !isfinite(ea)) set_err(w, LR_DERR_NAN, c);
    }
    nxt.k[a][c] = ka; nxt.r[a][c] = ra; nxt.e[a][c] = ea;
  }
  w.cc[c] = cmax;
}

// Dual-object reconstruction of a node velocity component along x or y:
// the primary formula with nodes as centres (Lagrangian positions x + d,
// dual width dx + (d_{q+1} - d_{q-1})/2, face displacement fdisp).
__device__ __forceinline__ double recon_dual_face(const LrGrid& g, const double* u, bool ucomp_x,
                                                  const double* dd, int qi, int qj, bool xdir,
                                                  double sg, double fdisp) {
  auto U = [&](int a, int b) { return ucomp_x ? nodeX(g, u, a, b) : nodeY(g, u, a, b); };
  auto Dd = [&](int a, int b) { return xdir ? nodeX(g, dd, a, b) : nodeY(g, dd, a, b); };
  int mi = xdir ? 1 : 0, mj = xdir ? 0 : 1;
  double u0 = U(qi, qj), up = U(qi + mi, qj + mj), um = U(qi - mi, qj - mj);
  double d0 = Dd(qi, qj), dp = Dd(qi + mi, qj + mj), dm = Dd(qi - mi, qj - mj);
  double h = xdir ? g.dx : g.dy;
  double sl = vl_slope(u0 - um, up - u0, h + d0 - dm, h + dp - d0);
  double wd = h + 0.5 * (dp - dm);
  return u0 + 0.5 * sl * (sg * wd - fdisp);
}

// K7a: dual-mesh fluxes (sections 2.1.1 and 2.3).  Dual X face between nodes
// (i,j),(i+1,j): 1/4 of the X-face mass fluxes bounding cells (i,j-1),(i,j).
// Dual Y face likewise.  Dual corners at the centre of cell (i,j): 1/4 of the
// corner mass fluxes of its four nodes running along ++ (joins nodes (i,j),
// (i+1,j+1)) or +- (joins (i,j+1),(i+1,j)).  Each object stores its mass flux
// and the momentum flux with the upwind-node velocity u^{lag} reconstructed
// on the dual mesh.  Objects just outside reflective walls are evaluated from
// the mirrored data, so every boundary node sees a full dual cell.
__global__ void __launch_bounds__(256) lr_dual_flux(LrGrid g, LrWork w) {
  int i = (int)(blockIdx.x * BX + threadIdx.x) - 1, j = (int)(blockIdx.y * BY + threadIdx.y) - 1;
  if (i > g.nx || j > g.ny) return;
  double dt = step_dt(g, w.scal);
  if (!(dt > 0.0)) return;
  bool xdual = g.perx ? (i >= 0 && i < g.nx) : true;   // dual index range in x
  bool ydual = g.pery ? (j >= 0 && j < g.ny) : true;
  bool xnode = i >= 0 && i < g.nxu;                     // canonical node in x
  bool ynode = j >= 0 && j < g.nyu;
  int o = (j + 1) * (g.nx + 2) + (i + 1);
  auto MXr = [&](int a, int b) { Ix q = xix(g, a, b); double v = w.MX[q.idx]; return q.fx ? -v : v; };
  auto MYr = [&](int a, int b) { Ix q = yix(g, a, b); double v = w.MY[q.idx]; return q.fy ? -v : v; };
  auto CPr = [&](int a, int b, double& pp, double& pm) {
    Ix q = nix(g, a, b);
    double x = w.Mpp[q.idx], y = w.Mpm[q.idx];
    if (q.fx) { double t = -y; y = -x; x = t; }
    if (q.fy) { double t = y; y = x; x = t; }
    pp = x; pm = y;
  };
  if (xdual && ynode) {  // dual X face between nodes (i,j), (i+1,j)
    double Dm = 0.25 * (MXr(i, j - 1) + MXr(i + 1, j - 1) + MXr(i, j) + MXr(i + 1, j));
    double px = 0.0, py = 0.0;
    if (Dm != 0.0) {
      int qi = Dm > 0.0 ? i : i + 1;
      double sg = Dm > 0.0 ? 1.0 : -1.0;
      double fd = 0.5 * (nodeX(g, w.ddx, i, j) + nodeX(g, w.ddx, i + 1, j));
      double vx, vy;
      if (g.face_o2) {
        vx = recon_dual_face(g, w.ulx, true, w.ddx, qi, j, true, sg, fd);
        vy = recon_dual_face(g, w.uly, false, w.ddx, qi, j, true, sg, fd);
      } else {
        vx = nodeX(g, w.ulx, qi, j); vy = nodeY(g, w.uly, qi, j);
      }
      px = Dm * vx; py = Dm * vy;
    }
    w.dX[0][o] = Dm; w.dX[1][o] = px; w.dX[2][o] = py;
  }
  if (xnode && ydual) {  // dual Y face between nodes (i,j), (i,j+1)
    double Dm = 0.25 * (MYr(i - 1, j) + MYr(i - 1, j + 1) + MYr(i, j) + MYr(i, j + 1));
    double px = 0.0, py = 0.0;
    if (Dm != 0.0) {
      int qj = Dm > 0.0 ? j : j + 1;
      double sg = Dm > 0.0 ? 1.0 : -1.0;
      double fd = 0.5 * (nodeY(g, w.ddy, i, j) + nodeY(g, w.ddy, i, j + 1));
      double vx, vy;
      if (g.face_o2) {
        vx = recon_dual_face(g, w.ulx, true, w.ddy, i, qj, false, sg, fd);
        vy = recon_dual_face(g, w.uly, false, w.ddy, i, qj, false, sg, fd);
      } else {
        vx = nodeX(g, w.ulx, i, qj); vy = nodeY(g, w.uly, i, qj);
      }
      px = Dm * vx; py = Dm * vy;
    }
    w.dY[0][o] = Dm; w.dY[1][o] = px; w.dY[2][o] = py;
  }
  if (xdual && ydual) {  // dual corners at the centre of cell (i,j)
    double p0, m0, p1, m1, p2, m2, p3, m3;
    CPr(i, j, p0, m0); CPr(i + 1, j, p1, m1); CPr(i, j + 1, p2, m2); CPr(i + 1, j + 1, p3, m3);
    double cdx = 0.25 * (nodeX(g, w.ddx, i, j) + nodeX(g, w.ddx, i + 1, j) + nodeX(g, w.ddx, i, j + 1) +
                         nodeX(g, w.ddx, i + 1, j + 1));
    double cdy = 0.25 * (nodeY(g, w.ddy, i, j) + nodeY(g, w.ddy, i + 1, j) + nodeY(g, w.ddy, i, j + 1) +
                         nodeY(g, w.ddy, i + 1, j + 1));
    for (int kind = 0; kind < 2; ++kind) {
      bool pp = kind == 0;
      double Dm = pp ? 0.25 * (p0 + p1 + p2 + p3) : 0.25 * (m0 + m1 + m2 + m3);
      double px = 0.0, py = 0.0;
      if (Dm != 0.0) {
        int ai = i, aj = pp ? j : j + 1, bi = i + 1, bj = pp ? j + 1 : j;
        int qi = Dm > 0.0 ? ai : bi, qj = Dm > 0.0 ? aj : bj;
        double sg = Dm > 0.0 ? 1.0 : -1.0;
        double vx = nodeX(g, w.ulx, qi, qj), vy = nodeY(g, w.uly, qi, qj);
        if (g.corner_o2) {
          double sy = pp ? 1.0 : -1.0;
          int sj = pp ? 1 : -1;
          double sdy = sy * g.dy;
          double dx0 = nodeX(g, w.ddx, qi, qj), dy0 = nodeY(g, w.ddy, qi, qj);
          double dxp = nodeX(g, w.ddx, qi + 1, qj + sj), dyp = nodeY(g, w.ddy, qi + 1, qj + sj);
          double dxm = nodeX(g, w.ddx, qi - 1, qj - sj), dym = nodeY(g, w.ddy, qi - 1, qj - sj);
          double hp = ((g.dx + dxp - dx0) * g.dx + (sdy + dyp - dy0) * sdy) * g.invD;
          double hm = ((g.dx + dx0 - dxm) * g.dx + (sdy + dy0 - dym) * sdy) * g.invD;
          double wxq = g.dx + 0.5 * (nodeX(g, w.ddx, qi + 1, qj) - nodeX(g, w.ddx, qi - 1, qj));
          double wyq = g.dy + 0.5 * (nodeY(g, w.ddy, qi, qj + 1) - nodeY(g, w.ddy, qi, qj - 1));
          double off = 0.5 * (sg * (wxq * g.dx + wyq * g.dy) - (cdx * g.dx + sy * cdy * g.dy)) * g.invD;
          double uxp = nodeX(g, w.ulx, qi + 1, qj + sj), uxm = nodeX(g, w.ulx, qi - 1, qj - sj);
          double uyp = nodeY(g, w.uly, qi + 1, qj + sj), uym = nodeY(g, w.uly, qi - 1, qj - sj);
          vx = vx + vl_slope(vx - uxm, uxp - vx, hm, hp) * off;
          vy = vy + vl_slope(vy - uym, uyp - vy, hm, hp) * off;
        }
        px = Dm * vx; py = Dm * vy;
      }
      if (pp) { w.dPP[0][o] = Dm; w.dPP[1][o] = px; w.dPP[2][o] = py; }
      else { w.dPM[0][o] = Dm; w.dPM[1][o] = px; w.dPM[2][o] = py; }
    }
  }
}

// Block-wide max of v >= 0 folded into red[0]; the last block of the grid
// turns it into the next CFL time step (and advances t when `advance`).
__device__ void cfl_finalize(const LrGrid& g, const LrWork& w, double v, bool advance, double dt) {
  __shared__ double sm[32];
  __shared__ int last;
  int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  if ((tid & 31) == 0) sm[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    int nw = (blockDim.x * blockDim.y) >> 5;
    double x = tid < nw ? sm[tid] : 0.0;
    for (int off = 16; off > 0; off >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, off));
    if (tid == 0) {
      atomicMax(&w.red[0], (unsigned long long)__double_as_longlong(x));
      __threadfence();
      unsigned long long nb = (unsigned long long)gridDim.x * gridDim.y;
      unsigned long long prev = atomicAdd(&w.red[1], 1ull);
      last = prev == nb - 1;
    }
  }
  __syncthreads();
  if (last && tid == 0) {
    __threadfence();
    double mx = __longlong_as_double((long long)atomicAdd(&w.red[0], 0ull));
    double best = mx > 0.0 ? g.hmin / mx : 1e300;
    double t = w.scal[0];
    if (advance) { t = t + dt; w.scal[2] = dt; w.scal[4] += 1.0; }
    w.scal[0] = t;
    w.scal[1] = g.cfl * best;
    w.red[0] = 0ull;
    w.red[1] = 0ull;
    w.red[2] = 0ull;
  }
}

// K7b: nodal momentum remap m_p' u_p' = m_p u_p^{lag} + sum of signed dual
// momentum fluxes, m_p' = m_p + sum of signed dual mass fluxes
// (m_p = 1/4 sum of the cell masses), wall-normal velocity zero; then the
// CFL rule for the next step from max over nodes of (max over the node's
// cells of c_c + |u_p|), which equals the per-cell form
// min_c min(dx,dy)/(c_c + max_{p in c} |u_p|).
__global__ void __launch_bounds__(256) lr_node_update(LrGrid g, LrState cur, LrState nxt, LrWork w) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  bool act = i < g.nxu && j < g.nyu;
  double dt = step_dt(g, w.scal);
  if (!(dt > 0.0)) {
    if (act) { int n = j * (g.nx + 1) + i; nxt.ux[n] = cur.ux[n]; nxt.uy[n] = cur.uy[n]; }
    if (i == 0 && j == 0) w.scal[2] = 0.0;
    return;
  }
  double val = 0.0;
  if (act) {
    int n = j * (g.nx + 1) + i;
    double ux1, uy1;
    if (g.presc) {
      ux1 = w.pux[n]; uy1 = w.puy[n];
    } else {
      int A = cix(g, i - 1, j - 1).idx, B = cix(g, i, j - 1).idx;
      int C = cix(g, i - 1, j).idx, Dd = cix(g, i, j).idx;
      double mp = 0.25 * (w.mc[A] + w.mc[B] + w.mc[C] + w.mc[Dd]);
      double mnew = mp, px = mp * w.ulx[n], py = mp * w.uly[n];
      int oR = dix(g, i, j), oL = dix(g, i - 1, j), oT = dix(g, i, j), oB = dix(g, i, j - 1);
      mnew += -w.dX[0][oR] + w.dX[0][oL]; px += -w.dX[1][oR] + w.dX[1][oL]; py += -w.dX[2][oR] + w.dX[2][oL];
      mnew += -w.dY[0][oT] + w.dY[0][oB]; px += -w.dY[1][oT] + w.dY[1][oB]; py += -w.dY[2][oT] + w.dY[2][oB];
      int c0 = dix(g, i, j), c1 = dix(g, i - 1, j - 1), c2 = dix(g, i, j - 1), c3 = dix(g, i - 1, j);
      mnew += -w.dPP[0][c0] + w.dPP[0][c1] - w.dPM[0][c2] + w.dPM[0][c3];
      px += -w.dPP[1][c0] + w.dPP[1][c1] - w.dPM[1][c2] + w.dPM[1][c3];
      py += -w.dPP[2][c0] + w.dPP[2][c1] - w.dPM[2][c2] + w.dPM[2][c3];
      if (!(mnew > 0.0)) set_err(w, LR_DERR_MASS, n);
      double im = 1.0 / mnew;
      ux1 = px * im;
      uy1 = py * im;
      if (!isfinite(ux1) || !isfinite(uy1)) set_err(w, LR_DERR_NAN, n);
    }
    if (!g.perx && (i == 0 || i == g.nx)) ux1 = 0.0;
    if (!g.pery && (j == 0 || j == g.ny)) uy1 = 0.0;
    nxt.ux[n] = ux1;
    nxt.uy[n] = uy1;
    double cm = fmax(fmax(w.cc[cix(g, i - 1, j - 1).idx], w.cc[cix(g, i, j - 1).idx]),
                     fmax(w.cc[cix(g, i - 1, j).idx], w.cc[cix(g, i, j).idx]));
    val = cm + sqrt(ux1 * ux1 + uy1 * uy1);
  }
  cfl_finalize(g, w, val, true, dt);
}

// CFL rule from the current state only (after lr_init).
__global__ void __launch_bounds__(256) lr_cfl_only(LrGrid g, LrState cur, LrWork w) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  double val = 0.0;
  if (i < g.nxu && j < g.nyu) {
    int n = j * (g.nx + 1) + i;
    double ux1 = cur.ux[n], uy1 = cur.uy[n];
    double cm = fmax(fmax(w.cc[cix(g, i - 1, j - 1).idx], w.cc[cix(g, i, j - 1).idx]),
                     fmax(w.cc[cix(g, i - 1, j).idx], w.cc[cix(g, i, j).idx]));
    val = cm + sqrt(ux1 * ux1 + uy1 * uy1);
  }
  cfl_finalize(g, w, val, false, 0.0);
}

// Initial state: the upload placed k, rho and p in the state arrays; drop
// materials with k <= EPS_K, renormalise, e = (p + pi)/((gamma-1) rho),
// sound speed; zero wall-normal node velocities.
template <int M>
__global__ void __launch_bounds__(256) lr_prepare(LrGrid g, LrState st, LrWork w) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  if (i <= g.nx && j <= g.ny) {
    int n = j * (g.nx + 1) + i;
    if (!g.perx && (i == 0 || i == g.nx)) st.ux[n] = 0.0;
    if (!g.pery && (j == 0 || j == g.ny)) st.uy[n] = 0.0;
  }
  if (i >= g.nx || j >= g.ny) return;
  int c = j * g.nx + i;
  double sum = 0.0, kept = 0.0;
  bool bad = false;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    double ka = st.k[a][c];
    if (!(ka >= -1e-12 && ka <= 1.0 + 1e-12)) bad = true;
    sum += ka;
    if (ka > EPS_K) kept += ka;
  }
  if (!(fabs(sum - 1.0) <= 1e-9)) bad = true;
  double cmax = 0.0;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    double ka = st.k[a][c];
    if (ka > EPS_K && !bad) {
      double ra = st.r[a][c], pa = st.e[a][c];
      if (!(ra > 0.0)) bad = true;
      double kn = ka / kept;
      double ea = (pa + g.pin[a]) / ((g.gam[a] - 1.0) * ra);
      st.k[a][c] = kn; st.e[a][c] = ea;
      double p2 = eos_p(g.gam[a], g.pin[a], ra, ea);
      double c2 = eos_c2(g.gam[a], g.pin[a], ra, p2);
      double wgt = kn / EPS_C < 1.0 ? kn / EPS_C : 1.0;
      double ca = sqrt(c2 > 0.0 ? c2 : 0.0);
      if (wgt * ca > cmax) cmax = wgt * ca;
    } else {
      st.k[a][c] = 0.0; st.r[a][c] = 0.0; st.e[a][c] = 0.0;
    }
  }
  if (bad) set_err(w, LR_DERR_MASS, c);
  w.cc[c] = cmax;
}

__global__ void lr_set_scalar_k(double* p, double v) { *p = v; }
__global__ void lr_reset_k(LrWork w) {
  w.red[0] = 0ull; w.red[1] = 0ull; w.red[2] = 0ull; w.err[0] = 0; w.err[1] = -1;
  w.scal[0] = 0.0; w.scal[1] = 0.0; w.scal[2] = 0.0; w.scal[3] = 0.0; w.scal[4] = 0.0;
}

// Debug view of the last step's corner fluxes: |dx dy| and total mass.
template <int M>
__global__ void lr_corner_dbg(LrGrid g, LrWork w, double* fc, double* mcn) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  if (i > g.nx || j > g.ny) return;
  int o = j * (g.nx + 1) + i;
  int n = nix(g, i, j).idx;
  double ddx = w.ddx[n], ddy = w.ddy[n];
  if (fc) fc[o] = fabs(ddx * ddy);
  if (mcn) {
    double m = 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a) m += w.cMm[a][n];
    mcn[o] = m;
  }
}

inline dim3 grid_for(int nxr, int nyr) { return dim3((nxr + BX - 1) / BX, (nyr + BY - 1) / BY); }

}  // namespace

#define LR_DISPATCH_M(KERNEL, GRID, ...)                                        \
  do {                                                                          \
    if (g.M == 1) KERNEL<1><<<GRID, dim3(BX, BY), 0, s>>>(__VA_ARGS__);         \
    else if (g.M == 2) KERNEL<2><<<GRID, dim3(BX, BY), 0, s>>>(__VA_ARGS__);    \
    else KERNEL<3><<<GRID, dim3(BX, BY), 0, s>>>(__VA_ARGS__);                  \
  } while (0)

cudaError_t lr_launch(int kid, const LrGrid& g, const LrState& cur, const LrState& nxt,
                      const LrWork& w, cudaStream_t s) {
  switch (kid) {
    case LRK_CELL_PRE: LR_DISPATCH_M(lr_cell_pre, grid_for(g.nx, g.ny), g, cur, w); break;
    case LRK_NODE_HALF: lr_node_half<<<grid_for(g.nxu, g.nyu), dim3(BX, BY), 0, s>>>(g, cur, w); break;
    case LRK_CELL_LAG: LR_DISPATCH_M(lr_cell_lag, grid_for(g.nxu, g.nyu), g, cur, w); break;
    case LRK_CELL_CF: LR_DISPATCH_M(lr_cell_cf, grid_for(g.nx, g.ny), g, cur, w); break;
    case LRK_MIXED: {
      int nb = (g.nx * g.ny + 127) / 128;
      if (nb > 152 * 8) nb = 152 * 8;
      if (g.M == 1) break;  // one material: no interfaces
      if (g.M == 2) lr_mixed<2><<<nb, 128, 0, s>>>(g, cur, w);
      else lr_mixed<3><<<nb, 128, 0, s>>>(g, cur, w);
      break;
    }
    case LRK_MAT_FLUX: LR_DISPATCH_M(lr_mat_flux, grid_for(g.nxu, g.nyu), g, cur, w); break;
    case LRK_CELL_UPDATE: LR_DISPATCH_M(lr_cell_update, grid_for(g.nx, g.ny), g, cur, nxt, w); break;
    case LRK_DUAL_FLUX: lr_dual_flux<<<grid_for(g.nx + 2, g.ny + 2), dim3(BX, BY), 0, s>>>(g, w); break;
    case LRK_NODE_UPDATE: lr_node_update<<<grid_for(g.nxu, g.nyu), dim3(BX, BY), 0, s>>>(g, cur, nxt, w); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t lr_launch_init_cfl(const LrGrid& g, const LrState& cur, const LrWork& w, cudaStream_t s) {
  lr_cfl_only<<<grid_for(g.nxu, g.nyu), dim3(BX, BY), 0, s>>>(g, cur, w);
  return cudaGetLastError();
}

cudaError_t lr_launch_prepare_init(const LrGrid& g, const LrState& st, const LrWork& w, cudaStream_t s) {
  LR_DISPATCH_M(lr_prepare, grid_for(g.nx + 1, g.ny + 1), g, st, w);
  return cudaGetLastError();
}

cudaError_t lr_launch_set_scalar(double* p, double v, cudaStream_t s) {
  lr_set_scalar_k<<<1, 1, 0, s>>>(p, v);
  return cudaGetLastError();
}

cudaError_t lr_launch_reset(const LrWork& w, cudaStream_t s) {
  lr_reset_k<<<1, 1, 0, s>>>(w);
  return cudaGetLastError();
}

cudaError_t lr_launch_corner_debug(const LrGrid& g, const LrWork& w, double* fc_out, double* mc_out,
                                   cudaStream_t s) {
  LR_DISPATCH_M(lr_corner_dbg, grid_for(g.nx + 1, g.ny + 1), g, w, fc_out, mc_out);
  return cudaGetLastError();
}
