/*
 * lr_oracle.c -- plain, slow FP64 reference of one time step of the staggered
 * Lagrange-Remap scheme of Chaudet (arXiv 2208.13409): SGPC Lagrange phase
 * (section 1.2 eqs. "prediction"/"correction", multi-material form of
 * section 4.1), one-step remap with face and corner fluxes (section 2.3),
 * the comparators of section 2 (one-step face-only "Direct" remap and the
 * alternate-directions "AD" remap, multi-material forms of section 4.3),
 * corner reconstructions (section 3.3), VOF/PLIC material fluxes on the
 * rectangular Lagrangian cell (section 4.4), dual-mesh momentum remap
 * (sections 2.1.1 and 2.3) and the CFL time step (annex CFL definition).
 *
 * TEST INFRASTRUCTURE ONLY (tests/, smoke check, bench.py CPU baseline).
 * It shares no code with the CUDA library; the product never calls it.
 *
 * Style: whole-array loops over arrays with G ghost layers, one phase at a
 * time; boundary conditions are re-applied to every intermediate field that
 * a later phase reads outside the interior (the analogue of a halo exchange
 * between phases).  No blocking, fusion or reordering.
 *
 * Readings of points the paper leaves open (garbled formulas, unstated
 * constants, inconsistent signs) are stated at each use below.  Pins
 * (tests/) cover:
 * EOS, cell volume F, Van Leer limiter, half-plane clipping and PLIC
 * placement, face/corner volume fluxes (one-node displacement expansion,
 * uniform translation), order-1 linear advection closed form, order-2 exact
 * translation of linear fields, uniform-state preservation, conservation,
 * Sod shock tube against the exact Riemann solution, translated planar
 * interfaces, volume-fraction bounds, mirror and transpose symmetry, CFL,
 * and the dual-mesh momentum remap: remapped nodal mass equal to a quarter
 * of the four remapped cell masses, the order-1 box formula on the dual
 * mesh, and exact dual face and corner fluxes of linear velocity fields
 * under uniform and axis-preserving affine displacements (the hook
 * orc_set_remap_velocity carries a given node field under a prescribed
 * displacement).
 * Parity unpinned beyond those invariants: the flux clipping near k=0 and
 * the material-removal threshold (clip_and_split, cell_update), the
 * 3-material nested interface order and the sound-speed ramp for nearly
 * empty materials; these follow the readings stated at their definitions.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "lr_oracle.h"

#define G 2          /* ghost layers */
#define MAXM 3
#define EPS_K 1e-12  /* material removed when Vol_a <= EPS_K * dx*dy */
#define EPS_C 1e-3   /* sound-speed weight min(1, k/EPS_C) */
#define MAXV 16      /* polygon vertex capacity */

struct orc {
  orc_config c;
  int nx, ny, M;
  double dx, dy, V;
  double gam[MAXM], pin[MAXM];
  int perx, pery;
  int cw, ch;     /* cell arrays:   (nx+2G) x (ny+2G)     */
  int nw, nh;     /* node arrays:   (nx+1+2G) x (ny+1+2G) */
  int xw, xh;     /* X-face arrays: (nx+1+2G) x (ny+2G)   */
  int yw, yh;     /* Y-face arrays: (nx+2G) x (ny+1+2G)   */
  double t, lastdt;
  int inited;
  /* state at t^n */
  double *k[MAXM], *r[MAXM], *e[MAXM];
  double *ux, *uy;
  int presc;
  double *pux, *puy;
  /* cell intermediates */
  double *mc, *cc, *Q, *Pi, *volh, *vollag, *vcf;
  double *Pa[MAXM], *Ph[MAXM], *elag[MAXM], *rcf[MAXM];
  double *ox, *oy, *wx, *wy;
  int *ncut;
  int *cutmat;                  /* [cell][MAXM]: present materials in order */
  double *cn[MAXM - 1][3];      /* per cut: normal x, normal y, constant d */
  double *cnY[MAXM - 1][3];     /* Direct remap: the cuts used for Y faces */
  double *fdx, *fdy;            /* AD remap: full displacement dt u^{n+1/2} */
  long nsteps;                  /* steps taken (AD sweep order) */
  double *outv[MAXM], *sclip[MAXM];
  int *dom;
  /* node intermediates */
  double *uhx, *uhy, *ulx, *uly, *ddx, *ddy;
  double *fc;                   /* corner |dVol| */
  double *cA[MAXM], *cMm[MAXM], *cE[MAXM]; /* corner per-material (positive) */
  double *Mpp, *Mpm;
  double *mpn;                  /* remapped nodal mass m_p' of the last step */
  double *dual[4][3];           /* dual X face, Y face, ++ and +- corner: mass, x- and y-momentum flux */
  int ruse;                     /* test hook: remap this node field under a prescribed velocity */
  double *rux, *ruy;
  /* face intermediates */
  double *fx, *fxlo, *fxhi, *fxb; /* X-faces */
  double *fy, *fylo, *fyhi, *fyb; /* Y-faces */
  double *xA[MAXM], *xMm[MAXM], *xE[MAXM];
  double *yA[MAXM], *yMm[MAXM], *yE[MAXM];
  double *MX, *MY;
  /* outputs kept for orc_get */
  double *cmass_mat_tot;
};

/* ---------------------------------------------------------------- indexing */
static inline int CI(const orc* s, int i, int j) { return (j + G) * s->cw + (i + G); }
static inline int NI(const orc* s, int i, int j) { return (j + G) * s->nw + (i + G); }
static inline int XI(const orc* s, int i, int j) { return (j + G) * s->xw + (i + G); }
static inline int YI(const orc* s, int i, int j) { return (j + G) * s->yw + (i + G); }

/* Cell index along one axis mapped into the interior: reflect mirrors about
 * the wall, periodic wraps.  *flip = 1 when a mirror was applied. */
static int map_cell(int i, int n, int per, int* flip) {
  *flip = 0;
  if (i >= 0 && i < n) return i;
  if (per) return ((i % n) + n) % n;
  *flip = 1;
  return i < 0 ? -1 - i : 2 * n - 1 - i;
}
/* Node index along one axis: reflect keeps nodes 0..n (mirror about node 0
 * and node n); periodic keeps 0..n-1 (node n is node 0). */
static int map_node(int i, int n, int per, int* flip) {
  *flip = 0;
  if (per) { int m = ((i % n) + n) % n; return m; }
  if (i >= 0 && i <= n) return i;
  *flip = 1;
  return i < 0 ? -i : 2 * n - i;
}
static int node_interior(int i, int n, int per) { return per ? (i >= 0 && i < n) : (i >= 0 && i <= n); }

/* ------------------------------------------------------------ ghost fills */
static void fill_cell(orc* s, double* a) {
  for (int j = -G; j < s->ny + G; ++j)
    for (int i = -G; i < s->nx + G; ++i) {
      if (i >= 0 && i < s->nx && j >= 0 && j < s->ny) continue;
      int fx, fy;
      int mi = map_cell(i, s->nx, s->perx, &fx), mj = map_cell(j, s->ny, s->pery, &fy);
      a[CI(s, i, j)] = a[CI(s, mi, mj)];
    }
}
static void fill_cell_int(orc* s, int* a) {
  for (int j = -G; j < s->ny + G; ++j)
    for (int i = -G; i < s->nx + G; ++i) {
      if (i >= 0 && i < s->nx && j >= 0 && j < s->ny) continue;
      int fx, fy;
      int mi = map_cell(i, s->nx, s->perx, &fx), mj = map_cell(j, s->ny, s->pery, &fy);
      a[CI(s, i, j)] = a[CI(s, mi, mj)];
    }
}
/* Node vector: the x component changes sign under an x mirror, y under y. */
static void fill_node_vec(orc* s, double* ax, double* ay) {
  for (int j = -G; j <= s->ny + G; ++j)
    for (int i = -G; i <= s->nx + G; ++i) {
      if (node_interior(i, s->nx, s->perx) && node_interior(j, s->ny, s->pery)) continue;
      int fx, fy;
      int mi = map_node(i, s->nx, s->perx, &fx), mj = map_node(j, s->ny, s->pery, &fy);
      int m = NI(s, mi, mj), d = NI(s, i, j);
      ax[d] = fx ? -ax[m] : ax[m];
      ay[d] = fy ? -ay[m] : ay[m];
    }
}
/* X-face signed flux: odd under an x mirror, even under a y mirror. */
static void fill_xface(orc* s, double* a) {
  for (int j = -G; j < s->ny + G; ++j)
    for (int i = -G; i <= s->nx + G; ++i) {
      if (node_interior(i, s->nx, s->perx) && j >= 0 && j < s->ny) continue;
      int fx, fy;
      int mi = map_node(i, s->nx, s->perx, &fx), mj = map_cell(j, s->ny, s->pery, &fy);
      double v = a[XI(s, mi, mj)];
      a[XI(s, i, j)] = fx ? -v : v;
    }
}
/* Y-face signed flux: even under an x mirror, odd under a y mirror. */
static void fill_yface(orc* s, double* a) {
  for (int j = -G; j <= s->ny + G; ++j)
    for (int i = -G; i < s->nx + G; ++i) {
      if (i >= 0 && i < s->nx && node_interior(j, s->ny, s->pery)) continue;
      int fx, fy;
      int mi = map_cell(i, s->nx, s->perx, &fx), mj = map_node(j, s->ny, s->pery, &fy);
      double v = a[YI(s, mi, mj)];
      a[YI(s, i, j)] = fy ? -v : v;
    }
}
/* Node diagonal fluxes: pp is signed along (+x,+y), pm along (+x,-y).  An x
 * mirror maps a (+x,+y) flux to (-x,+y) = -(+x,-y); a y mirror maps it to
 * (+x,-y). */
static void fill_corner(orc* s, double* pp, double* pm) {
  for (int j = -G; j <= s->ny + G; ++j)
    for (int i = -G; i <= s->nx + G; ++i) {
      if (node_interior(i, s->nx, s->perx) && node_interior(j, s->ny, s->pery)) continue;
      int fx, fy;
      int mi = map_node(i, s->nx, s->perx, &fx), mj = map_node(j, s->ny, s->pery, &fy);
      int m = NI(s, mi, mj), d = NI(s, i, j);
      double a = pp[m], b = pm[m];
      if (fx) { double ta = -b, tb = -a; a = ta; b = tb; }
      if (fy) { double ta = b, tb = a; a = ta; b = tb; }
      pp[d] = a;
      pm[d] = b;
    }
}
static void fill_node_scalar(orc* s, double* a) {
  for (int j = -G; j <= s->ny + G; ++j)
    for (int i = -G; i <= s->nx + G; ++i) {
      if (node_interior(i, s->nx, s->perx) && node_interior(j, s->ny, s->pery)) continue;
      int fx, fy;
      int mi = map_node(i, s->nx, s->perx, &fx), mj = map_node(j, s->ny, s->pery, &fy);
      a[NI(s, i, j)] = a[NI(s, mi, mj)];
    }
}

/* ------------------------------------------------------------------ EOS */
/* Stiffened gas p = (gamma-1) rho e - pi (section 5.2, water); pi = 0 is the
 * perfect gas of section 5.1.  Sound speed from the isentrope de = -p dv:
 * c^2 = (gamma p + pi) / rho. */
static double eos_p(double g, double pi, double rho, double e) { return (g - 1.0) * rho * e - pi; }
static double eos_c2(double g, double pi, double rho, double p) { return (g * p + pi) / rho; }

void orc_t_eos(double gamma, double pinf, double rho, double e, double* p, double* c2) {
  *p = eos_p(gamma, pinf, rho, e);
  *c2 = eos_c2(gamma, pinf, rho, *p);
}

/* ---------------------------------------------------------- geometry bits */
/* Cell volume F of section 1.2: two triangles split along the lr-ul diagonal,
 * 1/2|dx_{i-1/2,j} ^ dx_{i,j-1/2}| + 1/2|dx_{i+1/2,j} ^ dx_{i,j+1/2}|, with
 * the face vectors left = ul-ll, bottom = lr-ll, right = ur-lr, top = ur-ul. */
static double cell_volume(double llx, double lly, double lrx, double lry,
                          double ulx, double uly, double urx, double ury) {
  double lx = ulx - llx, ly = uly - lly;   /* left face   */
  double bx = lrx - llx, by = lry - lly;   /* bottom face */
  double rx = urx - lrx, ry = ury - lry;   /* right face  */
  double tx = urx - ulx, ty = ury - uly;   /* top face    */
  return 0.5 * fabs(lx * by - ly * bx) + 0.5 * fabs(rx * ty - ry * tx);
}
double orc_t_cell_volume(const double* p) {
  return cell_volume(p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7]);
}

/* Van Leer limited slope of section 2.1.1:
 * 1/2 (phi(r) d+ + phi(1/r) d-), r = d-/d+, phi(r) = (r+|r|)/(1+r).
 * Written out: phi(r) d+ = phi(1/r) d- = 2 d+ d- / (d+ + d-) when d+ d- > 0,
 * and both vanish otherwise (r <= 0), so the limited slope is the harmonic
 * mean 2 d+ d- / (d+ + d-) or 0. */
static double vanleer(double dm, double dp) {
  if (dm * dp > 0.0) return 2.0 * dm * dp / (dm + dp);
  return 0.0;
}
double orc_t_vanleer(double dm, double dp) { return vanleer(dm, dp); }

/* Sutherland-Hodgman clip of a convex polygon by the half-plane x.n <= d
 * (keep = +1) or x.n >= d (keep = -1). */
static int clip_poly(const double* in, int n, double nx, double ny, double d, int keep, double* out) {
  int m = 0;
  for (int a = 0; a < n; ++a) {
    int b = (a + 1) % n;
    double xa = in[2 * a], ya = in[2 * a + 1], xb = in[2 * b], yb = in[2 * b + 1];
    double fa = keep * (xa * nx + ya * ny - d), fb = keep * (xb * nx + yb * ny - d);
    if (fa <= 0.0) { out[2 * m] = xa; out[2 * m + 1] = ya; ++m; }
    if ((fa < 0.0 && fb > 0.0) || (fa > 0.0 && fb < 0.0)) {
      double tt = fa / (fa - fb);
      out[2 * m] = xa + tt * (xb - xa);
      out[2 * m + 1] = ya + tt * (yb - ya);
      ++m;
    }
  }
  return m;
}
static double poly_area(const double* p, int n) {
  double a = 0.0;
  for (int k = 0; k < n; ++k) {
    int l = (k + 1) % n;
    a += p[2 * k] * p[2 * l + 1] - p[2 * l] * p[2 * k + 1];
  }
  return 0.5 * fabs(a);
}
static double halfplane_area(const double* poly, int n, double nx, double ny, double d) {
  double tmp[2 * MAXV];
  int m = clip_poly(poly, n, nx, ny, d, +1, tmp);
  return m >= 3 ? poly_area(tmp, m) : 0.0;
}
double orc_t_halfplane_area(const double* poly, int nv, double nx, double ny, double d) {
  return halfplane_area(poly, nv, nx, ny, d);
}
/* PLIC line constant: the d for which the part {x.n <= d} of the polygon has
 * the prescribed area (section 4.1 "interface positioning").  The oracle
 * solves this definition by plain bisection to machine precision. */
static double plic_solve(const double* poly, int n, double nx, double ny, double target) {
  double lo = 1e300, hi = -1e300;
  for (int k = 0; k < n; ++k) {
    double v = poly[2 * k] * nx + poly[2 * k + 1] * ny;
    if (v < lo) lo = v;
    if (v > hi) hi = v;
  }
  for (int it = 0; it < 400; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (halfplane_area(poly, n, nx, ny, mid) < target) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}
double orc_t_plic(const double* poly, int nv, double nx, double ny, double target) {
  return plic_solve(poly, nv, nx, ny, target);
}
static void rect_poly(double x0, double x1, double y0, double y1, double* p) {
  p[0] = x0; p[1] = y0; p[2] = x1; p[3] = y0; p[4] = x1; p[5] = y1; p[6] = x0; p[7] = y1;
}

/* ------------------------------------------------------------- allocation */
static double* dalloc(long n) { return (double*)calloc((size_t)n, sizeof(double)); }

orc* orc_create(const orc_config* cfg, const double* gamma, const double* pinf) {
  if (!cfg || cfg->nx < 2 || cfg->ny < 2 || cfg->nmat < 1 || cfg->nmat > MAXM) return NULL;
  if (cfg->bc[0] != cfg->bc[1] || cfg->bc[2] != cfg->bc[3]) return NULL;
  if (!(cfg->x1 > cfg->x0) || !(cfg->y1 > cfg->y0)) return NULL;
  if (cfg->remap < ORC_REMAP_DIRECTCF || cfg->remap > ORC_REMAP_AD) return NULL;
  orc* s = (orc*)calloc(1, sizeof(orc));
  s->c = *cfg;
  s->nx = cfg->nx; s->ny = cfg->ny; s->M = cfg->nmat;
  s->dx = (cfg->x1 - cfg->x0) / cfg->nx;
  s->dy = (cfg->y1 - cfg->y0) / cfg->ny;
  s->V = s->dx * s->dy;
  for (int a = 0; a < s->M; ++a) { s->gam[a] = gamma[a]; s->pin[a] = pinf[a]; }
  s->perx = cfg->bc[0] == ORC_BC_PERIODIC;
  s->pery = cfg->bc[2] == ORC_BC_PERIODIC;
  s->cw = s->nx + 2 * G; s->ch = s->ny + 2 * G;
  s->nw = s->nx + 1 + 2 * G; s->nh = s->ny + 1 + 2 * G;
  s->xw = s->nx + 1 + 2 * G; s->xh = s->ny + 2 * G;
  s->yw = s->nx + 2 * G; s->yh = s->ny + 1 + 2 * G;
  long nc = (long)s->cw * s->ch, nn = (long)s->nw * s->nh;
  long nfx = (long)s->xw * s->xh, nfy = (long)s->yw * s->yh;
  for (int a = 0; a < MAXM; ++a) {
    s->k[a] = dalloc(nc); s->r[a] = dalloc(nc); s->e[a] = dalloc(nc);
    s->Pa[a] = dalloc(nc); s->Ph[a] = dalloc(nc); s->elag[a] = dalloc(nc); s->rcf[a] = dalloc(nc);
    s->outv[a] = dalloc(nc); s->sclip[a] = dalloc(nc);
    s->cA[a] = dalloc(nn); s->cMm[a] = dalloc(nn); s->cE[a] = dalloc(nn);
    s->xA[a] = dalloc(nfx); s->xMm[a] = dalloc(nfx); s->xE[a] = dalloc(nfx);
    s->yA[a] = dalloc(nfy); s->yMm[a] = dalloc(nfy); s->yE[a] = dalloc(nfy);
  }
  for (int q = 0; q < MAXM - 1; ++q)
    for (int z = 0; z < 3; ++z) { s->cn[q][z] = dalloc(nc); s->cnY[q][z] = dalloc(nc); }
  s->fdx = dalloc(nn); s->fdy = dalloc(nn);
  s->ncut = (int*)calloc((size_t)nc, sizeof(int));
  s->dom = (int*)calloc((size_t)nc, sizeof(int));
  s->cutmat = (int*)calloc((size_t)nc * MAXM, sizeof(int));
  s->ux = dalloc(nn); s->uy = dalloc(nn); s->pux = dalloc(nn); s->puy = dalloc(nn);
  s->mc = dalloc(nc); s->cc = dalloc(nc); s->Q = dalloc(nc); s->Pi = dalloc(nc);
  s->volh = dalloc(nc); s->vollag = dalloc(nc); s->vcf = dalloc(nc);
  s->ox = dalloc(nc); s->oy = dalloc(nc); s->wx = dalloc(nc); s->wy = dalloc(nc);
  s->uhx = dalloc(nn); s->uhy = dalloc(nn); s->ulx = dalloc(nn); s->uly = dalloc(nn);
  s->ddx = dalloc(nn); s->ddy = dalloc(nn); s->fc = dalloc(nn);
  s->Mpp = dalloc(nn); s->Mpm = dalloc(nn);
  s->mpn = dalloc(nn); s->rux = dalloc(nn); s->ruy = dalloc(nn);
  for (int q = 0; q < 4; ++q)
    for (int z = 0; z < 3; ++z) s->dual[q][z] = dalloc(nn);
  s->fx = dalloc(nfx); s->fxlo = dalloc(nfx); s->fxhi = dalloc(nfx); s->fxb = dalloc(nfx);
  s->fy = dalloc(nfy); s->fylo = dalloc(nfy); s->fyhi = dalloc(nfy); s->fyb = dalloc(nfy);
  s->MX = dalloc(nfx); s->MY = dalloc(nfy);
  return s;
}

void orc_destroy(orc* s) {
  if (!s) return;
  for (int a = 0; a < MAXM; ++a) {
    free(s->k[a]); free(s->r[a]); free(s->e[a]); free(s->Pa[a]); free(s->Ph[a]);
    free(s->elag[a]); free(s->rcf[a]); free(s->outv[a]); free(s->sclip[a]);
    free(s->cA[a]); free(s->cMm[a]); free(s->cE[a]);
    free(s->xA[a]); free(s->xMm[a]); free(s->xE[a]);
    free(s->yA[a]); free(s->yMm[a]); free(s->yE[a]);
  }
  for (int q = 0; q < MAXM - 1; ++q)
    for (int z = 0; z < 3; ++z) { free(s->cn[q][z]); free(s->cnY[q][z]); }
  free(s->fdx); free(s->fdy);
  free(s->ncut); free(s->dom); free(s->cutmat);
  free(s->ux); free(s->uy); free(s->pux); free(s->puy);
  free(s->mc); free(s->cc); free(s->Q); free(s->Pi); free(s->volh); free(s->vollag); free(s->vcf);
  free(s->ox); free(s->oy); free(s->wx); free(s->wy);
  free(s->uhx); free(s->uhy); free(s->ulx); free(s->uly); free(s->ddx); free(s->ddy); free(s->fc);
  free(s->Mpp); free(s->Mpm);
  free(s->mpn); free(s->rux); free(s->ruy);
  for (int q = 0; q < 4; ++q)
    for (int z = 0; z < 3; ++z) free(s->dual[q][z]);
  free(s->fx); free(s->fxlo); free(s->fxhi); free(s->fxb);
  free(s->fy); free(s->fylo); free(s->fyhi); free(s->fyb);
  free(s->MX); free(s->MY);
  free(s);
}

/* Normal velocity vanishes on reflective walls (free slip). */
static void apply_walls(orc* s, double* ax, double* ay) {
  if (!s->perx)
    for (int j = 0; j <= s->ny; ++j) { ax[NI(s, 0, j)] = 0.0; ax[NI(s, s->nx, j)] = 0.0; }
  if (!s->pery)
    for (int i = 0; i <= s->nx; ++i) { ay[NI(s, i, 0)] = 0.0; ay[NI(s, i, s->ny)] = 0.0; }
}

int orc_init(orc* s, const double* k, const double* rho, const double* p,
             const double* ux, const double* uy) {
  int nx = s->nx, ny = s->ny, M = s->M;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      long src = (long)j * nx + i;
      double sum = 0.0;
      for (int a = 0; a < M; ++a) {
        double ka = k[(long)a * nx * ny + src];
        if (!(ka >= -1e-12 && ka <= 1.0 + 1e-12)) return -1;
        sum += ka;
      }
      if (!(fabs(sum - 1.0) <= 1e-9)) return -1;
      double kept = 0.0;
      for (int a = 0; a < M; ++a) {
        double ka = k[(long)a * nx * ny + src];
        if (ka > EPS_K) kept += ka;
      }
      for (int a = 0; a < M; ++a) {
        double ka = k[(long)a * nx * ny + src];
        int c = CI(s, i, j);
        if (ka > EPS_K) {
          double ra = rho[(long)a * nx * ny + src], pa = p[(long)a * nx * ny + src];
          if (!(ra > 0.0)) return -1;
          s->k[a][c] = ka / kept;
          s->r[a][c] = ra;
          s->e[a][c] = (pa + s->pin[a]) / ((s->gam[a] - 1.0) * ra);
        } else {
          s->k[a][c] = 0.0; s->r[a][c] = 0.0; s->e[a][c] = 0.0;
        }
      }
    }
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      s->ux[NI(s, i, j)] = ux[(long)j * (nx + 1) + i];
      s->uy[NI(s, i, j)] = uy[(long)j * (nx + 1) + i];
    }
  apply_walls(s, s->ux, s->uy);
  s->t = 0.0;
  s->lastdt = 0.0;
  s->inited = 1;
  return 0;
}

int orc_set_prescribed(orc* s, const double* ux, const double* uy) {
  if (!ux || !uy) { s->presc = 0; return 0; }
  for (int j = 0; j <= s->ny; ++j)
    for (int i = 0; i <= s->nx; ++i) {
      s->pux[NI(s, i, j)] = ux[(long)j * (s->nx + 1) + i];
      s->puy[NI(s, i, j)] = uy[(long)j * (s->nx + 1) + i];
    }
  s->presc = 1;
  return 0;
}

int orc_set_remap_velocity(orc* s, const double* ux, const double* uy) {
  if (!ux || !uy) { s->ruse = 0; return 0; }
  for (int j = 0; j <= s->ny; ++j)
    for (int i = 0; i <= s->nx; ++i) {
      s->rux[NI(s, i, j)] = ux[(long)j * (s->nx + 1) + i];
      s->ruy[NI(s, i, j)] = uy[(long)j * (s->nx + 1) + i];
    }
  s->ruse = 1;
  return 0;
}

double orc_time(const orc* s) { return s->t; }

/* Fill ghosts of the state, then the pointwise cell quantities at t^n over the
 * whole ghosted array: material mass, cell mass, material pressure, sound
 * speed (reading: c_c = max_a min(1, k_a/EPS_C) c_a). */
static int state_derived(orc* s) {
  for (int a = 0; a < s->M; ++a) { fill_cell(s, s->k[a]); fill_cell(s, s->r[a]); fill_cell(s, s->e[a]); }
  fill_node_vec(s, s->ux, s->uy);
  int bad = 0;
  for (int j = -G; j < s->ny + G; ++j)
    for (int i = -G; i < s->nx + G; ++i) {
      int c = CI(s, i, j);
      double m = 0.0, cmax = 0.0;
      for (int a = 0; a < s->M; ++a) {
        double ka = s->k[a][c];
        if (ka > 0.0) {
          double ra = s->r[a][c];
          double pa = eos_p(s->gam[a], s->pin[a], ra, s->e[a][c]);
          double c2 = eos_c2(s->gam[a], s->pin[a], ra, pa);
          double w = ka / EPS_C < 1.0 ? ka / EPS_C : 1.0;
          if (w >= 1.0 && !(c2 > 0.0)) bad = 1;
          double ca = sqrt(c2 > 0.0 ? c2 : 0.0);
          s->Pa[a][c] = pa;
          if (w * ca > cmax) cmax = w * ca;
          m += ra * ka * s->V;
        } else {
          s->Pa[a][c] = 0.0;
        }
      }
      s->mc[c] = m;
      s->cc[c] = cmax;
    }
  return bad ? -3 : 0;
}

/* CFL time step (annex definition CFL = dt c / dx):
 * dt = CFL * min_c min(dx,dy) / (c_c + max_{p in c} |u_p|), capped at t_end. */
static double cfl_dt(orc* s) {
  double h = s->dx < s->dy ? s->dx : s->dy;
  double best = 1e300;
  for (int j = 0; j < s->ny; ++j)
    for (int i = 0; i < s->nx; ++i) {
      double um = 0.0;
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          int n = NI(s, i + a, j + b);
          double u = sqrt(s->ux[n] * s->ux[n] + s->uy[n] * s->uy[n]);
          if (u > um) um = u;
        }
      double v = h / (s->cc[CI(s, i, j)] + um);
      if (v < best) best = v;
    }
  return s->c.cfl * best;
}

/* -------------------------------------------------------- Lagrange phase */
/* Section 1.2 predictor and corrector, with the iso-deformation
 * multi-material form of section 4.1. */
static int lagrange(orc* s, double dt) {
  int nx = s->nx, ny = s->ny, M = s->M;
  double dx = s->dx, dy = s->dy, V = s->V;
  double L = sqrt(dx * dy), hdt = 0.5 * dt;
  /* pseudo-viscosity Q^n: Q = rho (a1 L c |div u| + a2 L^2 (div u)^2) if
   * div u < 0, with div u from the cell's four node velocities. */
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      int c = CI(s, i, j);
      int ll = NI(s, i, j), lr = NI(s, i + 1, j), ul = NI(s, i, j + 1), ur = NI(s, i + 1, j + 1);
      double div = ((s->ux[lr] + s->ux[ur]) - (s->ux[ll] + s->ux[ul])) / (2.0 * dx)
                 + ((s->uy[ul] + s->uy[ur]) - (s->uy[ll] + s->uy[lr])) / (2.0 * dy);
      double rc = s->mc[c] / V;
      s->Q[c] = div < 0.0 ? rc * (s->c.a1 * L * s->cc[c] * fabs(div) + s->c.a2 * L * L * div * div) : 0.0;
    }
  fill_cell(s, s->Q);
  /* predictor: x^{n+1/2} = x^n + dt/2 u^n, Vol^{n+1/2} = F(x^{n+1/2}),
   * rho_a^{n+1/2} = m_a / (k_a Vol^{n+1/2}),
   * e_a^{n+1/2} = e_a - (P_a + Q)(1/rho_a^{n+1/2} - 1/rho_a),
   * P_a^{n+1/2} = EOS, P^{n+1/2} = sum_a k_a P_a^{n+1/2}. */
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      int c = CI(s, i, j);
      int ll = NI(s, i, j), lr = NI(s, i + 1, j), ul = NI(s, i, j + 1), ur = NI(s, i + 1, j + 1);
      double vol = cell_volume(hdt * s->ux[ll], hdt * s->uy[ll],
                               dx + hdt * s->ux[lr], hdt * s->uy[lr],
                               hdt * s->ux[ul], dy + hdt * s->uy[ul],
                               dx + hdt * s->ux[ur], dy + hdt * s->uy[ur]);
      if (!(vol > 0.0)) return -3;
      s->volh[c] = vol;
      double P = 0.0;
      for (int a = 0; a < M; ++a) {
        double ka = s->k[a][c];
        if (ka > 0.0) {
          double ra = s->r[a][c];
          double rh = ra * V / vol;
          double eh = s->e[a][c] - (s->Pa[a][c] + s->Q[c]) * (1.0 / rh - 1.0 / ra);
          double ph = eos_p(s->gam[a], s->pin[a], rh, eh);
          s->Ph[a][c] = ph;
          P += ka * ph;
        } else {
          s->Ph[a][c] = 0.0;
        }
      }
      s->Pi[c] = P + s->Q[c];
    }
  fill_cell(s, s->Pi);
  /* nodal velocity: u^{n+1/2} = u^n - dt/2 grad(P+Q)_p / rho_p, gradient from
   * the four surrounding cells over 2dx, 2dy; rho_p = (1/4 sum m_c)/(dx dy). */
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      if (!node_interior(i, nx, s->perx) || !node_interior(j, ny, s->pery)) continue;
      int n = NI(s, i, j);
      if (s->presc) {
        s->uhx[n] = s->pux[n]; s->uhy[n] = s->puy[n];
        /* test hook: the node field the dual remap carries */
        s->ulx[n] = s->ruse ? s->rux[n] : s->pux[n];
        s->uly[n] = s->ruse ? s->ruy[n] : s->puy[n];
        continue;
      }
      int A = CI(s, i - 1, j - 1), B = CI(s, i, j - 1), C = CI(s, i - 1, j), D = CI(s, i, j);
      double gx = ((s->Pi[B] + s->Pi[D]) - (s->Pi[A] + s->Pi[C])) / (2.0 * dx);
      double gy = ((s->Pi[C] + s->Pi[D]) - (s->Pi[A] + s->Pi[B])) / (2.0 * dy);
      double mp = 0.25 * (s->mc[A] + s->mc[B] + s->mc[C] + s->mc[D]);
      double rp = mp / V;
      s->uhx[n] = s->ux[n] - hdt * gx / rp;
      s->uhy[n] = s->uy[n] - hdt * gy / rp;
    }
  apply_walls(s, s->uhx, s->uhy);
  if (!s->presc)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i <= nx; ++i) {
        int n = NI(s, i, j);
        s->ulx[n] = 2.0 * s->uhx[n] - s->ux[n];
        s->uly[n] = 2.0 * s->uhy[n] - s->uy[n];
      }
  apply_walls(s, s->ulx, s->uly);
  fill_node_vec(s, s->uhx, s->uhy);
  fill_node_vec(s, s->ulx, s->uly);
  /* corrector: x^{lag} = x^n + dt u^{n+1/2}, Vol^{lag} = F(x^{lag}),
   * e_a^{lag} = e_a - (P_a^{n+1/2} + Q)(1/rho_a^{lag} - 1/rho_a). */
  for (int j = -G; j <= ny + G; ++j)
    for (int i = -G; i <= nx + G; ++i) {
      int n = NI(s, i, j);
      s->ddx[n] = dt * s->uhx[n];
      s->ddy[n] = dt * s->uhy[n];
    }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      int c = CI(s, i, j);
      int ll = NI(s, i, j), lr = NI(s, i + 1, j), ul = NI(s, i, j + 1), ur = NI(s, i + 1, j + 1);
      double vol = cell_volume(s->ddx[ll], s->ddy[ll], dx + s->ddx[lr], s->ddy[lr],
                               s->ddx[ul], dy + s->ddy[ul], dx + s->ddx[ur], dy + s->ddy[ur]);
      if (!(vol > 0.0)) return -3;
      s->vollag[c] = vol;
      for (int a = 0; a < M; ++a) {
        if (s->k[a][c] > 0.0) {
          double ra = s->r[a][c];
          double rl = ra * V / vol;
          s->elag[a][c] = s->e[a][c] - (s->Ph[a][c] + s->Q[c]) * (1.0 / rl - 1.0 / ra);
        } else {
          s->elag[a][c] = 0.0;
        }
      }
    }
  for (int a = 0; a < M; ++a) fill_cell(s, s->elag[a]);
  return 0;
}

/* ----------------------------------------------------------- remap phase */
/* Face volume fluxes of section 2.3.  X-face (i,j) joins nodes p-=(i,j) and
 * p+=(i,j+1); in the face frame (face at x=0, p- at y=0):
 *   y- = max(0, dy_{p-}),  y+ = dy + min(0, dy_{p+}),
 *   x(y) = signed x-displacement of the straight Lagrangian face through
 *          (dx_{p-}, dy_{p-}) and (dx_{p+}, Dy + dy_{p+}),
 *   dVol = 1/2 (x(y-) + x(y+)) (y+ - y-),  > 0 towards +x.
 * The flux region is the rectangle [0, xbar] x [y-, y+], xbar = dVol/(y+-y-)
 * (the rectangular approximation of the trapezoid).  Y-faces swap x and y. */
static int face_fluxes(orc* s) {
  int nx = s->nx, ny = s->ny;
  double dx = s->dx, dy = s->dy;
  int nxu = s->perx ? nx : nx + 1, nyu = s->pery ? ny : ny + 1;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nxu; ++i) {
      int pm = NI(s, i, j), pp = NI(s, i, j + 1);
      double ax = s->ddx[pm], ay = s->ddy[pm], bx = s->ddx[pp], by = dy + s->ddy[pp];
      double ylo = ay > 0.0 ? ay : 0.0;
      double yhi = dy + (s->ddy[pp] < 0.0 ? s->ddy[pp] : 0.0);
      if (!(yhi > ylo)) return -3;
      double xlo = ax + (bx - ax) * (ylo - ay) / (by - ay);
      double xhi = ax + (bx - ax) * (yhi - ay) / (by - ay);
      double xb = 0.5 * (xlo + xhi);
      int f = XI(s, i, j);
      s->fx[f] = xb * (yhi - ylo);
      s->fxb[f] = xb; s->fxlo[f] = ylo; s->fxhi[f] = yhi;
    }
  for (int j = 0; j < nyu; ++j)
    for (int i = 0; i < nx; ++i) {
      int pm = NI(s, i, j), pp = NI(s, i + 1, j);
      double ax = s->ddx[pm], ay = s->ddy[pm], bx = dx + s->ddx[pp], by = s->ddy[pp];
      double xlo = ax > 0.0 ? ax : 0.0;
      double xhi = dx + (s->ddx[pp] < 0.0 ? s->ddx[pp] : 0.0);
      if (!(xhi > xlo)) return -3;
      double ylo = ay + (by - ay) * (xlo - ax) / (bx - ax);
      double yhi = ay + (by - ay) * (xhi - ax) / (bx - ax);
      double yb = 0.5 * (ylo + yhi);
      int f = YI(s, i, j);
      s->fy[f] = yb * (xhi - xlo);
      s->fyb[f] = yb; s->fylo[f] = xlo; s->fyhi[f] = xhi;
    }
  /* corner volume flux dVol_p = |dx_p dy_p| (section 2.3) */
  for (int j = 0; j < nyu; ++j)
    for (int i = 0; i < nxu; ++i) {
      int n = NI(s, i, j);
      s->fc[n] = fabs(s->ddx[n] * s->ddy[n]);
    }
  fill_xface(s, s->fx);
  fill_yface(s, s->fy);
  fill_node_scalar(s, s->fc);
  return 0;
}

/* Face volume fluxes of the Direct and AD remaps (sections 2.1 and 2.2):
 * the face moves with the mean of its two nodes' velocities, so an X face
 * sweeps the rectangle dVol = u_f.e_x dt dy = 1/2 (dx_{p-} + dx_{p+}) dy,
 * region [0, xbar] x [0, dy] in the face frame (> 0 towards +x); Y faces
 * likewise.  dirs: 1 = X faces, 2 = Y faces, 3 = both; the faces of a
 * direction not in dirs carry no flux.  There are no corner fluxes. */
static void face_fluxes_rect(orc* s, int dirs) {
  int nx = s->nx, ny = s->ny;
  double dx = s->dx, dy = s->dy;
  int nxu = s->perx ? nx : nx + 1, nyu = s->pery ? ny : ny + 1;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nxu; ++i) {
      int f = XI(s, i, j);
      double xb = (dirs & 1) ? 0.5 * (s->ddx[NI(s, i, j)] + s->ddx[NI(s, i, j + 1)]) : 0.0;
      s->fx[f] = xb * dy;
      s->fxb[f] = xb; s->fxlo[f] = 0.0; s->fxhi[f] = dy;
    }
  for (int j = 0; j < nyu; ++j)
    for (int i = 0; i < nx; ++i) {
      int f = YI(s, i, j);
      double yb = (dirs & 2) ? 0.5 * (s->ddy[NI(s, i, j)] + s->ddy[NI(s, i + 1, j)]) : 0.0;
      s->fy[f] = yb * dx;
      s->fyb[f] = yb; s->fylo[f] = 0.0; s->fyhi[f] = dx;
    }
  for (int j = 0; j < nyu; ++j)
    for (int i = 0; i < nxu; ++i) s->fc[NI(s, i, j)] = 0.0;
  fill_xface(s, s->fx);
  fill_yface(s, s->fy);
  fill_node_scalar(s, s->fc);
}

/* Corner donor table of section 3.3 (upwind corner value).  For node (i,j)
 * with displacement (dx,dy): dx>0,dy>0 -> donor (i-1,j-1), receiver (i,j);
 * dx<0,dy<0 -> donor (i,j), receiver (i-1,j-1); dx>0,dy<0 -> donor (i-1,j),
 * receiver (i,j-1); dx<0,dy>0 -> donor (i,j-1), receiver (i-1,j).
 * Returns 0 when there is no corner flux (dx or dy is zero). */
static int corner_cells(double ddx, double ddy, int i, int j, int* di, int* dj, int* ri, int* rj) {
  if (ddx > 0.0 && ddy > 0.0) { *di = i - 1; *dj = j - 1; *ri = i; *rj = j; return 1; }
  if (ddx < 0.0 && ddy < 0.0) { *di = i; *dj = j; *ri = i - 1; *rj = j - 1; return 1; }
  if (ddx > 0.0 && ddy < 0.0) { *di = i - 1; *dj = j; *ri = i; *rj = j - 1; return 1; }
  if (ddx < 0.0 && ddy > 0.0) { *di = i; *dj = j - 1; *ri = i - 1; *rj = j; return 1; }
  return 0;
}

/* Flux-consistent Lagrangian volume (section 2.3): each flux has a donor and a
 * receiver; Vol^{lagCF} = dx dy - (volume the cell receives) + (volume it
 * donates), so that the remapped volume is exactly dx dy.  Also the
 * Lagrangian rectangle of every cell: the rectangle through the midpoints of
 * its four Lagrangian faces (section 4.4), stored as centre offset (ox, oy)
 * from the Eulerian centre and widths (wx, wy). */
static int lagcf_volume(orc* s) {
  int nx = s->nx, ny = s->ny;
  double dx = s->dx, dy = s->dy;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double v = s->V + s->fx[XI(s, i + 1, j)] - s->fx[XI(s, i, j)]
                      + s->fy[YI(s, i, j + 1)] - s->fy[YI(s, i, j)];
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          int n = NI(s, i + a, j + b);
          int di, dj, ri, rj;
          if (!corner_cells(s->ddx[n], s->ddy[n], i + a, j + b, &di, &dj, &ri, &rj)) continue;
          if (di == i && dj == j) v += s->fc[n];
          if (ri == i && rj == j) v -= s->fc[n];
        }
      if (!(v > 0.0)) return -3;
      s->vcf[CI(s, i, j)] = v;
    }
  fill_cell(s, s->vcf);
  /* every cell of the ghosted array has its four nodes in the node array, and
   * the ghost node displacements already carry the boundary condition */
  for (int j = -G; j < ny + G; ++j)
    for (int i = -G; i < nx + G; ++i) {
      int c = CI(s, i, j);
      int ll = NI(s, i, j), lr = NI(s, i + 1, j), ul = NI(s, i, j + 1), ur = NI(s, i + 1, j + 1);
      double xl = 0.5 * (s->ddx[ll] + s->ddx[ul]), xr = dx + 0.5 * (s->ddx[lr] + s->ddx[ur]);
      double yb = 0.5 * (s->ddy[ll] + s->ddy[lr]), yt = dy + 0.5 * (s->ddy[ul] + s->ddy[ur]);
      s->ox[c] = 0.5 * (xl + xr) - 0.5 * dx;
      s->oy[c] = 0.5 * (yb + yt) - 0.5 * dy;
      s->wx[c] = xr - xl;
      s->wy[c] = yt - yb;
    }
  /* rho_a^{lagCF} = rho_a Vol^n / Vol^{lagCF}, e_a^{lagCF} = e_a^{lag} */
  for (int a = 0; a < s->M; ++a) {
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int c = CI(s, i, j);
        s->rcf[a][c] = s->k[a][c] > 0.0 ? s->r[a][c] * s->V / s->vcf[c] : 0.0;
      }
    fill_cell(s, s->rcf[a]);
  }
  return 0;
}

/* Interface placement (sections 4.1 and 4.4) for every mixed cell: Youngs
 * normal n_a = -grad k_a / |grad k_a| (outward from material a; reading: a
 * occupies {x.n_a <= d_a}) with the 9-point weights (1,2,1)/(8 dx),
 * (1,2,1)/(8 dy); zero gradient -> n = (1,0).  The line is placed in the
 * rectangular Lagrangian cell so that the material's area fraction there is
 * k_a^n.  Three materials (reading; the paper treats two): nested
 * dissection in material index order, each present material except the last
 * cut from what the previous cuts left, the last one taking the remainder. */
static void interfaces_in(orc* s, int rect, double* (*cn)[3]);
static void interfaces(orc* s) {
  if (s->c.remap == ORC_REMAP_DIRECT) {
    /* Direct remap (section 4.3): the interface i^n displaced along X with
     * its normal kept, placed so that k_a^n holds in the X-Lagrangian cell
     * [xl, xr] x [0, dy], cuts the X-face fluxes; i^n displaced along Y
     * (the Y-Lagrangian cell [0, dx] x [yb, yt]) cuts the Y-face fluxes. */
    interfaces_in(s, 1, s->cn);
    interfaces_in(s, 2, s->cnY);
  } else {
    interfaces_in(s, 0, s->cn);
  }
}
/* rect: 0 the Lagrangian rectangle, 1 its X extent by dy, 2 dx by its Y extent. */
static void interfaces_in(orc* s, int rect, double* (*cn)[3]) {
  int nx = s->nx, ny = s->ny, M = s->M;
  double dx = s->dx, dy = s->dy;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      int c = CI(s, i, j);
      int np = 0;
      int best = 0;
      for (int a = 0; a < M; ++a) {
        if (s->k[a][c] > 0.0) s->cutmat[(long)c * MAXM + np++] = a;
        if (s->k[a][c] > s->k[best][c]) best = a;
      }
      s->dom[c] = best;
      s->ncut[c] = np - 1;
      if (np < 2) continue;
      double xl = 0.5 * dx - 0.5 * s->wx[c] + s->ox[c] ;
      double xr = xl + s->wx[c];
      double yb = 0.5 * dy - 0.5 * s->wy[c] + s->oy[c];
      double yt = yb + s->wy[c];
      /* the rectangle is kept as centre offset and widths (wx, wy); its
       * area is the product of the widths (xr - xl would re-round wx) */
      double area = s->wx[c] * s->wy[c];
      if (rect == 1) { yb = 0.0; yt = dy; area = s->wx[c] * dy; }
      if (rect == 2) { xl = 0.0; xr = dx; area = dx * s->wy[c]; }
      double poly[2 * MAXV];
      rect_poly(xl, xr, yb, yt, poly);
      int nv = 4;
      for (int q = 0; q < np - 1; ++q) {
        int a = s->cutmat[(long)c * MAXM + q];
        double* K = s->k[a];
        double gx = ((K[CI(s, i + 1, j + 1)] + 2.0 * K[CI(s, i + 1, j)] + K[CI(s, i + 1, j - 1)])
                   - (K[CI(s, i - 1, j + 1)] + 2.0 * K[CI(s, i - 1, j)] + K[CI(s, i - 1, j - 1)])) / (8.0 * dx);
        double gy = ((K[CI(s, i + 1, j + 1)] + 2.0 * K[CI(s, i, j + 1)] + K[CI(s, i - 1, j + 1)])
                   - (K[CI(s, i + 1, j - 1)] + 2.0 * K[CI(s, i, j - 1)] + K[CI(s, i - 1, j - 1)])) / (8.0 * dy);
        double g = sqrt(gx * gx + gy * gy);
        double nxv = 1.0, nyv = 0.0;
        if (g > 0.0) { nxv = -gx / g; nyv = -gy / g; }
        double target = K[c] * area;
        double rem = poly_area(poly, nv);
        if (target > rem) target = rem;
        double d = plic_solve(poly, nv, nxv, nyv, target);
        cn[q][0][c] = nxv; cn[q][1][c] = nyv; cn[q][2][c] = d;
        double tmp[2 * MAXV];
        int m = clip_poly(poly, nv, nxv, nyv, d, -1, tmp);
        memcpy(poly, tmp, sizeof(double) * 2 * m);
        nv = m;
      }
    }
  fill_cell_int(s, s->ncut);
  fill_cell_int(s, s->dom);
}

/* Material split of one flux region (a rectangle in the donor's frame) by the
 * donor's interface lines: each cut material takes its part of what the
 * previous cuts left; the last present material takes the rest. */
static void split_region(orc* s, double* (*cn)[3], int c, double x0, double x1, double y0, double y1, double vol,
                         double* A) {
  for (int a = 0; a < MAXM; ++a) A[a] = 0.0;
  int nc = s->ncut[c];
  if (nc == 0) {
    for (int a = 0; a < s->M; ++a) if (s->k[a][c] > 0.0) A[a] = vol;
    return;
  }
  double poly[2 * MAXV], tmp[2 * MAXV];
  rect_poly(x0, x1, y0, y1, poly);
  int nv = 4;
  double used = 0.0;
  for (int q = 0; q < nc; ++q) {
    int a = s->cutmat[(long)c * MAXM + q];
    double nxv = cn[q][0][c], nyv = cn[q][1][c], d = cn[q][2][c];
    double part = nv >= 3 ? halfplane_area(poly, nv, nxv, nyv, d) : 0.0;
    A[a] = part;
    used += part;
    int m = nv >= 3 ? clip_poly(poly, nv, nxv, nyv, d, -1, tmp) : 0;
    memcpy(poly, tmp, sizeof(double) * 2 * m);
    nv = m;
  }
  int last = s->cutmat[(long)c * MAXM + nc];
  double rest = vol - used;
  A[last] = rest > 0.0 ? rest : 0.0;
}

/* Flux regions in the donor's frame (origin at the donor's Eulerian
 * lower-left node). */
static void xface_region(orc* s, int f, int donor_left, double* r) {
  double xb = s->fxb[f];
  if (donor_left) { r[0] = s->dx; r[1] = s->dx + xb; } else { r[0] = xb; r[1] = 0.0; }
  r[2] = s->fxlo[f]; r[3] = s->fxhi[f];
}
static void yface_region(orc* s, int f, int donor_below, double* r) {
  double yb = s->fyb[f];
  r[0] = s->fylo[f]; r[1] = s->fyhi[f];
  if (donor_below) { r[2] = s->dy; r[3] = s->dy + yb; } else { r[2] = yb; r[3] = 0.0; }
}
static void corner_region(orc* s, double ddx, double ddy, double* r) {
  /* the node sits at the donor's corner that points along (ddx,ddy) */
  double nxp = ddx > 0.0 ? s->dx : 0.0, nyp = ddy > 0.0 ? s->dy : 0.0;
  if (ddx > 0.0) { r[0] = nxp; r[1] = nxp + ddx; } else { r[0] = nxp + ddx; r[1] = nxp; }
  if (ddy > 0.0) { r[2] = nyp; r[3] = nyp + ddy; } else { r[2] = nyp + ddy; r[3] = nyp; }
}

static int wrapx(orc* s, int i) { return s->perx ? ((i % s->nx) + s->nx) % s->nx : i; }
static int wrapy(orc* s, int j) { return s->pery ? ((j % s->ny) + s->ny) % s->ny : j; }

/* Reconstructed value of a cell quantity q at a face (section 2.1.1):
 * a_f = a_d + delta_d/2 (sgn(dVol) dx_d^{lag} - dt u_f), with the Van Leer
 * slope over the Lagrangian centres of d-1, d, d+1 along the face normal,
 * dx_d^{lag} the donor rectangle width and dt u_f the mean displacement of
 * the face's two nodes. */
static double recon_face(orc* s, const double* q, int ci, int cj, int dirx, double sg, double fdisp) {
  int c = CI(s, ci, cj);
  int cm = dirx ? CI(s, ci - 1, cj) : CI(s, ci, cj - 1);
  int cp = dirx ? CI(s, ci + 1, cj) : CI(s, ci, cj + 1);
  double h = dirx ? s->dx : s->dy;
  const double* o = dirx ? s->ox : s->oy;
  const double* w = dirx ? s->wx : s->wy;
  double dp = (q[cp] - q[c]) / (h + o[cp] - o[c]);
  double dm = (q[c] - q[cm]) / (h + o[c] - o[cm]);
  double sl = vanleer(dm, dp);
  return q[c] + 0.5 * sl * (sg * w[c] - fdisp);
}
/* Diagonal limited reconstruction at a corner (section 3.3): along
 * v = (dx,dy)/|.| if ddx*ddy > 0, else v_perp = (dx,-dy)/|.|; slopes over the
 * Lagrangian centres of the donor's two diagonal neighbours; evaluated at
 * 1/2 (sgn(ddx) (wx, +-wy) - (ddx, ddy)) . w from the donor's centre. */
static double recon_corner(orc* s, const double* q, int ci, int cj, double ddx, double ddy) {
  double dx = s->dx, dy = s->dy, D = sqrt(dx * dx + dy * dy);
  int c = CI(s, ci, cj);
  double sy = (ddx * ddy > 0.0) ? 1.0 : -1.0; /* +1: v, -1: v_perp */
  int sj = sy > 0.0 ? 1 : -1;
  int cp = CI(s, ci + 1, cj + sj), cm = CI(s, ci - 1, cj - sj);
  double sp = ((dx + s->ox[cp] - s->ox[c]) * dx + (sy * dy + s->oy[cp] - s->oy[c]) * sy * dy) / D;
  double sm = ((dx + s->ox[c] - s->ox[cm]) * dx + (sy * dy + s->oy[c] - s->oy[cm]) * sy * dy) / D;
  double dp = (q[cp] - q[c]) / sp;
  double dm = (q[c] - q[cm]) / sm;
  double sl = vanleer(dm, dp);
  double sgx = ddx > 0.0 ? 1.0 : -1.0;
  double off = 0.5 * (sgx * (s->wx[c] * dx + s->wy[c] * dy) - (ddx * dx + sy * ddy * dy)) / D;
  return q[c] + sl * off;
}
static int pure_in(orc* s, int a, int ci, int cj) { return s->k[a][CI(s, ci, cj)] == 1.0; }

/* Van Leer limited slopes of q in cell (ci,cj) (section 2.1.1 and the
 * diagonal form of section 3.3): along x and y over the Lagrangian centres
 * of the two neighbours, along v = (dx,dy)/|.| and v_perp = (dx,-dy)/|.|
 * over the diagonal neighbours' Lagrangian centres projected on v, v_perp. */
static double slope_axis(orc* s, const double* q, int ci, int cj, int dirx) {
  int c = CI(s, ci, cj);
  int cm = dirx ? CI(s, ci - 1, cj) : CI(s, ci, cj - 1);
  int cp = dirx ? CI(s, ci + 1, cj) : CI(s, ci, cj + 1);
  double h = dirx ? s->dx : s->dy;
  const double* o = dirx ? s->ox : s->oy;
  return vanleer((q[c] - q[cm]) / (h + o[c] - o[cm]), (q[cp] - q[c]) / (h + o[cp] - o[c]));
}
static double slope_diag(orc* s, const double* q, int ci, int cj, int pp) {
  double dx = s->dx, dy = s->dy, D = sqrt(dx * dx + dy * dy);
  int c = CI(s, ci, cj);
  double sy = pp ? 1.0 : -1.0;
  int sj = pp ? 1 : -1;
  int cp = CI(s, ci + 1, cj + sj), cm = CI(s, ci - 1, cj - sj);
  double sp = ((dx + s->ox[cp] - s->ox[c]) * dx + (sy * dy + s->oy[cp] - s->oy[c]) * sy * dy) / D;
  double sm = ((dx + s->ox[c] - s->ox[cm]) * dx + (sy * dy + s->oy[c] - s->oy[cm]) * sy * dy) / D;
  return vanleer((q[c] - q[cm]) / sm, (q[cp] - q[c]) / sp);
}

/* x-y corner value (section 3.3): a_c + delta_x/2 (sgn(dVol_fx) dx_c^{lag}
 * - dt u_fx) + delta_y/2 (sgn(dVol_fy) dy_c^{lag} - dt u_fy), with f_x the
 * donor's X face on the side of the corner (in the donor's row), f_y its Y
 * face on that side (in its column); sgn(0) = 0. */
static double recon_corner_xy(orc* s, const double* q, int di, int dj, double ddx, double ddy) {
  int c = CI(s, di, dj);
  int fxi = di + (ddx > 0.0 ? 1 : 0), fyj = dj + (ddy > 0.0 ? 1 : 0);
  double vx = s->fx[XI(s, fxi, dj)], vy = s->fy[YI(s, di, fyj)];
  double sgx = vx > 0.0 ? 1.0 : vx < 0.0 ? -1.0 : 0.0;
  double sgy = vy > 0.0 ? 1.0 : vy < 0.0 ? -1.0 : 0.0;
  double fdx = 0.5 * (s->ddx[NI(s, fxi, dj)] + s->ddx[NI(s, fxi, dj + 1)]);
  double fdy = 0.5 * (s->ddy[NI(s, di, fyj)] + s->ddy[NI(s, di + 1, fyj)]);
  return q[c] + 0.5 * slope_axis(s, q, di, dj, 1) * (sgx * s->wx[c] - fdx)
              + 0.5 * slope_axis(s, q, di, dj, 0) * (sgy * s->wy[c] - fdy);
}

/* Multidimensional value (section 3.3): the plane a_c + G.(x - x_c) whose
 * cell means best fit the 9-point stencil in least squares, G solving the
 * normal equations (X^T X) G = X^T A with rows X = x_kl^{lag} - x_c^{lag}
 * (the Lagrangian rectangles' centres; a rectangle's mean of x - x_c is its
 * centre's offset) and A = a_kl - a_c; the gradient is scaled to the norm
 * min(|delta_x|, |delta_y|, |delta_v|, |delta_vperp|) of the limited 1D
 * slopes (direction kept) and evaluated at (px, py) in the donor's frame
 * (origin at its Eulerian lower-left node). */
static double recon_lsq(orc* s, const double* q, int di, int dj, double px, double py) {
  int c = CI(s, di, dj);
  double sxx = 0.0, sxy = 0.0, syy = 0.0, sxa = 0.0, sya = 0.0;
  for (int l = -1; l <= 1; ++l)
    for (int k = -1; k <= 1; ++k) {
      if (k == 0 && l == 0) continue;
      int n = CI(s, di + k, dj + l);
      double X1 = k * s->dx + s->ox[n] - s->ox[c];
      double X2 = l * s->dy + s->oy[n] - s->oy[c];
      double A = q[n] - q[c];
      sxx += X1 * X1; sxy += X1 * X2; syy += X2 * X2; sxa += X1 * A; sya += X2 * A;
    }
  double det = sxx * syy - sxy * sxy;
  double g1 = (syy * sxa - sxy * sya) / det;
  double g2 = (sxx * sya - sxy * sxa) / det;
  double gn = sqrt(g1 * g1 + g2 * g2);
  if (!(gn > 0.0)) return q[c];
  double m = fabs(slope_axis(s, q, di, dj, 1));
  double t = fabs(slope_axis(s, q, di, dj, 0)); if (t < m) m = t;
  t = fabs(slope_diag(s, q, di, dj, 1)); if (t < m) m = t;
  t = fabs(slope_diag(s, q, di, dj, 0)); if (t < m) m = t;
  double phi = m / gn;
  double cx = 0.5 * s->dx + s->ox[c], cy = 0.5 * s->dy + s->oy[c];
  return q[c] + phi * (g1 * (px - cx) + g2 * (py - cy));
}
static int pure_stencil(orc* s, int a, int di, int dj) {
  for (int l = -1; l <= 1; ++l)
    for (int k = -1; k <= 1; ++k)
      if (!pure_in(s, a, di + k, dj + l)) return 0;
  return 1;
}

/* For one flux: final material volumes after clipping, then mass and energy
 * fluxes from the reconstructed rho_a^{lagCF} and e_a^{lag}.
 * kind: 0 X-face, 1 Y-face, 2 corner.  Order 2 is used for material a only
 * when the donor and its two neighbours along the reconstruction direction
 * are pure in a (section 4.2 remark: order 1 next to interfaces). */
static void finish_flux(orc* s, int kind, int di, int dj, double sg, double fdisp,
                        double ddx, double ddy, const double* reg, const double* Araw,
                        double* Aout, double* Mout, double* Eout) {
  int c = CI(s, di, dj), M = s->M;
  double A[MAXM];
  for (int a = 0; a < M; ++a) A[a] = Araw[a];
  if (s->ncut[c] > 0) {
    double moved = 0.0;
    for (int a = 0; a < M; ++a) {
      double sc = s->sclip[a][c];
      if (sc < 1.0) { moved += (1.0 - sc) * A[a]; A[a] *= sc; }
    }
    A[s->dom[c]] += moved;
  }
  for (int a = 0; a < M; ++a) {
    Aout[a] = A[a]; Mout[a] = 0.0; Eout[a] = 0.0;
    if (!(A[a] > 0.0)) { Aout[a] = 0.0; continue; }
    double rf = s->rcf[a][c], ef = s->elag[a][c];
    int cr = s->c.corner_recon;
    int lsq = cr == ORC_CORNER_LSQ && (kind == 2 || s->c.face_order == 2);
    int o2 = 0;
    if (lsq)
      o2 = pure_stencil(s, a, di, dj);
    else if (kind == 0 && s->c.face_order == 2)
      o2 = pure_in(s, a, di - 1, dj) && pure_in(s, a, di, dj) && pure_in(s, a, di + 1, dj);
    else if (kind == 1 && s->c.face_order == 2)
      o2 = pure_in(s, a, di, dj - 1) && pure_in(s, a, di, dj) && pure_in(s, a, di, dj + 1);
    else if (kind == 2 && cr == ORC_CORNER_DIAG) {
      int sj = ddx * ddy > 0.0 ? 1 : -1;
      o2 = pure_in(s, a, di - 1, dj - sj) && pure_in(s, a, di, dj) && pure_in(s, a, di + 1, dj + sj);
    } else if (kind == 2 && cr == ORC_CORNER_AVG) {
      /* the donor and the receiver (the cell diagonally across the node) */
      o2 = pure_in(s, a, di, dj) && pure_in(s, a, di + (ddx > 0.0 ? 1 : -1), dj + (ddy > 0.0 ? 1 : -1));
    } else if (kind == 2 && cr == ORC_CORNER_XY) {
      o2 = pure_in(s, a, di - 1, dj) && pure_in(s, a, di, dj) && pure_in(s, a, di + 1, dj)
        && pure_in(s, a, di, dj - 1) && pure_in(s, a, di, dj + 1);
    }
    if (o2) {
      if (lsq) {
        double px = 0.5 * (reg[0] + reg[1]), py = 0.5 * (reg[2] + reg[3]);
        rf = recon_lsq(s, s->rcf[a], di, dj, px, py);
        ef = recon_lsq(s, s->elag[a], di, dj, px, py);
      } else if (kind == 2 && cr == ORC_CORNER_AVG) {
        /* 1/2 (a_donor + a_receiver), clamped to the donor value (section
         * 3.3: no negative donor mass) */
        int rc = CI(s, di + (ddx > 0.0 ? 1 : -1), dj + (ddy > 0.0 ? 1 : -1));
        double ra = 0.5 * (s->rcf[a][c] + s->rcf[a][rc]), ea = 0.5 * (s->elag[a][c] + s->elag[a][rc]);
        rf = ra < rf ? ra : rf;
        ef = ea < ef ? ea : ef;
      } else if (kind == 2 && cr == ORC_CORNER_XY) {
        rf = recon_corner_xy(s, s->rcf[a], di, dj, ddx, ddy);
        ef = recon_corner_xy(s, s->elag[a], di, dj, ddx, ddy);
      } else if (kind == 2) {
        rf = recon_corner(s, s->rcf[a], di, dj, ddx, ddy);
        ef = recon_corner(s, s->elag[a], di, dj, ddx, ddy);
      } else {
        rf = recon_face(s, s->rcf[a], di, dj, kind == 0, sg, fdisp);
        ef = recon_face(s, s->elag[a], di, dj, kind == 0, sg, fdisp);
      }
    }
    Mout[a] = rf * A[a];
    Eout[a] = rf * ef * A[a];
  }
}

/* Raw material split of every flux, the clipping factors per donor, then the
 * final per-material volume, mass and energy of every flux.
 * Clipping (reading; the paper is silent): if the outgoing volume of
 * material a from a mixed donor exceeds k_a Vol^{lagCF}, a's outgoing parts
 * are scaled down to fit and the removed volume is given, in the same
 * fluxes, to the donor's dominant material (largest k, lowest index). */
static void material_fluxes(orc* s) {
  int nx = s->nx, ny = s->ny, M = s->M;
  int nxu = s->perx ? nx : nx + 1, nyu = s->pery ? ny : ny + 1;
  long nfx = (long)s->xw * s->xh, nfy = (long)s->yw * s->yh, nn = (long)s->nw * s->nh;
  double* rawx[MAXM]; double* rawy[MAXM]; double* rawc[MAXM];
  for (int a = 0; a < MAXM; ++a) { rawx[a] = dalloc(nfx); rawy[a] = dalloc(nfy); rawc[a] = dalloc(nn); }
  for (int a = 0; a < M; ++a)
    for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) s->outv[a][CI(s, i, j)] = 0.0;
  double A[MAXM], r[4];
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nxu; ++i) {
      int f = XI(s, i, j);
      double v = s->fx[f];
      if (v == 0.0) continue;
      int left = v > 0.0;
      int di = wrapx(s, left ? i - 1 : i), dj = j;
      xface_region(s, f, left, r);
      split_region(s, s->cn, CI(s, di, dj), r[0], r[1], r[2], r[3], fabs(v), A);
      for (int a = 0; a < M; ++a) { rawx[a][f] = A[a]; s->outv[a][CI(s, di, dj)] += A[a]; }
    }
  for (int j = 0; j < nyu; ++j)
    for (int i = 0; i < nx; ++i) {
      int f = YI(s, i, j);
      double v = s->fy[f];
      if (v == 0.0) continue;
      int below = v > 0.0;
      int di = i, dj = wrapy(s, below ? j - 1 : j);
      yface_region(s, f, below, r);
      split_region(s, s->c.remap == ORC_REMAP_DIRECT ? s->cnY : s->cn, CI(s, di, dj), r[0], r[1], r[2], r[3],
                   fabs(v), A);
      for (int a = 0; a < M; ++a) { rawy[a][f] = A[a]; s->outv[a][CI(s, di, dj)] += A[a]; }
    }
  for (int j = 0; j < nyu; ++j)
    for (int i = 0; i < nxu; ++i) {
      int n = NI(s, i, j);
      int di, dj, ri, rj;
      if (s->fc[n] == 0.0 || !corner_cells(s->ddx[n], s->ddy[n], i, j, &di, &dj, &ri, &rj)) continue;
      di = wrapx(s, di); dj = wrapy(s, dj);
      corner_region(s, s->ddx[n], s->ddy[n], r);
      split_region(s, s->cn, CI(s, di, dj), r[0], r[1], r[2], r[3], s->fc[n], A);
      for (int a = 0; a < M; ++a) { rawc[a][n] = A[a]; s->outv[a][CI(s, di, dj)] += A[a]; }
    }
  /* clipping factors */
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      int c = CI(s, i, j);
      for (int a = 0; a < M; ++a) {
        s->sclip[a][c] = 1.0;
        if (s->ncut[c] == 0 || a == s->dom[c]) continue;
        double avail = s->k[a][c] * s->vcf[c];
        if (s->outv[a][c] > avail) s->sclip[a][c] = avail / s->outv[a][c];
      }
    }
  for (int a = 0; a < M; ++a) fill_cell(s, s->sclip[a]);
  /* final fluxes */
  double Ao[MAXM], Mo[MAXM], Eo[MAXM];
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nxu; ++i) {
      int f = XI(s, i, j);
      double v = s->fx[f];
      for (int a = 0; a < M; ++a) { s->xA[a][f] = 0.0; s->xMm[a][f] = 0.0; s->xE[a][f] = 0.0; }
      if (v == 0.0) continue;
      int left = v > 0.0;
      int di = wrapx(s, left ? i - 1 : i);
      for (int a = 0; a < M; ++a) A[a] = rawx[a][f];
      double fd = 0.5 * (s->ddx[NI(s, i, j)] + s->ddx[NI(s, i, j + 1)]);
      xface_region(s, f, left, r);
      finish_flux(s, 0, di, j, left ? 1.0 : -1.0, fd, 0.0, 0.0, r, A, Ao, Mo, Eo);
      double sg = left ? 1.0 : -1.0;
      for (int a = 0; a < M; ++a) { s->xA[a][f] = sg * Ao[a]; s->xMm[a][f] = sg * Mo[a]; s->xE[a][f] = sg * Eo[a]; }
    }
  for (int j = 0; j < nyu; ++j)
    for (int i = 0; i < nx; ++i) {
      int f = YI(s, i, j);
      double v = s->fy[f];
      for (int a = 0; a < M; ++a) { s->yA[a][f] = 0.0; s->yMm[a][f] = 0.0; s->yE[a][f] = 0.0; }
      if (v == 0.0) continue;
      int below = v > 0.0;
      int dj = wrapy(s, below ? j - 1 : j);
      for (int a = 0; a < M; ++a) A[a] = rawy[a][f];
      double fd = 0.5 * (s->ddy[NI(s, i, j)] + s->ddy[NI(s, i + 1, j)]);
      yface_region(s, f, below, r);
      finish_flux(s, 1, i, dj, below ? 1.0 : -1.0, fd, 0.0, 0.0, r, A, Ao, Mo, Eo);
      double sg = below ? 1.0 : -1.0;
      for (int a = 0; a < M; ++a) { s->yA[a][f] = sg * Ao[a]; s->yMm[a][f] = sg * Mo[a]; s->yE[a][f] = sg * Eo[a]; }
    }
  for (int j = 0; j < nyu; ++j)
    for (int i = 0; i < nxu; ++i) {
      int n = NI(s, i, j);
      for (int a = 0; a < M; ++a) { s->cA[a][n] = 0.0; s->cMm[a][n] = 0.0; s->cE[a][n] = 0.0; }
      int di, dj, ri, rj;
      if (s->fc[n] == 0.0 || !corner_cells(s->ddx[n], s->ddy[n], i, j, &di, &dj, &ri, &rj)) continue;
      di = wrapx(s, di); dj = wrapy(s, dj);
      for (int a = 0; a < M; ++a) A[a] = rawc[a][n];
      corner_region(s, s->ddx[n], s->ddy[n], r);
      finish_flux(s, 2, di, dj, 0.0, 0.0, s->ddx[n], s->ddy[n], r, A, Ao, Mo, Eo);
      for (int a = 0; a < M; ++a) { s->cA[a][n] = Ao[a]; s->cMm[a][n] = Mo[a]; s->cE[a][n] = Eo[a]; }
    }
  for (int a = 0; a < M; ++a) {
    fill_xface(s, s->xA[a]); fill_xface(s, s->xMm[a]); fill_xface(s, s->xE[a]);
    fill_yface(s, s->yA[a]); fill_yface(s, s->yMm[a]); fill_yface(s, s->yE[a]);
    fill_node_scalar(s, s->cA[a]); fill_node_scalar(s, s->cMm[a]); fill_node_scalar(s, s->cE[a]);
  }
  for (int a = 0; a < MAXM; ++a) { free(rawx[a]); free(rawy[a]); free(rawc[a]); }
}

/* Cell remap (sections 2.3 and 4.4):
 *   Vol_a^{proj} = k_a Vol^{lagCF} + sum_in dVol_a - sum_out dVol_a,
 *   m_a^{proj}   = m_a + sum_in rho_f dVol_a - sum_out ...,
 *   (me)_a^{proj}= m_a e_a^{lag} + sum_in rho_f e_f dVol_a - sum_out ...,
 *   k_a = Vol_a / sum_b Vol_b, rho_a = m_a / (k_a dx dy), e_a = (me)_a / m_a.
 * Reading: a material whose remapped volume is <= EPS_K dx dy is removed and
 * its mass and energy go to the cell's largest remaining material. */
static int cell_update(orc* s, double** nk, double** nr, double** ne) {
  int nx = s->nx, ny = s->ny, M = s->M;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      int c = CI(s, i, j);
      double vol[MAXM], mas[MAXM], ene[MAXM];
      for (int a = 0; a < M; ++a) {
        double ka = s->k[a][c];
        double m = s->r[a][c] * ka * s->V;
        vol[a] = ka * s->vcf[c];
        mas[a] = m;
        ene[a] = m * s->elag[a][c];
        int fl = XI(s, i, j), fr = XI(s, i + 1, j), fb = YI(s, i, j), ft = YI(s, i, j + 1);
        vol[a] += s->xA[a][fl] - s->xA[a][fr] + s->yA[a][fb] - s->yA[a][ft];
        mas[a] += s->xMm[a][fl] - s->xMm[a][fr] + s->yMm[a][fb] - s->yMm[a][ft];
        ene[a] += s->xE[a][fl] - s->xE[a][fr] + s->yE[a][fb] - s->yE[a][ft];
        for (int b = 0; b < 2; ++b)
          for (int q = 0; q < 2; ++q) {
            int n = NI(s, i + q, j + b);
            int di, dj, ri, rj;
            if (s->fc[n] == 0.0 || !corner_cells(s->ddx[n], s->ddy[n], i + q, j + b, &di, &dj, &ri, &rj)) continue;
            if (ri == i && rj == j) { vol[a] += s->cA[a][n]; mas[a] += s->cMm[a][n]; ene[a] += s->cE[a][n]; }
            if (di == i && dj == j) { vol[a] -= s->cA[a][n]; mas[a] -= s->cMm[a][n]; ene[a] -= s->cE[a][n]; }
          }
      }
      int keep[MAXM], big = -1;
      double tot = 0.0, lost_m = 0.0, lost_e = 0.0;
      for (int a = 0; a < M; ++a) {
        keep[a] = vol[a] > EPS_K * s->V;
        if (keep[a]) { tot += vol[a]; if (big < 0 || vol[a] > vol[big]) big = a; }
        else { lost_m += mas[a]; lost_e += ene[a]; }
      }
      if (big < 0) return -3;
      mas[big] += lost_m;
      ene[big] += lost_e;
      for (int a = 0; a < M; ++a) {
        if (!keep[a]) { nk[a][c] = 0.0; nr[a][c] = 0.0; ne[a][c] = 0.0; continue; }
        double ka = vol[a] / tot;
        if (!(mas[a] > 0.0)) return -3;
        nk[a][c] = ka;
        nr[a][c] = mas[a] / (ka * s->V);
        ne[a][c] = ene[a] / mas[a];
      }
    }
  return 0;
}

/* Dual-mesh momentum remap (sections 2.1.1 and 2.3).  Dual X-face between
 * nodes (i,j),(i+1,j): 1/4 of the four primary X-face mass fluxes that bound
 * cells (i,j-1) and (i,j); dual Y-face likewise.  Dual corner at the centre
 * of cell (i,j): 1/4 of the corner mass fluxes of the cell's four nodes that
 * run along that diagonal (++ joins nodes (i,j),(i+1,j+1); +- joins
 * (i,j+1),(i+1,j)).  m_p = 1/4 sum of the four cell masses,
 * m_p' = m_p + sum of signed dual fluxes, m_p' u_p' = m_p u_p^{lag} +
 * sum of signed dual fluxes times the reconstructed u^{lag}.  The dual
 * reconstruction repeats the primary one with the nodes as centres: Van
 * Leer over node Lagrangian positions, dual width dx + dt (u_{q+1}-u_{q-1})/2,
 * dual face displacement the mean of its two nodes', dual corner
 * displacement the mean of the cell's four nodes'. */
static double recon_dual_face(orc* s, const double* u, int qi, int qj, int dirx, double sg, double fdisp, int o2) {
  int q = NI(s, qi, qj);
  if (!o2) return u[q];
  int qm = dirx ? NI(s, qi - 1, qj) : NI(s, qi, qj - 1);
  int qp = dirx ? NI(s, qi + 1, qj) : NI(s, qi, qj + 1);
  double h = dirx ? s->dx : s->dy;
  const double* d = dirx ? s->ddx : s->ddy;
  double dp = (u[qp] - u[q]) / (h + d[qp] - d[q]);
  double dm = (u[q] - u[qm]) / (h + d[q] - d[qm]);
  double w = h + 0.5 * (d[qp] - d[qm]);
  return u[q] + 0.5 * vanleer(dm, dp) * (sg * w - fdisp);
}
static double recon_dual_corner(orc* s, const double* u, int qi, int qj, int diag_pp, double sg,
                                double cdx, double cdy, int o2) {
  int q = NI(s, qi, qj);
  if (!o2) return u[q];
  double dx = s->dx, dy = s->dy, D = sqrt(dx * dx + dy * dy);
  double sy = diag_pp ? 1.0 : -1.0;
  int sj = diag_pp ? 1 : -1;
  int qp = NI(s, qi + 1, qj + sj), qm = NI(s, qi - 1, qj - sj);
  double sp = ((dx + s->ddx[qp] - s->ddx[q]) * dx + (sy * dy + s->ddy[qp] - s->ddy[q]) * sy * dy) / D;
  double sm = ((dx + s->ddx[q] - s->ddx[qm]) * dx + (sy * dy + s->ddy[q] - s->ddy[qm]) * sy * dy) / D;
  double dp = (u[qp] - u[q]) / sp, dm = (u[q] - u[qm]) / sm;
  double wxq = dx + 0.5 * (s->ddx[NI(s, qi + 1, qj)] - s->ddx[NI(s, qi - 1, qj)]);
  double wyq = dy + 0.5 * (s->ddy[NI(s, qi, qj + 1)] - s->ddy[NI(s, qi, qj - 1)]);
  double off = 0.5 * (sg * (wxq * dx + wyq * dy) - (cdx * dx + sy * cdy * dy)) / D;
  return u[q] + vanleer(dm, dp) * off;
}

static void dual_remap(orc* s, double* nux, double* nuy) {
  int nx = s->nx, ny = s->ny, M = s->M;
  int nxu = s->perx ? nx : nx + 1, nyu = s->pery ? ny : ny + 1;
  /* total primary mass fluxes */
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nxu; ++i) {
      int f = XI(s, i, j); double m = 0.0;
      for (int a = 0; a < M; ++a) m += s->xMm[a][f];
      s->MX[f] = m;
    }
  for (int j = 0; j < nyu; ++j)
    for (int i = 0; i < nx; ++i) {
      int f = YI(s, i, j); double m = 0.0;
      for (int a = 0; a < M; ++a) m += s->yMm[a][f];
      s->MY[f] = m;
    }
  for (int j = 0; j < nyu; ++j)
    for (int i = 0; i < nxu; ++i) {
      int n = NI(s, i, j); double m = 0.0;
      for (int a = 0; a < M; ++a) m += s->cMm[a][n];
      double ddx = s->ddx[n], ddy = s->ddy[n];
      double sg = ddx > 0.0 ? m : -m;   /* signed along +x */
      s->Mpp[n] = (ddx * ddy > 0.0) ? sg : 0.0;
      s->Mpm[n] = (ddx * ddy < 0.0) ? sg : 0.0;
    }
  fill_xface(s, s->MX);
  fill_yface(s, s->MY);
  fill_corner(s, s->Mpp, s->Mpm);
  /* the dual mesh reconstructs corners along the diagonal for every
   * second-order corner choice (reading: section 3.3 defines the variants
   * for the cell-centred variables only) */
  int fo2 = s->c.face_order == 2, co2 = s->c.corner_recon != ORC_CORNER_UPWIND;
  long nn = (long)s->nw * s->nh;
  for (long v = 0; v < nn; ++v) {
    s->mpn[v] = 0.0;
    for (int q = 0; q < 4; ++q)
      for (int z = 0; z < 3; ++z) s->dual[q][z][v] = 0.0;
  }
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      if (!node_interior(i, nx, s->perx) || !node_interior(j, ny, s->pery)) continue;
      int p = NI(s, i, j);
      if (s->presc && !s->ruse) { nux[p] = s->pux[p]; nuy[p] = s->puy[p]; continue; }
      double mp = 0.25 * (s->mc[CI(s, i - 1, j - 1)] + s->mc[CI(s, i, j - 1)]
                        + s->mc[CI(s, i - 1, j)] + s->mc[CI(s, i, j)]);
      double mnew = mp, px = mp * s->ulx[p], py = mp * s->uly[p];
      /* dual X-faces: right (tail p), left (head p) */
      for (int side = 0; side < 2; ++side) {
        int fi = side == 0 ? i : i - 1;   /* dual face between nodes fi, fi+1 */
        double D = 0.25 * (s->MX[XI(s, fi, j - 1)] + s->MX[XI(s, fi + 1, j - 1)]
                         + s->MX[XI(s, fi, j)] + s->MX[XI(s, fi + 1, j)]);
        if (D == 0.0) continue;
        int qi = D > 0.0 ? fi : fi + 1;
        double fd = 0.5 * (s->ddx[NI(s, fi, j)] + s->ddx[NI(s, fi + 1, j)]);
        double sg = D > 0.0 ? 1.0 : -1.0;
        double vx = recon_dual_face(s, s->ulx, qi, j, 1, sg, fd, fo2);
        double vy = recon_dual_face(s, s->uly, qi, j, 1, sg, fd, fo2);
        double sgn = side == 0 ? -1.0 : 1.0;
        mnew += sgn * D; px += sgn * D * vx; py += sgn * D * vy;
        if (side == 0) { s->dual[0][0][p] = D; s->dual[0][1][p] = D * vx; s->dual[0][2][p] = D * vy; }
      }
      /* dual Y-faces: top (tail p), bottom (head p) */
      for (int side = 0; side < 2; ++side) {
        int fj = side == 0 ? j : j - 1;
        double D = 0.25 * (s->MY[YI(s, i - 1, fj)] + s->MY[YI(s, i - 1, fj + 1)]
                         + s->MY[YI(s, i, fj)] + s->MY[YI(s, i, fj + 1)]);
        if (D == 0.0) continue;
        int qj = D > 0.0 ? fj : fj + 1;
        double fd = 0.5 * (s->ddy[NI(s, i, fj)] + s->ddy[NI(s, i, fj + 1)]);
        double sg = D > 0.0 ? 1.0 : -1.0;
        double vx = recon_dual_face(s, s->ulx, i, qj, 0, sg, fd, fo2);
        double vy = recon_dual_face(s, s->uly, i, qj, 0, sg, fd, fo2);
        double sgn = side == 0 ? -1.0 : 1.0;
        mnew += sgn * D; px += sgn * D * vx; py += sgn * D * vy;
        if (side == 0) { s->dual[1][0][p] = D; s->dual[1][1][p] = D * vx; s->dual[1][2][p] = D * vy; }
      }
      /* dual corners: ++ at cells (i,j) [tail p] and (i-1,j-1) [head p];
       * +- at cells (i,j-1) [tail p = its upper-left node] and (i-1,j)
       * [head p = its lower-right node] */
      for (int kc = 0; kc < 4; ++kc) {
        int ci, cj, pp, tail;
        if (kc == 0) { ci = i; cj = j; pp = 1; tail = 1; }
        else if (kc == 1) { ci = i - 1; cj = j - 1; pp = 1; tail = 0; }
        else if (kc == 2) { ci = i; cj = j - 1; pp = 0; tail = 1; }
        else { ci = i - 1; cj = j; pp = 0; tail = 0; }
        int n0 = NI(s, ci, cj), n1 = NI(s, ci + 1, cj), n2 = NI(s, ci, cj + 1), n3 = NI(s, ci + 1, cj + 1);
        const double* Mv = pp ? s->Mpp : s->Mpm;
        double D = 0.25 * (Mv[n0] + Mv[n1] + Mv[n2] + Mv[n3]);
        if (D == 0.0) continue;
        int ai, aj, bi, bj;
        if (pp) { ai = ci; aj = cj; bi = ci + 1; bj = cj + 1; }
        else { ai = ci; aj = cj + 1; bi = ci + 1; bj = cj; }
        int qi = D > 0.0 ? ai : bi, qj = D > 0.0 ? aj : bj;
        double cdx = 0.25 * (s->ddx[n0] + s->ddx[n1] + s->ddx[n2] + s->ddx[n3]);
        double cdy = 0.25 * (s->ddy[n0] + s->ddy[n1] + s->ddy[n2] + s->ddy[n3]);
        double sg = D > 0.0 ? 1.0 : -1.0;
        double vx = recon_dual_corner(s, s->ulx, qi, qj, pp, sg, cdx, cdy, co2);
        double vy = recon_dual_corner(s, s->uly, qi, qj, pp, sg, cdx, cdy, co2);
        double sgn = tail ? -1.0 : 1.0;
        mnew += sgn * D; px += sgn * D * vx; py += sgn * D * vy;
        if (tail && cj >= 0) {  /* kept for the test hooks, at the cell's index */
          int o = NI(s, ci, cj), q = pp ? 2 : 3;
          s->dual[q][0][o] = D; s->dual[q][1][o] = D * vx; s->dual[q][2][o] = D * vy;
        }
      }
      s->mpn[p] = mnew;
      if (!(mnew > 0.0)) { nux[p] = NAN; nuy[p] = NAN; continue; }
      nux[p] = px / mnew;
      nuy[p] = py / mnew;
    }
  apply_walls(s, nux, nuy);
}

/* One remap of the state held in s (k, r, elag, ulx/uly, mc) with the
 * displacement in ddx/ddy: fluxes (kind 0 DirectCF faces and corners, 1
 * rectangle X and Y faces, 2 rectangle X faces only, 3 rectangle Y faces
 * only), Lagrangian volume and rectangles, interfaces, material fluxes,
 * cell remap into nk/nr/ne and dual remap into nux/nuy. */
static int remap_once(orc* s, int kind, double** nk, double** nr, double** ne, double* nux, double* nuy) {
  int rc = 0;
  if (kind == 0) rc = face_fluxes(s);
  else face_fluxes_rect(s, kind == 1 ? 3 : kind == 2 ? 1 : 2);
  if (rc) return rc;
  rc = lagcf_volume(s);
  if (rc) return rc;
  interfaces(s);
  material_fluxes(s);
  rc = cell_update(s, nk, nr, ne);
  if (!rc) dual_remap(s, nux, nuy);
  long nn = (long)s->nw * s->nh;
  if (!rc)
    for (long v = 0; v < nn; ++v) if (!(nux[v] == nux[v]) || !(nuy[v] == nuy[v])) rc = -3;
  return rc;
}

/* AD remap (section 2.1, multi-material section 4.3): an X remap with the
 * displacement along X only (the X-Lagrangian cell is the rectangle
 * [xl, xr] x [0, dy]; X-face fluxes u_f.e_x dt dy), whose result
 * (k, rho, e, u and the cell masses; e^{lagy} = e^{projx}, interfaces and
 * normals re-placed from k^{projx}) feeds a Y remap with the displacement
 * along Y only; X-Y on the steps numbered 0, 2, 4, ..., Y-X on the others
 * (section 2.1, remark 3). */
static int remap_ad(orc* s, double** nk, double** nr, double** ne, double* nux, double* nuy) {
  long nn = (long)s->nw * s->nh, nc = (long)s->cw * s->ch;
  memcpy(s->fdx, s->ddx, sizeof(double) * nn);
  memcpy(s->fdy, s->ddy, sizeof(double) * nn);
  int first_x = (s->nsteps % 2) == 0;
  for (int sweep = 0; sweep < 2; ++sweep) {
    int alongx = (sweep == 0) == first_x;
    for (long v = 0; v < nn; ++v) {
      s->ddx[v] = alongx ? s->fdx[v] : 0.0;
      s->ddy[v] = alongx ? 0.0 : s->fdy[v];
    }
    int rc = remap_once(s, alongx ? 2 : 3, nk, nr, ne, nux, nuy);
    if (rc) return rc;
    if (sweep == 1) break;
    /* the X (or Y) remap's result is the next sweep's Lagrangian state */
    for (int a = 0; a < s->M; ++a) {
      memcpy(s->k[a], nk[a], sizeof(double) * nc);
      memcpy(s->r[a], nr[a], sizeof(double) * nc);
      memcpy(s->elag[a], ne[a], sizeof(double) * nc);
      fill_cell(s, s->k[a]); fill_cell(s, s->r[a]); fill_cell(s, s->elag[a]);
    }
    for (int j = -G; j < s->ny + G; ++j)
      for (int i = -G; i < s->nx + G; ++i) {
        int c = CI(s, i, j);
        double m = 0.0;
        for (int a = 0; a < s->M; ++a) if (s->k[a][c] > 0.0) m += s->r[a][c] * s->k[a][c] * s->V;
        s->mc[c] = m;
      }
    memcpy(s->ulx, nux, sizeof(double) * nn);
    memcpy(s->uly, nuy, sizeof(double) * nn);
    apply_walls(s, s->ulx, s->uly);
    fill_node_vec(s, s->ulx, s->uly);
  }
  memcpy(s->ddx, s->fdx, sizeof(double) * nn);
  memcpy(s->ddy, s->fdy, sizeof(double) * nn);
  return 0;
}

int orc_step(orc* s, double t_end, double* dt_out) {
  if (!s->inited) return -5;
  int rc = state_derived(s);
  if (rc) return rc;
  double dt = s->c.dt_fixed > 0.0 ? s->c.dt_fixed : cfl_dt(s);
  if (t_end - s->t < dt) dt = t_end - s->t;
  if (dt_out) *dt_out = dt > 0.0 ? dt : 0.0;
  if (!(dt > 0.0)) return 0;
  s->lastdt = dt;
  rc = lagrange(s, dt);
  if (rc) return rc;
  long nc = (long)s->cw * s->ch, nn = (long)s->nw * s->nh;
  double *nk[MAXM], *nr[MAXM], *ne[MAXM];
  for (int a = 0; a < MAXM; ++a) { nk[a] = dalloc(nc); nr[a] = dalloc(nc); ne[a] = dalloc(nc); }
  double *nux = dalloc(nn), *nuy = dalloc(nn);
  /* the AD sweeps overwrite k, r with the intermediate state: keep t^n's */
  double *k0[MAXM], *r0[MAXM];
  int ad = s->c.remap == ORC_REMAP_AD;
  for (int a = 0; a < MAXM; ++a) { k0[a] = NULL; r0[a] = NULL; }
  if (ad)
    for (int a = 0; a < s->M; ++a) {
      k0[a] = dalloc(nc); r0[a] = dalloc(nc);
      memcpy(k0[a], s->k[a], sizeof(double) * nc); memcpy(r0[a], s->r[a], sizeof(double) * nc);
    }
  if (ad) rc = remap_ad(s, nk, nr, ne, nux, nuy);
  else rc = remap_once(s, s->c.remap == ORC_REMAP_DIRECT ? 1 : 0, nk, nr, ne, nux, nuy);
  if (rc && ad)
    for (int a = 0; a < s->M; ++a) {
      memcpy(s->k[a], k0[a], sizeof(double) * nc); memcpy(s->r[a], r0[a], sizeof(double) * nc);
    }
  if (!rc) {
    for (int a = 0; a < s->M; ++a) {
      double* t;
      t = s->k[a]; s->k[a] = nk[a]; nk[a] = t;
      t = s->r[a]; s->r[a] = nr[a]; nr[a] = t;
      t = s->e[a]; s->e[a] = ne[a]; ne[a] = t;
    }
    double* t;
    t = s->ux; s->ux = nux; nux = t;
    t = s->uy; s->uy = nuy; nuy = t;
    s->t += dt;
    s->nsteps += 1;
  }
  for (int a = 0; a < MAXM; ++a) { free(nk[a]); free(nr[a]); free(ne[a]); free(k0[a]); free(r0[a]); }
  free(nux); free(nuy);
  return rc;
}

long orc_size(const orc* s, int field) {
  long c = (long)s->nx * s->ny, n = (long)(s->nx + 1) * (s->ny + 1);
  switch (field) {
    case ORC_F_K: case ORC_F_RHO_MAT: case ORC_F_E_MAT: case ORC_F_E_LAG: case ORC_F_SCLIP: return c * s->M;
    case ORC_F_P: case ORC_F_RHO: case ORC_F_E: case ORC_F_C: case ORC_F_VOL_LAGCF: case ORC_F_Q: return c;
    case ORC_F_UX: case ORC_F_UY: case ORC_F_UHX: case ORC_F_UHY: case ORC_F_FC: case ORC_F_MC: return n;
    case ORC_F_FX: case ORC_F_MX: return (long)s->ny * (s->nx + 1);
    case ORC_F_FY: case ORC_F_MY: return (long)(s->ny + 1) * s->nx;
    case ORC_F_CONS: return 8;
    case ORC_F_DT: return 1;
    case ORC_F_CUTS: return 6 * c;
    case ORC_F_XA: return (long)s->M * s->ny * (s->nx + 1);
    case ORC_F_YA: return (long)s->M * (s->ny + 1) * s->nx;
    case ORC_F_CA: return (long)s->M * n;
    case ORC_F_MP_NEW: return n;
    case ORC_F_DUAL: return 12 * n;
  }
  return -1;
}

/* Node weight for domain sums: a reflective-wall node's dual cell is half
 * (corner: a quarter) inside the domain. */
static double node_weight(const orc* s, int i, int j) {
  double w = 1.0;
  if (!s->perx && (i == 0 || i == s->nx)) w *= 0.5;
  if (!s->pery && (j == 0 || j == s->ny)) w *= 0.5;
  return w;
}

int orc_get(orc* s, int field, double* out, long n) {
  long need = orc_size(s, field);
  if (need < 0 || n < need) return -1;
  int nx = s->nx, ny = s->ny, M = s->M;
  long cc = (long)nx * ny;
  switch (field) {
    case ORC_F_K: case ORC_F_RHO_MAT: case ORC_F_E_MAT: case ORC_F_E_LAG: case ORC_F_SCLIP:
      for (int a = 0; a < M; ++a)
        for (int j = 0; j < ny; ++j)
          for (int i = 0; i < nx; ++i) {
            int c = CI(s, i, j);
            double v = field == ORC_F_K ? s->k[a][c] : field == ORC_F_RHO_MAT ? s->r[a][c]
                     : field == ORC_F_E_MAT ? s->e[a][c] : field == ORC_F_SCLIP ? s->sclip[a][c]
                     : s->elag[a][c];
            out[a * cc + (long)j * nx + i] = v;
          }
      return 0;
    case ORC_F_P: case ORC_F_RHO: case ORC_F_E: case ORC_F_C:
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          int c = CI(s, i, j);
          double P = 0.0, R = 0.0, me = 0.0, m = 0.0, cmax = 0.0;
          for (int a = 0; a < M; ++a) {
            double ka = s->k[a][c];
            if (!(ka > 0.0)) continue;
            double ra = s->r[a][c], ea = s->e[a][c];
            double pa = eos_p(s->gam[a], s->pin[a], ra, ea);
            double c2 = eos_c2(s->gam[a], s->pin[a], ra, pa);
            double w = ka / EPS_C < 1.0 ? ka / EPS_C : 1.0;
            double ca = sqrt(c2 > 0.0 ? c2 : 0.0);
            if (w * ca > cmax) cmax = w * ca;
            P += ka * pa; R += ka * ra; me += ka * ra * ea; m += ka * ra;
          }
          double v = field == ORC_F_P ? P : field == ORC_F_RHO ? R : field == ORC_F_E ? me / m : cmax;
          out[(long)j * nx + i] = v;
        }
      return 0;
    case ORC_F_UX: case ORC_F_UY: case ORC_F_UHX: case ORC_F_UHY:
      fill_node_vec(s, s->ux, s->uy);
      for (int j = 0; j <= ny; ++j)
        for (int i = 0; i <= nx; ++i) {
          int p = NI(s, i, j);
          double v = field == ORC_F_UX ? s->ux[p] : field == ORC_F_UY ? s->uy[p]
                   : field == ORC_F_UHX ? s->uhx[p] : s->uhy[p];
          out[(long)j * (nx + 1) + i] = v;
        }
      return 0;
    case ORC_F_FC: case ORC_F_MC:
      for (int j = 0; j <= ny; ++j)
        for (int i = 0; i <= nx; ++i) {
          int p = NI(s, i, j);
          double v;
          if (field == ORC_F_FC) v = s->fc[p];
          else { v = 0.0; for (int a = 0; a < M; ++a) v += s->cMm[a][p]; }
          out[(long)j * (nx + 1) + i] = v;
        }
      return 0;
    case ORC_F_MP_NEW: case ORC_F_DUAL: {
      long nnode = (long)(nx + 1) * (ny + 1);
      int nq = field == ORC_F_DUAL ? 12 : 1;
      for (int q = 0; q < nq; ++q)
        for (int j = 0; j <= ny; ++j)
          for (int i = 0; i <= nx; ++i) {
            int p = NI(s, i, j);
            out[q * nnode + (long)j * (nx + 1) + i] = field == ORC_F_MP_NEW ? s->mpn[p] : s->dual[q / 3][q % 3][p];
          }
      return 0;
    }
    case ORC_F_VOL_LAGCF: case ORC_F_Q:
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
          out[(long)j * nx + i] = field == ORC_F_Q ? s->Q[CI(s, i, j)] : s->vcf[CI(s, i, j)];
      return 0;
    case ORC_F_FX: case ORC_F_MX:
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
          int f = XI(s, i, j);
          double v;
          if (field == ORC_F_FX) v = s->fx[f];
          else { v = 0.0; for (int a = 0; a < M; ++a) v += s->xMm[a][f]; }
          out[(long)j * (nx + 1) + i] = v;
        }
      return 0;
    case ORC_F_FY: case ORC_F_MY:
      for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
          int f = YI(s, i, j);
          double v;
          if (field == ORC_F_FY) v = s->fy[f];
          else { v = 0.0; for (int a = 0; a < M; ++a) v += s->yMm[a][f]; }
          out[(long)j * nx + i] = v;
        }
      return 0;
    case ORC_F_DT:
      out[0] = s->lastdt;
      return 0;
    case ORC_F_CUTS:
      for (int z = 0; z < 6; ++z)
        for (int j = 0; j < ny; ++j)
          for (int i = 0; i < nx; ++i) {
            int c = CI(s, i, j), q = z / 3;
            out[z * cc + (long)j * nx + i] = (q < s->ncut[c] && q < MAXM - 1) ? s->cn[q][z % 3][c] : 0.0;
          }
      return 0;
    case ORC_F_XA:
      for (int a = 0; a < M; ++a)
        for (int j = 0; j < ny; ++j)
          for (int i = 0; i <= nx; ++i)
            out[(long)a * ny * (nx + 1) + (long)j * (nx + 1) + i] = s->xA[a][XI(s, i, j)];
      return 0;
    case ORC_F_YA:
      for (int a = 0; a < M; ++a)
        for (int j = 0; j <= ny; ++j)
          for (int i = 0; i < nx; ++i)
            out[(long)a * (ny + 1) * nx + (long)j * nx + i] = s->yA[a][YI(s, i, j)];
      return 0;
    case ORC_F_CA:
      for (int a = 0; a < M; ++a)
        for (int j = 0; j <= ny; ++j)
          for (int i = 0; i <= nx; ++i)
            out[(long)a * (ny + 1) * (nx + 1) + (long)j * (nx + 1) + i] = s->cA[a][NI(s, i, j)];
      return 0;
    case ORC_F_CONS: {
      double ma[MAXM] = {0, 0, 0}, mt = 0.0, ei = 0.0, px = 0.0, py = 0.0, ek = 0.0;
      for (int a = 0; a < M; ++a) { fill_cell(s, s->k[a]); fill_cell(s, s->r[a]); fill_cell(s, s->e[a]); }
      fill_node_vec(s, s->ux, s->uy);
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          int c = CI(s, i, j);
          for (int a = 0; a < M; ++a) {
            double m = s->r[a][c] * s->k[a][c] * s->V;
            ma[a] += m; mt += m; ei += m * s->e[a][c];
          }
        }
      int nxu = s->perx ? nx : nx + 1, nyu = s->pery ? ny : ny + 1;
      for (int j = 0; j < nyu; ++j)
        for (int i = 0; i < nxu; ++i) {
          double mp = 0.0;
          for (int b = -1; b <= 0; ++b)
            for (int a2 = -1; a2 <= 0; ++a2) {
              int c = CI(s, i + a2, j + b);
              for (int a = 0; a < M; ++a) mp += 0.25 * s->r[a][c] * s->k[a][c] * s->V;
            }
          double w = node_weight(s, i, j) * mp;
          int p = NI(s, i, j);
          px += w * s->ux[p]; py += w * s->uy[p];
          ek += 0.5 * w * (s->ux[p] * s->ux[p] + s->uy[p] * s->uy[p]);
        }
      out[0] = ma[0]; out[1] = ma[1]; out[2] = ma[2];
      out[3] = mt; out[4] = px; out[5] = py; out[6] = ei; out[7] = ei + ek;
      return 0;
    }
  }
  return -1;
}
