/*
 * lr_oracle.h -- plain FP64 CPU reference ("oracle") of one time step of the
 * staggered Lagrange-Remap scheme with the one-step "Direct with Corner
 * Fluxes" (DirectCF) remap and VOF/PLIC sharp-interface material fluxes
 * (Chaudet, arXiv 2208.13409).
 *
 * TEST INFRASTRUCTURE.  Only tests/, the smoke check and the CPU-baseline leg
 * of bench.py may load this library.  It shares no code, header or constant
 * table with the CUDA library under paper_2208_13409_gb300/ and include/.
 *
 * Conventions (oracle side): cells (i,j), 0<=i<nx, 0<=j<ny, arrays [j][i];
 * nodes (i,j), 0<=i<=nx, 0<=j<=ny, arrays [(ny+1)][(nx+1)]; per-material
 * arrays are [nmat][ny][nx].  All floating point is IEEE double, compiled
 * with -ffp-contract=off.
 */
#ifndef LR_ORACLE_H
#define LR_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_REFLECT = 0, ORC_BC_PERIODIC = 1 };
/* Corner reconstruction (section 3.3): upwind, diagonal limited linear,
 * diagonal average (clamped to the donor value), x-y limited linear, and
 * multidimensional least-squares plane (which also gives the face values). */
enum { ORC_CORNER_UPWIND = 0, ORC_CORNER_DIAG = 1, ORC_CORNER_AVG = 2, ORC_CORNER_XY = 3, ORC_CORNER_LSQ = 4 };
/* Remap of the step: one-step with corner fluxes (section 2.3), one-step
 * with face fluxes only ("Direct", section 2.2), or alternate directions
 * ("AD", section 2.1: an X remap then a Y remap, the order swapped every
 * other step). */
enum { ORC_REMAP_DIRECTCF = 0, ORC_REMAP_DIRECT = 1, ORC_REMAP_AD = 2 };

typedef struct {
  int nx, ny;
  double x0, x1, y0, y1;
  int nmat;              /* 1..3 */
  double cfl, a1, a2;    /* CFL number, linear / quadratic pseudo-viscosity */
  int bc[4];             /* xlo, xhi, ylo, yhi; xlo==xhi and ylo==yhi required */
  int face_order;        /* 1 (upwind) or 2 (Van Leer limited linear) */
  int corner_recon;      /* ORC_CORNER_* */
  double dt_fixed;       /* >0: use this dt instead of the CFL rule */
  int remap;             /* ORC_REMAP_* */
} orc_config;

typedef struct orc orc;

/* Field identifiers for orc_get (same numbering as the product's enum). */
enum {
  ORC_F_K = 0,        /* [nmat][ny][nx] volume fractions */
  ORC_F_RHO_MAT = 1,  /* [nmat][ny][nx] material densities (0 where absent) */
  ORC_F_E_MAT = 2,    /* [nmat][ny][nx] material specific internal energies */
  ORC_F_P = 3,        /* [ny][nx] mixture pressure sum_a k_a P_a */
  ORC_F_RHO = 4,      /* [ny][nx] mixture density sum_a k_a rho_a */
  ORC_F_E = 5,        /* [ny][nx] mixture specific internal energy */
  ORC_F_UX = 6,       /* [(ny+1)][(nx+1)] node velocity x */
  ORC_F_UY = 7,       /* [(ny+1)][(nx+1)] node velocity y */
  ORC_F_CONS = 8,     /* [8]: mass_a (3 slots), mass, mom_x, mom_y, E_int, E_tot */
  ORC_F_C = 9,        /* [ny][nx] cell sound speed used by the CFL rule */
  /* intermediates of the last step (debug / per-phase checks) */
  ORC_F_UHX = 20,     /* [(ny+1)][(nx+1)] u^{n+1/2} x */
  ORC_F_UHY = 21,
  ORC_F_VOL_LAGCF = 22, /* [ny][nx] flux-consistent Lagrangian volume */
  ORC_F_E_LAG = 23,   /* [nmat][ny][nx] e_a^{n+1,lag} */
  ORC_F_FX = 24,      /* [ny][nx+1] X-face volume flux, + towards +x */
  ORC_F_FY = 25,      /* [ny+1][nx] Y-face volume flux, + towards +y */
  ORC_F_FC = 26,      /* [(ny+1)][(nx+1)] corner volume flux |dx dy| */
  ORC_F_MX = 27,      /* [ny][nx+1] X-face mass flux (all materials), signed */
  ORC_F_MY = 28,      /* [ny+1][nx] Y-face mass flux, signed */
  ORC_F_MC = 29,      /* [(ny+1)][(nx+1)] corner mass flux magnitude */
  ORC_F_Q = 30,       /* [ny][nx] pseudo-viscosity Q^n */
  ORC_F_DT = 31,      /* [1] last dt */
  ORC_F_CUTS = 32,    /* [6][ny][nx] interface lines of mixed cells: n0x, n0y, d0, n1x, n1y, d1 */
  ORC_F_XA = 33,      /* [nmat][ny][nx+1] per-material X-face volume flux, signed */
  ORC_F_YA = 34,      /* [nmat][ny+1][nx] per-material Y-face volume flux, signed */
  ORC_F_CA = 35,      /* [nmat][(ny+1)][(nx+1)] per-material corner volume flux */
  ORC_F_SCLIP = 37,   /* [nmat][ny][nx] factor on material a's outgoing volume
                         in the last step (1 unless clipped to what it holds) */
  ORC_F_MP_NEW = 38,  /* [(ny+1)][(nx+1)] remapped nodal mass m_p' of the last
                         step: m_p plus the signed dual mass fluxes (sections
                         2.1.1, 2.3); 0 at nodes the dual remap skipped */
  ORC_F_DUAL = 39     /* [4][3][(ny+1)][(nx+1)] dual fluxes of the last step:
                         kind 0 the dual X face between nodes (i,j),(i+1,j),
                         1 the dual Y face between (i,j),(i,j+1), 2 the ++
                         and 3 the +- dual corner at the centre of cell (i,j);
                         per kind the mass flux (signed along +x, or +y for
                         the Y face) and the x and y momentum fluxes (mass
                         flux times the upwind reconstructed velocity) */
};

orc* orc_create(const orc_config* cfg, const double* gamma, const double* pinf);
void orc_destroy(orc* s);
/* k, rho, p: [nmat][ny][nx]; ux, uy: [(ny+1)][(nx+1)].  Returns 0 or <0. */
int orc_init(orc* s, const double* k, const double* rho, const double* p,
             const double* ux, const double* uy);
/* Prescribed node velocity (re-imposed every step), NULL to clear. */
int orc_set_prescribed(orc* s, const double* ux, const double* uy);
/* Test hook for the dual remap (only with a prescribed velocity set): the
 * flux geometry still follows the prescribed velocity, but the dual remap
 * runs and carries this node field ([(ny+1)][(nx+1)] each) as u^{lag}
 * instead of the prescribed one.  NULL, NULL clears it. */
int orc_set_remap_velocity(orc* s, const double* ux, const double* uy);
/* One step, dt capped so that t does not pass t_end.  Returns 0 or <0. */
int orc_step(orc* s, double t_end, double* dt_out);
int orc_get(orc* s, int field, double* out, long n);
double orc_time(const orc* s);
long orc_size(const orc* s, int field);

/* Stand-alone geometric / constitutive pieces, exposed so the tests can pin
 * them one by one against closed forms. */
double orc_t_cell_volume(const double* xy8);          /* ll, lr, ul, ur */
double orc_t_vanleer(double dm, double dp);           /* limited slope */
double orc_t_halfplane_area(const double* poly, int nv, double nx, double ny,
                            double d);                /* area(poly & {x.n<=d}) */
double orc_t_plic(const double* poly, int nv, double nx, double ny,
                  double target);                     /* d: area = target */
void orc_t_eos(double gamma, double pinf, double rho, double e, double* p,
               double* c2);

#ifdef __cplusplus
}
#endif
#endif
