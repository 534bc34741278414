// lr_api.cu -- the C ABI of include/lr.h: context, device arena, launches,
// CUDA graphs for lr_run, field read-back and kernel timing.
#include "../../include/lr.h"
#include "lr_dev.cuh"
#include "lr_host.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <vector>

struct lr_ctx {
  lr_config cfg;
  LrGrid g;
  LrState st[2];
  int cur;
  LrWork w;
  char* arena;
  size_t arena_bytes;
  bool own_arena;
  cudaStream_t stream;
  bool own_stream;
  cudaStream_t aux;            // the interface kernels run here, beside lr_cell_cf and lr_mat_flux
  cudaEvent_t ev_fork, ev_cf, ev_join, ev_mf, ev_dual;
  bool have_mats, inited;
  int sticky;
  char msg[512];
  cudaGraphExec_t gexec[2];
  bool gvalid[2];
  bool prof;
  bool tiled;       // the tiled (fused, shared-memory) kernels replace kernel pairs of the step
  struct Pend { int kid; cudaEvent_t a, b; };
  std::vector<Pend> pend;
  double acc_ms[LRK_COUNT + 5];  // per kernel, then the tiled kernels and the interface-line placement
  long acc_n[LRK_COUNT + 5];
  double* tmp;      // device scratch for field views (max field size)
  size_t tmp_elems;
  double* rows;     // device scratch for conservation partial sums
};

// ---------------------------------------- shared with the batch API (lr_host.h)
bool lr_config_ok(const lr_config* c, char* why, size_t nwhy) {
  if (!c) { snprintf(why, nwhy, "null config"); return false; }
  if (c->nx < 2 || c->ny < 2) { snprintf(why, nwhy, "nx, ny must be >= 2"); return false; }
  if ((double)c->nx * (double)c->ny > (double)(1 << 28)) { snprintf(why, nwhy, "nx*ny above 2^28"); return false; }
  if (c->nmat < 1 || c->nmat > LR_MAXM) { snprintf(why, nwhy, "nmat must be 1..3"); return false; }
  if (!(c->x1 > c->x0) || !(c->y1 > c->y0)) { snprintf(why, nwhy, "empty domain"); return false; }
  if (c->bc[0] != c->bc[1] || c->bc[2] != c->bc[3]) { snprintf(why, nwhy, "bc[0]==bc[1] and bc[2]==bc[3] required"); return false; }
  for (int q = 0; q < 4; ++q)
    if (c->bc[q] != LR_BC_REFLECT && c->bc[q] != LR_BC_PERIODIC) { snprintf(why, nwhy, "bad bc"); return false; }
  if ((c->bc[0] == LR_BC_PERIODIC && c->nx < 3) || (c->bc[2] == LR_BC_PERIODIC && c->ny < 3)) {
    snprintf(why, nwhy, "a periodic direction needs at least 3 cells");
    return false;
  }
  if (!(c->cfl > 0.0) || c->cfl > 1.0) { snprintf(why, nwhy, "cfl must be in (0,1]"); return false; }
  if (c->a1 < 0.0 || c->a2 < 0.0) { snprintf(why, nwhy, "negative viscosity coefficient"); return false; }
  if (c->face_order != 1 && c->face_order != 2) { snprintf(why, nwhy, "face_order must be 1 or 2"); return false; }
  if (c->corner_recon < LR_CORNER_UPWIND || c->corner_recon > LR_CORNER_LSQ) { snprintf(why, nwhy, "bad corner_recon"); return false; }
  if (c->precision != LR_FP64 && c->precision != LR_DF64 && c->precision != LR_FP32) {
    snprintf(why, nwhy, "precision must be LR_FP64, LR_DF64 or LR_FP32");
    return false;
  }
  if (c->dt_fixed < 0.0) { snprintf(why, nwhy, "dt_fixed < 0"); return false; }
  if (c->remap != LR_REMAP_DIRECTCF && c->remap != LR_REMAP_DIRECT && c->remap != LR_REMAP_AD) {
    snprintf(why, nwhy, "remap must be LR_REMAP_DIRECTCF, LR_REMAP_DIRECT or LR_REMAP_AD");
    return false;
  }
  if (c->mixed_lanes != 0 && c->mixed_lanes != 1 && c->mixed_lanes != 2 && c->mixed_lanes != 4 &&
      c->mixed_lanes != 8) {
    snprintf(why, nwhy, "mixed_lanes must be 0, 1, 2, 4 or 8");
    return false;
  }
  return true;
}

void lr_fill_grid(const lr_config& f, LrGrid& g) {
  g.nx = f.nx; g.ny = f.ny; g.M = f.nmat;
  g.perx = f.bc[0] == LR_BC_PERIODIC;
  g.pery = f.bc[2] == LR_BC_PERIODIC;
  g.nxu = g.perx ? g.nx : g.nx + 1;
  g.nyu = g.pery ? g.ny : g.ny + 1;
  g.dx = (f.x1 - f.x0) / f.nx;
  g.dy = (f.y1 - f.y0) / f.ny;
  g.V = g.dx * g.dy;
  g.L = sqrt(g.dx * g.dy);
  g.hmin = g.dx < g.dy ? g.dx : g.dy;
  g.D = sqrt(g.dx * g.dx + g.dy * g.dy);
  g.inv2dx = 1.0 / (2.0 * g.dx);
  g.inv2dy = 1.0 / (2.0 * g.dy);
  g.inv8dx = 1.0 / (8.0 * g.dx);
  g.inv8dy = 1.0 / (8.0 * g.dy);
  g.invV = 1.0 / g.V;
  g.invD = 1.0 / g.D;
  g.cfl = f.cfl; g.a1 = f.a1; g.a2 = f.a2; g.dt_fixed = f.dt_fixed;
  g.face_o2 = f.face_order == 2;
  // the dual mesh reconstructs corners along the diagonal for every
  // second-order corner choice
  g.corner_o2 = f.corner_recon != LR_CORNER_UPWIND;
  g.corner_kind = f.corner_recon;
  g.mode = f.precision == LR_DF64 ? LR_MODE_DF64 : f.precision == LR_FP32 ? LR_MODE_FP32 : LR_MODE_FP64;
  g.mixed_lanes = f.mixed_lanes ? f.mixed_lanes : lr_default_mixed_lanes(g.mode);
  g.remap = f.remap;
  g.sweep = 0;
  g.corners = f.remap == LR_REMAP_DIRECTCF;
  g.lagrange = 1;
  g.finalize = 1;
}

// Field `field` of one simulation as doubles in dst (device); s is its
// current state, prev the other half of its double buffer.
cudaError_t lr_field_view(const LrGrid& g, const LrState& s, const LrState& prev, const LrWork& w, double* rows,
                          int field, double* dst, cudaStream_t st, bool* unknown) {
  size_t nc = (size_t)g.nx * g.ny;
  *unknown = false;
#define CK(call, where)                          \
  do {                                           \
    cudaError_t _e = (call);                     \
    if (_e != cudaSuccess) return _e;            \
  } while (0)
  switch (field) {
    case LR_F_K: case LR_F_RHO_MAT: case LR_F_E_MAT: case LR_F_E_LAG:
      for (int a = 0; a < g.M; ++a) {
        const void* src = field == LR_F_K ? s.k[a] : field == LR_F_RHO_MAT ? s.r[a]
                        : field == LR_F_E_MAT ? s.e[a] : w.elag[a];
        CK(lr_launch_view(g, src, dst + a * nc, nc, 0, st), "view");
      }
      return cudaSuccess;
    case LR_F_P: case LR_F_RHO: case LR_F_E:
      CK(lr_launch_mixture(g, s, dst, field == LR_F_P ? 0 : field == LR_F_RHO ? 1 : 2, st), "mixture");
      return cudaSuccess;
    case LR_F_C: case LR_F_VOL_LAGCF: case LR_F_Q:
      CK(lr_launch_view(g, field == LR_F_C ? w.cc : field == LR_F_Q ? w.Q : w.vcf, dst, nc, 0, st), "view");
      return cudaSuccess;
    case LR_F_UX: case LR_F_UY: case LR_F_UHX: case LR_F_UHY: {
      const void* src = field == LR_F_UX ? s.ux : field == LR_F_UY ? s.uy : field == LR_F_UHX ? w.uhx : w.uhy;
      CK(lr_launch_view(g, src, dst, 0, 1, st), "view");
      return cudaSuccess;
    }
    case LR_F_FX: case LR_F_MX:
      CK(lr_launch_view(g, field == LR_F_FX ? w.fx : w.MX, dst, 0, 2, st), "view");
      return cudaSuccess;
    case LR_F_FY: case LR_F_MY:
      CK(lr_launch_view(g, field == LR_F_FY ? w.fy : w.MY, dst, 0, 3, st), "view");
      return cudaSuccess;
    case LR_F_FC: case LR_F_MC:
      CK(lr_launch_corner_debug(g, w, field == LR_F_FC ? dst : nullptr, field == LR_F_MC ? dst : nullptr, st),
         "corner view");
      return cudaSuccess;
    case LR_F_DT:
      CK(cudaMemcpyAsync(dst, w.scal + 2, sizeof(double), cudaMemcpyDeviceToDevice, st), "dt");
      return cudaSuccess;
    case LR_F_NMIXED:
      CK(cudaMemcpyAsync(dst, w.scal + 6, sizeof(double), cudaMemcpyDeviceToDevice, st), "mixed count");
      return cudaSuccess;
    case LR_F_CONS:
      CK(lr_launch_cons(g, s, rows, dst, st), "cons");
      return cudaSuccess;
    case LR_F_CUTS:
      CK(lr_launch_cuts(g, prev, w, dst, st), "cuts");
      return cudaSuccess;
    case LR_F_XA: case LR_F_YA: case LR_F_CA:
      for (int a = 0; a < g.M; ++a) {
        if (field == LR_F_XA)
          CK(lr_launch_view(g, w.xA[a], dst + (size_t)a * (g.nx + 1) * g.ny, 0, 2, st), "view");
        else if (field == LR_F_YA)
          CK(lr_launch_view(g, w.yA[a], dst + (size_t)a * g.nx * (g.ny + 1), 0, 3, st), "view");
        else
          CK(lr_launch_view(g, w.cA[a], dst + (size_t)a * (g.nx + 1) * (g.ny + 1), 0, 1, st), "view");
      }
      return cudaSuccess;
  }
#undef CK
  *unknown = true;
  return cudaSuccess;
}


extern "C" lr_status lr_arith_check(int op, const double* a, const double* b, double* out, size_t n,
                                   void* cuda_stream) {
  if (op != LR_ARITH_DIV && op != LR_ARITH_SQRT) return LR_ERR_ARG;
  if (n > 0 && (!a || !b || !out)) return LR_ERR_ARG;
  return lr_launch_arith(op, a, b, out, n, static_cast<cudaStream_t>(cuda_stream)) == cudaSuccess ? LR_OK
                                                                                                   : LR_ERR_CUDA;
}

extern "C" lr_status lr_fp64_fma_probe(double* dev_out, int blocks, int threads, int iters, void* cuda_stream) {
  if (!dev_out || blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1) return LR_ERR_ARG;
  return lr_launch_dfma(dev_out, blocks, threads, iters, static_cast<cudaStream_t>(cuda_stream)) == cudaSuccess
             ? LR_OK
             : LR_ERR_CUDA;
}

cudaError_t lr_create_aux_stream(cudaStream_t* s) {
  int least = 0, greatest = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  if (e != cudaSuccess) return e;
  return cudaStreamCreateWithPriority(s, cudaStreamNonBlocking, greatest);
}

size_t lr_field_count(const LrGrid& g, int field) {
  size_t nx = g.nx, ny = g.ny, M = g.M;
  switch (field) {
    case LR_F_K: case LR_F_RHO_MAT: case LR_F_E_MAT: case LR_F_E_LAG: return M * nx * ny;
    case LR_F_P: case LR_F_RHO: case LR_F_E: case LR_F_C: case LR_F_VOL_LAGCF: case LR_F_Q: return nx * ny;
    case LR_F_UX: case LR_F_UY: case LR_F_UHX: case LR_F_UHY: case LR_F_FC: case LR_F_MC: return (nx + 1) * (ny + 1);
    case LR_F_FX: case LR_F_MX: return (nx + 1) * ny;
    case LR_F_FY: case LR_F_MY: return nx * (ny + 1);
    case LR_F_CONS: return 8;
    case LR_F_DT: return 1;
    case LR_F_NMIXED: return 1;
    case LR_F_CUTS: return 6 * nx * ny;
    case LR_F_XA: return M * (nx + 1) * ny;
    case LR_F_YA: return M * nx * (ny + 1);
    case LR_F_CA: return M * (nx + 1) * (ny + 1);
  }
  return 0;
}

namespace {

void setmsg(lr_ctx* c, const char* fmt, ...) {
  if (!c) return;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(c->msg, sizeof(c->msg), fmt, ap);
  va_end(ap);
}

lr_status cuda_fail(lr_ctx* c, cudaError_t e, const char* where) {
  setmsg(c, "CUDA error in %s: %s", where, cudaGetErrorString(e));
  return LR_ERR_CUDA;
}

#define CK(call, where)                                    \
  do {                                                     \
    cudaError_t _e = (call);                               \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, where); \
  } while (0)

// Bump allocator over the arena; with base == nullptr it only measures.
struct Bump {
  char* base;
  size_t off;
  template <class T>
  T* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};


// Lay out every device array; returns the arena size.  Real arrays have the
// element size of the step's arithmetic (8 bytes for double and double-float,
// 4 for float).
size_t layout(const lr_config* cfg, char* base, LrState* st, LrWork* w, double** tmp, size_t* tmp_elems,
              double** rows) {
  Bump b{base, 0};
  size_t nx = cfg->nx, ny = cfg->ny, M = cfg->nmat;
  size_t nc = nx * ny, nn = (nx + 1) * (ny + 1), nfx = (nx + 1) * ny, nfy = nx * (ny + 1);
  size_t nd = (nx + 2) * (ny + 2);
  size_t es = lr_real_size(cfg->precision == LR_DF64 ? LR_MODE_DF64 : cfg->precision == LR_FP32 ? LR_MODE_FP32 : LR_MODE_FP64);
  auto R = [&](size_t n) { return static_cast<void*>(b.take<char>(n * es)); };
  LrState s[2];
  LrWork W;
  memset(s, 0, sizeof(s));
  memset(&W, 0, sizeof(W));
  for (int q = 0; q < 2; ++q) {
    for (size_t a = 0; a < M; ++a) { s[q].k[a] = R(nc); s[q].r[a] = R(nc); s[q].e[a] = R(nc); }
    s[q].ux = R(nn); s[q].uy = R(nn);
  }
  W.scal = b.take<double>(LR_NSCAL);
  W.red = b.take<unsigned long long>(LR_RED_INST + 2);
  W.err = b.take<int>(2);
  W.mixed = b.take<int>(nc);
  W.minst = b.take<int>(nc);
  W.gdev = b.take<LrGrid>(1);
  W.mask = b.take<unsigned char>(nc);
  {
    int tw = 0, th = 0;
    lr_tiled_tile_shape(&tw, &th);
    size_t nt = ((nx + tw - 1) / tw) * ((ny + th - 1) / th);
    W.tflag = b.take<unsigned int>(nt);
    W.tlist = b.take<int>(nt);
    W.tcount = b.take<unsigned int>(2);
  }
  for (int q = 0; q < 6; ++q) W.cut[q] = b.take<double>(nc);
  if (cfg->remap == LR_REMAP_DIRECT)
    for (int q = 0; q < 6; ++q) W.cutY[q] = b.take<double>(nc);
  W.stage = b.take<double>(3 * M * nc + 2 * nn);
  W.dtR = R(1);
  W.pux = R(nn); W.puy = R(nn);
  W.mc = R(nc); W.Q = R(nc); W.Pi = R(nc); W.cc = R(nc);
  for (size_t a = 0; a < M; ++a) { W.elc[a] = R(nc); W.elag[a] = R(nc); W.rcf[a] = R(nc); }
  W.ox = R(nc); W.oy = R(nc); W.wx = R(nc); W.wy = R(nc); W.vcf = R(nc);
  W.uhx = R(nn); W.uhy = R(nn); W.ddx = R(nn); W.ddy = R(nn); W.ulx = R(nn); W.uly = R(nn);
  W.fx = R(nfx); W.fxb = R(nfx); W.fxlo = R(nfx); W.fxhi = R(nfx);
  W.fy = R(nfy); W.fyb = R(nfy); W.fylo = R(nfy); W.fyhi = R(nfy);
  if (M > 1)
    for (size_t a = 0; a < M; ++a) { W.xAm[a] = R(nfx); W.yAm[a] = R(nfy); W.cAm[a] = R(nn); }
  for (size_t a = 0; a < M; ++a) {
    W.xA[a] = R(nfx); W.xMm[a] = R(nfx); W.xE[a] = R(nfx);
    W.yA[a] = R(nfy); W.yMm[a] = R(nfy); W.yE[a] = R(nfy);
    W.cA[a] = R(nn); W.cMm[a] = R(nn); W.cE[a] = R(nn);
  }
  W.MX = R(nfx); W.MY = R(nfy); W.Mpp = R(nn); W.Mpm = R(nn);
  for (int q = 0; q < 3; ++q) { W.dX[q] = R(nd); W.dY[q] = R(nd); W.dPP[q] = R(nd); W.dPM[q] = R(nd); }
  size_t te = M * nc > nn ? M * nc : nn;
  if (6 * nc > te) te = 6 * nc;
  if (M * nn > te) te = M * nn;
  if (nd > te) te = nd;
  double* t = b.take<double>(te);
  double* r = b.take<double>(8 * ((ny + 1) > 64 ? (ny + 1) : 64));
  if (st) { st[0] = s[0]; st[1] = s[1]; }
  if (w) *w = W;
  if (tmp) *tmp = t;
  if (tmp_elems) *tmp_elems = te;
  if (rows) *rows = r;
  return b.off + 256;
}

void fill_grid(lr_ctx* c) { lr_fill_grid(c->cfg, c->g); }

// Captured graphs hold the grid by value: drop them when it changes, and
// refresh the device copy the interface kernel reads.
void drop_graphs(lr_ctx* c) {
  for (int q = 0; q < 2; ++q)
    if (c->gvalid[q]) { cudaGraphExecDestroy(c->gexec[q]); c->gvalid[q] = false; }
  if (c->w.gdev) {
    cudaMemcpyAsync(const_cast<LrGrid*>(c->w.gdev), &c->g, sizeof(LrGrid), cudaMemcpyHostToDevice, c->stream);
    cudaStreamSynchronize(c->stream);
  }
}

lr_status check_sticky(lr_ctx* ctx) {
  if (ctx->sticky != LR_OK) return (lr_status)ctx->sticky;
  int e[2];
  CK(cudaMemcpyAsync(e, ctx->w.err, sizeof(e), cudaMemcpyDeviceToHost, ctx->stream), "error word");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  if (e[0] != 0) {
    ctx->sticky = LR_ERR_NUMERIC;
    setmsg(ctx, "numeric failure (bits 0x%x: %s%s%s%s%s) first at index %d", e[0],
           (e[0] & LR_DERR_VOLUME) ? "volume " : "", (e[0] & LR_DERR_SOUND) ? "sound-speed " : "",
           (e[0] & LR_DERR_MASS) ? "mass " : "", (e[0] & LR_DERR_NAN) ? "nan " : "",
           (e[0] & LR_DERR_GEOM) ? "flux-geometry " : "", e[1]);
    return LR_ERR_NUMERIC;
  }
  return LR_OK;
}

// Timing slots: the step's kernels, then the tiled kernels.
enum { SLOT_T_LAG = LRK_COUNT, SLOT_T_CELL, SLOT_T_NODE, SLOT_PLACE, SLOT_T_FLAGGED, NSLOT };
const char* slot_name(int k) {
  switch (k) {
    case SLOT_T_LAG: return "lr_t_lagrange";
    case SLOT_T_CELL: return "lr_t_cell_remap";
    case SLOT_T_NODE: return "lr_t_node_remap";
    case SLOT_PLACE: return "lb_mixed_place";
    case SLOT_T_FLAGGED: return "lr_t_cell_flagged";
    default: return lr_kernel_names[k];
  }
}
int slot_of(int k) {
  switch (k) {
    case LRK_MIXED_PLACE: case LRK_MIXED_PLACE_PDL: return SLOT_PLACE;  // lr_mixed: the flux split after it
    case LRK_MIXED_PDL: return LRK_MIXED;
    case LRK_T_LAGRANGE: return SLOT_T_LAG;
    case LRK_T_CELL_REMAP: case LRK_T_CELL_CLEAN: return SLOT_T_CELL;
    case LRK_T_CELL_DIRTY: return SLOT_T_FLAGGED;
    case LRK_T_NODE_REMAP: return SLOT_T_NODE;
    default: return k < LRK_COUNT ? k : -1;
  }
}
// The tiled kernels cover the one-step remap with corner fluxes and upwind or
// diagonal corner values.
bool tiled_ok(const LrGrid& g) {
  return g.remap == LR_REMAP_DIRECTCF && (g.corner_kind == LR_CORNER_UPWIND || g.corner_kind == LR_CORNER_DIAG);
}
// The tiled step splits its cell remap around the interface kernels (tiles
// no mixed cell reaches beside them, the listed tiles after them) for three
// materials: there the nested cut of three-material cells makes the
// interface kernels a long FP64 latency chain (about 65 us on the 1400 x 600
// triple point) that the clean tiles hide, for about 20 us of latency-bound
// work on the listed tiles afterwards.  With two materials the interface
// kernels are short (about 30 us on the 4096 x 1024 shock-bubble) and the
// split costs more than it hides (measured on GB300).
bool split_cell_remap(const LrGrid& g) { return g.M == 3; }
// Cell tiles of the tiled step (one flag each).
size_t tile_count(const LrGrid& g) {
  int tw = 0, th = 0;
  lr_tiled_tile_shape(&tw, &th);
  return (size_t)((g.nx + tw - 1) / tw) * (size_t)((g.ny + th - 1) / th);
}

cudaError_t launch_on(lr_ctx* ctx, int k, const LrGrid& g, const LrState& cur, const LrState& nxt, cudaStream_t st) {
  int slot = slot_of(k);
  if (!ctx->prof || slot < 0) return lr_launch(k, g, cur, nxt, ctx->w, st);
  lr_ctx::Pend p;
  p.kid = slot;
  cudaEventCreate(&p.a);
  cudaEventCreate(&p.b);
  cudaEventRecord(p.a, st);
  cudaError_t e = lr_launch(k, g, cur, nxt, ctx->w, st);
  cudaEventRecord(p.b, st);
  ctx->pend.push_back(p);
  return e;
}

// One kernel of the step.  The interface kernels run on the auxiliary
// stream: the placement of the interface lines (it needs the mixed-cell list
// and the Lagrangian rectangles) forked after lr_cell_lag, beside
// lr_cell_cf; the flux split (it needs rho^{lagCF}) after lr_cell_cf, beside
// lr_mat_flux (each finishes a disjoint set of flux objects); joined before
// lr_cell_update.  lr_dual_flux needs only the mass fluxes (lr_mat_flux and
// the flux split), not the cell update: it runs on the auxiliary stream
// beside lr_cell_update, joined before lr_node_update.
cudaError_t launch_one(lr_ctx* ctx, int k, const LrGrid& g, const LrState& cur, const LrState& nxt) {
  cudaError_t e;
  // profiling mode times every kernel alone: the second stream's kernels
  // run on the main stream, in the same order
  cudaStream_t side = ctx->prof ? ctx->stream : ctx->aux;
  if (k == LRK_CELL_LAG && g.M > 1) {
    if ((e = launch_on(ctx, k, g, cur, nxt, ctx->stream)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ctx->ev_fork, ctx->stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(side, ctx->ev_fork, 0)) != cudaSuccess) return e;
    return launch_on(ctx, LRK_MIXED_PLACE, g, cur, nxt, side);
  }
  if (k == LRK_MIXED) {
    if (g.M == 1) return cudaSuccess;
    if ((e = cudaEventRecord(ctx->ev_cf, ctx->stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(side, ctx->ev_cf, 0)) != cudaSuccess) return e;
    if ((e = launch_on(ctx, k, g, cur, nxt, side)) != cudaSuccess) return e;
    return cudaEventRecord(ctx->ev_join, side);
  }
  if (k == LRK_CELL_UPDATE) {
    if ((e = cudaEventRecord(ctx->ev_mf, ctx->stream)) != cudaSuccess) return e;  // lr_mat_flux done
    if (g.M > 1 && (e = cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0)) != cudaSuccess) return e;
  }
  if (k == LRK_DUAL_FLUX) {
    if ((e = cudaStreamWaitEvent(side, ctx->ev_mf, 0)) != cudaSuccess) return e;
    if ((e = launch_on(ctx, k, g, cur, nxt, side)) != cudaSuccess) return e;
    return cudaEventRecord(ctx->ev_dual, side);
  }
  if (k == LRK_NODE_UPDATE && (e = cudaStreamWaitEvent(ctx->stream, ctx->ev_dual, 0)) != cudaSuccess) return e;
  return launch_on(ctx, k, g, cur, nxt, ctx->stream);
}

// One step from buffer `from`.  One-step remaps: the nine kernels, result in
// the other buffer.  Alternate directions: the Lagrange phase and the first
// sweep into the other buffer, then the sweep preparation and the second
// sweep back into `from` (the kernels read the sweep order from the step
// count on the device).
cudaError_t enqueue_step(lr_ctx* ctx, int from) {
  const LrState& cur = ctx->st[from];
  const LrState& nxt = ctx->st[1 - from];
  if (ctx->tiled) {
    // Tiled step: the Lagrange phase and remap geometry (it flags the cell
    // tiles a mixed cell reaches and lists them); the interface kernels of
    // the mixed cells on the second (high-priority) stream, beside the
    // material fluxes and cell update of the tiles no mixed cell reaches; the
    // listed tiles once the interface work is done; the dual remap and node
    // update (it reads the new sound speeds for the CFL rule).  The interface
    // kernels are latency-bound on the FP64 pipe and leave most issue slots
    // free, so the clean tiles run in their shadow.  Profiling mode runs
    // everything on one stream.
    const LrGrid& g = ctx->g;
    cudaError_t e;
    if ((e = launch_on(ctx, LRK_T_LAGRANGE, g, cur, nxt, ctx->stream)) != cudaSuccess) return e;
    if (g.M == 1) {
      if ((e = launch_on(ctx, LRK_T_CELL_REMAP, g, cur, nxt, ctx->stream)) != cudaSuccess) return e;
      return launch_on(ctx, LRK_T_NODE_REMAP, g, cur, nxt, ctx->stream);
    }
    if (!split_cell_remap(g)) {  // one stream: interface kernels, then every tile
      if ((e = launch_on(ctx, LRK_MIXED_PLACE_PDL, g, cur, nxt, ctx->stream)) != cudaSuccess) return e;
      if ((e = launch_on(ctx, LRK_MIXED_PDL, g, cur, nxt, ctx->stream)) != cudaSuccess) return e;
      if ((e = launch_on(ctx, LRK_T_CELL_REMAP, g, cur, nxt, ctx->stream)) != cudaSuccess) return e;
      return launch_on(ctx, LRK_T_NODE_REMAP, g, cur, nxt, ctx->stream);
    }
    cudaStream_t side = ctx->prof ? ctx->stream : ctx->aux;
    if ((e = cudaEventRecord(ctx->ev_fork, ctx->stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(side, ctx->ev_fork, 0)) != cudaSuccess) return e;
    // plain launches here: a programmatic launch of the flux split keeps its
    // blocks resident (and their registers held) through the placement,
    // taking them from the clean tiles that run meanwhile
    if ((e = launch_on(ctx, LRK_MIXED_PLACE, g, cur, nxt, side)) != cudaSuccess) return e;
    if ((e = launch_on(ctx, LRK_MIXED, g, cur, nxt, side)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ctx->ev_join, side)) != cudaSuccess) return e;
    if ((e = launch_on(ctx, LRK_T_CELL_CLEAN, g, cur, nxt, ctx->stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0)) != cudaSuccess) return e;
    if ((e = launch_on(ctx, LRK_T_CELL_DIRTY, g, cur, nxt, ctx->stream)) != cudaSuccess) return e;
    return launch_on(ctx, LRK_T_NODE_REMAP, g, cur, nxt, ctx->stream);
  }
  if (ctx->g.remap != LR_REMAP_AD) {
    for (int k = 0; k < LRK_COUNT; ++k) {
      cudaError_t e = launch_one(ctx, k, ctx->g, cur, nxt);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  LrGrid g1 = ctx->g, g2 = ctx->g;
  g1.sweep = 1; g1.finalize = 0;
  g2.sweep = 2; g2.lagrange = 0;
  for (int k = 0; k < LRK_COUNT; ++k) {
    cudaError_t e = launch_one(ctx, k, g1, cur, nxt);
    if (e != cudaSuccess) return e;
  }
  const int second[] = {LRK_SWEEP_PREP, LRK_CELL_LAG, LRK_CELL_CF, LRK_MIXED, LRK_MAT_FLUX,
                        LRK_CELL_UPDATE, LRK_DUAL_FLUX, LRK_NODE_UPDATE};
  for (int k : second) {
    cudaError_t e = launch_one(ctx, k, g2, nxt, cur);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Buffer holding the state after a step from `from`.
int after_step(const lr_ctx* ctx, int from) { return ctx->g.remap == LR_REMAP_AD ? from : 1 - from; }

lr_status ensure_graph(lr_ctx* ctx, int from) {
  if (ctx->gvalid[from]) return LR_OK;
  cudaGraph_t gr;
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t e = enqueue_step(ctx, from);
  cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &gr);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "capture launch");
  if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "end capture");
  e = cudaGraphInstantiate(&ctx->gexec[from], gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
  ctx->gvalid[from] = true;
  return LR_OK;
}

lr_status create_common(const lr_config* cfg, void* mem, size_t bytes, bool own, lr_ctx** out) {
  if (!out) return LR_ERR_ARG;
  *out = nullptr;
  char why[160];
  if (!lr_config_ok(cfg, why, sizeof(why))) return LR_ERR_ARG;
  lr_ctx* ctx = new lr_ctx();
  ctx->cfg = *cfg;
  fill_grid(ctx);
  size_t need = layout(cfg, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
  if (own) {
    cudaError_t e = cudaMalloc(&mem, need);
    if (e != cudaSuccess) { delete ctx; return LR_ERR_OOM; }
    bytes = need;
  } else {
    if (!mem || bytes < need || (reinterpret_cast<uintptr_t>(mem) & 255)) { delete ctx; return LR_ERR_OOM; }
  }
  ctx->arena = static_cast<char*>(mem);
  ctx->arena_bytes = bytes;
  ctx->own_arena = own;
  layout(cfg, ctx->arena, ctx->st, &ctx->w, &ctx->tmp, &ctx->tmp_elems, &ctx->rows);
  if (cfg->cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
    ctx->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      if (own) cudaFree(mem);
      delete ctx;
      return LR_ERR_CUDA;
    }
    ctx->own_stream = true;
  }
  if (lr_create_aux_stream(&ctx->aux) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_cf, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_mf, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_dual, cudaEventDisableTiming) != cudaSuccess) {
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    if (own) cudaFree(mem);
    delete ctx;
    return LR_ERR_CUDA;
  }
  ctx->sticky = LR_OK;
  ctx->tiled = tiled_ok(ctx->g) && ctx->g.mode == LR_MODE_FP32;
  if (lr_tiled_setup() != cudaSuccess ||
      cudaMemcpyAsync(const_cast<LrGrid*>(ctx->w.gdev), &ctx->g, sizeof(LrGrid), cudaMemcpyHostToDevice,
                      ctx->stream) != cudaSuccess ||
      lr_launch_reset(ctx->g.mode, ctx->w, 1, ctx->stream) != cudaSuccess ||
      cudaMemsetAsync(ctx->w.pux, 0, lr_real_size(ctx->g.mode) * (cfg->nx + 1) * (cfg->ny + 1), ctx->stream) != cudaSuccess ||
      cudaMemsetAsync(ctx->w.puy, 0, lr_real_size(ctx->g.mode) * (cfg->nx + 1) * (cfg->ny + 1), ctx->stream) != cudaSuccess ||
      cudaMemsetAsync(ctx->w.tflag, 0, sizeof(unsigned int) * tile_count(ctx->g), ctx->stream) != cudaSuccess ||
      cudaMemsetAsync(ctx->w.tcount, 0, 2 * sizeof(unsigned int), ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    if (own) cudaFree(mem);
    delete ctx;
    return LR_ERR_CUDA;
  }
  *out = ctx;
  return LR_OK;
}

// ------------------------------------------------ field views (device)
lr_status field_to_device(lr_ctx* ctx, int field, double* dst) {
  bool unknown = false;
  CK(lr_field_view(ctx->g, ctx->st[ctx->cur], ctx->st[1 - ctx->cur], ctx->w, ctx->rows, field, dst, ctx->stream,
                   &unknown), "field view");
  if (unknown) { setmsg(ctx, "unknown field %d", field); return LR_ERR_ARG; }
  return LR_OK;
}

}  // namespace

extern "C" {

void lr_config_default(lr_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->nmat = 1;
  c->x1 = 1.0;
  c->y1 = 1.0;
  c->cfl = 0.25;
  c->a1 = 0.5;
  c->a2 = 1.0;
  c->face_order = 2;
  c->corner_recon = LR_CORNER_DIAG;
  c->precision = LR_FP64;
}

lr_status lr_workspace_bytes(const lr_config* cfg, size_t* bytes) {
  char why[160];
  if (!bytes || !lr_config_ok(cfg, why, sizeof(why))) return LR_ERR_ARG;
  *bytes = layout(cfg, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
  return LR_OK;
}

lr_status lr_create(const lr_config* cfg, lr_ctx** out) { return create_common(cfg, nullptr, 0, true, out); }

lr_status lr_create_in(const lr_config* cfg, void* dev_mem, size_t bytes, lr_ctx** out) {
  return create_common(cfg, dev_mem, bytes, false, out);
}

lr_status lr_set_materials(lr_ctx* ctx, int nmat, const lr_material* mats) {
  if (!ctx) return LR_ERR_ARG;
  if (nmat != ctx->cfg.nmat || !mats) { setmsg(ctx, "lr_set_materials: need %d materials", ctx->cfg.nmat); return LR_ERR_ARG; }
  for (int a = 0; a < nmat; ++a) {
    if (!(mats[a].gamma > 1.0) || !(mats[a].pi >= 0.0)) { setmsg(ctx, "material %d: gamma > 1, pi >= 0 required", a); return LR_ERR_ARG; }
  }
  for (int a = 0; a < nmat; ++a) { ctx->g.gam[a] = mats[a].gamma; ctx->g.pin[a] = mats[a].pi; }
  ctx->have_mats = true;
  drop_graphs(ctx);
  return LR_OK;
}

lr_status lr_init(lr_ctx* ctx, const double* k, const double* rho, const double* p, const double* ux,
                  const double* uy) {
  if (!ctx) return LR_ERR_ARG;
  if (!ctx->have_mats) { setmsg(ctx, "lr_init before lr_set_materials"); return LR_ERR_STATE; }
  if (!k || !rho || !p || !ux || !uy) { setmsg(ctx, "lr_init: null array"); return LR_ERR_ARG; }
  const LrGrid& g = ctx->g;
  size_t nc = (size_t)g.nx * g.ny, nn = (size_t)(g.nx + 1) * (g.ny + 1);
  ctx->cur = 0;
  LrState& s = ctx->st[0];
  double* sk = ctx->w.stage;  // stream-ordered after any step still in flight
  CK(cudaMemcpyAsync(sk, k, g.M * nc * sizeof(double), cudaMemcpyHostToDevice, ctx->stream), "upload k");
  CK(cudaMemcpyAsync(sk + g.M * nc, rho, g.M * nc * sizeof(double), cudaMemcpyHostToDevice, ctx->stream), "upload rho");
  CK(cudaMemcpyAsync(sk + 2 * g.M * nc, p, g.M * nc * sizeof(double), cudaMemcpyHostToDevice, ctx->stream), "upload p");
  CK(cudaMemcpyAsync(sk + 3 * g.M * nc, ux, nn * sizeof(double), cudaMemcpyHostToDevice, ctx->stream), "upload ux");
  CK(cudaMemcpyAsync(sk + 3 * g.M * nc + nn, uy, nn * sizeof(double), cudaMemcpyHostToDevice, ctx->stream), "upload uy");
  CK(lr_launch_reset(g.mode, ctx->w, 1, ctx->stream), "reset");
  CK(lr_launch_init(g, s, ctx->w, ctx->stream), "prepare");
  ctx->sticky = LR_OK;
  ctx->inited = false;
  lr_status st = check_sticky(ctx);
  if (st != LR_OK) {
    setmsg(ctx, "lr_init: invalid initial state (k outside [0,1], sum k != 1, or rho <= 0)");
    ctx->sticky = LR_OK;
    return LR_ERR_ARG;
  }
  ctx->inited = true;
  return LR_OK;
}

// ---------------------------------------------------------- checkpoints
// Layout of a checkpoint: a header of 8 int64 (magic, nx, ny, nmat,
// precision, element size, remap, corner values), the scalars of the
// simulation (LR_NSCAL doubles), then in the step's element type the state
// (k, rho, e per material [nmat][ny][nx], ux, uy [(ny+1)][(nx+1)]), the cell
// sound speeds [ny][nx] and the dt of the step in flight (one element).
static const long long LR_CKPT_MAGIC = 0x4c52434b50543031ll;  // "LRCKPT01"
static size_t ckpt_bytes(const lr_ctx* c) {
  size_t es = lr_real_size(c->g.mode);
  size_t nc = (size_t)c->g.nx * c->g.ny, nn = (size_t)(c->g.nx + 1) * (c->g.ny + 1);
  return 8 * sizeof(long long) + LR_NSCAL * sizeof(double) + es * (3 * c->g.M * nc + 2 * nn + nc + 1);
}

size_t lr_checkpoint_bytes(const lr_ctx* ctx) { return ctx ? ckpt_bytes(ctx) : 0; }

lr_status lr_checkpoint_save(lr_ctx* ctx, void* host_buf, size_t bytes) {
  if (!ctx || !host_buf) return LR_ERR_ARG;
  if (!ctx->inited) { setmsg(ctx, "lr_checkpoint_save before lr_init"); return LR_ERR_STATE; }
  if (bytes < ckpt_bytes(ctx)) { setmsg(ctx, "checkpoint buffer too small"); return LR_ERR_ARG; }
  lr_status st = check_sticky(ctx);
  if (st != LR_OK) return st;
  const LrGrid& g = ctx->g;
  long long* h = static_cast<long long*>(host_buf);
  h[0] = LR_CKPT_MAGIC; h[1] = g.nx; h[2] = g.ny; h[3] = g.M; h[4] = g.mode;
  h[5] = (long long)lr_real_size(g.mode); h[6] = g.remap; h[7] = g.corner_kind;
  char* p = static_cast<char*>(host_buf) + 8 * sizeof(long long);
  size_t es = lr_real_size(g.mode);
  size_t nc = (size_t)g.nx * g.ny, nn = (size_t)(g.nx + 1) * (g.ny + 1);
  cudaStream_t s = ctx->stream;
  CK(cudaMemcpyAsync(p, ctx->w.scal, LR_NSCAL * sizeof(double), cudaMemcpyDeviceToHost, s), "checkpoint");
  p += LR_NSCAL * sizeof(double);
  const LrState& cs = ctx->st[ctx->cur];
  for (int a = 0; a < g.M; ++a) {
    void* src[3] = {cs.k[a], cs.r[a], cs.e[a]};
    for (int q = 0; q < 3; ++q) {
      CK(cudaMemcpyAsync(p, src[q], es * nc, cudaMemcpyDeviceToHost, s), "checkpoint");
      p += es * nc;
    }
  }
  CK(cudaMemcpyAsync(p, cs.ux, es * nn, cudaMemcpyDeviceToHost, s), "checkpoint");
  p += es * nn;
  CK(cudaMemcpyAsync(p, cs.uy, es * nn, cudaMemcpyDeviceToHost, s), "checkpoint");
  p += es * nn;
  CK(cudaMemcpyAsync(p, ctx->w.cc, es * nc, cudaMemcpyDeviceToHost, s), "checkpoint");
  p += es * nc;
  CK(cudaMemcpyAsync(p, ctx->w.dtR, es, cudaMemcpyDeviceToHost, s), "checkpoint");
  CK(cudaStreamSynchronize(s), "checkpoint");
  return LR_OK;
}

lr_status lr_checkpoint_load(lr_ctx* ctx, const void* host_buf, size_t bytes) {
  if (!ctx || !host_buf) return LR_ERR_ARG;
  if (!ctx->have_mats) { setmsg(ctx, "lr_checkpoint_load before lr_set_materials"); return LR_ERR_STATE; }
  const LrGrid& g = ctx->g;
  const long long* h = static_cast<const long long*>(host_buf);
  if (bytes < 8 * sizeof(long long) || h[0] != LR_CKPT_MAGIC) { setmsg(ctx, "not a checkpoint"); return LR_ERR_ARG; }
  if (h[1] != g.nx || h[2] != g.ny || h[3] != g.M || h[4] != g.mode || h[5] != (long long)lr_real_size(g.mode) ||
      h[6] != g.remap || h[7] != g.corner_kind || bytes < ckpt_bytes(ctx)) {
    setmsg(ctx, "checkpoint of another configuration");
    return LR_ERR_ARG;
  }
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  const char* p = static_cast<const char*>(host_buf) + 8 * sizeof(long long);
  size_t es = lr_real_size(g.mode);
  size_t nc = (size_t)g.nx * g.ny, nn = (size_t)(g.nx + 1) * (g.ny + 1);
  cudaStream_t s = ctx->stream;
  CK(lr_launch_reset(g.mode, ctx->w, 1, s), "reset");
  CK(cudaMemcpyAsync(ctx->w.scal, p, LR_NSCAL * sizeof(double), cudaMemcpyHostToDevice, s), "restore");
  p += LR_NSCAL * sizeof(double);
  const LrState& cs = ctx->st[ctx->cur];
  for (int a = 0; a < g.M; ++a) {
    void* dst[3] = {cs.k[a], cs.r[a], cs.e[a]};
    for (int q = 0; q < 3; ++q) {
      CK(cudaMemcpyAsync(dst[q], p, es * nc, cudaMemcpyHostToDevice, s), "restore");
      p += es * nc;
    }
  }
  CK(cudaMemcpyAsync(cs.ux, p, es * nn, cudaMemcpyHostToDevice, s), "restore");
  p += es * nn;
  CK(cudaMemcpyAsync(cs.uy, p, es * nn, cudaMemcpyHostToDevice, s), "restore");
  p += es * nn;
  CK(cudaMemcpyAsync(ctx->w.cc, p, es * nc, cudaMemcpyHostToDevice, s), "restore");
  p += es * nc;
  CK(cudaMemcpyAsync(ctx->w.dtR, p, es, cudaMemcpyHostToDevice, s), "restore");
  CK(cudaStreamSynchronize(s), "restore");
  ctx->sticky = LR_OK;
  ctx->inited = true;
  return LR_OK;
}

lr_status lr_set_prescribed_velocity(lr_ctx* ctx, const double* ux, const double* uy) {
  if (!ctx) return LR_ERR_ARG;
  size_t nn = (size_t)(ctx->g.nx + 1) * (ctx->g.ny + 1);
  if (!ux || !uy) {
    ctx->g.presc = 0;
  } else {
    double* sk = ctx->tmp;  // staging of one node field at a time
    CK(cudaMemcpyAsync(sk, ux, nn * sizeof(double), cudaMemcpyHostToDevice, ctx->stream), "upload pu");
    CK(lr_launch_from_double(ctx->g, sk, ctx->w.pux, nn, ctx->stream), "convert pu");
    CK(cudaMemcpyAsync(sk, uy, nn * sizeof(double), cudaMemcpyHostToDevice, ctx->stream), "upload pu");
    CK(lr_launch_from_double(ctx->g, sk, ctx->w.puy, nn, ctx->stream), "convert pu");
    CK(cudaStreamSynchronize(ctx->stream), "sync");
    ctx->g.presc = 1;
  }
  drop_graphs(ctx);
  return LR_OK;
}

lr_status lr_step(lr_ctx* ctx, double t_end, double* dt_taken) {
  if (!ctx) return LR_ERR_ARG;
  if (!ctx->inited) { setmsg(ctx, "lr_step before lr_init"); return LR_ERR_STATE; }
  if (ctx->sticky != LR_OK) return (lr_status)ctx->sticky;
  CK(lr_launch_set_tend(ctx->g, ctx->w, t_end, ctx->stream), "set t_end");
  CK(enqueue_step(ctx, ctx->cur), "step launch");
  ctx->cur = after_step(ctx, ctx->cur);
  if (dt_taken) {
    lr_status s = check_sticky(ctx);
    if (s != LR_OK) return s;
    CK(cudaMemcpy(dt_taken, ctx->w.scal + 2, sizeof(double), cudaMemcpyDeviceToHost), "read dt");
  }
  return LR_OK;
}

lr_status lr_run(lr_ctx* ctx, double t_end, long max_steps, long* steps_done, double* t_now) {
  if (!ctx) return LR_ERR_ARG;
  if (!ctx->inited) { setmsg(ctx, "lr_run before lr_init"); return LR_ERR_STATE; }
  if (ctx->sticky != LR_OK) return (lr_status)ctx->sticky;
  if (max_steps < 0) return LR_ERR_ARG;
  double s0[5];
  CK(cudaMemcpyAsync(s0, ctx->w.scal, sizeof(s0), cudaMemcpyDeviceToHost, ctx->stream), "read scalars");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  CK(lr_launch_set_tend(ctx->g, ctx->w, t_end, ctx->stream), "set t_end");
  // Steps are enqueued in chunks; after each chunk t and the next CFL dt are
  // read back and the next chunk is sized from the time left, so few no-op
  // steps (t already at t_end) are enqueued.
  long done = 0, chunk = 64;
  double t_cur = s0[0], dt_cur = ctx->g.dt_fixed > 0.0 ? ctx->g.dt_fixed : s0[1];
  while (done < max_steps && t_cur < t_end) {
    if (dt_cur > 0.0 && (t_end - t_cur) / dt_cur < 1e9) {
      long left = (long)((t_end - t_cur) / dt_cur) + 2;
      chunk = left < 64 ? left : 64;
    }
    long n = max_steps - done < chunk ? max_steps - done : chunk;
    for (long q = 0; q < n; ++q) {
      if (ctx->prof) {
        CK(enqueue_step(ctx, ctx->cur), "step launch");
      } else {
        lr_status s = ensure_graph(ctx, ctx->cur);
        if (s != LR_OK) return s;
        CK(cudaGraphLaunch(ctx->gexec[ctx->cur], ctx->stream), "graph launch");
      }
      ctx->cur = after_step(ctx, ctx->cur);
    }
    done += n;
    double sc[5];
    CK(cudaMemcpyAsync(sc, ctx->w.scal, sizeof(sc), cudaMemcpyDeviceToHost, ctx->stream), "read scalars");
    lr_status s = check_sticky(ctx);
    if (s != LR_OK) return s;
    t_cur = sc[0];
    dt_cur = ctx->g.dt_fixed > 0.0 ? ctx->g.dt_fixed : sc[1];
  }
  double sc[5];
  CK(cudaMemcpyAsync(sc, ctx->w.scal, sizeof(sc), cudaMemcpyDeviceToHost, ctx->stream), "read scalars");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  if (steps_done) *steps_done = (long)(sc[4] - s0[4] + 0.5);
  if (t_now) *t_now = sc[0];
  return LR_OK;
}

lr_status lr_sync(lr_ctx* ctx) {
  if (!ctx) return LR_ERR_ARG;
  return check_sticky(ctx);
}

size_t lr_field_size(const lr_ctx* ctx, int field) { return ctx ? lr_field_count(ctx->g, field) : 0; }

// Field into host memory, enqueued: pinned (page-locked, mapped) memory is
// written by the view kernel directly over the host link (no device staging,
// no separate copy); pageable memory through the staging buffer, the copy
// finishing before the call returns.
static lr_status field_to_host(lr_ctx* ctx, int field, double* host_out, size_t n_elems, const char* who) {
  if (!ctx || !host_out) return LR_ERR_ARG;
  size_t need = lr_field_size(ctx, field);
  if (need == 0 || n_elems < need) { setmsg(ctx, "%s: field %d needs %zu elements", who, field, need); return LR_ERR_ARG; }
  if (!ctx->inited) { setmsg(ctx, "%s before lr_init", who); return LR_ERR_STATE; }
  cudaPointerAttributes at;
  bool by_kernel = field != LR_F_DT && field != LR_F_NMIXED;  // the other fields are written by a kernel
  if (by_kernel && cudaPointerGetAttributes(&at, host_out) == cudaSuccess && at.type == cudaMemoryTypeHost &&
      at.devicePointer) {
    return field_to_device(ctx, field, static_cast<double*>(at.devicePointer));
  }
  cudaGetLastError();  // a failed query leaves an error state behind: clear it
  lr_status s = field_to_device(ctx, field, ctx->tmp);
  if (s != LR_OK) return s;
  CK(cudaMemcpyAsync(host_out, ctx->tmp, need * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "download");
  CK(cudaStreamSynchronize(ctx->stream), "sync");  // the staging buffer is reused by the next call
  return LR_OK;
}

lr_status lr_get_fields(lr_ctx* ctx, int field, double* host_out, size_t n_elems) {
  lr_status s = field_to_host(ctx, field, host_out, n_elems, "lr_get_fields");
  if (s != LR_OK) return s;
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  return LR_OK;
}

lr_status lr_get_fields_async(lr_ctx* ctx, int field, double* host_out, size_t n_elems) {
  if (field == LR_F_CONS) {
    if (ctx) setmsg(ctx, "lr_get_fields_async: LR_F_CONS is read with lr_get_fields");
    return LR_ERR_ARG;
  }
  return field_to_host(ctx, field, host_out, n_elems, "lr_get_fields_async");
}

lr_status lr_get_fields_device(lr_ctx* ctx, int field, double* dev_out, size_t n_elems) {
  if (!ctx || !dev_out) return LR_ERR_ARG;
  size_t need = lr_field_size(ctx, field);
  if (need == 0 || n_elems < need) return LR_ERR_ARG;
  if (!ctx->inited) return LR_ERR_STATE;
  return field_to_device(ctx, field, dev_out);
}

lr_status lr_time(lr_ctx* ctx, double* t, double* dt_next) {
  if (!ctx) return LR_ERR_ARG;
  double sc[5];
  CK(cudaMemcpyAsync(sc, ctx->w.scal, sizeof(sc), cudaMemcpyDeviceToHost, ctx->stream), "read scalars");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  if (t) *t = sc[0];
  if (dt_next) *dt_next = ctx->g.dt_fixed > 0.0 ? ctx->g.dt_fixed : sc[1];
  return LR_OK;
}

int lr_launches_per_step(const lr_ctx* ctx) {
  // the t_end/dt kernel, then the step's kernels (no interface kernel with one
  // material); alternate directions: a second sweep of eight kernels
  if (!ctx) return 0;
  // the interface work is two kernels (placement, then the flux split)
  int one = (int)LRK_COUNT + (ctx->g.M == 1 ? -1 : 1);
  // tiled: t_end/dt, Lagrange, cell remap, node remap; with two or more
  // materials the interface lines and flux split; with three the cell remap
  // in two launches (the tiles no mixed cell reaches, then the listed ones)
  if (ctx->tiled) return ctx->g.M == 1 ? 4 : ctx->g.M == 2 ? 6 : 7;
  return 1 + one + (ctx->g.remap == LR_REMAP_AD ? one - 1 : 0);
}

lr_status lr_set_tiled(lr_ctx* ctx, int on) {
  if (!ctx) return LR_ERR_ARG;
  if (on && !tiled_ok(ctx->g)) {
    setmsg(ctx, "the tiled step covers the DirectCF remap with upwind or diagonal corners only");
    return LR_ERR_ARG;
  }
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  ctx->tiled = on != 0;
  drop_graphs(ctx);
  return LR_OK;
}

int lr_get_tiled(const lr_ctx* ctx) { return ctx && ctx->tiled ? 1 : 0; }

lr_status lr_set_profiling(lr_ctx* ctx, int on) {
  if (!ctx) return LR_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  for (auto& p : ctx->pend) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  ctx->pend.clear();
  for (int k = 0; k < NSLOT; ++k) { ctx->acc_ms[k] = 0.0; ctx->acc_n[k] = 0; }
  ctx->prof = on != 0;
  return LR_OK;
}

int lr_kernel_times(lr_ctx* ctx, const char** names, long* launches, double* ms, int n) {
  if (!ctx) return 0;
  cudaStreamSynchronize(ctx->stream);
  for (auto& p : ctx->pend) {
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) { ctx->acc_ms[p.kid] += t; ctx->acc_n[p.kid] += 1; }
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  ctx->pend.clear();
  int m = n < (int)NSLOT ? n : (int)NSLOT;
  for (int k = 0; k < m; ++k) {
    if (names) names[k] = slot_name(k);
    if (launches) launches[k] = ctx->acc_n[k];
    if (ms) ms[k] = ctx->acc_ms[k];
  }
  return NSLOT;
}

void lr_destroy(lr_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  drop_graphs(ctx);
  for (auto& p : ctx->pend) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  cudaStreamSynchronize(ctx->aux);
  cudaStreamDestroy(ctx->aux);
  cudaEventDestroy(ctx->ev_fork);
  cudaEventDestroy(ctx->ev_cf);
  cudaEventDestroy(ctx->ev_join);
  cudaEventDestroy(ctx->ev_mf);
  cudaEventDestroy(ctx->ev_dual);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  if (ctx->own_arena) cudaFree(ctx->arena);
  delete ctx;
}

const char* lr_last_error(const lr_ctx* ctx) { return ctx ? ctx->msg : "null context"; }

}  // extern "C"
