// lr_batch.cu -- the C ABI of include/lr_batch.h: a device pool shared by
// many simulations, first-fit admission by units of the pool, tile tables
// grouped by material count, one batched launch per kernel of the step,
// CUDA graphs, per-member status, field read-back and the schedule
// autotuner.
#include "../../include/lr_batch.h"
#include "lr_dev.cuh"
#include "lr_host.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <algorithm>
#include <utility>
#include <vector>

namespace {

constexpr int NSHAPE = 4;
const int SHAPE_X[NSHAPE] = {32, 64, 16, 128};
const int SHAPE_Y[NSHAPE] = {8, 4, 16, 2};
constexpr int NBPS = 4;
const int BPS_OPTIONS[NBPS] = {0, 2, 4, 8};  // persistent blocks per SM; 0 = one block per tile
const int LANE_OPTIONS[3] = {2, 4, 8};

struct Member {
  bool used = false;
  int failed = 0;        // invalid initial state or numeric error seen by the host
  lr_config cfg;
  LrGrid g;
  long off = 0, units = 0;
};

struct Range { int start = 0, count = 0; };

struct Schedule {
  int shape[LRK_COUNT];
  int bps[LRK_COUNT];
  int lanes;
};

}  // namespace

struct lr_batch {
  lr_batch_config cfg;
  int mode;
  size_t es;             // bytes per real
  long P;                // pool units
  int S;                 // member slots
  int nsm;
  char* arena = nullptr;
  size_t state_bytes = 0;  // one state buffer (contiguous)
  size_t scal_bytes = 0;   // scal, red, err, dtR (contiguous)
  size_t cc_bytes = 0;     // w.cc: the state's sound-speed term, read by the next lb_cell_pre
  LrState st[2];
  int cur = 0;
  LrWork w;
  LrGrid* d_gs = nullptr;
  char* d_kcs = nullptr;
  size_t kcb = 0;
  double* tmp = nullptr;
  double* rows = nullptr;
  // tile tables
  LrTile* d_tiles = nullptr;
  size_t tiles_cap = 0;
  Range rng[NSHAPE][LR_NDOM][LR_MAXM + 1];   // [shape][domain][M], M=0: all groups
  Range prc, prn;                            // the persistent step's cell and node tiles (tiled-step shape)
  bool need_rebuild = true;
  long group_units[LR_MAXM + 1] = {0, 0, 0, 0};
  int group_members[LR_MAXM + 1] = {0, 0, 0, 0};
  LrTile* d_adm = nullptr;   // tiles of one member being admitted
  size_t adm_cap = 0;
  std::vector<Member> mem;
  std::vector<std::pair<long, long>> freel;  // free unit ranges (offset, length), sorted
  Schedule sch;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t aux = nullptr;   // interface kernels, beside lb_mat_flux
  cudaEvent_t ev_fork = nullptr, ev_cf = nullptr, ev_join = nullptr, ev_mf = nullptr, ev_dual = nullptr;
  cudaGraphExec_t gexec[2];
  bool gvalid[2] = {false, false};
  int launches = 0;
  bool prof = false;
  // persistent step: one cooperative launch per step (lb_t_step); by
  // default in FP32, and chosen by lr_batch_autotune unless the caller set it
  bool persistent = true;
  bool persistent_set = false;
  int pers_bps = 0;                 // resident blocks per SM of lb_t_step
  LrGridBar* bar = nullptr;         // its grid barrier (count, generation, status)
  unsigned int bar_extra = 0;       // test hook: arrivals no block makes
  unsigned long long bar_limit_ns = 1000000000ull;
  int sticky = LR_OK;               // LR_ERR_TIMEOUT after a barrier gave up
  struct Pend { int kid; cudaEvent_t a, b; };
  std::vector<Pend> pend;
  double acc_ms[LRK_COUNT + 1];     // per kernel; the last slot: the persistent step kernel
  long acc_n[LRK_COUNT + 1];
  char msg[512];
};

namespace {

void setmsg(lr_batch* b, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b->msg, sizeof(b->msg), fmt, ap);
  va_end(ap);
}

lr_status cuda_fail(lr_batch* b, cudaError_t e, const char* where) {
  setmsg(b, "CUDA error in %s: %s", where, cudaGetErrorString(e));
  return LR_ERR_CUDA;
}

#define CK(call, where)                                      \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return cuda_fail(b, _e, where);   \
  } while (0)

int mode_of(int precision) {
  return precision == LR_DF64 ? LR_MODE_DF64 : precision == LR_FP32 ? LR_MODE_FP32 : LR_MODE_FP64;
}

bool batch_config_ok(const lr_batch_config* c, char* why, size_t n) {
  if (!c) { snprintf(why, n, "null config"); return false; }
  if (c->precision != LR_FP64 && c->precision != LR_DF64 && c->precision != LR_FP32) {
    snprintf(why, n, "bad precision");
    return false;
  }
  if (c->nmat_max < 1 || c->nmat_max > LR_MAXM) { snprintf(why, n, "nmat_max must be 1..3"); return false; }
  if (c->capacity_members < 1 || c->capacity_members > (1 << 20)) { snprintf(why, n, "capacity_members"); return false; }
  if (c->capacity_units < 16 || c->capacity_units > (1L << 30)) { snprintf(why, n, "capacity_units"); return false; }
  if (c->max_member_cells < 4 || c->max_member_cells > (1L << 28)) { snprintf(why, n, "max_member_cells"); return false; }
  return true;
}

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

// Lay out the pool; every array of P units (so a member's cell, node,
// face and dual-cell arrays all start at its unit offset).
size_t layout(const lr_batch_config* c, char* base, lr_batch* b) {
  Bump m{base, 0};
  size_t P = (size_t)c->capacity_units, S = (size_t)c->capacity_members, M = (size_t)c->nmat_max;
  size_t es = lr_real_size(mode_of(c->precision));
  auto R = [&](size_t n) { return static_cast<void*>(m.take<char>(n * es)); };
  LrState s[2];
  LrWork W;
  memset(s, 0, sizeof(s));
  memset(&W, 0, sizeof(W));
  size_t s0 = 0;
  for (int q = 0; q < 2; ++q) {
    size_t a0 = (m.off + 255) & ~size_t(255);
    for (size_t a = 0; a < M; ++a) { s[q].k[a] = R(P); s[q].r[a] = R(P); s[q].e[a] = R(P); }
    s[q].ux = R(P); s[q].uy = R(P);
    if (q == 0) s0 = m.off - a0;
  }
  size_t sc0 = (m.off + 255) & ~size_t(255);
  W.scal = m.take<double>(LR_NSCAL * S);
  W.red = m.take<unsigned long long>(LR_RED_INST + 2 * S);
  W.err = m.take<int>(2 * S);
  W.dtR = R(S);
  size_t sc1 = m.off;
  W.mixed = m.take<int>(2 * P);
  W.minst = m.take<int>(2 * P);
  W.mask = m.take<unsigned char>(P);
  for (int q = 0; q < 6; ++q) W.cut[q] = m.take<double>(P);
  size_t C = (size_t)c->max_member_cells;
  W.stage = m.take<double>(3 * M * C + 2 * (2 * C + 1));
  W.pux = nullptr; W.puy = nullptr;
  W.mc = R(P); W.Q = R(P); W.Pi = R(P); W.cc = R(P);
  for (size_t a = 0; a < M; ++a) { W.elc[a] = R(P); W.elag[a] = R(P); W.rcf[a] = R(P); }
  W.ox = R(P); W.oy = R(P); W.wx = R(P); W.wy = R(P); W.vcf = R(P);
  W.uhx = R(P); W.uhy = R(P); W.ddx = R(P); W.ddy = R(P); W.ulx = R(P); W.uly = R(P);
  W.fx = R(P); W.fxb = R(P); W.fxlo = R(P); W.fxhi = R(P);
  W.fy = R(P); W.fyb = R(P); W.fylo = R(P); W.fyhi = R(P);
  for (size_t a = 0; a < M; ++a) {
    W.xAm[a] = R(P); W.yAm[a] = R(P); W.cAm[a] = R(P);
    W.xA[a] = R(P); W.xMm[a] = R(P); W.xE[a] = R(P);
    W.yA[a] = R(P); W.yMm[a] = R(P); W.yE[a] = R(P);
    W.cA[a] = R(P); W.cMm[a] = R(P); W.cE[a] = R(P);
  }
  W.MX = R(P); W.MY = R(P); W.Mpp = R(P); W.Mpm = R(P);
  for (int q = 0; q < 3; ++q) { W.dX[q] = R(P); W.dY[q] = R(P); W.dPP[q] = R(P); W.dPM[q] = R(P); }
  LrGridBar* bar = m.take<LrGridBar>(1);
  LrGrid* gs = m.take<LrGrid>(S);
  size_t kcb = lr_kc_bytes(mode_of(c->precision));
  char* kcs = m.take<char>(S * kcb);
  double* tmp = m.take<double>(6 * C + 8);
  double* rows = m.take<double>(8 * (C / 2 + 2 > 64 ? C / 2 + 2 : 64));
  if (b) {
    b->st[0] = s[0]; b->st[1] = s[1]; b->w = W;
    b->state_bytes = s0;
    b->scal_bytes = sc1 - sc0;
    b->cc_bytes = P * es;
    b->d_gs = gs; b->d_kcs = kcs; b->kcb = kcb;
    b->bar = bar;
    b->tmp = tmp; b->rows = rows;
  }
  return m.off + 256;
}

size_t unit_bytes(const lr_batch_config* c) {
  size_t es = lr_real_size(mode_of(c->precision)), M = (size_t)c->nmat_max;
  // state (two buffers), work reals, per-material work, dual, lists, mask, cuts
  return es * (2 * (3 * M + 2) + 29 + 15 * M + 12) + 2 * 4 + 2 * 4 + 1 + 6 * 8;
}

// ------------------------------------------------------------ unit pool
bool pool_alloc(lr_batch* b, long n, long* off) {
  for (size_t q = 0; q < b->freel.size(); ++q) {
    if (b->freel[q].second >= n) {
      *off = b->freel[q].first;
      b->freel[q].first += n;
      b->freel[q].second -= n;
      if (b->freel[q].second == 0) b->freel.erase(b->freel.begin() + q);
      return true;
    }
  }
  return false;
}
void pool_free(lr_batch* b, long off, long n) {
  auto it = std::lower_bound(b->freel.begin(), b->freel.end(), std::make_pair(off, 0L));
  it = b->freel.insert(it, std::make_pair(off, n));
  size_t q = it - b->freel.begin();
  if (q + 1 < b->freel.size() && b->freel[q].first + b->freel[q].second == b->freel[q + 1].first) {
    b->freel[q].second += b->freel[q + 1].second;
    b->freel.erase(b->freel.begin() + q + 1);
  }
  if (q > 0 && b->freel[q - 1].first + b->freel[q - 1].second == b->freel[q].first) {
    b->freel[q - 1].second += b->freel[q].second;
    b->freel.erase(b->freel.begin() + q);
  }
}

// ------------------------------------------------------------ tile tables
void dom_size(const LrGrid& g, int d, int* w, int* h) {
  switch (d) {
    case LR_DOM_CELLS: *w = g.nx; *h = g.ny; break;
    case LR_DOM_NODES: *w = g.nxu; *h = g.nyu; break;
    case LR_DOM_DUAL: *w = g.nx + 2; *h = g.ny + 2; break;
    default: *w = g.nx + 1; *h = g.ny + 1; break;
  }
}
void tiles_wh(const LrGrid& g, int slot, int d, int tw, int th, std::vector<LrTile>& out) {
  int w, h;
  dom_size(g, d, &w, &h);
  int tx = (w + tw - 1) / tw, ty = (h + th - 1) / th;
  for (int j = 0; j < ty; ++j)
    for (int i = 0; i < tx; ++i) out.push_back(LrTile{slot, i * tw, j * th, tx * ty});
}
void tiles_of(const LrGrid& g, int slot, int d, int s, std::vector<LrTile>& out) {
  tiles_wh(g, slot, d, SHAPE_X[s], SHAPE_Y[s], out);
}

lr_status rebuild(lr_batch* b) {
  bool use[NSHAPE][LR_NDOM];
  memset(use, 0, sizeof(use));
  for (int k = 0; k < LRK_COUNT; ++k)
    if (k != LRK_MIXED) use[b->sch.shape[k]][lr_kernel_domain(k)] = true;

  std::vector<LrTile> all;
  memset(b->rng, 0, sizeof(b->rng));
  for (int M = 0; M <= LR_MAXM; ++M) { b->group_units[M] = 0; b->group_members[M] = 0; }
  for (size_t q = 0; q < b->mem.size(); ++q)
    if (b->mem[q].used) { b->group_units[b->mem[q].g.M] += b->mem[q].units; b->group_members[b->mem[q].g.M] += 1; }
  for (int s = 0; s < NSHAPE; ++s)
    for (int d = 0; d < LR_NDOM; ++d) {
      if (!use[s][d]) continue;
      b->rng[s][d][0].start = (int)all.size();
      for (int M = 1; M <= LR_MAXM; ++M) {
        b->rng[s][d][M].start = (int)all.size();
        for (size_t q = 0; q < b->mem.size(); ++q)
          if (b->mem[q].used && b->mem[q].g.M == M) tiles_of(b->mem[q].g, (int)q, d, s, all);
        b->rng[s][d][M].count = (int)all.size() - b->rng[s][d][M].start;
      }
      b->rng[s][d][0].count = (int)all.size() - b->rng[s][d][0].start;
    }
  // the persistent step's tables: every member's cell and node tiles in the
  // tiled step's tile shape
  int tw = 0, th = 0;
  lr_tiled_tile_shape(&tw, &th);
  b->prc.start = (int)all.size();
  for (size_t q = 0; q < b->mem.size(); ++q)
    if (b->mem[q].used) tiles_wh(b->mem[q].g, (int)q, LR_DOM_CELLS, tw, th, all);
  b->prc.count = (int)all.size() - b->prc.start;
  b->prn.start = (int)all.size();
  for (size_t q = 0; q < b->mem.size(); ++q)
    if (b->mem[q].used) tiles_wh(b->mem[q].g, (int)q, LR_DOM_NODES, tw, th, all);
  b->prn.count = (int)all.size() - b->prn.start;
  if (all.size() > b->tiles_cap) {
    if (b->d_tiles) cudaFree(b->d_tiles);
    b->d_tiles = nullptr;
    size_t cap = all.size() + all.size() / 4 + 1024;
    CK(cudaMalloc(&b->d_tiles, cap * sizeof(LrTile)), "tile table");
    b->tiles_cap = cap;
  }
  if (!all.empty())
    CK(cudaMemcpyAsync(b->d_tiles, all.data(), all.size() * sizeof(LrTile), cudaMemcpyHostToDevice, b->stream),
       "upload tiles");
  CK(cudaStreamSynchronize(b->stream), "sync");
  for (int q = 0; q < 2; ++q)
    if (b->gvalid[q]) { cudaGraphExecDestroy(b->gexec[q]); b->gvalid[q] = false; }
  b->need_rebuild = false;
  return LR_OK;
}

LrBatchArgs base_args(lr_batch* b) {
  LrBatchArgs a;
  memset(&a, 0, sizeof(a));
  a.mode = b->mode;
  a.gs = b->d_gs;
  a.kcs = b->d_kcs;
  return a;
}

int grid_for_tiles(lr_batch* b, int bps, int ntiles) {
  if (bps <= 0) return ntiles;
  int g = b->nsm * bps;
  return g < ntiles ? g : ntiles;
}

cudaError_t launch_timed(lr_batch* b, int kid, const LrBatchArgs& a, const LrState& cur, const LrState& nxt,
                         cudaStream_t st) {
  b->launches += 1;
  if (!b->prof) return lr_launch_batch(kid, a, cur, nxt, b->w, st);
  lr_batch::Pend p;
  p.kid = kid == LRK_MIXED_PLACE ? (int)LRK_MIXED : kid;  // both interface kernels time as lr_mixed
  cudaEventCreate(&p.a);
  cudaEventCreate(&p.b);
  cudaEventRecord(p.a, st);
  cudaError_t e = lr_launch_batch(kid, a, cur, nxt, b->w, st);
  cudaEventRecord(p.b, st);
  b->pend.push_back(p);
  return e;
}

// Arguments of an interface kernel over material-count group M with `lanes`
// threads per mixed cell (blocks of 128 threads, at most 16 per SM).
void set_mixed_args(const lr_batch* b, int M, int lanes, LrBatchArgs& a) {
  a.M = M;
  a.lanes = lanes;
  a.mslot = M - 1;
  a.moff = (M - 2) * (int)b->P;
  long nb = ((long)lanes * b->group_units[M] + 127) / 128;
  a.grid = (int)(nb < (long)b->nsm * 16 ? nb : (long)b->nsm * 16);
}

bool persistent_on(const lr_batch* b) { return b->persistent && b->pers_bps > 0; }

// One step of every member in one cooperative launch (lb_t_step), after the
// barrier words are cleared.
cudaError_t enqueue_persistent(lr_batch* b, int from) {
  const LrState& cur = b->st[from];
  const LrState& nxt = b->st[1 - from];
  const Range& rc = b->prc;
  const Range& rn = b->prn;
  b->launches = 0;
  if (rc.count == 0) return cudaSuccess;
  LrPersistArgs p;
  memset(&p, 0, sizeof(p));
  p.gs = b->d_gs;
  p.kcs = b->d_kcs;
  p.ctiles = b->d_tiles + rc.start;
  p.nct = rc.count;
  p.ntiles = b->d_tiles + rn.start;
  p.nnt = rn.count;
  p.bar = b->bar;
  p.extra = b->bar_extra;
  p.limit_ns = b->bar_limit_ns;
  p.groups = (b->group_members[2] > 0 ? 4 : 0) | (b->group_members[3] > 0 ? 8 : 0);
  p.P = (int)b->P;
  int most = b->nsm * b->pers_bps;
  p.grid = rc.count < most ? rc.count : most;
  if (rn.count < p.grid) p.grid = rn.count > 0 ? rn.count : 1;
  cudaError_t e = cudaMemsetAsync(b->bar, 0, sizeof(LrGridBar), b->stream);
  if (e != cudaSuccess) return e;
  b->launches = 1;
  if (!b->prof) return lr_launch_batch_persistent(b->mode, p, cur, nxt, b->w, b->stream);
  lr_batch::Pend pe;
  pe.kid = LRK_COUNT;
  cudaEventCreate(&pe.a);
  cudaEventCreate(&pe.b);
  cudaEventRecord(pe.a, b->stream);
  e = lr_launch_batch_persistent(b->mode, p, cur, nxt, b->w, b->stream);
  cudaEventRecord(pe.b, b->stream);
  b->pend.push_back(pe);
  return e;
}

// One step of every member: for each kernel, one launch per material-count
// group (kernels that do not depend on it: one launch over all groups).
cudaError_t enqueue_step(lr_batch* b, int from) {
  if (persistent_on(b)) return enqueue_persistent(b, from);
  const LrState& cur = b->st[from];
  const LrState& nxt = b->st[1 - from];
  b->launches = 0;
  // profiling mode times every kernel alone: the second stream's kernels
  // run on the main stream, in the same order
  cudaStream_t side = b->prof ? b->stream : b->aux;
  for (int k = 0; k < LRK_COUNT; ++k) {
    LrBatchArgs a = base_args(b);
    bool any_mixed = b->group_members[2] + b->group_members[3] > 0;
    cudaStream_t ks = b->stream;
    if (k == LRK_CELL_UPDATE) {
      // lb_dual_flux needs only the mass fluxes: it runs on the auxiliary
      // stream beside lb_cell_update, joined before lb_node_update
      cudaError_t e = cudaEventRecord(b->ev_mf, b->stream);
      if (e == cudaSuccess && any_mixed) e = cudaStreamWaitEvent(b->stream, b->ev_join, 0);
      if (e != cudaSuccess) return e;
    }
    if (k == LRK_DUAL_FLUX) {
      cudaError_t e = cudaStreamWaitEvent(side, b->ev_mf, 0);
      if (e != cudaSuccess) return e;
      ks = side;
    }
    if (k == LRK_NODE_UPDATE) {
      cudaError_t e = cudaStreamWaitEvent(b->stream, b->ev_dual, 0);
      if (e != cudaSuccess) return e;
    }
    if (k == LRK_MIXED) {
      // the flux split of the mixed cells runs on the auxiliary stream after
      // lb_cell_cf, beside lb_mat_flux (disjoint flux objects), joined
      // before lb_cell_update
      if (!any_mixed) continue;
      cudaError_t e = cudaEventRecord(b->ev_cf, b->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(side, b->ev_cf, 0);
      if (e != cudaSuccess) return e;
      for (int M = 2; M <= LR_MAXM; ++M) {
        if (b->group_members[M] == 0) continue;
        set_mixed_args(b, M, b->sch.lanes, a);
        e = launch_timed(b, k, a, cur, nxt, side);
        if (e != cudaSuccess) return e;
      }
      e = cudaEventRecord(b->ev_join, side);
      if (e != cudaSuccess) return e;
      continue;
    }
    int s = b->sch.shape[k], d = lr_kernel_domain(k);
    a.bx = SHAPE_X[s];
    a.by = SHAPE_Y[s];
    a.tiles = b->d_tiles;
    bool per_m = !(k == LRK_NODE_HALF || k == LRK_DUAL_FLUX || k == LRK_NODE_UPDATE);
    for (int M = per_m ? 1 : 0; M <= (per_m ? LR_MAXM : 0); ++M) {
      const Range& r = b->rng[s][d][M];
      if (r.count == 0) continue;
      a.M = M == 0 ? 1 : M;
      a.tiles = b->d_tiles + r.start;
      a.ntiles = r.count;
      a.grid = grid_for_tiles(b, b->sch.bps[k], r.count);
      cudaError_t e = launch_timed(b, k, a, cur, nxt, ks);
      if (e != cudaSuccess) return e;
    }
    if (k == LRK_DUAL_FLUX) {
      cudaError_t e = cudaEventRecord(b->ev_dual, side);
      if (e != cudaSuccess) return e;
    }
    if (k == LRK_CELL_LAG && any_mixed) {
      // the interface lines of the mixed cells need the Lagrangian
      // rectangles: placed on the auxiliary stream beside lb_cell_cf
      cudaError_t e = cudaEventRecord(b->ev_fork, b->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(side, b->ev_fork, 0);
      if (e != cudaSuccess) return e;
      for (int M = 2; M <= LR_MAXM; ++M) {
        if (b->group_members[M] == 0) continue;
        LrBatchArgs pa = base_args(b);
        set_mixed_args(b, M, 8, pa);  // enough warps for four cells each
        e = launch_timed(b, LRK_MIXED_PLACE, pa, cur, nxt, side);
        if (e != cudaSuccess) return e;
      }
    }
  }
  return cudaSuccess;
}

lr_status ensure_graph(lr_batch* b, int from) {
  if (b->gvalid[from]) return LR_OK;
  cudaGraph_t gr;
  CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t e = enqueue_step(b, from);
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &gr);
  if (e != cudaSuccess) return cuda_fail(b, e, "capture launch");
  if (e2 != cudaSuccess) return cuda_fail(b, e2, "end capture");
  e = cudaGraphInstantiate(&b->gexec[from], gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return cuda_fail(b, e, "graph instantiate");
  b->gvalid[from] = true;
  return LR_OK;
}

// The persistent step's barrier status: a wait that gave up leaves the
// batch in error (LR_ERR_TIMEOUT) until it is destroyed.
lr_status check_barrier(lr_batch* b) {
  if (b->sticky != LR_OK) return (lr_status)b->sticky;
  if (!persistent_on(b)) return LR_OK;
  LrGridBar h;
  CK(cudaMemcpyAsync(&h, b->bar, sizeof(h), cudaMemcpyDeviceToHost, b->stream), "barrier status");
  CK(cudaStreamSynchronize(b->stream), "sync");
  if (h.status != 0) {
    b->sticky = LR_ERR_TIMEOUT;
    setmsg(b, "persistent step: a grid barrier waited longer than %.3f s and the step was abandoned",
           (double)b->bar_limit_ns * 1e-9);
    return LR_ERR_TIMEOUT;
  }
  return LR_OK;
}

lr_status run_steps(lr_batch* b, int nsteps) {
  if (b->sticky != LR_OK) return (lr_status)b->sticky;
  if (b->need_rebuild) {
    lr_status s = rebuild(b);
    if (s != LR_OK) return s;
  }
  for (int q = 0; q < nsteps; ++q) {
    if (b->prof) {
      CK(enqueue_step(b, b->cur), "step launch");
    } else {
      lr_status s = ensure_graph(b, b->cur);
      if (s != LR_OK) return s;
      CK(cudaGraphLaunch(b->gexec[b->cur], b->stream), "graph launch");
    }
    b->cur = 1 - b->cur;
  }
  return LR_OK;
}

bool member_ok(const lr_batch* b, int m) { return b && m >= 0 && m < (int)b->mem.size() && b->mem[m].used; }

// A member's arrays re-based at its offset, with a grid of offset 0 and
// slot 0 -- the form the single-simulation field views expect.
void member_view(const lr_batch* b, int m, LrGrid* g, LrState* s, LrState* prev, LrWork* w) {
  const Member& mb = b->mem[m];
  size_t off = (size_t)mb.off, es = b->es;
  auto rb = [&](void* p) -> void* { return p ? static_cast<char*>(p) + off * es : nullptr; };
  for (int q = 0; q < 2; ++q) {
    const LrState& src = b->st[q == 0 ? b->cur : 1 - b->cur];
    LrState& dst = q == 0 ? *s : *prev;
    memset(&dst, 0, sizeof(dst));
    for (int a = 0; a < b->cfg.nmat_max; ++a) { dst.k[a] = rb(src.k[a]); dst.r[a] = rb(src.r[a]); dst.e[a] = rb(src.e[a]); }
    dst.ux = rb(src.ux); dst.uy = rb(src.uy);
  }
  *w = b->w;
#define LR_F1(n) w->n = rb(b->w.n);
  LR_WORK_REALS(LR_F1)
#undef LR_F1
#define LR_F1(n) for (int a = 0; a < LR_MAXM; ++a) w->n[a] = rb(b->w.n[a]);
  LR_WORK_MAT_REALS(LR_F1)
#undef LR_F1
  for (int q = 0; q < 3; ++q) {
    w->dX[q] = rb(b->w.dX[q]); w->dY[q] = rb(b->w.dY[q]); w->dPP[q] = rb(b->w.dPP[q]); w->dPM[q] = rb(b->w.dPM[q]);
  }
  for (int q = 0; q < 6; ++q) w->cut[q] = b->w.cut[q] + off;
  w->mask = b->w.mask + off;
  w->scal = b->w.scal + LR_NSCAL * m;
  w->red = nullptr;
  w->err = b->w.err + 2 * m;
  w->dtR = static_cast<char*>(b->w.dtR) + (size_t)m * es;
  *g = mb.g;
  g->coff = g->noff = g->doff = 0;
  g->inst = 0;
  g->mslot = 0;
  g->moff = 0;
  g->stoff = 0;
}

void default_schedule(lr_batch* b) {
  for (int k = 0; k < LRK_COUNT; ++k) { b->sch.shape[k] = 0; b->sch.bps[k] = 0; }
  b->sch.lanes = lr_default_mixed_lanes(b->mode);
}

}  // namespace

extern "C" {

void lr_batch_config_default(lr_batch_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->precision = LR_FP64;
  c->nmat_max = 3;
  c->capacity_units = 1L << 20;
  c->capacity_members = 16;
  c->max_member_cells = 1L << 20;
}

lr_status lr_batch_workspace_bytes(const lr_batch_config* cfg, size_t* bytes) {
  char why[160];
  if (!bytes || !batch_config_ok(cfg, why, sizeof(why))) return LR_ERR_ARG;
  *bytes = layout(cfg, nullptr, nullptr);
  return LR_OK;
}

lr_status lr_batch_unit_bytes(const lr_batch_config* cfg, size_t* bytes) {
  char why[160];
  if (!bytes || !batch_config_ok(cfg, why, sizeof(why))) return LR_ERR_ARG;
  *bytes = unit_bytes(cfg);
  return LR_OK;
}

lr_status lr_batch_create(const lr_batch_config* cfg, lr_batch** out) {
  if (!out) return LR_ERR_ARG;
  *out = nullptr;
  char why[160];
  if (!batch_config_ok(cfg, why, sizeof(why))) return LR_ERR_ARG;
  lr_batch* b = new lr_batch();
  b->cfg = *cfg;
  b->mode = mode_of(cfg->precision);
  b->es = lr_real_size(b->mode);
  b->P = cfg->capacity_units;
  b->S = cfg->capacity_members;
  int dev = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) b->nsm = 152;
  size_t need = layout(cfg, nullptr, nullptr);
  if (cudaMalloc(&b->arena, need) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return LR_ERR_OOM;
  }
  layout(cfg, b->arena, b);
  if (cfg->cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
  } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess) {
    b->own_stream = true;
  } else {
    cudaFree(b->arena);
    delete b;
    return LR_ERR_CUDA;
  }
  if (lr_create_aux_stream(&b->aux) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_cf, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_mf, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_dual, cudaEventDisableTiming) != cudaSuccess) {
    if (b->own_stream) cudaStreamDestroy(b->stream);
    cudaFree(b->arena);
    delete b;
    return LR_ERR_CUDA;
  }
  b->mem.resize(b->S);
  b->freel.push_back(std::make_pair(0L, b->P));
  default_schedule(b);
  for (int k = 0; k <= LRK_COUNT; ++k) { b->acc_ms[k] = 0.0; b->acc_n[k] = 0; }
  if (lr_tiled_setup() != cudaSuccess) cudaGetLastError();
  b->pers_bps = lr_persistent_blocks_per_sm(b->mode);
  if (b->pers_bps > 4) b->pers_bps = 4;
  // the persistent step is the faster one in FP32 and the slower one in FP64
  // (the 512-member ensemble on GB300: 4.3e9 against 3.9e9 cell-updates/s in
  // FP32, 0.92e9 against 1.28e9 in FP64, whose interface phase inside the
  // persistent kernel runs with a fraction of the registers it needs)
  b->persistent = b->mode == LR_MODE_FP32;
  b->msg[0] = 0;
  if (lr_launch_reset(b->mode, b->w, b->S, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess) {
    if (b->own_stream) cudaStreamDestroy(b->stream);
    cudaFree(b->arena);
    delete b;
    return LR_ERR_CUDA;
  }
  *out = b;
  return LR_OK;
}

void lr_batch_destroy(lr_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (int q = 0; q < 2; ++q)
    if (b->gvalid[q]) cudaGraphExecDestroy(b->gexec[q]);
  for (auto& p : b->pend) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_adm) cudaFree(b->d_adm);
  cudaStreamSynchronize(b->aux);
  cudaStreamDestroy(b->aux);
  cudaEventDestroy(b->ev_fork);
  cudaEventDestroy(b->ev_cf);
  cudaEventDestroy(b->ev_join);
  cudaEventDestroy(b->ev_mf);
  cudaEventDestroy(b->ev_dual);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  cudaFree(b->arena);
  delete b;
}

const char* lr_batch_last_error(const lr_batch* b) { return b ? b->msg : "null batch"; }

lr_status lr_batch_add(lr_batch* b, const lr_config* cfg, const lr_material* mats, const double* k,
                       const double* rho, const double* p, const double* ux, const double* uy, double t_end,
                       long max_steps, int* member) {
  if (!b) return LR_ERR_ARG;
  if (member) *member = -1;
  char why[160];
  if (!cfg || !mats || !k || !rho || !p || !ux || !uy || !member) { setmsg(b, "lr_batch_add: null argument"); return LR_ERR_ARG; }
  if (!lr_config_ok(cfg, why, sizeof(why))) { setmsg(b, "lr_batch_add: %s", why); return LR_ERR_ARG; }
  if (cfg->precision != b->cfg.precision) { setmsg(b, "lr_batch_add: precision differs from the batch's"); return LR_ERR_ARG; }
  if (cfg->remap != LR_REMAP_DIRECTCF || cfg->corner_recon > LR_CORNER_DIAG) {
    setmsg(b, "lr_batch_add: batches run the DirectCF remap with upwind or diagonal corners only");
    return LR_ERR_ARG;
  }
  if (cfg->nmat > b->cfg.nmat_max) { setmsg(b, "lr_batch_add: nmat above nmat_max"); return LR_ERR_ARG; }
  if ((long)cfg->nx * cfg->ny > b->cfg.max_member_cells) { setmsg(b, "lr_batch_add: grid above max_member_cells"); return LR_ERR_ARG; }
  if (!(t_end >= 0.0)) { setmsg(b, "lr_batch_add: t_end must be >= 0"); return LR_ERR_ARG; }
  for (int a = 0; a < cfg->nmat; ++a)
    if (!(mats[a].gamma > 1.0) || !(mats[a].pi >= 0.0)) { setmsg(b, "material %d: gamma > 1, pi >= 0 required", a); return LR_ERR_ARG; }
  int slot = -1;
  for (int q = 0; q < b->S; ++q)
    if (!b->mem[q].used) { slot = q; break; }
  if (slot < 0) { setmsg(b, "lr_batch_add: all %d member slots in use", b->S); return LR_ERR_OOM; }
  long units = (long)(cfg->nx + 2) * (cfg->ny + 2), off = 0;
  if (!pool_alloc(b, units, &off)) { setmsg(b, "lr_batch_add: no free range of %ld units", units); return LR_ERR_OOM; }
  Member& mb = b->mem[slot];
  mb = Member();
  mb.used = true;
  mb.cfg = *cfg;
  mb.cfg.cuda_stream = nullptr;
  mb.off = off;
  mb.units = units;
  LrGrid& g = mb.g;
  memset(&g, 0, sizeof(g));
  lr_fill_grid(mb.cfg, g);
  for (int a = 0; a < cfg->nmat; ++a) { g.gam[a] = mats[a].gamma; g.pin[a] = mats[a].pi; }
  g.presc = 0;
  g.coff = g.noff = g.doff = (int)off;
  g.inst = slot;
  g.mslot = g.M >= 2 ? g.M - 1 : 0;
  g.moff = g.M >= 2 ? (g.M - 2) * (int)b->P : 0;
  g.stoff = 0;
  // the batch's lanes per mixed cell apply to every member
  g.mixed_lanes = b->sch.lanes;
  std::vector<char> kc(b->kcb);
  lr_make_kc(g, kc.data());
  size_t nc = (size_t)g.nx * g.ny, nn = (size_t)(g.nx + 1) * (g.ny + 1);
  double* sk = b->w.stage;
  cudaStream_t st = b->stream;
  double sc[LR_NSCAL] = {0.0, 0.0, 0.0, t_end, 0.0, 0.0, 0.0, max_steps > 0 ? (double)max_steps : 0.0};
  unsigned long long z[2] = {0ull, 0ull};
  int e0[2] = {0, -1};
  std::vector<LrTile> tl;
  tiles_of(g, slot, LR_DOM_NODES_ALL, 0, tl);
  int n_prep = (int)tl.size();
  tiles_of(g, slot, LR_DOM_NODES, 0, tl);
  int n_cfl = (int)tl.size() - n_prep;
  if (tl.size() > b->adm_cap) {
    CK(cudaStreamSynchronize(st), "sync");
    if (b->d_adm) cudaFree(b->d_adm);
    b->d_adm = nullptr;
    CK(cudaMalloc(&b->d_adm, tl.size() * sizeof(LrTile)), "admission tiles");
    b->adm_cap = tl.size();
  }
  CK(cudaMemcpyAsync(b->d_gs + slot, &g, sizeof(g), cudaMemcpyHostToDevice, st), "upload grid");
  CK(cudaMemcpyAsync(b->d_kcs + (size_t)slot * b->kcb, kc.data(), b->kcb, cudaMemcpyHostToDevice, st), "upload kc");
  CK(cudaMemcpyAsync(b->w.scal + LR_NSCAL * slot, sc, sizeof(sc), cudaMemcpyHostToDevice, st), "scalars");
  CK(cudaMemcpyAsync(b->w.red + LR_RED_INST + 2 * slot, z, sizeof(z), cudaMemcpyHostToDevice, st), "red");
  CK(cudaMemcpyAsync(b->w.err + 2 * slot, e0, sizeof(e0), cudaMemcpyHostToDevice, st), "err");
  CK(cudaMemcpyAsync(b->d_adm, tl.data(), tl.size() * sizeof(LrTile), cudaMemcpyHostToDevice, st), "tiles");
  CK(cudaMemcpyAsync(sk, k, g.M * nc * sizeof(double), cudaMemcpyHostToDevice, st), "upload k");
  CK(cudaMemcpyAsync(sk + g.M * nc, rho, g.M * nc * sizeof(double), cudaMemcpyHostToDevice, st), "upload rho");
  CK(cudaMemcpyAsync(sk + 2 * g.M * nc, p, g.M * nc * sizeof(double), cudaMemcpyHostToDevice, st), "upload p");
  CK(cudaMemcpyAsync(sk + 3 * g.M * nc, ux, nn * sizeof(double), cudaMemcpyHostToDevice, st), "upload ux");
  CK(cudaMemcpyAsync(sk + 3 * g.M * nc + nn, uy, nn * sizeof(double), cudaMemcpyHostToDevice, st), "upload uy");
  LrBatchArgs a = base_args(b);
  a.M = g.M;
  a.bx = SHAPE_X[0];
  a.by = SHAPE_Y[0];
  a.tiles = b->d_adm;
  a.ntiles = n_prep;
  a.grid = n_prep;
  const LrState& cs = b->st[b->cur];
  CK(lr_launch_batch(LRK_PREPARE, a, cs, cs, b->w, st), "prepare");
  a.M = 1;
  a.tiles = b->d_adm + n_prep;
  a.ntiles = n_cfl;
  a.grid = n_cfl;
  CK(lr_launch_batch(LRK_CFL_ONLY, a, cs, cs, b->w, st), "cfl");
  int e[2];
  CK(cudaMemcpyAsync(e, b->w.err + 2 * slot, sizeof(e), cudaMemcpyDeviceToHost, st), "error word");
  CK(cudaStreamSynchronize(st), "sync");
  *member = slot;
  b->need_rebuild = true;
  if (e[0] != 0) {
    mb.failed = 1;
    double zero = 0.0;
    CK(cudaMemcpyAsync(b->w.scal + LR_NSCAL * slot + 5, &zero, sizeof(zero), cudaMemcpyHostToDevice, st), "stop");
    CK(cudaStreamSynchronize(st), "sync");
    setmsg(b, "lr_batch_add: invalid initial state (k outside [0,1], sum k != 1, or rho <= 0)");
    return LR_ERR_ARG;
  }
  return LR_OK;
}

lr_status lr_batch_set_limits(lr_batch* b, int m, double t_end, long max_steps) {
  if (!member_ok(b, m) || !(t_end >= 0.0)) return LR_ERR_ARG;
  if (b->mem[m].failed) { setmsg(b, "member %d failed", m); return LR_ERR_STATE; }
  double lim = max_steps > 0 ? (double)max_steps : 0.0;
  CK(cudaMemcpyAsync(b->w.scal + LR_NSCAL * m + 7, &lim, sizeof(lim), cudaMemcpyHostToDevice, b->stream), "limit");
  CK(lr_launch_set_tend(b->mem[m].g, b->w, t_end, b->stream), "t_end");
  CK(cudaStreamSynchronize(b->stream), "sync");
  return LR_OK;
}

lr_status lr_batch_remove(lr_batch* b, int m) {
  if (!member_ok(b, m)) return LR_ERR_ARG;
  CK(cudaStreamSynchronize(b->stream), "sync");
  pool_free(b, b->mem[m].off, b->mem[m].units);
  b->mem[m] = Member();
  b->need_rebuild = true;
  return LR_OK;
}

lr_status lr_batch_step(lr_batch* b, int nsteps) {
  if (!b || nsteps < 0) return LR_ERR_ARG;
  return run_steps(b, nsteps);
}

lr_status lr_batch_sync(lr_batch* b) {
  if (!b) return LR_ERR_ARG;
  CK(cudaStreamSynchronize(b->stream), "sync");
  return check_barrier(b);
}

lr_status lr_batch_set_persistent(lr_batch* b, int on) {
  if (!b) return LR_ERR_ARG;
  if (on && b->pers_bps <= 0) { setmsg(b, "the persistent step cannot be resident on this device"); return LR_ERR_ARG; }
  CK(cudaStreamSynchronize(b->stream), "sync");
  b->persistent = on != 0;
  b->persistent_set = true;
  b->need_rebuild = true;
  return LR_OK;
}

int lr_batch_get_persistent(const lr_batch* b) { return b && persistent_on(b) ? 1 : 0; }

lr_status lr_batch_test_barrier(lr_batch* b, unsigned int extra_arrivals, double limit_s) {
  if (!b || !(limit_s > 0.0) || limit_s > 10.0) return LR_ERR_ARG;
  CK(cudaStreamSynchronize(b->stream), "sync");
  b->bar_extra = extra_arrivals;
  b->bar_limit_ns = (unsigned long long)(limit_s * 1e9);
  for (int q = 0; q < 2; ++q)
    if (b->gvalid[q]) { cudaGraphExecDestroy(b->gexec[q]); b->gvalid[q] = false; }
  return LR_OK;
}

lr_status lr_batch_status_all(lr_batch* b, int* state, long* steps, int n) {
  if (!b || n < b->S) return LR_ERR_ARG;
  std::vector<double> sc((size_t)LR_NSCAL * b->S);
  std::vector<int> er((size_t)2 * b->S);
  CK(cudaMemcpyAsync(sc.data(), b->w.scal, sc.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "scalars");
  CK(cudaMemcpyAsync(er.data(), b->w.err, er.size() * sizeof(int), cudaMemcpyDeviceToHost, b->stream), "errors");
  CK(cudaStreamSynchronize(b->stream), "sync");
  for (int q = 0; q < b->S; ++q) {
    Member& mb = b->mem[q];
    if (!mb.used) {
      if (state) state[q] = -2;
      if (steps) steps[q] = 0;
      continue;
    }
    if (er[2 * q] != 0 && !mb.failed) {
      mb.failed = 1;
      double zero = 0.0;  // stop the member; the others go on
      CK(cudaMemcpyAsync(b->w.scal + LR_NSCAL * q + 5, &zero, sizeof(zero), cudaMemcpyHostToDevice, b->stream), "stop");
    }
    if (state) state[q] = mb.failed ? -1 : (sc[LR_NSCAL * q + 5] > 0.0 ? 0 : 1);
    if (steps) steps[q] = (long)sc[LR_NSCAL * q + 4];
  }
  CK(cudaStreamSynchronize(b->stream), "sync");
  return LR_OK;
}

lr_status lr_batch_status(lr_batch* b, int m, double* t, long* steps, int* state) {
  if (!member_ok(b, m)) return LR_ERR_ARG;
  double sc[LR_NSCAL];
  int er[2];
  CK(cudaMemcpyAsync(sc, b->w.scal + LR_NSCAL * m, sizeof(sc), cudaMemcpyDeviceToHost, b->stream), "scalars");
  CK(cudaMemcpyAsync(er, b->w.err + 2 * m, sizeof(er), cudaMemcpyDeviceToHost, b->stream), "errors");
  CK(cudaStreamSynchronize(b->stream), "sync");
  Member& mb = b->mem[m];
  if (er[0] != 0 && !mb.failed) {
    mb.failed = 1;
    double zero = 0.0;
    CK(cudaMemcpyAsync(b->w.scal + LR_NSCAL * m + 5, &zero, sizeof(zero), cudaMemcpyHostToDevice, b->stream), "stop");
    CK(cudaStreamSynchronize(b->stream), "sync");
    setmsg(b, "member %d: numeric failure (bits 0x%x) at index %d", m, er[0], er[1]);
  }
  if (t) *t = sc[0];
  if (steps) *steps = (long)sc[4];
  if (state) *state = mb.failed ? -1 : (sc[5] > 0.0 ? 0 : 1);
  return LR_OK;
}

size_t lr_batch_field_size(const lr_batch* b, int m, int field) {
  if (!member_ok(b, m)) return 0;
  return lr_field_count(b->mem[m].g, field);
}

lr_status lr_batch_get_fields(lr_batch* b, int m, int field, double* host_out, size_t n_elems) {
  if (!member_ok(b, m) || !host_out) return LR_ERR_ARG;
  size_t need = lr_field_count(b->mem[m].g, field);
  if (need == 0 || n_elems < need) { setmsg(b, "lr_batch_get_fields: field %d needs %zu elements", field, need); return LR_ERR_ARG; }
  LrGrid g;
  LrState s, prev;
  LrWork w;
  member_view(b, m, &g, &s, &prev, &w);
  bool unknown = false;
  CK(lr_field_view(g, s, prev, w, b->rows, field, b->tmp, b->stream, &unknown), "field view");
  if (unknown) { setmsg(b, "unknown field %d", field); return LR_ERR_ARG; }
  CK(cudaMemcpyAsync(host_out, b->tmp, need * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "download");
  CK(cudaStreamSynchronize(b->stream), "sync");
  return LR_OK;
}

int lr_batch_launches_per_step(const lr_batch* b) {
  if (!b) return 0;
  if (persistent_on(b)) return 1;
  int n = 0;
  for (int k = 0; k < LRK_COUNT; ++k) {
    if (k == LRK_MIXED) {  // placement and flux split: two kernels per group
      for (int M = 2; M <= LR_MAXM; ++M) n += 2 * (b->group_members[M] > 0);
      continue;
    }
    bool per_m = !(k == LRK_NODE_HALF || k == LRK_DUAL_FLUX || k == LRK_NODE_UPDATE);
    if (per_m) {
      for (int M = 1; M <= LR_MAXM; ++M) n += b->group_members[M] > 0;
    } else {
      int any = 0;
      for (int M = 1; M <= LR_MAXM; ++M) any |= b->group_members[M] > 0;
      n += any;
    }
  }
  return n;
}

lr_status lr_batch_set_profiling(lr_batch* b, int on) {
  if (!b) return LR_ERR_ARG;
  CK(cudaStreamSynchronize(b->stream), "sync");
  for (auto& p : b->pend) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  b->pend.clear();
  for (int k = 0; k <= LRK_COUNT; ++k) { b->acc_ms[k] = 0.0; b->acc_n[k] = 0; }
  b->prof = on != 0;
  return LR_OK;
}

int lr_batch_kernel_times(lr_batch* b, const char** names, long* launches, double* ms, int n) {
  if (!b) return 0;
  cudaStreamSynchronize(b->stream);
  for (auto& p : b->pend) {
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) { b->acc_ms[p.kid] += t; b->acc_n[p.kid] += 1; }
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  b->pend.clear();
  int m = n < (int)LRK_COUNT + 1 ? n : (int)LRK_COUNT + 1;
  for (int k = 0; k < m; ++k) {
    if (names) names[k] = k < LRK_COUNT ? lr_kernel_names[k] : "lb_t_step";
    if (launches) launches[k] = b->acc_n[k];
    if (ms) ms[k] = b->acc_ms[k];
  }
  return LRK_COUNT + 1;
}

lr_status lr_batch_schedule(const lr_batch* b, int* shape, int* bps, int* lanes) {
  if (!b) return LR_ERR_ARG;
  for (int k = 0; k < LRK_COUNT; ++k) {
    if (shape) shape[k] = b->sch.shape[k];
    if (bps) bps[k] = b->sch.bps[k];
  }
  if (lanes) *lanes = b->sch.lanes;
  return LR_OK;
}

lr_status lr_batch_autotune(lr_batch* b, int trial_steps) {
  if (!b) return LR_ERR_ARG;
  if (trial_steps < 1) trial_steps = 1;
  bool any = false;
  for (auto& m : b->mem) any |= m.used;
  if (!any) { setmsg(b, "lr_batch_autotune: no members"); return LR_ERR_STATE; }
  if (b->sticky != LR_OK) return (lr_status)b->sticky;
  CK(cudaStreamSynchronize(b->stream), "sync");
  // the schedule belongs to the per-kernel step; the persistent step is off
  // while the trials run
  const bool pers0 = b->persistent;
  b->persistent = false;
  // snapshot of the current state buffer, the scalars and the sound-speed
  // term the next step's lb_cell_pre reads
  char* snap = nullptr;
  size_t nb = b->state_bytes + b->scal_bytes + b->cc_bytes;
  char* cc0 = static_cast<char*>(b->w.cc);
  CK(cudaMalloc(&snap, nb), "autotune snapshot");
  const int cur0 = b->cur;
  char* st0 = static_cast<char*>(b->st[cur0].k[0]);
  char* sc0 = reinterpret_cast<char*>(b->w.scal);
  lr_status rs = LR_OK;
  auto restore = [&]() -> lr_status {
    CK(cudaMemcpyAsync(static_cast<char*>(b->st[cur0].k[0]), snap, b->state_bytes, cudaMemcpyDeviceToDevice, b->stream), "restore");
    CK(cudaMemcpyAsync(sc0, snap + b->state_bytes, b->scal_bytes, cudaMemcpyDeviceToDevice, b->stream), "restore");
    CK(cudaMemcpyAsync(cc0, snap + b->state_bytes + b->scal_bytes, b->cc_bytes, cudaMemcpyDeviceToDevice, b->stream),
       "restore");
    b->cur = cur0;
    CK(cudaStreamSynchronize(b->stream), "sync");
    return LR_OK;
  };
  auto trial = [&](const Schedule& s, double* per_kernel) -> lr_status {
    b->sch = s;
    b->need_rebuild = true;
    lr_status q = lr_batch_set_profiling(b, 1);
    if (q != LR_OK) return q;
    q = run_steps(b, 1);  // warm-up
    if (q != LR_OK) return q;
    lr_batch_kernel_times(b, nullptr, nullptr, nullptr, 0);
    for (int k = 0; k < LRK_COUNT; ++k) { b->acc_ms[k] = 0.0; b->acc_n[k] = 0; }
    q = run_steps(b, trial_steps);
    if (q != LR_OK) return q;
    lr_batch_kernel_times(b, nullptr, nullptr, per_kernel, LRK_COUNT);
    q = lr_batch_set_profiling(b, 0);
    if (q != LR_OK) return q;
    return restore();
  };
  CK(cudaMemcpyAsync(snap, st0, b->state_bytes, cudaMemcpyDeviceToDevice, b->stream), "snapshot");
  CK(cudaMemcpyAsync(snap + b->state_bytes, sc0, b->scal_bytes, cudaMemcpyDeviceToDevice, b->stream), "snapshot");
  CK(cudaMemcpyAsync(snap + b->state_bytes + b->scal_bytes, cc0, b->cc_bytes, cudaMemcpyDeviceToDevice, b->stream),
     "snapshot");
  Schedule best = b->sch;
  double bestt[LRK_COUNT];
  for (int k = 0; k < LRK_COUNT; ++k) bestt[k] = 1e300;
  double t[LRK_COUNT];
  // 1. tile shape per kernel (one block per tile)
  for (int s = 0; s < NSHAPE && rs == LR_OK; ++s) {
    Schedule c = best;
    for (int k = 0; k < LRK_COUNT; ++k) { c.shape[k] = s; c.bps[k] = 0; }
    rs = trial(c, t);
    for (int k = 0; k < LRK_COUNT && rs == LR_OK; ++k)
      if (k != LRK_MIXED && t[k] < bestt[k]) { bestt[k] = t[k]; best.shape[k] = s; best.bps[k] = 0; }
    if (rs == LR_OK && s == 0) bestt[LRK_MIXED] = t[LRK_MIXED];
  }
  // 2. persistent blocks per SM at each kernel's best shape
  for (int q = 1; q < NBPS && rs == LR_OK; ++q) {
    Schedule c = best;
    for (int k = 0; k < LRK_COUNT; ++k) c.bps[k] = BPS_OPTIONS[q];
    rs = trial(c, t);
    for (int k = 0; k < LRK_COUNT && rs == LR_OK; ++k)
      if (k != LRK_MIXED && t[k] < bestt[k]) { bestt[k] = t[k]; best.bps[k] = BPS_OPTIONS[q]; }
  }
  // 3. lanes per mixed cell
  for (int q = 0; q < 3 && rs == LR_OK; ++q) {
    Schedule c = best;
    c.lanes = LANE_OPTIONS[q];
    if (c.lanes == best.lanes) continue;
    rs = trial(c, t);
    if (rs == LR_OK && t[LRK_MIXED] < bestt[LRK_MIXED]) { bestt[LRK_MIXED] = t[LRK_MIXED]; best.lanes = c.lanes; }
  }
  // 4. unless the caller chose, the whole step: the tuned per-kernel step
  // against the persistent step (CUDA events around trial_steps steps each)
  bool pers = pers0;
  if (rs == LR_OK && !b->persistent_set && b->pers_bps > 0) {
    double ms[2] = {0.0, 0.0};
    for (int q = 0; q < 2 && rs == LR_OK; ++q) {
      b->sch = best;
      b->persistent = q == 1;
      b->need_rebuild = true;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rs = LR_ERR_CUDA;
      } else {
        rs = run_steps(b, 1);  // warm-up (tables and graphs)
        if (rs == LR_OK && cudaEventRecord(e0, b->stream) != cudaSuccess) rs = LR_ERR_CUDA;
        if (rs == LR_OK) rs = run_steps(b, trial_steps);
        if (rs == LR_OK && cudaEventRecord(e1, b->stream) != cudaSuccess) rs = LR_ERR_CUDA;
        float el = 0.0f;
        if (rs == LR_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&el, e0, e1) != cudaSuccess))
          rs = LR_ERR_CUDA;
        ms[q] = el;
        if (rs == LR_OK) rs = check_barrier(b);
        if (rs == LR_OK) rs = restore();
      }
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
    }
    if (rs == LR_OK) pers = ms[1] < ms[0];
  }
  cudaFree(snap);
  b->sch = best;
  b->persistent = pers;
  b->need_rebuild = true;
  if (rs != LR_OK) return rs;
  // the members' grids carry the lanes of lr_mixed only through the launch
  return LR_OK;
}

}  // extern "C"
