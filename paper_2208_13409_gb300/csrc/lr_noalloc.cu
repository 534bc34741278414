// lr_noalloc.cu -- lr_cfl_dt_noalloc: the CFL time-step reduction over a
// state that lives in caller-owned device memory, using only a fixed scratch
// array compiled into the library (no cudaMalloc, no cudaFree, no allocating
// library call on any path).
//
// Who needs it: code that may not allocate device memory at the moment it
// asks for a time step -- for example a host application whose device memory
// is entirely reserved by another framework's caching allocator, or a
// latency-critical loop that must not hit cudaMalloc (which can synchronise
// the device and can fail when memory is fragmented).  Such callers hand in
// their own state arrays and their own one-double output.
//
// The scratch below is shared by every call in the process: a call
// overwrites what the previous call left, and calls whose work overlaps on
// the GPU (two streams, or two host threads) race on it.  Serialise them.
// The scratch's device address is looked up once per device and kept; a
// device reset (cudaDeviceReset) invalidates it, so no call may follow a
// reset of the device in the same process.
#include "../../include/lr.h"

#include <cuda_runtime.h>
#include <math.h>
#include <mutex>

#define LR_NOALLOC_MAX_CELLS (1 << 20)   // 8 MiB of per-cell scratch
#define LR_NOALLOC_MAX_DEVICES 64

namespace {

// [0 .. MAX_CELLS): per-cell CFL sound speed; then 2 reduction words.
static __device__ __align__(256) double g_noalloc_scratch[LR_NOALLOC_MAX_CELLS + 32];

constexpr double kEpsC = 1e-3;  // same sound-speed weight min(1, k/1e-3) as lr_step

struct NaGrid {
  int nx, ny, M, perx, pery, nxu, nyu;
  double hmin, cfl;
  double gam[3], pin[3];
};

// Order-preserving key of a value >= 0 (or NaN, which orders above every
// number, so a NaN anywhere reaches the result).
__device__ __forceinline__ unsigned long long na_key(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

__device__ __forceinline__ int na_map(int i, int n, int per) {
  if (per) return (i + n) % n;
  if (i < 0) return -1 - i;
  if (i >= n) return 2 * n - 1 - i;
  return i;
}

// Pass 1: c_c = max_a min(1, k_a/1e-3) sqrt(c_a^2) of every cell into scratch
// (NaN for a cell whose state is not finite or where a material of full
// weight has c^2 <= 0); thread 0 also clears the two reduction words.
__global__ void na_sound(NaGrid g, const double* k, const double* r, const double* e, double* scr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  size_t nc = (size_t)g.nx * g.ny;
  if (i == 0 && j == 0) {
    unsigned long long* red = reinterpret_cast<unsigned long long*>(scr + LR_NOALLOC_MAX_CELLS);
    red[0] = 0ull;
    red[1] = 0ull;
  }
  if (i >= g.nx || j >= g.ny) return;
  size_t c = (size_t)j * g.nx + i;
  double cmax = 0.0;
  bool bad = false;
  for (int a = 0; a < g.M; ++a) {
    double ka = k[a * nc + c];
    if (isnan(ka)) bad = true;
    if (!(ka > 0.0)) continue;
    double ra = r[a * nc + c], ea = e[a * nc + c];
    double pa = (g.gam[a] - 1.0) * ra * ea - g.pin[a];
    double c2 = (g.gam[a] * pa + g.pin[a]) / ra;
    double wgt = ka / kEpsC < 1.0 ? ka / kEpsC : 1.0;
    if (!isfinite(ka) || !isfinite(ra) || !isfinite(ea) || !isfinite(c2) || (wgt >= 1.0 && !(c2 > 0.0))) bad = true;
    double ca = sqrt(c2 > 0.0 ? c2 : 0.0);
    if (wgt * ca > cmax) cmax = wgt * ca;
  }
  scr[c] = bad ? __longlong_as_double(0x7ff8000000000000ll) : cmax;
}

// Pass 2: max over nodes of (max over the node's cells of c_c) + |u_p|; the
// last block writes dt = cfl * min(dx,dy) / max to *dt_out.
__global__ void na_reduce(NaGrid g, const double* ux, const double* uy, double* scr, double* dt_out) {
  __shared__ unsigned long long sm[32];
  __shared__ int last;
  unsigned long long* red = reinterpret_cast<unsigned long long*>(scr + LR_NOALLOC_MAX_CELLS);
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  unsigned long long v = 0ull;  // key of max over the node's cells of c_c, plus |u_p|
  if (i < g.nxu && j < g.nyu) {
    size_t n = (size_t)j * (g.nx + 1) + i;
    unsigned long long cm = 0ull;
    for (int b = -1; b <= 0; ++b)
      for (int a = -1; a <= 0; ++a) {
        size_t c = (size_t)na_map(j + b, g.ny, g.pery) * g.nx + na_map(i + a, g.nx, g.perx);
        unsigned long long kc = na_key(scr[c]);
        cm = kc > cm ? kc : cm;
      }
    v = na_key(__longlong_as_double((long long)cm) + sqrt(ux[n] * ux[n] + uy[n] * uy[n]));
  }
  int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int off = 16; off > 0; off >>= 1) {
    unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
    v = o > v ? o : v;
  }
  if ((tid & 31) == 0) sm[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    int nw = (blockDim.x * blockDim.y) >> 5;
    unsigned long long x = tid < nw ? sm[tid] : 0ull;
    for (int off = 16; off > 0; off >>= 1) {
      unsigned long long o = __shfl_xor_sync(0xffffffffu, x, off);
      x = o > x ? o : x;
    }
    if (tid == 0) {
      atomicMax(&red[0], x);
      __threadfence();
      unsigned long long nb = (unsigned long long)gridDim.x * gridDim.y;
      last = atomicAdd(&red[1], 1ull) == nb - 1;
    }
  }
  __syncthreads();
  if (last && tid == 0) {
    __threadfence();
    double mx = __longlong_as_double((long long)atomicAdd(&red[0], 0ull));
    // a NaN or infinite maximum (a state that is not finite, or a material
    // without a real sound speed) gives a NaN time step
    *dt_out = !isfinite(mx) ? __longlong_as_double(0x7ff8000000000000ll) : g.cfl * (mx > 0.0 ? g.hmin / mx : 1e300);
  }
}

std::mutex g_setup_mu;
double* g_scratch_ptr[LR_NOALLOC_MAX_DEVICES];

}  // namespace

extern "C" lr_status lr_cfl_dt_noalloc(const lr_config* cfg, const lr_material* mats,
                                       const double* k, const double* rho, const double* e,
                                       const double* ux, const double* uy, double* dt_out) {
  if (!cfg || !mats || !k || !rho || !e || !ux || !uy || !dt_out) return LR_ERR_ARG;
  if (cfg->nx < 2 || cfg->ny < 2 || cfg->nmat < 1 || cfg->nmat > 3) return LR_ERR_ARG;
  if ((long long)cfg->nx * cfg->ny > LR_NOALLOC_MAX_CELLS) return LR_ERR_ARG;  // beyond the fixed scratch
  if (!(cfg->x1 > cfg->x0) || !(cfg->y1 > cfg->y0) || !(cfg->cfl > 0.0) || cfg->cfl > 1.0) return LR_ERR_ARG;
  for (int q = 0; q < 4; ++q)
    if (cfg->bc[q] != LR_BC_REFLECT && cfg->bc[q] != LR_BC_PERIODIC) return LR_ERR_ARG;
  if (cfg->bc[0] != cfg->bc[1] || cfg->bc[2] != cfg->bc[3]) return LR_ERR_ARG;
  if ((cfg->bc[0] == LR_BC_PERIODIC && cfg->nx < 3) || (cfg->bc[2] == LR_BC_PERIODIC && cfg->ny < 3)) return LR_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= LR_NOALLOC_MAX_DEVICES) return LR_ERR_CUDA;
  double* scr;
  {
    // one-time set-up per device, with that device current: the host-side
    // symbol is only a stand-in, the kernels need its device address
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LR_ERR_CUDA;
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scr = g_scratch_ptr[dev];
  }
  NaGrid g;
  g.nx = cfg->nx; g.ny = cfg->ny; g.M = cfg->nmat;
  g.perx = cfg->bc[0] == LR_BC_PERIODIC;
  g.pery = cfg->bc[2] == LR_BC_PERIODIC;
  g.nxu = g.perx ? g.nx : g.nx + 1;
  g.nyu = g.pery ? g.ny : g.ny + 1;
  double dx = (cfg->x1 - cfg->x0) / cfg->nx, dy = (cfg->y1 - cfg->y0) / cfg->ny;
  g.hmin = dx < dy ? dx : dy;
  g.cfl = cfg->cfl;
  for (int a = 0; a < 3; ++a) {
    g.gam[a] = a < g.M ? mats[a].gamma : 1.4;
    g.pin[a] = a < g.M ? mats[a].pi : 0.0;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cfg->cuda_stream);
  dim3 blk(32, 8);
  na_sound<<<dim3((g.nx + 31) / 32, (g.ny + 7) / 8), blk, 0, s>>>(g, k, rho, e, scr);
  na_reduce<<<dim3((g.nxu + 31) / 32, (g.nyu + 7) / 8), blk, 0, s>>>(g, ux, uy, scr, dt_out);
  return cudaGetLastError() == cudaSuccess ? LR_OK : LR_ERR_CUDA;
}
