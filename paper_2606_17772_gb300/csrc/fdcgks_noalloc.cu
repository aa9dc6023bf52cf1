// Allocation-free CFL time step: a variant of the CFL reduction of
// fdcgks_api.cu that works on the caller's own state arrays and keeps its
// per-tile partial maxima in a fixed device array owned by the library
// instead of memory obtained from cudaMalloc.
//
// Some callers cannot allocate device memory at the moment they need a time
// step: applications that hand the library a fixed share of the GPU's memory
// and forbid further allocations, or time loops that must not risk an
// allocation failure or the implicit synchronisation that cudaMalloc and
// cudaFree can cause.  They keep their state in their own buffers and call
// fdcgks_cfl_dt_noalloc, which needs neither a context nor any allocation.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/fdcgks.h"
#include "fdcgks_internal.cuh"

namespace {

const int TILE_THREADS = 256;
const int TILE_NODES = FDCGKS_NOALLOC_TILE_NODES;    // nodes reduced by one block
const int MAX_TILES = FDCGKS_NOALLOC_MAX_TILES;

// Partial maxima (wave rate, kinematic viscosity) of each tile, then the
// final pair in the last two slots.  Every GPU that loads the library holds
// this array until the process exits; all calls share it, and it keeps the
// contents of the last call.
static __device__ __align__(256) double g_cfl_scratch[2 * MAX_TILES + 2];

// host-side addresses of g_cfl_scratch, one per device, filled on first use
// and kept for the process (valid while the device's primary context lives)
const int MAX_DEVICES = 64;
static void* g_scratch_addr[MAX_DEVICES];
static std::mutex g_scratch_lock;

__global__ void cfl_tiles_kernel(const double* Wp, const double* Wd, long np, long nd, double gamma, double mu,
                                 double ihx, double ihy, double* partial) {
  const long base = (long)blockIdx.x * TILE_NODES;
  double rate = 0.0, numax = 0.0;
  for (int k = threadIdx.x; k < TILE_NODES; k += TILE_THREADS) {
    long t = base + k;
    if (t >= np + nd) break;
    const double* W = t < np ? Wp : Wd;
    long n = t < np ? np : nd;
    long q = t < np ? t : t - np;
    double r = W[q], U = W[n + q] / r, V = W[2 * n + q] / r;
    double p = (gamma - 1.0) * (W[3 * n + q] - 0.5 * r * (U * U + V * V));
    double c = sqrt(gamma * p / r);
    rate = fmax(rate, fmax((fabs(U) + c) * ihx, (fabs(V) + c) * ihy));
    numax = fmax(numax, mu / r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
    numax = fmax(numax, __shfl_xor_sync(0xffffffffu, numax, o));
  }
  __shared__ double sr[TILE_THREADS / 32], sn[TILE_THREADS / 32];
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) { sr[w] = rate; sn[w] = numax; }
  __syncthreads();
  if (threadIdx.x == 0) {   // rate, numax already hold warp 0's maxima
    for (int k = 1; k < TILE_THREADS / 32; ++k) { rate = fmax(rate, sr[k]); numax = fmax(numax, sn[k]); }
    partial[2 * blockIdx.x] = rate;
    partial[2 * blockIdx.x + 1] = numax;
  }
}

// one block folds the partials of this call's tiles into the final pair
__global__ void cfl_final_kernel(double* partial, int tiles) {
  double rate = 0.0, numax = 0.0;
  for (int k = threadIdx.x; k < tiles; k += blockDim.x) {
    rate = fmax(rate, partial[2 * k]);
    numax = fmax(numax, partial[2 * k + 1]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
    numax = fmax(numax, __shfl_xor_sync(0xffffffffu, numax, o));
  }
  __shared__ double sr[32], sn[32];
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) { sr[w] = rate; sn[w] = numax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x / 32); ++k) { rate = fmax(rate, sr[k]); numax = fmax(numax, sn[k]); }
    rate = fmax(rate, sr[0]);
    numax = fmax(numax, sn[0]);
    partial[2 * MAX_TILES] = rate;
    partial[2 * MAX_TILES + 1] = numax;
  }
}

// failures are reported through fdcgks_last_error(NULL)
fdcgks_status nfail(fdcgks_status s, const char* msg, cudaError_t e = cudaSuccess) {
  char m[300];
  if (e != cudaSuccess) snprintf(m, sizeof(m), "%s: %s", msg, cudaGetErrorString(e));
  else snprintf(m, sizeof(m), "%s", msg);
  fdk::set_global_error(m);
  return s;
}

// Device address of g_cfl_scratch for the current device.  In host code the
// symbol's name only stands in for the device array; its address must be
// obtained from the runtime, once per device, with that device current.
fdcgks_status scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail(FDCGKS_ERR_CUDA, "cudaGetDevice", e);
  if (dev < 0 || dev >= MAX_DEVICES) return nfail(FDCGKS_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> guard(g_scratch_lock);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_cfl_scratch);
    if (e != cudaSuccess || !p) return nfail(FDCGKS_ERR_CUDA, "cudaGetSymbolAddress(g_cfl_scratch)", e);
    g_scratch_addr[dev] = p;
  }
  *out = (double*)g_scratch_addr[dev];
  return FDCGKS_OK;
}

}  // namespace

extern "C" fdcgks_status fdcgks_cfl_dt_noalloc(const fdcgks_params* p, const double* Wp, const double* Wd, double cfl,
                                               double* dt_out) {
  if (!p || !Wp || !Wd || !dt_out) return nfail(FDCGKS_ERR_ARG, "NULL argument");
  if (p->nx < 1 || p->ny < 1) return nfail(FDCGKS_ERR_ARG, "nx and ny must be >= 1");
  if (!(p->x1 > p->x0) || !(p->y1 > p->y0)) return nfail(FDCGKS_ERR_ARG, "domain extents must be positive");
  if (!(p->gamma > 1.0) || !(p->mu >= 0.0)) return nfail(FDCGKS_ERR_ARG, "gamma must be > 1 and mu >= 0");
  if (!(cfl > 0.0) || !std::isfinite(cfl)) return nfail(FDCGKS_ERR_ARG, "cfl must be positive and finite");
  const long nxd = p->nx + (p->bc[0] == FDCGKS_BC_PERIODIC ? 0 : 1);
  const long nyd = p->ny + (p->bc[2] == FDCGKS_BC_PERIODIC ? 0 : 1);
  const long np = (long)p->nx * p->ny, nd = nxd * nyd;
  const long tiles = (np + nd + TILE_NODES - 1) / TILE_NODES;
  if (tiles > MAX_TILES) {
    char m[200];
    snprintf(m, sizeof(m), "%ld nodes exceed the allocation-free limit of %ld nodes (%d tiles of %d)", np + nd,
             (long)MAX_TILES * TILE_NODES, MAX_TILES, TILE_NODES);
    return nfail(FDCGKS_ERR_ARG, m);
  }
  double* scratch = nullptr;
  fdcgks_status st = scratch_for_current_device(&scratch);
  if (st != FDCGKS_OK) return st;
  cudaStream_t s = (cudaStream_t)p->stream;
  const double hx = (p->x1 - p->x0) / p->nx, hy = (p->y1 - p->y0) / p->ny;
  cfl_tiles_kernel<<<(unsigned)tiles, TILE_THREADS, 0, s>>>(Wp, Wd, np, nd, p->gamma, p->mu, 1.0 / hx, 1.0 / hy,
                                                          scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return nfail(FDCGKS_ERR_CUDA, "cfl tile kernel", e);
  cfl_final_kernel<<<1, 1024, 0, s>>>(scratch, (int)tiles);
  e = cudaGetLastError();
  if (e != cudaSuccess) return nfail(FDCGKS_ERR_CUDA, "cfl final kernel", e);
  double h[2] = {0.0, 0.0};
  e = cudaMemcpyAsync(h, scratch + 2 * MAX_TILES, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return nfail(FDCGKS_ERR_CUDA, "reading the reduced maxima", e);
  if (!(h[0] > 0.0) || !std::isfinite(h[0])) return nfail(FDCGKS_ERR_NONPHYSICAL, "no finite wave speed");
  double dt = cfl / h[0];
  if (h[1] > 0.0) {
    double hm = std::fmin(hx, hy);
    dt = std::fmin(dt, cfl * hm * hm / (8.0 * h[1]));
  }
  *dt_out = dt;
  return FDCGKS_OK;
}
