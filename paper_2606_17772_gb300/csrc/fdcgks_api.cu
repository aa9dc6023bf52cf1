// Host runtime and C entry points of the FD-CGKS library: context and device
// buffers, ghost-layer fill, CFL reduction, stage sequencing of the S2O4 step.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/fdcgks.h"
#include "fdcgks_internal.cuh"
#include "fdcgks_replay.h"

using namespace fdk;
using fdk::check_params;

struct fdcgks_ctx {
  fdcgks_params p;
  Layout L;
  double hx, hy;
  cudaStream_t stream;
  double* S = nullptr;      // state [2][12][plane] (FP64 path; staging of set/get_state in the mixed path)
  double* S2 = nullptr;     // stage state (FP64 path)
  // mixed path: the state as float-float pairs (high parts with ghost layers,
  // read by the nodal/point kernels), the stage state (high parts) and the
  // S2O4 accumulators as pairs
  float* Sf = nullptr;
  float* Slo = nullptr;
  float* S2f = nullptr;
  float* Acc_hi = nullptr;
  float* Acc_lo = nullptr;
  float* Gb_hi = nullptr;
  float* Gb_lo = nullptr;
  double* Wacc = nullptr;   // [2][4][plane]
  double* gB = nullptr;     // [2][8][plane]
  void* NF = nullptr;       // nodal fluxes [2][16][plane] of the compute type
  void* PA = nullptr;       // point outputs [50][pplane]
  void* PB = nullptr;
  int* flag = nullptr;      // device flags
  double* red = nullptr;    // reduction scratch
  int red_blocks = 0;
  bool has_state = false;
  // kernel-class timing with CUDA events on the context stream (optional)
  int profiling = 0;
  cudaEvent_t* ev = nullptr;  // event pool
  int ev_cap = 0, ev_used = 0;
  int* ev_class = nullptr;    // class of the interval that ends at event 2k+1
  long long launches = 0;     // kernels launched by the stepping path
  // split sides (fdcgks_set_sides) and the context time they are evaluated at
  bool has_sides = false;
  fdcgks_side sides[4];
  double t = 0.0;
  char err[512];
};

static char g_err[512] = "";

void fdk::set_global_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

bool fdk::ctx_view(fdcgks_t c, CtxView* v) {
  if (!c || !v) return false;
  v->p = c->p;
  v->L = c->L;
  v->hx = c->hx;
  v->hy = c->hy;
  v->stream = c->stream;
  v->S = c->S;
  v->has_state = c->has_state;
  v->has_sides = c->has_sides;
  return true;
}

void fdk::ctx_set_error(fdcgks_t c, const char* msg) {
  if (c) snprintf(c->err, sizeof(c->err), "%s", msg);
  else set_global_error(msg);
}

static fdcgks_status fail(fdcgks_t c, fdcgks_status s, const char* fmt, ...) {
  char* dst = c ? c->err : g_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return s;
}

#define CUDA_TRY(ctx, expr)                                                                              \
  do {                                                                                                   \
    cudaError_t e_ = (expr);                                                                             \
    if (e_ != cudaSuccess) return fail(ctx, FDCGKS_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                              \
  } while (0)

// ---------------------------------------------------------------------------
// run constants
// ---------------------------------------------------------------------------
const char* fdk::check_params(const fdcgks_params* p) {
  if (!p) return "params is NULL";
  if (p->nx < 1 || p->ny < 1) return "nx and ny must be >= 1";
  if (p->nx > (1 << 20) || p->ny > (1 << 20)) return "nx or ny too large";
  if (!(p->x1 > p->x0) || !(p->y1 > p->y0)) return "domain extents must be positive";
  if (!(p->gamma > 1.0) || !std::isfinite(p->gamma)) return "gamma must be > 1";
  if (!(p->mu >= 0.0) || !std::isfinite(p->mu)) return "mu must be >= 0";
  if (!(p->Pr > 0.0) || !std::isfinite(p->Pr)) return "Pr must be > 0";
  for (int k = 0; k < 4; ++k)
    if (p->bc[k] < 0 || p->bc[k] > 3) return "unknown boundary condition";
  for (int d = 0; d < 2; ++d)
    if ((p->bc[2 * d] == FDCGKS_BC_PERIODIC) != (p->bc[2 * d + 1] == FDCGKS_BC_PERIODIC))
      return "periodic boundaries must be paired";
  if ((p->bc[0] != FDCGKS_BC_PERIODIC && p->nx < 3) || (p->bc[2] != FDCGKS_BC_PERIODIC && p->ny < 3))
    return "a bounded direction needs at least 3 nodes";
  if (p->flux_variant != 62 && p->flux_variant != 64) return "flux_variant must be 62 or 64";
  if (p->geno_variant < 0 || p->geno_variant > 2) return "geno_variant must be 0, 1 or 2";
  if (p->grad_base != 0 && p->grad_base != 1) return "grad_base must be 0 or 1";
  if (p->precision != FDCGKS_FP64 && p->precision != FDCGKS_MIXED) return "precision must be 0 or 1";
  if (!(p->tau_c1 >= 0.0) || !(p->tau_c2 >= 0.0)) return "tau constants must be >= 0";
  if (p->recon_vars != 0 && p->recon_vars != 1) return "recon_vars must be 0 or 1";
  return nullptr;
}

static size_t rsize(const fdcgks_params& p) { return p.precision == FDCGKS_MIXED ? sizeof(float) : sizeof(double); }

// ---------------------------------------------------------------------------
// ghost fill: periodic wrap, mirror (symmetry / no-slip) or constant
// extrapolation (transmissive); x pass over interior rows, then y pass over
// all columns so that corners are filled consistently
// ---------------------------------------------------------------------------
template <class T>
__global__ void ghost_kernel(T* S, Layout L, int bc0, int bc1, int dir) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  ghost_body(S, L, bc0, bc1, dir, blockIdx.z, idx);
}

template <class T>
__global__ void ghost_sides_kernel(T* S, Layout L, GhostSides gs, int dir) {
  ghost_body_sides(S, L, gs, dir, blockIdx.z, blockIdx.x * blockDim.x + threadIdx.x);
}

// split sides evaluated at time t
static GhostSides ghost_sides(fdcgks_t c, double t) {
  GhostSides gs;
  const double gm1 = c->p.gamma - 1.0;
  for (int k = 0; k < 4; ++k) {
    const fdcgks_side& sd = c->sides[k];
    gs.split[k] = std::fma(sd.split_speed, t, sd.split0);
    for (int q = 0; q < 2; ++q) {
      gs.kind[k][q] = sd.kind[q];
      const double* pr = sd.prim[q];
      gs.W[k][q][0] = pr[0];
      gs.W[k][q][1] = pr[0] * pr[1];
      gs.W[k][q][2] = pr[0] * pr[2];
      gs.W[k][q][3] = pr[3] / gm1 + 0.5 * pr[0] * (pr[1] * pr[1] + pr[2] * pr[2]);
    }
  }
  gs.x0 = c->p.x0;
  gs.y0 = c->p.y0;
  gs.hx = c->hx;
  gs.hy = c->hy;
  return gs;
}

// ghost layers at stage time t (t matters only for split sides)
template <class T>
static cudaError_t fill_ghosts(fdcgks_t c, T* S, double t) {
  const Layout& L = c->L;
  int tx = (L.ny > L.nyd ? L.ny : L.nyd) * 2 * GH;
  int ty = ((L.nx > L.nxd ? L.nx : L.nxd) + 2 * GH) * 2 * GH;
  if (c->has_sides) {
    const GhostSides gs = ghost_sides(c, t);
    ghost_sides_kernel<T><<<dim3((tx + 127) / 128, 1, 2), 128, 0, c->stream>>>(S, L, gs, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ghost_sides_kernel<T><<<dim3((ty + 127) / 128, 1, 2), 128, 0, c->stream>>>(S, L, gs, 1);
    return cudaGetLastError();
  }
  ghost_kernel<T><<<dim3((tx + 127) / 128, 1, 2), 128, 0, c->stream>>>(S, L, c->p.bc[0], c->p.bc[1], 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ghost_kernel<T><<<dim3((ty + 127) / 128, 1, 2), 128, 0, c->stream>>>(S, L, c->p.bc[2], c->p.bc[3], 1);
  return cudaGetLastError();
}

// mixed path: FP64 state <-> float-float pairs (whole padded planes)
__global__ void split_ff_kernel(const double* S, float* hi, float* lo, long n) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    float h = (float)S[t];
    hi[t] = h;
    lo[t] = (float)(S[t] - (double)h);
  }
}
__global__ void join_ff_kernel(const float* hi, const float* lo, double* S, long n) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    S[t] = (double)hi[t] + (double)lo[t];
}

cudaError_t fdk::launch_split_ff(const double* S, float* hi, float* lo, long n, cudaStream_t s) {
  split_ff_kernel<<<1024, 256, 0, s>>>(S, hi, lo, n);
  return cudaGetLastError();
}
cudaError_t fdk::launch_join_ff(const float* hi, const float* lo, double* S, long n, cudaStream_t s) {
  join_ff_kernel<<<1024, 256, 0, s>>>(hi, lo, S, n);
  return cudaGetLastError();
}

static cudaError_t join_state(fdcgks_t c) {
  if (!c->Sf) return cudaSuccess;
  return launch_join_ff(c->Sf, c->Slo, c->S, 2L * NFLD * c->L.plane, c->stream);
}

// ---------------------------------------------------------------------------
// state validation and CFL reduction
// ---------------------------------------------------------------------------
__global__ void validate_kernel(const double* S, Layout L, double gamma, int* flag) {
  const int g = blockIdx.z;
  const int nxg = g == 0 ? L.nx : L.nxd, nyg = g == 0 ? L.ny : L.nyd;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= nxg || j >= nyg) return;
  const double* Sg = S + (long)g * NFLD * L.plane;
  const long c0 = cell(L, i, j);
  double r = Sg[c0], mu_ = Sg[L.plane + c0], mv_ = Sg[2 * L.plane + c0], E = Sg[3 * L.plane + c0];
  double p = (gamma - 1.0) * (E - 0.5 * (mu_ * mu_ + mv_ * mv_) / r);
  bool ok = r > 0.0 && p > 0.0 && r < INFINITY && p < INFINITY;
  for (int f = 4; f < NFLD; ++f) ok = ok && fabs(Sg[(long)f * L.plane + c0]) < INFINITY;
  if (!ok) atomicOr(flag, 1);
}

cudaError_t fdk::launch_validate(const double* S, const Layout& L, double gamma, int* flag, cudaStream_t s) {
  const int mx = L.nx > L.nxd ? L.nx : L.nxd, my = L.ny > L.nyd ? L.ny : L.nyd;
  validate_kernel<<<dim3((mx + 127) / 128, my, 2), 128, 0, s>>>(S, L, gamma, flag);
  return cudaGetLastError();
}

// the rates of cfl_rates added over the directions, (|U|+c)/hx + (|V|+c)/hy
// (the two-dimensional form of the CFL bound), and nu = mu/rho, folded into
// running maxima
__device__ void cfl_rates_sum(double r, double ru, double rv, double E, double gamma, double mu, double ihx,
                              double ihy, double& rate, double& numax) {
  const double ir = 1.0 / r;
  const double U = ru * ir, V = rv * ir;
  const double p = (gamma - 1.0) * (E - 0.5 * r * (U * U + V * V));
  const double cs = sqrt(gamma * p * ir);
  rate = fmax(rate, (fabs(U) + cs) * ihx + (fabs(V) + cs) * ihy);
  numax = fmax(numax, mu * ir);
}

// the state the CFL reduction reads: FP64 entries, or the mixed path's
// float-float pairs joined in FP64 (no FP64 copy of the state is made); est
// gives the FP32 rounding of an entry (the high part of a pair)
struct StateF64 {
  const double* S;
  __device__ double operator()(long k) const { return S[k]; }
  __device__ float est(long k) const { return (float)S[k]; }
};
struct StatePair {
  const float* hi;
  const float* lo;
  __device__ double operator()(long k) const { return (double)hi[k] + (double)lo[k]; }
  __device__ float est(long k) const { return hi[k]; }
};

// Work split of the CFL passes: the rows of both grids (primary first), each
// cut into segments of CFL_SEG nodes; an item is one segment of one row.
// The FP32 constants of the screening go with it.
const int CFL_SEG = 1024;
struct CflGrid {
  Layout L;
  int segs;   // segments per row (of the wider grid)
  double gamma, mu, ihx, ihy;
  float gf, muf, ihxf, ihyf;
  int sum;
};

// Calls f(c0) for the node offset c0 of every node of item `it`
template <class F>
__device__ __forceinline__ void cfl_item(const CflGrid& G, int it, F f) {
  const Layout& L = G.L;
  const int row = it / G.segs, seg = it - row * G.segs;
  const int g = row < L.ny ? 0 : 1, j = g == 0 ? row : row - L.ny;
  const int nxg = g == 0 ? L.nx : L.nxd;
  const int i1 = min(nxg, (seg + 1) * CFL_SEG);
  const long base = (long)g * NFLD * L.plane;
  for (int i = seg * CFL_SEG + threadIdx.x; i < i1; i += blockDim.x) f(base + cell(L, i, j));
}

// block-wide maxima of two values (>= 0) into thread 0; blockDim.x <= 1024
template <class T>
__device__ __forceinline__ void block_max2(T& a, T& b, T* sa, T* sb) {
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  const int w = threadIdx.x / 32;
  if ((threadIdx.x & 31) == 0) { sa[w] = a; sb[w] = b; }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 1; k < (int)(blockDim.x / 32); ++k) { a = fmax(a, sa[k]); b = fmax(b, sb[k]); }
}

// First pass: the largest reliable FP32 estimates (cfl_estimate_f) of the
// rate and of nu over all nodes, folded into mxf[0..1] (zeroed before) with
// atomicMax on the bit patterns (non-negative floats order as their bits).
template <class ST>
__global__ void cfl_screen_kernel(ST S, CflGrid G, int items, unsigned* mxf) {
  __shared__ float sa[32], sb[32];
  float mr = 0.0f, mn = 0.0f;
  const long P = G.L.plane;
  for (int it = blockIdx.x; it < items; it += gridDim.x)
    cfl_item(G, it, [&](long c0) {
      float rt, nu;
      bool ok;
      cfl_estimate_f(S.est(c0), S.est(c0 + P), S.est(c0 + 2 * P), S.est(c0 + 3 * P), G.gf, G.muf, G.ihxf, G.ihyf,
                     G.sum != 0, rt, nu, ok);
      if (ok) {
        mr = fmaxf(mr, rt);
        mn = fmaxf(mn, nu);
      }
    });
  block_max2(mr, mn, sa, sb);
  if (threadIdx.x == 0) {
    if (mr > 0.0f) atomicMax(mxf, __float_as_uint(mr));
    if (mn > 0.0f) atomicMax(mxf + 1, __float_as_uint(mn));
  }
}

// Second pass: per-block maxima of the FP64 rate and nu, evaluated (from the
// FP64 entries or the joined pairs) only at nodes whose estimate is
// unreliable or within CFL_SCREEN_MARGIN of the first pass's maxima; the
// maxima are exactly those of evaluating every node.
template <class ST>
__global__ void cfl_kernel(ST S, CflGrid G, int items, const unsigned* mxf, double* out) {
  __shared__ double sa[32], sb[32];
  double rate = 0.0, numax = 0.0;
  const long P = G.L.plane;
  const float mr = __uint_as_float(mxf[0]), mn = __uint_as_float(mxf[1]);
  const float tr = mr * (1.0f - CFL_SCREEN_MARGIN);
  const float tn = mn > 0.0f ? mn * (1.0f - CFL_SCREEN_MARGIN) : INFINITY;   // mu = 0: nu never decides
  for (int it = blockIdx.x; it < items; it += gridDim.x)
    cfl_item(G, it, [&](long c0) {
      float rt, nu;
      bool ok;
      cfl_estimate_f(S.est(c0), S.est(c0 + P), S.est(c0 + 2 * P), S.est(c0 + 3 * P), G.gf, G.muf, G.ihxf, G.ihyf,
                     G.sum != 0, rt, nu, ok);
      if (ok && rt < tr && nu < tn) return;
      const double r = S(c0), ru = S(c0 + P), rv = S(c0 + 2 * P), E = S(c0 + 3 * P);
      if (G.sum)
        cfl_rates_sum(r, ru, rv, E, G.gamma, G.mu, G.ihx, G.ihy, rate, numax);
      else
        cfl_rates(r, ru, rv, E, G.gamma, G.mu, G.ihx, G.ihy, rate, numax);
    });
  block_max2(rate, numax, sa, sb);
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = rate;
    out[2 * blockIdx.x + 1] = numax;
  }
}

// ---------------------------------------------------------------------------
// optional timing of kernel classes (events recorded around each launch group)
// ---------------------------------------------------------------------------
enum { KC_GHOST = 0, KC_NODAL = 1, KC_POINTS = 2, KC_UPDATE = 3, KC_CFL = 4, KC_N = 5 };

static cudaError_t prof_mark(fdcgks_t c, int cls, bool begin) {
  if (!c->profiling) return cudaSuccess;
  if (c->ev_used + 1 > c->ev_cap) {
    int cap = c->ev_cap ? 2 * c->ev_cap : 256;
    cudaEvent_t* ev = new cudaEvent_t[cap];
    int* cl = new int[cap / 2];
    for (int k = 0; k < c->ev_cap; ++k) ev[k] = c->ev[k];
    for (int k = 0; k < c->ev_cap / 2; ++k) cl[k] = c->ev_class[k];
    for (int k = c->ev_cap; k < cap; ++k) {
      cudaError_t e = cudaEventCreate(&ev[k]);
      if (e != cudaSuccess) { delete[] ev; delete[] cl; return e; }
    }
    delete[] c->ev;
    delete[] c->ev_class;
    c->ev = ev;
    c->ev_class = cl;
    c->ev_cap = cap;
  }
  if (!begin) c->ev_class[c->ev_used / 2] = cls;
  return cudaEventRecord(c->ev[c->ev_used++], c->stream);
}

// ---------------------------------------------------------------------------
// stage sequencing
// ---------------------------------------------------------------------------
template <class R>
static KArgs<R> make_args(fdcgks_t c, double dt, const double* S, double* Sout, int want_n) {
  KArgs<R> a;
  std::memset(&a, 0, sizeof(a));
  a.L = c->L;
  a.S = S;
  a.Sn = c->S;
  a.Sout = Sout;
  a.Wacc = c->Wacc;
  a.gB = c->gB;
  a.NF = (R*)c->NF;
  a.PA = (R*)c->PA;
  a.PB = (R*)c->PB;
  a.geno = make_geno<R>(c->p.geno_variant);
  a.gas = make_gas<R>(c->p, dt);
  a.hd[0] = c->hx; a.hd[1] = c->hy;
  a.ihd[0] = 1.0 / c->hx; a.ihd[1] = 1.0 / c->hy;
  a.h[0] = (R)c->hx; a.h[1] = (R)c->hy;
  a.ih[0] = (R)(1.0 / c->hx); a.ih[1] = (R)(1.0 / c->hy);
  // the no-slip wall reset reads bc: an unsplit side's kind, else a non-wall kind
  for (int k = 0; k < 4; ++k)
    a.bc[k] = !c->has_sides ? c->p.bc[k]
                            : (c->sides[k].kind[0] == c->sides[k].kind[1] ? c->sides[k].kind[0] : FDCGKS_BC_FIXED);
  a.flux_variant = c->p.flux_variant;
  a.grad_base = c->p.grad_base;
  a.recon_vars = c->p.recon_vars;
  a.want_n = want_n;
  a.dt = dt;
  a.flag = c->flag;
  return a;
}

// precision-specific state pointers of one stage
static void stage_state(fdcgks_t c, int mode, KArgs<double>& a) {
  a.S = mode == UPD_STAGE2 ? c->S2 : c->S;
  a.Sout = mode == UPD_STAGE1 ? c->S2 : c->S;
  a.Sr = a.S;
}
static void stage_state(fdcgks_t c, int mode, KArgs<float>& a) {
  a.Sr = mode == UPD_STAGE2 ? c->S2f : c->Sf;
  a.Sn_hi = c->Sf;
  a.Sn_lo = c->Slo;
  a.Out_hi = mode == UPD_STAGE1 ? c->S2f : c->Sf;
  a.Out_lo = mode == UPD_STAGE1 ? nullptr : c->Slo;
  a.Acc_hi = c->Acc_hi;
  a.Acc_lo = c->Acc_lo;
  a.Gb_hi = c->Gb_hi;
  a.Gb_lo = c->Gb_lo;
}

template <class R>
static fdcgks_status run_stage(fdcgks_t c, double dt, int mode, double* const* op) {
  KArgs<R> a = make_args<R>(c, dt, nullptr, nullptr, mode != UPD_STAGE2);
  stage_state(c, mode, a);
  CUDA_TRY(c, prof_mark(c, KC_GHOST, true));
  CUDA_TRY(c, fill_ghosts(c, const_cast<R*>(a.Sr), mode == UPD_STAGE2 ? c->t + 0.5 * dt : c->t));
  CUDA_TRY(c, prof_mark(c, KC_GHOST, false));
  if (op)
    for (int k = 0; k < 8; ++k) a.op[k] = op[k];
  CUDA_TRY(c, prof_mark(c, KC_NODAL, true));
  CUDA_TRY(c, launch_nodal<R>(a, c->stream));
  CUDA_TRY(c, prof_mark(c, KC_NODAL, false));
  CUDA_TRY(c, prof_mark(c, KC_POINTS, true));
  CUDA_TRY(c, launch_points<R>(a, c->stream));
  CUDA_TRY(c, prof_mark(c, KC_POINTS, false));
  CUDA_TRY(c, prof_mark(c, KC_UPDATE, true));
  CUDA_TRY(c, launch_update<R>(a, mode, c->stream));
  CUDA_TRY(c, prof_mark(c, KC_UPDATE, false));
  c->launches += 6;   // 2 ghost passes, nodal, 2 point types, update
  return FDCGKS_OK;
}

template <class R>
static fdcgks_status run_step(fdcgks_t c, double dt) {
  fdcgks_status s = run_stage<R>(c, dt, UPD_STAGE1, nullptr);
  if (s != FDCGKS_OK) return s;
  s = run_stage<R>(c, dt, UPD_STAGE2, nullptr);
  if (s == FDCGKS_OK) c->t += dt;
  return s;
}

// Load a padded FP64 state [2][12][plane] (interior valid) into the context:
// the state itself on the FP64 path, split into float-float pairs on the
// mixed path (as fdcgks_set_state does, without validation).
fdcgks_status fdk::ctx_load_padded(fdcgks_t c, const double* in) {
  CUDA_TRY(c, cudaMemcpyAsync(c->S, in, sizeof(double) * 2 * NFLD * c->L.plane, cudaMemcpyDeviceToDevice,
                              c->stream));
  if (c->Sf) CUDA_TRY(c, launch_split_ff(c->S, c->Sf, c->Slo, 2L * NFLD * c->L.plane, c->stream));
  c->has_state = true;
  return FDCGKS_OK;
}

// One step of the context's own precision from the padded FP64 state `in`
// to `out`, through the context's buffers (its state is overwritten, its time
// kept).  A float-float pair joined to FP64 splits back into a pair of the
// same FP64 value; the low part keeps its bits unless it lies more than 29
// bits below the high part, when it loses those below 2^-53 of the value, so
// steps chained through FP64 buffers follow the mixed run to FP64 rounding.
fdcgks_status fdk::ctx_replay_step(fdcgks_t c, double dt, const double* in, double* out) {
  fdcgks_status s = ctx_load_padded(c, in);
  if (s != FDCGKS_OK) return s;
  const double t = c->t;
  s = c->p.precision == FDCGKS_MIXED ? run_step<float>(c, dt) : run_step<double>(c, dt);
  c->t = t;
  if (s != FDCGKS_OK) return s;
  CUDA_TRY(c, join_state(c));
  CUDA_TRY(c, cudaMemcpyAsync(out, c->S, sizeof(double) * 2 * NFLD * c->L.plane, cudaMemcpyDeviceToDevice,
                              c->stream));
  return FDCGKS_OK;
}

// ---------------------------------------------------------------------------
// C entry points
// ---------------------------------------------------------------------------
extern "C" {

const char* fdcgks_status_string(fdcgks_status s) {
  switch (s) {
    case FDCGKS_OK: return "ok";
    case FDCGKS_ERR_ARG: return "invalid argument";
    case FDCGKS_ERR_CUDA: return "CUDA error";
    case FDCGKS_ERR_NONPHYSICAL: return "non-physical state";
    case FDCGKS_ERR_STATE: return "no state loaded";
    case FDCGKS_ERR_TIMEOUT: return "device wait timed out";
    case FDCGKS_ERR_NOMEM: return "out of device memory";
  }
  return "unknown status";
}

const char* fdcgks_last_error(fdcgks_t ctx) { return ctx ? ctx->err : g_err; }

void fdcgks_destroy(fdcgks_t c) {
  if (!c) return;
  for (int k = 0; k < c->ev_cap; ++k) cudaEventDestroy(c->ev[k]);
  delete[] c->ev;
  delete[] c->ev_class;
  void* bufs[] = {c->S, c->S2, c->Sf, c->Slo, c->S2f, c->Acc_hi, c->Acc_lo, c->Gb_hi, c->Gb_lo,
                  c->Wacc, c->gB, c->NF, c->PA, c->PB, c->flag, c->red};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete c;
}

fdcgks_status fdcgks_create(const fdcgks_params* p, fdcgks_t* out) {
  if (!out) return fail(nullptr, FDCGKS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (const char* m = check_params(p)) return fail(nullptr, FDCGKS_ERR_ARG, "%s", m);
  fdcgks_t c = new (std::nothrow) fdcgks_ctx();
  if (!c) return fail(nullptr, FDCGKS_ERR_NOMEM, "host allocation failed");
  c->p = *p;
  c->err[0] = 0;
  c->stream = (cudaStream_t)p->stream;
  c->hx = (p->x1 - p->x0) / p->nx;
  c->hy = (p->y1 - p->y0) / p->ny;
  c->L = make_layout(*p);
  const Layout& L = c->L;
  const size_t rs = rsize(*p);
  const bool mixed = p->precision == FDCGKS_MIXED;
  const size_t fp = sizeof(float) * L.plane;
  struct { void** ptr; size_t bytes; } allocs[] = {
      {(void**)&c->S, sizeof(double) * 2 * NFLD * L.plane},
      {(void**)&c->S2, mixed ? 0 : sizeof(double) * 2 * NFLD * L.plane},
      {(void**)&c->Wacc, mixed ? 0 : sizeof(double) * 2 * 4 * L.plane},
      {(void**)&c->gB, mixed ? 0 : sizeof(double) * 2 * 8 * L.plane},
      {(void**)&c->Sf, mixed ? fp * 2 * NFLD : 0},
      {(void**)&c->Slo, mixed ? fp * 2 * NFLD : 0},
      {(void**)&c->S2f, mixed ? fp * 2 * NFLD : 0},
      {(void**)&c->Acc_hi, mixed ? fp * 2 * 4 : 0},
      {(void**)&c->Acc_lo, mixed ? fp * 2 * 4 : 0},
      {(void**)&c->Gb_hi, mixed ? fp * 2 * 8 : 0},
      {(void**)&c->Gb_lo, mixed ? fp * 2 * 8 : 0},
      {&c->NF, rs * 2 * NNF * L.plane},
      {&c->PA, rs * NPT * L.pplane},
      {&c->PB, rs * NPT * L.pplane},
      {(void**)&c->flag, sizeof(int) * 4},
  };
  for (auto& a : allocs) {
    if (a.bytes == 0) continue;
    cudaError_t e = cudaMalloc(a.ptr, a.bytes);
    if (e != cudaSuccess) {
      fail(nullptr, e == cudaErrorMemoryAllocation ? FDCGKS_ERR_NOMEM : FDCGKS_ERR_CUDA, "cudaMalloc(%zu): %s",
           a.bytes, cudaGetErrorString(e));
      fdcgks_destroy(c);
      return e == cudaErrorMemoryAllocation ? FDCGKS_ERR_NOMEM : FDCGKS_ERR_CUDA;
    }
  }
  c->red_blocks = 1024;
  // per-block maxima, then the two screening maxima (2 unsigned in one more double)
  if (cudaMalloc((void**)&c->red, sizeof(double) * (2 * c->red_blocks + 1)) != cudaSuccess) {
    fdcgks_destroy(c);
    return fail(nullptr, FDCGKS_ERR_NOMEM, "cudaMalloc of the reduction scratch failed");
  }
  // zero everything once so that ghost corners and unused entries are defined
  cudaError_t e = cudaSuccess;
  e = e == cudaSuccess ? cudaMemsetAsync(c->S, 0, sizeof(double) * 2 * NFLD * L.plane, c->stream) : e;
  if (c->S2) e = e == cudaSuccess ? cudaMemsetAsync(c->S2, 0, sizeof(double) * 2 * NFLD * L.plane, c->stream) : e;
  if (c->Sf) e = e == cudaSuccess ? cudaMemsetAsync(c->Sf, 0, sizeof(float) * 2 * NFLD * L.plane, c->stream) : e;
  if (c->S2f) e = e == cudaSuccess ? cudaMemsetAsync(c->S2f, 0, sizeof(float) * 2 * NFLD * L.plane, c->stream) : e;
  e = e == cudaSuccess ? cudaMemsetAsync(c->flag, 0, sizeof(int) * 4, c->stream) : e;
  e = e == cudaSuccess ? cudaStreamSynchronize(c->stream) : e;
  if (e != cudaSuccess) {
    fdcgks_destroy(c);
    return fail(nullptr, FDCGKS_ERR_CUDA, "initialisation: %s", cudaGetErrorString(e));
  }
  *out = c;
  return FDCGKS_OK;
}

fdcgks_status fdcgks_dims(fdcgks_t c, int* nx, int* ny, int* nxd, int* nyd) {
  if (!c) return fail(nullptr, FDCGKS_ERR_ARG, "ctx is NULL");
  if (nx) *nx = c->L.nx;
  if (ny) *ny = c->L.ny;
  if (nxd) *nxd = c->L.nxd;
  if (nyd) *nyd = c->L.nyd;
  return FDCGKS_OK;
}

// copy one interior field plane between a dense [ny][nx] array and the padded layout
static cudaError_t copy_field(fdcgks_t c, double* dev_plane, const double* src, double* dst, int nxg, int nyg,
                              bool to_dev, int on_device) {
  const Layout& L = c->L;
  double* d0 = dev_plane + cell(L, 0, 0);
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : (to_dev ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
  if (to_dev)
    return cudaMemcpy2DAsync(d0, sizeof(double) * L.pitch, src, sizeof(double) * nxg, sizeof(double) * nxg, nyg, k,
                             c->stream);
  return cudaMemcpy2DAsync(dst, sizeof(double) * nxg, d0, sizeof(double) * L.pitch, sizeof(double) * nxg, nyg, k,
                           c->stream);
}

// Dense state [grid][field][nyg][nxg] (the four caller arrays back to back:
// Wp, Gp, Wd, Gd) <-> the padded layout of both grids, on the device.
// blockIdx.z = grid * NFLD + field; rows strided over gridDim.y.
__global__ void dense_padded_kernel(double* dense, double* S, Layout L, int to_padded) {
  const int g = blockIdx.z / NFLD, f = blockIdx.z % NFLD;
  const int nxg = g == 0 ? L.nx : L.nxd, nyg = g == 0 ? L.ny : L.nyd;
  const long goff = g == 0 ? 0 : (long)NFLD * L.nx * L.ny;
  double* Sf = S + ((long)g * NFLD + f) * L.plane;
  for (int j = blockIdx.y; j < nyg; j += gridDim.y) {
    double* d = dense + goff + ((long)f * nyg + j) * nxg;
    double* p = Sf + cell(L, 0, j);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nxg; i += gridDim.x * blockDim.x) {
      if (to_padded) p[i] = d[i];
      else d[i] = p[i];
    }
  }
}

// Host state <-> device: the whole state in four contiguous copies through a
// dense staging area (the point-output buffer, free between steps), and one
// kernel between the staging area and the padded layout; contiguous copies
// run at the host link's full rate where per-row (pitched) copies do not.
// Returns false (nothing done) when the staging area is too small.
static bool staged_size_ok(fdcgks_t c) {
  const Layout& L = c->L;
  const size_t need = sizeof(double) * NFLD * ((size_t)L.nx * L.ny + (size_t)L.nxd * L.nyd);
  return need <= rsize(c->p) * NPT * (size_t)L.pplane;
}

static cudaError_t launch_dense_padded(fdcgks_t c, double* dense, int to_padded) {
  const Layout& L = c->L;
  const int mx = std::max(L.nx, L.nxd), my = std::max(L.ny, L.nyd);
  const dim3 grid((unsigned)std::min((mx + 255) / 256, 64), (unsigned)std::min(my, 65535), 2 * NFLD);
  dense_padded_kernel<<<grid, 256, 0, c->stream>>>(dense, c->S, L, to_padded);
  return cudaGetLastError();
}

static cudaError_t host_state_copy(fdcgks_t c, double* const* host, bool to_dev) {
  const Layout& L = c->L;
  double* st = (double*)c->PA;
  const long N0 = (long)L.nx * L.ny, N1 = (long)L.nxd * L.nyd;
  const long off[4] = {0, 4 * N0, NFLD * N0, NFLD * N0 + 4 * N1};
  const long len[4] = {4 * N0, 8 * N0, 4 * N1, 8 * N1};
  cudaError_t e = cudaSuccess;
  if (!to_dev) e = launch_dense_padded(c, st, 0);
  for (int k = 0; k < 4 && e == cudaSuccess; ++k)
    e = to_dev ? cudaMemcpyAsync(st + off[k], host[k], sizeof(double) * len[k], cudaMemcpyHostToDevice, c->stream)
               : cudaMemcpyAsync(host[k], st + off[k], sizeof(double) * len[k], cudaMemcpyDeviceToHost, c->stream);
  if (to_dev && e == cudaSuccess) e = launch_dense_padded(c, st, 1);
  return e;
}

fdcgks_status fdcgks_set_state(fdcgks_t c, const double* Wp, const double* Gp, const double* Wd, const double* Gd,
                               int on_device) {
  if (!c) return fail(nullptr, FDCGKS_ERR_ARG, "ctx is NULL");
  if (!Wp || !Gp || !Wd || !Gd) return fail(c, FDCGKS_ERR_ARG, "NULL state pointer");
  const Layout& L = c->L;
  if (!on_device && staged_size_ok(c)) {
    double* const host[4] = {const_cast<double*>(Wp), const_cast<double*>(Gp), const_cast<double*>(Wd),
                             const_cast<double*>(Gd)};
    CUDA_TRY(c, host_state_copy(c, host, true));
  } else {
    const double* srcW[2] = {Wp, Wd};
    const double* srcG[2] = {Gp, Gd};
    for (int g = 0; g < 2; ++g) {
      int nxg = g == 0 ? L.nx : L.nxd, nyg = g == 0 ? L.ny : L.nyd;
      long NN = (long)nxg * nyg;
      double* Sg = c->S + (long)g * NFLD * L.plane;
      for (int f = 0; f < NFLD; ++f) {
        const double* src = f < 4 ? srcW[g] + f * NN : srcG[g] + (f - 4) * NN;
        CUDA_TRY(c, copy_field(c, Sg + (long)f * L.plane, src, nullptr, nxg, nyg, true, on_device));
      }
    }
  }
  if (c->Sf) CUDA_TRY(c, launch_split_ff(c->S, c->Sf, c->Slo, 2L * NFLD * L.plane, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
  CUDA_TRY(c, launch_validate(c->S, L, c->p.gamma, c->flag, c->stream));
  int h = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&h, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (h) {
    c->has_state = false;
    CUDA_TRY(c, cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
    return fail(c, FDCGKS_ERR_NONPHYSICAL, "state has non-positive or non-finite density/pressure");
  }
  c->has_state = true;
  c->t = 0.0;
  return FDCGKS_OK;
}

fdcgks_status fdcgks_get_state(fdcgks_t c, double* Wp, double* Gp, double* Wd, double* Gd, int on_device) {
  if (!c) return fail(nullptr, FDCGKS_ERR_ARG, "ctx is NULL");
  if (!c->has_state) return fail(c, FDCGKS_ERR_STATE, "no state loaded");
  if (!Wp || !Gp || !Wd || !Gd) return fail(c, FDCGKS_ERR_ARG, "NULL state pointer");
  const Layout& L = c->L;
  CUDA_TRY(c, join_state(c));
  if (!on_device && staged_size_ok(c)) {
    double* const host[4] = {Wp, Gp, Wd, Gd};
    CUDA_TRY(c, host_state_copy(c, host, false));
  } else {
    double* dstW[2] = {Wp, Wd};
    double* dstG[2] = {Gp, Gd};
    for (int g = 0; g < 2; ++g) {
      int nxg = g == 0 ? L.nx : L.nxd, nyg = g == 0 ? L.ny : L.nyd;
      long NN = (long)nxg * nyg;
      double* Sg = c->S + (long)g * NFLD * L.plane;
      for (int f = 0; f < NFLD; ++f) {
        double* dst = f < 4 ? dstW[g] + f * NN : dstG[g] + (f - 4) * NN;
        CUDA_TRY(c, copy_field(c, Sg + (long)f * L.plane, nullptr, dst, nxg, nyg, false, on_device));
      }
    }
  }
  if (!on_device) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return FDCGKS_OK;
}

fdcgks_status fdcgks_steps(fdcgks_t c, double dt, int nsteps) {
  if (!c) return fail(nullptr, FDCGKS_ERR_ARG, "ctx is NULL");
  if (!c->has_state) return fail(c, FDCGKS_ERR_STATE, "no state loaded");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, FDCGKS_ERR_ARG, "dt must be positive and finite");
  if (nsteps < 0) return fail(c, FDCGKS_ERR_ARG, "nsteps must be >= 0");
  for (int s = 0; s < nsteps; ++s) {
    fdcgks_status st = c->p.precision == FDCGKS_MIXED ? run_step<float>(c, dt) : run_step<double>(c, dt);
    if (st != FDCGKS_OK) return st;
  }
  return FDCGKS_OK;
}

fdcgks_status fdcgks_step(fdcgks_t c, double dt) { return fdcgks_steps(c, dt, 1); }

fdcgks_status fdcgks_check(fdcgks_t c, int* nonphysical) {
  if (!c || !nonphysical) return fail(c, FDCGKS_ERR_ARG, "NULL argument");
  int h = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&h, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
  *nonphysical = h & 1;
  return FDCGKS_OK;
}

static fdcgks_status cfl_dt_impl(fdcgks_t c, double cfl, int sum, double* dt_out) {
  if (!c || !dt_out) return fail(c, FDCGKS_ERR_ARG, "NULL argument");
  if (!c->has_state) return fail(c, FDCGKS_ERR_STATE, "no state loaded");
  if (!(cfl > 0.0) || !std::isfinite(cfl)) return fail(c, FDCGKS_ERR_ARG, "cfl must be positive and finite");
  CflGrid G;
  G.L = c->L;
  G.segs = (std::max(c->L.nx, c->L.nxd) + CFL_SEG - 1) / CFL_SEG;
  G.gamma = c->p.gamma;
  G.mu = c->p.mu;
  G.ihx = 1.0 / c->hx;
  G.ihy = 1.0 / c->hy;
  G.gf = (float)G.gamma;
  G.muf = (float)G.mu;
  G.ihxf = (float)G.ihx;
  G.ihyf = (float)G.ihy;
  G.sum = sum;
  const long items = (long)(c->L.ny + c->L.nyd) * G.segs;
  if (items > INT_MAX) return fail(c, FDCGKS_ERR_ARG, "grid too large for the CFL reduction");
  unsigned* mxf = (unsigned*)(c->red + 2 * c->red_blocks);
  CUDA_TRY(c, prof_mark(c, KC_CFL, true));
  CUDA_TRY(c, cudaMemsetAsync(mxf, 0, 2 * sizeof(unsigned), c->stream));
  if (c->Sf) {
    const StatePair st{c->Sf, c->Slo};
    cfl_screen_kernel<<<c->red_blocks, 256, 0, c->stream>>>(st, G, (int)items, mxf);
    CUDA_TRY(c, cudaGetLastError());
    cfl_kernel<<<c->red_blocks, 256, 0, c->stream>>>(st, G, (int)items, mxf, c->red);
  } else {
    const StateF64 st{c->S};
    cfl_screen_kernel<<<c->red_blocks, 256, 0, c->stream>>>(st, G, (int)items, mxf);
    CUDA_TRY(c, cudaGetLastError());
    cfl_kernel<<<c->red_blocks, 256, 0, c->stream>>>(st, G, (int)items, mxf, c->red);
  }
  CUDA_TRY(c, cudaGetLastError());
  c->launches += 2;
  CUDA_TRY(c, prof_mark(c, KC_CFL, false));
  double* h = new double[2 * c->red_blocks];
  cudaError_t e = cudaMemcpyAsync(h, c->red, sizeof(double) * 2 * c->red_blocks, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    delete[] h;
    return fail(c, FDCGKS_ERR_CUDA, "cfl reduction: %s", cudaGetErrorString(e));
  }
  double rate = 0.0, numax = 0.0;
  for (int b = 0; b < c->red_blocks; ++b) {
    rate = std::fmax(rate, h[2 * b]);
    numax = std::fmax(numax, h[2 * b + 1]);
  }
  delete[] h;
  if (!(rate > 0.0) || !std::isfinite(rate)) return fail(c, FDCGKS_ERR_NONPHYSICAL, "no finite wave speed");
  double dt = cfl / rate;
  if (numax > 0.0) {
    double hm = std::fmin(c->hx, c->hy);
    dt = std::fmin(dt, cfl * hm * hm / (8.0 * numax));
  }
  *dt_out = dt;
  return FDCGKS_OK;
}

fdcgks_status fdcgks_cfl_dt(fdcgks_t c, double cfl, double* dt_out) { return cfl_dt_impl(c, cfl, 0, dt_out); }

fdcgks_status fdcgks_cfl_dt_sum(fdcgks_t c, double cfl, double* dt_out) { return cfl_dt_impl(c, cfl, 1, dt_out); }

fdcgks_status fdcgks_stage_operator(fdcgks_t c, double dt, double* Lp, double* Ltp, double* gbp, double* gtp,
                                    double* Ld, double* Ltd, double* gbd, double* gtd) {
  if (!c) return fail(nullptr, FDCGKS_ERR_ARG, "ctx is NULL");
  if (!c->has_state) return fail(c, FDCGKS_ERR_STATE, "no state loaded");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, FDCGKS_ERR_ARG, "dt must be positive and finite");
  double* op[8] = {Lp, Ltp, gbp, gtp, Ld, Ltd, gbd, gtd};
  for (double* q : op)
    if (!q) return fail(c, FDCGKS_ERR_ARG, "NULL output pointer");
  return c->p.precision == FDCGKS_MIXED ? run_stage<float>(c, dt, UPD_OPERATOR, op)
                                        : run_stage<double>(c, dt, UPD_OPERATOR, op);
}

fdcgks_status fdcgks_set_sides(fdcgks_t c, const fdcgks_side* sides) {
  if (!c) return fail(nullptr, FDCGKS_ERR_ARG, "ctx is NULL");
  if (!sides) {
    c->has_sides = false;
    return FDCGKS_OK;
  }
  for (int k = 0; k < 4; ++k) {
    const fdcgks_side& sd = sides[k];
    const bool periodic = c->p.bc[k] == FDCGKS_BC_PERIODIC;
    for (int q = 0; q < 2; ++q) {
      const int kind = sd.kind[q];
      if (periodic != (kind == FDCGKS_BC_PERIODIC))
        return fail(c, FDCGKS_ERR_ARG, "side %d: a periodic direction stays periodic, a bounded one bounded", k);
      if (kind < 0 || kind > FDCGKS_BC_FIXED) return fail(c, FDCGKS_ERR_ARG, "side %d: unknown kind %d", k, kind);
      if (kind == FDCGKS_BC_NOSLIP && sd.kind[1 - q] != FDCGKS_BC_NOSLIP)
        return fail(c, FDCGKS_ERR_ARG, "side %d: a no-slip wall cannot be split", k);
      if (kind == FDCGKS_BC_FIXED) {
        const double* pr = sd.prim[q];
        if (!(pr[0] > 0.0) || !(pr[3] > 0.0) || !std::isfinite(pr[1]) || !std::isfinite(pr[2]) ||
            !std::isfinite(pr[0]) || !std::isfinite(pr[3]))
          return fail(c, FDCGKS_ERR_ARG, "side %d: fixed state needs positive finite density and pressure", k);
      }
    }
    if (!std::isfinite(sd.split0) || !std::isfinite(sd.split_speed))
      return fail(c, FDCGKS_ERR_ARG, "side %d: split must be finite", k);
  }
  for (int k = 0; k < 4; ++k) c->sides[k] = sides[k];
  c->has_sides = true;
  return FDCGKS_OK;
}

fdcgks_status fdcgks_set_time(fdcgks_t c, double t) {
  if (!c) return fail(nullptr, FDCGKS_ERR_ARG, "ctx is NULL");
  if (!std::isfinite(t)) return fail(c, FDCGKS_ERR_ARG, "t must be finite");
  c->t = t;
  return FDCGKS_OK;
}

fdcgks_status fdcgks_get_time(fdcgks_t c, double* t) {
  if (!c || !t) return fail(c, FDCGKS_ERR_ARG, "NULL argument");
  *t = c->t;
  return FDCGKS_OK;
}

fdcgks_status fdcgks_set_profiling(fdcgks_t c, int enable) {
  if (!c) return fail(nullptr, FDCGKS_ERR_ARG, "ctx is NULL");
  c->profiling = enable ? 1 : 0;
  c->ev_used = 0;
  return FDCGKS_OK;
}

fdcgks_status fdcgks_get_profile(fdcgks_t c, double* ms, int* count, long long* launches) {
  if (!c) return fail(nullptr, FDCGKS_ERR_ARG, "ctx is NULL");
  if (ms)
    for (int k = 0; k < KC_N; ++k) ms[k] = 0.0;
  if (count)
    for (int k = 0; k < KC_N; ++k) count[k] = 0;
  if (c->ev_used) CUDA_TRY(c, cudaEventSynchronize(c->ev[c->ev_used - 1]));
  for (int k = 0; k + 1 < c->ev_used; k += 2) {
    float t = 0.f;
    CUDA_TRY(c, cudaEventElapsedTime(&t, c->ev[k], c->ev[k + 1]));
    int cls = c->ev_class[k / 2];
    if (ms) ms[cls] += t;
    if (count) count[cls] += 1;
  }
  c->ev_used = 0;
  if (launches) *launches = c->launches;
  return FDCGKS_OK;
}

fdcgks_status fdcgks_iface_batch(const fdcgks_params* p, int normal, double dt, int n, const double* in, double* out) {
  if (const char* m = check_params(p)) return fail(nullptr, FDCGKS_ERR_ARG, "%s", m);
  if (normal != 0 && normal != 1) return fail(nullptr, FDCGKS_ERR_ARG, "normal must be 0 or 1");
  if (n < 0 || (n > 0 && (!in || !out))) return fail(nullptr, FDCGKS_ERR_ARG, "bad batch arguments");
  if (!(dt > 0.0)) return fail(nullptr, FDCGKS_ERR_ARG, "dt must be positive");
  cudaError_t e = p->precision == FDCGKS_MIXED
                      ? launch_iface_batch<float>(make_gas<float>(*p, dt), normal, n, in, out, (cudaStream_t)p->stream)
                      : launch_iface_batch<double>(make_gas<double>(*p, dt), normal, n, in, out, (cudaStream_t)p->stream);
  if (e != cudaSuccess) return fail(nullptr, FDCGKS_ERR_CUDA, "iface batch: %s", cudaGetErrorString(e));
  return FDCGKS_OK;
}

fdcgks_status fdcgks_nodal_batch(const fdcgks_params* p, double dt, int n, const double* in, double* out) {
  if (const char* m = check_params(p)) return fail(nullptr, FDCGKS_ERR_ARG, "%s", m);
  if (n < 0 || (n > 0 && (!in || !out))) return fail(nullptr, FDCGKS_ERR_ARG, "bad batch arguments");
  if (!(dt > 0.0)) return fail(nullptr, FDCGKS_ERR_ARG, "dt must be positive");
  cudaError_t e = p->precision == FDCGKS_MIXED
                      ? launch_nodal_batch<float>(make_gas<float>(*p, dt), n, in, out, (cudaStream_t)p->stream)
                      : launch_nodal_batch<double>(make_gas<double>(*p, dt), n, in, out, (cudaStream_t)p->stream);
  if (e != cudaSuccess) return fail(nullptr, FDCGKS_ERR_CUDA, "nodal batch: %s", cudaGetErrorString(e));
  return FDCGKS_OK;
}

fdcgks_status fdcgks_recon_batch(const fdcgks_params* p, int kind, double h, int n, const double* in, double* out) {
  if (const char* m = check_params(p)) return fail(nullptr, FDCGKS_ERR_ARG, "%s", m);
  if (kind != 0 && kind != 1) return fail(nullptr, FDCGKS_ERR_ARG, "kind must be 0 or 1");
  if (!(h > 0.0) || n < 0 || (n > 0 && (!in || !out))) return fail(nullptr, FDCGKS_ERR_ARG, "bad batch arguments");
  cudaError_t e = p->precision == FDCGKS_MIXED
                      ? launch_recon_batch<float>(make_geno<float>(p->geno_variant), kind, h, n, in, out,
                                                  (cudaStream_t)p->stream)
                      : launch_recon_batch<double>(make_geno<double>(p->geno_variant), kind, h, n, in, out,
                                                   (cudaStream_t)p->stream);
  if (e != cudaSuccess) return fail(nullptr, FDCGKS_ERR_CUDA, "recon batch: %s", cudaGetErrorString(e));
  return FDCGKS_OK;
}

}  // extern "C"
