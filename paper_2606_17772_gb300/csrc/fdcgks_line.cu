// The paper's one-dimensional scheme (Sec. 2, with the reconstruction of
// Sec. 3) on a batch of independent lines.
//
// One line is one grid of n nodes carrying W = (rho, rho U, rho E) and the
// averaged gradient W_x (Eq. define-averaged-gradient).  One thread block
// owns one line for a whole call: a step is
//
//   stage 1: ghosts(S) -> interface solves + nodal fluxes -> update S -> T
//   stage 2: ghosts(T) -> interface solves + nodal fluxes -> update T -> S
//
// with barriers between the phases, so a call runs any number of steps
// (fixed dt, or each line's own CFL dt found by a reduction) in a single
// launch, and the lines of a batch run side by side on the SMs.  A line can
// also be spread over a thread-block cluster of 2, 4 or 8 blocks (on as many
// SMs): the phases' work items are dealt out over the cluster's threads and
// the phases are separated by cluster barriers, whose release/acquire
// ordering makes each block's global-memory writes visible to the others.
// A single line then runs at the FP64 rate of several SMs instead of one.  The line's working arrays stay in global memory (L2-resident for
// the line sizes of Sec. 5); the per-node device functions are the 2-D
// path's: the line reconstruction of the 2-D interface points with the
// y-momentum set to zero, the x-normal kinetic solve with V = 0 and no
// tangential variation (the 1-D BGK gas is the 2-D one restricted so), and
// the nodal solve with W_y = 0.  The compute type R is FP64, or FP32 (the
// mixed path: reconstruction, kinetic solves and compact fluxes in FP32 with
// the 2-D mixed path's FP64 time coefficients, the interface and nodal
// outputs stored in FP32); the state, its stage copy and the S2O4
// accumulation are FP64 in both.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include <cooperative_groups.h>

#include "../../include/fdcgks.h"
#include "fdcgks_kernels.cuh"

namespace cg = cooperative_groups;

using namespace fdk;

namespace {

constexpr int LT = 128;    // threads per line block
constexpr int NPF = 19;    // interface outputs: F, F_t, W^l, W^r, W^l_t, W^r_t (3 each), chi

enum { LINE_STEPS = 0, LINE_RUN = 1, LINE_OPERATOR = 2 };

template <class R>
struct LineArgs {
  int n, np;                 // nodes; padded length n + 2 GH
  int cs;                    // blocks per line (a cluster when > 1)
  int bc0, bc1, fv, grad_base, recon_vars;
  double h, ih, gamma, mu;
  GenoK<R> geno;
  GasK<R> gas;               // the time-step fields are set per step
  double* S;                 // [batch][6][np] state (W 3, W_x 3)
  double* T;                 // [batch][6][np] stage-1 state
  R* P;                      // [batch][NPF][n + 3] interfaces k + 1/2, k = -2..n
  R* NF;                     // [batch][6][n + 2] nodal F, F_t at nodes -1..n
  double* A;                 // [batch][6][n] S2O4 accumulator and gradient base
  double* tl;                // [batch] line time
  int* ns;                   // [batch] steps taken by the last run
  int* flag;                 // [batch] status bits
  double* part;              // [batch][cs][2] per-block CFL maxima
  double* op[4];             // LINE_OPERATOR outputs [batch][3][n]
};

// this thread's index among the line's threads, and their number
template <class R>
__device__ __forceinline__ int lt_index(const LineArgs<R>& a) { return (blockIdx.x % a.cs) * blockDim.x + threadIdx.x; }
template <class R>
__device__ __forceinline__ int lt_count(const LineArgs<R>& a) { return a.cs * blockDim.x; }

// barrier over the line's threads (block or cluster), ordering their memory accesses
template <class R>
__device__ __forceinline__ void line_sync(const LineArgs<R>& a) {
  if (a.cs == 1) __syncthreads();
  else cg::this_cluster().sync();
}

// conservative component c (0..2) of a line <-> slot of the 2-D 4-vector
__device__ __forceinline__ int slot4(int c) { return c == 2 ? 3 : c; }

// ghost nodes of buffer B: periodic wrap, constant extrapolation with zero
// gradient (transmissive), mirror with U odd and each gradient of the
// opposite parity to its field (reflecting)
template <class R>
__device__ void line_ghosts(const LineArgs<R>& a, double* B) {
  for (int idx = lt_index(a); idx < 2 * GH; idx += lt_count(a)) {
    const int side = idx / GH, k = 1 + idx % GH;
    const int b = side == 0 ? a.bc0 : a.bc1;
    const int ghost = side == 0 ? -k : a.n - 1 + k;
    int src;
    if (b == FDCGKS_BC_PERIODIC) src = ((ghost % a.n) + a.n) % a.n;
    else if (b == FDCGKS_BC_TRANSMISSIVE) src = side == 0 ? 0 : a.n - 1;
    else src = side == 0 ? k - 1 : a.n - k;
    for (int c = 0; c < 3; ++c) {
      double w = B[c * a.np + GH + src], gx = B[(3 + c) * a.np + GH + src];
      if (b == FDCGKS_BC_TRANSMISSIVE) {
        gx = 0.0;
      } else if (b == FDCGKS_BC_SYMMETRY) {
        const double s = c == 1 ? -1.0 : 1.0;
        w *= s;
        gx *= -s;
      }
      B[c * a.np + GH + ghost] = w;
      B[(3 + c) * a.np + GH + ghost] = gx;
    }
  }
}

// interface solves (k = -2..n) and nodal fluxes (j = -1..n) of buffer B
template <class R>
__device__ void line_fluxes(const LineArgs<R>& a, const GasK<R>& gas, const double* B, R* P, R* NF) {
  const int ni = a.n + 3, nn = a.n + 2;
  const R h = (R)a.h, ih = (R)a.ih;
  for (int idx = lt_index(a); idx < ni + nn; idx += lt_count(a)) {
    if (idx < ni) {
      const int k = idx - 2;   // interface k + 1/2 from nodes k-1..k+2
      auto ld = [&](int, int e, int f) -> R {
        const int s = f & 3;
        if (s == 2) return R(0);                      // rho V
        const int c = s == 3 ? 2 : s;
        return (R)B[((f < 4 ? 0 : 3) + c) * a.np + GH + (k - 1 + e)];
      };
      R vl[4], dl[4], vr[4], dr[4], chi;
      if (a.recon_vars) recon_line_char(a.geno, gas.gm1, 0, ld, 0, h, ih, vl, dl, vr, dr, chi);
      else recon_line_ld(a.geno, ld, 0, h, ih, vl, dl, vr, dr, chi);
      const R zero[4] = {R(0), R(0), R(0), R(0)};
      IfaceOut<R> o;
      iface_solve(gas, 0, vl, vr, dl, dr, zero, true, o);
      R* q = P + idx;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int s = slot4(c);
        q[(0 + c) * ni] = o.F[s];
        q[(3 + c) * ni] = o.Ft[s];
        q[(6 + c) * ni] = o.Wl[s];
        q[(9 + c) * ni] = o.Wr[s];
        q[(12 + c) * ni] = o.Wlt[s];
        q[(15 + c) * ni] = o.Wrt[s];
      }
      q[18 * ni] = chi;
    } else {
      const int j = idx - ni - 1;   // node j: value and GENO x-derivative
      R W[4] = {R(0), R(0), R(0), R(0)}, Wx[4] = {R(0), R(0), R(0), R(0)}, Wy[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double* w = B + c * a.np + GH + j;
        const double* g = B + (3 + c) * a.np + GH + j;
        const R q[3] = {(R)w[-1], (R)w[0], (R)w[1]}, gx[3] = {(R)g[-1], (R)g[0], (R)g[1]};
        W[slot4(c)] = q[1];
        Wx[slot4(c)] = recon_node(a.geno, q, gx, h, ih);
      }
      R F[4], G[4], Ft[4], Gt[4];
      nodal_flux(gas, W, Wx, Wy, F, G, Ft, Gt);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        NF[c * nn + j + 1] = F[slot4(c)];
        NF[(3 + c) * nn + j + 1] = Ft[slot4(c)];
      }
    }
  }
}

// node operator (Eqs. fd-conservative-form, fd-conservative-flux*,
// define-averaged-gradient) and the S2O4 stage update Bin -> Bout
template <class R>
__device__ void line_update(const LineArgs<R>& a, int mode, int stage, double dt, const R* P, const R* NF,
                            const double* Bin, double* Bout, double* A, int line, int* flag) {
  const int ni = a.n + 3, nn = a.n + 2;
  const R ih = (R)a.ih;
  for (int j = lt_index(a); j < a.n; j += lt_count(a)) {
    const R chip = P[18 * ni + j + 2], chim = P[18 * ni + j + 1];
    double L[3], Lt[3], gb[3], gt[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R* F = P + c * ni;
      const R* Ft = P + (3 + c) * ni;
      const R* nF = NF + c * nn;
      const R* nFt = NF + (3 + c) * nn;
      // interface k + 1/2 sits at P index k + 2, node k at NF index k + 1
      const R fp = compact_flux(a.fv, chip, F[j + 1], F[j + 2], F[j + 3], nF[j + 1], nF[j + 2]);
      const R fm = compact_flux(a.fv, chim, F[j], F[j + 1], F[j + 2], nF[j], nF[j + 1]);
      const R ftp = compact_flux(a.fv, chip, Ft[j + 1], Ft[j + 2], Ft[j + 3], nFt[j + 1], nFt[j + 2]);
      const R ftm = compact_flux(a.fv, chim, Ft[j], Ft[j + 1], Ft[j + 2], nFt[j], nFt[j + 1]);
      L[c] = (double)(-(fp - fm) * ih);
      Lt[c] = (double)(-(ftp - ftm) * ih);
      gb[c] = (double)((P[(6 + c) * ni + j + 2] - P[(9 + c) * ni + j + 1]) * ih);
      gt[c] = (double)((P[(12 + c) * ni + j + 2] - P[(15 + c) * ni + j + 1]) * ih);
    }
    if (mode == LINE_OPERATOR) {
      const long o = (long)line * 3 * a.n + j;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        a.op[0][o + c * a.n] = L[c];
        a.op[1][o + c * a.n] = Lt[c];
        a.op[2][o + c * a.n] = gb[c];
        a.op[3][o + c * a.n] = gt[c];
      }
      continue;
    }
    double W[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (stage == 0) {
        const double Wn = Bin[c * a.np + GH + j];
        W[c] = Wn + 0.5 * dt * L[c] + 0.125 * dt * dt * Lt[c];
        A[c * a.n + j] = Wn + dt * L[c] + dt * dt / 6.0 * Lt[c];
        const double base = a.grad_base ? Bin[(3 + c) * a.np + GH + j] : gb[c];
        A[(3 + c) * a.n + j] = base;
        Bout[(3 + c) * a.np + GH + j] = base + 0.5 * dt * gt[c];
      } else {
        W[c] = A[c * a.n + j] + dt * dt / 3.0 * Lt[c];
        Bout[(3 + c) * a.np + GH + j] = A[(3 + c) * a.n + j] + dt * gt[c];
      }
      Bout[c * a.np + GH + j] = W[c];
    }
    const double p = W[2] - 0.5 * W[1] * W[1] / W[0];
    if (!(W[0] > 0.0) || !(p > 0.0)) atomicOr(flag, 1);
  }
}

// the line's CFL time step (the same in every thread of the line): block
// maxima of (|U| + c)/h and nu, then across the cluster through global memory
// (k alternates the partial buffer between consecutive steps)
template <class R>
__device__ double line_cfl(const LineArgs<R>& a, const double* B, double cfl, int line, int k) {
  __shared__ double sr[LT / 32], sn[LT / 32];
  double rate = 0.0, numax = 0.0;
  for (int j = lt_index(a); j < a.n; j += lt_count(a))
    cfl_rates(B[GH + j], B[a.np + GH + j], 0.0, B[2 * a.np + GH + j], a.gamma, a.mu, a.ih, 0.0, rate, numax);
  for (int o = 16; o > 0; o >>= 1) {
    rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
    numax = fmax(numax, __shfl_xor_sync(0xffffffffu, numax, o));
  }
  if (threadIdx.x % 32 == 0) {
    sr[threadIdx.x / 32] = rate;
    sn[threadIdx.x / 32] = numax;
  }
  __syncthreads();
  rate = 0.0;
  numax = 0.0;
  for (int w = 0; w < LT / 32; ++w) {
    rate = fmax(rate, sr[w]);
    numax = fmax(numax, sn[w]);
  }
  __syncthreads();   // sr, sn are rewritten by the next call
  if (a.cs > 1) {
    double* part = a.part + ((long)line * 2 + (k & 1)) * a.cs * 2;
    if (threadIdx.x == 0) {
      part[2 * (blockIdx.x % a.cs)] = rate;
      part[2 * (blockIdx.x % a.cs) + 1] = numax;
    }
    line_sync(a);
    for (int r = 0; r < a.cs; ++r) {
      rate = fmax(rate, part[2 * r]);
      numax = fmax(numax, part[2 * r + 1]);
    }
  }
  double dt = cfl / rate;
  if (numax > 0.0) dt = fmin(dt, cfl * a.h * a.h / (8.0 * numax));
  return dt;
}

template <class R>
__device__ void line_stage(const LineArgs<R>& a, const GasK<R>& gas, int mode, int stage, double dt, double* Bin,
                           double* Bout, R* P, R* NF, double* A, int line, int* flag) {
  line_ghosts(a, Bin);
  line_sync(a);
  line_fluxes(a, gas, Bin, P, NF);
  line_sync(a);
  line_update(a, mode, stage, dt, P, NF, Bin, Bout, A, line, flag);
  line_sync(a);
}

// the time-step fields of the gas constants (FP64 and compute-type copies)
template <class R>
__device__ __forceinline__ void gas_set_dt(GasK<R>& gas, double dt) {
  gas.dt = dt;
  gas.inv_dt = 1.0 / dt;
  gas.dt_r = (R)dt;
  gas.inv_dt_r = (R)(1.0 / dt);
}

template <class R>
__global__ void __launch_bounds__(LT) line_kernel(LineArgs<R> a, int mode, double dt_fixed, int nsteps, double t_end,
                                                  double cfl, int max_steps) {
  const int b = blockIdx.x / a.cs;
  const bool lead = blockIdx.x % a.cs == 0 && threadIdx.x == 0;
  const long pad = 6L * a.np;
  double* S = a.S + b * pad;
  double* T = a.T + b * pad;
  R* P = a.P + (long)b * NPF * (a.n + 3);
  R* NF = a.NF + (long)b * 6 * (a.n + 2);
  double* A = a.A + (long)b * 6 * a.n;
  int* flag = a.flag + b;
  GasK<R> gas = a.gas;
  if (mode == LINE_OPERATOR) {
    gas_set_dt(gas, dt_fixed);
    line_stage(a, gas, mode, 0, dt_fixed, S, T, P, NF, A, b, flag);
    return;
  }
  double t = a.tl[b];
  int k = 0;
  // every thread runs the same sequence of time steps, so the loop and its
  // barriers are uniform over the block
  while (mode == LINE_STEPS ? k < nsteps : (k < max_steps && t < t_end * (1.0 - 1e-14))) {
    double dt = dt_fixed;
    if (mode == LINE_RUN) {
      dt = fmin(line_cfl(a, S, cfl, b, k), t_end - t);
      if (!(dt > 0.0) || !(dt < INFINITY)) {
        if (lead) atomicOr(flag, 2);
        break;
      }
    }
    gas_set_dt(gas, dt);
    line_stage(a, gas, mode, 0, dt, S, T, P, NF, A, b, flag);
    line_stage(a, gas, mode, 1, dt, T, S, P, NF, A, b, flag);
    t += dt;
    ++k;
    // a run stops a line that left the physical states (the flag is read
    // after the stage's closing barrier, so every thread of the line sees the
    // same value and the line's blocks leave the loop together)
    if (mode == LINE_RUN && (*(volatile int*)flag & 1)) break;
  }
  if (lead) {
    a.tl[b] = t;
    a.ns[b] = k;
  }
}

// W, W_x [batch][3][n] <-> the padded state (set_state / get_state)
__global__ void line_scatter_kernel(const double* W, const double* Wx, double* S, int n, int np, long total) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long b = t / (3L * n);
    const int c = (int)((t / n) % 3), j = (int)(t % n);
    S[b * 6 * np + (long)c * np + GH + j] = W[t];
    S[b * 6 * np + (long)(3 + c) * np + GH + j] = Wx[t];
  }
}
__global__ void line_gather_kernel(const double* S, double* W, double* Wx, int n, int np, long total) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long b = t / (3L * n);
    const int c = (int)((t / n) % 3), j = (int)(t % n);
    W[t] = S[b * 6 * np + (long)c * np + GH + j];
    Wx[t] = S[b * 6 * np + (long)(3 + c) * np + GH + j];
  }
}

}  // namespace

struct fdcgks_line_ctx {
  fdcgks_line_params p;
  LineArgs<double> a;        // FP64 path (the shared buffers; a32 aliases them for the mixed path)
  LineArgs<float> a32;
  cudaStream_t stream;
  void* mem = nullptr;       // one allocation for every array
  double* stage = nullptr;   // [2][batch][3][n] host-copy staging
  long long launches = 0;
  char err[512];
};

namespace {

fdcgks_status lfail(fdcgks_line_t c, fdcgks_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) snprintf(c->err, sizeof(c->err), "%s", buf);
  else set_global_error(buf);
  return s;
}

#define LINE_TRY(c, expr)                                                                          \
  do {                                                                                             \
    cudaError_t e_ = (expr);                                                                       \
    if (e_ != cudaSuccess) return lfail((c), FDCGKS_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

const char* check_line_params(const fdcgks_line_params* p) {
  if (!p) return "params is NULL";
  if (p->n < 1 || p->n > (1 << 20)) return "n must be in [1, 2^20]";
  if (p->batch < 1 || p->batch > (1 << 20)) return "batch must be in [1, 2^20]";
  if ((long long)p->n * p->batch > (1LL << 28)) return "n * batch too large";
  for (int k = 0; k < 2; ++k)
    if (p->bc[k] != FDCGKS_BC_PERIODIC && p->bc[k] != FDCGKS_BC_TRANSMISSIVE && p->bc[k] != FDCGKS_BC_SYMMETRY)
      return "line ends take PERIODIC, TRANSMISSIVE or SYMMETRY";
  if ((p->bc[0] == FDCGKS_BC_PERIODIC) != (p->bc[1] == FDCGKS_BC_PERIODIC))
    return "a periodic line is periodic at both ends";
  if (p->bc[0] != FDCGKS_BC_PERIODIC && p->n < 3) return "a bounded line needs n >= 3";
  if (p->cluster != 0 && p->cluster != 1 && p->cluster != 2 && p->cluster != 4 && p->cluster != 8)
    return "cluster must be 0 (automatic), 1, 2, 4 or 8";
  if (p->precision != FDCGKS_FP64 && p->precision != FDCGKS_MIXED) return "precision must be FP64 or MIXED";
  // the remaining options are those of the 2-D scheme
  fdcgks_params q;
  std::memset(&q, 0, sizeof(q));
  q.nx = p->n;
  q.ny = 1;
  q.x0 = p->x0;
  q.x1 = p->x1;
  q.y0 = 0.0;
  q.y1 = 1.0;
  q.gamma = p->gamma;
  q.mu = p->mu;
  q.Pr = p->Pr;
  q.bc[0] = p->bc[0];
  q.bc[1] = p->bc[1];
  q.flux_variant = p->flux_variant;
  q.geno_variant = p->geno_variant;
  q.grad_base = p->grad_base;
  q.precision = FDCGKS_FP64;
  q.tau_c1 = p->tau_c1;
  q.tau_c2 = p->tau_c2;
  q.recon_vars = p->recon_vars;
  return check_params(&q);
}

fdcgks_status launch_line(fdcgks_line_t c, int mode, double dt, int nsteps, double t_end, double cfl, int max_steps) {
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)(c->p.batch * c->a.cs));
  cfg.blockDim = dim3(LT);
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)c->a.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (c->p.precision == FDCGKS_MIXED) {
    LineArgs<float> a = c->a32;
    for (int k = 0; k < 4; ++k) a.op[k] = c->a.op[k];
    LINE_TRY(c, cudaLaunchKernelEx(&cfg, line_kernel<float>, a, mode, dt, nsteps, t_end, cfl, max_steps));
  } else {
    LINE_TRY(c, cudaLaunchKernelEx(&cfg, line_kernel<double>, c->a, mode, dt, nsteps, t_end, cfl, max_steps));
  }
  ++c->launches;
  return FDCGKS_OK;
}

}  // namespace

extern "C" {

fdcgks_status fdcgks_line_create(const fdcgks_line_params* p, fdcgks_line_t* out) {
  if (!out) return lfail(nullptr, FDCGKS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (const char* m = check_line_params(p)) return lfail(nullptr, FDCGKS_ERR_ARG, "%s", m);
  fdcgks_line_t c = new (std::nothrow) fdcgks_line_ctx();
  if (!c) return lfail(nullptr, FDCGKS_ERR_CUDA, "out of host memory");
  c->p = *p;
  c->err[0] = 0;
  c->stream = (cudaStream_t)p->stream;
  const int n = p->n, B = p->batch, np = n + 2 * GH;
  LineArgs<double>& a = c->a;
  a.n = n;
  a.np = np;
  // blocks per line: as asked, or automatic: spread lines over clusters of up
  // to 8 blocks while the batch leaves SMs idle (two blocks fit an SM), with
  // at least 32 nodes per block
  a.cs = p->cluster;
  if (a.cs == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    a.cs = 1;
    while (a.cs < 8 && (long)B * a.cs * 2 <= 2L * sms && n / (a.cs * 2) >= 32) a.cs *= 2;
  }
  a.bc0 = p->bc[0];
  a.bc1 = p->bc[1];
  a.fv = p->flux_variant;
  a.grad_base = p->grad_base;
  a.recon_vars = p->recon_vars;
  a.h = (p->x1 - p->x0) / n;
  a.ih = 1.0 / a.h;
  a.gamma = p->gamma;
  a.mu = p->mu;
  a.geno = make_geno<double>(p->geno_variant);
  fdcgks_params q;
  std::memset(&q, 0, sizeof(q));
  q.gamma = p->gamma;
  q.mu = p->mu;
  q.Pr = p->Pr;
  q.tau_c1 = p->tau_c1;
  q.tau_c2 = p->tau_c2;
  a.gas = make_gas<double>(q, 1.0);
  // doubles: S, T, P, NF, A, tl, staging, CFL partials; ints: ns, flag
  const size_t nS = (size_t)B * 6 * np, nP = (size_t)B * NPF * (n + 3), nN = (size_t)B * 6 * (n + 2),
               nA = (size_t)B * 6 * n, nStage = (size_t)B * 6 * n, nPart = (size_t)B * 4 * a.cs;
  const size_t nd = 2 * nS + nP + nN + nA + B + nStage + nPart;
  const size_t bytes = nd * sizeof(double) + 2 * (size_t)B * sizeof(int);
  cudaError_t e = cudaMalloc(&c->mem, bytes);
  if (e != cudaSuccess) {
    delete c;
    return lfail(nullptr, FDCGKS_ERR_CUDA, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  double* d = (double*)c->mem;
  a.S = d;
  d += nS;
  a.T = d;
  d += nS;
  a.P = d;
  d += nP;
  a.NF = d;
  d += nN;
  a.A = d;
  d += nA;
  a.tl = d;
  d += B;
  c->stage = d;
  d += nStage;
  a.part = d;
  d += nPart;
  a.ns = (int*)d;
  a.flag = a.ns + B;
  for (int k = 0; k < 4; ++k) a.op[k] = nullptr;
  // the mixed path's view: the same buffers, FP32 interface and nodal outputs
  // in the (larger) FP64 arrays' space, FP32 constants
  LineArgs<float>& f = c->a32;
  f.n = a.n; f.np = a.np; f.cs = a.cs;
  f.bc0 = a.bc0; f.bc1 = a.bc1; f.fv = a.fv; f.grad_base = a.grad_base; f.recon_vars = a.recon_vars;
  f.h = a.h; f.ih = a.ih; f.gamma = a.gamma; f.mu = a.mu;
  f.geno = make_geno<float>(p->geno_variant);
  f.gas = make_gas<float>(q, 1.0);
  f.S = a.S; f.T = a.T; f.A = a.A; f.tl = a.tl; f.ns = a.ns; f.flag = a.flag; f.part = a.part;
  f.P = (float*)a.P;
  f.NF = (float*)a.NF;
  for (int k = 0; k < 4; ++k) f.op[k] = nullptr;
  e = cudaMemsetAsync(c->mem, 0, bytes, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    cudaFree(c->mem);
    delete c;
    return lfail(nullptr, FDCGKS_ERR_CUDA, "initialisation: %s", cudaGetErrorString(e));
  }
  *out = c;
  return FDCGKS_OK;
}

void fdcgks_line_destroy(fdcgks_line_t c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  cudaFree(c->mem);
  delete c;
}

fdcgks_status fdcgks_line_set_state(fdcgks_line_t c, const double* W, const double* Wx, int on_device) {
  if (!c) return lfail(nullptr, FDCGKS_ERR_ARG, "ctx is NULL");
  if (!W || !Wx) return lfail(c, FDCGKS_ERR_ARG, "W or Wx is NULL");
  const long total = 3L * c->p.n * c->p.batch;
  const double *w = W, *wx = Wx;
  if (!on_device) {
    LINE_TRY(c, cudaMemcpyAsync(c->stage, W, total * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    LINE_TRY(c, cudaMemcpyAsync(c->stage + total, Wx, total * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    w = c->stage;
    wx = c->stage + total;
  }
  const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  line_scatter_kernel<<<blocks, 256, 0, c->stream>>>(w, wx, c->a.S, c->p.n, c->a.np, total);
  LINE_TRY(c, cudaGetLastError());
  LINE_TRY(c, cudaMemsetAsync(c->a.tl, 0, c->p.batch * sizeof(double), c->stream));
  LINE_TRY(c, cudaMemsetAsync(c->a.flag, 0, c->p.batch * sizeof(int), c->stream));
  if (!on_device) LINE_TRY(c, cudaStreamSynchronize(c->stream));
  return FDCGKS_OK;
}

fdcgks_status fdcgks_line_get_state(fdcgks_line_t c, double* W, double* Wx, int on_device) {
  if (!c) return lfail(nullptr, FDCGKS_ERR_ARG, "ctx is NULL");
  if (!W || !Wx) return lfail(c, FDCGKS_ERR_ARG, "W or Wx is NULL");
  const long total = 3L * c->p.n * c->p.batch;
  double* w = on_device ? W : c->stage;
  double* wx = on_device ? Wx : c->stage + total;
  const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  line_gather_kernel<<<blocks, 256, 0, c->stream>>>(c->a.S, w, wx, c->p.n, c->a.np, total);
  LINE_TRY(c, cudaGetLastError());
  if (!on_device) {
    LINE_TRY(c, cudaMemcpyAsync(W, w, total * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LINE_TRY(c, cudaMemcpyAsync(Wx, wx, total * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LINE_TRY(c, cudaStreamSynchronize(c->stream));
  }
  return FDCGKS_OK;
}

fdcgks_status fdcgks_line_steps(fdcgks_line_t c, double dt, int nsteps) {
  if (!c) return lfail(nullptr, FDCGKS_ERR_ARG, "ctx is NULL");
  if (!(dt > 0.0) || !std::isfinite(dt)) return lfail(c, FDCGKS_ERR_ARG, "dt must be positive and finite");
  if (nsteps < 0) return lfail(c, FDCGKS_ERR_ARG, "nsteps must be >= 0");
  if (nsteps == 0) return FDCGKS_OK;
  return launch_line(c, LINE_STEPS, dt, nsteps, 0.0, 0.0, 0);
}

fdcgks_status fdcgks_line_run(fdcgks_line_t c, double t_end, double cfl, int max_steps, double* t, int* steps) {
  if (!c) return lfail(nullptr, FDCGKS_ERR_ARG, "ctx is NULL");
  if (!std::isfinite(t_end)) return lfail(c, FDCGKS_ERR_ARG, "t_end must be finite");
  if (!(cfl > 0.0) || !std::isfinite(cfl)) return lfail(c, FDCGKS_ERR_ARG, "cfl must be positive and finite");
  if (max_steps < 0) return lfail(c, FDCGKS_ERR_ARG, "max_steps must be >= 0");
  fdcgks_status s = launch_line(c, LINE_RUN, 0.0, 0, t_end, cfl, max_steps);
  if (s != FDCGKS_OK) return s;
  if (t) LINE_TRY(c, cudaMemcpyAsync(t, c->a.tl, c->p.batch * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (steps) LINE_TRY(c, cudaMemcpyAsync(steps, c->a.ns, c->p.batch * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  LINE_TRY(c, cudaStreamSynchronize(c->stream));
  return FDCGKS_OK;
}

fdcgks_status fdcgks_line_stage_operator(fdcgks_line_t c, double dt, double* L, double* Lt, double* gb, double* gt) {
  if (!c) return lfail(nullptr, FDCGKS_ERR_ARG, "ctx is NULL");
  if (!(dt > 0.0) || !std::isfinite(dt)) return lfail(c, FDCGKS_ERR_ARG, "dt must be positive and finite");
  if (!L || !Lt || !gb || !gt) return lfail(c, FDCGKS_ERR_ARG, "output pointer is NULL");
  c->a.op[0] = L;
  c->a.op[1] = Lt;
  c->a.op[2] = gb;
  c->a.op[3] = gt;
  fdcgks_status s = launch_line(c, LINE_OPERATOR, dt, 0, 0.0, 0.0, 0);
  for (int k = 0; k < 4; ++k) c->a.op[k] = nullptr;
  return s;
}

fdcgks_status fdcgks_line_check(fdcgks_line_t c, int* flags, int* any) {
  if (!c) return lfail(nullptr, FDCGKS_ERR_ARG, "ctx is NULL");
  const int B = c->p.batch;
  int* h = new (std::nothrow) int[B];
  if (!h) return lfail(c, FDCGKS_ERR_CUDA, "out of host memory");
  cudaError_t e = cudaMemcpyAsync(h, c->a.flag, B * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    delete[] h;
    return lfail(c, FDCGKS_ERR_CUDA, "flag read: %s", cudaGetErrorString(e));
  }
  int o = 0;
  for (int b = 0; b < B; ++b) o |= h[b];
  if (flags) std::memcpy(flags, h, B * sizeof(int));
  if (any) *any = o;
  delete[] h;
  return FDCGKS_OK;
}

const char* fdcgks_line_last_error(fdcgks_line_t c) { return c ? c->err : fdcgks_last_error(nullptr); }

}  // extern "C"
