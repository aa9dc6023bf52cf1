// Batched ensemble: many independent FD-CGKS runs of different sizes and
// parameters advanced together on one GPU.
//
// Every run ("member") keeps the padded layout and buffers a single context
// would have, carved out of one device allocation.  One step of the whole
// ensemble is a fixed sequence of launches, each covering one phase of the
// stage for all members at once:
//
//   [CFL reduction] -> per-member dt -> stage 1 -> stage 2,
//   stage = ghost fill (x, then y) -> nodal -> points A+B -> update.
//
// Each phase launch drains a list of tiles (member, kind, tile coordinates)
// with a persistent grid of resident blocks that take tiles from an atomic
// queue head, or (autotuner's choice) with one block per tile.  A tile's
// block copies its member's argument block into shared memory and runs the
// same per-node bodies as the single-run kernels, so every member's result
// is identical to a single-context run with the same time steps.
//
// The time step of each member is computed on the device every step (CFL
// reduction into per-member maxima, then a one-thread-per-member kernel that
// writes dt into the member's argument blocks), so a step needs no host
// round trip and is captured once into a CUDA graph that is replayed.
//
// The queue involves no waiting: a block that finds the queue empty exits.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fdcgks.h"
#include "fdcgks_kernels.cuh"

using namespace fdk;

namespace {

const int ENS_THREADS = 128;   // threads per block of every phase kernel
const int CFL_TILE = 1024;     // nodes per CFL tile (8 per thread)

// launch phases of one stage
enum { PH_GHOSTX = 0, PH_GHOSTY, PH_NODAL, PH_POINTS, PH_UPDATE, PH_CFL, PH_N };
// queue heads of one step: the 5 stage phases twice, then the CFL passes
const int N_COUNTERS = 2 * 5 + 2;

// per-member constants of the CFL time step
struct MemberMeta {
  double gamma, mu, ihx, ihy, hm;
};

// one phase launch
struct PhaseQ {
  const int4* tiles;   // (member, kind, tile x, tile y)
  int ntiles;
  int* head;           // queue head (persistent dispatch)
  int stage;           // 0 or 1
  int lbx;             // tile width 2^lbx nodes, height ENS_THREADS >> lbx
  int persistent;
  const int* mstat;    // member status bits
};

// tile width of the points phase in the pair form (two lanes per point, so
// ENS_THREADS / 2 points per tile): 2^min(lbx, 6)
__host__ __device__ inline int ens_points_lbx(int lbx) { return lbx < 6 ? lbx : 6; }

template <class R, int PH> struct EnsMinB { static constexpr int v = 1; };
template <class R> struct EnsMinB<R, PH_NODAL> { static constexpr int v = PointTune<R>::nodal_minb; };
template <class R> struct EnsMinB<R, PH_POINTS> {
  static constexpr int v = PointTune<R>::pair ? PointTune<R>::pair_minb : PointTune<R>::minb;
};
template <class R> struct EnsMinB<R, PH_UPDATE> { static constexpr int v = PointTune<R>::update_minb; };

template <class R>
__device__ __forceinline__ void copy_args(KArgs<R>& dst, const KArgs<R>* src) {
  static_assert(sizeof(KArgs<R>) % sizeof(int) == 0, "argument block is not a whole number of words");
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(&dst);
  for (int k = threadIdx.x; k < (int)(sizeof(KArgs<R>) / sizeof(int)); k += ENS_THREADS) d[k] = s[k];
}

// next tile of this block: from the queue head (persistent) or the block index
template <int PERSIST>
__device__ __forceinline__ int next_tile(const PhaseQ& q, int iter, int* s_tile) {
  if (!PERSIST) return iter == 0 ? (int)blockIdx.x : q.ntiles;
  if (threadIdx.x == 0) *s_tile = atomicAdd(q.head, 1);
  __syncthreads();
  return *s_tile;
}

// one phase for all members; PERSIST 1: resident blocks loop over the queue,
// 0: one block per tile (compiled separately: the loop costs registers)
template <class R, int PH, int PERSIST>
__global__ void __launch_bounds__(ENS_THREADS, (EnsMinB<R, PH>::v)) ens_phase_kernel(const KArgs<R>* args, PhaseQ q) {
  __shared__ KArgs<R> sa;
  __shared__ int s_tile;
  for (int iter = 0;; ++iter) {
    const int t = next_tile<PERSIST>(q, iter, &s_tile);
    if (t >= q.ntiles) break;
    const int4 tl = q.tiles[t];
    if (!(q.mstat[tl.x] & FDCGKS_ENS_FROZEN)) {   // uniform over the block
      copy_args(sa, args + 2 * tl.x + q.stage);
      __syncthreads();
      const int li = threadIdx.x & ((1 << q.lbx) - 1), lj = threadIdx.x >> q.lbx;
      const int i = (tl.z << q.lbx) + li, j = tl.w * (ENS_THREADS >> q.lbx) + lj;
      if (PH == PH_GHOSTX) {
        ghost_body(const_cast<R*>(sa.Sr), sa.L, sa.bc[0], sa.bc[1], 0, tl.y, tl.z * ENS_THREADS + threadIdx.x);
      } else if (PH == PH_GHOSTY) {
        ghost_body(const_cast<R*>(sa.Sr), sa.L, sa.bc[2], sa.bc[3], 1, tl.y, tl.z * ENS_THREADS + threadIdx.x);
      } else if (PH == PH_NODAL) {
        nodal_body(sa, tl.y, i - 1, j - 1);
      } else if (PH == PH_POINTS) {
        if constexpr (PointTune<R>::pair) {
          // two lanes per point (point_pair_body): the tile holds ENS_THREADS / 2
          // points, 2^lbp wide with lbp = min(lbx, 6) (ens_points_lbx)
          const int lbp = ens_points_lbx(q.lbx), pi = threadIdx.x >> 1;
          const int pi_x = (tl.z << lbp) + (pi & ((1 << lbp) - 1));
          const int pj = tl.w * ((ENS_THREADS / 2) >> lbp) + (pi >> lbp);
          if (tl.y == 0) point_pair_body<R, 0, false>(sa, pi_x - 2, pj - 2, threadIdx.x & 1);
          else point_pair_body<R, 1, false>(sa, pi_x - 2, pj - 2, threadIdx.x & 1);
        } else {
          if (tl.y == 0) point_body<R, 0>(sa, i - 2, j - 2);
          else point_body<R, 1>(sa, i - 2, j - 2);
        }
      } else {
        update_body(sa, q.stage == 0 ? UPD_STAGE1 : UPD_STAGE2, tl.y, i, j);
      }
    }
    __syncthreads();   // sa and s_tile are rewritten by the next tile
  }
}

// state at t^n of one node as FP64 (the float-float pair joined in the mixed path)
__device__ __forceinline__ double state_at(const KArgs<double>& a, long off) { return a.Sn[off]; }
__device__ __forceinline__ double state_at(const KArgs<float>& a, long off) {
  return (double)a.Sn_hi[off] + (double)a.Sn_lo[off];
}

// FP32 estimate of one node's CFL rate and viscosity from the high parts of
// the mixed state (cfl_estimate_f: reliable to 1e-5 while p > 0.05 E)
__device__ __forceinline__ void cfl_estimate(const float* hi, long c0, long plane, float gf, float muf, float ihxf,
                                             float ihyf, float& rt, float& nu, bool& ok) {
  cfl_estimate_f(hi[c0], hi[c0 + plane], hi[c0 + 2 * plane], hi[c0 + 3 * plane], gf, muf, ihxf, ihyf, false, rt, nu,
                 ok);
}

// mixed path, first pass: each member's largest reliable FP32 estimates,
// folded with atomicMax on the bit patterns (non-negative floats)
template <class R>
__global__ void __launch_bounds__(ENS_THREADS) ens_cfl_screen_kernel(const KArgs<R>* args, const MemberMeta* meta,
                                                                     PhaseQ q, unsigned* mxf) {
  __shared__ float sr[ENS_THREADS / 32], sn[ENS_THREADS / 32];
  __shared__ int s_tile;
  for (int iter = 0;; ++iter) {
    const int t = q.persistent ? next_tile<1>(q, iter, &s_tile) : next_tile<0>(q, iter, &s_tile);
    if (t >= q.ntiles) break;
    const int4 tl = q.tiles[t];
    const int m = tl.x, g = tl.y;
    float mr = 0.0f, mn = 0.0f;
    if (!(q.mstat[m] & FDCGKS_ENS_FROZEN)) {
      const KArgs<R>& a = args[2 * m];
      const Layout L = a.L;
      const MemberMeta mm = meta[m];
      const int nxg = g == 0 ? L.nx : L.nxd, nyg = g == 0 ? L.ny : L.nyd, nn = nxg * nyg;
      const float* hi = a.Sn_hi + (long)g * NFLD * L.plane;
      for (int k = threadIdx.x; k < CFL_TILE; k += ENS_THREADS) {
        const int n = tl.z + k;
        if (n >= nn) break;
        float rt, nu;
        bool ok;
        cfl_estimate(hi, cell(L, n % nxg, n / nxg), L.plane, (float)mm.gamma, (float)mm.mu, (float)mm.ihx,
                     (float)mm.ihy, rt, nu, ok);
        if (ok) {
          mr = fmaxf(mr, rt);
          mn = fmaxf(mn, nu);
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, o));
      mn = fmaxf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    const int w = threadIdx.x / 32;
    if ((threadIdx.x & 31) == 0) { sr[w] = mr; sn[w] = mn; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int k = 1; k < ENS_THREADS / 32; ++k) { mr = fmaxf(mr, sr[k]); mn = fmaxf(mn, sn[k]); }
      if (mr > 0.0f) atomicMax(mxf + 2 * m, __float_as_uint(mr));
      if (mn > 0.0f) atomicMax(mxf + 2 * m + 1, __float_as_uint(mn));
    }
    __syncthreads();
  }
}

// CFL maxima of each member: tiles (member, grid, first node, -) of CFL_TILE
// nodes of one grid; block maxima folded into the member's pair with
// atomicMax on the bit patterns (both maxima are >= 0, where the order of the
// patterns is the order of the values).  FP64 path: every node evaluated.
// Mixed path: the FP64 rates (from the joined float-float pairs) only where
// the FP32 estimate is unreliable or within CFL_SCREEN_MARGIN of the member's
// largest estimate (first pass); the maxima are exactly those of evaluating
// every node.
template <class R>
__global__ void __launch_bounds__(ENS_THREADS) ens_cfl_kernel(const KArgs<R>* args, const MemberMeta* meta, PhaseQ q,
                                                              const unsigned* mxf, unsigned long long* mx) {
  __shared__ double sr[ENS_THREADS / 32], sn[ENS_THREADS / 32];
  __shared__ int s_tile;
  for (int iter = 0;; ++iter) {
    const int t = q.persistent ? next_tile<1>(q, iter, &s_tile) : next_tile<0>(q, iter, &s_tile);
    if (t >= q.ntiles) break;
    const int4 tl = q.tiles[t];
    const int m = tl.x, g = tl.y;
    double rate = 0.0, numax = 0.0;
    if (!(q.mstat[m] & FDCGKS_ENS_FROZEN)) {
      const KArgs<R>& a = args[2 * m];
      const Layout L = a.L;
      const MemberMeta mm = meta[m];
      const int nxg = g == 0 ? L.nx : L.nxd, nyg = g == 0 ? L.ny : L.nyd, nn = nxg * nyg;
      const long base = (long)g * NFLD * L.plane;
      float tr = 0.0f, tn = INFINITY;
      if constexpr (IsF32<R>::v) {
        const float mr = __uint_as_float(mxf[2 * m]), mn = __uint_as_float(mxf[2 * m + 1]);
        tr = mr * (1.0f - CFL_SCREEN_MARGIN);
        if (mn > 0.0f) tn = mn * (1.0f - CFL_SCREEN_MARGIN);   // with mu = 0 nu never decides
      }
      for (int k = threadIdx.x; k < CFL_TILE; k += ENS_THREADS) {
        const int n = tl.z + k;
        if (n >= nn) break;
        const long c0 = cell(L, n % nxg, n / nxg);
        if constexpr (IsF32<R>::v) {
          float rt, nu;
          bool ok;
          cfl_estimate(a.Sn_hi + base, c0, L.plane, (float)mm.gamma, (float)mm.mu, (float)mm.ihx, (float)mm.ihy,
                       rt, nu, ok);
          if (ok && rt < tr && nu < tn) continue;
        }
        const long cg = base + c0;
        cfl_rates(state_at(a, cg), state_at(a, cg + L.plane), state_at(a, cg + 2 * L.plane),
                  state_at(a, cg + 3 * L.plane), mm.gamma, mm.mu, mm.ihx, mm.ihy, rate, numax);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
      numax = fmax(numax, __shfl_xor_sync(0xffffffffu, numax, o));
    }
    const int w = threadIdx.x / 32;
    if ((threadIdx.x & 31) == 0) { sr[w] = rate; sn[w] = numax; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int k = 1; k < ENS_THREADS / 32; ++k) { rate = fmax(rate, sr[k]); numax = fmax(numax, sn[k]); }
      if (rate > 0.0) atomicMax(mx + 2 * m, (unsigned long long)__double_as_longlong(rate));
      if (numax > 0.0) atomicMax(mx + 2 * m + 1, (unsigned long long)__double_as_longlong(numax));
    }
    __syncthreads();
  }
}

// per-member time step, written into both stage argument blocks: from the
// CFL maxima (the formula of fdcgks_cfl_dt) or from a fixed per-member array;
// members flagged non-physical (or without a finite wave speed) are frozen
template <class R>
__global__ void ens_dt_kernel(KArgs<R>* args, const MemberMeta* meta, const unsigned long long* mx,
                              const double* fixed_dt, const double* cfl_p, int* mstat, double* time, double* last_dt,
                              int M) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  int st = mstat[m];
  if (st & FDCGKS_ENS_NONPHYSICAL) st |= FDCGKS_ENS_FROZEN;
  double dt = 0.0;
  if (!(st & FDCGKS_ENS_FROZEN)) {
    if (fixed_dt) {
      dt = fixed_dt[m];
    } else {
      const double rate = __longlong_as_double((long long)mx[2 * m]);
      const double numax = __longlong_as_double((long long)mx[2 * m + 1]);
      const double cfl = *cfl_p;
      if (!(rate > 0.0) || !(rate < INFINITY)) {
        st |= FDCGKS_ENS_NO_WAVE_SPEED | FDCGKS_ENS_FROZEN;
      } else {
        dt = cfl / rate;
        if (numax > 0.0) {
          const double hm = meta[m].hm;
          dt = fmin(dt, cfl * hm * hm / (8.0 * numax));
        }
      }
    }
  }
  mstat[m] = st;
  if (st & FDCGKS_ENS_FROZEN) {
    last_dt[m] = 0.0;
    return;
  }
  for (int s = 0; s < 2; ++s) {
    KArgs<R>& a = args[2 * m + s];
    a.dt = dt;
    a.gas.dt = dt;
    a.gas.inv_dt = 1.0 / dt;
    a.gas.dt_r = (R)dt;
    a.gas.inv_dt_r = (R)(1.0 / dt);
  }
  time[m] += dt;
  last_dt[m] = dt;
}

// tile shape of the three tiled phases and the dispatch mode
struct TileCfg {
  int lbx[3];      // nodal, points, update: log2 of the tile width (0..7)
  int persistent;  // 1: persistent grid + queue, 0: one block per tile
};

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct fdcgks_ens {
  int M = 0;
  int precision = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  std::vector<fdcgks_params> p;
  std::vector<Layout> L;
  std::vector<double> hx, hy;
  std::vector<char> has_state;
  // one allocation holding every member's buffers
  char* arena = nullptr;
  size_t arena_bytes = 0;
  std::vector<size_t> st_off, st_bytes;   // per member: offset/size of the state buffer(s) to back up
  void* args = nullptr;                   // KArgs<R>[2 M] (stage 1, stage 2 per member)
  std::vector<char> h_args;               // host copy
  MemberMeta* meta = nullptr;
  int* mstat = nullptr;
  double* time = nullptr;
  double* last_dt = nullptr;
  double* fixed_dt = nullptr;
  double* cfl = nullptr;
  unsigned long long* mx = nullptr;
  unsigned* mxf = nullptr;
  int* heads = nullptr;
  int* vflag = nullptr;
  double* staging = nullptr;              // FP64 padded state of the largest member
  // per member: padded FP64 state S (FP64 path) or the float-float pair (mixed)
  std::vector<double*> S;
  std::vector<float*> Shi, Slo;
  // tile lists
  TileCfg cfg;
  int4* tiles = nullptr;
  size_t tiles_cap = 0;
  int t_off[PH_N], t_cnt[PH_N];
  int resident[PH_N];
  cudaGraphExec_t graph[2] = {nullptr, nullptr};   // [0]: CFL time steps, [1]: fixed time steps
  long long launches = 0;
  char err[512];
};

namespace {

fdcgks_status efail(fdcgks_ens_t e, fdcgks_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (e) snprintf(e->err, sizeof(e->err), "%s", buf);
  else set_global_error(buf);
  return s;
}

#define ENS_TRY(e, expr)                                                                                        \
  do {                                                                                                          \
    cudaError_t e_ = (expr);                                                                                    \
    if (e_ != cudaSuccess)                                                                                      \
      return efail(e, e_ == cudaErrorMemoryAllocation ? FDCGKS_ERR_NOMEM : FDCGKS_ERR_CUDA, "%s: %s (%s:%d)", \
                   #expr, cudaGetErrorString(e_), __FILE__, __LINE__);                                          \
  } while (0)

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

template <class R>
size_t args_bytes() { return sizeof(KArgs<R>); }

void drop_graphs(fdcgks_ens_t e) {
  for (auto& g : e->graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

// tile lists of every phase for the current tile configuration
fdcgks_status build_tiles(fdcgks_ens_t e) {
  std::vector<int4> t;
  auto rect = [&](int m, int kind, int w, int h, int lbx) {
    const int bx = 1 << lbx, by = ENS_THREADS >> lbx;
    for (int ty = 0; ty < (h + by - 1) / by; ++ty)
      for (int tx = 0; tx < (w + bx - 1) / bx; ++tx) t.push_back(make_int4(m, kind, tx, ty));
  };
  for (int ph = 0; ph < PH_N; ++ph) {
    e->t_off[ph] = (int)t.size();
    for (int m = 0; m < e->M; ++m) {
      const Layout& L = e->L[m];
      for (int g = 0; g < 2; ++g) {
        const int nxg = g == 0 ? L.nx : L.nxd, nyg = g == 0 ? L.ny : L.nyd;
        switch (ph) {
          case PH_GHOSTX: {
            const int items = nyg * 2 * GH;
            for (int k = 0; k < (items + ENS_THREADS - 1) / ENS_THREADS; ++k) t.push_back(make_int4(m, g, k, 0));
            break;
          }
          case PH_GHOSTY: {
            const int items = (nxg + 2 * GH) * 2 * GH;
            for (int k = 0; k < (items + ENS_THREADS - 1) / ENS_THREADS; ++k) t.push_back(make_int4(m, g, k, 0));
            break;
          }
          case PH_NODAL: rect(m, g, nxg + 2, nyg + 2, e->cfg.lbx[0]); break;
          case PH_POINTS: {  // kind = point type: A (g = 0) over (nx + 3) x (nyd + 3), B over (nxd + 3) x (ny + 3)
            const bool pair = e->precision == FDCGKS_MIXED ? PointTune<float>::pair : PointTune<double>::pair;
            if (pair) {
              // ENS_THREADS / 2 points per tile, 2^lbp wide
              const int lbp = ens_points_lbx(e->cfg.lbx[1]);
              const int bx = 1 << lbp, by = (ENS_THREADS / 2) >> lbp;
              const int w = g == 0 ? L.nx + 3 : L.nxd + 3, h = g == 0 ? L.nyd + 3 : L.ny + 3;
              for (int ty = 0; ty < (h + by - 1) / by; ++ty)
                for (int tx = 0; tx < (w + bx - 1) / bx; ++tx) t.push_back(make_int4(m, g, tx, ty));
            } else if (g == 0) {
              rect(m, 0, L.nx + 3, L.nyd + 3, e->cfg.lbx[1]);
            } else {
              rect(m, 1, L.nxd + 3, L.ny + 3, e->cfg.lbx[1]);
            }
            break;
          }
          case PH_UPDATE: rect(m, g, nxg, nyg, e->cfg.lbx[2]); break;
          case PH_CFL: {
            const long nn = (long)nxg * nyg;
            for (long k = 0; k < nn; k += CFL_TILE) t.push_back(make_int4(m, g, (int)k, 0));
            break;
          }
        }
      }
    }
    e->t_cnt[ph] = (int)t.size() - e->t_off[ph];
  }
  if (t.size() > e->tiles_cap) {
    if (e->tiles) cudaFree(e->tiles);
    e->tiles = nullptr;
    e->tiles_cap = 0;
    ENS_TRY(e, cudaMalloc((void**)&e->tiles, t.size() * sizeof(int4)));
    e->tiles_cap = t.size();
  }
  ENS_TRY(e, cudaMemcpyAsync(e->tiles, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice, e->stream));
  ENS_TRY(e, cudaStreamSynchronize(e->stream));
  drop_graphs(e);
  return FDCGKS_OK;
}

PhaseQ phase_q(fdcgks_ens_t e, int ph, int stage, int head) {
  PhaseQ q;
  q.tiles = e->tiles + e->t_off[ph];
  q.ntiles = e->t_cnt[ph];
  q.head = e->heads + head;
  q.stage = stage;
  q.lbx = ph == PH_NODAL ? e->cfg.lbx[0] : ph == PH_POINTS ? e->cfg.lbx[1] : ph == PH_UPDATE ? e->cfg.lbx[2] : 0;
  q.persistent = e->cfg.persistent;
  q.mstat = e->mstat;
  return q;
}

unsigned grid_of(fdcgks_ens_t e, int ph) {
  const int n = e->t_cnt[ph];
  if (!e->cfg.persistent) return (unsigned)n;
  return (unsigned)(n < e->resident[ph] ? n : e->resident[ph]);
}

template <class R, int PH>
cudaError_t launch_phase(fdcgks_ens_t e, int stage, int head) {
  if (e->t_cnt[PH] == 0) return cudaSuccess;
  const PhaseQ q = phase_q(e, PH, stage, head);
  if (e->cfg.persistent)
    ens_phase_kernel<R, PH, 1><<<grid_of(e, PH), ENS_THREADS, 0, e->stream>>>((const KArgs<R>*)e->args, q);
  else
    ens_phase_kernel<R, PH, 0><<<grid_of(e, PH), ENS_THREADS, 0, e->stream>>>((const KArgs<R>*)e->args, q);
  return cudaGetLastError();
}

// optional per-phase timing (untimed runs pass ev = nullptr)
struct PhaseTimer {
  cudaEvent_t* ev;
  int n;
  cudaError_t mark(cudaStream_t s) { return ev ? cudaEventRecord(ev[n++], s) : cudaSuccess; }
};

// enqueue one step of every member on e->stream (captured into a graph, or
// run directly when timing phases); returns kernels launched via *nk
template <class R>
fdcgks_status enqueue_step(fdcgks_ens_t e, bool fixed, PhaseTimer* tm, int* nk) {
  int k = 0;
  ENS_TRY(e, cudaMemsetAsync(e->heads, 0, sizeof(int) * N_COUNTERS, e->stream));
  if (!fixed) {
    ENS_TRY(e, cudaMemsetAsync(e->mx, 0, sizeof(unsigned long long) * 2 * e->M, e->stream));
    if constexpr (IsF32<R>::v) {
      ENS_TRY(e, cudaMemsetAsync(e->mxf, 0, sizeof(unsigned) * 2 * e->M, e->stream));
      ens_cfl_screen_kernel<R><<<grid_of(e, PH_CFL), ENS_THREADS, 0, e->stream>>>(
          (const KArgs<R>*)e->args, e->meta, phase_q(e, PH_CFL, 0, 11), e->mxf);
      ENS_TRY(e, cudaGetLastError());
      ++k;
    }
    ens_cfl_kernel<R><<<grid_of(e, PH_CFL), ENS_THREADS, 0, e->stream>>>(
        (const KArgs<R>*)e->args, e->meta, phase_q(e, PH_CFL, 0, 10), e->mxf, e->mx);
    ENS_TRY(e, cudaGetLastError());
    ++k;
  }
  ens_dt_kernel<R><<<(e->M + 127) / 128, 128, 0, e->stream>>>((KArgs<R>*)e->args, e->meta, e->mx,
                                                               fixed ? e->fixed_dt : nullptr, e->cfl, e->mstat,
                                                               e->time, e->last_dt, e->M);
  ENS_TRY(e, cudaGetLastError());
  ++k;
  if (tm) ENS_TRY(e, tm->mark(e->stream));
  for (int s = 0; s < 2; ++s) {
    const int h0 = 5 * s;
    ENS_TRY(e, (launch_phase<R, PH_GHOSTX>(e, s, h0)));
    ENS_TRY(e, (launch_phase<R, PH_GHOSTY>(e, s, h0 + 1)));
    if (tm) ENS_TRY(e, tm->mark(e->stream));
    ENS_TRY(e, (launch_phase<R, PH_NODAL>(e, s, h0 + 2)));
    if (tm) ENS_TRY(e, tm->mark(e->stream));
    ENS_TRY(e, (launch_phase<R, PH_POINTS>(e, s, h0 + 3)));
    if (tm) ENS_TRY(e, tm->mark(e->stream));
    ENS_TRY(e, (launch_phase<R, PH_UPDATE>(e, s, h0 + 4)));
    if (tm) ENS_TRY(e, tm->mark(e->stream));
    k += 5;
  }
  if (nk) *nk = k;
  return FDCGKS_OK;
}

fdcgks_status enqueue(fdcgks_ens_t e, bool fixed, PhaseTimer* tm, int* nk) {
  return e->precision == FDCGKS_MIXED ? enqueue_step<float>(e, fixed, tm, nk) : enqueue_step<double>(e, fixed, tm, nk);
}

int kernels_per_step(fdcgks_ens_t e, bool fixed) {
  return (fixed ? 0 : (e->precision == FDCGKS_MIXED ? 2 : 1)) + 1 + 10;
}

fdcgks_status ensure_graph(fdcgks_ens_t e, bool fixed) {
  cudaGraphExec_t& ge = e->graph[fixed ? 1 : 0];
  if (ge) return FDCGKS_OK;
  ENS_TRY(e, cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
  fdcgks_status st = enqueue(e, fixed, nullptr, nullptr);
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
  if (st != FDCGKS_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return efail(e, FDCGKS_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
  }
  ce = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (ce != cudaSuccess) {
    ge = nullptr;
    return efail(e, FDCGKS_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(ce));
  }
  return FDCGKS_OK;
}

fdcgks_status check_member(fdcgks_ens_t e, int m) {
  if (!e) return efail(nullptr, FDCGKS_ERR_ARG, "ensemble is NULL");
  if (m < 0 || m >= e->M) return efail(e, FDCGKS_ERR_ARG, "member %d out of range [0, %d)", m, e->M);
  return FDCGKS_OK;
}

fdcgks_status check_all_loaded(fdcgks_ens_t e) {
  for (int m = 0; m < e->M; ++m)
    if (!e->has_state[m]) return efail(e, FDCGKS_ERR_STATE, "member %d has no state loaded", m);
  return FDCGKS_OK;
}

template <class R>
void fill_args(fdcgks_ens_t e, int m, char* base, const std::vector<size_t>& off) {
  // off: S, S2 (FP64) / Shi, Slo, S2hi (mixed), Acc(_hi, _lo), Gb(_hi, _lo), NF, PA, PB
  const fdcgks_params& p = e->p[m];
  for (int s = 0; s < 2; ++s) {
    KArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    a.L = e->L[m];
    a.geno = make_geno<R>(p.geno_variant);
    a.gas = make_gas<R>(p, 1.0);   // dt fields are written on the device every step
    a.hd[0] = e->hx[m];
    a.hd[1] = e->hy[m];
    a.ihd[0] = 1.0 / e->hx[m];
    a.ihd[1] = 1.0 / e->hy[m];
    a.h[0] = (R)e->hx[m];
    a.h[1] = (R)e->hy[m];
    a.ih[0] = (R)(1.0 / e->hx[m]);
    a.ih[1] = (R)(1.0 / e->hy[m]);
    for (int k = 0; k < 4; ++k) a.bc[k] = p.bc[k];
    a.flux_variant = p.flux_variant;
    a.grad_base = p.grad_base;
    a.want_n = s == 0 ? 1 : 0;
    a.dt = 1.0;
    a.flag = e->mstat + m;
    if (e->precision == FDCGKS_MIXED) {
      float* Shi = (float*)(base + off[0]);
      float* Slo = (float*)(base + off[1]);
      float* S2 = (float*)(base + off[2]);
      a.Sr = (R*)(s == 0 ? Shi : S2);
      a.Sn_hi = (R*)Shi;
      a.Sn_lo = (R*)Slo;
      a.Out_hi = (R*)(s == 0 ? S2 : Shi);
      a.Out_lo = s == 0 ? nullptr : (R*)Slo;
      a.Acc_hi = (R*)(base + off[3]);
      a.Acc_lo = (R*)(base + off[4]);
      a.Gb_hi = (R*)(base + off[5]);
      a.Gb_lo = (R*)(base + off[6]);
      a.NF = (R*)(base + off[7]);
      a.PA = (R*)(base + off[8]);
      a.PB = (R*)(base + off[9]);
    } else {
      double* S = (double*)(base + off[0]);
      double* S2 = (double*)(base + off[1]);
      a.S = s == 0 ? S : S2;
      a.Sr = (R*)a.S;
      a.Sn = S;
      a.Sout = s == 0 ? S2 : S;
      a.Wacc = (double*)(base + off[2]);
      a.gB = (double*)(base + off[3]);
      a.NF = (R*)(base + off[4]);
      a.PA = (R*)(base + off[5]);
      a.PB = (R*)(base + off[6]);
    }
    std::memcpy(e->h_args.data() + (2 * m + s) * sizeof(KArgs<R>), &a, sizeof(a));
  }
}

template <class R, int PH>
cudaError_t occupancy(int* out) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, ens_phase_kernel<R, PH, 1>, ENS_THREADS, 0);
}

template <class R>
cudaError_t all_occupancy(fdcgks_ens_t e) {
  int b[PH_N] = {0};
  cudaError_t r;
  if ((r = occupancy<R, PH_GHOSTX>(&b[PH_GHOSTX])) != cudaSuccess) return r;
  if ((r = occupancy<R, PH_GHOSTY>(&b[PH_GHOSTY])) != cudaSuccess) return r;
  if ((r = occupancy<R, PH_NODAL>(&b[PH_NODAL])) != cudaSuccess) return r;
  if ((r = occupancy<R, PH_POINTS>(&b[PH_POINTS])) != cudaSuccess) return r;
  if ((r = occupancy<R, PH_UPDATE>(&b[PH_UPDATE])) != cudaSuccess) return r;
  if ((r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[PH_CFL], ens_cfl_kernel<R>, ENS_THREADS, 0)) !=
      cudaSuccess)
    return r;
  for (int k = 0; k < PH_N; ++k) e->resident[k] = (b[k] > 0 ? b[k] : 1) * e->num_sms;
  return cudaSuccess;
}

// copy of every member's state buffers (kept by the tuner, which must leave
// the ensemble as it found it)
struct Backup {
  char* buf = nullptr;
  size_t bytes = 0;
};

fdcgks_status backup_take(fdcgks_ens_t e, Backup& b) {
  b.bytes = 0;
  for (int m = 0; m < e->M; ++m) b.bytes += align256(e->st_bytes[m]);
  b.bytes += align256(sizeof(double) * 2 * e->M) + align256(sizeof(int) * e->M);
  ENS_TRY(e, cudaMalloc((void**)&b.buf, b.bytes));
  size_t o = 0;
  for (int m = 0; m < e->M; ++m) {
    ENS_TRY(e, cudaMemcpyAsync(b.buf + o, e->arena + e->st_off[m], e->st_bytes[m], cudaMemcpyDeviceToDevice,
                               e->stream));
    o += align256(e->st_bytes[m]);
  }
  ENS_TRY(e, cudaMemcpyAsync(b.buf + o, e->time, sizeof(double) * e->M, cudaMemcpyDeviceToDevice, e->stream));
  ENS_TRY(e, cudaMemcpyAsync(b.buf + o + sizeof(double) * e->M, e->last_dt, sizeof(double) * e->M,
                             cudaMemcpyDeviceToDevice, e->stream));
  o += align256(sizeof(double) * 2 * e->M);
  ENS_TRY(e, cudaMemcpyAsync(b.buf + o, e->mstat, sizeof(int) * e->M, cudaMemcpyDeviceToDevice, e->stream));
  return FDCGKS_OK;
}

fdcgks_status backup_restore(fdcgks_ens_t e, const Backup& b) {
  size_t o = 0;
  for (int m = 0; m < e->M; ++m) {
    ENS_TRY(e, cudaMemcpyAsync(e->arena + e->st_off[m], b.buf + o, e->st_bytes[m], cudaMemcpyDeviceToDevice,
                               e->stream));
    o += align256(e->st_bytes[m]);
  }
  ENS_TRY(e, cudaMemcpyAsync(e->time, b.buf + o, sizeof(double) * e->M, cudaMemcpyDeviceToDevice, e->stream));
  ENS_TRY(e, cudaMemcpyAsync(e->last_dt, b.buf + o + sizeof(double) * e->M, sizeof(double) * e->M,
                             cudaMemcpyDeviceToDevice, e->stream));
  o += align256(sizeof(double) * 2 * e->M);
  ENS_TRY(e, cudaMemcpyAsync(e->mstat, b.buf + o, sizeof(int) * e->M, cudaMemcpyDeviceToDevice, e->stream));
  return FDCGKS_OK;
}

fdcgks_status set_cfl(fdcgks_ens_t e, double cfl) {
  ENS_TRY(e, cudaMemcpyAsync(e->cfl, &cfl, sizeof(double), cudaMemcpyHostToDevice, e->stream));
  return FDCGKS_OK;
}

// ms per step of the current configuration: warm-up step, then `steps` timed steps
fdcgks_status time_config(fdcgks_ens_t e, int steps, double* ms) {
  fdcgks_status st = ensure_graph(e, false);
  if (st != FDCGKS_OK) return st;
  cudaEvent_t a, b;
  ENS_TRY(e, cudaEventCreate(&a));
  ENS_TRY(e, cudaEventCreate(&b));
  cudaError_t r = cudaGraphLaunch(e->graph[0], e->stream);
  if (r == cudaSuccess) r = cudaEventRecord(a, e->stream);
  for (int k = 0; k < steps && r == cudaSuccess; ++k) r = cudaGraphLaunch(e->graph[0], e->stream);
  if (r == cudaSuccess) r = cudaEventRecord(b, e->stream);
  if (r == cudaSuccess) r = cudaEventSynchronize(b);
  float t = 0.f;
  if (r == cudaSuccess) r = cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (r != cudaSuccess) return efail(e, FDCGKS_ERR_CUDA, "tuning run: %s", cudaGetErrorString(r));
  e->launches += (long long)(steps + 1) * kernels_per_step(e, false);
  *ms = t / steps;
  return FDCGKS_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points
// ---------------------------------------------------------------------------
extern "C" {

void fdcgks_ens_destroy(fdcgks_ens_t e) {
  if (!e) return;
  drop_graphs(e);
  void* bufs[] = {e->arena, e->args, e->meta, e->mstat, e->time, e->last_dt, e->fixed_dt, e->cfl,
                  e->mx, e->mxf, e->heads, e->vflag, e->staging, e->tiles};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (e->stream) cudaStreamDestroy(e->stream);
  delete e;
}

fdcgks_status fdcgks_ens_create(const fdcgks_params* params, int count, fdcgks_ens_t* out) {
  if (!out) return efail(nullptr, FDCGKS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!params || count < 1) return efail(nullptr, FDCGKS_ERR_ARG, "need at least one member");
  for (int m = 0; m < count; ++m) {
    if (const char* msg = check_params(params + m)) return efail(nullptr, FDCGKS_ERR_ARG, "member %d: %s", m, msg);
    if (params[m].precision != params[0].precision)
      return efail(nullptr, FDCGKS_ERR_ARG, "member %d: all members must share one precision", m);
    if (params[m].recon_vars != 0)
      return efail(nullptr, FDCGKS_ERR_ARG, "member %d: the ensemble reconstructs conservative components only", m);
  }
  fdcgks_ens_t e = new (std::nothrow) fdcgks_ens();
  if (!e) return efail(nullptr, FDCGKS_ERR_NOMEM, "host allocation failed");
  e->err[0] = 0;
  e->M = count;
  e->precision = params[0].precision;
  e->p.assign(params, params + count);
  e->cfg.lbx[0] = 5;
  e->cfg.lbx[1] = 5;
  e->cfg.lbx[2] = 5;
  e->cfg.persistent = 0;
  const bool mixed = e->precision == FDCGKS_MIXED;
  const size_t rs = mixed ? sizeof(float) : sizeof(double);
  auto bail = [&](fdcgks_status s, const char* what, cudaError_t r) {
    efail(nullptr, s, "%s: %s", what, cudaGetErrorString(r));
    fdcgks_ens_destroy(e);
    return s;
  };
  cudaError_t r;
  int dev = 0;
  if ((r = cudaGetDevice(&dev)) != cudaSuccess) return bail(FDCGKS_ERR_CUDA, "cudaGetDevice", r);
  if ((r = cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return bail(FDCGKS_ERR_CUDA, "SM count", r);
  if ((r = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(FDCGKS_ERR_CUDA, "stream creation", r);

  // member layouts and the arena plan
  std::vector<std::vector<size_t>> offs(count);
  size_t total = 0;
  long max_plane = 0;
  for (int m = 0; m < count; ++m) {
    const fdcgks_params& p = params[m];
    Layout L = make_layout(p);
    e->L.push_back(L);
    e->hx.push_back((p.x1 - p.x0) / p.nx);
    e->hy.push_back((p.y1 - p.y0) / p.ny);
    if (L.plane > max_plane) max_plane = L.plane;
    std::vector<size_t> sizes;
    if (mixed) {
      const size_t fp = sizeof(float) * L.plane;
      sizes = {fp * 2 * NFLD, fp * 2 * NFLD, fp * 2 * NFLD, fp * 2 * 4, fp * 2 * 4, fp * 2 * 8, fp * 2 * 8};
    } else {
      const size_t dp = sizeof(double) * L.plane;
      sizes = {dp * 2 * NFLD, dp * 2 * NFLD, dp * 2 * 4, dp * 2 * 8};
    }
    sizes.push_back(rs * 2 * NNF * L.plane);
    sizes.push_back(rs * NPT * L.pplane);
    sizes.push_back(rs * NPT * L.pplane);
    for (size_t b : sizes) {
      offs[m].push_back(total);
      total += align256(b);
    }
    // the state itself: S (FP64) or the high and low parts (mixed), adjacent
    e->st_off.push_back(offs[m][0]);
    e->st_bytes.push_back(mixed ? offs[m][1] - offs[m][0] + sizes[1] : sizes[0]);
  }
  e->arena_bytes = total;
  if ((r = cudaMalloc((void**)&e->arena, total)) != cudaSuccess)
    return bail(r == cudaErrorMemoryAllocation ? FDCGKS_ERR_NOMEM : FDCGKS_ERR_CUDA, "ensemble arena", r);
  const size_t ab = mixed ? args_bytes<float>() : args_bytes<double>();
  struct { void** ptr; size_t bytes; } allocs[] = {
      {&e->args, ab * 2 * count},
      {(void**)&e->meta, sizeof(MemberMeta) * count},
      {(void**)&e->mstat, sizeof(int) * count},
      {(void**)&e->time, sizeof(double) * count},
      {(void**)&e->last_dt, sizeof(double) * count},
      {(void**)&e->fixed_dt, sizeof(double) * count},
      {(void**)&e->cfl, sizeof(double)},
      {(void**)&e->mx, sizeof(unsigned long long) * 2 * count},
      {(void**)&e->mxf, sizeof(unsigned) * 2 * count},
      {(void**)&e->heads, sizeof(int) * N_COUNTERS},
      {(void**)&e->vflag, sizeof(int)},
      {(void**)&e->staging, mixed ? sizeof(double) * 2 * NFLD * max_plane : 0},
  };
  for (auto& a : allocs) {
    if (!a.bytes) continue;
    if ((r = cudaMalloc(a.ptr, a.bytes)) != cudaSuccess)
      return bail(r == cudaErrorMemoryAllocation ? FDCGKS_ERR_NOMEM : FDCGKS_ERR_CUDA, "ensemble buffers", r);
  }
  // argument blocks and constants
  e->h_args.assign(ab * 2 * count, 0);
  std::vector<MemberMeta> meta(count);
  for (int m = 0; m < count; ++m) {
    if (mixed) fill_args<float>(e, m, e->arena, offs[m]);
    else fill_args<double>(e, m, e->arena, offs[m]);
    meta[m].gamma = params[m].gamma;
    meta[m].mu = params[m].mu;
    meta[m].ihx = 1.0 / e->hx[m];
    meta[m].ihy = 1.0 / e->hy[m];
    meta[m].hm = std::fmin(e->hx[m], e->hy[m]);
    if (mixed) {
      e->S.push_back(nullptr);
      e->Shi.push_back((float*)(e->arena + offs[m][0]));
      e->Slo.push_back((float*)(e->arena + offs[m][1]));
    } else {
      e->S.push_back((double*)(e->arena + offs[m][0]));
      e->Shi.push_back(nullptr);
      e->Slo.push_back(nullptr);
    }
  }
  e->has_state.assign(count, 0);
  r = cudaMemsetAsync(e->arena, 0, total, e->stream);
  if (r == cudaSuccess) r = cudaMemcpyAsync(e->args, e->h_args.data(), e->h_args.size(), cudaMemcpyHostToDevice,
                                            e->stream);
  if (r == cudaSuccess) r = cudaMemcpyAsync(e->meta, meta.data(), sizeof(MemberMeta) * count, cudaMemcpyHostToDevice,
                                            e->stream);
  if (r == cudaSuccess) r = cudaMemsetAsync(e->mstat, 0, sizeof(int) * count, e->stream);
  if (r == cudaSuccess) r = cudaMemsetAsync(e->time, 0, sizeof(double) * count, e->stream);
  if (r == cudaSuccess) r = cudaMemsetAsync(e->last_dt, 0, sizeof(double) * count, e->stream);
  if (r == cudaSuccess) r = cudaStreamSynchronize(e->stream);
  if (r != cudaSuccess) return bail(FDCGKS_ERR_CUDA, "ensemble initialisation", r);
  r = mixed ? all_occupancy<float>(e) : all_occupancy<double>(e);
  if (r != cudaSuccess) return bail(FDCGKS_ERR_CUDA, "occupancy query", r);
  fdcgks_status st = build_tiles(e);
  if (st != FDCGKS_OK) {
    efail(nullptr, st, "%s", e->err);
    fdcgks_ens_destroy(e);
    return st;
  }
  *out = e;
  return FDCGKS_OK;
}

fdcgks_status fdcgks_ens_set_state(fdcgks_ens_t e, int m, const double* Wp, const double* Gp, const double* Wd,
                                   const double* Gd, int on_device) {
  fdcgks_status st = check_member(e, m);
  if (st != FDCGKS_OK) return st;
  if (!Wp || !Gp || !Wd || !Gd) return efail(e, FDCGKS_ERR_ARG, "NULL state pointer");
  const Layout& L = e->L[m];
  const bool mixed = e->precision == FDCGKS_MIXED;
  double* S = mixed ? e->staging : e->S[m];
  const double* srcW[2] = {Wp, Wd};
  const double* srcG[2] = {Gp, Gd};
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  e->has_state[m] = 0;
  for (int g = 0; g < 2; ++g) {
    const int nxg = g == 0 ? L.nx : L.nxd, nyg = g == 0 ? L.ny : L.nyd;
    const long NN = (long)nxg * nyg;
    for (int f = 0; f < NFLD; ++f) {
      const double* src = f < 4 ? srcW[g] + f * NN : srcG[g] + (f - 4) * NN;
      double* dst = S + ((long)g * NFLD + f) * L.plane + cell(L, 0, 0);
      ENS_TRY(e, cudaMemcpy2DAsync(dst, sizeof(double) * L.pitch, src, sizeof(double) * nxg, sizeof(double) * nxg,
                                   nyg, kind, e->stream));
    }
  }
  if (mixed) ENS_TRY(e, launch_split_ff(S, e->Shi[m], e->Slo[m], 2L * NFLD * L.plane, e->stream));
  ENS_TRY(e, cudaMemsetAsync(e->vflag, 0, sizeof(int), e->stream));
  ENS_TRY(e, launch_validate(S, L, e->p[m].gamma, e->vflag, e->stream));
  ENS_TRY(e, cudaMemsetAsync(e->mstat + m, 0, sizeof(int), e->stream));
  ENS_TRY(e, cudaMemsetAsync(e->time + m, 0, sizeof(double), e->stream));
  ENS_TRY(e, cudaMemsetAsync(e->last_dt + m, 0, sizeof(double), e->stream));
  int h = 0;
  ENS_TRY(e, cudaMemcpyAsync(&h, e->vflag, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
  ENS_TRY(e, cudaStreamSynchronize(e->stream));
  if (h) return efail(e, FDCGKS_ERR_NONPHYSICAL, "member %d: state has non-positive or non-finite density/pressure", m);
  e->has_state[m] = 1;
  return FDCGKS_OK;
}

fdcgks_status fdcgks_ens_get_state(fdcgks_ens_t e, int m, double* Wp, double* Gp, double* Wd, double* Gd,
                                   int on_device) {
  fdcgks_status st = check_member(e, m);
  if (st != FDCGKS_OK) return st;
  if (!e->has_state[m]) return efail(e, FDCGKS_ERR_STATE, "member %d has no state loaded", m);
  if (!Wp || !Gp || !Wd || !Gd) return efail(e, FDCGKS_ERR_ARG, "NULL state pointer");
  const Layout& L = e->L[m];
  double* S = e->S[m];
  if (e->precision == FDCGKS_MIXED) {
    S = e->staging;
    ENS_TRY(e, launch_join_ff(e->Shi[m], e->Slo[m], S, 2L * NFLD * L.plane, e->stream));
  }
  double* dstW[2] = {Wp, Wd};
  double* dstG[2] = {Gp, Gd};
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int g = 0; g < 2; ++g) {
    const int nxg = g == 0 ? L.nx : L.nxd, nyg = g == 0 ? L.ny : L.nyd;
    const long NN = (long)nxg * nyg;
    for (int f = 0; f < NFLD; ++f) {
      double* dst = f < 4 ? dstW[g] + f * NN : dstG[g] + (f - 4) * NN;
      const double* src = S + ((long)g * NFLD + f) * L.plane + cell(L, 0, 0);
      ENS_TRY(e, cudaMemcpy2DAsync(dst, sizeof(double) * nxg, src, sizeof(double) * L.pitch, sizeof(double) * nxg,
                                   nyg, kind, e->stream));
    }
  }
  ENS_TRY(e, cudaStreamSynchronize(e->stream));
  return FDCGKS_OK;
}

fdcgks_status fdcgks_ens_run(fdcgks_ens_t e, double cfl, const double* dt, int nsteps) {
  if (!e) return efail(nullptr, FDCGKS_ERR_ARG, "ensemble is NULL");
  if (nsteps < 0) return efail(e, FDCGKS_ERR_ARG, "nsteps must be >= 0");
  fdcgks_status st = check_all_loaded(e);
  if (st != FDCGKS_OK) return st;
  const bool fixed = dt != nullptr;
  if (fixed) {
    for (int m = 0; m < e->M; ++m)
      if (!(dt[m] > 0.0) || !std::isfinite(dt[m])) return efail(e, FDCGKS_ERR_ARG, "dt[%d] must be positive", m);
    ENS_TRY(e, cudaMemcpyAsync(e->fixed_dt, dt, sizeof(double) * e->M, cudaMemcpyHostToDevice, e->stream));
  } else {
    if (!(cfl > 0.0) || !std::isfinite(cfl)) return efail(e, FDCGKS_ERR_ARG, "cfl must be positive and finite");
    st = set_cfl(e, cfl);
    if (st != FDCGKS_OK) return st;
  }
  st = ensure_graph(e, fixed);
  if (st != FDCGKS_OK) return st;
  for (int k = 0; k < nsteps; ++k) ENS_TRY(e, cudaGraphLaunch(e->graph[fixed ? 1 : 0], e->stream));
  e->launches += (long long)nsteps * kernels_per_step(e, fixed);
  return FDCGKS_OK;
}

fdcgks_status fdcgks_ens_status(fdcgks_ens_t e, double* t, double* last_dt, int* status) {
  if (!e) return efail(nullptr, FDCGKS_ERR_ARG, "ensemble is NULL");
  if (t) ENS_TRY(e, cudaMemcpyAsync(t, e->time, sizeof(double) * e->M, cudaMemcpyDeviceToHost, e->stream));
  if (last_dt)
    ENS_TRY(e, cudaMemcpyAsync(last_dt, e->last_dt, sizeof(double) * e->M, cudaMemcpyDeviceToHost, e->stream));
  if (status) ENS_TRY(e, cudaMemcpyAsync(status, e->mstat, sizeof(int) * e->M, cudaMemcpyDeviceToHost, e->stream));
  ENS_TRY(e, cudaStreamSynchronize(e->stream));
  return FDCGKS_OK;
}

fdcgks_status fdcgks_ens_set_tiles(fdcgks_ens_t e, const int* cfg) {
  if (!e || !cfg) return efail(e, FDCGKS_ERR_ARG, "NULL argument");
  for (int k = 0; k < 3; ++k)
    if (cfg[k] < 0 || cfg[k] > 7) return efail(e, FDCGKS_ERR_ARG, "tile width exponent must be in [0, 7]");
  if (cfg[3] != 0 && cfg[3] != 1) return efail(e, FDCGKS_ERR_ARG, "dispatch must be 0 or 1");
  for (int k = 0; k < 3; ++k) e->cfg.lbx[k] = cfg[k];
  e->cfg.persistent = cfg[3];
  return build_tiles(e);
}

fdcgks_status fdcgks_ens_get_tiles(fdcgks_ens_t e, int* cfg) {
  if (!e || !cfg) return efail(e, FDCGKS_ERR_ARG, "NULL argument");
  for (int k = 0; k < 3; ++k) cfg[k] = e->cfg.lbx[k];
  cfg[3] = e->cfg.persistent;
  return FDCGKS_OK;
}

fdcgks_status fdcgks_ens_tune(fdcgks_ens_t e, double cfl, int trial_steps, int* cfg_out, double* ms_out) {
  if (!e) return efail(nullptr, FDCGKS_ERR_ARG, "ensemble is NULL");
  if (trial_steps < 1) return efail(e, FDCGKS_ERR_ARG, "trial_steps must be >= 1");
  if (!(cfl > 0.0) || !std::isfinite(cfl)) return efail(e, FDCGKS_ERR_ARG, "cfl must be positive and finite");
  fdcgks_status st = check_all_loaded(e);
  if (st != FDCGKS_OK) return st;
  Backup b;
  st = backup_take(e, b);
  if (st == FDCGKS_OK) st = set_cfl(e, cfl);
  TileCfg best = e->cfg;
  double best_ms = 1e300;
  // the current configuration first, then coordinate descent: each phase's
  // tile width with the others held, then the dispatch mode
  auto trial = [&](const TileCfg& c) -> fdcgks_status {
    e->cfg = c;
    fdcgks_status s = build_tiles(e);
    if (s == FDCGKS_OK) s = backup_restore(e, b);
    double ms = 0.0;
    if (s == FDCGKS_OK) s = time_config(e, trial_steps, &ms);
    if (s == FDCGKS_OK && ms < best_ms) {
      best_ms = ms;
      best = c;
    }
    return s;
  };
  if (st == FDCGKS_OK) st = trial(e->cfg);
  for (int ph = 0; ph < 3 && st == FDCGKS_OK; ++ph) {
    const TileCfg base = best;
    for (int lbx = 3; lbx <= 7 && st == FDCGKS_OK; ++lbx) {
      if (lbx == base.lbx[ph]) continue;
      TileCfg c = base;
      c.lbx[ph] = lbx;
      st = trial(c);
    }
  }
  if (st == FDCGKS_OK) {
    TileCfg c = best;
    c.persistent = 1 - c.persistent;
    st = trial(c);
  }
  e->cfg = best;
  fdcgks_status st2 = build_tiles(e);
  if (st2 == FDCGKS_OK && b.buf) st2 = backup_restore(e, b);
  if (b.buf) {
    cudaStreamSynchronize(e->stream);
    cudaFree(b.buf);
  }
  if (st != FDCGKS_OK) return st;
  if (st2 != FDCGKS_OK) return st2;
  if (cfg_out) fdcgks_ens_get_tiles(e, cfg_out);
  if (ms_out) *ms_out = best_ms;
  return FDCGKS_OK;
}

fdcgks_status fdcgks_ens_profile(fdcgks_ens_t e, double cfl, int nsteps, double* ms) {
  if (!e || !ms) return efail(e, FDCGKS_ERR_ARG, "NULL argument");
  if (nsteps < 1) return efail(e, FDCGKS_ERR_ARG, "nsteps must be >= 1");
  if (!(cfl > 0.0) || !std::isfinite(cfl)) return efail(e, FDCGKS_ERR_ARG, "cfl must be positive and finite");
  fdcgks_status st = check_all_loaded(e);
  if (st != FDCGKS_OK) return st;
  st = set_cfl(e, cfl);
  if (st != FDCGKS_OK) return st;
  // events: start, after dt, then per stage 4 marks -> 10 per step
  const int per = 10;
  std::vector<cudaEvent_t> ev((size_t)per * nsteps);
  for (auto& v : ev) ENS_TRY(e, cudaEventCreate(&v));
  for (int k = 0; k < 5; ++k) ms[k] = 0.0;
  fdcgks_status out = FDCGKS_OK;
  for (int s = 0; s < nsteps && out == FDCGKS_OK; ++s) {
    PhaseTimer tm{ev.data() + (size_t)per * s, 0};
    cudaError_t r = tm.mark(e->stream);
    if (r != cudaSuccess) {
      out = efail(e, FDCGKS_ERR_CUDA, "event record: %s", cudaGetErrorString(r));
      break;
    }
    int nk = 0;
    out = enqueue(e, false, &tm, &nk);
    e->launches += nk;
  }
  if (out == FDCGKS_OK) {
    cudaError_t r = cudaEventSynchronize(ev.back());
    // classes: 0 CFL + dt, 1 ghost, 2 nodal, 3 points, 4 update
    const int cls[per - 1] = {0, 1, 2, 3, 4, 1, 2, 3, 4};
    for (int s = 0; s < nsteps && r == cudaSuccess; ++s)
      for (int k = 0; k + 1 < per && r == cudaSuccess; ++k) {
        float t = 0.f;
        r = cudaEventElapsedTime(&t, ev[(size_t)per * s + k], ev[(size_t)per * s + k + 1]);
        ms[cls[k]] += t;
      }
    if (r != cudaSuccess) out = efail(e, FDCGKS_ERR_CUDA, "event timing: %s", cudaGetErrorString(r));
  }
  for (auto& v : ev) cudaEventDestroy(v);
  return out;
}

fdcgks_status fdcgks_ens_info(fdcgks_ens_t e, void** stream, long long* launches, long long* nodes) {
  if (!e) return efail(nullptr, FDCGKS_ERR_ARG, "ensemble is NULL");
  if (stream) *stream = (void*)e->stream;
  if (launches) *launches = e->launches;
  if (nodes) {
    long long n = 0;
    for (int m = 0; m < e->M; ++m) n += (long long)e->L[m].nx * e->L[m].ny + (long long)e->L[m].nxd * e->L[m].nyd;
    *nodes = n;
  }
  return FDCGKS_OK;
}

const char* fdcgks_ens_last_error(fdcgks_ens_t e) { return e ? e->err : fdcgks_last_error(nullptr); }

}  // extern "C"
