// Internal declarations shared by the CUDA translation units of the FD-CGKS
// library: padded data layout, kernel argument block and launchers.
#pragma once

#include <cuda_runtime.h>

#include "fdcgks_math.cuh"

namespace fdk {

const int GH = 3;        // ghost layers of every state plane
const int NFLD = 12;     // fields per grid: W[4], averaged x-gradient[4], averaged y-gradient[4]
const int NNF = 16;      // nodal outputs: F[4], G[4], F_t[4], G_t[4]
const int NPS = 25;      // outputs of one interface solve (see PO_* below)
const int NPT = 2 * NPS; // outputs of one virtual-interface point (primary solve, dual solve)

// field offsets inside one solve's 25 outputs
enum { PO_F = 0, PO_FT = 4, PO_CHI = 8, PO_WL = 9, PO_WR = 13, PO_WLT = 17, PO_WRT = 21 };

// Both grids share one padded plane geometry.  A state buffer holds
// [grid 2][field 12][plane]; node (i, j) of a grid sits at
// (j + GH) * pitch + (i + GH), i in [-GH, n + GH).
// Interface-point arrays (Type A: (i+1/2, j), Type B: (i, j+1/2)) hold
// [NPT][pplane] with point (i, j) at (j + 2) * ppitch + (i + 2).
struct Layout {
  int nx, ny, nxd, nyd;
  int pitch, rows;
  long plane;
  int ppitch, prows;
  long pplane;
};

FD_HD long cell(const Layout& L, int i, int j) { return (long)(j + GH) * L.pitch + (i + GH); }
FD_HD long pcell(const Layout& L, int i, int j) { return (long)(j + 2) * L.ppitch + (i + 2); }

template <class R>
struct KArgs {
  Layout L;
  const R* Sr;           // state read by the nodal and point kernels, in the compute type
                         // (the FP64 state itself, or the high parts in the mixed path)
  // mixed path: the state and the S2O4 accumulators are float-float pairs
  const R* Sn_hi;        // state at t^n [2][12][plane], high and low parts
  const R* Sn_lo;
  R* Out_hi;             // stage 1: W*, grad* (high parts only); stage 2: the new state
  R* Out_lo;             // stage 2: low parts of the new state (null at stage 1)
  R* Acc_hi;             // W_acc pairs [2][4][plane]
  R* Acc_lo;
  R* Gb_hi;              // gradient-base pairs [2][8][plane]
  R* Gb_lo;
  const double* S;       // state read by this stage [2][12][plane] (FP64 path)
  const double* Sn;      // state at t^n (stage 1 base, reading-A gradient base)
  double* Sout;          // stage 1: W*, grad*;  stage 2: W^{n+1}, grad^{n+1}
  double* Wacc;          // [2][4][plane]  W^n + dt L + dt^2/6 L_t
  double* gB;            // [2][8][plane]  gradient base of Eq. (eq-interface-update)
  R* NF;                 // [2][16][plane] nodal fluxes
  R* PA;                 // [50][pplane]   Type A point outputs
  R* PB;                 // [50][pplane]   Type B point outputs
  GenoK<R> geno;
  GasK<R> gas;
  R h[2], ih[2];
  double hd[2], ihd[2];
  int bc[4];
  int flux_variant, grad_base, want_n;
  double dt;
  int* flag;             // bit 0: non-physical state found
  double* op[8];         // operator outputs (Lp, Ltp, gbp, gtp, Ld, Ltd, gbd, gtd), interior layout
};

enum { UPD_STAGE1 = 0, UPD_STAGE2 = 1, UPD_OPERATOR = 2 };

// message returned by fdcgks_last_error(NULL)
void set_global_error(const char* msg);

template <class R> cudaError_t launch_nodal(const KArgs<R>& a, cudaStream_t s);
template <class R> cudaError_t launch_points(const KArgs<R>& a, cudaStream_t s);
template <class R> cudaError_t launch_update(const KArgs<R>& a, int mode, cudaStream_t s);

// component-level batches (device arrays), for parity tests of the kernels' arithmetic
template <class R> cudaError_t launch_iface_batch(const GasK<R>& gas, int normal, int n, const double* in,
                                                  double* out, cudaStream_t s);
template <class R> cudaError_t launch_nodal_batch(const GasK<R>& gas, int n, const double* in, double* out,
                                                  cudaStream_t s);
template <class R> cudaError_t launch_recon_batch(const GenoK<R>& g, int kind, double h, int n, const double* in,
                                                  double* out, cudaStream_t s);

}  // namespace fdk
