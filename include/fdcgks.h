/*
 * fdcgks.h -- C ABI of the GB300 FD-CGKS library (libfdcgks.so).
 *
 * The library advances the two-dimensional finite-difference compact
 * gas-kinetic scheme of "Finite Difference Implementation of a High-order
 * Space-Time Coupled Compact Gas-Kinetic Scheme" (Zhao, Chen, Xu) on one GPU:
 * the conservative variables W = (rho, rho U, rho V, rho E) and the averaged
 * spatial gradients of W on a primary grid and on a dual grid offset by half a
 * spacing in both directions (Sec. 4), evolved by the S2O4 two-stage scheme
 * (Sec. 2.4) with the space-time coupled BGK interface solution (App. A) and
 * GENO-blended compact reconstruction (Sec. 3).
 *
 * Conventions for every entry point:
 *   - Status codes; nothing aborts, exits or traps on the device.  A failed
 *     call leaves a message readable with fdcgks_last_error().  Unless an
 *     entry point says otherwise: FDCGKS_ERR_ARG for a NULL context or array
 *     or an out-of-range argument (nothing is changed then); FDCGKS_ERR_STATE
 *     for a call that needs a state before fdcgks_set_state; FDCGKS_ERR_NOMEM
 *     when a device allocation fails; FDCGKS_ERR_CUDA for a failed launch or
 *     copy, after which the context's state is unspecified (load one again).
 *   - Arrays are float64, C order.  Conservative fields W: [4][ny][nx];
 *     gradients: [2][4][ny][nx] (averaged x-gradient, then y-gradient).
 *     Dual-grid arrays use (nyd, nxd) from fdcgks_dims().
 *   - "on_device" selects device pointers (stream-ordered on the context's
 *     stream) or host pointers (the call returns after the copy completed).
 *   - The caller owns every pointer it passes; the library never frees or
 *     retains caller memory.  The context owns its device buffers.
 *   - All work is issued on params.stream (a cudaStream_t; NULL = legacy
 *     default stream).
 *   - Node placement: primary nodes at cell centres x0 + (i + 1/2) hx, dual
 *     nodes at x0 + i hx.  A bounded direction carries n + 1 dual nodes (the
 *     outermost lie on the boundaries); a periodic one carries n.
 */
#ifndef FDCGKS_H
#define FDCGKS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fdcgks_ctx* fdcgks_t;

typedef enum {
  FDCGKS_OK = 0,
  FDCGKS_ERR_ARG = 1,          /* invalid argument (sizes, variants, dt, pointers) */
  FDCGKS_ERR_CUDA = 2,         /* a CUDA call failed; see fdcgks_last_error */
  FDCGKS_ERR_NONPHYSICAL = 3,  /* non-positive or non-finite density or pressure found */
  FDCGKS_ERR_STATE = 4,        /* step or get_state before set_state */
  FDCGKS_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
  FDCGKS_ERR_NOMEM = 6         /* device allocation failed */
} fdcgks_status;

/* Boundary conditions (Sec. 5 test problems; ghost rules are this library's
 * reading, the paper does not describe them):
 *   PERIODIC      wrap (must be set on both sides of a direction)
 *   TRANSMISSIVE  zero-gradient: ghosts copy the boundary node, zero gradients
 *   SYMMETRY      mirror; normal momentum odd, all else even
 *   NOSLIP        adiabatic no-slip wall: mirror with both momenta odd; dual
 *                 nodes on the wall have their velocity set to zero after each stage */
typedef enum {
  FDCGKS_BC_PERIODIC = 0,
  FDCGKS_BC_TRANSMISSIVE = 1,
  FDCGKS_BC_SYMMETRY = 2,
  FDCGKS_BC_NOSLIP = 3,
  FDCGKS_BC_FIXED = 4          /* fixed state (inflow, or the state on either side of a tracked shock):
                                  ghosts hold the given state with zero gradients; only through
                                  fdcgks_set_sides */
} fdcgks_bc;

typedef enum { FDCGKS_FP64 = 0, FDCGKS_MIXED = 1 } fdcgks_precision;

typedef struct {
  int nx, ny;                 /* primary nodes per direction (>= 1) */
  double x0, x1, y0, y1;      /* domain; hx = (x1 - x0)/nx, hy = (y1 - y0)/ny */
  double gamma;               /* ratio of specific heats (> 1) */
  double mu;                  /* dynamic viscosity (>= 0; 0 = inviscid) */
  double Pr;                  /* Prandtl number (> 0) */
  int bc[4];                  /* fdcgks_bc for x-low, x-high, y-low, y-high */
  int flux_variant;           /* 64: FD-CGKS(6-4), Eq. fd-conservative-flux-2 (default);
                                 62: FD-CGKS(6-2), Eq. fd-conservative-flux-1 */
  int geno_variant;           /* 0: Sec. 3.2 constants (r=2, eps=1e-12, d=(8,1,1));
                                 1: App. D constants (r=3, eps=1e-15, d=8 on the central stencil);
                                 2: linear reconstruction and flux (chi = 1) */
  int grad_base;              /* Eq. eq-interface-update base: 0 = re-evaluated from the
                                 interface solution at t^n (default), 1 = stored gradient */
  int precision;              /* fdcgks_precision: FP64, or MIXED (FP32 reconstruction and
                                 flux arithmetic, FP64 state, accumulation and time coefficients) */
  double tau_c1, tau_c2;      /* collision time tau = c1 dt + mu/p + c2 dt |pl - pr|/(pl + pr)
                                 at interfaces, c1 dt + mu/p at nodes (paper App. A cites the
                                 GKS literature for tau; these constants are run parameters) */
  void* stream;               /* cudaStream_t for all work; NULL = legacy default stream */
  int recon_vars;             /* interface reconstruction (Sec. 3.1) on 0: conservative components
                                 (default), 1: characteristic components along the interface normal
                                 (eigenvectors of the Euler flux Jacobian at the mean of the two
                                 adjacent nodes; chi of the flux from the U +- c fields, Sec. 3.2).
                                 Single contexts only: the ensemble and the adjoint take 0. */
} fdcgks_params;

/* Create a context: validates params and allocates the device buffers of the
 * state (both grids, padded with 3 ghost layers), the S2O4 stage state and
 * the per-stage interface/nodal intermediates.  *out is NULL on failure. */
fdcgks_status fdcgks_create(const fdcgks_params* params, fdcgks_t* out);

/* Release a context and its device memory.  NULL is accepted. */
void fdcgks_destroy(fdcgks_t ctx);

/* Interior node counts of the primary (nx, ny) and dual (nxd, nyd) grids. */
fdcgks_status fdcgks_dims(fdcgks_t ctx, int* nx, int* ny, int* nxd, int* nyd);

/* Load W and averaged gradients of both grids (layouts above).  Validates
 * that density and pressure are positive and finite everywhere
 * (FDCGKS_ERR_NONPHYSICAL otherwise; the state is then not marked loaded). */
fdcgks_status fdcgks_set_state(fdcgks_t ctx, const double* Wp, const double* Gp, const double* Wd,
                               const double* Gd, int on_device);

/* Copy W and averaged gradients of both grids out (layouts above). */
fdcgks_status fdcgks_get_state(fdcgks_t ctx, double* Wp, double* Gp, double* Wd, double* Gd, int on_device);

/* One S2O4 step of size dt (> 0, finite): Eqs. eq-nodal-update and
 * eq-interface-update, each stage evaluating the compact nonlinear flux
 * (Eqs. fd-conservative-flux, -flux-1/-2) of GENO-reconstructed (Sec. 3)
 * kinetic interface and nodal fluxes (App. A) on both grids (Sec. 4).
 * Asynchronous on the context stream.  A non-physical result sets a device
 * flag read by fdcgks_check(). */
fdcgks_status fdcgks_step(fdcgks_t ctx, double dt);

/* nsteps consecutive steps of size dt (same semantics as fdcgks_step). */
fdcgks_status fdcgks_steps(fdcgks_t ctx, double dt, int nsteps);

/* CFL time step (Sec. 5): cfl * min over all nodes of both grids of
 * min(hx/(|U|+c), hy/(|V|+c)); with mu > 0 also bounded by
 * cfl * min(hx,hy)^2 / (8 nu_max), nu = mu/rho.  Synchronizes the stream.
 * The bound is per direction: for smooth flow oblique to the grid, cfl 0.4
 * lets the scheme's grid-scale diagonal modes grow slowly (visible over
 * thousands of steps, first in mixed precision); cfl 0.2 is stable.
 * Evaluated in FP64 (on the joined float-float pairs in a mixed context) at
 * the nodes that can hold the maxima: a first pass takes FP32 estimates of
 * every node's rates, a second evaluates the FP64 rates only where the
 * estimate is unreliable or within a relative 5e-5 of the largest estimate,
 * which is more than twice the estimates' error; the result equals the
 * all-node FP64 value. */
fdcgks_status fdcgks_cfl_dt(fdcgks_t ctx, double cfl, double* dt_out);

/* The two-dimensional form of the same bound: cfl / max over all nodes of
 * both grids of ((|U|+c)/hx + (|V|+c)/hy), with the same viscous bound.  At
 * most the per-direction step, half of it for flow at 45 degrees; cfl 0.4 in
 * this form is stable for smooth oblique flow.  Synchronizes the stream;
 * evaluated with the same screening. */
fdcgks_status fdcgks_cfl_dt_sum(fdcgks_t ctx, double cfl, double* dt_out);

/* Read and clear the device non-physical flag (synchronizes the stream).
 * *nonphysical = 1 if a step produced non-positive/non-finite rho or p. */
fdcgks_status fdcgks_check(fdcgks_t ctx, int* nonphysical);

/* One stage's spatial operator on the current state, without advancing it:
 * L and dL/dt (Eq. eq-conservation-law-2d applied to the fluxes and their time
 * derivatives), the averaged gradients re-evaluated from the interface
 * solution (Eq. define-averaged-gradient) and their time derivatives.  Device
 * pointers, interior layouts: L* [4][ny][nx], g* [2][4][ny][nx] (dual arrays
 * over nyd, nxd).  Used to check the kernels stage by stage. */
fdcgks_status fdcgks_stage_operator(fdcgks_t ctx, double dt, double* Lp, double* Ltp, double* gbp, double* gtp,
                                    double* Ld, double* Ltd, double* gbd, double* gtd);

/* Kernel-class timing: with profiling enabled, every stage records CUDA
 * events on the context stream around its ghost fill, nodal kernel, point
 * kernels (Type A and B) and update kernel, and fdcgks_cfl_dt /
 * fdcgks_cfl_dt_sum around their reduction kernel (with the float-float to
 * FP64 join of the state on mixed contexts).  fdcgks_get_profile waits for
 * the recorded events, returns the summed milliseconds and the number of
 * launch groups per class in ms[5] / count[5] (order: ghost, nodal, points,
 * update, cfl; either may be NULL), clears the record, and returns in
 * *launches (may be NULL) the total number of kernels the stepping path has
 * launched on this context. */
fdcgks_status fdcgks_set_profiling(fdcgks_t ctx, int enable);
fdcgks_status fdcgks_get_profile(fdcgks_t ctx, double* ms, int* count, long long* launches);

/* Boundary sides beyond params.bc (the paper names inflow, outflow, reflecting
 * walls starting part way along a side, and a top boundary that tracks an
 * exact moving shock, Sec. 5 double Mach reflection, without describing their
 * implementation).  Each side (x-low, x-high, y-low, y-high) is split at a
 * point that moves along it, split0 + split_speed * t (x for the y-sides, y
 * for the x-sides): ghost nodes whose coordinate along the side lies below
 * the split take kind[0], the others kind[1].  FIXED parts hold prim[part] =
 * (rho, U, V, p) in their ghosts with zero gradients.  The ghost fill of stage
 * 1 uses the context time t, that of stage 2 t + dt/2; each step advances t
 * by dt (fdcgks_set_time, fdcgks_get_time; fdcgks_set_state resets t to 0).
 *   - sides == NULL restores params.bc.  A periodic direction stays periodic
 *     on both sides and parts; a bounded side takes TRANSMISSIVE, SYMMETRY,
 *     FIXED, or NOSLIP (NOSLIP only for an unsplit side, kind[0] == kind[1]).
 *   - Single contexts only (the ensemble and the adjoint take params.bc). */
typedef struct {
  int kind[2];
  double split0, split_speed;
  double prim[2][4];
} fdcgks_side;
fdcgks_status fdcgks_set_sides(fdcgks_t ctx, const fdcgks_side* sides);
fdcgks_status fdcgks_set_time(fdcgks_t ctx, double t);
fdcgks_status fdcgks_get_time(fdcgks_t ctx, double* t);

/* Batched kinetic interface solve (App. A1-A2, Eq. eq:W-model), normal 0 = x,
 * 1 = y, on device arrays: in [n][20] = Wl[4], Wr[4], normal derivatives
 * Wl_n[4], Wr_n[4], tangential derivative Wt[4]; out [n][24] = F[4], F_t[4],
 * W^l[4], W^r[4], W^l_t[4], W^r_t[4].  Uses params' gas, tau constants and
 * precision; dt is the step size.  Asynchronous on params->stream. */
fdcgks_status fdcgks_iface_batch(const fdcgks_params* params, int normal, double dt, int n, const double* in,
                                 double* out);

/* Batched nodal flux (Sec. 2.1) on device arrays: in [n][12] = W[4], W_x[4],
 * W_y[4]; out [n][16] = F[4], G[4], F_t[4], G_t[4]. */
fdcgks_status fdcgks_nodal_batch(const fdcgks_params* params, double dt, int n, const double* in, double* out);

/* Batched GENO reconstruction (Sec. 3) on device arrays.  kind 0: interface
 * between entries 1 and 2 of a 4-point line, in [n][8] = Q[4], Qx[4];
 * out [n][6] = value_l, derivative_l, chi_l, value_r, derivative_r, chi_r.
 * kind 1: node derivative, in [n][6] = Q[3], Qx[3]; out [n][6] = derivative, 0...
 * h is the spacing. */
fdcgks_status fdcgks_recon_batch(const fdcgks_params* params, int kind, double h, int n, const double* in,
                                 double* out);

/* Allocation-free CFL time step.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they need
 * a time step, e.g. an application that gives the library a fixed share of
 * the GPU's memory and forbids further allocations, or a time loop that must
 * not risk an allocation failure or the synchronisation cudaMalloc/cudaFree
 * can imply.  It computes the same
 * time step as fdcgks_cfl_dt, from the caller's device arrays Wp [4][ny][nx]
 * and Wd [4][nyd][nxd] (float64, read only), without a context and without
 * allocating: its partial maxima live in a fixed device array of the library
 * (FDCGKS_NOALLOC_MAX_TILES tiles of FDCGKS_NOALLOC_TILE_NODES nodes, 64 KB),
 * which every GPU that loads the library holds until the process exits.
 *   - Uses params' nx, ny, bc (for nxd, nyd), domain, gamma, mu and stream;
 *     runs on params->stream and synchronizes it to read the result.
 *   - Grids with more than FDCGKS_NOALLOC_MAX_TILES * FDCGKS_NOALLOC_TILE_NODES
 *     primary plus dual nodes are rejected with FDCGKS_ERR_ARG.
 *   - The first call on each device looks up the device address of the
 *     library's array (once per device, with that device current); make that
 *     first call before any stream capture.  The address is kept for the rest
 *     of the process: it belongs to the device's primary context, so the
 *     caller must not reset the device (cudaDeviceReset) or make another
 *     context current between calls.
 *   - All calls share the one array and it keeps the last call's contents;
 *     each call writes every entry it reads, so nothing needs clearing, but
 *     calls that overlap on the GPU (other streams, other host threads) race
 *     on it and must be serialized by the caller.
 *   - Errors are reported through fdcgks_last_error(NULL). */
#define FDCGKS_NOALLOC_TILE_NODES 4096
#define FDCGKS_NOALLOC_MAX_TILES 4096
fdcgks_status fdcgks_cfl_dt_noalloc(const fdcgks_params* params, const double* Wp, const double* Wd, double cfl,
                                    double* dt_out);

/* Adjoint of nsteps steps (reverse mode).  The paper has no counterpart: the
 * gradient of a scalar objective J of the state after nsteps steps of size dt
 * with respect to the initial state, for sensitivity studies and
 * optimisation through the solver.
 *   - Inputs (device arrays, the layouts of fdcgks_set_state): the initial
 *     state Wp0, Gp0, Wd0, Gd0, and dJ/d(final state) aWp, aGp, aWd, aGd.
 *   - Output (device arrays, same layouts): dJ/d(initial state) gWp, gGp,
 *     gWd, gGd.  The derivative is that of the discrete FP64 step, taking at
 *     every branch (GENO saturation, the positivity safeguard, the no-slip
 *     reset) the one the forward took; at exact ties of min/max and at
 *     |p_l - p_r| = 0 in tau it takes the mean of the one-sided derivatives.
 *   - The context runs the nsteps steps from the initial state and keeps
 *     the final state, as after fdcgks_set_state + fdcgks_steps.
 *   - Memory: checkpoints every checkpoint_every steps; each segment's states
 *     are recomputed from its checkpoint, each step's stage intermediates once
 *     more before its reverse pass (about three forward sweeps in all).  The
 *     call allocates a workspace of about ceil(nsteps / checkpoint_every) +
 *     checkpoint_every + 20 padded states and frees it before returning.
 *   - Mixed-precision contexts: the trajectory (checkpoints, recomputed
 *     segments, the final state the context keeps) is the context's own mixed
 *     run, kept between steps in FP64 buffers (a float-float pair round-trips
 *     to the same FP64 value; its low part can lose bits below 2^-53 of it,
 *     so the state follows the mixed run to FP64 rounding, about 1e-14
 *     relative after 50 steps); each step's reverse pass is the FP64 step's at those
 *     states, so the adjoint accumulates in FP64 and the result is the FP64
 *     step's derivative along the mixed trajectory.  With the linear
 *     reconstruction it matches the mixed run's own derivative to the FP32
 *     rounding of its fluxes.  With GENO it does not where the data vary by
 *     less than about 4e-6 of their size (a vortex's far field): the mixed
 *     step's GENO takes such data as smooth (an FP32 rounding floor in its
 *     smoothness indicators), the FP64 step's weights follow them.
 *   - Conservative reconstruction (recon_vars 0) and the boundary kinds of
 *     params.bc only (no fdcgks_set_sides); FDCGKS_ERR_ARG otherwise.
 *     A non-physical initial state returns FDCGKS_ERR_NONPHYSICAL (as
 *     fdcgks_set_state); FDCGKS_ERR_NOMEM when the workspace cannot be
 *     allocated; FDCGKS_ERR_CUDA on a failed launch or copy, after which the
 *     gradient arrays and the context's state are unspecified (load a state
 *     again with fdcgks_set_state).  Synchronizes the context stream. */
fdcgks_status fdcgks_vjp_steps(fdcgks_t ctx, double dt, int nsteps, int checkpoint_every, const double* Wp0,
                               const double* Gp0, const double* Wd0, const double* Gd0, const double* aWp,
                               const double* aGp, const double* aWd, const double* aGd, double* gWp, double* gGp,
                               double* gWd, double* gGd);

/* ------------------------------------------------------------------------
 * Batched ensemble.  The paper has no counterpart: its runs are independent,
 * and batching them is an execution strategy for parameter sweeps and
 * uncertainty studies with many small and mid-sized grids, which one at a
 * time cannot fill the GPU.  An ensemble holds `count` independent runs
 * ("members"), each with its own fdcgks_params (grid size, domain, boundary
 * conditions, gas constants, variants); every member advances exactly as a
 * context created with the same params would (same kernels per node, same
 * time-step formula), so member results equal single-context results.
 *   - All members share params[0].precision (FDCGKS_ERR_ARG otherwise).
 *   - params[m].stream is ignored: the ensemble owns one CUDA stream, given
 *     by fdcgks_ens_info, and every entry point below synchronizes it before
 *     returning except fdcgks_ens_run.
 *   - A step of the ensemble: each member's CFL time step is reduced on the
 *     device (the formula of fdcgks_cfl_dt, in FP64; the mixed path screens
 *     nodes with FP32 estimates first and evaluates in FP64 only those that
 *     can hold the maxima, which leaves the result unchanged), or taken from
 *     a fixed array, and both S2O4 stages of every member follow; one step
 *     is captured into a CUDA graph on first use and replayed.
 *   - Per-member status bits (fdcgks_ens_status): NONPHYSICAL when a stage
 *     produced non-positive or non-finite density or pressure; NO_WAVE_SPEED
 *     when no finite CFL rate was found; FROZEN once either happened (at the
 *     start of the next step): a frozen member is no longer advanced and its
 *     time stops, the others continue.  fdcgks_ens_set_state clears them.
 *   - Errors are reported through fdcgks_ens_last_error(ens); a failed
 *     fdcgks_ens_create reports through fdcgks_last_error(NULL).
 * ------------------------------------------------------------------------ */
typedef struct fdcgks_ens* fdcgks_ens_t;

#define FDCGKS_ENS_NONPHYSICAL 1
#define FDCGKS_ENS_NO_WAVE_SPEED 2
#define FDCGKS_ENS_FROZEN 4

/* Create an ensemble of `count` >= 1 members described by params[count]
 * (each validated as by fdcgks_create).  Allocates every member's buffers
 * in one device allocation.  *out is NULL on failure. */
fdcgks_status fdcgks_ens_create(const fdcgks_params* params, int count, fdcgks_ens_t* out);

/* Release an ensemble and its device memory.  NULL is accepted. */
void fdcgks_ens_destroy(fdcgks_ens_t ens);

/* Load / read the state of member m (arrays as for fdcgks_set_state /
 * fdcgks_get_state with that member's dims; host or device pointers per
 * on_device).  set_state validates density and pressure
 * (FDCGKS_ERR_NONPHYSICAL otherwise, member not loaded) and resets the
 * member's time and status. */
fdcgks_status fdcgks_ens_set_state(fdcgks_ens_t ens, int m, const double* Wp, const double* Gp, const double* Wd,
                                   const double* Gd, int on_device);
fdcgks_status fdcgks_ens_get_state(fdcgks_ens_t ens, int m, double* Wp, double* Gp, double* Wd, double* Gd,
                                   int on_device);

/* Advance every member nsteps steps.  dt == NULL: each member takes its own
 * CFL time step (number cfl > 0) at every step, computed on the device.
 * dt != NULL: host array dt[count] of fixed positive time steps (cfl is
 * ignored).  Asynchronous on the ensemble's stream (the host array is
 * copied before the call returns).  Every member must have a state. */
fdcgks_status fdcgks_ens_run(fdcgks_ens_t ens, double cfl, const double* dt, int nsteps);

/* Per-member elapsed time since its set_state, last time step taken and
 * status bits (FDCGKS_ENS_*), into host arrays [count]; any may be NULL. */
fdcgks_status fdcgks_ens_status(fdcgks_ens_t ens, double* t, double* last_dt, int* status);

/* Tile configuration cfg[4]: log2 of the tile width (0..7; the tile height is
 * 128 / width) of the nodal, point and update phases, then the dispatch
 * (1: persistent grid of resident blocks taking tiles from an atomic queue;
 * 0: one block per tile).  Default {5, 5, 5, 0}.  Results do not depend on
 * it. */
fdcgks_status fdcgks_ens_set_tiles(fdcgks_ens_t ens, const int* cfg);
fdcgks_status fdcgks_ens_get_tiles(fdcgks_ens_t ens, int* cfg);

/* Autotuner: times trial_steps CFL steps (number cfl) per candidate
 * configuration (coordinate descent over the three tile widths 8..128,
 * then the dispatch), keeps the fastest, and writes it to cfg_out[4] and
 * its ms per step to *ms_out (either may be NULL).  Every member's state,
 * time and status are restored afterwards (the tuner allocates a temporary
 * copy of all states).  Every member must have a state. */
fdcgks_status fdcgks_ens_tune(fdcgks_ens_t ens, double cfl, int trial_steps, int* cfg_out, double* ms_out);

/* Phase timing: runs nsteps CFL steps outside the graph with CUDA events
 * between phases and returns the summed milliseconds in ms[5]: CFL + time
 * step, ghost fill, nodal, points, update.  Advances the members. */
fdcgks_status fdcgks_ens_profile(fdcgks_ens_t ens, double cfl, int nsteps, double* ms);

/* The ensemble's cudaStream_t, the number of kernels its stepping path has
 * launched, and the total number of primary plus dual nodes (the node
 * updates of one step); any may be NULL. */
fdcgks_status fdcgks_ens_info(fdcgks_ens_t ens, void** stream, long long* launches, long long* nodes);

/* Message of the last failed call on ens (NULL: as fdcgks_last_error(NULL)). */
const char* fdcgks_ens_last_error(fdcgks_ens_t ens);

/* ---- The paper's one-dimensional scheme (Sec. 2) on a batch of lines ----
 * Each line is one grid of n nodes at x0 + (j + 1/2) h, h = (x1 - x0) / n,
 * carrying W = (rho, rho U, rho E) and the averaged gradient W_x over
 * [x_{j-1/2}, x_{j+1/2}] (Eq. define-averaged-gradient).  A stage
 * reconstructs the interface states (Sec. 3, GENO, the same options as the
 * 2-D scheme), solves the BGK interface problem (App. A; the 1-D gas is the
 * 2-D one with V = 0 and no y-variation), forms the nodal fluxes and the
 * compact flux (Eqs. fd-conservative-flux*) and updates W and W_x with
 * S2O4 (Eqs. eq-nodal-update, eq-interface-update); the interface values
 * of the gradient update are the solve's own W^(l,r) (Eq. eq:W-model).
 * The lines share grid, gas and options and evolve independently: one
 * thread block (or a cluster of blocks, see cluster) advances one line
 * through whole steps, so a call is one kernel launch whatever the number of
 * steps.  FP64 or mixed precision (see precision).
 *   - bc[0], bc[1]: PERIODIC (both ends), TRANSMISSIVE or SYMMETRY
 *     (a reflecting wall); n >= 3 (bounded) or >= 1 (periodic); batch >= 1.
 *   - State arrays W [batch][3][n] and Wx [batch][3][n], row-major; host or
 *     device (on_device) memory owned by the caller.
 *   - Each line keeps its own time (0 after set_state), advanced by every
 *     step of fdcgks_line_steps and fdcgks_line_run.
 *   - Errors: FDCGKS_ERR_ARG for invalid arguments (nothing changed),
 *     FDCGKS_ERR_CUDA for a failed allocation, copy or launch; messages via
 *     fdcgks_line_last_error (fdcgks_last_error(NULL) for a failed create). */
typedef struct {
  int n, batch;
  double x0, x1;
  double gamma, mu, Pr;
  int bc[2];
  int flux_variant, geno_variant, grad_base;
  double tau_c1, tau_c2;
  int recon_vars;
  void* stream;                /* cudaStream_t, NULL = default stream */
  int cluster;                 /* blocks per line: 1, 2, 4 or 8 (a thread-block cluster
                                  on as many SMs), or 0: automatic (clusters while the
                                  batch leaves SMs idle, >= 32 nodes per block).  The
                                  results do not depend on it. */
  int precision;               /* FDCGKS_FP64, or FDCGKS_MIXED: reconstruction, kinetic
                                  solves and compact fluxes in FP32 (FP64 time
                                  coefficients, as the 2-D mixed path); state and S2O4
                                  accumulation in FP64 either way */
} fdcgks_line_params;
typedef struct fdcgks_line_ctx* fdcgks_line_t;
fdcgks_status fdcgks_line_create(const fdcgks_line_params* params, fdcgks_line_t* out);
void fdcgks_line_destroy(fdcgks_line_t ctx);
fdcgks_status fdcgks_line_set_state(fdcgks_line_t ctx, const double* W, const double* Wx, int on_device);
fdcgks_status fdcgks_line_get_state(fdcgks_line_t ctx, double* W, double* Wx, int on_device);
/* nsteps steps of size dt > 0 on every line (one launch, asynchronous). */
fdcgks_status fdcgks_line_steps(fdcgks_line_t ctx, double dt, int nsteps);
/* Each line advances from its own time to t_end with its own CFL steps,
 * dt = cfl min h/(|U| + c) (and cfl h^2/(8 nu_max) when mu > 0), the last
 * one clipped to land on t_end, at most max_steps steps; a line whose time
 * step is not positive and finite stops and sets status bit 1, a line with
 * a non-physical node after a step stops there (bit 0).  One launch;
 * waits for it.  t[batch] and steps[batch] (host, either may be NULL)
 * receive each line's time and the number of steps it took. */
fdcgks_status fdcgks_line_run(fdcgks_line_t ctx, double t_end, double cfl, int max_steps, double* t, int* steps);
/* One stage's operator of the current state with time step dt: L, dL/dt,
 * the averaged gradient re-evaluated from the interface solution and its
 * time derivative, [batch][3][n] device arrays each. */
fdcgks_status fdcgks_line_stage_operator(fdcgks_line_t ctx, double dt, double* L, double* Lt, double* gb,
                                         double* gt);
/* Status bits of each line since set_state (bit 0: a node left the physical
 * states after a stage; bit 1: no positive finite CFL time step): flags
 * [batch] (host, may be NULL) and their OR in *any (may be NULL).  Waits. */
fdcgks_status fdcgks_line_check(fdcgks_line_t ctx, int* flags, int* any);
/* Message of the last failed call on ctx (NULL: as fdcgks_last_error(NULL)). */
const char* fdcgks_line_last_error(fdcgks_line_t ctx);

/* Message of the last failed call on ctx (or of the last failed
 * context-free call when ctx is NULL). */
const char* fdcgks_last_error(fdcgks_t ctx);

/* Static name of a status code. */
const char* fdcgks_status_string(fdcgks_status s);

#ifdef __cplusplus
}
#endif

#endif /* FDCGKS_H */
