/* hzn.h -- C-ABI of the GB300 GRMHD finite-volume library (libhzn.so, sm_103a).
 *
 * The library advances the conservation form of ideal general-relativistic MHD in a fixed
 * spacetime (§2.1 Eq. 2, compact form §2.2 Eq. 3) on a uniform Cartesian mesh with the
 * scheme of §2.2/§3.2: MC-limited reconstruction of the primitive variables, HLLE fluxes,
 * flux divergence plus metric source, third-order Runge-Kutta, Newton-Raphson recovery of
 * the primitive variables and hyperbolic divergence cleaning.  One full RK3 step is three
 * fused stencil launches (one per substep) on the caller's CUDA stream.
 *
 * Conventions shared by every call
 *   - Return value: HZ_OK (0) on success, a negative HZ_ERR_* on error, HZ_WARN_C2P (> 0)
 *     when the call completed but cells were reset to atmosphere (count in hz_stats).
 *     No call aborts, throws or prints.  hz_strerror() names every code.
 *   - Pointers named d_* are CUDA device pointers owned by the caller; the library never
 *     frees them and never keeps them beyond the call (inputs are copied into the workspace).
 *     Host pointers are named h_* or are plain out-parameters.
 *   - Grid functions are field-major, x fastest, no padding: field f of cell (i, j, k) is at
 *     [f * N + (k * ny + j) * nx + i], N = nx * ny * nz.  The metric carries one ghost layer
 *     on every active axis (an axis with n > 1): Nm = (nx + 2gx)(ny + 2gy)(nz + 2gz), g = 1
 *     on an active axis and 0 otherwise, and cell (i, j, k) sits at (i + gx, j + gy, k + gz).
 *   - Primitive fields (9): rho, p, u~^x, u~^y, u~^z, B^x, B^y, B^z, psi.  u~^i = W v^i =
 *     u^i + W beta^i / alpha is the primitive velocity of §5.2 (footnote); B^i = *F^{it} (§2.1);
 *     psi is the divergence-cleaning scalar (ignored and kept 0 when cleaning is off).
 *   - Conserved fields (9): sqrt(-g) rho u^t, sqrt(-g) T^t_t, sqrt(-g) T^t_x,y,z,
 *     sqrt(-g) B^x,y,z (§2.1, the eight conservative quantities), Psi = sqrt(gamma) psi.
 *   - Metric fields (10): alpha, beta^x, beta^y, beta^z, gamma_xx, _xy, _xz, _yy, _yz, _zz.
 *   - All device work is enqueued on the stream given to hz_create and is asynchronous unless
 *     the call says it synchronises.  A context must not be used from two host threads at once.
 */
#ifndef HZN_H
#define HZN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HZN_VERSION 1

enum {
  HZ_OK = 0,
  HZ_WARN_C2P = 1,       /* completed; some cells were reset to atmosphere              */
  HZ_ERR_ARG = -1,       /* invalid argument (null pointer, bad size, bad option)        */
  HZ_ERR_CUDA = -2,      /* a CUDA runtime call failed (the context may be unusable)     */
  HZ_ERR_STATE = -3,     /* call out of order (e.g. step before metric and primitives)   */
  HZ_ERR_WORKSPACE = -4, /* workspace pointer misaligned or smaller than required        */
  HZ_ERR_UNSUPPORTED = -5,/* option combination not built                                */
  HZ_ERR_TOO_LARGE = -6  /* grid needs more than HZ_NOALLOC_SCRATCH_BYTES (hz_step_noalloc) */
};

enum { HZ_BC_OUTFLOW = 0, HZ_BC_PERIODIC = 1 };
enum { HZ_FP64 = 0, HZ_MIXED = 1, HZ_FP64_DW = 2 };
enum { HZ_RECON_MC = 0, HZ_RECON_PPM = 1 };
enum { HZ_C2P_2D = 0, HZ_C2P_1D = 1 };

typedef struct hz_ctx hz_ctx; /* opaque; host-side bookkeeping, owned by the library */

/* Uniform Cartesian mesh.  An axis with n = 1 is inactive (no flux, no metric derivative).
 * Active axes need n >= 2; outflow boundaries copy the nearest interior cell (zero gradient),
 * periodic ones wrap. */
typedef struct {
  int n[3];
  int bc[3];
  double dx[3];
} hz_grid;

/* Physics and numerics options (§3.2 lists the scheme choices; the values are run inputs). */
typedef struct {
  double gamma;     /* ideal-gas index, p = (gamma - 1) rho eps; 1 < gamma <= 3          */
  int precision;    /* HZ_FP64: every step in FP64.  HZ_MIXED: primitives and metric stored
                       in FP32; reconstruction, HLLE fluxes and sources in FP32 with the flux
                       divergence accumulated in FP32; the conserved state (stored in FP64),
                       its RK update, the recovery and the CFL maximum in FP64 (§3.2, §6).
                       HZ_FP64_DW: FP64 storage, RK update, recovery and CFL maximum as for
                       HZ_FP64; reconstruction, face states, HLLE fluxes, flux divergence and
                       sources in double-word arithmetic (a value is the sum of two FP32
                       numbers, about 48 significant bits) on the FP32 pipes.  MC
                       reconstruction only (HZ_ERR_UNSUPPORTED with HZ_RECON_PPM); the
                       adjoint and the ensemble take HZ_FP64 only                          */
  int cleaning;     /* 1: hyperbolic divergence cleaning with the field psi (§3.2)         */
  double ch;        /* cleaning speed as a fraction of light speed (0 < ch <= 1)          */
  double kappa;     /* cleaning damping rate (>= 0)                                       */
  double rho_floor; /* atmosphere density; a recovered rho below it resets the cell        */
  double rho_atm;   /* a cell whose D / sqrt(gamma) (= rho W) is below rho_atm is set to the
                       atmosphere without a recovery (0 disables)                           */
  double p_floor;   /* pressure floor                                                    */
  double atm_K;     /* atmosphere pressure = atm_K rho_floor^gamma when > 0, else p_floor */
  int c2p_maxit;    /* Newton iteration cap of the recovery (1 .. 200)                    */
  double c2p_tol;   /* recovery accuracy (1e-15 .. 1e-6): the FP64 stage (corrections with the
                       Jacobian of the FP32 root, each of which multiplies the error by about
                       2^-24; Newton steps if they do not settle) stops after a step
                       |dZ| <= 0.01 sqrt(c2p_tol) Z, which leaves an error below c2p_tol      */
  int recon;        /* HZ_RECON_MC: TVD with the MC limiter.  HZ_RECON_PPM: the piecewise
                       parabolic method (§3.2; interface parabola from MC-limited slopes, then
                       the monotonicity constraints; no steepening or flattening); needs at
                       least 3 cells on every active axis (HZ_ERR_UNSUPPORTED otherwise)       */
  int c2p;          /* HZ_C2P_2D: Newton in (Z, v^2), FP32 then FP64 (§3.2 "2D").  HZ_C2P_1D:
                       Newton in Z alone with v^2 eliminated, kept in its bracket by bisection
                       (§3.2 "1D").  Both return the same root to round-off                    */
} hz_options;

typedef struct {
  long long c2p_failures; /* cells reset to atmosphere since the last hz_set_primitives     */
  int c2p_max_iters;      /* largest Newton iteration count seen since then                 */
  double max_speed;       /* CFL rate of the newest state (see hz_max_speed)                */
  double t;               /* simulated time since the last hz_set_primitives               */
  double dt;              /* step size of the last step                                     */
  long long steps;        /* full RK3 steps since the last hz_set_primitives               */
} hz_stats;

/* Device bytes the caller must provide to hz_create for this grid and options.
 * Errors: HZ_ERR_ARG for null pointers or invalid grid/options. */
int hz_workspace_bytes(const hz_grid* grid, const hz_options* opts, size_t* bytes);

/* Create a context on the current CUDA device.  d_workspace: caller-owned device memory of at
 * least hz_workspace_bytes, 256-byte aligned, valid until hz_destroy; the library allocates
 * no device memory of its own.  stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: HZ_ERR_ARG, HZ_ERR_WORKSPACE, HZ_ERR_UNSUPPORTED, HZ_ERR_CUDA. */
int hz_create(hz_ctx** ctx, const hz_grid* grid, const hz_options* opts, void* d_workspace,
              size_t bytes, void* stream);

/* Release the host-side context (the workspace stays with the caller).  Null is accepted. */
int hz_destroy(hz_ctx* ctx);

/* Copy the metric at cell centres, ghost layer included (10 x Nm doubles, layout above) into
 * the workspace.  The metric is the fixed spacetime of §2.1 (Cowling approximation).  The copy
 * also checks whether the shift and the off-diagonal gamma_ij vanish everywhere; if they do,
 * the kernels drop those identically zero terms.  Synchronises the stream. */
int hz_set_metric(hz_ctx* ctx, const double* d_metric);

/* Copy the primitive state (9 x N doubles) into the workspace and compute the conserved
 * state w(u) per cell (§2.2: algebraic).  Resets time, step count and statistics, and
 * computes the CFL rate of the new state (see hz_max_speed).  Requires hz_set_metric. */
int hz_set_primitives(hz_ctx* ctx, const double* d_prim);

/* Copy out the current primitive / conserved state (9 x N doubles each). */
int hz_get_primitives(hz_ctx* ctx, double* d_prim);
int hz_get_conserved(hz_ctx* ctx, double* d_cons);

/* One full RK3 step (three substeps, §3.2) of size dt > 0, asynchronous on the stream. */
int hz_step(hz_ctx* ctx, double dt);

/* One full RK3 step with dt = cfl / max_speed taken on the device from the newest state and
 * clipped so that t does not pass t_end (dt = 0 once t = t_end).  Asynchronous: no host
 * synchronisation, so a sequence of calls can be captured in a CUDA graph. */
int hz_step_cfl(hz_ctx* ctx, double cfl, double t_end);

/* CFL rate of the current state: the maximum over cells of the sum over active axes of
 * max(|lambda+|, |lambda-|)/dx (each axis's bound widened to the cleaning speed when cleaning is
 * on), so that dt = cfl / rate; the RK3 update treats all axes at once (§3.2), so their Courant
 * numbers add.  In 1-D, the per-axis maximum.  Synchronises the stream. */
int hz_max_speed(hz_ctx* ctx, double* h_out);

/* Statistics of the run so far.  Synchronises the stream.  Returns HZ_WARN_C2P when
 * c2p_failures > 0. */
int hz_get_stats(hz_ctx* ctx, hz_stats* h_out);

/* Static description of a return code. */
const char* hz_strerror(int code);

/* HZN_VERSION of the loaded library. */
int hz_version(void);

/* The CUDA runtime error code (a cudaError_t value) behind the last HZ_ERR_CUDA that a call of
 * this library returned on the calling host thread; 0 if none has.  Not cleared by later calls
 * that succeed.  No counterpart in the paper: it makes HZ_ERR_CUDA diagnosable. */
int hz_last_cuda_error(void);

/* Static description of a CUDA runtime error code (cudaGetErrorString). */
const char* hz_cuda_error_string(int cuda_code);

/* ---- Ensembles of independent 1-D tubes ------------------------------------------------
 * Many independent 1-D Riemann problems (the shock tubes of §5.1) advanced to a common end
 * time in one persistent launch.  Each tube has its own cell count n[t] >= 2, cell width dx[t]
 * and adiabatic index gamma[t], Minkowski spacetime, outflow boundaries, and its own CFL time
 * step; the scheme is that of the grid path (MC, HLLE, RK3, Newton recovery; §2.2, §3.2) in
 * FP64 without divergence cleaning (opts->precision = HZ_FP64, opts->cleaning = 0,
 * opts->recon = HZ_RECON_MC, opts->c2p = HZ_C2P_2D; the floors, rho_atm, atm_K and the recovery
 * options of hz_options apply).  A persistent grid of thread
 * blocks takes tubes from a work queue, most cells first; one block owns a tube for all its
 * steps, so no grid-wide synchronisation is needed.
 *
 * Caller layout of primitives: the tubes concatenated without padding and field-major over
 * the concatenation: field f of cell c of tube t at [f * Ncat + off[t] + c] with
 * off[t] = n[0] + ... + n[t-1], Ncat = sum n[t]; fields as for the grid (the ninth, psi, is
 * ignored), 9 x Ncat doubles. */
typedef struct hz_ensemble hz_ensemble;

/* Device bytes hz_ensemble_create needs for these tube sizes. */
int hz_ensemble_workspace_bytes(int ntubes, const int* h_n, size_t* bytes);

/* Create an ensemble over caller-owned device workspace (256-byte aligned).  Host arrays of
 * length ntubes.  Synchronises the device (uploads its tables).  Errors: HZ_ERR_ARG,
 * HZ_ERR_WORKSPACE, HZ_ERR_UNSUPPORTED (mixed precision or cleaning), HZ_ERR_CUDA. */
int hz_ensemble_create(hz_ensemble** ens, int ntubes, const int* h_n, const double* h_dx,
                       const double* h_gamma, const hz_options* opts, void* d_workspace,
                       size_t bytes, void* stream);
int hz_ensemble_destroy(hz_ensemble* ens);

/* Copy in the primitive state of every tube (layout above) and compute the conserved state. */
int hz_ensemble_set_primitives(hz_ensemble* ens, const double* d_prim);

/* Launch shape: threads per block and blocks per SM, one of (64,4), (128,1), (128,2),
 * (128,3), (256,1).  Default (128,2). */
int hz_ensemble_set_launch(hz_ensemble* ens, int threads, int ctas_per_sm);

/* Advance every tube from t = 0 to t_end with dt = cfl / max|lambda|/dx of that tube, at most
 * max_steps steps per tube, in one kernel launch.  use_graph = 1 captures the launch (with
 * its queue reset) in a CUDA graph on first use and replays the graph afterwards; capture
 * needs a stream other than the legacy default stream.  Asynchronous. */
int hz_ensemble_run(hz_ensemble* ens, double t_end, double cfl, long long max_steps, int use_graph);

/* Copy out the primitive state of every tube (layout above). */
int hz_ensemble_get_primitives(hz_ensemble* ens, double* d_prim);

/* Per-tube time reached, steps taken and recovery failures of the last run (host arrays of
 * length ntubes).  Synchronises the stream; HZ_WARN_C2P if any tube had failures. */
int hz_ensemble_results(hz_ensemble* ens, double* h_t, long long* h_steps, long long* h_fails);

/* Autotuner: time a probe run to t_probe for each launch shape above, keep the fastest, and
 * restore the state from d_prim.  Outputs the chosen shape and, if h_ms is not null, the five
 * probe times in ms.  Synchronises the stream. */
int hz_ensemble_autotune(hz_ensemble* ens, const double* d_prim, double t_probe, double cfl,
                         int* h_threads, int* h_ctas_per_sm, float* h_ms);

/* ---- Adjoint (reverse-mode gradient) of a fixed-step run -------------------------------
 * The paper motivates the method by inverse problems on astrophysical sources (§1) but has no
 * adjoint; these calls differentiate the discrete update of §2.2/§3.2 exactly.  A forward run
 * of nsteps RK3 steps of fixed size dt from a primitive state P(0) stores checkpoints; the
 * backward call takes dJ/dP(n) (and optionally dJ/dU(n)) for any scalar J of the final state
 * and returns dJ/dP(0).  Every branch of the forward update (MC limiter case, HLLE wave-speed
 * bound, discriminant clamp, atmosphere reset, pressure floor) is frozen at the forward state;
 * the Newton recovery of §2.2 is differentiated by the implicit-function theorem
 * (dP/dU = (dU/dP)^{-1} at the recovered state).  At a pressure-floor reset the Jacobian is
 * taken at the floored state.
 *
 * Memory: sqrt(nsteps)-step checkpointing.  The forward pass stores (P, U) every ckpt_every
 * steps (ckpt_every <= 0 picks ceil(sqrt(nsteps))); the backward pass recomputes one segment
 * at a time with the forward kernels into a tape of its 3 ckpt_every + 1 substep states.
 * FP64 with MC reconstruction only (HZ_ERR_UNSUPPORTED for HZ_MIXED or HZ_RECON_PPM); cleaning
 * on or off; either recovery scheme; any metric, 1-3 axes.
 * Layouts of the gradients are those of the primitive / conserved state (9 x N doubles). */
typedef struct hz_adjoint hz_adjoint;
/* Device bytes hz_adjoint_create needs. */
int hz_adjoint_workspace_bytes(const hz_grid* grid, const hz_options* opts, int nsteps,
                               int ckpt_every, size_t* bytes);
/* Create an adjoint driver on a context whose metric is set (hz_set_metric).  It uses the
 * context's stream and kernels; d_workspace: caller-owned, 256-byte aligned, at least
 * hz_adjoint_workspace_bytes.  The context must outlive the driver. */
int hz_adjoint_create(hz_adjoint** adj, hz_ctx* ctx, int nsteps, double dt, int ckpt_every,
                      void* d_workspace, size_t bytes);
int hz_adjoint_destroy(hz_adjoint* adj);
/* Checkpoint interval and number of segments in use (host outputs, either may be null). */
int hz_adjoint_checkpoint_interval(const hz_adjoint* adj, int* h_every, int* h_segments);
/* Set the context's primitive state to d_prim_in, advance nsteps steps of size dt storing the
 * checkpoints, and copy the final primitive state to d_prim_out (may be null).  The context
 * holds the final state afterwards, as after hz_step.  Asynchronous. */
int hz_adjoint_forward(hz_adjoint* adj, const double* d_prim_in, double* d_prim_out);
/* Reverse sweep of the last hz_adjoint_forward: d_gprim_out = dJ/dP(n), d_gcons_out =
 * dJ/dU(n) or null (zero); writes d_gprim_in = dJ/dP(0).  The context's primitive and
 * conserved state are left as the forward pass left them; its statistics (time, steps,
 * maximum speed) are those of the recomputation.  Asynchronous.  HZ_ERR_STATE before a
 * forward pass. */
int hz_adjoint_backward(hz_adjoint* adj, const double* d_gprim_out, const double* d_gcons_out,
                        double* d_gprim_in);
/* ---- Whole update without allocation --------------------------------------------------
 * The paper has no counterpart to this call; it is a convenience of this library.
 *
 * hz_create needs a caller-provided device workspace.  Some callers cannot allocate one: a
 * solver embedded as a plug-in in a host framework that owns all device memory through its
 * own pool and does not let plug-ins call cudaMalloc (an allocation outside the pool breaks
 * its accounting or fragments it), or a thin foreign-function layer that can only pass
 * pointers it was given.  hz_step_noalloc serves them: it takes the metric, the primitive
 * state in and a buffer for the primitive state out, advances nsteps RK3 steps of fixed size
 * dt (nsteps = 0 only converts to conserved and back), and writes the result.  It calls no
 * cudaMalloc, cudaFree or other allocating routine, on the device or the host.
 *
 * Its scratch (the workspace hz_create would take) is one static device array of
 * HZ_NOALLOC_SCRATCH_BYTES (16 MiB) inside libhzn.so; every GPU that loads the library holds
 * it until the process exits.  A grid whose hz_workspace_bytes exceeds that size is rejected
 * with HZ_ERR_TOO_LARGE (for example 24^3 cells with cleaning fit, 32^3 do not).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call before any
 *     stream capture.
 *   - Every call shares the one array and leaves its own state in it; each call overwrites
 *     everything it reads (and clears its counters) before use.  Calls whose GPU work
 *     overlaps (two streams, or two host threads) race on the array and give wrong results:
 *     serialise them.
 *   - Arguments and layouts are those of hz_set_metric / hz_set_primitives /
 *     hz_get_primitives; the work runs on stream.  The call synchronises the stream twice:
 *     after the metric scan (it reads back the metric class to choose the kernels, as
 *     hz_set_metric does) and at the end, so it returns with d_prim_out written.
 *   - Returns HZ_OK, or HZ_WARN_C2P when the recovery failed in some cells during the run
 *     (those cells were reset to the atmosphere, as hz_get_stats reports for a context);
 *     HZ_ERR_ARG, HZ_ERR_TOO_LARGE, HZ_ERR_UNSUPPORTED or HZ_ERR_CUDA otherwise. */
#define HZ_NOALLOC_SCRATCH_BYTES (16u << 20)
int hz_step_noalloc(const hz_grid* grid, const hz_options* opts, const double* d_metric,
                    const double* d_prim_in, double* d_prim_out, double dt, int nsteps,
                    void* stream);

/* ---- Self-test of the double-word arithmetic of HZ_FP64_DW ------------------------------
 * Not a step of the method: it exposes the pair-of-FP32 operations the HZ_FP64_DW kernels use,
 * so that their error bounds can be checked against exact arithmetic on the host.  For each
 * i < n it splits d_a[i] and d_b[i] into pairs x, y (integer split, as the kernels load
 * doubles) and writes, as the two floats (hi, lo) of each result widened to double,
 *   d_out[(2 q) n + i] = hi, d_out[(2 q + 1) n + i] = lo   for q = 0 .. HZ_DW_NRESULTS - 1:
 *   q = 0 x, 1 y, 2 x + y, 3 x - y, 4 x * y, 5 x / y, 6 sqrt(|x|), 7 1 / sqrt(|x|),
 *   8 the half MC slope of (x, y) (the reconstruction's limited slope).
 * d_a, d_b (n doubles) and d_out (2 HZ_DW_NRESULTS n doubles) are caller-owned device
 * memory; the work is enqueued on stream.  Returns HZ_ERR_ARG for null pointers or n < 0,
 * HZ_ERR_CUDA if the launch fails. */
#define HZ_DW_NRESULTS 9
int hz_dw_selftest(const double* d_a, const double* d_b, double* d_out, long long n,
                   void* stream);

/* ---- Self-test of the FP64 reciprocal of the FP64 kernels --------------------------------
 * Not a step of the method: d_out[i] = the reciprocal of d_x[i] as the FP64 kernels form it
 * (the hardware approximation refined by two Newton-Raphson steps, r <- r + r (1 - x r)), so
 * that its error against the correctly rounded 1/x can be checked.  Defined for normal x whose
 * reciprocal is normal.  d_x, d_out: n doubles of caller-owned device memory; work enqueued on
 * stream.  Returns HZ_ERR_ARG for null pointers or n < 0, HZ_ERR_CUDA if the launch fails. */
int hz_rcp_selftest(const double* d_x, double* d_out, long long n, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HZN_H */
