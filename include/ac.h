/*
 * ac.h -- C ABI of the GB300 pseudo-time residual sweep for the 2D inviscid
 * variable-density artificial-compressibility (AC) equations.
 *
 * Method: Leakey, Glenis & Hewett, "Riemann solvers and pressure gradients
 * in Godunov-type schemes for variable density incompressible flows"
 * (arXiv 2108.08769).  Equation and section numbers below refer to it.
 *
 *   governing equations        Sec. 2.1.1 (Eqs. AC_start - AC_end)
 *   compact form, Q = (rho, rho u, rho v, p/beta)           Sec. 2.1.2
 *   dual time stepping, RK stages, point-implicit scaling   Sec. 2.2, Alg. 1,
 *                                         Eqs. RK1, RK2, bdf, point_implicit
 *   local pseudo-time step                                  Sec. 2.2.3
 *   MUSCL + k-limiter, new pressure gradient                Sec. 2.3, Eq. new_gradp
 *   face rotation, Osher / Bassi / Roe fluxes               Sec. 2.4, Alg. 2
 *   ghost-cell boundaries, reversed gravity in wall ghosts  Sec. 2.5
 *
 * Conventions (all entry points):
 *  - Grids are uniform, cell-centred, nx * ny interior cells.  Host field
 *    arrays are caller-owned, nx*ny doubles, row-major with x fastest
 *    (index j*nx + i), interior cells only.  Every call copies; no host
 *    pointer is retained after a call returns.
 *  - The library owns all device memory of a context.  Device work runs on
 *    the context's stream (default stream unless ac_set_stream was called).
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - Return codes: AC_OK (0) on success, AC_NOT_CONVERGED (1) when a
 *    physical step hit max_iters (the state is advanced), negative values
 *    for errors.  After an error the state is the one before the call, and
 *    ac_last_error() describes the failure.
 */
#ifndef AC_H
#define AC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define AC_OK 0
#define AC_NOT_CONVERGED 1
#define AC_ERR_ARG (-1)       /* invalid argument (sizes, kinds, NULL, beta <= 0, ...) */
#define AC_ERR_CUDA (-2)      /* a CUDA runtime call failed */
#define AC_ERR_NONFINITE (-3) /* a residual norm or an input became NaN/Inf */
#define AC_ERR_TIMEOUT (-4)   /* reserved for a bounded device wait that gives up; no kernel here waits
                                 on another (every CTA is independent), so no call returns it */
#define AC_ERR_OOM (-5)       /* device allocation failed */
#define AC_ERR_STATE (-6)     /* call out of order (e.g. a step before ac_set_state) */

/* ---- boundary kinds (Sec. 2.5) ---------------------------------------- */
#define AC_BC_WALL_SLIP 0      /* mirror: rho, p copied; normal velocity negated */
#define AC_BC_WALL_NOSLIP 1    /* as slip, tangential velocity negated too */
#define AC_BC_TRANSMISSIVE 2   /* zero gradient: boundary cell copied */
#define AC_BC_PERIODIC 3       /* wrap; must be set on both sides of an axis */

/* ---- pressure-gradient methods (Sec. 2.3.2) --------------------------- */
#define AC_GRADP_NEW 0         /* rearranged momentum equation (Eq. new_gradp), default */
#define AC_GRADP_MINMOD 1      /* standard k-limiter on p, k = 1 */
#define AC_GRADP_SUPERBEE 2    /* standard k-limiter on p, k = 2 */
#define AC_GRADP_SPLIT_MINMOD 3   /* Qian et al. hydrostatic/kinematic split, k = 1 */
#define AC_GRADP_SPLIT_SUPERBEE 4 /* Qian et al. hydrostatic/kinematic split, k = 2 */

/* ---- Riemann solvers (Sec. 2.4) ---------------------------------------- */
#define AC_RIEMANN_OSHER 0     /* Dumbser-Toro Osher flux, 3-point Gauss path (default) */
#define AC_RIEMANN_BASSI 1     /* flux of the exact solution of Bassi et al. (Sec. 2.4.1) */
#define AC_RIEMANN_ROE 2       /* Roe flux with the Roe averages of Sec. 2.4.2 */

/* ---- arithmetic -------------------------------------------------------- */
#define AC_PREC_FP64 0         /* every step in FP64 */
#define AC_PREC_MIXED 1        /* FP32 sweep; FP64 time levels, reference pressure, norms */

typedef struct {
    int nx, ny;        /* interior cells, >= 1 each */
    double lx, ly;     /* domain extent (m); dx = lx/nx, dy = ly/ny */
    double gx, gy;     /* gravity (m/s^2), body force rho g (Sec. 2.1.2) */
} ac_grid;

typedef struct {
    double rho_heavy;  /* densest fluid present (kg/m^3) */
    double rho_light;  /* lightest fluid present (kg/m^3) */
} ac_fluids;

typedef struct {
    int xlo, xhi, ylo, yhi;   /* AC_BC_* per side */
} ac_bc;

typedef struct {
    int rk_stages;       /* s_max, 1..4 (default 3); alpha_s = 1/(s_max - s + 1) */
    int riemann;         /* AC_RIEMANN_* (default Osher) */
    int gradp;           /* AC_GRADP_* (default AC_GRADP_NEW) */
    int limiter_k;       /* k of the limiter on rho, u, v: 1 minmod (default), 2 superbee */
    int local_dtau;      /* 1: local pseudo-time step (default); 0: global minimum */
    int realtime;        /* 1: real-time term on (default); 0: pure pseudo-time */
    int alpha_pi_p_row;  /* 1: alpha_PI also scales the pressure row (default) */
    int precision;       /* AC_PREC_* (default AC_PREC_FP64) */
    double cfl_tau;      /* pseudo-time Courant number (default 0.45) */
    double abs_tol[4];   /* absolute residual floors for rho, rho u, rho v, p (default 0) */
    int bdf_order;       /* real-time derivative (Eq. bdf, Table BDF): 1 Backward-Euler (default),
                            2 BDF2, 3 BDF3; a context's first step after ac_set_state is always
                            Backward-Euler, its second at most BDF2 (Sec. 2.2.2) */
} ac_options;

typedef struct ac_ctx ac_ctx;

/* Fill *opt with the defaults listed above.  Returns AC_OK, or AC_ERR_ARG
 * for NULL. */
int ac_default_options(ac_options *opt);

/* beta (Pa) that gives the fluid of density rho_ref the artificial sound
 * speed sqrt(4 beta/rho_ref)/2 = c0 at rest, i.e. beta = rho_ref * c0^2
 * (Sec. 2.1.3: c = sqrt(u^2 + 4 beta/rho), acoustic speeds (u +- c)/2). */
double ac_beta_from_speed(double c0, double rho_ref);

/* Create a context for one tank.  grid, bc must be non-NULL; fluids may be
 * NULL (when given, ac_set_state rejects densities outside
 * [rho_light/2, 2 rho_heavy]); opt may be NULL (defaults).  beta > 0 in Pa
 * (Eq. AC_end).  Allocates the device state on the current device.  Cells
 * are indexed with 32-bit integers on the device: nx*ny may not exceed 2^31
 * (AC_ERR_ARG).
 * Errors: AC_ERR_ARG, AC_ERR_OOM, AC_ERR_CUDA.  *out is NULL on error. */
int ac_create(const ac_grid *grid, const ac_fluids *fluids, double beta, const ac_bc *bc,
              const ac_options *opt, ac_ctx **out);

/* Release all device and host memory of ctx (NULL is ignored). */
void ac_destroy(ac_ctx *ctx);

/* Run the context's device work on `stream` (a cudaStream_t passed as
 * void*; NULL = default stream).  Captured graphs are rebuilt lazily. */
int ac_set_stream(ac_ctx *ctx, void *stream);

/* Set the state Q = (rho, rho u, rho v, p) from host arrays (nx*ny doubles
 * each); the solvers see p as p/beta, the fifth component of the compact
 * form (Sec. 2.1.2).  Also sets the real-time level Q^n := Q, the
 * assignment that opens every physical step of Alg. 1, and clears the older
 * levels (Sec. 2.2.2: the next step starts from Backward-Euler).  rho must
 * be finite and > 0; all values finite (AC_ERR_NONFINITE otherwise,
 * AC_ERR_ARG for rho <= 0). */
int ac_set_state(ac_ctx *ctx, const double *rho, const double *rhou, const double *rhov,
                 const double *p);

/* Copy the current state Q = (rho, rho u, rho v, p) (Sec. 2.1.2, with p in
 * Pa rather than p/beta) to host arrays (nx*ny doubles each; any pointer may
 * be NULL to skip that field): after a physical step this is Q^{n+1}, the
 * converged pseudo-time state of Alg. 1.  Synchronises the context's
 * stream. */
int ac_get_state(const ac_ctx *ctx, double *rho, double *rhou, double *rhov, double *p);

/* One real-time step of dual time stepping (Alg. 1): Q^n <- Q, then
 * pseudo-iterations of s_max Runge-Kutta stages (Eqs. RK1-RK2) until every
 * field's residual norm R_k <= max(tol * R0_k, abs_tol_k) or max_iters
 * iterations have run.  R_k is the RMS over cells of the stage-1 bracket of
 * Eq. RK2 (pressure row in Pa/s); R0 is the first iteration's norm.  tol < 0
 * runs exactly max_iters iterations.  dt > 0 (ignored when the real-time
 * term is off), max_iters >= 1.
 * Returns AC_OK (converged, or tol < 0), AC_NOT_CONVERGED, or an error;
 * *iters_out (may be NULL) receives the iterations completed.  On
 * AC_ERR_NONFINITE the state is restored to its value before the call. */
int ac_physical_step(ac_ctx *ctx, double dt, double tol, int max_iters, int *iters_out);

/* Pure pseudo-time evolution (the set-up of the Riemann problems of Sec.
 * 3.1): with the real-time term off and the global pseudo-time step
 * (options realtime = 0, local_dtau = 0), run pseudo-iterations of s_max
 * Runge-Kutta stages (Eq. RK2) from the current state until the pseudo-time
 * reaches tau_end, the last step shortened to land on it, or max_iters
 * iterations have run.  The state is advanced in place (no stopping test).
 * Returns AC_OK when tau_end was reached, AC_NOT_CONVERGED when max_iters
 * came first, AC_ERR_ARG for other options or tau_end not finite and > 0;
 * *iters_out (may be NULL) receives the iterations run. */
int ac_pseudo_time_run(ac_ctx *ctx, double tau_end, int max_iters, int *iters_out);

/* Residual norms of the last physical step (Alg. 1's convergence test;
 * the paper does not define the norm, and this library reads it as the RMS
 * over cells of the stage-1 bracket of Eq. RK2, pressure row in Pa/s):
 * out[4] = final R (rho, rho u, rho v, p), out0[4] (may be NULL) =
 * first-iteration R0. */
int ac_residual_norms(const ac_ctx *ctx, double out[4], double out0[4]);

/* Global real-time step from a real-time Courant number (Sec. 2.2.4):
 * dt = min over cells of CFL_t |Omega| / (|u| dy + |v| dx), from the current
 * state; +inf when the fluid is at rest everywhere.  cfl_t > 0.  The
 * real-time term is point-implicit, so this sets resolution, not
 * stability.  Synchronises the context's stream. */
int ac_realtime_dt(ac_ctx *ctx, double cfl_t, double *dt_out);

/* Real-time history, for checkpointing and for BDF2/BDF3: level k (1 or 2)
 * is (rho, rho u, rho v) of the state k physical steps before the current
 * one.  Level 1 exists after one step (or ac_set_history(ctx, 1, ...)),
 * level 2 after two steps and only when bdf_order >= 2.  Restoring a
 * checkpoint: ac_set_state, then ac_set_history for level 1, then level 2.
 * ac_set_state forgets the history; so does a step that fails with
 * AC_ERR_NONFINITE (the next step is Backward-Euler).
 * Errors: AC_ERR_ARG (k out of range, level 2 without bdf_order >= 2),
 * AC_ERR_STATE (level not available yet, or level 2 set before level 1). */
int ac_get_history(const ac_ctx *ctx, int k, double *rho, double *rhou, double *rhov);
int ac_set_history(ac_ctx *ctx, int k, const double *rho, const double *rhou, const double *rhov);

/* Number of kernels this context has launched since creation (device work
 * inside captured graphs is counted per replay). */
long long ac_kernel_launches(const ac_ctx *ctx);

/* Per-kernel timing.  With profiling on, ac_physical_step launches each
 * pseudo-iteration's kernels from the host (no captured graph, one host
 * wait per iteration) and brackets every stage-sweep launch with a pair of
 * CUDA events on the context's stream; the numerical result is the same.
 * ac_stage_kernel_time returns the summed event time (ms) and the number
 * of stage-sweep launches measured since profiling was switched on. */
int ac_set_profiling(ac_ctx *ctx, int on);
int ac_stage_kernel_time(const ac_ctx *ctx, double *total_ms, long long *launches);

/* The stage-sweep variant the autotuner chose at the first physical step
 * (AC_ERR_STATE before it): tile width tx, height ty, threads per CTA and
 * the variant's index in the library's table.  Setting the environment
 * variable AC_TILE (mixed form) or AC_TILE_F64 (FP64) to an index before the
 * first step forces that variant.  The Bassi and Roe fluxes always run
 * variant 0, and so does BDF2/BDF3 in the mixed form; the mixed form's
 * column-strip variants implement the new pressure gradient only and are
 * replaced by variant 0 for the others. */
int ac_tile_shape(const ac_ctx *ctx, int *tx, int *ty, int *threads, int *variant);

/* Measurement helper, not part of the method: the device's FP64 fused
 * multiply-add rate in TFLOP/s (an FMA counted as 2 flops), timed with CUDA
 * events over a kernel of independent FMA chains on the current device
 * (about 10 ms, default stream; allocates and frees 1.2 MiB).  The FP64
 * sweep's roofline is checked against it.  Errors: AC_ERR_ARG, AC_ERR_OOM,
 * AC_ERR_CUDA. */
int ac_probe_fp64_fma_tflops(double *tflops);

/* ---- many tanks at once (mixed form) -------------------------------------
 * A batch advances n independent tanks of any sizes, densities and beta in
 * the mixed form (FP32 sweep; FP64 time levels, reference pressure and
 * norms).  Every Runge-Kutta stage of every tank is one kernel launch over
 * the flattened tiles of all tanks; each tank keeps its own pseudo-iteration
 * count, residual norms and convergence flag (Alg. 1 per tank), and a tank
 * that has converged stops consuming work while the others iterate.  One
 * physical step is one graph launch whose WHILE loop runs until every tank
 * has stopped.  The tile shape (cells per CTA, threads per CTA) is chosen by
 * timing every compiled shape on the batch at its first step.
 * The tanks' own numbers do not depend on the rest of the batch.  With the
 * column-strip sweep they equal a single-tank context's bit for bit; with
 * the tile sweep (a separately compiled kernel, whose multiply-adds the
 * compiler may contract differently) they agree with it to round-off. */
typedef struct ac_batch ac_batch;

/* Create a batch: each tank is one instance of the problem of ac_create
 * (Sec. 2.1.1 equations, Sec. 2.5 boundaries, beta of Eq. AC_end).
 * grids[n], beta[n] (Pa) and bcs[n] describe the tanks, 1 <= n <= 65535;
 * opt (may be NULL) applies to all of them and must select AC_PREC_MIXED and
 * the local pseudo-time step.  The tanks together may hold at most 2^31
 * cells (each rounded up to its aligned slot).
 * Errors: AC_ERR_ARG, AC_ERR_OOM, AC_ERR_CUDA. */
int ac_batch_create(int n, const ac_grid *grids, const double *beta, const ac_bc *bcs, const ac_options *opt,
                    ac_batch **out);
void ac_batch_destroy(ac_batch *b);
int ac_batch_set_stream(ac_batch *b, void *stream);
/* State of tank k (0 <= k < n) from host arrays, as ac_set_state (Q^n := Q
 * of Alg. 1 for that tank). */
int ac_batch_set_state(ac_batch *b, int k, const double *rho, const double *rhou, const double *rhov,
                       const double *p);
/* State of tank k to host arrays, as ac_get_state (Q^{n+1} of Alg. 1 after
 * a step). */
int ac_batch_get_state(const ac_batch *b, int k, double *rho, double *rhou, double *rhov, double *p);
/* One physical step of every tank with its own dt[k]: Alg. 1 per tank
 * (Q^n <- Q, pseudo-iterations of the Runge-Kutta stages of Eq. RK2 until
 * that tank's residual test passes); tol and max_iters as in
 * ac_physical_step.  iters_out[n] and status_out[n] (may be NULL)
 * receive each tank's iterations and status (AC_OK, AC_NOT_CONVERGED,
 * AC_ERR_NONFINITE).  Returns AC_OK when every tank converged (or tol < 0),
 * AC_NOT_CONVERGED when some tank hit max_iters, AC_ERR_NONFINITE when some
 * tank's norm became non-finite (those tanks are restored to the start of
 * the step, the others advanced). */
int ac_batch_physical_step(ac_batch *b, const double *dt, double tol, int max_iters, int *iters_out,
                           int *status_out);
/* Residual norms of tank k's last step, as ac_residual_norms (Alg. 1). */
int ac_batch_residual_norms(const ac_batch *b, int k, double out[4], double out0[4]);
/* The tile shape the autotuner chose (AC_ERR_STATE before the first step). */
int ac_batch_tile_shape(const ac_batch *b, int *tx, int *ty, int *threads);
int ac_batch_set_profiling(ac_batch *b, int on);
int ac_batch_stage_kernel_time(const ac_batch *b, double *total_ms, long long *launches);
long long ac_batch_kernel_launches(const ac_batch *b);

/* ---- stage sweep without device allocation ------------------------------
 * This entry point has no counterpart in the paper: it exists for callers
 * that cannot allocate device memory -- code running inside a memory pool
 * it does not own, a sandbox or plug-in host that forbids allocation after
 * start-up, or a real-time loop where an allocation could stall or fail.
 *
 * One FP64 Runge-Kutta stage sweep (the same kernel ac_physical_step runs)
 * on caller-owned DEVICE arrays of nx*ny doubles (row-major, x fastest):
 *   q_prev  Q^{s-1} = (rho, rho u, rho v, p)   (ignored for stage 1)
 *   q0      Q^{m}, the state at the start of the pseudo-iteration
 *   qn      Q^n = (rho, rho u, rho v), the real-time level (may be NULL
 *           when opt->realtime is 0)
 *   q_out   receives Q^s (must not alias any input)
 *   norms   device array of 4 doubles receiving the residual norms R of
 *           the stage-1 bracket (stage 1 only; may be NULL)
 * grid, beta, bc and opt mean what they mean for ac_create; opt->precision
 * must be AC_PREC_FP64 and opt->bdf_order 1 (Backward-Euler real-time
 * term); stage is 1..opt->rk_stages; dt as in
 * ac_physical_step.  Work is enqueued on `stream` (a cudaStream_t; NULL =
 * default stream) and the call returns without waiting.
 *
 * No cudaMalloc, cudaFree or allocating library call is made.  The sweep's
 * scratch (control block and per-tile partial sums) is a fixed 1 MiB array
 * inside the library, so grids are limited to 32760 tiles of 32x8 cells
 * (about 8.39 million cells); larger grids are rejected with AC_ERR_ARG.
 * Every GPU that loads the library holds that 1 MiB until the process
 * exits.  All calls share the array: calls whose work overlaps on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller.  Every call looks up the array's address on the current device
 * and sets the kernel's shared-memory limit (host-side calls that allocate
 * nothing, so the address stays valid across a device reset); the first
 * call on a device may also load the library's kernels, so make that first
 * call before any stream capture.  The grid size is checked before any
 * field pointer is looked at. */
int ac_stage_sweep_noalloc(const ac_grid *grid, double beta, const ac_bc *bc, const ac_options *opt,
                           int stage, double dt, const double *const q_prev[4], const double *const q0[4],
                           const double *const qn[3], double *const q_out[4], double *norms, void *stream);

/* Message describing the last error on this thread ("" if none). */
const char *ac_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
