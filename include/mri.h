/*
 * mri.h -- C ABI of the GB300 fast-partition solver for multirate infinitesimal
 * (MRI) time integration of reacting flow.
 *
 * The method (Loffeld et al., "Performance of explicit and IMEX MRI multirate
 * methods on complex reactive flow problems ...", arXiv 2211.03293):
 *   y' = f^F(t, y) + f^S(t, y)                                   (Eq. 1)
 * One slow step H: Y_1 = y_n; for i = 2..s, with T_i = t_n + c_i H and
 * dc_i = c_i - c_{i-1}, solve the modified fast IVP
 *   v'(theta) = f^F(theta, v) + r_i(theta),  theta in [T_{i-1}, T_i],
 *   v(T_{i-1}) = Y_{i-1},  Y_i = v(T_i)                          (Eq. 3)
 * where the forcing r_i is built from f^S(T_j, Y_j), j <= i; y_{n+1} = Y_s
 * (Sec. 2.1, the stage algorithm).  f^F is the chemistry of each grid cell
 * (Sec. 3.2: f^F = omega_k W_k / rho for Eq. 6), f^S the transport.
 *
 * Conventions for every call:
 *   - state layout is cell-major y[ncell][n], n = Ns + 1, entries
 *     (Y_1 .. Y_Ns, T): mass fractions then temperature [K]; SI units;
 *   - all array arguments are DEVICE pointers owned by the caller (cudaMalloc,
 *     torch tensors, ...).  The library allocates device memory only in
 *     mri_mech_load (freed by mri_mech_free);
 *   - calls are asynchronous and ordered on `stream` (a cudaStream_t, NULL =
 *     legacy default stream); the return value covers host-side argument
 *     checks and launch errors only.  Per-cell results (Newton failure, bad
 *     input state) are written to cell_status on the device;
 *   - no call aborts or traps: errors are negative return codes;
 *   - a mechanism belongs to the device that was current when mri_mech_load ran:
 *     every call that uses it must be made with that device current (MRI_EINVAL
 *     otherwise, before anything is launched);
 *   - fast-stage launches on one mechanism may run concurrently on different
 *     streams: each takes its own device work-queue counter, eager launches from a
 *     ring of 256 (so at most 256 of them in flight at once) and launches recorded
 *     into a CUDA graph by stream capture from a second ring of 256 that eager
 *     launches never use, since a graph keeps its counter for every replay.  Graphs
 *     whose captured launches wrapped that ring (more than 256 captured stage
 *     launches on one mechanism) may share a counter and must not be replayed at
 *     the same time.
 */
#ifndef MRI_H
#define MRI_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define MRI_OK 0
#define MRI_EINVAL (-1)    /* bad argument, rejected on the host before any launch */
#define MRI_ENEWTON (-2)   /* at least one cell failed (see cell_status) */
#define MRI_ECUDA (-3)     /* a CUDA call failed (launch, copy, allocation) */
#define MRI_ETIMEOUT (-4)  /* a device work budget ran out */
#define MRI_ENOMEM (-5)    /* workspace too small */
#define MRI_ECONV (-6)     /* an iterative linear solve missed its tolerance in max_iter iterations */

/* ---- per-cell status written by the kernels -------------------------- */
#define MRI_CELL_OK 0
#define MRI_CELL_ENEWTON 1 /* Newton did not converge in max_newton iterations,
                              or produced a non-finite iterate; the cell keeps
                              the state at the start of the failed substep and
                              takes no further substeps in this call */
#define MRI_CELL_EINPUT 2  /* non-finite input state, T <= 0 or p <= 0: the
                              cell is left unchanged */
#define MRI_CELL_TIMEOUT 3 /* not run: the time budget of the call ran out before a
                              warp took the cell; the cell is left unchanged */

/* ---- fast integrators ------------------------------------------------ */
#define MRI_SDIRK2 2       /* Alexander (1977) 2-stage, order 2, L-stable, stiffly accurate */
#define MRI_SDIRK3 3       /* Alexander (1977) 3-stage, order 3, L-stable, stiffly accurate */
/* The paper's explicit fast methods (Sec. 3.2, the MRI-P(k) runs use explicit Runge-Kutta
 * fast integrators): fixed substeps only (no adaptive option), no Jacobian and no Newton
 * iteration, so the Newton, precision, solve-layout and matrix-cache options are ignored;
 * stable only where h times the chemistry's largest eigenvalue is small (a cell whose
 * state becomes non-finite stops with MRI_CELL_ENEWTON at the state before that substep).
 * cell_stats[1] counts right-hand-side evaluations, cell_stats[2] stays 0.
 * mri_stage_fast_guided and mri_stage_fast_batch reject them. */
#define MRI_ERK2 12        /* Heun's method: c = (0, 1), a21 = 1, b = (1/2, 1/2) */
#define MRI_ERK3 13        /* Kutta's third-order method: c = (0, 1/2, 1), a21 = 1/2,
                              a31 = -1, a32 = 2, b = (1/6, 2/3, 1/6) */
#define MRI_ERK4 14        /* classical fourth-order Runge-Kutta method */

/* ---- slow (MRI) methods ---------------------------------------------- */
#define MRI_KW3 1          /* explicit third-order method of Knoth & Wolke (1998) in
                              MIS form, the paper's "MRI3" slow method (Sec. 3.2) */

/* ---- mechanism ------------------------------------------------------- */
typedef struct mri_mech mri_mech;

/* Parse a mechanism blob and upload its tables to the current device.
 * blob: host bytes in the "MRIMECH1" layout (magic; int32 header
 *   [Ns, R, E, n_eff, n_troe, 0, 0, 0]; float64 W[Ns] kg/mol; float64
 *   nasa[Ns][7]; int32 elem[Ns][E]; int32 rtype[R] (0 plain, 1 third body,
 *   2 Troe falloff); int32 reac[R][3]; int32 prod[R][3] (species index,
 *   repeated for stoichiometry, -1 pad); int32 eff_row[R]; int32 troe_row[R];
 *   float64 A[R] (SI), b[R], Ta[R] (K); float64 eff[n_eff][Ns];
 *   float64 troe[n_troe][7] = (A0, b0, Ta0, a, T***, T*, T**); every int32
 *   section zero-padded to 8 bytes).  Production rates follow the standard
 *   Chemkin definitions the paper refers to (Sec. 3: omega_k of Eq. 4 and 6).
 * Limits: 1 <= Ns <= 127, 0 <= R <= 1023.
 * On success *out owns device memory until mri_mech_free.  Returns MRI_EINVAL
 * for a malformed blob, MRI_ECUDA if the upload fails. */
int mri_mech_load(const void* blob, size_t nbytes, mri_mech** out);
void mri_mech_free(mri_mech* mech);
int mri_mech_info(const mri_mech* mech, int* n_species, int* n_reactions);

/* ---- fast solve options ---------------------------------------------- */
#define MRI_JAC_PER_SUBSTEP 0 /* Jacobian + LU at the start of every substep, reused
                                 by all stages; refreshed inside Newton when the
                                 contraction is slow */
#define MRI_JAC_LAZY 1        /* the factorised Newton matrix also carries over to the
                                 next substeps of the call while h gamma is unchanged
                                 up to rounding (at most 12 substeps); refreshed inside
                                 Newton when the
                                 contraction is slow.  The converged stage values do not
                                 depend on the policy, only the cost does. */
#define MRI_PREC_FP64 0       /* plain path: everything in FP64 */
#define MRI_PREC_FP32_LU 1    /* mixed precision: Jacobian assembly, Newton matrix, LU and
                                 triangular solves in FP32; rates, residual, state update
                                 and convergence test in FP64.  Each Newton iteration's FP64
                                 residual refines the FP32 correction, so the converged
                                 stage values meet the same tolerance as the FP64 form. */

typedef struct {
  int method;            /* MRI_SDIRK2, MRI_SDIRK3 or an explicit MRI_ERK2/3/4 */
  double newton_rtol;    /* WRMS weights w_k = rtol |Z_k| + atol_k; converged when WRMS(delta) <= 1 */
  double newton_atol_Y;  /* absolute tolerance of the mass fractions */
  double newton_atol_T;  /* absolute tolerance of T [K] */
  int max_newton;        /* Newton iterations per SDIRK stage, 1..100 */
  int jac_policy;        /* MRI_JAC_PER_SUBSTEP or MRI_JAC_LAZY */
  int precision;         /* MRI_PREC_FP64 or MRI_PREC_FP32_LU */
  int ramp;              /* 0 = off; R in 1..40: the first substep of the call is
                            replaced by R+1 substeps of sizes hh 2^-R, hh 2^-R,
                            hh 2^(1-R), ..., hh/2 (sum hh), for states far from
                            the fast manifold */
  /* Launch shape of the persistent kernel (one warp per cell at a time; warps take
   * cells from a device work queue).  They change the cost only, never a result. */
  int warps_per_block;   /* 0 = automatic (as many as the shared memory holds, at most
                            12); else 1..12, rejected (MRI_EINVAL) if they do not fit */
  int blocks_per_sm;     /* 0 = automatic (1); else 1..8 resident CTAs per SM, each
                            with 1/blocks_per_sm of the SM's shared memory */
  double time_budget_s;  /* 0 = none.  > 0: warps stop taking new cells once this much
                            time has passed since they started (cells already taken
                            are finished).  The cells not taken are always the tail
                            [ncell - m, ncell) of the range: they keep their input
                            state, get status MRI_CELL_TIMEOUT and count in n_failed,
                            so a caller resumes by calling again on that tail.
                            mri_step rejects a budget. */
  /* Newton-matrix cache (nullable): a device buffer of mri_matrix_cache_size bytes
   * in which each cell's factorised Newton matrix, its h gamma and age survive from
   * one call to the next, so that MRI_JAC_LAZY reuses it across the stages and
   * steps of a run instead of refactorising at the start of every call.  The
   * caller zeroes it once (a zeroed entry is empty), keeps the cell order fixed
   * between calls that share it, and uses one cache per mechanism and precision;
   * entries of another n or precision are ignored.  Each entry also keeps f^F at
   * the cell's output state; with MRI_START_PREDICTOR the next call adds its own
   * forcing at the stage start to it and so predicts the Newton start of its first
   * stage too (a state changed by the caller in between only makes that start
   * worse).  Like the lazy policy itself the cache changes the cost, not the
   * converged results.  Calls that share a cache must not overlap on the GPU.
   * mri_stage_fast_batch rejects a cache. */
  void* matrix_cache;
  size_t matrix_cache_bytes;
  /* Adaptive substeps (the paper's fast steps are fixed; adaptivity is its stated
   * future work).  1: starting from the uniform substep Hstage/n_sub, each SDIRK step
   * is accepted when the WRMS norm (weights ctrl_rtol |y| + ctrl_atol) of the
   * embedded estimate h sum_i (b_i - bhat_i) F_i is at most 1, with bhat the weights
   * of one order lower on the same stages (SDIRK3: bhat_3 = 0, sum bhat = 1,
   * bhat . c = 1/2; SDIRK2: bhat = (1, 0)); the next size is the step's times the
   * largest of 4, 2, 1, 1/2 not above 0.9 err^(-1/q) (q = 3 for SDIRK3, 2 for SDIRK2;
   * 1/2 or 1/4 after a rejection, 1/4 after a Newton failure), never above Hstage,
   * and the last step ends exactly at Hstage.  A cell fails when a step falls below
   * Hstage 2^-40 or after 10000 attempts.  ramp is ignored; cell_stats[0] counts
   * accepted steps, [1] and [2] include rejected attempts.  h sets the first step. */
  int adaptive;
  double ctrl_rtol;
  double ctrl_atol_Y;
  double ctrl_atol_T;
  /* Acceptance of a Newton iterate computed with an older matrix (modified Newton,
   * linear convergence at the rate rho = WRMS(delta_k) / WRMS(delta_k-1)): besides
   * WRMS(delta_k) <= 1, the estimated remaining error rho WRMS(delta_k) must be at
   * most newton_safety, 0 < newton_safety <= 1 (default 3e-4).  The default keeps
   * each accepted stage value within about 1e-12 relative of the exact solution of
   * the stage equation, so whole MRI steps match a full-Newton solution to 1e-10;
   * a larger value accepts an iteration earlier more often, with the remaining error
   * still inside the Newton tolerance.  Iterates of a fresh matrix are accepted at
   * WRMS(delta) <= 1 either way. */
  double newton_safety;
  /* How warps get their cells (results are the same either way):
   * MRI_SCHED_QUEUE (default) from the launch's device work queue, so cells of uneven
   * cost balance; MRI_SCHED_STATIC a fixed mapping, warp w of the grid's W warps
   * integrates cells w, w + W, w + 2W, ... (the mapping the queue is measured
   * against).  Static scheduling takes no time budget and is rejected by
   * mri_stage_fast_batch (MRI_EINVAL). */
  int schedule;
  /* How the Newton matrix is factorised and every Newton iteration solved
   * (MRI_LU_*).  The triangular-solve layouts (AUTO, REGS, REGS_SPLIT, SHARED) share
   * the arithmetic and its order, so their results are bitwise identical; only the
   * cost differs.  MRI_LU_INVERSE computes the inverse instead, so its corrections
   * differ from the others by rounding (the converged stage values still meet the
   * Newton tolerance).  A dimension of the autotuner.  A matrix cache entry records
   * whether it holds LU factors or an inverse; an entry of the other kind counts as
   * empty. */
  int lu_variant;
} mri_fast_opts;

#define MRI_SCHED_QUEUE 0
#define MRI_SCHED_STATIC 1
#define MRI_LU_AUTO 0        /* n <= 64: in registers (FP64 factors with n > 32: the split
                                forward layout); larger n: shared memory */
#define MRI_LU_REGS 1        /* solution in registers, row lane + 32 r in register r
                                (n <= 64; larger n use MRI_LU_SHARED) */
#define MRI_LU_REGS_SPLIT 2  /* registers; for 32 < n <= 64 the forward pass holds rows
                                n - 32 + lane and the short block, then moves to the
                                MRI_LU_REGS layout for the backward pass (fewer FP64
                                instructions); n <= 32 as MRI_LU_REGS, larger n shared */
#define MRI_LU_SHARED 3      /* substitutions on the right-hand side in shared memory */
#define MRI_LU_INVERSE 4     /* Gauss-Jordan inversion with partial pivoting (the pivot
                                rule of the LU) at every Jacobian evaluation; every
                                Newton solve is then a matrix-vector product, with no
                                chain of dependent steps (one warp instruction of a
                                narrow FP64 unit costs the same whatever its active
                                lanes, and a substitution step waits on the previous) */

/* Fill opts with the defaults (SDIRK3, rtol 1e-10, atol_Y 1e-20, atol_T 1e-10 K,
 * 10 Newton iterations, per-substep Jacobian, FP64, no ramp, automatic launch
 * shape, no time budget, no matrix cache, fixed substeps; controller tolerances
 * 1e-6, 1e-12, 1e-6 K for the adaptive option; Newton safety 3e-4; work-queue
 * scheduling; automatic solve layout). */
void mri_fast_opts_default(mri_fast_opts* opts);

/* One MRI stage of the fast partition for every cell (Eq. 3):
 *   v' = f^F(v) + r(theta),  r(theta) = sum_{k<K} rhohat^k phi[cell][k][:],
 *   rhohat = (theta - t0) / Hstage in [0, 1],
 * integrated from v = y over [t0, t0 + Hstage] with n_sub = max(1,
 * ceil(Hstage/h (1 - 1e-12))) uniform SDIRK substeps of size Hstage/n_sub;
 * y is overwritten with v(t0 + Hstage).  f^F: dY_k/dt = omega_k W_k / rho,
 * dT/dt = -sum_k h_k omega_k / (rho cp) at the constant pressure p[cell]
 * (ideal gas, Eq. 5).
 *   y           [ncell][n] in/out
 *   p           [ncell] pressure [Pa]
 *   phi         [ncell][K][n] forcing coefficients (may be NULL when K == 0)
 *   K           0..4 forcing polynomial terms
 *   t0, Hstage  stage start time and length dc_i H [s] (Hstage > 0)
 *   h           target substep [s] (h > 0)
 *   cell_status [ncell] MRI_CELL_* or NULL
 *   cell_stats  [ncell][4] int32 or NULL: substeps taken, Newton iterations,
 *               Jacobian/LU factorizations, failures -- ADDED to what is there
 *   n_failed    one int32 or NULL: incremented by the number of cells whose
 *               status is not MRI_CELL_OK (caller zeroes it)
 * Returns MRI_OK once launched, MRI_EINVAL for bad sizes/options,
 * MRI_ECUDA on a launch failure. */
int mri_stage_fast(double* y, const double* p, int ncell, const double* phi, int K,
                   double t0, double Hstage, double h, const mri_mech* mech,
                   const mri_fast_opts* opts, int32_t* cell_status, int32_t* cell_stats,
                   int32_t* n_failed, void* stream);

/* ---- Newton starts and the learned form's guess ---------------------------- */
#define MRI_START_PREDICTOR 0   /* base + h gamma F_prev once a stage derivative is known,
                                   else the previous stage value (mri_stage_fast) */
#define MRI_START_PREVIOUS 1    /* always the previous stage value (y_n for the first stage) */
#define MRI_START_GUESS 2       /* the caller's predicted states at the substep ends,
                                   interpolated linearly to the stage's time */
#define MRI_START_GUESS_FIRST 3 /* the guess where the predictor has no derivative yet
                                   (the first SDIRK stage of the call), else the predictor */

/* mri_stage_fast with a chosen start for every Newton iteration and, for the
 * MRI_START_GUESS modes, predicted states guess [ncell][guess_steps][n] (device)
 * at the ends of the call's substeps: guess_steps must equal the call's substep
 * count n_sub = max(1, ceil(Hstage/h (1 - 1e-12))).  The Newton start of an SDIRK
 * stage at time theta in substep j (theta/hh - j = f in [0, 1)) is
 * (1 - f) guess[j-1] + f guess[j], with guess[-1] the input state (for example
 * the learned form's prediction, mri_mlp.h).  The start changes the
 * Newton path, not the stage equations: every stage value is still accepted only
 * by the FP64 residual and WRMS test, and where Newton does not converge from the
 * chosen start the stage is solved again with full Newton from the previous stage
 * value; n_fallback (device int32, nullable, added to) counts those restarts.  The
 * paper's explicit fast methods need no Newton start; this is part of the learned
 * form.  step_exp (device int8 [ncell], nullable; adaptive substeps only): each
 * cell's first step is the uniform substep Hstage/n_sub times 2^step_exp[c], with
 * step_exp clamped to [-20, 10] (the learned form's substep-size prediction; the
 * controller takes over from the second step).  Other arguments, results and codes
 * as mri_stage_fast. */
int mri_stage_fast_guided(double* y, const double* p, int ncell, const double* phi, int K, double t0,
                          double Hstage, double h, const double* guess, int guess_steps, int start,
                          const mri_mech* mech,
                          const mri_fast_opts* opts, int32_t* cell_status, int32_t* cell_stats,
                          int32_t* n_failed, int32_t* n_fallback, const int8_t* step_exp, void* stream);

/* ---- several mechanisms in one launch ------------------------------------ */
#define MRI_MAX_GROUPS 8

typedef struct {
  const mri_mech* mech;  /* mechanism of this group's cells (on the current device) */
  double* y;             /* [ncell][n] in/out, n = that mechanism's Ns + 1 */
  const double* p;       /* [ncell] */
  int ncell;             /* >= 0 */
  const double* phi;     /* [ncell][K][n] or NULL when K == 0 */
  int K;                 /* 0..4 */
  int32_t* cell_status;  /* [ncell] or NULL */
  int32_t* cell_stats;   /* [ncell][4] or NULL, added to */
} mri_stage_group;

/* mri_stage_fast over up to MRI_MAX_GROUPS groups of cells with different
 * mechanisms in ONE kernel launch (for example a batch of independent 0-D reactors
 * on a 9-, a 40- and an 80-species mechanism: K = 0 and no slow partition).  Every
 * group is integrated exactly as mri_stage_fast integrates it (same Hstage, h and
 * opts for all groups; the results are bitwise those of one mri_stage_fast call per
 * group).  The SMs are first split between the groups in proportion to an estimate
 * of their work; each group's CTAs hold its tables and take its cells from its own
 * queue, and a CTA whose group has no cells left stages the next group's tables and
 * takes cells from that group's queue, so the costliest group gets help at the end.
 * opts->warps_per_block and opts->time_budget_s must be 0, opts->blocks_per_sm 0 or
 * 1, opts->schedule the work queue and the method implicit (MRI_EINVAL otherwise).  n_failed (nullable) counts
 * failed cells over all groups.  The paper solves one mechanism at a time; mixing
 * mechanisms in one launch is a batching service of this library. */
int mri_stage_fast_batch(const mri_stage_group* groups, int ngroups, double t0, double Hstage, double h,
                         const mri_fast_opts* opts, int32_t* n_failed, void* stream);

/* Launch shape mri_stage_fast would use for ncell cells and K forcing terms with
 * these options on the current device: warps (= cells in flight) per CTA, CTAs in
 * the persistent grid and dynamic shared memory per CTA (staged tables plus one
 * workspace per warp).  A query for autotuning and reports; the paper has no
 * counterpart.  Returns MRI_EINVAL if the requested shape does not fit. */
int mri_stage_fast_shape(const mri_mech* mech, const mri_fast_opts* opts, int ncell, int K,
                         int* warps_per_block, int* blocks, size_t* smem_bytes);

/* Bytes of the Newton-matrix cache (mri_fast_opts.matrix_cache) for ncell cells of
 * a mechanism in a precision form (0 on bad arguments). */
size_t mri_matrix_cache_size(const mri_mech* mech, int ncell, int precision);

/* ---- slow partition ---------------------------------------------------- */
typedef struct {
  int nx, ny, nz;        /* periodic box; cell index (k*ny + j)*nx + i */
  double dx;             /* spacing [m], same on every axis */
  double u[3];           /* constant advection velocity [m/s] */
  double D;              /* diffusivity [m^2/s], same for every component */
  int order;             /* 2 or 4: central differences of that order */
} mri_grid;

/* f^S(y) = -u . grad(y) + D lap(y) for every component (Eq. 6 transport with
 * the advection sign taken as -div(Y u); Sec. 3.1: 2nd-order central stencils,
 * periodic).  Axes with one cell are skipped.  y, fS: [ncell][n] device.
 * The slow partition is autonomous: t is accepted for the interface only. */
int mri_slow_rhs(const double* y, double* fS, int n, const mri_grid* grid, double t, void* stream);

/* Stage forcing of the MIS form of an explicit MRI method: the polynomial r_i of
 * Eq. 3 built from slow evaluations (Sec. 2.1, step 2a), here its constant term
 *   phi[e] = sum_{j < nslow} coeffs[j] * fS[j * len + e],  e < len,
 * fS: nslow consecutive device arrays of len doubles (f^S(Y_1), f^S(Y_2), ...),
 * coeffs: host array of nslow values (a row of mri_method_coupling's G),
 * phi: device output of len doubles.  1 <= nslow <= 3. */
int mri_stage_forcing(const double* fS, int nslow, long long len, const double* coeffs, double* phi,
                      void* stream);

/* Host-side coupling table of the MRI method: stage times c[0..s) and, for stage
 * i = 1..s-1, G[i*3 + j] = (a_ij - a_{i-1,j}) / (c_i - c_{i-1}) -- the weight of
 * f^S(Y_j) in stage i's constant forcing.  For MRI_KW3 (Knoth & Wolke ERK3 with
 * c = (0, 1/3, 3/4), a21 = 1/3, a31 = -3/16, a32 = 15/16, b = (1/6, 3/10, 8/15),
 * b appended as the last stage row) s = 4.  c needs 4 doubles, G 12. */
int mri_method_coupling(int mri_method, double* c, double* G, int* nstages);

/* Bytes of device workspace mri_step needs for a grid and n unknowns per cell. */
size_t mri_step_workspace_size(const mri_grid* grid, int n);

/* One slow step of the explicit MRI method `mri_method` (MRI_KW3) over the
 * grid: three f^S evaluations and three fast stages (Sec. 3.2, "MRI3").
 * workspace: device buffer of at least mri_step_workspace_size bytes, owned by
 * the caller and overwritten.  The other arguments are those of
 * mri_stage_fast; opts->ramp applies to the first fast stage only, and
 * opts->time_budget_s must be 0 (MRI_EINVAL otherwise). */
int mri_step(double* y, const double* p, const mri_grid* grid, double t, double H, double h,
             int mri_method, const mri_mech* mech, const mri_fast_opts* opts, void* workspace,
             size_t workspace_bytes, int32_t* cell_status, int32_t* cell_stats, int32_t* n_failed,
             void* stream);

/* ---- IMEX: implicit slow diffusion ---------------------------------------
 * The paper's IMEX-MRI runs (Sec. 3.2, problem 2 of Sec. 3.1) split the slow
 * partition into explicit advection f^E and implicit diffusion f^I and solve the
 * implicit stages' linear systems with Krylov solvers.  The third- and fourth-order
 * IMEX-MRI-GARK coupling tables the paper uses are not printed in it, so this
 * library provides the implicit solve and a first-order solve-decoupled IMEX-MRI
 * step built from it (its own, first order):
 *
 * mri_diffusion_solve: (I - a L) x = b for every component of [ncell][n], L = D lap_h
 * the periodic 7-point (2nd-order) Laplacian of the grid (axes with one cell
 * skipped; grid->u and grid->order are not used), by Jacobi-preconditioned
 * conjugate gradients for all components at once (each with its own scalars),
 * until |r|_2 <= tol |b|_2 per component (a component with b = 0: tol times its
 * initial residual); n <= 1024.  x holds the initial guess on entry and the
 * solution on return.  workspace: mri_diffusion_workspace_size bytes (device).
 *   check_every > 0: the host reads the solve's device state every check_every
 *     iterations (synchronising `stream`) and stops once every component has
 *     converged; *iterations (host, nullable) receives the iterations taken.
 *     Returns MRI_ECONV when max_iter iterations did not converge.
 *   check_every = 0: all max_iter iterations are enqueued without synchronisation
 *     (their launches do nothing once the solve has converged), so the call can be
 *     captured in a CUDA graph; convergence is reported only through cg_info.
 * cg_info (device, nullable, 2 ints): [0] 1 if every component converged, else 0;
 * [1] iterations taken.  Returns MRI_OK, MRI_ECONV, MRI_EINVAL, MRI_ENOMEM or
 * MRI_ECUDA. */
size_t mri_diffusion_workspace_size(const mri_grid* grid, int n);
int mri_diffusion_solve(double* x, const double* b, int n, const mri_grid* grid, double a, double tol,
                        int max_iter, int check_every, void* workspace, size_t workspace_bytes, int* iterations,
                        int32_t* cg_info, void* stream);

/* One first-order IMEX-MRI step over [t, t + H]: with f^E the grid's advection
 * (its order) and f^I = D lap_h y (7-point), the fast stage integrates
 *   v' = f^F(v) + f^E(y_n) + f^I(y_n)   on [t, t + H] from y_n
 * (mri_stage_fast with K = 1 and step h), then the solve-decoupled implicit stage
 *   (I - H L) y_{n+1} = v - H L y_n
 * (mri_diffusion_solve from x = v, with cg_tol, cg_max_iter, cg_check_every).  With
 * f^F = 0 and u = 0 it is backward Euler for the diffusion.  workspace:
 * mri_step_imex1_workspace_size bytes.  Status, stats and n_failed as mri_step;
 * cg_iterations and cg_info as mri_diffusion_solve.  With cg_check_every = 0 the
 * step does not synchronise and can be captured in a CUDA graph. */
size_t mri_step_imex1_workspace_size(const mri_grid* grid, int n);
int mri_step_imex1(double* y, const double* p, const mri_grid* grid, double t, double H, double h,
                   const mri_mech* mech, const mri_fast_opts* opts, double cg_tol, int cg_max_iter,
                   int cg_check_every, void* workspace, size_t workspace_bytes, int32_t* cell_status,
                   int32_t* cell_stats, int32_t* n_failed, int* cg_iterations, int32_t* cg_info, void* stream);

/* One second-order IMEX multirate step over [t, t + H], Strang-split (its own
 * scheme; the paper's IMEX-MRI-GARK tables are not printed): a Crank-Nicolson half
 * step of the diffusion, (I - (H/4) L) y* = (I + (H/4) L) y_n with L = D lap_h
 * (7-point), then mri_step over H with the chemistry fast and the advection (the
 * grid with D = 0) as the explicit slow partition, then a second Crank-Nicolson
 * half step; each half step by mri_diffusion_solve from x = y (cg_tol,
 * cg_max_iter, cg_check_every).  mri_method: MRI_KW3.  workspace:
 * mri_step_imex2_workspace_size bytes.  Status, stats and n_failed as mri_step;
 * cg_iterations (host, nullable) the CG iterations of both half steps (-1 with
 * cg_check_every = 0); cg_info (device, nullable, 2 ints) covers both half steps:
 * [0] 1 only if both converged, [1] their iterations summed.  With host checks
 * (cg_check_every > 0) a first half step that misses its tolerance ends the call
 * with MRI_ECONV (cg_info then describes that half step alone).  With
 * cg_check_every = 0 the step does not synchronise. */
size_t mri_step_imex2_workspace_size(const mri_grid* grid, int n);
int mri_step_imex2(double* y, const double* p, const mri_grid* grid, double t, double H, double h,
                   int mri_method, const mri_mech* mech, const mri_fast_opts* opts, double cg_tol,
                   int cg_max_iter, int cg_check_every, void* workspace, size_t workspace_bytes,
                   int32_t* cell_status, int32_t* cell_stats, int32_t* n_failed, int* cg_iterations,
                   int32_t* cg_info, void* stream);

/* Allocation-free variant of mri_step.  The paper has no counterpart: this is a
 * service for callers that must not allocate device memory while they run --
 * for example a host application that hands all of the GPU's memory to its own
 * pool manager at start-up, or code on a latency-critical path with a rule
 * against any call into the CUDA allocator.  Such a caller cannot provide
 * mri_step's workspace, so this entry point uses a fixed scratch array built into
 * the library instead; it never calls cudaMalloc or cudaFree.
 * Limits and behaviour:
 *   - the scratch is 16 MiB per device, held from library load until process
 *     exit; grids whose mri_step_workspace_size exceeds 16 MiB
 *     (4 * ncell * n * 8 bytes > 16 MiB, i.e. ncell * n > 524288) are rejected
 *     with MRI_ENOMEM before anything is launched;
 *   - the first call on a device looks up the scratch address for that device
 *     (cudaGetSymbolAddress), so make that first call before any stream capture;
 *   - every call on a device shares the one array and it keeps the previous
 *     call's contents; nothing in it needs to start at zero because each step
 *     writes every scratch value before reading it.  Calls whose work overlaps on
 *     the GPU (other streams, other threads) race on the array: order them on one
 *     stream or synchronise between them.
 * Arguments, results and return codes are those of mri_step. */
int mri_step_noalloc(double* y, const double* p, const mri_grid* grid, double t, double H, double h,
                     int mri_method, const mri_mech* mech, const mri_fast_opts* opts, int32_t* cell_status,
                     int32_t* cell_stats, int32_t* n_failed, void* stream);

/* ---- the separate kernels of the fast path, for per-kernel checks ------ */
/* f^F(y) of every cell (no forcing): f [ncell][n]. */
int mri_fast_rhs(const double* y, const double* p, int ncell, const mri_mech* mech, double* f,
                 void* stream);
/* Analytic Jacobian d f^F / d y of every cell: J [ncell][n][n], row-major. */
int mri_fast_jac(const double* y, const double* p, int ncell, const mri_mech* mech, double* J,
                 void* stream);
/* Batched dense solve A x = b with LU and partial pivoting (largest |a|, ties
 * to the lowest row): A [nbatch][n][n] row-major is overwritten by its LU
 * factors, b [nbatch][n] by x; info [nbatch] (may be NULL) gets 0 or k+1 for a
 * zero pivot in column k.  1 <= n <= 128. */
int mri_lu_solve_batched(double* A, double* b, int n, int nbatch, int32_t* info, void* stream);
/* Batched dense solve A x = b through the Gauss-Jordan inverse of MRI_LU_INVERSE
 * (FP64): A [nbatch][n][n] row-major is overwritten by A^-1, b [nbatch][n] by
 * x = A^-1 b computed as the stage kernel does (W (P b), W = (P A)^-1); info as for
 * mri_lu_solve_batched.  1 <= n <= 128. */
int mri_inverse_solve_batched(double* A, double* b, int n, int nbatch, int32_t* info, void* stream);

const char* mri_status_str(int code);

#ifdef __cplusplus
}
#endif
#endif
