/*
 * CPU oracle of the MRI fast-partition solve: plain, slow, FP64.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code with the CUDA path: its own mechanism reader, thermodynamics, rates,
 * Jacobian, LU, SDIRK tableaux, MRI coupling table and stencils.
 *
 * What it computes, and where each piece comes from:
 *   - the two-rate problem y' = f^F(t,y) + f^S(t,y) (paper Eq. 1);
 *   - the infinitesimal (MIS / MRI-GARK) step: Y_1 = y_n; for i = 2..s solve the
 *     modified fast IVP v' = f^F(theta, v) + r_i(theta) on [T_{i-1}, T_i] from
 *     v = Y_{i-1}, Y_i = v(T_i); y_{n+1} = Y_s (Sec. 2.1, Eq. 3 and the stage
 *     algorithm above it).  The slow method is the third-order explicit scheme
 *     of Knoth and Wolke (Sec. 3.2, "MRI3") in MIS form: constant forcing
 *     r_i = (1/dc_i) sum_j (a_ij - a_{i-1,j}) f^S(Y_j);
 *   - the fast partition f^F = omega_k W_k / rho for the mass fractions (Sec. 3.2,
 *     partitioning of Eq. 6) plus the constant-pressure energy equation for T,
 *     with rho from the ideal-gas law (Eq. 5); production rates follow the
 *     standard Chemkin definitions (Arrhenius, third body, Lindemann-Troe
 *     falloff, equilibrium constants from NASA-7 Gibbs polynomials), which the
 *     paper names but does not print;
 *   - explicit fast integrators (Sec. 3.2, the MRI-P(k) methods): Heun's second-
 *     order, Kutta's third-order and the classical fourth-order Runge-Kutta method,
 *     fixed substeps, no Jacobian;
 *   - fast integrator: L-stable SDIRK2 / SDIRK3 (Alexander 1977) with full
 *     Newton (fresh analytic Jacobian and LU with partial pivoting every
 *     iteration), fixed substeps n_i = ceil(dc_i H / h), optionally a geometric
 *     start-up sequence in place of the first substep; or (adaptive) substep
 *     sizes from an embedded error estimate with a power-of-two controller;
 *   - slow partition: periodic central advection-diffusion, 2nd or 4th order,
 *     same u and D for every component (Sec. 3.1 for the 2nd-order form).
 *
 * Conventions: state per cell y = (Y_1..Y_Ns, T), cell-major [ncell][n],
 * n = Ns + 1; SI units; Jacobians row-major J[i*n + j] = d f_i / d y_j.
 * Every function returns 0 on success and a negative value on bad input.
 */
#ifndef MRI_ORACLE_H
#define MRI_ORACLE_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int method;          /* 2 = SDIRK2, 3 = SDIRK3; explicit (fixed substeps only): 12 = Heun,
                          13 = Kutta's third-order method, 14 = classical RK4 */
  double rtol;         /* Newton WRMS relative tolerance */
  double atol_Y;       /* absolute tolerance, mass fractions */
  double atol_T;       /* absolute tolerance, temperature [K] */
  int max_newton;      /* Newton iterations per stage before the cell fails */
  int ramp;            /* >0: first substep of the stage replaced by a geometric start-up
                          sequence of ramp+1 substeps (hh 2^-ramp, hh 2^-ramp, ..., hh/2) */
  int adaptive;        /* 1: substep sizes chosen by the embedded error estimate (ramp ignored) */
  double ctrl_rtol;    /* adaptive: local error tolerance, relative */
  double ctrl_atol_Y;  /* adaptive: absolute, mass fractions */
  double ctrl_atol_T;  /* adaptive: absolute, temperature [K] */
} orc_opts;

typedef struct {
  int nx, ny, nz;      /* periodic grid; cell index (k*ny + j)*nx + i */
  double dx;           /* spacing [m], same on every axis */
  double u[3];         /* advection velocity [m/s] */
  double D;            /* diffusivity [m^2/s] */
  int order;           /* 2 or 4 */
} orc_grid;

void* orc_mech_load(const void* blob, size_t nbytes);
void orc_mech_free(void* mech);
int orc_mech_info(const void* mech, int* n_species, int* n_reactions);

int orc_thermo(const void* mech, double T, double* cpR, double* hRT, double* sR, double* gRT);
/* forward / reverse rate coefficients and K_c at T for concentrations C (C enters
   only through [M] of falloff reactions) */
int orc_rate_coeffs(const void* mech, double T, const double* C, double* kf, double* kr, double* Kc);
/* rates of progress q[R] and molar production rates wdot[Ns] at (T, C) */
int orc_progress(const void* mech, double T, const double* C, double* q, double* wdot);
int orc_rhs(const void* mech, const double* y, double p, double* f);
int orc_jac(const void* mech, const double* y, double p, double* J);
int orc_jac_cs(const void* mech, const double* y, double p, double* J);

int orc_lu_solve(int n, double* A, int* piv, double* b);
/* Floating-point operations of the oracle's own formulas at state y, counted by
 * category: out[row * 6 + col], rows 0 one f^F evaluation, 1 one analytic Jacobian
 * (its rate evaluation included), 2 one LU factorisation of I - hg J, 3 one solve with
 * those factors; columns add/subtract, multiply, divide, exp, log (natural or decimal),
 * pow.  Returns 0, 1 if the matrix is singular, -1 on bad arguments. */
int orc_flop_counts(const void* mech, const double* y, double p, double hg, long long* out);
int orc_sdirk_tableau(int method, double* A, double* b, double* c, int* s);
/* embedded weights of the adaptive error estimate (one order lower than the method)
   and the estimate's order q (the controller scales steps by err^(-1/q)) */
int orc_sdirk_embedded(int method, double* bhat, int* q);
/* explicit Runge-Kutta tableau of method 12, 13 or 14 (A row-major s x s) */
int orc_erk_tableau(int method, double* A, double* b, double* c, int* s);
/* the explicit methods on the scalar test problems of orc_sdirk_scalar */
int orc_erk_scalar(int method, int problem, double lam, double t0, double t1, int nsteps, double y0,
                   double* y_out);
int orc_mri_tableau(double* A, double* c, int* s);
/* coupling coefficients of the MIS form: G[i*s + j] multiplies f^S(Y_j) in the
   constant forcing of stage i (i = 1..s-1, zero-based) */
int orc_mri_coupling(double* G, int* s);

int orc_stage_fast(const void* mech, double* y, const double* p, int ncell, const double* phi, int K,
                   double Hs, double h, const orc_opts* o, int32_t* status, int32_t* stats, int nthreads);
/* orc_stage_fast with, in adaptive mode, each cell's first step set to the uniform
 * substep times 2^step_exp[c] (step_exp clamped to [-20, 10]; NULL: all 0). */
int orc_stage_fast_exp(const void* mech, double* y, const double* p, int ncell, const double* phi, int K,
                       double Hs, double h, const orc_opts* o, const int8_t* step_exp, int32_t* status,
                       int32_t* stats, int nthreads);
int orc_slow_rhs(const double* y, double* f, int n, const orc_grid* g);
/* one MRI3 slow step; o->ramp applies to the first fast stage only */
int orc_mri_step(const void* mech, double* y, const double* p, const orc_grid* g, double H, double h,
                 const orc_opts* o, int32_t* status, int32_t* stats, int nthreads);
/* coupled single-rate SDIRK over f^F + f^S for all cells at once (dense Newton);
   for brute-force references on a few cells */
int orc_single_rate(const void* mech, double* y, const double* p, const orc_grid* g, double t_end,
                    int nsteps, const orc_opts* o);

/* scalar/test problems: problem 0 = y' = lam*y; 1 = Prothero-Robinson
   y' = lam*(y - cos t) - sin t */
int orc_sdirk_scalar(int method, int problem, double lam, double t0, double t1, int nsteps, double y0,
                     double* y_out);
/* KPR multirate problem, MIS/KW3 slow + SDIRK or explicit fast method (fast_method
   2, 3, 12, 13, 14) with m substeps per unit of slow step: returns max-norm error at t1 */
int orc_kpr_mri(int fast_method, double G, double e, double beta, double omega, double t1, int nsteps,
                int m_fast, double* err, double* y_out);

#ifdef __cplusplus
}
#endif
#endif
