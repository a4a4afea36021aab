/*
 * Reference oracle for the sigma-transformed mixed-stage Poisson solve of
 * "Subspace Acceleration for Efficient Nonlinear Water Wave Simulation"
 * (Sorensen, Guido, Engsig-Karup, Kressner).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, serial FP64 CPU restatement
 * of the method, written to check the CUDA library against.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load it;
 * the product path never calls it and shares no code with it.
 *
 * What it computes, and where the paper defines it:
 *   - grid and finite-difference weights (Fornberg's algorithm) ........ fd.c
 *   - the discrete operator A(eta_prev, eta_cur) of Eq. (16)-(18),
 *     assembled row by row as an explicit sparse matrix ................ operator.c
 *   - ILU(0) of A at still water and its triangular solves (Sec. 3) .... krylov.c
 *   - left-preconditioned restarted GMRES with CGS2 (Sec. 3) ........... krylov.c
 *   - EWMA sketch and least-squares guess (Algorithms 2 and 4) ......... subspace.c
 *   - randomized range finder over the K newest solutions (Algorithm 3)  subspace.c
 *   - optional orthonormal basis V = Q of either sketch ................ subspace.c
 *   - counter-based Gaussian draws for the sketch vectors .............. subspace.c
 *   - vertical walls with ghost columns and relaxation zones (Sec. 5.2)  operator.c, physics.c
 *   - LSERK45 stage driver, Eq. (14)-(17) and Algorithm 1 .............. physics.c
 *
 * Parity status of each function is listed in oracle/README.md.
 */
#ifndef SAWAVE_ORACLE_H
#define SAWAVE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_W 7        /* stencil width: sixth-order, 7-point (Sec. 5.2) */
#define OR_HALF 3

enum { OR_OK = 0, OR_BAD_ARG = -1, OR_NOT_CONVERGED = -3, OR_SINGULAR = -4, OR_NAN = -5 };
enum { OR_GUESS_COLD = 0, OR_GUESS_PREV = 1, OR_GUESS_EWMA = 2, OR_GUESS_RRF = 3 };

typedef struct {
    int nx, ny, nz;   /* columns in x and y (ny = 1 in 2D), sigma levels 0..nz-1 (ghost level -1 extra) */
    double lx, ly;    /* periodic lengths in x and y; with walls, lx is the wall-to-wall length */
    int walls;        /* 0: periodic in x.  1 (2-D only): vertical walls at x = 0 and x = lx, with
                         columns 0 and nx-1 the ghost columns outside them (Sec. 3, Sec. 5.2):
                         physical columns 1..nx-2 sit at x = (ix-1) lx/(nx-3) */
} or_grid;

typedef struct {
    int restart;       /* GMRES restart length m */
    int max_restarts;  /* cycles allowed after the first */
    double tol;        /* relative tolerance on the preconditioned residual */
    int guess;         /* OR_GUESS_* */
    int k;             /* sketch width of the EWMA subspace */
    double decay;      /* forgetting factor r applied once per solve */
    int n_init_solves; /* solves that use the previous-solution guess before EWMA starts */
    uint64_t seed;     /* seed of the Gaussian sketch vectors */
    int history;       /* K: past solutions kept for the randomized range finder (Algorithm 3) */
    int orthonormalize;/* 1: V = Q, an orthonormal basis of the sketch's span (the optional QR step of
                          Algorithms 3 and 4); 0: V = Y */
} or_params;

typedef struct {
    int iterations;     /* Arnoldi steps, all cycles */
    int restarts;       /* cycles started after the first */
    int converged;
    double res0;        /* ||M^-1(b - A x0)|| / ||M^-1 b|| */
    double res_final;   /* same, at the returned x */
    double true_res;    /* ||b - A x|| / ||b|| */
    double guess_res;   /* ||b - A x0|| / ||b|| */
} or_stats;

/* ---- finite differences (fd.c) ---- */
/* Fornberg (1988) weights c[d*n + i] for derivative order d = 0..mmax at z over nodes x[0..n-1]. */
void or_fornberg(double z, const double *x, int n, int mmax, double *c);
/* First sigma level of the 7-node window used at level j (j = -1..nz-1). */
int or_sigma_window(int nz, int j);
/* x coordinate of column ix (periodic: ix lx/nx; walls: (ix-1) lx/(nx-3)). */
typedef struct or_problem or_problem;
double or_xcoord(const or_problem *P, int ix);

/* ---- operator (operator.c) ---- */
typedef struct {
    int n;
    int *rowptr, *col;
    double *val;
} or_csr;

/* Node index of (ix, iy, j), j = -1 (ghost) .. nz-1 (surface); x fastest, ghost plane first. */
long or_index(const or_grid *g, int ix, int iy, int j);

or_problem *or_create(const or_grid *g, const or_params *p, const double *h, int *status);
void or_destroy(or_problem *P);
int or_size(const or_problem *P);
int or_is_box_pattern(const or_problem *P);

/* Assemble A(eta_prev, eta_cur) (Eq. 16-18) into an internal CSR; returns nnz. */
int or_assemble(or_problem *P, const double *eta_prev, const double *eta_cur);
/* Export the last assembled matrix (arrays sized n+1, nnz, nnz). */
void or_export_matrix(const or_problem *P, int *rowptr, int *col, double *val);
/* y = A x with the last assembled matrix. */
void or_matvec(const or_problem *P, const double *x, double *y);

/* ---- preconditioner and GMRES (krylov.c) ---- */
/* ILU(0) of the still-water matrix; order[new] = old (NULL = natural). */
int or_build_ilu(or_problem *P, const int *order);
int or_ilu_nnz(const or_problem *P);
void or_export_ilu(const or_problem *P, int *rowptr, int *col, double *val);
void or_ilu_apply(const or_problem *P, const double *v, double *out);
/* Left-preconditioned GMRES(m) on the last assembled matrix, from x (in/out). */
int or_gmres(or_problem *P, const double *b, double *x, or_stats *st);
/* Same, recording the preconditioned residual estimate after every Arnoldi step. */
int or_gmres_trace(or_problem *P, const double *b, double *x, or_stats *st, double *trace, int trace_len);

/* ---- subspace acceleration (subspace.c) ---- */
uint64_t or_splitmix64(uint64_t seed, uint64_t i);
void or_draw_omega(uint64_t seed, long solve_index, int k, double *omega);
/* Least-squares z = argmin ||W z - b|| by Householder QR; returns the numerical rank. */
int or_lstsq_qr(int m, int k, const double *W, const double *b, double *z);
/* Guess of Algorithm 2 with V = Y: x0 = Y z*, z* = argmin ||A Y z - b||. */
int or_ewma_guess(or_problem *P, const double *b, double *x0);
/* Y <- decay * Y + x omega_s^T (Algorithm 4), s = index of the solve that produced x. */
void or_ewma_update(or_problem *P, const double *x, long solve_index);
void or_get_sketch(const or_problem *P, double *Y);
void or_set_sketch(or_problem *P, const double *Y);
/* Randomized range finder (Algorithm 3) with V = Y: Y = X Omega for the K_e = min(solves,
 * K) newest solutions X (column r = the r-th newest) and Omega = the first K_e rows of the
 * K x k Gaussian matrix of this solve (entry (r, c) = draw r k + c of or_draw_omega with
 * K k values); k_e = min(k, K_e) columns.  Writes Y (m x k_e, column-major), returns k_e. */
int or_rrf_sketch(const or_problem *P, double *Y);
/* Guess of Algorithm 2 with V = Y of the range finder; returns the numerical rank. */
int or_rrf_guess(or_problem *P, const double *b, double *x0);
/* Orthonormal basis Q (m x r, column-major) of the span of Y (m x k): the Q of
 * Y = Q R by classical Gram-Schmidt applied twice per column, dropping columns
 * whose remainder is below 1e-12 of the largest column norm.  Returns r. */
int or_orth_basis(int m, int k, const double *Y, double *Q);
/* Full solve of Algorithm 2: assemble A(eta_prev, eta_cur), guess, GMRES, history update. */
int or_solve(or_problem *P, const double *eta_prev, const double *eta_cur, const double *b,
             double *x_out, or_stats *st);
long or_solve_count(const or_problem *P);

/* ---- time integration (physics.c) ---- */
typedef struct {
    double g, rho;    /* gravity and density; inviscid */
    double dt;
} or_physics;

/* LSERK45 coefficients alpha_i, beta_i, c_i (i = 1..5, stored 0..4). */
void or_lserk45(double *alpha, double *beta, double *c);
/* f_eta of Eq. (14b) at the surface nodes; out has one value per column. */
void or_f_eta(const or_problem *P, const double *u, const double *v, const double *w,
              const double *eta, double *out);
/* Right-hand side b of Eq. (16)-(17) for stage i (1..5). */
void or_rhs(const or_problem *P, const or_physics *ph, int stage,
            const double *u, const double *v, const double *w,
            const double *Ku, const double *Kv, const double *Kw,
            const double *eta_prev, const double *eta_cur, const double *deta_dt, double *b);
/* One stage i (1..5) of Algorithm 1 in place; p receives the stage pressure. */
int or_stage(or_problem *P, const or_physics *ph, int stage,
             double *u, double *v, double *w, double *eta,
             double *Ku, double *Kv, double *Kw, double *Keta, double *p, or_stats *st);

/* ---- wave generation and absorption zones (physics.c, Sec. 5.2) ---- */
typedef struct {
    double gen_x0, gen_x1;   /* generation zone [gen_x0, gen_x1] (empty when gen_x1 <= gen_x0) */
    double abs_x0, abs_x1;   /* absorption zone [abs_x0, abs_x1] (empty when abs_x1 <= abs_x0) */
    double height, period;   /* incident linear wave: height H and period T */
    double depth;            /* still-water depth the incident wave is computed for */
    double ramp_time;        /* the incident amplitude ramps up smoothly over [0, ramp_time] */
    double g;
} or_relaxation;

/* Relaxation weight Gamma(xi) = 1 - (exp(xi^3.5) - 1)/(e - 1): 1 at the inner end of a zone
 * (xi = 0), 0 at its outer end (xi = 1). */
double or_relax_weight(double xi);
/* Wavenumber k of the linear dispersion relation omega^2 = g k tanh(k depth) (Newton). */
double or_wavenumber(double omega, double depth, double g);
/* phi <- Gamma phi + (1 - Gamma) phi_target for eta, then u and w (2-D), at time t. */
void or_relax(const or_problem *P, const or_relaxation *rl, double t, double *u, double *w, double *eta);

#ifdef __cplusplus
}
#endif
#endif
