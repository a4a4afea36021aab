/*
 * sawave: subspace-accelerated sigma-transformed Poisson solve on one GB300.
 *
 * C ABI of the library libsawave.so.  The method is that of
 * "Subspace Acceleration for Efficient Nonlinear Water Wave Simulation"
 * (Sorensen, Guido, Engsig-Karup, Kressner): every stage of a low-storage
 * Runge-Kutta step of the free-surface Navier-Stokes model solves
 *     A(tau) x(tau) = b(tau)                                   (Eq. 1, Eq. 19)
 * with the mixed-stage sigma-transformed operator of Eq. (16)-(18), by GMRES
 * left-preconditioned with one fixed ILU factorisation (Sec. 3), started from
 * the exponentially weighted subspace guess of Algorithms 2 and 4.
 *
 * Conventions for every entry point:
 *   - the return value is a status code (SW_OK or a negative SW_ERR_*);
 *   - pointers named d_* are device pointers (cudaMalloc or torch memory on the
 *     current device), pointers named h_* are host pointers; the caller owns
 *     every buffer it passes and the library never frees or keeps them;
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Work is enqueued on that stream; calls that return
 *     statistics synchronise it;
 *   - the library owns everything it allocates (ILU factors, Krylov basis,
 *     subspace sketch, scratch) and releases it in sw_destroy_problem;
 *   - there is no CPU fallback: without a usable CUDA device every call that
 *     needs one returns SW_ERR_CUDA.
 *
 * Grid and node numbering.  The sigma grid has nx * ny columns (ny = 1 in 2-D),
 * periodic in x (and y), and nz sigma levels sigma_j = j/(nz-1), j = 0..nz-1,
 * plus one ghost level j = -1 below the bed (Sec. 5.1).  A field on the grid
 * is an array of m = nx*ny*(nz+1) doubles, node (ix, iy, j) at index
 * ((j+1)*ny + iy)*nx + ix.  Surface fields (eta, h) hold nx*ny doubles,
 * index iy*nx + ix.  Requirements: nz >= 7; nx and ny (when ny > 1) are
 * multiples of 4 and at least 8.
 *
 * Walls (sw_grid.walls = 1; 2-D only, nx >= 16 and a multiple of 4): vertical walls at
 * x = 0 and x = lx with impermeable (Neumann) conditions imposed through
 * ghost nodes (Sec. 3; the flume of Sec. 5.2).  Columns 0 and nx-1 are ghost
 * columns one spacing outside the walls; the physical columns 1..nx-2 sit at
 * x = (ix-1) lx/(nx-3).  The row of ghost node (0, j), j = -1..nz-2, is the
 * wall condition n . grad^(i-1) p = n . G at the wall node (1, j) (likewise
 * nx-1 for the wall node nx-2); surface ghost nodes are Dirichlet rows.  x
 * stencils next to a wall are shifted inside the grid (off-centred 7-point
 * formulas); x derivatives of surface data and velocities use the physical
 * columns only.  The stage driver keeps the ghost columns' flow at rest.
 */
#ifndef SAWAVE_H
#define SAWAVE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SW_OK 0
#define SW_ERR_BAD_ARG (-1)          /* invalid argument or unsupported size */
#define SW_ERR_CUDA (-2)             /* a CUDA call failed (message via sw_last_error) */
#define SW_ERR_NOT_CONVERGED (-3)    /* iteration cap reached; x holds the last iterate */
#define SW_ERR_SINGULAR_PRECOND (-4) /* zero pivot in the ILU factorisation */
#define SW_ERR_NAN (-5)              /* non-finite residual during a solve */
#define SW_ERR_TIMEOUT (-6)          /* a wait inside a solve kernel ran past its bound (2 s of device time);
                                        the solve was abandoned and x is incomplete */

#define SW_GUESS_COLD 0      /* x0 = 0 */
#define SW_GUESS_PREVIOUS 1  /* x0 = previous solution (the paper's baseline, Sec. 5.1) */
#define SW_GUESS_EWMA 2      /* Algorithm 4 with V = Y (Algorithm 2) */
#define SW_GUESS_RRF 3       /* Algorithm 3 (randomized range finder) with V = Y = X Omega over the
                                `history` newest solutions, a fresh Gaussian Omega per solve */
#define SW_RRF_MAX_HISTORY 16

#define SW_PRECISION_FP64 0  /* every step in FP64 */
#define SW_PRECISION_MIXED 1 /* FP32 inner GMRES cycles, FP64 outer residual */

#define SW_EXEC_AUTO 0        /* resident where it applies (see SW_EXEC_RESIDENT) and the problem fits in
                                 shared memory; else persistent below SW_EXEC_STREAMED_MIN unknowns,
                                 streamed above */
#define SW_EXEC_PERSISTENT 1  /* one cooperative kernel per solve, one block per SM: no host round
                                 trip inside a solve, lowest latency for small problems */
#define SW_EXEC_STREAMED 2    /* one high-occupancy kernel per phase, small control kernels in
                                 between, one stream synchronisation per restart cycle: keeps HBM
                                 busy on large problems (sw_solve_poisson then returns once the
                                 solve has finished) */
#define SW_EXEC_RESIDENT 3    /* small periodic 2-D FP64 problems: one block per slab of columns with the
                                 slab's vectors and constants in shared memory; neighbouring blocks
                                 exchange boundary columns through flags (no grid barrier) and inner
                                 products are all-reduced with one atomic per block; same arithmetic
                                 up to rounding, the norm of the twice-orthogonalised Krylov vector from
                                 ||w||^2 - ||h'||^2 */
#define SW_EXEC_STREAMED_MIN 262144

typedef struct sw_problem sw_problem;

typedef struct {
    int nx, ny, nz;  /* columns in x and y, sigma levels (ghost level not counted) */
    double lx, ly;   /* periodic domain lengths (ly ignored when ny == 1); with walls, lx is the
                        wall-to-wall length */
    int walls;       /* 0: periodic in x; 1: walls with ghost columns (2-D, see above) */
} sw_grid;

typedef struct {
    int restart;        /* GMRES restart length m (Sec. 3; 20 for the workloads here) */
    int max_restarts;   /* restart cycles allowed after the first one */
    double tol;         /* stop when ||M^-1(b - A x)|| <= tol ||M^-1 b|| */
    int guess;          /* SW_GUESS_* */
    int k;              /* EWMA sketch width k (Algorithm 4), 1..16 */
    double decay;       /* forgetting rate r of Algorithm 4, applied once per solve, in (0, 1] */
    int n_init_solves;  /* solves run with the previous-solution guess before EWMA starts (N_init, Sec. 5.1) */
    int precision;      /* SW_PRECISION_* */
    uint64_t seed;      /* seed of the Gaussian sketch vectors omega */
    int executor;       /* SW_EXEC_*: how a solve is run on the GPU (same arithmetic) */
    int history;        /* K of the range finder: solutions kept, k..SW_RRF_MAX_HISTORY (SW_GUESS_RRF) */
    int orthonormalize; /* 1: the guess uses V = Q, an orthonormal basis of the sketch's span (the optional
                           QR step of Algorithms 3 and 4), by CholeskyQR2 with columns below the rank guard
                           dropped; 0: V = Y.  Same x0 in exact arithmetic; costs three passes over the
                           sketch and a k x m buffer */
} sw_params;

typedef struct {
    int iterations;        /* Arnoldi steps of the last solve (all cycles) */
    int restarts;          /* cycles after the first in the last solve */
    int converged;         /* 1 when the last solve met the tolerance */
    int status;            /* status of the last solve */
    double res0;           /* ||M^-1(b - A x0)|| / ||M^-1 b|| of the last solve */
    double res_final;      /* same at the returned solution */
    double true_res;       /* ||b - A x|| / ||b|| at the returned solution */
    double guess_res;      /* ||b - A x0|| / ||b|| */
    long long n_solves;    /* solves since creation */
    long long total_iterations;
    long long launches;    /* CUDA kernels this library launched since creation */
    double model_flops;    /* algorithmic FP operations of all solves so far (cost model of the
                              operator, preconditioner, Gram-Schmidt and guess; not counters) */
    double model_bytes;    /* algorithmic bytes moved by all solves so far (same model) */
    int executor;          /* SW_EXEC_* the solves run on (resolved from SW_EXEC_AUTO) */
} sw_stats;

typedef struct {
    double g;    /* gravity */
    double rho;  /* density */
    double dt;   /* time step Delta tau */
} sw_physics;

/* Wave generation and absorption zones of a flume (Sec. 5.2).  After every
 * stage, eta, u and w of the physical columns inside a zone are blended
 * towards a target, phi <- Gamma phi + (1 - Gamma) phi_target, with
 * Gamma(xi) = 1 - (exp(xi^3.5) - 1)/(e - 1) (Engsig-Karup, Bingham & Lindberg
 * 2009), xi = 0 at the inner end of the zone and 1 at its outer end.  The
 * generation target is the incident linear wave of height H and period T on
 * the still-water depth `depth`, amplitude ramped in time by
 * (1 - cos(pi t / ramp_time))/2 up to t = ramp_time; the absorption target is
 * still water.  The zone x ranges are in the coordinates of the grid. */
typedef struct {
    double gen_x0, gen_x1;   /* generation zone (empty when gen_x1 <= gen_x0); xi = 1 at gen_x0 */
    double abs_x0, abs_x1;   /* absorption zone (empty when abs_x1 <= abs_x0); xi = 1 at abs_x1 */
    double height, period;   /* incident wave height H and period T */
    double depth;            /* still-water depth of the incident wave */
    double ramp_time;        /* 0 for no ramp */
    double g;                /* gravity of the dispersion relation */
} sw_relaxation;

/* Build a problem on the current CUDA device.  h_depth: host array of nx*ny
 * still-water depths h > 0.  Computes the ILU(0) factors of the operator at
 * still water (eta = 0) on the host in FP64 (Sec. 3 and Sec. 5), in the
 * four-colour column ordering, and uploads them.  On success *out owns all
 * device memory of the problem.  Errors: SW_ERR_BAD_ARG (sizes, parameters),
 * SW_ERR_SINGULAR_PRECOND, SW_ERR_CUDA. */
int sw_create_problem(const sw_grid *grid, const sw_params *params, const double *h_depth, sw_problem **out);

/* Release everything the problem owns.  NULL is accepted. */
int sw_destroy_problem(sw_problem *p);

/* Number of unknowns m = nx*ny*(nz+1). */
int sw_problem_size(const sw_problem *p, long long *m);

/* Solve A(eta_prev, eta_cur) x = b (Eq. 16-18; Algorithm 2 with the guess
 * selected in the parameters; for EWMA the sketch is updated with the new
 * solution, Algorithm 4).  d_eta_prev, d_eta_cur: nx*ny surfaces at stages
 * i-1 and i; d_b, d_x: m doubles.  Enqueued on `stream`; returns SW_OK once
 * enqueued.  The outcome (status, iterations, residuals) is read with
 * sw_get_stats. */
int sw_solve_poisson(sw_problem *p, const double *d_eta_prev, const double *d_eta_cur,
                     const double *d_b, double *d_x, void *stream);

/* The same solve with host buffers: copies eta_prev, eta_cur and b to the
 * device, solves, copies x back and synchronises `stream`.  Returns the
 * solve status. */
int sw_solve_poisson_host(sw_problem *p, const double *h_eta_prev, const double *h_eta_cur,
                          const double *h_b, double *h_x, void *stream);

/* Statistics of the last solve (synchronises the stream of that solve). */
int sw_get_stats(sw_problem *p, sw_stats *out);

/* y = A(eta_prev, eta_cur) x, matrix-free (Eq. 16-18).  Device pointers. */
int sw_apply_operator(sw_problem *p, const double *d_eta_prev, const double *d_eta_cur,
                      const double *d_x, double *d_y, void *stream);

/* out = U^-1 L^-1 v with the fixed ILU(0) factors (Sec. 3).  Device pointers,
 * out must not alias v. */
int sw_apply_preconditioner(sw_problem *p, const double *d_v, double *d_out, void *stream);

/* EWMA guess alone (Algorithm 2 with V = Y): x0 = Y z*, z* = argmin ||A Y z - b||,
 * with A = A(eta_prev, eta_cur) and the problem's current sketch Y. */
int sw_subspace_guess(sw_problem *p, const double *d_eta_prev, const double *d_eta_cur,
                      const double *d_b, double *d_x0, void *stream);

/* Sketch access: Y is m x k, column c at offset c*m.  Device pointers. */
int sw_get_sketch(sw_problem *p, double *d_Y, void *stream);
int sw_set_sketch(sw_problem *p, const double *d_Y, long long n_solves, void *stream);

/* The Gaussian sketch vector omega of a given solve (host): SplitMix64
 * outputs 2(s k + c) + 1 and 2(s k + c) + 2 through Box-Muller, c = 0..k-1.
 * The range finder's K x k matrix Omega of solve s is the draw with K k
 * values, entry (r, c) at r k + c, row r weighting the r-th newest solution;
 * with fewer than K solutions stored, the first K_e rows and min(k, K_e)
 * columns are used. */
int sw_draw_omega(uint64_t seed, long long solve_index, int k, double *h_omega);

/* ---- stage driver: Algorithm 1 with LSERK45 (Sec. 3 and Sec. 5) ---- */

/* Physical constants and time step for the stage driver. */
int sw_set_physics(sw_problem *p, const sw_physics *phys);
/* Load the state: u, w (and v in 3-D, else NULL) on the m nodes, eta on the
 * surface; the Runge-Kutta registers are zeroed, the stage counter and the
 * time (t = 0) reset.  Device pointers, copied. */
int sw_set_state(sw_problem *p, const double *d_u, const double *d_v, const double *d_w,
                 const double *d_eta, void *stream);
/* Copy the state out (any of the pointers may be NULL). */
int sw_get_state(sw_problem *p, double *d_u, double *d_v, double *d_w, double *d_eta,
                 double *d_p, void *stream);
/* One stage i (cycling 1..5) of Algorithm 1: K_eta and eta^(i), the right-hand
 * side of Eq. (16)-(17), the Poisson solve, K_u and u^(i); then, when
 * relaxation zones are set, the blend of eta, u, w at the stage's end time
 * t = (n + c_(i+1)) dt (n completed steps, c_6 = 1). */
int sw_advance_stage(sw_problem *p, void *stream);
/* Generation/absorption zones applied after every stage (2-D); NULL removes
 * them.  Copied.  SW_ERR_BAD_ARG for a 3-D problem or a non-positive period,
 * height or depth when a generation zone is set. */
int sw_set_relaxation(sw_problem *p, const sw_relaxation *relax);
/* Set the number of completed Runge-Kutta steps n (the next stage is stage 1
 * of step n + 1, at time n dt), e.g. to continue a run from a saved state.
 * Call between steps.  SW_ERR_BAD_ARG for n < 0. */
int sw_set_step(sw_problem *p, long long n_steps);
/* The system A(eta_prev, eta_cur) p = b of the last stage (copies; any pointer may be NULL). */
int sw_get_last_system(sw_problem *p, double *d_eta_prev, double *d_eta_cur, double *d_b, void *stream);

/* ---- batch form: many independent problems in one launch per step ---- */

typedef struct sw_batch sw_batch;

/* Group existing two-dimensional problems (all with the same precision; walled
 * and periodic grids may be mixed) so that their solves and stages run
 * together: each Poisson solve on one thread block, problems
 * handed out largest first; each driver step one launch over (problem, node).
 * The batch keeps pointers to the problems, which must outlive it.  The
 * many-query setting of Sec. 1 (many wave simulations at once) is the use.
 * SW_ERR_BAD_ARG for a three-dimensional member or mixed precisions. */
int sw_create_batch(sw_problem *const *problems, int n, sw_batch **out);
int sw_destroy_batch(sw_batch *b);
/* Solve every member's system A_i x_i = b_i (Algorithm 2 per member, as
 * sw_solve_poisson).  Host arrays of n device pointers, in the order the
 * problems were given to sw_create_batch.  Per-member results via sw_get_stats. */
int sw_batch_solve(sw_batch *b, const double *const *d_eta_prev, const double *const *d_eta_cur,
                   const double *const *d_b, double *const *d_x, void *stream);
/* Thread blocks per member for the batch's solves, the same for every member:
 * 1 gives every member one thread block, so that up to one member per SM run
 * at once; 2, 4, 8 or 16 give every member a thread-block cluster of that many
 * blocks (one per SM, cluster barriers and partial sums through distributed
 * shared memory), which shortens large members at the cost of fewer members
 * at once.  Replaces a split (sw_batch_set_split).  SW_ERR_BAD_ARG for other
 * values or when the device cannot place such a cluster with this batch's
 * shared memory.
 *
 * The default set by sw_create_batch is the launch shape with the shortest
 * modelled makespan (a member's time taken as its unknowns over the SMs of
 * its team times a per-SM efficiency measured for each cluster size): one
 * block for every member, clusters of one size for every member, or a split
 * (sw_batch_set_split). */
int sw_batch_set_cluster(sw_batch *b, int blocks_per_member);
/* Split launch: the n_big largest members (by unknowns) on clusters of
 * blocks_per_member (2, 4, 8 or 16) blocks, the other n - n_big on one block
 * each, the two launches side by side (the single-block one on a stream of
 * the batch, joined back to the caller's stream by events).  Each big member
 * gets a cluster of its own where the device can place that many clusters
 * beside at least one single block; the single blocks take the remaining SMs.
 * SW_ERR_BAD_ARG unless 1 <= n_big < n and the device can place such a
 * cluster. */
int sw_batch_set_split(sw_batch *b, int n_big, int blocks_per_member);
/* The batch's launch shape: members on clusters, blocks per cluster member,
 * blocks of the cluster launch, blocks of the single-block launch. */
int sw_batch_get_launch(sw_batch *b, int *n_big, int *blocks_per_member, int *cluster_blocks, int *single_blocks);
/* Tile autotuner of the batch: sw_create_batch times the operator apply of
 * every member at once (one block per member, the inner precision) with tiles
 * of 8, 16, 32 and 64 columns (each cut to the largest width that divides the
 * member's nx) and keeps the fastest for the members' applies; the tile shape
 * changes no output value.  *tile_x = the width kept; us[0..n) = microseconds
 * per batched apply for each candidate (n <= 4 values written, 0 where not
 * timed). */
int sw_batch_autotuned_tile(sw_batch *b, int *tile_x, double *us, int n);
/* One Runge-Kutta stage of every member (each needs its state and physics set).
 * Relaxation zones set with sw_set_relaxation are not applied here. */
int sw_batch_advance_stage(sw_batch *b, void *stream);

/* Allocation-free operator apply: y = A(eta_prev, eta_cur) x as in
 * sw_apply_operator, but without a problem handle and without allocating
 * device memory.  The paper has no counterpart; this exists for callers that
 * cannot call cudaMalloc (a memory budget or pool that forbids new device
 * allocations, or a framework that hands over only its own buffers).
 * All pointers except `grid` are device pointers owned by the caller: d_h
 * (nx*ny depths), d_eta_prev and d_eta_cur (nx*ny), d_x and d_y (m each).
 * Scratch lives in one static device array sized for at most 65,536 columns
 * (nx*ny; about 12.6 MB held by every GPU that loads the library until exit);
 * larger grids return SW_ERR_BAD_ARG.  The first call on a device resolves
 * the array's address and should come before any stream capture.  A call
 * enqueues kernels only (the weights travel as kernel arguments, no copy from
 * host memory).  Calls share the array: two calls that overlap on the GPU
 * race.  Same grid rules as sw_create_problem; periodic grids only (walls:
 * SW_ERR_BAD_ARG). */
int sw_apply_operator_noalloc(const sw_grid *grid, const double *d_h, const double *d_eta_prev,
                              const double *d_eta_cur, const double *d_x, double *d_y, void *stream);

/* Per-launch timing of the solve kernel with CUDA events recorded on the
 * launching stream around each solve (off by default).  sw_get_solve_time
 * synchronises and returns the summed duration in milliseconds and the number
 * of timed solves since timing was switched on. */
int sw_enable_timing(sw_problem *p, int on);
int sw_get_solve_time(sw_problem *p, double *total_ms, long long *n_timed);

/* Profiling aid: cumulative device time in microseconds spent in each phase of
 * all solves so far, as seen by one thread between grid barriers (n <= 16
 * values): 0 geometry, 1 ||M^-1 b||, 2 sketch update and W = A Y, 3 Gram and
 * least squares, 4 residual apply, 5 residual preconditioner and norm,
 * 6 Arnoldi apply, 7 Arnoldi preconditioner, 8-10 the three Gram-Schmidt
 * passes, 11 Givens rotations, 12 solution update, 13 true residual. */
int sw_get_phase_times(sw_problem *p, double *us, int n);

/* Profiling aid for problems on the streamed executor, after at least one
 * solve: the hot kernels of an Arnoldi step timed alone on the problem's own
 * buffers with CUDA events on a private stream, `reps` launches each after
 * one untimed launch, a 256 MiB buffer written before every launch so that
 * inputs come from HBM (allocated and freed by the call).  us[i] (i < n <= 8)
 * receives the mean duration in microseconds of: 0 the operator apply of the
 * Arnoldi step (autotuned form), 1 the forward ILU gathers of every colour,
 * 2 the in-column block products of both sweeps, 3 the backward ILU gathers,
 * 4-6 the three Gram-Schmidt passes at Arnoldi index j = 10, 7 one whole ILU
 * application (on periodic grids the products read the packed triangular
 * inverse blocks).  The control state of the last solve is restored. */
int sw_profile_kernels(sw_problem *p, int reps, double *us, int n);
/* The operator form the streamed executor's autotuner picked: *column_form 1
 * for the column-marching kernel (tile tile_x x tile_y columns), 0 for the
 * staged tile kernel of tile_x x tile_y columns. */
int sw_autotuned_apply(sw_problem *p, int *column_form, int *tile_x, int *tile_y);
/* Override the autotuner's choice for the streamed executor's Arnoldi apply:
 * 1 the column-marching kernel (periodic grids with 10, 18 or 34 levels, nx a
 * multiple of 32 and ny of 8 in 3-D, nx a multiple of 256 in 2-D), 0 the
 * staged tile kernel.  Same result up to rounding.  SW_ERR_BAD_ARG when the
 * column form does not serve the grid or another executor runs the solves. */
int sw_set_apply_form(sw_problem *p, int column_form);

/* Testing aid for failure detection without a GPU fault: in the next solve of
 * a problem on the resident executor, block 0 stops raising its flag from its
 * `exchange`-th boundary exchange on (1 = the first), so the neighbouring
 * blocks' bounded waits run out, every block leaves the kernel and the solve's
 * status (sw_get_stats) is SW_ERR_TIMEOUT; later solves are unaffected.
 * SW_ERR_BAD_ARG for another executor or exchange < 1. */
int sw_test_stall_exchange(sw_problem *p, int exchange);

/* Last error message of the calling thread (static storage). */
const char *sw_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
