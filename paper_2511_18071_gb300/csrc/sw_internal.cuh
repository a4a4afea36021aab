// Internal definitions of libsawave: the device-side problem descriptor, the
// ILU slot layout, and host-side bookkeeping.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/sawave.h"

namespace sw {

constexpr int W = 7;     // stencil width (sixth order, Sec. 5.2)
constexpr int HALF = 3;
constexpr int MAX_LEVELS = 64;      // nz + 1 <= 64 (two levels per lane in the ILU column sweeps)
constexpr int MAX_RESTART = 32;
constexpr int MAX_K = 16;

// Sparsity layouts of the preconditioner rows ("slots").  An x position t =
// 0..6 is the t-th column of the row's 7-column x window (t = dx + 3 when
// the window is centred; next to a wall the window is shifted and the row's
// own column sits at position o != 3).
//   CROSS2D: x positions other than the own column at the row's level (6),
//            sigma window of the own column (7)                                -> 13
//   BOX2D:   (x position, window level) (7 x 7); own column at position o      -> 49
//   CROSS3D: x (6) and y (6) neighbours at the own level, sigma window (7)     -> 19
//   BOX3D:   x box (7 x 7) and y box without its centre column (6 x 7)         -> 91
enum Layout { CROSS2D = 0, BOX2D = 1, CROSS3D = 2, BOX3D = 3 };

__host__ __device__ inline int layout_nslot(int L) {
    return L == CROSS2D ? 13 : L == BOX2D ? 49 : L == CROSS3D ? 19 : 91;
}
// Slot holding the sigma-window entry kk (same column) of a row with a centred x window.
__host__ __device__ inline int sigma_slot(int L, int kk) {
    return (L == CROSS2D ? 6 : L == CROSS3D ? 12 : 21) + kk;
}
// The same for a row whose own column is at x position o (2-D layouts).
__host__ __device__ inline int own_slot(int L, int kk, int o) {
    return L == BOX2D ? o * 7 + kk : sigma_slot(L, kk);
}

constexpr int MAX_GROUPS = 7;   // column groups of the ILU sweeps: 4 colours (+3 next to walls)

// Device view of one problem (plain pointers; passed to kernels by value).
struct Dev {
    int nx, ny, nz, P, ncol, three_d, layout, nslot;
    long long m;
    double dx, dy;
    // Walls (2-D): ghost columns 0 and nx-1 outside the walls, x windows
    // shifted inside the grid next to them (see include/sawave.h).
    int walls;
    // ILU column groups in sweep order; columns of one group are uncoupled.
    // Periodic: colour (ix + iy) mod 4.  Walls: colours ix mod 4 of columns
    // 3..nx-4, then {0, nx-1}, {1, nx-2}, {2, nx-3}.
    int ngroups;
    const int *goff;                       // walls: first column rank of each group (ngroups + 1);
                                           // periodic groups are the four equal colours
    const int *gcol;                       // walls: column of each column rank (ncol)
    const unsigned char *grp;              // walls: group of each column (ncol)
    const double *wx1, *wx2, *wy1, *wy2;   // 7 each
    const double *wxo1, *wxo2;             // walls: 7 x 7 each, weights at node o of a 7-node window
    const double *ws1, *ws2;               // P x 7, row j+1
    const int *win;                        // P, first level of the sigma window of level j
    const double *h, *hx, *hy, *hxx, *hyy; // ncol
    double *gp;                            // per-column coefficients of the current geometry pair
    float *gp32;                           // the same in FP32 (for the FP32 operator; may be null)
    const float *w32;                      // weights in FP32: wx1, wx2, wy1, wy2 (7 each), ws1, ws2 (P x 7),
                                           // wxo1, wxo2 (7 x 7 each)
    const double *lu64;                    // nslot x m (rank-major), FP64 factors
    const float *lu32;                     // same, FP32 copy (mixed precision)
    const double *udinv64;                 // 1 / u_jj per rank
    const float *udinv32;
    // Per-column inverses of the in-column blocks of L and U (P x P each),
    // transposed: blk[(colrank * P + jp) * P + j] = inv[j][jp].
    const double *linv64, *uinv64;
    const float *linv32, *uinv32;
};

// Algorithmic cost per grid point of the building blocks (FP64 words).
struct CostModel {
    double fA, bA;   // operator apply
    double fM, bM;   // preconditioner application
};

struct Problem {
    sw_grid grid;
    sw_params params;
    sw_physics phys;
    int device;
    Dev dev;
    long long m;
    int ncol, P;
    // device allocations
    std::vector<void *> allocs;
    double *d_weights = nullptr;
    int *d_win = nullptr;
    double *d_hcols = nullptr;     // h, hx, hy, hxx, hyy
    double *d_geom = nullptr;      // per-column coefficients (20 x ncol)
    float *d_geom32 = nullptr;     // FP32 copy (20 x ncol)
    float *d_weights32 = nullptr;
    double *d_lu64 = nullptr, *d_udinv64 = nullptr;
    float *d_lu32 = nullptr, *d_udinv32 = nullptr;
    double *d_linv64 = nullptr, *d_uinv64 = nullptr;
    float *d_linv32 = nullptr, *d_uinv32 = nullptr;
    double *d_V = nullptr;         // (restart + 1) x m Krylov basis
    float *d_V32 = nullptr;
    double *d_work = nullptr;      // 6 x m work vectors
    double *d_Y[2] = {nullptr, nullptr};  // EWMA sketch, double buffered
    double *d_W = nullptr;         // k x m, A Y
    double *d_xprev = nullptr;
    double *d_X = nullptr;         // range finder: history x m past solutions
    double *d_Q = nullptr;         // k x m orthonormal basis of the sketch (orthonormalize)
    double *d_part = nullptr;      // per-block partial sums
    double *d_omega = nullptr;     // k doubles
    void *d_stats = nullptr;       // DevStats
    void *d_sync = nullptr;        // grid barrier / flags
    // stage driver state
    double *d_u = nullptr, *d_v = nullptr, *d_w = nullptr, *d_eta = nullptr;
    double *d_Ku = nullptr, *d_Kv = nullptr, *d_Kw = nullptr, *d_Keta = nullptr;
    double *d_p = nullptr, *d_rhs = nullptr, *d_eta_new = nullptr, *d_feta = nullptr;
    double *d_drv = nullptr;       // driver scratch (several fields)
    double *d_host_io = nullptr;   // staging for the host-buffer entry point
    int *d_gcol = nullptr;         // walls: column order of the ILU sweeps
    int *d_goff = nullptr;         // walls: group offsets (device copy of goff_h)
    int goff_h[MAX_GROUPS + 1] = {};   // first column rank of each group (host)
    unsigned char *d_grp = nullptr;
    bool relax_on = false;         // generation/absorption zones after each stage
    sw_relaxation relax{};
    double relax_k = 0.0;          // wavenumber of the incident wave
    long long step_index = 0;      // completed Runge-Kutta steps since sw_set_state
    int ybuf = 0;                  // which sketch buffer holds Y
    bool pending = false;          // Y still lacks the newest solution (folded in by the next solve)
    long long n_solves = 0;
    long long total_iterations = 0;
    int stage = 0;                 // next Runge-Kutta stage, 0..4
    int nblocks = 0, nthreads = 0;
    int exec = SW_EXEC_PERSISTENT;  // resolved executor of the solves
    void *streamed = nullptr;      // state of the streamed executor
    void *resident = nullptr;      // state of the resident executor
    int resident_stall = -1;       // testing aid of sw_test_stall_exchange (next solve only)
    size_t smem = 0;
    cudaStream_t last_stream = nullptr;
    bool has_state = false;
    long long launches = 0;        // kernels launched by this problem
    CostModel cost{};
    // solve-kernel timing (events on the launching stream)
    bool timing = false;
    std::vector<cudaEvent_t> ev;   // pairs (start, stop)
    int ev_used = 0;
    double timed_ms = 0.0;
    long long n_timed = 0;
};

// Statistics written by the device at the end of a solve.
struct DevStats {
    int iterations, restarts, converged, status;
    double res0, res_final, true_res, guess_res, bnorm, braw;
    int guess_rank, guess_mode, cholesky_shift, pad;
    long long total_iterations;
    double model_flops, model_bytes;
    double phase_ns[16];   // cumulative device time per solve phase (block 0's view)
};


// Host helpers of the finite-difference set-up (setup.cu), shared by every
// entry point that builds weights.
// 7-point derivative weights w1 (first) and w2 (second derivative) at z over
// the nodes x[0..6], from the derivatives of the Lagrange basis polynomials.
void lagrange_weights(const long double *x, long double z, double *w1, double *w2);
// First level of the 7-level sigma window used at level j (j = -1..nz-1).
int sigma_window(int nz, int j);
// Centred x and y weights (7 each) and the sigma weights and windows of every
// level (ws1, ws2: (nz + 1) x 7, row j + 1; win: nz + 1) of a grid.
void grid_weights(const sw_grid &g, double *wx1, double *wx2, double *wy1, double *wy2, double *ws1, double *ws2,
                  int *win);

// Raise the dynamic shared-memory limit of kernel `kern` to at least `bytes`.
// The limit is one setting per kernel function shared by every problem, so it
// only ever grows (a problem created later with a smaller need must not lower
// it under an earlier one's); thread-safe.
cudaError_t ensure_smem(const void *kern, size_t bytes);

void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

}  // namespace sw
