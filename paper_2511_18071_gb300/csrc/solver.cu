// The Poisson solve of one Runge-Kutta stage as one persistent cooperative
// kernel (Algorithm 2 with the EWMA subspace of Algorithm 4, then restarted
// GMRES left-preconditioned with the fixed ILU(0) factors, Sec. 3 and 4).
// All control flow stays on the device: every block runs the same loop, the
// decisions (convergence, breakdown, restarts) are made on values that every
// block reduces identically, and grid barriers separate the phases.
#include <cmath>
#include <cstring>

#include "sw_device.cuh"

namespace sw {

struct SolveArgs {
    const double *eta_prev, *eta_cur, *b;
    double *x;
    double *V;        // (restart + 1) x m
    double *r;        // work
    double *t;        // work
    double *Yold, *Ynew, *Wm, *xprev;
    double *part;     // 2 x PART_STRIDE x nb
    DevStats *stats;
    Tiling tl;
    int restart, max_restarts, guess_mode, k, pending, nb;
    int guess_only;   // stop after writing x0 (sw_subspace_guess)
    double tol, decay;
    double omega[MAX_K];
    CostModel cm;
};

// Phases of a solve, timed by block 0 between grid barriers (profiling aid).
enum Phase {
    PH_GEOM = 0, PH_BNORM, PH_GUESS_W, PH_GUESS_LS, PH_RES_APPLY, PH_RES_ILU, PH_ARN_APPLY, PH_ARN_ILU,
    PH_CGS1, PH_CGS2, PH_CGS3, PH_GIVENS, PH_UPDATE, PH_TRUERES, PH_COUNT
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// ---- shared-memory layout of the solve kernel ----
struct SmemFixed {
    double red[NWARPS * 32];
    double res[PART_STRIDE + 8];
    double H[(MAX_RESTART + 1) * MAX_RESTART];
    double cs[MAX_RESTART], sn[MAX_RESTART], g[MAX_RESTART + 1], y[MAX_RESTART];
    double scale[MAX_RESTART + 1];
    double hs[MAX_RESTART];        // projection coefficients of the current Gram-Schmidt pass, times scale
    double G[MAX_K * MAX_K], R1[MAX_K * MAX_K], R2[MAX_K * MAX_K], R[MAX_K * MAX_K];
    double c1[MAX_K], c2[MAX_K], z[MAX_K], tmp[MAX_K];
    int flags[8];
    unsigned char ga[PART_STRIDE], gb[PART_STRIDE];   // Gram entry e -> (row, column), row <= column
};

struct LdVec {
    const double *v;
    double s;
    __device__ double operator()(long long i) const { return s * v[i]; }
};
struct LdEwma {
    const double *Y, *x;
    double rho, om;
    __device__ double operator()(long long i) const { return rho * Y[i] + om * x[i]; }
};
struct StVec {
    double *y;
    __device__ void operator()(long long i, double v) const { y[i] = v; }
};
struct StResid {
    const double *b;
    double *r;
    double acc;
    __device__ void operator()(long long i, double v) {
        double t = b[i] - v;
        r[i] = t;
        acc += t * t;
    }
};

template <class L, class S>
__device__ inline void apply_grid(const Dev &D, const Tiling &tl, double *sp, double *sq, L &ld, S &st) {
    for (int tile = blockIdx.x; tile < tl.ntiles; tile += gridDim.x) apply_tile<double>(D, tl, tile, sp, sq, ld, st);
}

// out = U^-1 L^-1 in over the whole grid (7 grid barriers, the last one included).
__device__ inline void ilu_apply_grid(const Dev &D, cg::grid_group &grid, const double *in, double *out) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int per = D.ncol >> 2;
    for (int c = 0; c < 4; ++c) {
        for (int q = gw; q < per; q += nw) ilu_fwd_column<double, double>(D, c, q, in, out, lane);
        if (c < 3) grid.sync();
    }
    for (int q = gw; q < per; q += nw) ilu_bwd_column<double>(D, 3, q, out, lane);
    grid.sync();
    for (int c = 2; c >= 0; --c) {
        for (int q = gw; q < per; q += nw) ilu_bwd_column<double>(D, c, q, out, lane);
        grid.sync();
    }
}

// Sum n <= 32 per-thread values over the grid into out[] (shared, all blocks).
__device__ inline void grid_sum32(cg::grid_group &grid, double (&v)[32], int n, SmemFixed &S, double *part, int nb,
                                  double *out, bool active = true) {
    block_partials32(v, n, S.red, part, nb, active);
    grid.sync();
    gather_partials(part, n, nb, out, S.red);
}

// Distributed variant for many values: block b finishes values b, b + nb, ...
// and publishes them; a second barrier makes them visible to everyone.
__device__ inline void grid_sum_many(cg::grid_group &grid, const double *part, int n, int nb, double *finals,
                                     double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = blockIdx.x * NWARPS + warp; i < n; i += nb * NWARPS) {
        double t[5];
#pragma unroll
        for (int u = 0; u < 5; ++u) t[u] = lane + 32 * u < nb ? part[i * nb + lane + 32 * u] : 0.0;
        double s = (t[0] + t[1]) + (t[2] + t[3]) + t[4];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) finals[i] = s;
    }
    grid.sync();
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = finals[i];
    __syncthreads();
}

// Upper-triangular Cholesky G = R^T R of a k x k matrix by one warp.
// Returns false on a non-positive pivot.
__device__ inline bool warp_cholesky(double *G, double *R, int k) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < k * k; i += 32) R[i] = 0.0;
    __syncwarp();
    bool ok = true;
    for (int j = 0; j < k; ++j) {
        double piv = G[j * k + j];
        if (!(piv > 0.0)) { ok = false; break; }
        double rjj = sqrt(piv);
        double inv = 1.0 / rjj;
        if (lane == 0) R[j * k + j] = rjj;
        for (int l = j + 1 + lane; l < k; l += 32) R[j * k + l] = G[j * k + l] * inv;
        __syncwarp();
        // trailing update G[a][b] -= R[j][a] R[j][b], a <= b, a, b > j
        for (int e = lane; e < k * k; e += 32) {
            int a = e / k, b = e % k;
            if (a > j && b >= a) {
                double v = G[a * k + b] - R[j * k + a] * R[j * k + b];
                G[a * k + b] = v;
                G[b * k + a] = v;
            }
        }
        __syncwarp();
    }
    __syncwarp();
    return ok;
}

// One warp: solve U z = rhs (U upper k x k), z written to out; rows whose
// |U_jj| <= tiny are skipped with z_j = 0.
__device__ inline void warp_backsub(const double *U, const double *rhs, double *out, int k, double tiny) {
    const int lane = threadIdx.x & 31;
    double acc = lane < k ? rhs[lane] : 0.0;
    for (int j = k - 1; j >= 0; --j) {
        double ujj = U[j * k + j];
        bool keep = fabs(ujj) > tiny;
        double zj = __shfl_sync(0xffffffffu, acc, j);
        zj = keep ? zj / ujj : 0.0;
        if (lane == j) out[j] = zj;
        if (lane < j) acc -= U[lane * k + j] * zj;
    }
    __syncwarp();
}

// One warp: solve U^T w = rhs (forward substitution with the transpose).
__device__ inline void warp_fwdsub_t(const double *U, const double *rhs, double *out, int k) {
    const int lane = threadIdx.x & 31;
    double acc = lane < k ? rhs[lane] : 0.0;
    for (int j = 0; j < k; ++j) {
        double wj = __shfl_sync(0xffffffffu, acc, j) / U[j * k + j];
        if (lane == j) out[j] = wj;
        if (lane > j && lane < k) acc -= U[j * k + lane] * wj;
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// The solve kernel.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NTHREADS, 1) solve_kernel(Dev D, SolveArgs A) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemFixed &S = *reinterpret_cast<SmemFixed *>(smem_raw);
    double *sp = reinterpret_cast<double *>(smem_raw + ((sizeof(SmemFixed) + 255) & ~size_t(255)));
    double *sq = sp + (size_t)D.P * A.tl.HW;
    const long long m = D.m;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gnth = gridDim.x * blockDim.x;
    const int nb = A.nb;
    const int k = A.k;
    int pbuf = 0;
    auto part = [&]() {
        double *p = A.part + (size_t)pbuf * PART_STRIDE * nb;
        pbuf ^= 1;
        return p;
    };
    double *finals = A.part + (size_t)2 * PART_STRIDE * nb;   // PART_STRIDE values
    // algorithmic cost of this solve (per grid point unit costs times m)
    double mf = 0.0, mb = 0.0;
    const double md = (double)m;
    auto cost = [&](double f, double b) { mf += f * md; mb += b * md; };
    double ph[PH_COUNT];
    for (int i = 0; i < PH_COUNT; ++i) ph[i] = 0.0;
    unsigned long long t_last = global_ns();
    auto tick = [&](int phase) {
        if (gtid == 0) {
            unsigned long long t = global_ns();
            ph[phase] += (double)(t - t_last);
            t_last = t;
        }
    };
    if (threadIdx.x == 0) {
        int e = 0;
        for (int a = 0; a < k; ++a)
            for (int b = a; b < k; ++b, ++e) { S.ga[e] = (unsigned char)a; S.gb[e] = (unsigned char)b; }
    }

    // a1: geometry of the stage pair
    geometry_columns(D, A.eta_prev, A.eta_cur, gtid, gnth);
    grid.sync();
    tick(PH_GEOM);

    // reference norms ||b|| and ||M^-1 b||
    ilu_apply_grid(D, grid, A.b, A.t);
    {
        double v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.0;
        for (long long p = gtid; p < m; p += gnth) {
            double bb = A.b[p], tt = A.t[p];
            v[0] += bb * bb;
            v[1] += tt * tt;
        }
        grid_sum32(grid, v, 2, S, part(), nb, S.res);
    }
    const double braw = sqrt(S.res[0]);
    const double bnorm = sqrt(S.res[1]);
    cost(A.cm.fM + 4.0, A.cm.bM + 8.0);
    tick(PH_BNORM);

    // ---- a7-a10: initial guess (Algorithm 2) ----
    int guess_rank = -1, shifted = 0;
    if (A.pending || A.guess_mode == SW_GUESS_EWMA) {
        // Y_new = r Y_old + x_prev omega^T (Algorithm 4) and W = A Y_new
        const bool upd = A.pending != 0;
        if (upd) cost(3.0 * k, (2.0 * k + 1.0) * 8.0);
        if (A.guess_mode == SW_GUESS_EWMA) cost(k * A.cm.fA, k * (A.cm.bA + 8.0));
        for (int c = 0; c < k; ++c) {
            const double *Yc = A.Yold + (size_t)c * m;
            double *Ync = A.Ynew + (size_t)c * m;
            if (upd)
                for (long long p = gtid; p < m; p += gnth) Ync[p] = A.decay * Yc[p] + A.omega[c] * A.xprev[p];
            if (A.guess_mode == SW_GUESS_EWMA) {
                StVec st{A.Wm + (size_t)c * m};
                if (upd) {
                    LdEwma ld{Yc, A.xprev, A.decay, A.omega[c]};
                    apply_grid(D, A.tl, sp, sq, ld, st);
                } else {
                    LdVec ld{Yc, 1.0};
                    apply_grid(D, A.tl, sp, sq, ld, st);
                }
            }
        }
        grid.sync();
    }
    tick(PH_GUESS_W);
    const double *Ycur = A.pending ? A.Ynew : A.Yold;
    if (A.guess_mode == SW_GUESS_EWMA) {
        // Gram G = W^T W and c = W^T b (a8), k(k+1)/2 + k values in chunks of 32
        const int ng = k * (k + 1) / 2;
        const int nv = ng + k;
        cost(2.0 * nv, (k + 1.0) * 8.0);
        double *pt = part();
        for (int c0 = 0; c0 < nv; c0 += 32) {
            double v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = 0.0;
            for (long long p = gtid; p < m; p += gnth) {
                double wv[MAX_K];
#pragma unroll
                for (int c = 0; c < MAX_K; ++c) wv[c] = c < k ? A.Wm[(size_t)c * m + p] : 0.0;
                double bp = A.b[p];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    int e = c0 + i;
                    if (e >= nv) break;
                    double prod;
                    if (e < ng) {
                        prod = wv[S.ga[e]] * wv[S.gb[e]];
                    } else {
                        prod = wv[e - ng] * bp;
                    }
                    v[i] += prod;
                }
            }
            block_partials32(v, min(32, nv - c0), S.red, pt + (size_t)c0 * nb, nb);
        }
        grid.sync();
        grid_sum_many(grid, pt, nv, nb, finals, S.res);
        // unpack
        if (threadIdx.x < 32) {
            for (int e = threadIdx.x; e < ng; e += 32) {
                S.G[S.ga[e] * k + S.gb[e]] = S.res[e];
                S.G[S.gb[e] * k + S.ga[e]] = S.res[e];
            }
            for (int c = threadIdx.x; c < k; c += 32) S.c1[c] = S.res[ng + c];
            __syncwarp();
            // a9: CholeskyQR2 step 1, shifted (Fukaya et al. 2020) if the Gram is not numerically SPD
            double tr = 0.0;
            for (int c = 0; c < k; ++c) tr += S.G[c * k + c];
            for (int i = threadIdx.x; i < k * k; i += 32) S.R[i] = S.G[i];   // keep a copy
            __syncwarp();
            bool ok = tr > 0.0 && warp_cholesky(S.G, S.R1, k);
            if (!ok && tr > 0.0) {
                double sh = 11.0 * ((double)m * k + (double)k * (k + 1)) * 1.1102230246251565e-16 * tr;
                for (int i = threadIdx.x; i < k * k; i += 32) S.G[i] = S.R[i] + ((i / k == i % k) ? sh : 0.0);
                __syncwarp();
                ok = warp_cholesky(S.G, S.R1, k);
                shifted = 1;
            }
            if (threadIdx.x == 0) S.flags[0] = ok ? 1 : 0;
        }
        __syncthreads();
        const bool ok1 = S.flags[0] != 0;
        if (ok1) {
            cost((double)k * k + 2.0 * nv, (k + 1.0) * 8.0);
            // second pass: Q1 = W R1^-1, G2 = Q1^T Q1, c2 = Q1^T b
            double *pt2 = part();
            for (int c0 = 0; c0 < nv; c0 += 32) {
                double v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.0;
                for (long long p = gtid; p < m; p += gnth) {
                    double q[MAX_K];
#pragma unroll
                    for (int c = 0; c < MAX_K; ++c) {
                        if (c >= k) { q[c] = 0.0; continue; }
                        double s = A.Wm[(size_t)c * m + p];
                        for (int i = 0; i < c; ++i) s -= q[i] * S.R1[i * k + c];
                        q[c] = s / S.R1[c * k + c];
                    }
                    double bp = A.b[p];
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        int e = c0 + i;
                        if (e >= nv) break;
                        double prod;
                        if (e < ng) {
                            prod = q[S.ga[e]] * q[S.gb[e]];
                        } else {
                            prod = q[e - ng] * bp;
                        }
                        v[i] += prod;
                    }
                }
                block_partials32(v, min(32, nv - c0), S.red, pt2 + (size_t)c0 * nb, nb);
            }
            grid.sync();
            grid_sum_many(grid, pt2, nv, nb, finals, S.res);
            if (threadIdx.x < 32) {
                for (int e = threadIdx.x; e < ng; e += 32) {
                    S.G[S.ga[e] * k + S.gb[e]] = S.res[e];
                    S.G[S.gb[e] * k + S.ga[e]] = S.res[e];
                }
                for (int c = threadIdx.x; c < k; c += 32) S.c2[c] = S.res[ng + c];
                __syncwarp();
                bool ok2 = warp_cholesky(S.G, S.R2, k);
                if (!ok2) {
                    // Q1 is far from orthonormal: fall back on R = R1 and Q^T b = R1^-T W^T b
                    for (int i = threadIdx.x; i < k * k; i += 32) S.R[i] = S.R1[i];
                    __syncwarp();
                    warp_fwdsub_t(S.R1, S.c1, S.tmp, k);
                } else {
                    // R = R2 R1; Q^T b = R2^-T (Q1^T b)
                    for (int e = threadIdx.x; e < k * k; e += 32) {
                        int a = e / k, bc = e % k;
                        double s = 0.0;
                        for (int l = a; l <= bc; ++l) s += S.R2[a * k + l] * S.R1[l * k + bc];
                        S.R[e] = bc >= a ? s : 0.0;
                    }
                    __syncwarp();
                    warp_fwdsub_t(S.R2, S.c2, S.tmp, k);
                }
                // rank guard as in the reference: drop columns with |R_jj| <= 1e-12 |R_00|
                double tiny = 1e-12 * fabs(S.R[0]);
                warp_backsub(S.R, S.tmp, S.z, k, tiny);
                if (threadIdx.x == 0) {
                    int rk = 0;
                    for (int j = 0; j < k; ++j) rk += fabs(S.R[j * k + j]) > tiny;
                    S.flags[1] = rk;
                }
            }
            __syncthreads();
            guess_rank = S.flags[1];
        } else {
            if (threadIdx.x < MAX_K) S.z[threadIdx.x] = 0.0;
            __syncthreads();
            guess_rank = 0;
        }
        // a10: x0 = Y z
        cost(2.0 * k, (k + 1.0) * 8.0);
        for (long long p = gtid; p < m; p += gnth) {
            double s = 0.0;
            for (int c = 0; c < k; ++c) s += Ycur[(size_t)c * m + p] * S.z[c];
            A.x[p] = s;
        }
    } else if (A.guess_mode == SW_GUESS_PREVIOUS) {
        cost(0.0, 16.0);
        for (long long p = gtid; p < m; p += gnth) A.x[p] = A.xprev[p];
    } else {
        for (long long p = gtid; p < m; p += gnth) A.x[p] = 0.0;
    }
    grid.sync();
    tick(PH_GUESS_LS);
    if (A.guess_only) {
        if (gtid == 0) {
            A.stats->guess_rank = guess_rank;
            A.stats->cholesky_shift = shifted;
        }
        return;
    }

    // ---- GMRES(m), left-preconditioned (Sec. 3) ----
    int iters = 0, restarts = 0, converged = 0, status = SW_ERR_NOT_CONVERGED;
    double res0 = 0.0, res_last = 0.0, guess_res = 0.0;
    const int mr = A.restart;
    if (bnorm == 0.0) {
        for (long long p = gtid; p < m; p += gnth) A.x[p] = 0.0;
        converged = 1;
        status = SW_OK;
    } else {
        for (int cycle = 0;; ++cycle) {
            // r = b - A x ; V0 = M^-1 r
            {
                StResid st{A.b, A.r, 0.0};
                LdVec ld{A.x, 1.0};
                apply_grid(D, A.tl, sp, sq, ld, st);
                double v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.0;
                v[0] = st.acc;
                grid.sync();
                tick(PH_RES_APPLY);
                ilu_apply_grid(D, grid, A.r, A.V);
                for (long long p = gtid; p < m; p += gnth) v[1] += A.V[p] * A.V[p];
                grid_sum32(grid, v, 2, S, part(), nb, S.res);
                tick(PH_RES_ILU);
            }
            const double beta = sqrt(S.res[1]);
            cost(A.cm.fA + A.cm.fM + 4.0, A.cm.bA + A.cm.bM + 8.0);
            if (cycle == 0) {
                res0 = beta / bnorm;
                guess_res = braw > 0.0 ? sqrt(S.res[0]) / braw : sqrt(S.res[0]);
            }
            res_last = beta / bnorm;
            if (!isfinite(beta)) { status = SW_ERR_NAN; break; }
            if (beta <= A.tol * bnorm) { converged = 1; status = SW_OK; break; }
            if (cycle == A.max_restarts + 1) break;
            if (cycle > 0) ++restarts;
            if (threadIdx.x == 0) {
                S.scale[0] = 1.0 / beta;
                for (int i = 0; i <= mr; ++i) S.g[i] = 0.0;
                S.g[0] = beta;
            }
            __syncthreads();
            int jend = 0;
            for (int j = 0; j < mr; ++j) {
                double *w = A.V + (size_t)(j + 1) * m;
                // w = M^-1 A v_j  (v_j = scale_j * V_j)
                {
                    LdVec ld{A.V + (size_t)j * m, S.scale[j]};
                    StVec st{A.t};
                    apply_grid(D, A.tl, sp, sq, ld, st);
                    grid.sync();
                    tick(PH_ARN_APPLY);
                    ilu_apply_grid(D, grid, A.t, w);
                    tick(PH_ARN_ILU);
                }
                // CGS2 pass 1: d_i = V_i . w
                // Gram-Schmidt passes: warp w of block b takes 32-point chunks
                // b + nb w, b + nb (w + NWARPS), ... so that the warps holding
                // data are spread over the blocks and sub-partitions
                const int wlane = threadIdx.x & 31, wid = threadIdx.x >> 5;
                const long long k0 = blockIdx.x + (long long)nb * wid, kstep = (long long)nb * NWARPS;
                const bool wactive = 32 * k0 < m;
                double v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.0;
                for (long long kc = k0; 32 * kc < m; kc += kstep) {
                    const long long p = 32 * kc + wlane;
                    if (p >= m) continue;
                    double vb[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) vb[i] = i <= j ? A.V[(size_t)i * m + p] : 0.0;
                    const double wv = w[p];
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        if (i > j) break;
                        v[i] += vb[i] * wv;
                    }
                }
                grid_sum32(grid, v, j + 1, S, part(), nb, S.res, wactive);
                tick(PH_CGS1);
                if (threadIdx.x < MAX_RESTART) {
                    const int i = threadIdx.x;
                    double hi = i <= j ? S.res[i] * S.scale[i] : 0.0;
                    if (i <= j) S.H[i * MAX_RESTART + j] = hi;
                    S.hs[i] = i <= j ? hi * S.scale[i] : 0.0;
                }
                __syncthreads();
                // pass 2: w -= V h ; d'_i = V_i . w
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.0;
                for (long long kc = k0; 32 * kc < m; kc += kstep) {
                    const long long p = 32 * kc + wlane;
                    if (p >= m) continue;
                    double vb[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) vb[i] = i <= j ? A.V[(size_t)i * m + p] : 0.0;
                    double wv = w[p];
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        if (i > j) break;
                        wv -= S.hs[i] * vb[i];
                    }
                    w[p] = wv;
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        if (i > j) break;
                        v[i] += vb[i] * wv;
                    }
                }
                grid_sum32(grid, v, j + 1, S, part(), nb, S.res, wactive);
                tick(PH_CGS2);
                if (threadIdx.x < MAX_RESTART) {
                    const int i = threadIdx.x;
                    double hi = i <= j ? S.res[i] * S.scale[i] : 0.0;
                    if (i <= j) S.H[i * MAX_RESTART + j] += hi;
                    S.hs[i] = i <= j ? hi * S.scale[i] : 0.0;
                }
                __syncthreads();
                // pass 3: w -= V h' ; ||w||^2
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.0;
                for (long long kc = k0; 32 * kc < m; kc += kstep) {
                    const long long p = 32 * kc + wlane;
                    if (p >= m) continue;
                    double vb[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) vb[i] = i <= j ? A.V[(size_t)i * m + p] : 0.0;
                    double wv = w[p];
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        if (i > j) break;
                        wv -= S.hs[i] * vb[i];
                    }
                    w[p] = wv;
                    v[0] += wv * wv;
                }
                grid_sum32(grid, v, 1, S, part(), nb, S.res, wactive);
                tick(PH_CGS3);
                // a5: Hessenberg column, Givens rotations, residual estimate
                if (threadIdx.x == 0) {
                    double hn = sqrt(S.res[0]);
                    S.scale[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
                    double *Hc = S.H;
                    for (int i = 0; i < j; ++i) {
                        double a = Hc[i * MAX_RESTART + j], bb = Hc[(i + 1) * MAX_RESTART + j];
                        Hc[i * MAX_RESTART + j] = S.cs[i] * a + S.sn[i] * bb;
                        Hc[(i + 1) * MAX_RESTART + j] = -S.sn[i] * a + S.cs[i] * bb;
                    }
                    double a = Hc[j * MAX_RESTART + j];
                    double den = hypot(a, hn);
                    S.cs[j] = a / den;
                    S.sn[j] = hn / den;
                    Hc[j * MAX_RESTART + j] = den;
                    S.g[j + 1] = -S.sn[j] * S.g[j];
                    S.g[j] = S.cs[j] * S.g[j];
                    S.flags[2] = (fabs(S.g[j + 1]) <= A.tol * bnorm) || hn == 0.0;
                }
                __syncthreads();
                tick(PH_GIVENS);
                cost(A.cm.fA + A.cm.fM + 8.0 * (j + 1) + 2.0, A.cm.bA + A.cm.bM + (3.0 * j + 8.0) * 8.0);
                ++iters;
                jend = j + 1;
                if (S.flags[2]) break;
            }
            // a6: y = R^-1 g, x += V (scale y)
            if (threadIdx.x < 32) {
                const int lane = threadIdx.x;
                double acc = lane < jend ? S.g[lane] : 0.0;
                for (int i = jend - 1; i >= 0; --i) {
                    double yi = __shfl_sync(0xffffffffu, acc, i) / S.H[i * MAX_RESTART + i];
                    if (lane == i) S.y[i] = yi * S.scale[i];
                    if (lane < i) acc -= S.H[lane * MAX_RESTART + i] * yi;
                }
            }
            __syncthreads();
            cost(2.0 * jend, (jend + 2.0) * 8.0);
            for (long long p = gtid; p < m; p += gnth) {
                double s = A.x[p];
                for (int i = 0; i < jend; ++i) s += S.y[i] * A.V[(size_t)i * m + p];
                A.x[p] = s;
            }
            grid.sync();
            tick(PH_UPDATE);
        }
    }
    // true residual ||b - A x|| / ||b||, solution kept for the next guess
    double true_res;
    {
        StResid st{A.b, A.r, 0.0};
        LdVec ld{A.x, 1.0};
        apply_grid(D, A.tl, sp, sq, ld, st);
        double v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.0;
        v[0] = st.acc;
        for (long long p = gtid; p < m; p += gnth) A.xprev[p] = A.x[p];
        grid_sum32(grid, v, 1, S, part(), nb, S.res);
        true_res = braw > 0.0 ? sqrt(S.res[0]) / braw : sqrt(S.res[0]);
        cost(A.cm.fA + 3.0, A.cm.bA + 24.0);
    }
    tick(PH_TRUERES);
    if (gtid == 0) {
        DevStats &st = *A.stats;
        st.iterations = iters;
        st.restarts = restarts;
        st.converged = converged;
        st.status = status;
        st.res0 = res0;
        st.res_final = res_last;
        st.true_res = true_res;
        st.guess_res = guess_res;
        st.bnorm = bnorm;
        st.braw = braw;
        st.guess_rank = guess_rank;
        st.guess_mode = A.guess_mode;
        st.cholesky_shift = shifted;
        st.total_iterations += iters;
        st.model_flops += mf;
        st.model_bytes += mb;
        for (int i = 0; i < PH_COUNT; ++i) st.phase_ns[i] += ph[i];
    }
}

// ---------------------------------------------------------------------------
// Standalone kernels for the per-step entry points.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NTHREADS) geometry_kernel(Dev D, const double *ep, const double *ec) {
    geometry_columns(D, ep, ec, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void __launch_bounds__(NTHREADS) apply_kernel(Dev D, Tiling tl, const double *x, double *y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *sp = reinterpret_cast<double *>(smem_raw);
    double *sq = sp + (size_t)D.P * tl.HW;
    LdVec ld{x, 1.0};
    StVec st{y};
    for (int tile = blockIdx.x; tile < tl.ntiles; tile += gridDim.x) apply_tile<double>(D, tl, tile, sp, sq, ld, st);
}

__global__ void __launch_bounds__(NTHREADS) ilu_fwd_kernel(Dev D, int c, const double *in, double *out) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int q = gw; q < (D.ncol >> 2); q += nw) ilu_fwd_column<double, double>(D, c, q, in, out, lane);
}

struct SketchUpd {
    double om[MAX_K];
};

// Y <- r Y + x omega^T (Algorithm 4), column c at Y + c m.
__global__ void __launch_bounds__(NTHREADS) sketch_update_kernel(double *Y, const double *x, SketchUpd u, int k,
                                                                 long long m, double rho) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m; p += (long long)gridDim.x * blockDim.x) {
        double xp = x[p];
        for (int c = 0; c < k; ++c) Y[(size_t)c * m + p] = rho * Y[(size_t)c * m + p] + u.om[c] * xp;
    }
}

__global__ void __launch_bounds__(NTHREADS) ilu_bwd_kernel(Dev D, int c, double *out) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int q = gw; q < (D.ncol >> 2); q += nw) ilu_bwd_column<double>(D, c, q, out, lane);
}

// ---------------------------------------------------------------------------
// Launch configuration.
// ---------------------------------------------------------------------------
static Tiling make_tiling(const Dev &D) {
    Tiling t{};
    if (!D.three_d) {
        // enough tiles to spread over the SMs, at most 64 columns per tile
        int TX = 64;
        while (TX > 4 && (D.nx % TX != 0 || D.nx / TX < 304)) TX >>= 1;
        t.TX = TX; t.TY = 1;
    } else {
        int TX = 16, TY = 8;
        while ((size_t)(TX + 6) * (TY + 6) * D.P * 2 * sizeof(double) > 150 * 1024 && TX > 4) {
            if (TX > TY) TX >>= 1; else TY >>= 1;
        }
        while (D.nx % TX) TX >>= 1;
        while (D.ny % TY) TY >>= 1;
        t.TX = TX; t.TY = TY;
    }
    t.HX = t.TX + 2 * HALF;
    t.HY = D.three_d ? t.TY + 2 * HALF : 1;
    t.HW = t.HX * t.HY;
    t.ntx = D.nx / t.TX;
    t.nty = D.three_d ? D.ny / t.TY : 1;
    t.ntiles = t.ntx * t.nty;
    return t;
}

static size_t solve_smem(const Dev &D, const Tiling &t) {
    return ((sizeof(SmemFixed) + 255) & ~size_t(255)) + 2 * (size_t)D.P * t.HW * sizeof(double);
}

int setup_solver_launch(Problem *P) {
    Tiling t = make_tiling(P->dev);
    size_t smem = solve_smem(P->dev, t);
    cudaError_t e = cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "solve_kernel smem attribute");
    e = cudaFuncSetAttribute(apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * (size_t)P->dev.P * t.HW * sizeof(double)));
    if (e != cudaSuccess) return cuda_fail(e, "apply_kernel smem attribute");
    int nsm = 0, per = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P->device);
    if (e != cudaSuccess) return cuda_fail(e, "SM count");
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, solve_kernel, NTHREADS, smem);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    if (per < 1) { set_error("solve kernel does not fit on an SM"); return SW_ERR_BAD_ARG; }
    // one block per SM; the cross-block gathers are sized for at most 160 blocks
    P->nblocks = nsm < NWARPS * GATHER_PER_WARP ? nsm : NWARPS * GATHER_PER_WARP;
    P->nthreads = NTHREADS;
    P->smem = smem;
    return SW_OK;
}

static Tiling tiling_of(const Problem *P) { return make_tiling(P->dev); }

// Fold the recorded event pairs into the running total.
static int flush_timing(Problem *P) {
    for (int i = 0; i < P->ev_used; ++i) {
        cudaError_t e = cudaEventSynchronize(P->ev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "event sync");
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, P->ev[2 * i], P->ev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "event time");
        P->timed_ms += ms;
        P->n_timed++;
    }
    P->ev_used = 0;
    return SW_OK;
}

static int launch_solve(Problem *P, const double *ep, const double *ec, const double *b, double *x,
                        cudaStream_t s, int guess_only) {
    const sw_params &pr = P->params;
    SolveArgs A{};
    A.eta_prev = ep; A.eta_cur = ec; A.b = b; A.x = x;
    A.V = P->d_V; A.r = P->d_work; A.t = P->d_work + P->m;
    A.Yold = P->d_Y[P->ybuf]; A.Ynew = P->d_Y[P->ybuf ^ 1];
    A.Wm = P->d_W; A.xprev = P->d_xprev; A.part = P->d_part; A.stats = (DevStats *)P->d_stats;
    A.tl = tiling_of(P);
    A.restart = pr.restart; A.max_restarts = pr.max_restarts; A.k = pr.k; A.nb = P->nblocks;
    A.tol = pr.tol; A.decay = pr.decay; A.guess_only = guess_only;
    int mode = pr.guess;
    if (mode == SW_GUESS_EWMA && P->n_solves < pr.n_init_solves) mode = SW_GUESS_PREVIOUS;
    if (guess_only) mode = SW_GUESS_EWMA;
    A.guess_mode = mode;
    A.cm = P->cost;
    A.pending = P->pending ? 1 : 0;
    if (A.pending) sw_draw_omega(pr.seed, P->n_solves - 1, pr.k, A.omega);
    Dev D = P->dev;
    void *args[] = {&D, &A};
    cudaError_t e = cudaSuccess;
    int evi = -1;
    if (P->timing) {
        if (P->ev_used * 2 + 2 > (int)P->ev.size()) {
            int rc = flush_timing(P);
            if (rc != SW_OK) return rc;
        }
        evi = P->ev_used++;
        e = cudaEventRecord(P->ev[2 * evi], s);
        if (e != cudaSuccess) return cuda_fail(e, "event record");
    }
    e = cudaLaunchCooperativeKernel((const void *)solve_kernel, P->nblocks, NTHREADS, args, P->smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "solve launch");
    P->launches++;
    if (evi >= 0) {
        e = cudaEventRecord(P->ev[2 * evi + 1], s);
        if (e != cudaSuccess) return cuda_fail(e, "event record");
    }
    if (A.pending) P->ybuf ^= 1;
    P->pending = false;
    if (!guess_only) {
        P->n_solves++;
        P->pending = pr.guess == SW_GUESS_EWMA;
    }
    P->last_stream = s;
    return SW_OK;
}

int solve_device(Problem *P, const double *ep, const double *ec, const double *b, double *x, cudaStream_t s) {
    return launch_solve(P, ep, ec, b, x, s, 0);
}

int read_stats(Problem *P, DevStats *out) {
    cudaError_t e = cudaStreamSynchronize(P->last_stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream sync");
    e = cudaMemcpy(out, P->d_stats, sizeof(DevStats), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "stats copy");
    return SW_OK;
}

}  // namespace sw

using namespace sw;

extern "C" int sw_solve_poisson(sw_problem *pp, const double *ep, const double *ec, const double *b, double *x,
                                void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !ep || !ec || !b || !x) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    return solve_device(P, ep, ec, b, x, (cudaStream_t)stream);
}

extern "C" int sw_solve_poisson_host(sw_problem *pp, const double *hep, const double *hec, const double *hb,
                                     double *hx, void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !hep || !hec || !hb || !hx) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    double *db = P->d_host_io, *dx = db + P->m, *dep = dx + P->m, *dec = dep + P->ncol;
    cudaError_t e = cudaMemcpyAsync(db, hb, P->m * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dep, hep, P->ncol * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dec, hec, P->ncol * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    int rc = solve_device(P, dep, dec, db, dx, s);
    if (rc != SW_OK) return rc;
    e = cudaMemcpyAsync(hx, dx, P->m * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    DevStats st;
    rc = read_stats(P, &st);
    if (rc != SW_OK) return rc;
    return st.status;
}

extern "C" int sw_get_stats(sw_problem *pp, sw_stats *out) {
    Problem *P = (Problem *)pp;
    if (!P || !out) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    DevStats st;
    std::memset(&st, 0, sizeof(st));
    if (P->n_solves > 0) {
        int rc = read_stats(P, &st);
        if (rc != SW_OK) return rc;
    }
    out->iterations = st.iterations;
    out->restarts = st.restarts;
    out->converged = st.converged;
    out->status = P->n_solves > 0 ? st.status : SW_OK;
    out->res0 = st.res0;
    out->res_final = st.res_final;
    out->true_res = st.true_res;
    out->guess_res = st.guess_res;
    out->n_solves = P->n_solves;
    out->total_iterations = st.total_iterations;
    out->launches = P->launches;
    out->model_flops = st.model_flops;
    out->model_bytes = st.model_bytes;
    return SW_OK;
}

extern "C" int sw_get_phase_times(sw_problem *pp, double *us, int n) {
    Problem *P = (Problem *)pp;
    if (!P || !us || n < 1) { set_error("bad argument"); return SW_ERR_BAD_ARG; }
    DevStats st;
    std::memset(&st, 0, sizeof(st));
    if (P->n_solves > 0) {
        int rc = read_stats(P, &st);
        if (rc != SW_OK) return rc;
    }
    for (int i = 0; i < n && i < 16; ++i) us[i] = i < PH_COUNT ? st.phase_ns[i] * 1e-3 : 0.0;
    return SW_OK;
}

extern "C" int sw_enable_timing(sw_problem *pp, int on) {
    Problem *P = (Problem *)pp;
    if (!P) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    if (on && P->ev.empty()) {
        P->ev.resize(512);
        for (auto &ev : P->ev) {
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return cuda_fail(e, "event create");
        }
    }
    if (P->timing && !on) {
        int rc = flush_timing(P);
        if (rc != SW_OK) return rc;
    }
    P->timing = on != 0;
    P->timed_ms = 0.0;
    P->n_timed = 0;
    P->ev_used = 0;
    return SW_OK;
}

extern "C" int sw_get_solve_time(sw_problem *pp, double *total_ms, long long *n_timed) {
    Problem *P = (Problem *)pp;
    if (!P || !total_ms || !n_timed) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    int rc = flush_timing(P);
    if (rc != SW_OK) return rc;
    *total_ms = P->timed_ms;
    *n_timed = P->n_timed;
    return SW_OK;
}

extern "C" int sw_apply_operator(sw_problem *pp, const double *ep, const double *ec, const double *x, double *y,
                                 void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !ep || !ec || !x || !y) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    Tiling tl = tiling_of(P);
    int gb = (P->ncol + NTHREADS - 1) / NTHREADS;
    geometry_kernel<<<gb, NTHREADS, 0, s>>>(P->dev, ep, ec);
    apply_kernel<<<tl.ntiles, NTHREADS, 2 * (size_t)P->dev.P * tl.HW * sizeof(double), s>>>(P->dev, tl, x, y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "apply launch");
    P->launches += 2;
    P->last_stream = s;
    return SW_OK;
}

extern "C" int sw_apply_preconditioner(sw_problem *pp, const double *v, double *out, void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !v || !out || v == out) { set_error("bad argument"); return SW_ERR_BAD_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    int per = P->ncol >> 2;
    int blocks = (per * 32 + NTHREADS - 1) / NTHREADS;
    for (int c = 0; c < 4; ++c) ilu_fwd_kernel<<<blocks, NTHREADS, 0, s>>>(P->dev, c, v, out);
    for (int c = 3; c >= 0; --c) ilu_bwd_kernel<<<blocks, NTHREADS, 0, s>>>(P->dev, c, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "preconditioner launch");
    P->launches += 8;
    P->last_stream = s;
    return SW_OK;
}

extern "C" int sw_subspace_guess(sw_problem *pp, const double *ep, const double *ec, const double *b, double *x0,
                                 void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !ep || !ec || !b || !x0) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    return launch_solve(P, ep, ec, b, x0, (cudaStream_t)stream, 1);
}

extern "C" int sw_get_sketch(sw_problem *pp, double *Y, void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !Y) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    // The update with the newest solution is applied lazily at the start of
    // the next solve; apply it here on a copy when one is pending.
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = (size_t)P->params.k * P->m * sizeof(double);
    cudaError_t e = cudaMemcpyAsync(Y, P->d_Y[P->ybuf], bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "sketch copy");
    if (P->pending) {
        SketchUpd u;
        sw_draw_omega(P->params.seed, P->n_solves - 1, P->params.k, u.om);
        int blocks = (int)((P->m + NTHREADS - 1) / NTHREADS);
        if (blocks > 4096) blocks = 4096;
        sketch_update_kernel<<<blocks, NTHREADS, 0, s>>>(Y, P->d_xprev, u, P->params.k, P->m, P->params.decay);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "sketch update launch");
        P->launches++;
    }
    P->last_stream = s;
    return SW_OK;
}

extern "C" int sw_set_sketch(sw_problem *pp, const double *Y, long long n_solves, void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !Y || n_solves < 0) { set_error("bad argument"); return SW_ERR_BAD_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = (size_t)P->params.k * P->m * sizeof(double);
    cudaError_t e = cudaMemcpyAsync(P->d_Y[P->ybuf], Y, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "sketch copy");
    // the loaded sketch is complete: no update pending; later draws continue at n_solves
    P->n_solves = n_solves;
    P->pending = false;
    P->last_stream = s;
    return SW_OK;
}
