// One Poisson solve (Algorithm 2 with the EWMA subspace of Algorithm 4, then
// restarted GMRES left-preconditioned with the fixed ILU(0) factors, Sec. 3
// and 4) written once for two kinds of "team":
//   GridTeam  - every block of a cooperative grid works on one instance and
//               grid barriers separate the phases (single large instance);
//   BlockTeam - one thread block owns one instance and __syncthreads
//               separates the phases (batches of independent instances).
// and two inner precisions TI:
//   double - every step in FP64;
//   float  - the operator, the preconditioner and the Krylov vectors of the
//            GMRES cycles in FP32, with every reduction accumulated in FP64,
//            Gram-Schmidt coefficients, Hessenberg/Givens, the subspace sketch,
//            W = A Y and its least squares in FP64, and each restart
//            recomputing the residual b - A x and updating x in FP64
//            (GMRES-based iterative refinement).
#pragma once
#include "sw_device.cuh"

namespace sw {

struct SolveArgs {
    const double *eta_prev, *eta_cur, *b;
    double *x;
    void *V;          // (restart + 1) x m, inner type
    double *r;        // FP64 residual
    void *t;          // inner work vector
    double *Yold, *Ynew;      // k x m each; the sketch stays FP64 in both forms (an FP32 sketch
                              // loses the fine structure the least-squares combination relies on)
    double *Wm;               // k x m, A Y in FP64
    double *xprev;
    double *part;     // grid team: 2 x PART_STRIDE x nb partials + PART_STRIDE finals
    DevStats *stats;
    Tiling tl;
    int restart, max_restarts, guess_mode, k, pending, nb;
    int guess_only;   // stop after writing x0 (sw_subspace_guess)
    double tol, decay;
    double inner_rtol;   // inner cycle stop relative to its starting residual (FP32 inner only)
    double omega[MAX_K];
    CostModel cm;
    // range finder (Algorithm 3): Y = X Omega over the ke newest of K stored solutions
    const double *ring;       // K x m past solutions, slot = solve index mod K
    double *ring_store;       // slot that receives this solve's solution (null: none)
    int ring_K, ring_Ke, ring_newest;   // slots, solutions used, slot of the newest
    double omega_rrf[SW_RRF_MAX_HISTORY * MAX_K];   // row r (r-th newest) x column c at r k + c
    // optional V = Q of the sketch (the QR step of Algorithms 3 and 4)
    double *Vq;               // k x m, null unless orthonormalize
};

// Phases of a solve, timed between barriers by the team's first thread (profiling aid).
enum Phase {
    PH_GEOM = 0, PH_BNORM, PH_GUESS_W, PH_GUESS_LS, PH_RES_APPLY, PH_RES_ILU, PH_ARN_APPLY, PH_ARN_ILU,
    PH_CGS1, PH_CGS2, PH_CGS3, PH_GIVENS, PH_UPDATE, PH_TRUERES, PH_COUNT
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

struct SmemFixed {
    double red[NWARPS * 32];
    double res[PART_STRIDE + 8];
    double H[(MAX_RESTART + 1) * MAX_RESTART];
    double cs[MAX_RESTART], sn[MAX_RESTART], g[MAX_RESTART + 1], y[MAX_RESTART];
    double scale[MAX_RESTART + 1];
    double hs[MAX_RESTART];   // projection coefficients of the current Gram-Schmidt pass, times scale
    float hs32[MAX_RESTART];  // the same rounded to FP32 (FP32 inner form)
    double G[MAX_K * MAX_K], R1[MAX_K * MAX_K], R2[MAX_K * MAX_K], R[MAX_K * MAX_K];
    double c1[MAX_K], c2[MAX_K], z[MAX_K], tmp[MAX_K];
    int flags[8];
    unsigned char ga[PART_STRIDE], gb[PART_STRIDE];   // Gram entry e -> (row, column), row <= column
    double xchg[2 * PART_STRIDE];   // cluster team: this block's partial sums, read by the other blocks
};

// ---- teams ----
struct GridTeam {
    cg::grid_group g;
    int nb, bid;
    double *part;
    int pbuf;
    __device__ GridTeam(double *p, int nblocks) : g(cg::this_grid()), nb(nblocks), bid(blockIdx.x), part(p), pbuf(0) {}
    __device__ void sync() { g.sync(); }
    __device__ double *next_part() {
        double *q = part + (size_t)pbuf * PART_STRIDE * nb;
        pbuf ^= 1;
        return q;
    }
    __device__ double *finals() { return part + (size_t)2 * PART_STRIDE * nb; }
    // sum of n <= 32 per-thread values over the team into out[] (shared memory)
    __device__ void sum32(double (&v)[32], int n, SmemFixed &S, double *out, bool active = true) {
        double *pt = next_part();
        block_partials32(v, n, S.red, pt, nb, active);
        g.sync();
        gather_partials(pt, n, nb, out, S.red);
    }
    // sums of nv <= PART_STRIDE values computed in 32-value chunks by fill(c0, v)
    template <class Fill>
    __device__ void sum_many(int nv, SmemFixed &S, double *out, Fill fill) {
        double *pt = next_part();
        for (int c0 = 0; c0 < nv; c0 += 32) {
            double v[32];
            fill(c0, v);
            block_partials32(v, min(32, nv - c0), S.red, pt + (size_t)c0 * nb, nb);
        }
        g.sync();
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        double *fin = finals();
        for (int i = bid * NWARPS + warp; i < nv; i += nb * NWARPS) {
            double t[5];
#pragma unroll
            for (int u = 0; u < 5; ++u) t[u] = lane + 32 * u < nb ? pt[i * nb + lane + 32 * u] : 0.0;
            double s = (t[0] + t[1]) + (t[2] + t[3]) + t[4];
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) fin[i] = s;
        }
        g.sync();
        for (int i = threadIdx.x; i < nv; i += blockDim.x) out[i] = fin[i];
        __syncthreads();
    }
};

struct BlockTeam {
    int nb, bid;
    __device__ BlockTeam() : nb(1), bid(0) {}
    __device__ void sync() { __syncthreads(); }
    __device__ void sum32(double (&v)[32], int n, SmemFixed &S, double *out, bool active = true) {
        block_partials32(v, n, S.red, out, 1, active, 0);
    }
    template <class Fill>
    __device__ void sum_many(int nv, SmemFixed &S, double *out, Fill fill) {
        for (int c0 = 0; c0 < nv; c0 += 32) {
            double v[32];
            fill(c0, v);
            block_partials32(v, min(32, nv - c0), S.red, out + c0, 1, true, 0);
        }
    }
};

// A thread-block cluster owns the instance (batch members): hardware cluster
// barriers separate the phases, and partial sums are exchanged through
// distributed shared memory.  Every block sums the blocks' partials in rank
// order, so all blocks hold bit-identical totals and take the same decisions.
// Partial buffers alternate: a buffer is rewritten only after the next
// reduction's barrier, which every reader of it has passed.
constexpr int MAX_CLUSTER = 16;
struct ClusterTeam {
    cg::cluster_group cl;
    int nb, bid;
    double *xbuf;
    int pbuf;
    __device__ ClusterTeam(double *xb)
        : cl(cg::this_cluster()), nb((int)cg::this_cluster().num_blocks()),
          bid((int)cg::this_cluster().block_rank()), xbuf(xb), pbuf(0) {}
    __device__ void sync() { cl.sync(); }
    __device__ double *next_part() {
        double *q = xbuf + pbuf * PART_STRIDE;
        pbuf ^= 1;
        return q;
    }
    // out[i] = sum over the cluster's blocks of pt[i], i < nv, in rank order
    __device__ void cluster_sum(double *pt, int nv, double *out) {
        for (int i = threadIdx.x; i < nv; i += blockDim.x) {
            double t[MAX_CLUSTER];
#pragma unroll
            for (int r = 0; r < MAX_CLUSTER; ++r) t[r] = r < nb ? cl.map_shared_rank(pt, r)[i] : 0.0;
            double s = 0.0;
#pragma unroll
            for (int r = 0; r < MAX_CLUSTER; ++r) s += t[r];
            out[i] = s;
        }
        __syncthreads();
    }
    __device__ void sum32(double (&v)[32], int n, SmemFixed &S, double *out, bool active = true) {
        double *pt = next_part();
        block_partials32(v, n, S.red, pt, 1, active, 0);
        cl.sync();
        cluster_sum(pt, n, out);
    }
    template <class Fill>
    __device__ void sum_many(int nv, SmemFixed &S, double *out, Fill fill) {
        double *pt = next_part();
        for (int c0 = 0; c0 < nv; c0 += 32) {
            double v[32];
            fill(c0, v);
            block_partials32(v, min(32, nv - c0), S.red, pt + c0, 1, true, 0);
        }
        cl.sync();
        cluster_sum(pt, nv, out);
    }
};

// Compensated FP32 accumulation of products a*b (TwoProduct with fmaf, TwoSum;
// Ogita, Rump & Oishi 2005): about twice FP32 precision, all on FP32 pipes.
struct Dot2f {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = a * b;
        const float ep = fmaf(a, b, -p);
        const float t = s + p;
        const float bp = t - s;
        const float es = (s - (t - bp)) + (p - bp);
        s = t;
        c += es + ep;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// ---- loaders / stores for the tiled operator ----
template <typename TV, typename TC>
struct LdVec {
    const TV *v;
    TC s;
    __device__ TC operator()(long long i) const { return s * TC(v[i]); }
};
template <typename TV, typename TC>
struct LdEwma {
    const TV *Y;
    const double *x;
    TC rho, om;
    __device__ TC operator()(long long i) const { return rho * TC(Y[i]) + om * TC(x[i]); }
};
template <typename TV, typename TC>
struct StVec {
    TV *y;
    __device__ void operator()(long long i, TC v) const { y[i] = TV(v); }
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

template <class Team, typename TC, int WM, class L, class S>
__device__ inline void team_apply(Team &tm, const Dev &D, const Tiling &tl, void *smem_tiles, L &ld, S &st) {
    TC *sp = reinterpret_cast<TC *>(smem_tiles);
    TC *sq = sp + (size_t)D.P * tl.HW;
    for (int tile = tm.bid; tile < tl.ntiles; tile += tm.nb) apply_tile<TC, WM>(D, tl, tile, sp, sq, ld, st);
}

// out = U^-1 L^-1 in by column-group sweeps; the last barrier is included.
template <class Team, typename TI, typename TIn, int WM>
__device__ inline void team_ilu(Team &tm, const Dev &D, const TIn *in, TI *out) {
    const int lane = threadIdx.x & 31;
    // warp-major numbering: a group with fewer columns than blocks gets one
    // warp on each of as many SMs, instead of all warps of a few SMs sharing
    // their FP64 pipes and load units
    const int gw = (threadIdx.x >> 5) * tm.nb + tm.bid;
    const int nw = tm.nb * NWARPS;
    const int ng = (WM & 3) == 0 ? 4 : D.ngroups;   // periodic grids: the four colours
    if (group_size<WM>(D, 0) > 4 * nw) {
        // large problem: row-parallel coupling gathers, then per-column products
        const long long tid = (long long)tm.bid * NTHREADS + threadIdx.x, nth = (long long)tm.nb * NTHREADS;
        for (int c = 0; c < ng; ++c) {
            const int per = group_size<WM>(D, c);
            const long long rows = (long long)per * D.P;
            for (long long r = tid; r < rows; r += nth) ilu_gather_row<TI, TIn, true, WM>(D, c, r, in, out);
            tm.sync();
            for (int q = gw; q < per; q += nw) ilu_column_product<TI, WM>(D, c, q, out, lane, false);
            tm.sync();
        }
        for (int c = ng - 1; c >= 0; --c) {
            const int per = group_size<WM>(D, c);
            const long long rows = (long long)per * D.P;
            if (c < ng - 1) {
                for (long long r = tid; r < rows; r += nth) ilu_gather_row<TI, TI, false, WM>(D, c, r, out, out);
                tm.sync();
            }
            for (int q = gw; q < per; q += nw) ilu_column_product<TI, WM>(D, c, q, out, lane, true);
            tm.sync();
        }
        return;
    }
    for (int c = 0; c < ng; ++c) {
        const int per = group_size<WM>(D, c);
        for (int q = gw; q < per; q += nw) ilu_fwd_column<TI, TIn, WM>(D, c, q, in, out, lane);
        if (c < ng - 1) tm.sync();
    }
    for (int c = ng - 1; c >= 0; --c) {
        const int per = group_size<WM>(D, c);
        for (int q = gw; q < per; q += nw) ilu_bwd_column<TI, WM>(D, c, q, out, lane);
        tm.sync();
    }
}

// Upper-triangular Cholesky G = R^T R of a k x k matrix by one warp; false on a non-positive pivot.
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

// One warp: solve U z = rhs (U upper k x k); rows with |U_jj| <= tiny give z_j = 0.
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

// One warp: solve U^T w = rhs.
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
// The solve body.
// ---------------------------------------------------------------------------
template <class Team, typename TI, int WM>
__device__ void solve_body(Team &tm, const Dev &D, const SolveArgs &A, SmemFixed &S, void *tiles, double *ph) {
    const long long m = D.m;
    const int nb = tm.nb;
    const int tid = tm.bid * NTHREADS + threadIdx.x;
    const int nth = nb * NTHREADS;
    const int k = A.k;
    TI *V = reinterpret_cast<TI *>(A.V);
    TI *tw = reinterpret_cast<TI *>(A.t);
    double *Yold = A.Yold;
    double *Ynew = A.Ynew;
    double *Wm = A.Wm;
    const bool timer = ph != nullptr && tid == 0;
    double mf = 0.0, mb = 0.0;
    const double md = (double)m;
    auto cost = [&](double f, double b) { mf += f * md; mb += b * md; };
    unsigned long long t_last = timer ? global_ns() : 0ull;
    auto tick = [&](int phase) {
        if (timer) {
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
    geometry_columns(D, A.eta_prev, A.eta_cur, tid, nth);
    tm.sync();
    tick(PH_GEOM);

    // reference norms ||b|| and ||M^-1 b||
    team_ilu<Team, TI, double, WM>(tm, D, A.b, tw);
    {
        double v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.0;
        for (long long p = tid; p < m; p += nth) {
            double bb = A.b[p], tt = (double)tw[p];
            v[0] += bb * bb;
            v[1] += tt * tt;
        }
        tm.sum32(v, 2, S, S.res);
    }
    const double braw = sqrt(S.res[0]);
    const double bnorm = sqrt(S.res[1]);
    cost(A.cm.fM + 4.0, A.cm.bM + 8.0);
    tick(PH_BNORM);

    // ---- a7-a10: initial guess (Algorithm 2) ----
    int guess_rank = -1, shifted = 0;
    if (A.guess_mode == SW_GUESS_RRF) {
        // Algorithm 3: Y = X Omega over the newest solutions, then W = A Y (FP64)
        cost(2.0 * A.ring_Ke * k, (A.ring_Ke + k) * 8.0);
        if (!A.Vq) cost(k * A.cm.fA, k * (A.cm.bA + 8.0));
        for (int c = 0; c < k; ++c) {
            double *Ync = Ynew + (size_t)c * m;
            for (long long p = tid; p < m; p += nth) {
                double s = 0.0;
                for (int r = 0; r < A.ring_Ke; ++r) {
                    const int slot = (A.ring_newest - r + A.ring_K) % A.ring_K;
                    s += A.ring[(size_t)slot * m + p] * A.omega_rrf[r * k + c];
                }
                Ync[p] = s;
            }
        }
        tm.sync();
        if (!A.Vq) {
            for (int c = 0; c < k; ++c) {
                StVec<double, double> st{Wm + (size_t)c * m};
                LdVec<double, double> ld{Ynew + (size_t)c * m, 1.0};
                team_apply<Team, double, WM>(tm, D, A.tl, tiles, ld, st);
            }
            tm.sync();
        }
    } else if (A.pending || A.guess_mode == SW_GUESS_EWMA) {
        // Y_new = r Y_old + x_prev omega^T (Algorithm 4) and W = A Y_new
        const bool upd = A.pending != 0;
        if (upd) cost(3.0 * k, (2.0 * k + 1.0) * 8.0);
        if (A.guess_mode == SW_GUESS_EWMA && !A.Vq) cost(k * A.cm.fA, k * (A.cm.bA + 8.0));
        for (int c = 0; c < k; ++c) {
            const double *Yc = Yold + (size_t)c * m;
            double *Ync = Ynew + (size_t)c * m;
            if (upd)
                for (long long p = tid; p < m; p += nth) Ync[p] = A.decay * Yc[p] + A.omega[c] * A.xprev[p];
            if (A.guess_mode == SW_GUESS_EWMA && !A.Vq) {
                // W = A Y in FP64 (the least squares needs it accurate)
                StVec<double, double> st{Wm + (size_t)c * m};
                if (upd) {
                    LdEwma<double, double> ld{Yc, A.xprev, A.decay, A.omega[c]};
                    team_apply<Team, double, WM>(tm, D, A.tl, tiles, ld, st);
                } else {
                    LdVec<double, double> ld{Yc, 1.0};
                    team_apply<Team, double, WM>(tm, D, A.tl, tiles, ld, st);
                }
            }
        }
        tm.sync();
    }
    const double *Ycur = (A.pending || A.guess_mode == SW_GUESS_RRF) ? Ynew : Yold;
    if (A.Vq && (A.guess_mode == SW_GUESS_EWMA || A.guess_mode == SW_GUESS_RRF)) {
        // the optional QR step of Algorithms 3 and 4: V = Y R^-1 with R from CholeskyQR2 of Y
        // (shifted Cholesky when Y^T Y is not numerically SPD), then W = A V
        const int ng = k * (k + 1) / 2;
        cost(2.0 * ng + (double)k * k + 2.0 * ng + (double)k * k, 3.0 * k * 8.0 + k * 8.0);
        cost(k * A.cm.fA, k * (A.cm.bA + 8.0));
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1 && !S.flags[0]) break;
            tm.sum_many(ng, S, S.res, [&](int c0, double (&v)[32]) {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.0;
                for (long long p = tid; p < m; p += nth) {
                    double q[MAX_K];
#pragma unroll
                    for (int c = 0; c < MAX_K; ++c) {
                        if (c >= k) { q[c] = 0.0; continue; }
                        double sv = Ycur[(size_t)c * m + p];
                        if (pass == 1) {
                            for (int i = 0; i < c; ++i) sv -= q[i] * S.R1[i * k + c];
                            sv /= S.R1[c * k + c];
                        }
                        q[c] = sv;
                    }
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int e = c0 + i;
                        if (e >= ng) break;
                        v[i] += q[S.ga[e]] * q[S.gb[e]];
                    }
                }
            });
            if (threadIdx.x < 32) {
                for (int e = threadIdx.x; e < ng; e += 32) {
                    S.G[S.ga[e] * k + S.gb[e]] = S.res[e];
                    S.G[S.gb[e] * k + S.ga[e]] = S.res[e];
                }
                __syncwarp();
                if (pass == 0) {
                    double tr = 0.0;
                    for (int c = 0; c < k; ++c) tr += S.G[c * k + c];
                    for (int i = threadIdx.x; i < k * k; i += 32) S.R[i] = S.G[i];
                    __syncwarp();
                    bool ok = tr > 0.0 && warp_cholesky(S.G, S.R1, k);
                    if (!ok && tr > 0.0) {
                        double sh = 11.0 * ((double)m * k + (double)k * (k + 1)) * 1.1102230246251565e-16 * tr;
                        for (int i = threadIdx.x; i < k * k; i += 32) S.G[i] = S.R[i] + ((i / k == i % k) ? sh : 0.0);
                        __syncwarp();
                        ok = warp_cholesky(S.G, S.R1, k);
                    }
                    // R = R1 unless the second pass refines it
                    for (int i = threadIdx.x; i < k * k; i += 32) S.R[i] = S.R1[i];
                    if (threadIdx.x == 0) S.flags[0] = ok ? 1 : 0;
                } else if (warp_cholesky(S.G, S.R2, k)) {
                    for (int e = threadIdx.x; e < k * k; e += 32) {
                        int a = e / k, bc = e % k;
                        double sv = 0.0;
                        for (int l = a; l <= bc; ++l) sv += S.R2[a * k + l] * S.R1[l * k + bc];
                        S.R[e] = bc >= a ? sv : 0.0;
                    }
                }
            }
            __syncthreads();
        }
        // V = Y R^-1, or V = Y when the Gram matrix is zero or not factorable
        const bool ok = S.flags[0] != 0;
        for (long long p = tid; p < m; p += nth) {
            double q[MAX_K];
#pragma unroll
            for (int c = 0; c < MAX_K; ++c) {
                if (c >= k) break;
                double sv = Ycur[(size_t)c * m + p];
                if (ok) {
                    for (int i = 0; i < c; ++i) sv -= q[i] * S.R[i * k + c];
                    sv /= S.R[c * k + c];
                }
                q[c] = sv;
                A.Vq[(size_t)c * m + p] = sv;
            }
        }
        tm.sync();
        for (int c = 0; c < k; ++c) {
            StVec<double, double> st{Wm + (size_t)c * m};
            LdVec<double, double> ld{A.Vq + (size_t)c * m, 1.0};
            team_apply<Team, double, WM>(tm, D, A.tl, tiles, ld, st);
        }
        tm.sync();
        Ycur = A.Vq;
    }
    tick(PH_GUESS_W);
    if (A.guess_mode == SW_GUESS_EWMA || A.guess_mode == SW_GUESS_RRF) {
        // Gram G = W^T W and c = W^T b (a8)
        const int ng = k * (k + 1) / 2;
        const int nv = ng + k;
        cost(2.0 * nv, (k + 1.0) * 8.0);
        tm.sum_many(nv, S, S.res, [&](int c0, double (&v)[32]) {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = 0.0;
            for (long long p = tid; p < m; p += nth) {
                double wv[MAX_K];
#pragma unroll
                for (int c = 0; c < MAX_K; ++c) wv[c] = c < k ? (double)Wm[(size_t)c * m + p] : 0.0;
                const double bp = A.b[p];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int e = c0 + i;
                    if (e >= nv) break;
                    v[i] += e < ng ? wv[S.ga[e]] * wv[S.gb[e]] : wv[e - ng] * bp;
                }
            }
        });
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
            for (int i = threadIdx.x; i < k * k; i += 32) S.R[i] = S.G[i];
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
        if (S.flags[0]) {
            // second pass: Q1 = W R1^-1, G2 = Q1^T Q1, c2 = Q1^T b
            cost((double)k * k + 2.0 * nv, (k + 1.0) * 8.0);
            tm.sum_many(nv, S, S.res, [&](int c0, double (&v)[32]) {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.0;
                for (long long p = tid; p < m; p += nth) {
                    double q[MAX_K];
#pragma unroll
                    for (int c = 0; c < MAX_K; ++c) {
                        if (c >= k) { q[c] = 0.0; continue; }
                        double s = (double)Wm[(size_t)c * m + p];
                        for (int i = 0; i < c; ++i) s -= q[i] * S.R1[i * k + c];
                        q[c] = s / S.R1[c * k + c];
                    }
                    const double bp = A.b[p];
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int e = c0 + i;
                        if (e >= nv) break;
                        v[i] += e < ng ? q[S.ga[e]] * q[S.gb[e]] : q[e - ng] * bp;
                    }
                }
            });
            if (threadIdx.x < 32) {
                for (int e = threadIdx.x; e < ng; e += 32) {
                    S.G[S.ga[e] * k + S.gb[e]] = S.res[e];
                    S.G[S.gb[e] * k + S.ga[e]] = S.res[e];
                }
                for (int c = threadIdx.x; c < k; c += 32) S.c2[c] = S.res[ng + c];
                __syncwarp();
                bool ok2 = warp_cholesky(S.G, S.R2, k);
                if (!ok2) {
                    // Q1 far from orthonormal: use R = R1 and Q^T b = R1^-T W^T b
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
                // rank guard: drop columns with |R_jj| <= 1e-12 |R_00|
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
        cost(2.0 * k, k * 8.0 + 8.0);
        for (long long p = tid; p < m; p += nth) {
            double s = 0.0;
            for (int c = 0; c < k; ++c) s += Ycur[(size_t)c * m + p] * S.z[c];
            A.x[p] = s;
        }
    } else if (A.guess_mode == SW_GUESS_PREVIOUS) {
        cost(0.0, 16.0);
        for (long long p = tid; p < m; p += nth) A.x[p] = A.xprev[p];
    } else {
        for (long long p = tid; p < m; p += nth) A.x[p] = 0.0;
    }
    tm.sync();
    tick(PH_GUESS_LS);
    if (A.guess_only) {
        if (tid == 0) {
            A.stats->guess_rank = guess_rank;
            A.stats->cholesky_shift = shifted;
        }
        return;
    }

    // ---- restarted GMRES(m), left-preconditioned (Sec. 3) ----
    int iters = 0, restarts = 0, converged = 0, status = SW_ERR_NOT_CONVERGED;
    double res0 = 0.0, res_last = 0.0, guess_res = 0.0;
    const int mr = A.restart;
    const int wlane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // Gram-Schmidt point mapping: warp w of team block b takes 32-point chunks
    // b + nb w, b + nb (w + NWARPS), ... so that the warps holding data are
    // spread over blocks and sub-partitions
    const long long k0 = tm.bid + (long long)nb * wid, kstep = (long long)nb * NWARPS;
    const bool wactive = 32 * k0 < m;
    if (bnorm == 0.0) {
        for (long long p = tid; p < m; p += nth) A.x[p] = 0.0;
        converged = 1;
        status = SW_OK;
    } else {
        for (int cycle = 0;; ++cycle) {
            // r = b - A x (FP64) ; V0 = M^-1 r
            {
                StResid st{A.b, A.r, 0.0};
                LdVec<double, double> ld{A.x, 1.0};
                team_apply<Team, double, WM>(tm, D, A.tl, tiles, ld, st);
                double v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.0;
                v[0] = st.acc;
                tm.sync();
                tick(PH_RES_APPLY);
                team_ilu<Team, TI, double, WM>(tm, D, A.r, V);
                for (long long p = tid; p < m; p += nth) {
                    const double vv = (double)V[p];
                    v[1] += vv * vv;
                }
                tm.sum32(v, 2, S, S.res);
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
            const double inner_stop = fmax(A.tol * bnorm, A.inner_rtol * beta);
            if (threadIdx.x == 0) {
                S.scale[0] = 1.0 / beta;
                for (int i = 0; i <= mr; ++i) S.g[i] = 0.0;
                S.g[0] = beta;
            }
            __syncthreads();
            int jend = 0;
            for (int j = 0; j < mr; ++j) {
                TI *w = V + (size_t)(j + 1) * m;
                // w = M^-1 A v_j  (v_j = scale_j V_j)
                {
                    LdVec<TI, TI> ld{V + (size_t)j * m, TI(S.scale[j])};
                    StVec<TI, TI> st{tw};
                    team_apply<Team, TI, WM>(tm, D, A.tl, tiles, ld, st);
                    tm.sync();
                    tick(PH_ARN_APPLY);
                    team_ilu<Team, TI, TI, WM>(tm, D, tw, w);
                    tick(PH_ARN_ILU);
                }
                // CGS2 pass 1: d_i = V_i . w
                double v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.0;
                if constexpr (sizeof(TI) == 4) {
                    Dot2f acc[32];
                    for (long long kc = k0; 32 * kc < m; kc += kstep) {
                        const long long p = 32 * kc + wlane;
                        if (p >= m) continue;
                        float vb[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i) vb[i] = i <= j ? (float)V[(size_t)i * m + p] : 0.f;
                        const float wv = (float)w[p];
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            if (i > j) break;
                            acc[i].add(vb[i], wv);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        if (i > j) break;
                        v[i] = acc[i].value();
                    }
                } else {
                    for (long long kc = k0; 32 * kc < m; kc += kstep) {
                        const long long p = 32 * kc + wlane;
                        if (p >= m) continue;
                        double vb[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i) vb[i] = i <= j ? (double)V[(size_t)i * m + p] : 0.0;
                        const double wv = (double)w[p];
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            if (i > j) break;
                            v[i] += vb[i] * wv;
                        }
                    }
                }
                tm.sum32(v, j + 1, S, S.res, wactive);
                tick(PH_CGS1);
                if (threadIdx.x < MAX_RESTART) {
                    const int i = threadIdx.x;
                    const double hi = i <= j ? S.res[i] * S.scale[i] : 0.0;
                    if (i <= j) S.H[i * MAX_RESTART + j] = hi;
                    S.hs[i] = i <= j ? hi * S.scale[i] : 0.0;
                    S.hs32[i] = (float)S.hs[i];
                }
                __syncthreads();
                // pass 2: w -= V h ; d'_i = V_i . w
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.0;
                if constexpr (sizeof(TI) == 4) {
                    Dot2f acc[32];
                    for (long long kc = k0; 32 * kc < m; kc += kstep) {
                        const long long p = 32 * kc + wlane;
                        if (p >= m) continue;
                        float vb[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i) vb[i] = i <= j ? (float)V[(size_t)i * m + p] : 0.f;
                        float wv = (float)w[p];
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            if (i > j) break;
                            wv = fmaf(-S.hs32[i], vb[i], wv);
                        }
                        w[p] = TI(wv);
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            if (i > j) break;
                            acc[i].add(vb[i], wv);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        if (i > j) break;
                        v[i] = acc[i].value();
                    }
                } else {
                    for (long long kc = k0; 32 * kc < m; kc += kstep) {
                        const long long p = 32 * kc + wlane;
                        if (p >= m) continue;
                        double vb[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i) vb[i] = i <= j ? (double)V[(size_t)i * m + p] : 0.0;
                        double wv = (double)w[p];
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            if (i > j) break;
                            wv -= S.hs[i] * vb[i];
                        }
                        w[p] = TI(wv);
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            if (i > j) break;
                            v[i] += vb[i] * wv;
                        }
                    }
                }
                tm.sum32(v, j + 1, S, S.res, wactive);
                tick(PH_CGS2);
                if (threadIdx.x < MAX_RESTART) {
                    const int i = threadIdx.x;
                    const double hi = i <= j ? S.res[i] * S.scale[i] : 0.0;
                    if (i <= j) S.H[i * MAX_RESTART + j] += hi;
                    S.hs[i] = i <= j ? hi * S.scale[i] : 0.0;
                    S.hs32[i] = (float)S.hs[i];
                }
                __syncthreads();
                // pass 3: w -= V h' ; ||w||^2
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.0;
                if constexpr (sizeof(TI) == 4) {
                    Dot2f acc;
                    for (long long kc = k0; 32 * kc < m; kc += kstep) {
                        const long long p = 32 * kc + wlane;
                        if (p >= m) continue;
                        float vb[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i) vb[i] = i <= j ? (float)V[(size_t)i * m + p] : 0.f;
                        float wv = (float)w[p];
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            if (i > j) break;
                            wv = fmaf(-S.hs32[i], vb[i], wv);
                        }
                        w[p] = TI(wv);
                        acc.add(wv, wv);
                    }
                    v[0] = acc.value();
                } else {
                    for (long long kc = k0; 32 * kc < m; kc += kstep) {
                        const long long p = 32 * kc + wlane;
                        if (p >= m) continue;
                        double vb[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i) vb[i] = i <= j ? (double)V[(size_t)i * m + p] : 0.0;
                        double wv = (double)w[p];
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            if (i > j) break;
                            wv -= S.hs[i] * vb[i];
                        }
                        w[p] = TI(wv);
                        v[0] += wv * wv;
                    }
                }
                tm.sum32(v, 1, S, S.res, wactive);
                tick(PH_CGS3);
                // a5: Hessenberg column, Givens rotations, residual estimate
                if (threadIdx.x == 0) {
                    const double hn = sqrt(S.res[0]);
                    S.scale[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
                    double *Hc = S.H;
                    for (int i = 0; i < j; ++i) {
                        const double a = Hc[i * MAX_RESTART + j], bb = Hc[(i + 1) * MAX_RESTART + j];
                        Hc[i * MAX_RESTART + j] = S.cs[i] * a + S.sn[i] * bb;
                        Hc[(i + 1) * MAX_RESTART + j] = -S.sn[i] * a + S.cs[i] * bb;
                    }
                    const double a = Hc[j * MAX_RESTART + j];
                    const double den = hypot(a, hn);
                    S.cs[j] = a / den;
                    S.sn[j] = hn / den;
                    Hc[j * MAX_RESTART + j] = den;
                    S.g[j + 1] = -S.sn[j] * S.g[j];
                    S.g[j] = S.cs[j] * S.g[j];
                    S.flags[2] = (fabs(S.g[j + 1]) <= inner_stop) || hn == 0.0;
                }
                __syncthreads();
                tick(PH_GIVENS);
                cost(A.cm.fA + A.cm.fM + 8.0 * (j + 1) + 2.0,
                     A.cm.bA + A.cm.bM + (3.0 * j + 8.0) * (double)sizeof(TI));
                ++iters;
                jend = j + 1;
                if (S.flags[2]) break;
            }
            // a6: y = R^-1 g, x += V (scale y) in FP64
            if (threadIdx.x < 32) {
                const int lane = threadIdx.x;
                double acc = lane < jend ? S.g[lane] : 0.0;
                for (int i = jend - 1; i >= 0; --i) {
                    const double yi = __shfl_sync(0xffffffffu, acc, i) / S.H[i * MAX_RESTART + i];
                    if (lane == i) S.y[i] = yi * S.scale[i];
                    if (lane < i) acc -= S.H[lane * MAX_RESTART + i] * yi;
                }
            }
            __syncthreads();
            cost(2.0 * jend, jend * (double)sizeof(TI) + 16.0);
            for (long long p = tid; p < m; p += nth) {
                double s = A.x[p];
                for (int i = 0; i < jend; ++i) s += S.y[i] * (double)V[(size_t)i * m + p];
                A.x[p] = s;
            }
            tm.sync();
            tick(PH_UPDATE);
        }
    }
    // true residual ||b - A x|| / ||b|| in FP64; the solution is kept for the next guess
    double true_res;
    {
        StResid st{A.b, A.r, 0.0};
        LdVec<double, double> ld{A.x, 1.0};
        team_apply<Team, double, WM>(tm, D, A.tl, tiles, ld, st);
        double v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.0;
        v[0] = st.acc;
        for (long long p = tid; p < m; p += nth) {
            A.xprev[p] = A.x[p];
            if (A.ring_store) A.ring_store[p] = A.x[p];
        }
        tm.sum32(v, 1, S, S.res);
        true_res = braw > 0.0 ? sqrt(S.res[0]) / braw : sqrt(S.res[0]);
        cost(A.cm.fA + 3.0, A.cm.bA + 24.0);
    }
    tick(PH_TRUERES);
    if (tid == 0) {
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
        if (ph)
            for (int i = 0; i < PH_COUNT; ++i) st.phase_ns[i] += ph[i];
    }
}

}  // namespace sw
