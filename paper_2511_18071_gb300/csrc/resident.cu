// The Poisson solve of one stage for small two-dimensional periodic problems,
// with every vector and constant of the solve resident in shared memory (the
// resident executor).
//
// Same algorithm, in the same order, as the persistent solve kernel
// (sw_solve.cuh): reference norms, the subspace guess of Algorithm 2 (the EWMA
// sketch of Algorithm 4 or the range finder of Algorithm 3; W = A Y, Gram,
// CholeskyQR2 with the shifted fallback and the rank guard, x0 = Y z), then
// restarted GMRES left-preconditioned with the fixed ILU(0) factors (Sec. 3).
// The difference is where the data live and how the blocks synchronise:
//
//  - block b owns the C consecutive columns [bC, bC + C) (C a multiple of 4,
//    so one column per colour in every group of four), all levels; its slab
//    of every vector (Krylov basis, sketch, W, x, b, r) and its constants
//    (the off-column ILU factors and the inverses of its columns' in-column
//    blocks) stay in shared memory for the whole solve;
//  - the operator and the ILU colour sweeps couple a column only to columns at
//    most three away, i.e. to the two neighbouring blocks: before every sweep
//    and apply that needs them, a block publishes its three leftmost and three
//    rightmost columns in a mailbox in global memory, raises its sequence flag
//    and waits for its two neighbours' flags, instead of a grid barrier;
//  - inner products are all-reduced: every block writes its partial sums,
//    counts itself in with one atomic, waits until every block has, and sums
//    the partials in a fixed order (so every block holds bit-identical values
//    and takes the same decisions);
//  - the Gram-Schmidt step takes two all-reduces instead of three: the second
//    pass returns the projections and ||w||^2 together, and the norm of the
//    twice-orthogonalised vector is ||w||^2 - ||h'||^2 (V orthonormal), with a
//    direct third reduction when that difference loses accuracy.
//
// Every wait is bounded (R_WAIT_NS of device time, checked against the global
// timer); a wait that runs out sets a shared abort flag that makes every other
// wait give up too, and the solve returns SW_ERR_TIMEOUT.
#include <cmath>
#include <cstring>
#include <vector>

#include "sw_solve.cuh"

namespace sw {

constexpr unsigned long long R_WAIT_NS = 2000000000ull;   // 2 s

// Device description of the resident layout of one problem.
struct ResDev {
    int C, NB, nl, nlp, mv, blob, noff;
    int stall;             // testing aid: from this exchange on, block 0 withholds its flag (-1: never)
    const double *cblob;   // NB x blob: off-column factors fac[i][l][cx], then Linv and Uinv of the block's columns
    double *mail;          // 2 x NB x mv x P x 6 boundary columns
    unsigned *sync;        // [0] all-reduce arrivals, [1] abort, [2 + b] exchange flag of block b
    double *part;          // 2 x NB x PART_STRIDE partial sums
};

__device__ __forceinline__ unsigned r_ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until *a >= target and *b >= target (thread 0 only).  False when the
// bound runs out (the abort flag is then raised) or another block aborted.
__device__ inline bool r_wait_ge(const unsigned *a, const unsigned *b, unsigned target, unsigned *abortp) {
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (r_ld_acquire(a) >= target && r_ld_acquire(b) >= target) return true;
        if ((it & 31) == 0) {
            if (r_ld_acquire(abortp)) return false;
            if (global_ns() - t0 > R_WAIT_NS) {
                atomicExch(abortp, 1u);
                return false;
            }
        }
    }
}

// Per-block view of the solve's shared memory and synchronisation state.
struct RCtx {
    int b, bl, br, C, P, nl, nlp, HX, NB;
    unsigned seq, round;
    double *fac, *linv, *uinv;          // constants
    double *V, *t, *x, *bb, *r, *xp;    // vectors (nlp stride between Krylov vectors)
    double *Y, *Wm, *halo, *sp, *sq, *cc, *ws1, *ws2;
    int *win;
};

// ---- exchange of boundary columns with the two neighbouring blocks ----------

// Publish the three leftmost and three rightmost columns of nv local vectors
// (vector c at vec + c * stride) and fill halo[c][l][0..5] with the left
// neighbour's three rightmost and the right neighbour's three leftmost columns.
__device__ bool r_exchange(RCtx &X, const ResDev &R, SmemFixed &S, const double *vec, int stride, int nv) {
    const int P = X.P, C = X.C, n6 = P * 6;
    X.seq++;
    const int par = X.seq & 1;
    double *mine = R.mail + ((size_t)(par * X.NB + X.b) * R.mv) * n6;
    for (int i = threadIdx.x; i < nv * n6; i += NTHREADS) {
        const int c = i / n6, rr = i - c * n6, l = rr / 6, e = rr - l * 6;
        mine[i] = vec[(size_t)c * stride + l * C + (e < 3 ? e : C - 6 + e)];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (!(X.b == 0 && R.stall > 0 && (int)X.seq >= R.stall)) atomicExch(R.sync + 2 + X.b, X.seq);
        S.flags[7] = r_wait_ge(R.sync + 2 + X.bl, R.sync + 2 + X.br, X.seq, R.sync + 1) ? 1 : 0;
    }
    __syncthreads();
    if (!S.flags[7]) return false;
    const double *ml = R.mail + ((size_t)(par * X.NB + X.bl) * R.mv) * n6;
    const double *mr = R.mail + ((size_t)(par * X.NB + X.br) * R.mv) * n6;
    for (int i = threadIdx.x; i < nv * n6; i += NTHREADS) {
        const int e = i % 6;
        X.halo[i] = e < 3 ? __ldcg(ml + i + 3) : __ldcg(mr + i - 3);
    }
    __syncthreads();
    return true;
}

// ---- all-reduce of block partial sums ----------------------------------------

// out[v] = sum over blocks of bp[v] (v < nv <= PART_STRIDE), summed in the same
// order by every block.  bp is in shared memory; out may be S.res.
__device__ bool r_allreduce(RCtx &X, const ResDev &R, SmemFixed &S, const double *bp, int nv, double *out) {
    const int par = X.round & 1;
    double *mine = R.part + (size_t)(par * X.NB + X.b) * PART_STRIDE;
    for (int i = threadIdx.x; i < nv; i += NTHREADS) mine[i] = bp[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(R.sync, 1u);
        const unsigned target = (X.round + 1) * (unsigned)X.NB;
        S.flags[7] = r_wait_ge(R.sync, R.sync, target, R.sync + 1) ? 1 : 0;
    }
    X.round++;
    __syncthreads();
    if (!S.flags[7]) return false;
    const double *pp = R.part + (size_t)par * X.NB * PART_STRIDE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v0 = 0; v0 < nv; v0 += 32) {
        const int v = v0 + lane;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        if (v < nv) {
            int bq = warp;
            for (; bq + 3 * NWARPS < X.NB; bq += 4 * NWARPS) {
                a0 += __ldcg(pp + (size_t)bq * PART_STRIDE + v);
                a1 += __ldcg(pp + (size_t)(bq + NWARPS) * PART_STRIDE + v);
                a2 += __ldcg(pp + (size_t)(bq + 2 * NWARPS) * PART_STRIDE + v);
                a3 += __ldcg(pp + (size_t)(bq + 3 * NWARPS) * PART_STRIDE + v);
            }
            for (; bq < X.NB; bq += NWARPS) a0 += __ldcg(pp + (size_t)bq * PART_STRIDE + v);
        }
        S.red[warp * 32 + lane] = (a0 + a1) + (a2 + a3);
        __syncthreads();
        if (warp == 0 && v < nv) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < NWARPS; ++w) s += S.red[w * 32 + lane];
            out[v] = s;
        }
        __syncthreads();
    }
    return true;
}

// ---- block partial sums -------------------------------------------------------

// bp[i] = sum over the block's points of f(p, i), i < nv <= 4 (norms).
template <class F>
__device__ void r_block_sums(const RCtx &X, SmemFixed &S, int nv, F f, double *bp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool active = warp * 32 < X.nl;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (active) {
        for (int p = threadIdx.x; p < X.nl; p += NTHREADS) f(p, v);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i >= nv) break;
            double s = v[i];
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            v[i] = s;
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) S.red[warp * 32 + i] = active && i < nv ? v[i] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        double s = 0.0;
        for (int w = 0; w < NWARPS; ++w) s += S.red[w * 32 + threadIdx.x];
        bp[threadIdx.x] = s;
    }
    __syncthreads();
}

// bp[i] = V_i . w over the block's points, i < nv <= 32 (lane = i, warps take
// slices of the points), plus bp[nv] = w . w when with_norm.
__device__ void r_block_dots(const RCtx &X, SmemFixed &S, int nv, const double *w, bool with_norm, double *bp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pw = (X.nl + NWARPS - 1) / NWARPS;
    const int p0 = warp * pw, p1 = min(X.nl, p0 + pw);
    double a = 0.0;
    const int nval = nv + (with_norm ? 1 : 0);
    if (lane < nval) {
        const double *vv = lane < nv ? X.V + (size_t)lane * X.nlp : w;
        for (int p = p0; p < p1; ++p) a += vv[p] * w[p];
    }
    S.red[warp * 32 + lane] = a;
    __syncthreads();
    if (warp == 0 && lane < nval) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < NWARPS; ++q) s += S.red[q * 32 + lane];
        bp[lane] = s;
    }
    __syncthreads();
}

// ---- operator apply on the block's slab -------------------------------------

// The value of a local vector at level index l and block column xe in
// [-3, C + 3): own columns from the slab, the others from the halo.
__device__ __forceinline__ double r_ext(const RCtx &X, const double *vec, const double *halo, int l, int xe) {
    if (xe < 0) return halo[l * 6 + xe + 3];
    if (xe >= X.C) return halo[l * 6 + xe - X.C + 3];
    return vec[l * X.C + xe];
}

// y = A (s vec) on the block's columns (Eq. 16-18), vec's halo in `halo`;
// with resid, y = bb - A vec and the block's sum of y^2 is returned (thread 0).
__device__ double r_apply(const RCtx &X, const Dev &D, const double *vec, const double *halo, double s, double *y,
                          bool resid) {
    const int P = X.P, C = X.C, HX = X.HX, HW = HX;
    for (int i = threadIdx.x; i < P * HX; i += NTHREADS) {
        const int l = i / HX, a = i - l * HX;
        X.sp[i] = s * r_ext(X, vec, halo, l, a - HALF);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P * HX; i += NTHREADS) {
        const int l = i / HX, a = i - l * HX;
        const double *w1 = X.ws1 + l * W;
        const int base = (X.win[l] + 1) * HW + a;
        double sv = 0.0;
#pragma unroll
        for (int k = 0; k < W; ++k) sv += w1[k] * X.sp[base + k * HW];
        X.sq[i] = sv;
    }
    __syncthreads();
    const double inv_nzm1 = 1.0 / (double)(D.nz - 1);
    const double *wx1 = D.wx1, *wx2 = D.wx2;
    double acc = 0.0;
    for (int i = threadIdx.x; i < P * C; i += NTHREADS) {
        const int l = i / C, cx = i - l * C;
        const int hr = cx + HALF;
        const double *cc = X.cc;
        double yv;
        if (l == P - 1) {
            yv = X.sp[l * HW + hr];
        } else if (l == 0) {
            double px = 0.0;
#pragma unroll
            for (int t = -HALF; t <= HALF; ++t) px += wx1[t + HALF] * X.sp[HW + hr + t];
            yv = cc[CC_GS * C + cx] * X.sq[HW + hr] + cc[CC_GX * C + cx] * px;
        } else {
            const double sg = (double)(l - 1) * inv_nzm1;
            const double ap1 = cc[CC_AP1 * C + cx];
            const double aa = cc[CC_AP0 * C + cx] - sg * ap1;
            const double bbv = cc[CC_BP0 * C + cx] - sg * cc[CC_BP1 * C + cx];
            const double ax = cc[CC_AXP0 * C + cx] - sg * cc[CC_AXP1 * C + cx] - aa * ap1;
            const double c_xs = aa + bbv;
            const double c_ss = aa * bbv + cc[CC_EF * C + cx];
            const double c_s = ax - bbv * ap1;
            const double *pl = X.sp + l * HW + hr;
            const double *ql = X.sq + l * HW + hr;
            double pxx = 0.0, pxs = 0.0;
#pragma unroll
            for (int t = -HALF; t <= HALF; ++t) {
                pxx += wx2[t + HALF] * pl[t];
                pxs += wx1[t + HALF] * ql[t];
            }
            const double *w2 = X.ws2 + l * W;
            const double *pc = X.sp + (X.win[l] + 1) * HW + hr;
            double pss = 0.0;
#pragma unroll
            for (int k = 0; k < W; ++k) pss += w2[k] * pc[k * HW];
            yv = pxx + c_xs * pxs + c_s * ql[0];
            yv += c_ss * pss;
        }
        if (resid) {
            const double tv = X.bb[i] - yv;
            y[i] = tv;
            acc += tv * tv;
        } else {
            y[i] = yv;
        }
    }
    __syncthreads();
    return acc;
}

// ---- ILU(0) colour sweeps on the block's slab -------------------------------

// Sum over the off-column factor slots of column cx (colour CC) whose
// neighbour colour is below (LOWER) or above CC, neighbours from `out` and its halo.
template <int L, bool LOWER, int CC>
__device__ __forceinline__ double r_offsum(const RCtx &X, const double *out, int cx, int l) {
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < Off<L>::N; ++i) {
        const int ox = Off<L>::ox(i);
        const int nc = (CC + ox) & 3;
        if (LOWER ? (nc >= CC) : (nc <= CC)) continue;
        const int lev = Off<L>::kk(i) < 0 ? l : X.win[l] + 1 + Off<L>::kk(i);
        acc += X.fac[((size_t)i * X.P + l) * X.C + cx] * r_ext(X, out, X.halo, lev, cx + ox);
    }
    return acc;
}

// forward sweep of colour CC: out = Linv (in - lower couplings); with UP, the
// backward sweep of the same colour follows at once (the last colour)
template <int L, int CC, bool UP>
__device__ void r_fwd(const RCtx &X, const double *in, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = warp; 4 * q + CC < X.C; q += NWARPS) {
        const int cx = 4 * q + CC;
        double g[2], y[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int l = lane + 32 * h;
            g[h] = l < X.P ? in[l * X.C + cx] - r_offsum<L, true, CC>(X, out, cx, l) : 0.0;
        }
        column_block_product<double>(X.linv + (size_t)cx * X.P * X.P, g, y, X.P, lane);
        if (UP) {
            double z[2];
            column_block_product<double>(X.uinv + (size_t)cx * X.P * X.P, y, z, X.P, lane);
            y[0] = z[0];
            y[1] = z[1];
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (lane + 32 * h < X.P) out[(lane + 32 * h) * X.C + cx] = y[h];
    }
    __syncthreads();
}

template <int L, int CC>
__device__ void r_bwd(const RCtx &X, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = warp; 4 * q + CC < X.C; q += NWARPS) {
        const int cx = 4 * q + CC;
        double g[2], y[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int l = lane + 32 * h;
            g[h] = l < X.P ? out[l * X.C + cx] - r_offsum<L, false, CC>(X, out, cx, l) : 0.0;
        }
        __syncwarp();
        column_block_product<double>(X.uinv + (size_t)cx * X.P * X.P, g, y, X.P, lane);
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (lane + 32 * h < X.P) out[(lane + 32 * h) * X.C + cx] = y[h];
    }
    __syncthreads();
}

// out = U^-1 L^-1 in: four forward colours, four backward colours (the last
// forward and first backward colour together), six boundary exchanges.
template <int L>
__device__ bool r_ilu(RCtx &X, const ResDev &R, SmemFixed &S, const double *in, double *out) {
    r_fwd<L, 0, false>(X, in, out);
    if (!r_exchange(X, R, S, out, 0, 1)) return false;
    r_fwd<L, 1, false>(X, in, out);
    if (!r_exchange(X, R, S, out, 0, 1)) return false;
    r_fwd<L, 2, false>(X, in, out);
    if (!r_exchange(X, R, S, out, 0, 1)) return false;
    r_fwd<L, 3, true>(X, in, out);
    if (!r_exchange(X, R, S, out, 0, 1)) return false;
    r_bwd<L, 2>(X, out);
    if (!r_exchange(X, R, S, out, 0, 1)) return false;
    r_bwd<L, 1>(X, out);
    if (!r_exchange(X, R, S, out, 0, 1)) return false;
    r_bwd<L, 0>(X, out);
    return true;
}

// ---- the solve ----------------------------------------------------------------

template <int L>
__global__ void __launch_bounds__(NTHREADS, 1) resident_kernel(Dev D, SolveArgs A, ResDev R) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemFixed &S = *reinterpret_cast<SmemFixed *>(smem_raw);
    double *base = reinterpret_cast<double *>(smem_raw + ((sizeof(SmemFixed) + 255) & ~size_t(255)));
    const int tid = threadIdx.x;
    const int k = A.k, mr = A.restart;
    RCtx X;
    X.b = blockIdx.x;
    X.NB = R.NB;
    X.bl = X.b == 0 ? R.NB - 1 : X.b - 1;
    X.br = X.b == R.NB - 1 ? 0 : X.b + 1;
    X.C = R.C;
    X.P = D.P;
    X.nl = R.nl;
    X.nlp = R.nlp;
    X.HX = R.C + 2 * HALF;
    X.seq = 0;
    X.round = 0;
    const int C = X.C, P = X.P, nl = X.nl, nlp = X.nlp;
    const int noff = R.noff;
    // shared-memory carve-out (doubles)
    double *q = base;
    X.fac = q; q += (size_t)noff * nl;
    X.linv = q; q += (size_t)C * P * P;
    X.uinv = q; q += (size_t)C * P * P;
    X.V = q; q += (size_t)(mr + 1) * nlp;
    X.t = q; q += nlp;
    X.x = q; q += nlp;
    X.bb = q; q += nlp;
    X.r = q; q += nlp;
    X.xp = q; q += nlp;
    X.Y = q; q += (size_t)k * nl;
    X.Wm = q; q += (size_t)k * nl;
    X.halo = q; q += (size_t)R.mv * P * 6;
    X.sp = q; q += (size_t)P * X.HX;
    X.sq = q; q += (size_t)P * X.HX;
    X.cc = q; q += (size_t)NCC * C;
    X.ws1 = q; q += (size_t)P * W;
    X.ws2 = q; q += (size_t)P * W;
    X.win = reinterpret_cast<int *>(q);
    double *bp = S.xchg;   // block partial sums
    const long long col0 = (long long)X.b * C;
    const long long m = D.m;
    const bool timer = X.b == 0 && tid == 0;
    double ph[PH_COUNT];
    for (int i = 0; i < PH_COUNT; ++i) ph[i] = 0.0;
    unsigned long long t_last = timer ? global_ns() : 0ull;
    auto tick = [&](int phase) {
        if (timer) {
            const unsigned long long tn = global_ns();
            ph[phase] += (double)(tn - t_last);
            t_last = tn;
        }
    };
    double mf = 0.0, mb = 0.0;
    const double md = (double)m;
    auto cost = [&](double f, double bq) { mf += f * md; mb += bq * md; };
    // global index of local point i = l * C + cx
    auto gidx = [&](int i) { const int l = i / C; return (long long)l * D.ncol + col0 + (i - l * C); };

    // constants, weights, b and the previous solution into shared memory
    {
        const double *cb = R.cblob + (size_t)X.b * R.blob;
        for (int i = tid; i < R.blob; i += NTHREADS) X.fac[i] = __ldg(cb + i);
        for (int i = tid; i < P * W; i += NTHREADS) { X.ws1[i] = D.ws1[i]; X.ws2[i] = D.ws2[i]; }
        for (int i = tid; i < P; i += NTHREADS) X.win[i] = D.win[i];
        for (int i = tid; i < nl; i += NTHREADS) {
            const long long g = gidx(i);
            X.bb[i] = A.b[g];
            X.xp[i] = A.xprev[g];
        }
        if (tid == 0) {
            int e = 0;
            for (int a = 0; a < k; ++a)
                for (int b2 = a; b2 < k; ++b2, ++e) { S.ga[e] = (unsigned char)a; S.gb[e] = (unsigned char)b2; }
        }
        // a1: geometry of the block's columns
        for (int cx = tid; cx < C; cx += NTHREADS) {
            double v[NCC];
            column_coefs(D, A.eta_prev, A.eta_cur, (int)(col0 + cx), v);
            for (int kk = 0; kk < NCC; ++kk) X.cc[kk * C + cx] = v[kk];
        }
        __syncthreads();
    }
    tick(PH_GEOM);

    int status = SW_ERR_NOT_CONVERGED;
    int iters = 0, restarts = 0, converged = 0, guess_rank = -1, shifted = 0;
    double res0 = 0.0, res_last = 0.0, guess_res = 0.0, true_res = 0.0, braw = 0.0, bnorm = 0.0;
#define R_TRY(expr) do { if (!(expr)) goto aborted; } while (0)

    // reference norms ||b|| and ||M^-1 b||
    R_TRY(r_ilu<L>(X, R, S, X.bb, X.t));
    r_block_sums(X, S, 2, [&](int p, double (&v)[4]) { v[0] += X.bb[p] * X.bb[p]; v[1] += X.t[p] * X.t[p]; }, bp);
    R_TRY(r_allreduce(X, R, S, bp, 2, S.res));
    braw = sqrt(S.res[0]);
    bnorm = sqrt(S.res[1]);
    cost(A.cm.fM + 4.0, A.cm.bM + 8.0);
    tick(PH_BNORM);

    // ---- a7-a10: the initial guess (Algorithm 2) ----
    {
        const bool sub = A.guess_mode == SW_GUESS_EWMA || A.guess_mode == SW_GUESS_RRF;
        const bool upd = A.pending != 0 && A.guess_mode != SW_GUESS_RRF;
        if (A.guess_mode == SW_GUESS_RRF) {
            // Algorithm 3: Y = X Omega over the newest stored solutions
            cost(2.0 * A.ring_Ke * k, (A.ring_Ke + k) * 8.0);
            for (int i = tid; i < k * nl; i += NTHREADS) {
                const int c = i / nl, p = i - c * nl;
                const long long g = gidx(p);
                double sv = 0.0;
                for (int rr = 0; rr < A.ring_Ke; ++rr) {
                    const int slot = (A.ring_newest - rr + A.ring_K) % A.ring_K;
                    sv += A.ring[(size_t)slot * m + g] * A.omega_rrf[rr * k + c];
                }
                X.Y[i] = sv;
                A.Ynew[(size_t)c * m + g] = sv;
            }
        } else if (upd || A.guess_mode == SW_GUESS_EWMA) {
            // Y_new = r Y_old + x_prev omega^T (Algorithm 4), kept as the sketch
            if (upd) cost(3.0 * k, (2.0 * k + 1.0) * 8.0);
            for (int i = tid; i < k * nl; i += NTHREADS) {
                const int c = i / nl, p = i - c * nl;
                const long long g = gidx(p);
                const double yo = A.Yold[(size_t)c * m + g];
                double yn = yo;
                if (upd) {
                    yn = A.decay * yo + A.omega[c] * X.xp[p];
                    A.Ynew[(size_t)c * m + g] = yn;
                }
                X.Y[i] = yn;
            }
        }
        __syncthreads();
        if (sub) {
            // W = A Y in FP64 (a8): one exchange for all k columns, then k applies
            cost(k * A.cm.fA, k * (A.cm.bA + 8.0));
            R_TRY(r_exchange(X, R, S, X.Y, nl, k));
            for (int c = 0; c < k; ++c)
                r_apply(X, D, X.Y + (size_t)c * nl, X.halo + (size_t)c * P * 6, 1.0, X.Wm + (size_t)c * nl, false);
        }
        tick(PH_GUESS_W);
        if (sub) {
            const int ng = k * (k + 1) / 2, nv = ng + k;
            // Gram G = W^T W and c = W^T b: value e on threads e, e + nv, ...
            auto gram = [&]() {
                const int G = max(1, NTHREADS / nv);
                double a = 0.0;
                const int e = tid % nv, gq = tid / nv;
                if (gq < G) {
                    const double *wa = e < ng ? X.Wm + (size_t)S.ga[e] * nl : X.Wm + (size_t)(e - ng) * nl;
                    const double *wb = e < ng ? X.Wm + (size_t)S.gb[e] * nl : X.bb;
                    for (int p = gq; p < nl; p += G) a += wa[p] * wb[p];
                }
                __syncthreads();
                if (gq < G) S.red[tid] = a;
                __syncthreads();
                for (int ee = tid; ee < nv; ee += NTHREADS) {
                    double sv = 0.0;
                    for (int g2 = 0; g2 < G && g2 * nv + ee < NTHREADS; ++g2) sv += S.red[g2 * nv + ee];
                    bp[ee] = sv;
                }
                __syncthreads();
            };
            cost(2.0 * nv, (k + 1.0) * 8.0);
            gram();
            R_TRY(r_allreduce(X, R, S, bp, nv, S.res));
            if (tid < 32) {
                for (int e = tid; e < ng; e += 32) {
                    S.G[S.ga[e] * k + S.gb[e]] = S.res[e];
                    S.G[S.gb[e] * k + S.ga[e]] = S.res[e];
                }
                for (int c = tid; c < k; c += 32) S.c1[c] = S.res[ng + c];
                __syncwarp();
                double tr = 0.0;
                for (int c = 0; c < k; ++c) tr += S.G[c * k + c];
                for (int i = tid; i < k * k; i += 32) S.R[i] = S.G[i];
                __syncwarp();
                bool ok = tr > 0.0 && warp_cholesky(S.G, S.R1, k);
                if (!ok && tr > 0.0) {
                    const double sh = 11.0 * ((double)m * k + (double)k * (k + 1)) * 1.1102230246251565e-16 * tr;
                    for (int i = tid; i < k * k; i += 32) S.G[i] = S.R[i] + ((i / k == i % k) ? sh : 0.0);
                    __syncwarp();
                    ok = warp_cholesky(S.G, S.R1, k);
                    shifted = 1;
                }
                if (tid == 0) S.flags[0] = ok ? 1 : 0;
            }
            __syncthreads();
            if (S.flags[0]) {
                // second pass: Q1 = W R1^-1 in place, G2 = Q1^T Q1, c2 = Q1^T b
                cost((double)k * k + 2.0 * nv, (k + 1.0) * 8.0);
                for (int p = tid; p < nl; p += NTHREADS) {
                    double qv[MAX_K];
#pragma unroll
                    for (int c = 0; c < MAX_K; ++c) {
                        if (c >= k) break;
                        double sv = X.Wm[(size_t)c * nl + p];
                        for (int i = 0; i < c; ++i) sv -= qv[i] * S.R1[i * k + c];
                        qv[c] = sv / S.R1[c * k + c];
                    }
#pragma unroll
                    for (int c = 0; c < MAX_K; ++c) {
                        if (c >= k) break;
                        X.Wm[(size_t)c * nl + p] = qv[c];
                    }
                }
                __syncthreads();
                gram();
                R_TRY(r_allreduce(X, R, S, bp, nv, S.res));
                if (tid < 32) {
                    for (int e = tid; e < ng; e += 32) {
                        S.G[S.ga[e] * k + S.gb[e]] = S.res[e];
                        S.G[S.gb[e] * k + S.ga[e]] = S.res[e];
                    }
                    for (int c = tid; c < k; c += 32) S.c2[c] = S.res[ng + c];
                    __syncwarp();
                    const bool ok2 = warp_cholesky(S.G, S.R2, k);
                    if (!ok2) {
                        for (int i = tid; i < k * k; i += 32) S.R[i] = S.R1[i];
                        __syncwarp();
                        warp_fwdsub_t(S.R1, S.c1, S.tmp, k);
                    } else {
                        for (int e = tid; e < k * k; e += 32) {
                            const int a = e / k, bc = e % k;
                            double sv = 0.0;
                            for (int l2 = a; l2 <= bc; ++l2) sv += S.R2[a * k + l2] * S.R1[l2 * k + bc];
                            S.R[e] = bc >= a ? sv : 0.0;
                        }
                        __syncwarp();
                        warp_fwdsub_t(S.R2, S.c2, S.tmp, k);
                    }
                    // rank guard: drop columns with |R_jj| <= 1e-12 |R_00|
                    const double tiny = 1e-12 * fabs(S.R[0]);
                    warp_backsub(S.R, S.tmp, S.z, k, tiny);
                    if (tid == 0) {
                        int rk = 0;
                        for (int j = 0; j < k; ++j) rk += fabs(S.R[j * k + j]) > tiny;
                        S.flags[1] = rk;
                    }
                }
                __syncthreads();
                guess_rank = S.flags[1];
            } else {
                if (tid < MAX_K) S.z[tid] = 0.0;
                __syncthreads();
                guess_rank = 0;
            }
            // a10: x0 = Y z
            cost(2.0 * k, k * 8.0 + 8.0);
            for (int p = tid; p < nl; p += NTHREADS) {
                double sv = 0.0;
                for (int c = 0; c < k; ++c) sv += X.Y[(size_t)c * nl + p] * S.z[c];
                X.x[p] = sv;
            }
        } else if (A.guess_mode == SW_GUESS_PREVIOUS) {
            cost(0.0, 16.0);
            for (int p = tid; p < nl; p += NTHREADS) X.x[p] = X.xp[p];
        } else {
            for (int p = tid; p < nl; p += NTHREADS) X.x[p] = 0.0;
        }
        __syncthreads();
    }
    tick(PH_GUESS_LS);
    if (A.guess_only) {
        for (int p = tid; p < nl; p += NTHREADS) A.x[gidx(p)] = X.x[p];
        if (X.b == 0 && tid == 0) {
            A.stats->guess_rank = guess_rank;
            A.stats->cholesky_shift = shifted;
        }
        return;
    }

    // ---- restarted GMRES(m), left-preconditioned (Sec. 3) ----
    if (bnorm == 0.0) {
        for (int p = tid; p < nl; p += NTHREADS) X.x[p] = 0.0;
        __syncthreads();
        converged = 1;
        status = SW_OK;
    } else {
        for (int cycle = 0;; ++cycle) {
            // r = b - A x (FP64); V0 = M^-1 r
            R_TRY(r_exchange(X, R, S, X.x, 0, 1));
            const double racc = r_apply(X, D, X.x, X.halo, 1.0, X.r, true);
            tick(PH_RES_APPLY);
            R_TRY(r_ilu<L>(X, R, S, X.r, X.V));
            {
                double rsum = racc;
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
                if ((tid & 31) == 0) S.red[tid >> 5] = rsum;
                __syncthreads();
                double vsum = 0.0;
                for (int p = tid; p < nl; p += NTHREADS) vsum += X.V[p] * X.V[p];
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) vsum += __shfl_xor_sync(0xffffffffu, vsum, o);
                if ((tid & 31) == 0) S.red[NWARPS + (tid >> 5)] = vsum;
                __syncthreads();
                if (tid < 2) {
                    double sv = 0.0;
                    for (int w = 0; w < NWARPS; ++w) sv += S.red[tid * NWARPS + w];
                    bp[tid] = sv;
                }
                __syncthreads();
            }
            R_TRY(r_allreduce(X, R, S, bp, 2, S.res));
            tick(PH_RES_ILU);
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
            if (tid == 0) {
                S.scale[0] = 1.0 / beta;
                for (int i = 0; i <= mr; ++i) S.g[i] = 0.0;
                S.g[0] = beta;
            }
            __syncthreads();
            int jend = 0;
            for (int j = 0; j < mr; ++j) {
                double *w = X.V + (size_t)(j + 1) * nlp;
                const double *vj = X.V + (size_t)j * nlp;
                // w = M^-1 A v_j  (v_j = scale_j V_j)
                R_TRY(r_exchange(X, R, S, vj, 0, 1));
                r_apply(X, D, vj, X.halo, S.scale[j], X.t, false);
                tick(PH_ARN_APPLY);
                R_TRY(r_ilu<L>(X, R, S, X.t, w));
                tick(PH_ARN_ILU);
                // Gram-Schmidt pass 1: d_i = V_i . w
                r_block_dots(X, S, j + 1, w, false, bp);
                R_TRY(r_allreduce(X, R, S, bp, j + 1, S.res));
                tick(PH_CGS1);
                if (tid < MAX_RESTART) {
                    const int i = tid;
                    const double hi = i <= j ? S.res[i] * S.scale[i] : 0.0;
                    if (i <= j) S.H[i * MAX_RESTART + j] = hi;
                    S.hs[i] = i <= j ? hi * S.scale[i] : 0.0;
                }
                __syncthreads();
                // pass 2: w -= V h; d'_i = V_i . w and w . w in one reduction
                for (int p = tid; p < nl; p += NTHREADS) {
                    double wv = w[p];
                    for (int i = 0; i <= j; ++i) wv -= S.hs[i] * X.V[(size_t)i * nlp + p];
                    w[p] = wv;
                }
                __syncthreads();
                r_block_dots(X, S, j + 1, w, true, bp);
                R_TRY(r_allreduce(X, R, S, bp, j + 2, S.res));
                tick(PH_CGS2);
                double hn2;
                {
                    double hh = 0.0;
                    for (int i = 0; i <= j; ++i) {
                        const double hi = S.res[i] * S.scale[i];
                        hh += hi * hi;
                    }
                    hn2 = S.res[j + 1] - hh;
                    __syncthreads();
                    if (tid < MAX_RESTART) {
                        const int i = tid;
                        const double hi = i <= j ? S.res[i] * S.scale[i] : 0.0;
                        if (i <= j) S.H[i * MAX_RESTART + j] += hi;
                        S.hs[i] = i <= j ? hi * S.scale[i] : 0.0;
                    }
                    __syncthreads();
                }
                // pass 3 (local): w -= V h'
                for (int p = tid; p < nl; p += NTHREADS) {
                    double wv = w[p];
                    for (int i = 0; i <= j; ++i) wv -= S.hs[i] * X.V[(size_t)i * nlp + p];
                    w[p] = wv;
                }
                __syncthreads();
                // ||w||^2 - ||h'||^2 has lost accuracy when it is far below ||w||^2: reduce directly
                if (!(hn2 > 1e-4 * S.res[j + 1])) {
                    r_block_sums(X, S, 1, [&](int p, double (&v)[4]) { v[0] += w[p] * w[p]; }, bp);
                    R_TRY(r_allreduce(X, R, S, bp, 1, S.res));
                    hn2 = S.res[0];
                }
                tick(PH_CGS3);
                // a5: Hessenberg column, Givens rotations, residual estimate
                if (tid == 0) {
                    const double hn = sqrt(fmax(hn2, 0.0));
                    S.scale[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
                    double *Hc = S.H;
                    for (int i = 0; i < j; ++i) {
                        const double a = Hc[i * MAX_RESTART + j], bq = Hc[(i + 1) * MAX_RESTART + j];
                        Hc[i * MAX_RESTART + j] = S.cs[i] * a + S.sn[i] * bq;
                        Hc[(i + 1) * MAX_RESTART + j] = -S.sn[i] * a + S.cs[i] * bq;
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
                cost(A.cm.fA + A.cm.fM + 8.0 * (j + 1) + 2.0, A.cm.bA + A.cm.bM + (3.0 * j + 8.0) * 8.0);
                ++iters;
                jend = j + 1;
                if (S.flags[2]) break;
            }
            // a6: y = R^-1 g, x += V (scale y)
            if (tid < 32) {
                const int lane = tid;
                double acc = lane < jend ? S.g[lane] : 0.0;
                for (int i = jend - 1; i >= 0; --i) {
                    const double yi = __shfl_sync(0xffffffffu, acc, i) / S.H[i * MAX_RESTART + i];
                    if (lane == i) S.y[i] = yi * S.scale[i];
                    if (lane < i) acc -= S.H[lane * MAX_RESTART + i] * yi;
                }
            }
            __syncthreads();
            cost(2.0 * jend, jend * 8.0 + 16.0);
            for (int p = tid; p < nl; p += NTHREADS) {
                double sv = X.x[p];
                for (int i = 0; i < jend; ++i) sv += S.y[i] * X.V[(size_t)i * nlp + p];
                X.x[p] = sv;
            }
            __syncthreads();
            tick(PH_UPDATE);
        }
    }
    // true residual ||b - A x|| / ||b||; the solution is kept for the next guess
    {
        R_TRY(r_exchange(X, R, S, X.x, 0, 1));
        const double racc = r_apply(X, D, X.x, X.halo, 1.0, X.r, true);
        double rsum = racc;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
        if ((tid & 31) == 0) S.red[tid >> 5] = rsum;
        for (int p = tid; p < nl; p += NTHREADS) {
            const long long g = gidx(p);
            A.x[g] = X.x[p];
            A.xprev[g] = X.x[p];
            if (A.ring_store) A.ring_store[g] = X.x[p];
        }
        __syncthreads();
        if (tid == 0) {
            double sv = 0.0;
            for (int w = 0; w < NWARPS; ++w) sv += S.red[w];
            bp[0] = sv;
        }
        __syncthreads();
        R_TRY(r_allreduce(X, R, S, bp, 1, S.res));
        true_res = braw > 0.0 ? sqrt(S.res[0]) / braw : sqrt(S.res[0]);
        cost(A.cm.fA + 3.0, A.cm.bA + 24.0);
    }
    tick(PH_TRUERES);
    if (X.b == 0 && tid == 0) {
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
    return;
aborted:
    // a wait ran out (or another block's did): report and leave; no work of
    // this block is in flight (every copy above is a plain load or store)
    if (tid == 0) A.stats->status = SW_ERR_TIMEOUT;
#undef R_TRY
}

// Per-block constants: the off-column factor slots of the block's columns
// (fac[i][l][cx], i in the order of Off<L>), then the inverses of their
// in-column L and U blocks (P x P each, transposed as in Dev).
template <int L>
__global__ void resident_blob_kernel(Dev D, ResDev R, double *blob) {
    const int b = blockIdx.x, C = R.C, P = D.P, nl = R.nl;
    double *out = blob + (size_t)b * R.blob;
    const int per = D.ncol >> 2;
    for (int i = threadIdx.x; i < Off<L>::N * nl; i += blockDim.x) {
        const int s = i / nl, rr = i - s * nl, l = rr / C, cx = rr - l * C;
        const int col = b * C + cx, c = col & 3, qq = col >> 2;
        int slot = 0;
#pragma unroll
        for (int u = 0; u < Off<L>::N; ++u)
            if (u == s) slot = Off<L>::slot(u);
        const long long row = (long long)c * per * P + (long long)l * per + qq;
        out[i] = D.lu64[(size_t)slot * D.m + row];
    }
    for (int i = threadIdx.x; i < 2 * C * P * P; i += blockDim.x) {
        const int which = i / (C * P * P), rr = i - which * C * P * P, cx = rr / (P * P), e = rr - cx * P * P;
        const int col = b * C + cx, c = col & 3, qq = col >> 2;
        const long long cr = (long long)c * per + qq;
        out[(size_t)Off<L>::N * nl + i] = (which ? D.uinv64 : D.linv64)[(size_t)cr * P * P + e];
    }
}

// ---- host side ---------------------------------------------------------------

struct Resident {
    ResDev R{};
    size_t smem = 0;
    const void *kern = nullptr;
};

static size_t resident_smem(const Dev &D, int C, int mr, int k, int noff) {
    const int P = D.P, nl = C * P, nlp = nl | 1, mv = k > 1 ? k : 1;
    size_t d = (size_t)noff * nl + 2 * (size_t)C * P * P + (size_t)(mr + 1) * nlp + 5 * (size_t)nlp +
               2 * (size_t)k * nl + (size_t)mv * P * 6 + 2 * (size_t)P * (C + 2 * HALF) + (size_t)NCC * C +
               2 * (size_t)P * W + (size_t)(P + 1) / 2 + 1;
    return ((sizeof(SmemFixed) + 255) & ~size_t(255)) + d * sizeof(double);
}

static const void *resident_kernel_for(int layout) {
    return layout == BOX2D ? (const void *)resident_kernel<BOX2D> : (const void *)resident_kernel<CROSS2D>;
}

// Whether problem P can run on the resident executor, and its slab width.
bool resident_fits(const Problem *P, int nsm, int *C_out, size_t *smem_out) {
    const Dev &D = P->dev;
    const sw_params &p = P->params;
    if (D.three_d || D.walls || p.precision != SW_PRECISION_FP64 || p.orthonormalize) return false;
    if (D.layout != CROSS2D && D.layout != BOX2D) return false;
    if (p.restart > MAX_RESTART || p.restart + 2 > 32) return false;
    const int noff = D.layout == BOX2D ? Off<BOX2D>::N : Off<CROSS2D>::N;
    for (int C = 4; C <= 16; C += 4) {
        if (D.nx % C) continue;
        const int NB = D.nx / C;
        if (NB > nsm || NB > 160 || NB < 2) continue;
        const size_t sm = resident_smem(D, C, p.restart, p.k, noff);
        if (sm > 227 * 1024) return false;
        *C_out = C;
        *smem_out = sm;
        return true;
    }
    return false;
}

int setup_resident(Problem *P) {
    int nsm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P->device);
    if (e != cudaSuccess) return cuda_fail(e, "SM count");
    int C = 0;
    size_t smem = 0;
    if (!resident_fits(P, nsm, &C, &smem)) {
        set_error("the resident executor needs a small periodic 2-D FP64 problem (no orthonormalisation)");
        return SW_ERR_BAD_ARG;
    }
    const Dev &D = P->dev;
    Resident *Rs = new (std::nothrow) Resident();
    if (!Rs) { set_error("out of host memory"); return SW_ERR_BAD_ARG; }
    P->resident = Rs;
    ResDev &R = Rs->R;
    R.stall = -1;
    R.C = C;
    R.NB = D.nx / C;
    R.nl = C * D.P;
    R.nlp = R.nl | 1;
    R.mv = P->params.k > 1 ? P->params.k : 1;
    R.noff = D.layout == BOX2D ? Off<BOX2D>::N : Off<CROSS2D>::N;
    R.blob = R.noff * R.nl + 2 * C * D.P * D.P;
    double *blob = nullptr, *mail = nullptr, *part = nullptr;
    unsigned *sync = nullptr;
    e = cudaMalloc((void **)&blob, (size_t)R.NB * R.blob * sizeof(double));
    if (e == cudaSuccess) { P->allocs.push_back(blob); e = cudaMalloc((void **)&mail, 2 * (size_t)R.NB * R.mv * D.P * 6 * sizeof(double)); }
    if (e == cudaSuccess) { P->allocs.push_back(mail); e = cudaMalloc((void **)&part, 2 * (size_t)R.NB * PART_STRIDE * sizeof(double)); }
    if (e == cudaSuccess) { P->allocs.push_back(part); e = cudaMalloc((void **)&sync, (2 + (size_t)R.NB) * sizeof(unsigned)); }
    if (e == cudaSuccess) P->allocs.push_back(sync);
    if (e != cudaSuccess) return cuda_fail(e, "resident executor set-up");
    R.cblob = blob;
    R.mail = mail;
    R.part = part;
    R.sync = sync;
    if (D.layout == BOX2D) resident_blob_kernel<BOX2D><<<R.NB, 256>>>(D, R, blob);
    else resident_blob_kernel<CROSS2D><<<R.NB, 256>>>(D, R, blob);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "resident constants");
    Rs->kern = resident_kernel_for(D.layout);
    Rs->smem = smem;
    e = cudaFuncSetAttribute(Rs->kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "resident smem attribute");
    int per = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, Rs->kern, NTHREADS, smem);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    if (per < 1) { set_error("resident kernel does not fit on an SM"); return SW_ERR_BAD_ARG; }
    P->launches++;
    return SW_OK;
}

void destroy_resident(Problem *P) {
    delete (Resident *)P->resident;
    P->resident = nullptr;
}

int solve_resident(Problem *P, const SolveArgs &A, cudaStream_t s) {
    Resident *Rs = (Resident *)P->resident;
    ResDev R = Rs->R;
    R.stall = P->resident_stall;
    P->resident_stall = -1;
    cudaError_t e = cudaMemsetAsync(R.sync, 0, (2 + (size_t)R.NB) * sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_fail(e, "resident sync reset");
    Dev D = P->dev;
    SolveArgs Ac = A;
    void *args[] = {&D, &Ac, &R};
    e = cudaLaunchCooperativeKernel(Rs->kern, R.NB, NTHREADS, args, Rs->smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "resident solve launch");
    P->launches++;
    return SW_OK;
}

}  // namespace sw

using namespace sw;

extern "C" int sw_test_stall_exchange(sw_problem *pp, int exchange) {
    Problem *P = (Problem *)pp;
    if (!P || exchange < 1) { set_error("bad argument"); return SW_ERR_BAD_ARG; }
    if (P->exec != SW_EXEC_RESIDENT) { set_error("the problem does not use the resident executor"); return SW_ERR_BAD_ARG; }
    P->resident_stall = exchange;
    return SW_OK;
}
