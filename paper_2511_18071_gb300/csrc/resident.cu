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
//    rightmost columns in a mailbox in global memory and reads its two
//    neighbours' mailboxes, instead of a grid barrier;
//  - inner products are all-reduced: every block publishes its partial sums
//    and sums every block's partials in a fixed order (so every block holds
//    bit-identical values and takes the same decisions);
//  - mailbox and partial-sum words are self-validating: each 8-byte word holds
//    32 bits of data and a 32-bit tag (launch epoch and exchange or reduction
//    number), written and read as single 8-byte accesses, so a reader polls
//    the data itself until its tag appears (one round trip through L2 once the
//    data have landed; no fence, flag or counter); slots alternate between two
//    buffers, and a block cannot get two exchanges ahead of its neighbours;
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
    int stall;             // testing aid: from this exchange on, block 0 publishes nothing (-1: never)
    unsigned epoch;        // launch epoch, 1..4095, in the high bits of every tag
    const double *cblob;   // NB x blob: off-column factors fac[i][l][cx], then Linv and Uinv of the block's columns
    unsigned long long *mail;   // 2 x NB x mv x P x 6 boundary values, two tagged words each
    unsigned *sync;             // [0] abort flag
    unsigned long long *part;   // 2 x NB x PART_STRIDE partial sums, two tagged words each
};

__device__ __forceinline__ void r_st64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long r_ld64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
// A double as two tagged words: (tag << 32) | low 32 bits, (tag << 32) | high 32 bits.
__device__ __forceinline__ void r_put(unsigned long long *p, double v, unsigned tag) {
    const unsigned long long t = (unsigned long long)tag << 32;
    r_st64(p, t | (unsigned)__double2loint(v));
    r_st64(p + 1, t | (unsigned)__double2hiint(v));
}

__device__ __forceinline__ unsigned r_ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Up to N tagged doubles at addr(0..n-1): every round loads all words still
// missing their tag at once (one round trip per round), until all carry it.
template <int N, class Addr>
__device__ __forceinline__ bool r_get_n(Addr addr, int n, unsigned tag, unsigned *abortp, double (&out)[N]) {
    unsigned long long lo[N], hi[N];
    unsigned missing = n >= 32 ? 0xffffffffu : (1u << n) - 1u;
    unsigned long long t0 = 0;
    for (unsigned it = 0;; ++it) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            if (missing & (1u << q)) {
                lo[q] = r_ld64(addr(q));
                hi[q] = r_ld64(addr(q) + 1);
            }
        }
#pragma unroll
        for (int q = 0; q < N; ++q)
            if ((missing & (1u << q)) && (unsigned)(lo[q] >> 32) == tag && (unsigned)(hi[q] >> 32) == tag) {
                out[q] = __hiloint2double((int)(unsigned)hi[q], (int)(unsigned)lo[q]);
                missing &= ~(1u << q);
            }
        if (!missing) return true;
        if (it == 0) t0 = global_ns();
        if ((it & 31) == 31) {
            if (r_ld_acquire(abortp)) return false;
            if (global_ns() - t0 > R_WAIT_NS) {
                atomicExch(abortp, 1u);
                return false;
            }
        }
    }
}

// Per-block view of the solve's shared memory (set once, then read-only; kept
// in shared memory itself to leave registers to the arithmetic).
struct RCtx {
    int b, bl, br, C, P, nl, nlp, HX, NB;
    double *fac, *linv, *uinv;          // constants
    double *V, *t, *x, *bb, *r, *xp;    // vectors (nlp stride between Krylov vectors)
    double *Y, *Wm, *halo, *sp, *sq, *cc, *ws1, *ws2;
    int *win;
};

// ---- exchange of boundary columns with the two neighbouring blocks ----------

// Publish the three leftmost and three rightmost columns of nv local vectors
// (vector c at vec + c * stride) and fill halo[c][l][0..5] with the left
// neighbour's three rightmost and the right neighbour's three leftmost columns.
// Publication and collection may be separated by other work (the collection
// of exchange seq must come before the publication of exchange seq + 1).
__device__ __noinline__ void r_publish(const RCtx &X, const ResDev &R, const double *vec, int stride, int nv,
                                       unsigned seq) {
    const int P = X.P, C = X.C, n6 = P * 6;
    const unsigned tag = (R.epoch << 20) | seq;
    const int par = seq & 1;
    unsigned long long *mine = R.mail + 2 * ((size_t)(par * X.NB + X.b) * R.mv) * n6;
    if (!(X.b == 0 && R.stall > 0 && (int)seq >= R.stall)) {
        for (int i = threadIdx.x; i < nv * n6; i += NTHREADS) {
            const int c = i / n6, rr = i - c * n6, l = rr / 6, e = rr - l * 6;
            r_put(mine + 2 * i, vec[(size_t)c * stride + l * C + (e < 3 ? e : C - 6 + e)], tag);
        }
    }
}

__device__ __noinline__ bool r_collect(const RCtx &X, const ResDev &R, int nv, unsigned seq) {
    const int P = X.P, n6 = P * 6;
    const unsigned tag = (R.epoch << 20) | seq;
    const int par = seq & 1;
    const unsigned long long *ml = R.mail + 2 * ((size_t)(par * X.NB + X.bl) * R.mv) * n6;
    const unsigned long long *mr = R.mail + 2 * ((size_t)(par * X.NB + X.br) * R.mv) * n6;
    bool ok = true;
    constexpr int CH = 8;
    for (int i0 = threadIdx.x; i0 < nv * n6 && ok; i0 += CH * NTHREADS) {
        const int cnt = min(CH, (nv * n6 - i0 + NTHREADS - 1) / NTHREADS);
        double v[CH];
        ok = r_get_n<CH>([&](int q) {
            const int i = i0 + q * NTHREADS;
            return i % 6 < 3 ? ml + 2 * (i + 3) : mr + 2 * (i - 3);
        }, cnt, tag, R.sync, v);
#pragma unroll
        for (int q = 0; q < CH; ++q)
            if (q < cnt) X.halo[i0 + q * NTHREADS] = v[q];
    }
    return __syncthreads_and(ok) != 0;
}

__device__ bool r_exchange(const RCtx &X, const ResDev &R, const double *vec, int stride, int nv, unsigned seq) {
    r_publish(X, R, vec, stride, nv, seq);
    return r_collect(X, R, nv, seq);
}

// ---- all-reduce of block partial sums ----------------------------------------

// out[v] = sum over blocks of bp[v] (v < nv <= PART_STRIDE), summed in the same
// order by every block.  bp is in shared memory; out may be S.res.
__device__ __noinline__ bool r_allreduce(const RCtx &X, const ResDev &R, SmemFixed &S, const double *bp, int nv,
                                         double *out, unsigned round) {
    const unsigned tag = (R.epoch << 20) | (0x80000u + round);
    const int par = round & 1;
    unsigned long long *mine = R.part + 2 * (size_t)(par * X.NB + X.b) * PART_STRIDE;
    for (int i = threadIdx.x; i < nv; i += NTHREADS) r_put(mine + 2 * i, bp[i], tag);
    const unsigned long long *pp = R.part + 2 * (size_t)par * X.NB * PART_STRIDE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool ok = true;
    for (int v0 = 0; v0 < nv; v0 += 32) {
        const int v = v0 + lane;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        if (v < nv && ok) {
            // blocks warp, warp + 8, ...: at most 20 (NB <= 160), loaded together
            const int nmine = (X.NB - warp + NWARPS - 1) / NWARPS;
            constexpr int CH = 20;
            for (int u0 = 0; u0 < nmine && ok; u0 += CH) {
                double t[CH];
                const int cnt = min(CH, nmine - u0);
                ok = r_get_n<CH>([&](int q) {
                    return pp + 2 * ((size_t)(warp + NWARPS * (u0 + q)) * PART_STRIDE + v);
                }, cnt, tag, R.sync, t);
#pragma unroll
                for (int q = 0; q < CH; ++q) {
                    if (q >= cnt) break;
                    // block warp + 8u goes to accumulator u mod 4 (a fixed order)
                    const int u = u0 + q;
                    if ((u & 3) == 0) a0 += t[q];
                    else if ((u & 3) == 1) a1 += t[q];
                    else if ((u & 3) == 2) a2 += t[q];
                    else a3 += t[q];
                }
            }
        }
        S.red[warp * 32 + lane] = (a0 + a1) + (a2 + a3);
        if (!__syncthreads_and(ok)) return false;
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

// One colour phase with the work of each column spread over several warps
// (levels one per lane, P <= 32): the warps of a column take every nwc-th
// off-column slot, then a slice of the rows of the column's inverse block,
// and the slices are added; the warps' partial sums meet in shared memory.
// Forward: out = Linv (in - lower couplings), then with UP the backward step
// of the same colour, out = Uinv out; backward: out = Uinv (out - upper couplings).
template <int L, int CC, bool FWD, bool UP>
__device__ void r_phase(const RCtx &X, SmemFixed &S, const double *in, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int P = X.P, C = X.C;
    const int ncc = C >> 2;                   // columns of this colour in the block (1..4)
    const int nwc = ncc > 2 ? 2 : 4;          // warps per column
    const int cs = warp / nwc, part = warp - cs * nwc;
    const bool act = cs < ncc;
    const int cx = 4 * cs + CC;
    double *po = S.red, *py = S.xchg;
    // off-column couplings, slots part, part + nwc, ...
    double o = 0.0;
    if (act && lane < P) {
#pragma unroll
        for (int i = 0; i < Off<L>::N; ++i) {
            const int ox = Off<L>::ox(i);
            const int nc = (CC + ox) & 3;
            if (FWD ? (nc >= CC) : (nc <= CC)) continue;
            if (i % nwc != part) continue;
            const int lev = Off<L>::kk(i) < 0 ? lane : X.win[lane] + 1 + Off<L>::kk(i);
            o += X.fac[((size_t)i * P + lane) * C + cx] * r_ext(X, out, X.halo, lev, cx + ox);
        }
    }
    po[warp * 32 + lane] = o;
    __syncthreads();
    double g = 0.0;
    if (act && lane < P) {
        double os = 0.0;
        for (int p = 0; p < nwc; ++p) os += po[(cs * nwc + p) * 32 + lane];
        g = (FWD ? in[lane * C + cx] : out[lane * C + cx]) - os;
    }
    const int rng = (P + nwc - 1) / nwc, a0 = part * rng, a1 = min(P, a0 + rng);
    const double *B = (FWD ? X.linv : X.uinv) + (size_t)(act ? cx : 0) * P * P;
    double y = 0.0;
    for (int a2 = a0; a2 < a1; ++a2) {
        const double ga = __shfl_sync(0xffffffffu, g, a2);
        if (act && lane < P) y += B[a2 * P + lane] * ga;
    }
    py[warp * 32 + lane] = y;
    __syncthreads();
    if (UP) {
        // backward step of the last colour on the forward result
        double yf = 0.0;
        if (act && lane < P)
            for (int p = 0; p < nwc; ++p) yf += py[(cs * nwc + p) * 32 + lane];
        const double *U = X.uinv + (size_t)(act ? cx : 0) * P * P;
        double z = 0.0;
        for (int a2 = a0; a2 < a1; ++a2) {
            const double ga = __shfl_sync(0xffffffffu, yf, a2);
            if (act && lane < P) z += U[a2 * P + lane] * ga;
        }
        po[warp * 32 + lane] = z;
        __syncthreads();
        if (act && part == 0 && lane < P) {
            double zs = 0.0;
            for (int p = 0; p < nwc; ++p) zs += po[(cs * nwc + p) * 32 + lane];
            out[lane * C + cx] = zs;
        }
    } else if (act && part == 0 && lane < P) {
        double ys = 0.0;
        for (int p = 0; p < nwc; ++p) ys += py[(cs * nwc + p) * 32 + lane];
        out[lane * C + cx] = ys;
    }
    __syncthreads();
}

// out = U^-1 L^-1 in: four forward colours, four backward colours (the last
// forward and first backward colour together), six boundary exchanges.
template <int L>
__device__ bool r_ilu(const RCtx &X, const ResDev &R, SmemFixed &S, const double *in, double *out, unsigned &seq) {
    if (X.P <= 32) {
        r_phase<L, 0, true, false>(X, S, in, out);
        if (!r_exchange(X, R, out, 0, 1, ++seq)) return false;
        r_phase<L, 1, true, false>(X, S, in, out);
        if (!r_exchange(X, R, out, 0, 1, ++seq)) return false;
        r_phase<L, 2, true, false>(X, S, in, out);
        if (!r_exchange(X, R, out, 0, 1, ++seq)) return false;
        r_phase<L, 3, true, true>(X, S, in, out);
        if (!r_exchange(X, R, out, 0, 1, ++seq)) return false;
        r_phase<L, 2, false, false>(X, S, in, out);
        if (!r_exchange(X, R, out, 0, 1, ++seq)) return false;
        r_phase<L, 1, false, false>(X, S, in, out);
        if (!r_exchange(X, R, out, 0, 1, ++seq)) return false;
        r_phase<L, 0, false, false>(X, S, in, out);
        return true;
    }
    r_fwd<L, 0, false>(X, in, out);
    if (!r_exchange(X, R, out, 0, 1, ++seq)) return false;
    r_fwd<L, 1, false>(X, in, out);
    if (!r_exchange(X, R, out, 0, 1, ++seq)) return false;
    r_fwd<L, 2, false>(X, in, out);
    if (!r_exchange(X, R, out, 0, 1, ++seq)) return false;
    r_fwd<L, 3, true>(X, in, out);
    if (!r_exchange(X, R, out, 0, 1, ++seq)) return false;
    r_bwd<L, 2>(X, out);
    if (!r_exchange(X, R, out, 0, 1, ++seq)) return false;
    r_bwd<L, 1>(X, out);
    if (!r_exchange(X, R, out, 0, 1, ++seq)) return false;
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
    __shared__ RCtx Xs;
    if (tid == 0) {
        RCtx &X0 = Xs;
        X0.b = blockIdx.x;
        X0.NB = R.NB;
        X0.bl = X0.b == 0 ? R.NB - 1 : X0.b - 1;
        X0.br = X0.b == R.NB - 1 ? 0 : X0.b + 1;
        X0.C = R.C;
        X0.P = D.P;
        X0.nl = R.nl;
        X0.nlp = R.nlp;
        X0.HX = R.C + 2 * HALF;
        // shared-memory carve-out (doubles)
        const int C0 = X0.C, P0 = X0.P, nl0 = X0.nl, nlp0 = X0.nlp;
        double *q = base;
        X0.fac = q; q += (size_t)R.noff * nl0;
        X0.linv = q; q += (size_t)C0 * P0 * P0;
        X0.uinv = q; q += (size_t)C0 * P0 * P0;
        X0.V = q; q += (size_t)(mr + 1) * nlp0;
        X0.t = q; q += nlp0;
        X0.x = q; q += nlp0;
        X0.bb = q; q += nlp0;
        X0.r = q; q += nlp0;
        X0.xp = q; q += nlp0;
        X0.Y = q; q += (size_t)k * nl0;
        X0.Wm = q; q += (size_t)k * nl0;
        X0.halo = q; q += (size_t)R.mv * P0 * 6;
        X0.sp = q; q += (size_t)P0 * X0.HX;
        X0.sq = q; q += (size_t)P0 * X0.HX;
        X0.cc = q; q += (size_t)NCC * C0;
        X0.ws1 = q; q += (size_t)P0 * W;
        X0.ws2 = q; q += (size_t)P0 * W;
        X0.win = reinterpret_cast<int *>(q);
    }
    __syncthreads();
    const RCtx &X = Xs;
    unsigned seq = 0, round = 0;   // exchanges and reductions so far (the same in every block)
    const int C = X.C, P = X.P, nl = X.nl, nlp = X.nlp;
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
    R_TRY(r_ilu<L>(X, R, S, X.bb, X.t, seq));
    r_block_sums(X, S, 2, [&](int p, double (&v)[4]) { v[0] += X.bb[p] * X.bb[p]; v[1] += X.t[p] * X.t[p]; }, bp);
    R_TRY(r_allreduce(X, R, S, bp, 2, S.res, ++round));
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
            R_TRY(r_exchange(X, R, X.Y, nl, k, ++seq));
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
            R_TRY(r_allreduce(X, R, S, bp, nv, S.res, ++round));
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
                R_TRY(r_allreduce(X, R, S, bp, nv, S.res, ++round));
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
            R_TRY(r_exchange(X, R, X.x, 0, 1, ++seq));
            const double racc = r_apply(X, D, X.x, X.halo, 1.0, X.r, true);
            tick(PH_RES_APPLY);
            R_TRY(r_ilu<L>(X, R, S, X.r, X.V, seq));
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
            R_TRY(r_allreduce(X, R, S, bp, 2, S.res, ++round));
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
                // w = M^-1 A v_j  (v_j = scale_j V_j); the boundary of V_j was
                // published when it was formed (V_0 here, the others after pass 3)
                if (j == 0) r_publish(X, R, vj, 0, 1, ++seq);
                R_TRY(r_collect(X, R, 1, seq));
                r_apply(X, D, vj, X.halo, S.scale[j], X.t, false);
                tick(PH_ARN_APPLY);
                R_TRY(r_ilu<L>(X, R, S, X.t, w, seq));
                tick(PH_ARN_ILU);
                // Gram-Schmidt pass 1: d_i = V_i . w
                r_block_dots(X, S, j + 1, w, false, bp);
                R_TRY(r_allreduce(X, R, S, bp, j + 1, S.res, ++round));
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
                R_TRY(r_allreduce(X, R, S, bp, j + 2, S.res, ++round));
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
                // the next apply's boundary exchange, in flight during the rotations
                // (w is final now; its scale comes with the apply)
                r_publish(X, R, w, 0, 1, ++seq);
                // ||w||^2 - ||h'||^2 has lost accuracy when it is far below ||w||^2: reduce directly
                if (!(hn2 > 1e-4 * S.res[j + 1])) {
                    r_block_sums(X, S, 1, [&](int p, double (&v)[4]) { v[0] += w[p] * w[p]; }, bp);
                    R_TRY(r_allreduce(X, R, S, bp, 1, S.res, ++round));
                    hn2 = S.res[0];
                }
                tick(PH_CGS3);
                // a5: Hessenberg column, Givens rotations, residual estimate
                if (tid == 0) {
                    const double hn = sqrt(fmax(hn2, 0.0));
                    S.scale[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
                    // the earlier rotations on the new column: row i + 1 as
                    // rotated so far is the only carried value, one fused
                    // multiply-add per rotation on the dependent chain
                    double *Hc = S.H;
                    double tr = Hc[j];
                    for (int i = 0; i < j; ++i) {
                        const double h1 = Hc[(i + 1) * MAX_RESTART + j], ci = S.cs[i], si = S.sn[i];
                        const double ch = ci * h1;
                        Hc[i * MAX_RESTART + j] = fma(ci, tr, si * h1);
                        tr = fma(-si, tr, ch);
                    }
                    const double a = tr;
                    const double den = sqrt(fma(a, a, hn * hn));
                    const double rden = 1.0 / den;
                    S.cs[j] = a * rden;
                    S.sn[j] = hn * rden;
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
        R_TRY(r_exchange(X, R, X.x, 0, 1, ++seq));
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
        R_TRY(r_allreduce(X, R, S, bp, 1, S.res, ++round));
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
    unsigned epoch = 0;   // launches so far (the tag epoch is 1 + epoch mod 4095)
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
    double *blob = nullptr;
    unsigned long long *mail = nullptr, *part = nullptr;
    unsigned *sync = nullptr;
    const size_t mail_bytes = 2 * 2 * (size_t)R.NB * R.mv * D.P * 6 * sizeof(unsigned long long);
    const size_t part_bytes = 2 * 2 * (size_t)R.NB * PART_STRIDE * sizeof(unsigned long long);
    e = cudaMalloc((void **)&blob, (size_t)R.NB * R.blob * sizeof(double));
    if (e == cudaSuccess) { P->allocs.push_back(blob); e = cudaMalloc((void **)&mail, mail_bytes); }
    if (e == cudaSuccess) { P->allocs.push_back(mail); e = cudaMemset(mail, 0, mail_bytes); }
    if (e == cudaSuccess) e = cudaMalloc((void **)&part, part_bytes);
    if (e == cudaSuccess) { P->allocs.push_back(part); e = cudaMemset(part, 0, part_bytes); }
    if (e == cudaSuccess) e = cudaMalloc((void **)&sync, sizeof(unsigned));
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
    e = ensure_smem((const void *)Rs->kern, (size_t)(int)smem);
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
    // consecutive launches never share an epoch, so a word left by the last
    // launch never carries a tag this launch waits for
    R.epoch = 1 + (Rs->epoch++ % 4095u);
    cudaError_t e = cudaMemsetAsync(R.sync, 0, sizeof(unsigned), s);
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
