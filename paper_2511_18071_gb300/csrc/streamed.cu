// The Poisson solve of one stage for large problems, as a sequence of
// high-occupancy kernels (the streamed executor).
//
// Same algorithm, in the same order, as the persistent solve kernel
// (sw_solve.cuh): reference norms, the EWMA guess of Algorithms 2 and 4
// (sketch update, W = A Y in FP64, Gram, CholeskyQR2 with the shifted
// fallback and the rank guard, x0 = Y z), then restarted GMRES
// left-preconditioned with the fixed ILU(0) factors (Sec. 3) with CGS2,
// Givens rotations and the FP64 restart residual.  The difference is the
// execution: a persistent kernel has one block per SM (8 warps), too few to
// keep enough loads in flight when the factors, the Krylov basis and the
// sketch live in HBM; here every bandwidth-bound phase is its own kernel with
// as many blocks as the data needs, and the small dense steps (Hessenberg
// column, Givens, Cholesky, stop tests) run in one-block control kernels that
// keep their state in device memory.  Kernels of an Arnoldi step return at
// once when the control state says the cycle or the solve has ended, so the
// host enqueues a whole restart cycle and synchronises once per cycle.
#include <cmath>
#include <cstring>
#include <mutex>
#include <set>
#include <type_traits>
#include <utility>
#include <vector>

#include "sw_colapply.cuh"
#include "sw_ilu_packed.cuh"
#include "sw_solve.cuh"

namespace sw {

constexpr int SNB = 4 * 152;   // blocks of the streaming reduction kernels

// Control state of one streamed solve (device memory).
struct SState {
    double H[(MAX_RESTART + 1) * MAX_RESTART];
    double cs[MAX_RESTART], sn[MAX_RESTART], g[MAX_RESTART + 1], y[MAX_RESTART];
    double scale[MAX_RESTART + 1];
    double hs[MAX_RESTART];
    float hs32[MAX_RESTART];
    double G[MAX_K * MAX_K], R1[MAX_K * MAX_K], R2[MAX_K * MAX_K], R[MAX_K * MAX_K];
    double c1[MAX_K], c2[MAX_K], z[MAX_K], tmp[MAX_K];
    double res[PART_STRIDE];
    double braw, bnorm, res0, res_last, guess_res, inner_stop, mf, mb;
    int iters, restarts, converged, status, stop, done, jend, guess_rank, shifted, chol_ok;
};

// ---- reductions ----------------------------------------------------------

// One block: out[i] = sum over b < nb of part[i * nb + b], i < n (fixed order).
__device__ inline void reduce_parts(const double *part, int n, int nb, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < n; i += NWARPS) {
        // four independent accumulators keep four loads in flight per lane
        const double *pi = part + (size_t)i * nb;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int b = lane;
        for (; b + 96 < nb; b += 128) {
            s0 += pi[b];
            s1 += pi[b + 32];
            s2 += pi[b + 64];
            s3 += pi[b + 96];
        }
        for (; b < nb; b += 32) s0 += pi[b];
        double s = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[i] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ void zero32(double (&v)[32]) {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = 0.0;
}

// ---- operator kernels ------------------------------------------------------

__global__ void __launch_bounds__(NTHREADS) sk_geometry(Dev D, const double *ep, const double *ec) {
    geometry_columns(D, ep, ec, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

template <typename TI, int WM>
__global__ void __launch_bounds__(NTHREADS) sk_apply_vj(Dev D, Tiling tl, const TI *V, int j, const SState *ss,
                                                          TI *t) {
    if (ss->stop || ss->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TI *sp = reinterpret_cast<TI *>(smem_raw);
    TI *sq = sp + (size_t)D.P * tl.HW;
    LdVec<TI, TI> ld{V + (size_t)j * D.m, TI(ss->scale[j])};
    StVec<TI, TI> st{t};
    for (int tile = blockIdx.x; tile < tl.ntiles; tile += gridDim.x) apply_tile<TI, WM>(D, tl, tile, sp, sq, ld, st);
}

// The same apply in column-marching form (periodic grids with 10, 18 or 34
// levels; sw_colapply.cuh), one CX x CY tile per block.  Up to 18 levels in
// FP32 the kernel is held to 80 registers, three blocks per SM: 28.3 us per
// launch on the 512^2 x 17 field against 31.4 us at two blocks (128
// registers) and 31.1 us at four (64 registers, with spills).
template <typename TI, int P, bool TD>
__global__ void __launch_bounds__(NTHREADS, (P > 18 ? (sizeof(TI) == 4 ? 2 : 1) : (sizeof(TI) == 4 ? 3 : 2)))
    sk_apply_col(Dev D, ColXY<TI> xy, const TI *V, int j, const SState *ss, TI *t) {
    if (ss->stop || ss->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LdVec<TI, TI> ld{V + (size_t)j * D.m, TI(ss->scale[j])};
    StVec<TI, TI> st{t};
    col_apply_tile<TI, P, TD>(D, xy, blockIdx.x, smem_raw, ld, st);
}



template <typename TI, int P, bool TD>
static const void *col_kernel() { return (const void *)sk_apply_col<TI, P, TD>; }

// Kernel, grid and shared memory of the column-marching apply for this
// problem, or false when it does not serve the grid.
template <typename TI>
static bool col_launch_shape(const Dev &D, const void **k, int *grid, size_t *smem) {
    if (!colapply_ok(D, D.P)) return false;
    const bool td = D.three_d != 0;
    *grid = td ? (D.nx / ColShape<true>::CX) * (D.ny / ColShape<true>::CY) : D.nx / ColShape<false>::CX;
    switch (D.P) {
    case 10: *k = td ? col_kernel<TI, 10, true>() : col_kernel<TI, 10, false>();
             *smem = td ? ColGeom<TI, 10, true>::smem() : ColGeom<TI, 10, false>::smem(); break;
    case 18: *k = td ? col_kernel<TI, 18, true>() : col_kernel<TI, 18, false>();
             *smem = td ? ColGeom<TI, 18, true>::smem() : ColGeom<TI, 18, false>::smem(); break;
    default: *k = td ? col_kernel<TI, 34, true>() : col_kernel<TI, 34, false>();
             *smem = td ? ColGeom<TI, 34, true>::smem() : ColGeom<TI, 34, false>::smem(); break;
    }
    return *smem <= 227 * 1024;
}

struct Streamed;
template <typename TI> static const ColXY<TI> &xy_of(const Streamed *S);

template <typename TI>
static cudaError_t launch_col(const Problem *P, const TI *V, int j, const SState *ss, TI *t, cudaStream_t s) {
    const Dev &D = P->dev;
    const void *k = nullptr;
    int grid = 0;
    size_t smem = 0;
    if (!col_launch_shape<TI>(D, &k, &grid, &smem)) return cudaErrorInvalidValue;
    Dev Dc = D;
    ColXY<TI> xy = xy_of<TI>((const Streamed *)P->streamed);
    void *args[] = {&Dc, &xy, (void *)&V, &j, (void *)&ss, &t};
    return cudaLaunchKernel(k, dim3(grid), dim3(NTHREADS), args, smem, s);
}

// r = b - A x with per-block partial sums of r^2 in part[blockIdx.x]
template <int WM>
__global__ void __launch_bounds__(NTHREADS) sk_apply_resid(Dev D, Tiling tl, const double *x, const double *b,
                                                             double *r, double *part, const SState *ss,
                                                             int skip_when_done) {
    if (skip_when_done && ss->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[NWARPS * 32];
    double *sp = reinterpret_cast<double *>(smem_raw);
    double *sq = sp + (size_t)D.P * tl.HW;
    StResid st{b, r, 0.0};
    LdVec<double, double> ld{x, 1.0};
    for (int tile = blockIdx.x; tile < tl.ntiles; tile += gridDim.x) apply_tile<double, WM>(D, tl, tile, sp, sq, ld, st);
    double v[32];
    zero32(v);
    v[0] = st.acc;
    block_partials32(v, 1, red, part, gridDim.x);
}

// W_c = A (r Y_c + omega_c x_prev) or A Y_c, FP64
template <int WM>
__global__ void __launch_bounds__(NTHREADS) sk_apply_w(Dev D, Tiling tl, const double *Yc, const double *xprev,
                                                         double decay, double om, int upd, double *Wc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *sp = reinterpret_cast<double *>(smem_raw);
    double *sq = sp + (size_t)D.P * tl.HW;
    StVec<double, double> st{Wc};
    if (upd) {
        LdEwma<double, double> ld{Yc, xprev, decay, om};
        for (int tile = blockIdx.x; tile < tl.ntiles; tile += gridDim.x) apply_tile<double, WM>(D, tl, tile, sp, sq, ld, st);
    } else {
        LdVec<double, double> ld{Yc, 1.0};
        for (int tile = blockIdx.x; tile < tl.ntiles; tile += gridDim.x) apply_tile<double, WM>(D, tl, tile, sp, sq, ld, st);
    }
}

// ---- preconditioner kernels (one column group per launch) ----------------

template <typename TI, typename TIn, bool LOWER, int WM>
__global__ void __launch_bounds__(NTHREADS) sk_ilu_gather(Dev D, int c, const TIn *in, TI *out, const SState *ss,
                                                            int skip) {
    if (skip && (ss->stop || ss->done)) return;
    const long long rows = (long long)group_size<WM>(D, c) * D.P;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x)
        ilu_gather_row<TI, TIn, LOWER, WM>(D, c, r, in, out);
}

// periodic grids: one kernel per colour and layout, slot selection resolved at compile time
template <typename TI, typename TIn, bool LOWER, int L, int CC>
__global__ void __launch_bounds__(NTHREADS) sk_ilu_gather_cc(Dev D, const TIn *in, TI *out, const SState *ss,
                                                               int skip) {
    if (skip && (ss->stop || ss->done)) return;
    const long long rows = (long long)(D.ncol >> 2) * D.P;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x)
        ilu_gather_row_cc<L, TI, TIn, LOWER, CC>(D, r, in, out);
}

template <typename TI, typename TIn, bool LOWER, int L>
static void launch_gather_cc(const Dev &D, int c, int gb, const TIn *in, TI *out, const SState *ss, int skip,
                             cudaStream_t s) {
    switch (c) {
    case 0: sk_ilu_gather_cc<TI, TIn, LOWER, L, 0><<<gb, NTHREADS, 0, s>>>(D, in, out, ss, skip); break;
    case 1: sk_ilu_gather_cc<TI, TIn, LOWER, L, 1><<<gb, NTHREADS, 0, s>>>(D, in, out, ss, skip); break;
    case 2: sk_ilu_gather_cc<TI, TIn, LOWER, L, 2><<<gb, NTHREADS, 0, s>>>(D, in, out, ss, skip); break;
    default: sk_ilu_gather_cc<TI, TIn, LOWER, L, 3><<<gb, NTHREADS, 0, s>>>(D, in, out, ss, skip); break;
    }
}

template <typename TI, typename TIn, bool LOWER, int WM>
static void launch_gather(const Dev &D, int c, int gb, const TIn *in, TI *out, const SState *ss, int skip,
                          cudaStream_t s) {
    if (WM == 1) {
        sk_ilu_gather<TI, TIn, LOWER, WM><<<gb, NTHREADS, 0, s>>>(D, c, in, out, ss, skip);
        return;
    }
    switch (D.layout) {
    case CROSS2D: launch_gather_cc<TI, TIn, LOWER, CROSS2D>(D, c, gb, in, out, ss, skip, s); break;
    case BOX2D: launch_gather_cc<TI, TIn, LOWER, BOX2D>(D, c, gb, in, out, ss, skip, s); break;
    case CROSS3D: launch_gather_cc<TI, TIn, LOWER, CROSS3D>(D, c, gb, in, out, ss, skip, s); break;
    default: launch_gather_cc<TI, TIn, LOWER, BOX3D>(D, c, gb, in, out, ss, skip, s); break;
    }
}

template <typename TI, int WM>
__global__ void __launch_bounds__(NTHREADS) sk_ilu_product(Dev D, int c, TI *out, int upper, const SState *ss,
                                                             int skip) {
    if (skip && (ss->stop || ss->done)) return;
    const int lane = threadIdx.x & 31;
    const int per = group_size<WM>(D, c);
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < per; q += nw)
        ilu_column_product<TI, WM>(D, c, q, out, lane, upper != 0);
}

// ---- streaming vector kernels --------------------------------------------

template <typename TI>
__global__ void __launch_bounds__(NTHREADS) sk_norms_b(const double *b, const TI *t, long long m, double *part) {
    __shared__ double red[NWARPS * 32];
    double v[32];
    zero32(v);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m; p += (long long)gridDim.x * blockDim.x) {
        const double bb = b[p], tt = (double)t[p];
        v[0] += bb * bb;
        v[1] += tt * tt;
    }
    block_partials32(v, 2, red, part, gridDim.x);
}

// Range finder: column c of Y = X Omega over the Ke newest stored solutions
struct RrfCol {
    double w[SW_RRF_MAX_HISTORY];   // Omega[r][c], r-th newest solution
    int Ke, K, newest;
};
__global__ void __launch_bounds__(NTHREADS) sk_rrf_y(const double *ring, RrfCol rc, double *Yc, long long m) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m; p += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < rc.Ke; ++r) {
            const int slot = (rc.newest - r + rc.K) % rc.K;
            s += ring[(size_t)slot * m + p] * rc.w[r];
        }
        Yc[p] = s;
    }
}

__global__ void __launch_bounds__(NTHREADS) sk_ynew(const double *Yc, const double *xprev, double decay, double om,
                                                     double *Ync, long long m) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m; p += (long long)gridDim.x * blockDim.x)
        Ync[p] = decay * Yc[p] + om * xprev[p];
}

// Gram entries of W (first pass) or of Q1 = W R1^-1 (second pass), and W^T b / Q1^T b, in
// chunks of 32 values: part[(c0 + i) * nb + block]
__global__ void __launch_bounds__(NTHREADS) sk_gram(const double *Wm, const double *b, long long m, int k,
                                                     const SState *ss, int second, double *part) {
    __shared__ double red[NWARPS * 32];
    __shared__ unsigned char ga[PART_STRIDE], gb[PART_STRIDE];
    __shared__ double R1[MAX_K * MAX_K];
    if (second && !ss->chol_ok) return;
    if (threadIdx.x == 0) {
        int e = 0;
        for (int a = 0; a < k; ++a)
            for (int bb = a; bb < k; ++bb, ++e) { ga[e] = (unsigned char)a; gb[e] = (unsigned char)bb; }
    }
    for (int i = threadIdx.x; i < k * k; i += blockDim.x) R1[i] = ss->R1[i];
    __syncthreads();
    const int ng = k * (k + 1) / 2, nv = ng + k;
    for (int c0 = 0; c0 < nv; c0 += 32) {
        double v[32];
        zero32(v);
        for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m;
             p += (long long)gridDim.x * blockDim.x) {
            double q[MAX_K];
#pragma unroll
            for (int c = 0; c < MAX_K; ++c) {
                if (c >= k) { q[c] = 0.0; continue; }
                double s = Wm[(size_t)c * m + p];
                if (second) {
                    for (int i = 0; i < c; ++i) s -= q[i] * R1[i * k + c];
                    s = s / R1[c * k + c];
                }
                q[c] = s;
            }
            const double bp = b[p];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int e = c0 + i;
                if (e >= nv) break;
                v[i] += e < ng ? q[ga[e]] * q[gb[e]] : q[e - ng] * bp;
            }
        }
        block_partials32(v, min(32, nv - c0), red, part + (size_t)c0 * gridDim.x, gridDim.x);
    }
}

// V = Y R^-1 with R from CholeskyQR2 of the sketch (the optional QR step of
// Algorithms 3 and 4), or V = Y when its Gram matrix could not be factored
__global__ void __launch_bounds__(NTHREADS) sk_orth_v(const double *Y, const SState *ss, int k, double *Vq,
                                                       long long m) {
    __shared__ double R[MAX_K * MAX_K];
    for (int i = threadIdx.x; i < k * k; i += blockDim.x) R[i] = ss->R[i];
    __syncthreads();
    const bool ok = ss->chol_ok != 0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m; p += (long long)gridDim.x * blockDim.x) {
        double q[MAX_K];
#pragma unroll
        for (int c = 0; c < MAX_K; ++c) {
            if (c >= k) break;
            double sv = Y[(size_t)c * m + p];
            if (ok) {
                for (int i = 0; i < c; ++i) sv -= q[i] * R[i * k + c];
                sv /= R[c * k + c];
            }
            q[c] = sv;
            Vq[(size_t)c * m + p] = sv;
        }
    }
}

// x0 = Y z (EWMA), x_prev (previous solution) or 0 (cold start)
__global__ void __launch_bounds__(NTHREADS) sk_x0(const double *Y, const double *xprev, const SState *ss, int k,
                                                   int mode, double *x, long long m) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m; p += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        if (mode == SW_GUESS_EWMA || mode == SW_GUESS_RRF) {
            for (int c = 0; c < k; ++c) s += Y[(size_t)c * m + p] * ss->z[c];
        } else if (mode == SW_GUESS_PREVIOUS) {
            s = xprev[p];
        }
        x[p] = s;
    }
}

// ||V_0||^2 after the preconditioner: part[blockIdx.x]
template <typename TI>
__global__ void __launch_bounds__(NTHREADS) sk_norm(const TI *v0, long long m, double *part, const SState *ss) {
    __shared__ double red[NWARPS * 32];
    if (ss->done) return;
    double v[32];
    zero32(v);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m; p += (long long)gridDim.x * blockDim.x) {
        const double a = (double)v0[p];
        v[0] += a * a;
    }
    block_partials32(v, 1, red, part, gridDim.x);
}

// Sum of two compensated FP32 partial sums (s, c): TwoSum of the leading
// parts, both compensation terms carried (Ogita, Rump and Oishi 2005).
__device__ __forceinline__ void ds_add(float &s, float &c, float s2, float c2) {
    const float t = s + s2;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (s2 - bp);
    s = t;
    c = (c + c2) + e;
}

// Warp reduce-scatter of N compensated FP32 sums (N = 1, 2, 4, 8, 16 or 32):
// afterwards lane l holds the warp total of value l % N in s[0] + c[0].  The
// halving steps follow warp_reduce_scatter; the remaining lane bits are
// summed by plain butterflies.  Only FP32 instructions: the FP64 pipe of this
// chip issues one warp instruction per ~64 cycles per scheduler.
template <int N>
__device__ __forceinline__ void warp_reduce_scatter_ds(float (&s)[N], float (&c)[N], int lane) {
#pragma unroll
    for (int o = N / 2; o >= 1; o >>= 1) {
        const bool upper = lane & o;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float ss = upper ? s[i] : s[i + o], cs = upper ? c[i] : c[i + o];
            float ks = upper ? s[i + o] : s[i], kc = upper ? c[i + o] : c[i];
            const float rs = __shfl_xor_sync(0xffffffffu, ss, o);
            const float rc = __shfl_xor_sync(0xffffffffu, cs, o);
            ds_add(ks, kc, rs, rc);
            s[i] = ks;
            c[i] = kc;
        }
    }
#pragma unroll
    for (int o = N; o < 32; o <<= 1) {
        const float rs = __shfl_xor_sync(0xffffffffu, s[0], o);
        const float rc = __shfl_xor_sync(0xffffffffu, c[0], o);
        ds_add(s[0], c[0], rs, rc);
    }
}

// CGS2 pass 1 (d_i = V_i . w), pass 2 (w -= V h; d'_i = V_i . w) and pass 3
// (w -= V h'; ||w||^2), as in the persistent kernel: FP32 inner vectors use
// compensated products, the coefficient sums are FP64.  NJ >= j + 1 sizes the
// per-thread arrays, so short Arnoldi prefixes need few registers and the
// kernel keeps more warps resident.
//
// FP32 vectors are read VW points at a time (16-byte loads for VW = 4, 8-byte for VW = 2): a
// thread has NJ + 1 independent vector loads in flight per iteration.  The
// block's partial sums are reduced across each warp in compensated FP32
// (double-single) and only then converted to FP64, so the epilogue issues a
// handful of FP64 instructions per warp instead of a 32-value FP64 butterfly.
template <typename V4T, int VW> struct VecOf;
template <> struct VecOf<float4, 4> {
    __device__ static float get(const float4 &v, int u) { return u == 0 ? v.x : (u == 1 ? v.y : (u == 2 ? v.z : v.w)); }
    __device__ static void set(float4 &v, int u, float a) {
        if (u == 0) v.x = a; else if (u == 1) v.y = a; else if (u == 2) v.z = a; else v.w = a;
    }
    __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
template <> struct VecOf<float, 1> {
    __device__ static float get(const float &v, int) { return v; }
    __device__ static void set(float &v, int, float a) { v = a; }
    __device__ static float zero() { return 0.f; }
};
template <> struct VecOf<float2, 2> {
    __device__ static float get(const float2 &v, int u) { return u == 0 ? v.x : v.y; }
    __device__ static void set(float2 &v, int u, float a) { if (u == 0) v.x = a; else v.y = a; }
    __device__ static float2 zero() { return make_float2(0.f, 0.f); }
};

template <int PASS, int NJ, int VW>
__device__ __forceinline__ void cgs_f32_body(const float *V, int j, float *w, long long m, const float *hs32,
                                             Dot2f (&acc)[PASS == 3 ? 1 : NJ]) {
    using VT = typename std::conditional<VW == 4, float4, typename std::conditional<VW == 2, float2, float>::type>::type;
    using Op = VecOf<VT, VW>;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long mv = m / VW;
    const VT *Vv = reinterpret_cast<const VT *>(V);
    VT *wvp = reinterpret_cast<VT *>(w);
    for (long long p = t0; p < mv; p += stride) {
        VT vb[NJ];
#pragma unroll
        for (int i = 0; i < NJ; ++i) vb[i] = i <= j ? Vv[(size_t)i * mv + p] : Op::zero();
        VT wv = wvp[p];
        if (PASS > 1) {
#pragma unroll
            for (int i = 0; i < NJ; ++i) {
                if (i > j) break;
                const float h = -hs32[i];
#pragma unroll
                for (int u = 0; u < VW; ++u) Op::set(wv, u, fmaf(h, Op::get(vb[i], u), Op::get(wv, u)));
            }
            wvp[p] = wv;
        }
#pragma unroll
        for (int u = 0; u < VW; ++u) {
            const float wu = Op::get(wv, u);
            if (PASS == 3) {
                acc[0].add(wu, wu);
            } else {
#pragma unroll
                for (int i = 0; i < NJ; ++i) {
                    if (i > j) break;
                    acc[i].add(Op::get(vb[i], u), wu);
                }
            }
        }
    }
}

template <typename TI, int PASS, int NJ>
__global__ void __launch_bounds__(NTHREADS, (sizeof(TI) == 4 && NJ <= 16) ? 2 : 1) sk_cgs(const TI *V, int j, TI *w, long long m, const SState *ss,
                                                    double *part) {
    __shared__ double red[NWARPS * 32];
    __shared__ double hs[MAX_RESTART];
    __shared__ float hs32[MAX_RESTART];
    if (ss->stop || ss->done) return;
    if (threadIdx.x < MAX_RESTART) {
        hs[threadIdx.x] = ss->hs[threadIdx.x];
        hs32[threadIdx.x] = ss->hs32[threadIdx.x];
    }
    __syncthreads();
    constexpr int NA = PASS == 3 ? 1 : NJ;
    const long long stride = (long long)gridDim.x * blockDim.x;
    if constexpr (sizeof(TI) == 4) {
        Dot2f acc[NA];
        // the basis vectors start m points apart: with m a multiple of the
        // vector width (always so for the library's grids, where m is a
        // multiple of 4) every load is aligned; other m take single points
        constexpr int VWD = NJ <= 16 ? 4 : 2;
        if (m % VWD == 0) cgs_f32_body<PASS, NJ, VWD>((const float *)V, j, (float *)w, m, hs32, acc);
        else cgs_f32_body<PASS, NJ, 1>((const float *)V, j, (float *)w, m, hs32, acc);
        // block partials: compensated warp reduce-scatter, FP64 across warps
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        constexpr int NR = NA == 1 ? 1 : (NA <= 4 ? 4 : (NA <= 8 ? 8 : (NA <= 16 ? 16 : 32)));
        float rs[NR], rc[NR];
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            rs[i] = i < NA ? acc[i < NA ? i : 0].s : 0.f;
            rc[i] = i < NA ? acc[i < NA ? i : 0].c : 0.f;
        }
        warp_reduce_scatter_ds<NR>(rs, rc, lane);
        red[warp * 32 + lane] = (double)rs[0] + (double)rc[0];
        __syncthreads();
        const int n = PASS == 3 ? 1 : j + 1;
        if (warp == 0 && lane < n) {
            double t = 0.0;
            for (int w2 = 0; w2 < NWARPS; ++w2) t += red[w2 * 32 + lane];
            part[lane * gridDim.x + blockIdx.x] = t;
        }
    } else {
        double d[NA];
#pragma unroll
        for (int i = 0; i < NA; ++i) d[i] = 0.0;
        for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m; p += stride) {
            double vb[NJ];
#pragma unroll
            for (int i = 0; i < NJ; ++i) vb[i] = i <= j ? (double)V[(size_t)i * m + p] : 0.0;
            double wv = (double)w[p];
            if (PASS > 1) {
#pragma unroll
                for (int i = 0; i < NJ; ++i) {
                    if (i > j) break;
                    wv -= hs[i] * vb[i];
                }
                w[p] = TI(wv);
            }
            if (PASS == 3) {
                d[0] += wv * wv;
            } else {
#pragma unroll
                for (int i = 0; i < NA; ++i) {
                    if (i > j) break;
                    d[i] += vb[i] * wv;
                }
            }
        }
        double v[32];
        zero32(v);
#pragma unroll
        for (int i = 0; i < NA; ++i) v[i] = d[i];
        block_partials32(v, PASS == 3 ? 1 : j + 1, red, part, gridDim.x);
    }
}

// Launches one Gram-Schmidt pass and returns its number of blocks (the
// partial sums the control kernel then reduces).  FP32: per-thread arrays
// sized to the next multiple of four above j, so that the vector loads of a
// pass stay in registers, and as many blocks as stay resident at once (two
// per SM up to 16 basis vectors, one above: 128 registers or more), so a pass
// runs in one round and its control kernel reduces few partial sums.
template <typename TI, int PASS>
static int launch_cgs(const TI *V, int j, TI *w, long long m, const SState *ss, double *part, cudaStream_t s) {
    if constexpr (sizeof(TI) == 4) {
        const int nj = 4 * ((j + 4) / 4);
        const int nb = (nj <= 16 ? 2 : 1) * (SNB / 4);
        switch (nj / 4) {
        case 1: sk_cgs<TI, PASS, 4><<<nb, NTHREADS, 0, s>>>(V, j, w, m, ss, part); break;
        case 2: sk_cgs<TI, PASS, 8><<<nb, NTHREADS, 0, s>>>(V, j, w, m, ss, part); break;
        case 3: sk_cgs<TI, PASS, 12><<<nb, NTHREADS, 0, s>>>(V, j, w, m, ss, part); break;
        case 4: sk_cgs<TI, PASS, 16><<<nb, NTHREADS, 0, s>>>(V, j, w, m, ss, part); break;
        case 5: sk_cgs<TI, PASS, 20><<<nb, NTHREADS, 0, s>>>(V, j, w, m, ss, part); break;
        case 6: sk_cgs<TI, PASS, 24><<<nb, NTHREADS, 0, s>>>(V, j, w, m, ss, part); break;
        case 7: sk_cgs<TI, PASS, 28><<<nb, NTHREADS, 0, s>>>(V, j, w, m, ss, part); break;
        default: sk_cgs<TI, PASS, 32><<<nb, NTHREADS, 0, s>>>(V, j, w, m, ss, part); break;
        }
        return nb;
    } else {
        if (j < 4) sk_cgs<TI, PASS, 4><<<SNB, NTHREADS, 0, s>>>(V, j, w, m, ss, part);
        else if (j < 8) sk_cgs<TI, PASS, 8><<<SNB, NTHREADS, 0, s>>>(V, j, w, m, ss, part);
        else if (j < 16) sk_cgs<TI, PASS, 16><<<SNB, NTHREADS, 0, s>>>(V, j, w, m, ss, part);
        else sk_cgs<TI, PASS, 32><<<SNB, NTHREADS, 0, s>>>(V, j, w, m, ss, part);
        return SNB;
    }
}

// x += V y (y already carries the basis scales), FP64
template <typename TI>
__global__ void __launch_bounds__(NTHREADS) sk_update_x(double *x, const TI *V, long long m, const SState *ss) {
    __shared__ double y[MAX_RESTART];
    __shared__ int jend;
    if (threadIdx.x == 0) jend = ss->jend;
    if (threadIdx.x < MAX_RESTART) y[threadIdx.x] = ss->y[threadIdx.x];
    __syncthreads();
    if (jend == 0) return;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m; p += (long long)gridDim.x * blockDim.x) {
        double s = x[p];
        for (int i = 0; i < jend; ++i) s += y[i] * (double)V[(size_t)i * m + p];
        x[p] = s;
    }
}

__global__ void __launch_bounds__(NTHREADS) sk_final_x(double *x, double *xprev, double *ring_store, long long m,
                                                        const SState *ss) {
    const bool zero = ss->bnorm == 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m; p += (long long)gridDim.x * blockDim.x) {
        if (zero) x[p] = 0.0;
        xprev[p] = x[p];
        if (ring_store) ring_store[p] = x[p];
    }
}

// ---- one-block control kernels -------------------------------------------

struct CtlArgs {
    double tol, inner_rtol, md;
    int k, mr, max_restarts, guess_mode;
    CostModel cm;
    int isz;   // bytes of an inner-precision value
};

__device__ __forceinline__ void add_cost(SState *ss, const CtlArgs &c, double f, double b) {
    ss->mf += f * c.md;
    ss->mb += b * c.md;
}

__global__ void sk_ctl_bnorm(const double *part, int nb, SState *ss, CtlArgs c) {
    __shared__ double out[2];
    reduce_parts(part, 2, nb, out);
    if (threadIdx.x == 0) {
        ss->braw = sqrt(out[0]);
        ss->bnorm = sqrt(out[1]);
        ss->iters = 0;
        ss->restarts = 0;
        ss->converged = 0;
        ss->status = SW_ERR_NOT_CONVERGED;
        ss->stop = 1;
        ss->done = 0;
        ss->jend = 0;
        ss->guess_rank = -1;
        ss->shifted = 0;
        ss->chol_ok = 0;
        ss->res0 = ss->res_last = ss->guess_res = 0.0;
        ss->mf = 0.0;
        ss->mb = 0.0;
        add_cost(ss, c, c.cm.fM + 4.0, c.cm.bM + 8.0);
        for (int i = 0; i < MAX_K; ++i) ss->z[i] = 0.0;
        if (ss->bnorm == 0.0) {   // b = 0: x = 0 (written at the end), no iterations
            ss->converged = 1;
            ss->status = SW_OK;
            ss->done = 1;
        }
    }
}

// a9, step 1: G = W^T W, c1 = W^T b, Cholesky (shifted when not numerically SPD)
__global__ void sk_ctl_chol1(const double *part, int nb, SState *ss, CtlArgs c, long long m, int upd, int w_cost) {
    __shared__ double res[PART_STRIDE];
    const int k = c.k, ng = k * (k + 1) / 2, nv = ng + k;
    reduce_parts(part, nv, nb, res);
    if (threadIdx.x == 0) {
        if (upd) add_cost(ss, c, 3.0 * k, (2.0 * k + 1.0) * 8.0);
        if (w_cost) add_cost(ss, c, k * c.cm.fA, k * (c.cm.bA + 8.0));
        add_cost(ss, c, 2.0 * nv, (k + 1.0) * 8.0);
    }
    if (threadIdx.x < 32) {
        int e = 0;
        for (int a = 0; a < k; ++a)
            for (int b = a; b < k; ++b, ++e)
                if ((e & 31) == (int)threadIdx.x) {
                    ss->G[a * k + b] = res[e];
                    ss->G[b * k + a] = res[e];
                }
        for (int i = threadIdx.x; i < k; i += 32) ss->c1[i] = res[ng + i];
        __syncwarp();
        double tr = 0.0;
        for (int i = 0; i < k; ++i) tr += ss->G[i * k + i];
        for (int i = threadIdx.x; i < k * k; i += 32) ss->R[i] = ss->G[i];
        __syncwarp();
        bool ok = tr > 0.0 && warp_cholesky(ss->G, ss->R1, k);
        int shifted = 0;
        if (!ok && tr > 0.0) {
            double sh = 11.0 * ((double)m * k + (double)k * (k + 1)) * 1.1102230246251565e-16 * tr;
            for (int i = threadIdx.x; i < k * k; i += 32) ss->G[i] = ss->R[i] + ((i / k == i % k) ? sh : 0.0);
            __syncwarp();
            ok = warp_cholesky(ss->G, ss->R1, k);
            shifted = 1;
        }
        if (threadIdx.x == 0) {
            ss->chol_ok = ok ? 1 : 0;
            ss->shifted = shifted;
            if (!ok) ss->guess_rank = 0;
        }
    }
}

// a9, step 2: G2 = Q1^T Q1, c2 = Q1^T b; R = R2 R1 (or R1 if G2 is not SPD); z with the rank guard
__global__ void sk_ctl_chol2(const double *part, int nb, SState *ss, CtlArgs c) {
    __shared__ double res[PART_STRIDE];
    if (!ss->chol_ok) return;
    const int k = c.k, ng = k * (k + 1) / 2, nv = ng + k;
    reduce_parts(part, nv, nb, res);
    if (threadIdx.x == 0) add_cost(ss, c, (double)k * k + 2.0 * nv, (k + 1.0) * 8.0);
    if (threadIdx.x < 32) {
        int e = 0;
        for (int a = 0; a < k; ++a)
            for (int b = a; b < k; ++b, ++e)
                if ((e & 31) == (int)threadIdx.x) {
                    ss->G[a * k + b] = res[e];
                    ss->G[b * k + a] = res[e];
                }
        for (int i = threadIdx.x; i < k; i += 32) ss->c2[i] = res[ng + i];
        __syncwarp();
        bool ok2 = warp_cholesky(ss->G, ss->R2, k);
        if (!ok2) {
            for (int i = threadIdx.x; i < k * k; i += 32) ss->R[i] = ss->R1[i];
            __syncwarp();
            warp_fwdsub_t(ss->R1, ss->c1, ss->tmp, k);
        } else {
            for (int e2 = threadIdx.x; e2 < k * k; e2 += 32) {
                int a = e2 / k, bc = e2 % k;
                double s = 0.0;
                for (int l = a; l <= bc; ++l) s += ss->R2[a * k + l] * ss->R1[l * k + bc];
                ss->R[e2] = bc >= a ? s : 0.0;
            }
            __syncwarp();
            warp_fwdsub_t(ss->R2, ss->c2, ss->tmp, k);
        }
        double tiny = 1e-12 * fabs(ss->R[0]);
        warp_backsub(ss->R, ss->tmp, ss->z, k, tiny);
        if (threadIdx.x == 0) {
            int rk = 0;
            for (int j = 0; j < k; ++j) rk += fabs(ss->R[j * k + j]) > tiny;
            ss->guess_rank = rk;
        }
    }
}

__global__ void sk_ctl_guess_cost(SState *ss, CtlArgs c, int upd, int rrf_Ke) {
    if (threadIdx.x != 0) return;
    if (c.guess_mode == SW_GUESS_RRF) add_cost(ss, c, 2.0 * rrf_Ke * c.k, (rrf_Ke + c.k) * 8.0);
    if (c.guess_mode == SW_GUESS_EWMA || c.guess_mode == SW_GUESS_RRF) {
        add_cost(ss, c, 2.0 * c.k, c.k * 8.0 + 8.0);
    } else {
        if (upd) add_cost(ss, c, 3.0 * c.k, (2.0 * c.k + 1.0) * 8.0);
        if (c.guess_mode == SW_GUESS_PREVIOUS) add_cost(ss, c, 0.0, 16.0);
    }
}

// Start of a restart cycle: beta = ||M^-1 (b - A x)||, stop tests, reset of the Arnoldi state
__global__ void sk_ctl_cycle(const double *partA, int nbA, const double *partB, int nbB, SState *ss, CtlArgs c,
                             int cycle) {
    __shared__ double r2[1], b2[1];
    if (ss->done) return;
    reduce_parts(partA, 1, nbA, r2);
    reduce_parts(partB, 1, nbB, b2);
    if (threadIdx.x != 0) return;
    const double beta = sqrt(b2[0]);
    add_cost(ss, c, c.cm.fA + c.cm.fM + 4.0, c.cm.bA + c.cm.bM + 8.0);
    if (cycle == 0) {
        ss->res0 = beta / ss->bnorm;
        ss->guess_res = ss->braw > 0.0 ? sqrt(r2[0]) / ss->braw : sqrt(r2[0]);
    }
    ss->res_last = beta / ss->bnorm;
    ss->stop = 1;
    ss->jend = 0;
    if (!isfinite(beta)) { ss->status = SW_ERR_NAN; ss->done = 1; return; }
    if (beta <= c.tol * ss->bnorm) { ss->converged = 1; ss->status = SW_OK; ss->done = 1; return; }
    if (cycle == c.max_restarts + 1) { ss->done = 1; return; }
    if (cycle > 0) ss->restarts++;
    ss->inner_stop = fmax(c.tol * ss->bnorm, c.inner_rtol * beta);
    ss->scale[0] = 1.0 / beta;
    for (int i = 0; i <= c.mr; ++i) ss->g[i] = 0.0;
    ss->g[0] = beta;
    ss->stop = 0;
}

// Hessenberg column from pass 1 (PASS 1) or its correction from pass 2 (PASS 2)
template <int PASS>
__global__ void sk_ctl_h(const double *part, int nb, int j, SState *ss) {
    __shared__ double res[MAX_RESTART];
    if (ss->stop || ss->done) return;
    reduce_parts(part, j + 1, nb, res);
    if (threadIdx.x < MAX_RESTART) {
        const int i = threadIdx.x;
        const double hi = i <= j ? res[i] * ss->scale[i] : 0.0;
        if (i <= j) {
            if (PASS == 1) ss->H[i * MAX_RESTART + j] = hi;
            else ss->H[i * MAX_RESTART + j] += hi;
        }
        ss->hs[i] = i <= j ? hi * ss->scale[i] : 0.0;
        ss->hs32[i] = (float)ss->hs[i];
    }
}

// a5: norm of the new vector, Givens rotations, residual estimate, stop test
__global__ void sk_ctl_givens(const double *part, int nb, int j, SState *ss, CtlArgs c) {
    __shared__ double res[1];
    if (ss->stop || ss->done) return;
    reduce_parts(part, 1, nb, res);
    if (threadIdx.x != 0) return;
    const double hn = sqrt(res[0]);
    ss->scale[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
    double *Hc = ss->H;
    for (int i = 0; i < j; ++i) {
        const double a = Hc[i * MAX_RESTART + j], bb = Hc[(i + 1) * MAX_RESTART + j];
        Hc[i * MAX_RESTART + j] = ss->cs[i] * a + ss->sn[i] * bb;
        Hc[(i + 1) * MAX_RESTART + j] = -ss->sn[i] * a + ss->cs[i] * bb;
    }
    const double a = Hc[j * MAX_RESTART + j];
    const double den = hypot(a, hn);
    ss->cs[j] = a / den;
    ss->sn[j] = hn / den;
    Hc[j * MAX_RESTART + j] = den;
    ss->g[j + 1] = -ss->sn[j] * ss->g[j];
    ss->g[j] = ss->cs[j] * ss->g[j];
    add_cost(ss, c, c.cm.fA + c.cm.fM + 8.0 * (j + 1) + 2.0, c.cm.bA + c.cm.bM + (3.0 * j + 8.0) * (double)c.isz);
    ss->iters++;
    ss->jend = j + 1;
    if ((fabs(ss->g[j + 1]) <= ss->inner_stop) || hn == 0.0 || j + 1 == c.mr) ss->stop = 1;
}

// a6: y = R^-1 g (scaled by the basis scales) for the update x += V y
__global__ void sk_ctl_y(SState *ss, CtlArgs c) {
    if (ss->done || threadIdx.x >= 32) return;
    const int jend = ss->jend;
    const int lane = threadIdx.x;
    double acc = lane < jend ? ss->g[lane] : 0.0;
    for (int i = jend - 1; i >= 0; --i) {
        const double yi = __shfl_sync(0xffffffffu, acc, i) / ss->H[i * MAX_RESTART + i];
        if (lane == i) ss->y[i] = yi * ss->scale[i];
        if (lane < i) acc -= ss->H[lane * MAX_RESTART + i] * yi;
    }
    if (lane == 0) add_cost(ss, c, 2.0 * jend, jend * (double)c.isz + 16.0);
}

__global__ void sk_ctl_final(const double *partA, int nbA, SState *ss, CtlArgs c, DevStats *stats, int guess_only) {
    __shared__ double r2[1];
    if (!guess_only) reduce_parts(partA, 1, nbA, r2);
    if (threadIdx.x != 0) return;
    DevStats &st = *stats;
    if (guess_only) {
        st.guess_rank = ss->guess_rank;
        st.cholesky_shift = ss->shifted;
        return;
    }
    const double true_res = ss->braw > 0.0 ? sqrt(r2[0]) / ss->braw : sqrt(r2[0]);
    add_cost(ss, c, c.cm.fA + 3.0, c.cm.bA + 24.0);
    if (ss->bnorm == 0.0) { ss->converged = 1; ss->status = SW_OK; }
    st.iterations = ss->iters;
    st.restarts = ss->restarts;
    st.converged = ss->converged;
    st.status = ss->status;
    st.res0 = ss->res0;
    st.res_final = ss->res_last;
    st.true_res = true_res;
    st.guess_res = ss->guess_res;
    st.bnorm = ss->bnorm;
    st.braw = ss->braw;
    st.guess_rank = ss->guess_rank;
    st.guess_mode = c.guess_mode;
    st.cholesky_shift = ss->shifted;
    st.total_iterations += ss->iters;
    st.model_flops += ss->mf;
    st.model_bytes += ss->mb;
}

// ---- host side -------------------------------------------------------------

struct Streamed {
    bool col = false;                            // Arnoldi apply in column-marching form (autotuned)
    cudaGraphExec_t cycle = nullptr;             // the Arnoldi steps of one restart cycle
    long long cycle_kernels = 0;
    SState *ss = nullptr;
    double *partA = nullptr, *partB = nullptr;   // apply-grid partials, streaming partials
    int *h_done = nullptr;                       // pinned flag read once per cycle
    Tiling tl{};
    int nbA = 0;
    ColXY<float> xy32{};                         // x / y weights of the column-marching apply
    ColXY<double> xy64{};
    void *ltri = nullptr, *utri = nullptr;       // packed inverse blocks (periodic grids)
};

template <> const ColXY<float> &xy_of<float>(const Streamed *S) { return S->xy32; }
template <> const ColXY<double> &xy_of<double>(const Streamed *S) { return S->xy64; }

static Tiling st_tiling(const Dev &D) {
    // as for the standalone operator: at least 304 tiles, at most 64 columns wide
    Tiling t{};
    if (!D.three_d) {
        int TX = 64;
        while (TX > 4 && (D.nx % TX != 0 || D.nx / TX < 304)) TX >>= 1;
        t.TX = TX;
        t.TY = 1;
    } else {
        int TX = 16, TY = 8;
        while ((size_t)(TX + 6) * (TY + 6) * D.P * 2 * sizeof(double) > 150 * 1024 && TX > 4) {
            if (TX > TY) TX >>= 1; else TY >>= 1;
        }
        while (D.nx % TX) TX >>= 1;
        while (D.ny % TY) TY >>= 1;
        t.TX = TX;
        t.TY = TY;
    }
    t.HX = t.TX + 2 * HALF;
    t.HY = D.three_d ? t.TY + 2 * HALF : 1;
    t.HW = t.HX * t.HY;
    t.ntx = D.nx / t.TX;
    t.nty = D.three_d ? D.ny / t.TY : 1;
    t.ntiles = t.ntx * t.nty;
    return t;
}

template <typename TC>
static size_t tile_smem(const Dev &D, const Tiling &t) { return 2 * (size_t)D.P * t.HW * sizeof(TC); }

template <typename TI, int WM>
static cudaError_t set_smem_attrs(const Dev &D, const Tiling &t) {
    cudaError_t e = ensure_smem((const void *)sk_apply_vj<TI, WM>, (size_t)(int)tile_smem<TI>(D, t));
    if (e == cudaSuccess)
        e = ensure_smem((const void *)sk_apply_resid<WM>, (size_t)(int)tile_smem<double>(D, t));
    if (e == cudaSuccess)
        e = ensure_smem((const void *)sk_apply_w<WM>, (size_t)(int)tile_smem<double>(D, t));
    return e;
}

static Tiling tiling_with(const Dev &D, int TX, int TY) {
    Tiling t{};
    t.TX = TX;
    t.TY = D.three_d ? TY : 1;
    t.HX = t.TX + 2 * HALF;
    t.HY = D.three_d ? t.TY + 2 * HALF : 1;
    t.HW = t.HX * t.HY;
    t.ntx = D.nx / t.TX;
    t.nty = D.three_d ? D.ny / t.TY : 1;
    t.ntiles = t.ntx * t.nty;
    return t;
}

// Tile autotuner: time the Arnoldi operator kernel (the precision the solves
// use) for every admissible tile shape on the problem's own buffers, three
// launches each after one warm-up, and keep the fastest.  The tile shape
// changes no output value, only the staging of the halos.
template <typename TI, int WM>
static Tiling tune_tiles(Problem *P) {
    const Dev &D = P->dev;
    Streamed *S = (Streamed *)P->streamed;
    Tiling best = st_tiling(D);
    std::vector<std::pair<int, int>> cand;
    if (!D.three_d) {
        for (int TX : {8, 16, 32, 64}) cand.push_back({TX, 1});
    } else {
        for (int TX : {8, 16, 32})
            for (int TY : {4, 8, 16}) cand.push_back({TX, TY});
    }
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) { (void)cudaGetLastError(); return best; }
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    TI *V = P->params.precision == SW_PRECISION_MIXED ? (TI *)P->d_V32 : (TI *)P->d_V;
    TI *tw = (TI *)(P->d_work + P->m);
    float best_ms = 1e30f;
    for (auto &c : cand) {
        if (D.nx % c.first || (D.three_d && D.ny % c.second)) continue;
        Tiling t = tiling_with(D, c.first, c.second);
        const size_t sm = tile_smem<TI>(D, t);
        if (sm > 200 * 1024 || t.ntiles < 152) continue;
        if (ensure_smem((const void *)sk_apply_vj<TI, WM>, (size_t)(int)sm) !=
            cudaSuccess) { (void)cudaGetLastError(); continue; }
        sk_apply_vj<TI, WM><<<t.ntiles, NTHREADS, sm, cs>>>(D, t, V, 0, S->ss, tw);
        cudaEventRecord(a, cs);
        for (int r = 0; r < 3; ++r) sk_apply_vj<TI, WM><<<t.ntiles, NTHREADS, sm, cs>>>(D, t, V, 0, S->ss, tw);
        cudaEventRecord(b, cs);
        if (cudaEventSynchronize(b) != cudaSuccess) { (void)cudaGetLastError(); continue; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best_ms) { best_ms = ms; best = t; }
    }
    // the column-marching form competes with the best tile shape
    {
        const void *k = nullptr;
        int grid = 0;
        size_t smc = 0;
        if (WM == 0 && col_launch_shape<TI>(D, &k, &grid, &smc) &&
            ensure_smem((const void *)k, (size_t)(int)smc) == cudaSuccess) {
            bool ok = launch_col<TI>(P, V, 0, S->ss, tw, cs) == cudaSuccess;
            ok = ok && cudaEventRecord(a, cs) == cudaSuccess;
            for (int r = 0; r < 3 && ok; ++r) ok = launch_col<TI>(P, V, 0, S->ss, tw, cs) == cudaSuccess;
            ok = ok && cudaEventRecord(b, cs) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess;
            float ms = 0.f;
            if (ok && cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms < best_ms) {
                best_ms = ms;
                S->col = true;
            }
        }
        (void)cudaGetLastError();
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(cs);
    (void)cudaGetLastError();
    return best;
}

// Write the constant-memory sigma weights of the column form for P's number of
// levels (once per device and P; every problem with those levels has the same
// weights, so a later write would store the same values).
static cudaError_t colapply_set_weights(const Problem *P) {
    static std::mutex mu;
    static std::set<std::pair<int, int>> done;
    const int nl = P->dev.P;
    if (nl != 10 && nl != 18 && nl != 34) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({dev, nl})) return cudaSuccess;
    double wx1[W], wx2[W], wy1[W], wy2[W];
    std::vector<double> ws(2 * (size_t)nl * W);
    std::vector<int> win(nl);
    grid_weights(P->grid, wx1, wx2, wy1, wy2, ws.data(), ws.data() + (size_t)nl * W, win.data());
    std::vector<float> ws32(ws.begin(), ws.end());
    const int off = nl == 10 ? colw_off<10>() : (nl == 18 ? colw_off<18>() : colw_off<34>());
    e = cudaMemcpyToSymbol(c_colw64, ws.data(), ws.size() * sizeof(double), off * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbol(c_colw32, ws32.data(), ws32.size() * sizeof(float), off * sizeof(float));
    if (e == cudaSuccess) done.insert({dev, nl});
    return e;
}

int setup_streamed(Problem *P) {
    Streamed *S = new (std::nothrow) Streamed();
    if (!S) { set_error("out of host memory"); return SW_ERR_BAD_ARG; }
    P->streamed = S;
    const Dev &D = P->dev;
    S->tl = st_tiling(D);
    S->nbA = S->tl.ntiles < SNB ? S->tl.ntiles : SNB;
    cudaError_t e = cudaMalloc((void **)&S->ss, sizeof(SState));
    if (e == cudaSuccess) { P->allocs.push_back(S->ss); e = cudaMemset(S->ss, 0, sizeof(SState)); }
    if (e == cudaSuccess) e = cudaMalloc((void **)&S->partA, (size_t)SNB * 2 * sizeof(double));
    if (e == cudaSuccess) P->allocs.push_back(S->partA);
    if (e == cudaSuccess) e = cudaMalloc((void **)&S->partB, (size_t)SNB * PART_STRIDE * sizeof(double));
    if (e == cudaSuccess) P->allocs.push_back(S->partB);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&S->h_done, sizeof(int));
    if (e == cudaSuccess && !D.walls) e = colapply_set_weights(P);
    {
        double wx1[W], wx2[W], wy1[W], wy2[W];
        std::vector<double> ws(2 * (size_t)D.P * W);
        std::vector<int> win(D.P);
        grid_weights(P->grid, wx1, wx2, wy1, wy2, ws.data(), ws.data() + (size_t)D.P * W, win.data());
        for (int t = 0; t < W; ++t) {
            S->xy64.wx1[t] = wx1[t]; S->xy64.wx2[t] = wx2[t]; S->xy64.wy1[t] = wy1[t]; S->xy64.wy2[t] = wy2[t];
            S->xy32.wx1[t] = (float)wx1[t]; S->xy32.wx2[t] = (float)wx2[t];
            S->xy32.wy1[t] = (float)wy1[t]; S->xy32.wy2[t] = (float)wy2[t];
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "streamed executor set-up");
    // periodic grids: packed triangles of the in-column inverse blocks (built
    // once on the device from the dense blocks)
    if (!D.walls) {
        const bool f32 = P->params.precision == SW_PRECISION_MIXED;
        const size_t es = f32 ? sizeof(float) : sizeof(double);
        {
            const size_t bytes = (size_t)D.ncol * tri_stride(D.P) * es;
            void *lt = nullptr, *ut = nullptr;
            e = cudaMalloc(&lt, bytes);
            if (e == cudaSuccess) { P->allocs.push_back(lt); e = cudaMalloc(&ut, bytes); }
            if (e == cudaSuccess) { P->allocs.push_back(ut); e = cudaMemset(lt, 0, bytes); }
            if (e == cudaSuccess) e = cudaMemset(ut, 0, bytes);
            if (e == cudaSuccess) {
                if (f32) sk_pack_tri<float><<<4 * 152, NTHREADS>>>(D.linv32, D.uinv32, D.P, D.ncol, (float *)lt, (float *)ut);
                else sk_pack_tri<double><<<4 * 152, NTHREADS>>>(D.linv64, D.uinv64, D.P, D.ncol, (double *)lt, (double *)ut);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_fail(e, "packed inverse blocks");
            S->ltri = lt;
            S->utri = ut;
        }
    }
    {
        const bool f32 = P->params.precision == SW_PRECISION_MIXED;
        if (D.walls) S->tl = f32 ? tune_tiles<float, 1>(P) : tune_tiles<double, 1>(P);
        else S->tl = f32 ? tune_tiles<float, 0>(P) : tune_tiles<double, 0>(P);
        S->nbA = S->tl.ntiles < SNB ? S->tl.ntiles : SNB;
    }
    if (D.walls) {
        e = set_smem_attrs<double, 1>(D, S->tl);
        if (e == cudaSuccess) e = set_smem_attrs<float, 1>(D, S->tl);
    } else {
        e = set_smem_attrs<double, 0>(D, S->tl);
        if (e == cudaSuccess) e = set_smem_attrs<float, 0>(D, S->tl);
    }
    if (e != cudaSuccess) return cuda_fail(e, "streamed kernel attributes");
    return SW_OK;
}

void destroy_streamed(Problem *P) {
    Streamed *S = (Streamed *)P->streamed;
    if (!S) return;
    if (S->h_done) cudaFreeHost(S->h_done);
    if (S->cycle) cudaGraphExecDestroy(S->cycle);
    delete S;
    P->streamed = nullptr;
}

// In-column products of colour c with the packed blocks (periodic grids)
template <typename TI>
static void launch_product_tri(const Problem *P, int c, bool upper, TI *out, const SState *ss, int skip,
                               cudaStream_t s) {
    const Dev &D = P->dev;
    const Streamed *S = (const Streamed *)P->streamed;
    const int per = D.ncol >> 2;
    const int pb = (per * 32 + NTHREADS - 1) / NTHREADS;
    const TI *tri = (const TI *)(upper ? S->utri : S->ltri);
#define SW_TRI_LAUNCH(PC)                                                                                      \
    do {                                                                                                       \
        if (upper) sk_ilu_product_tri<TI, false, PC, SState><<<pb, NTHREADS, 0, s>>>(D, c, tri, out, ss, skip); \
        else sk_ilu_product_tri<TI, true, PC, SState><<<pb, NTHREADS, 0, s>>>(D, c, tri, out, ss, skip);        \
    } while (0)
    switch (D.P) {
    case 10: SW_TRI_LAUNCH(10); break;
    case 18: SW_TRI_LAUNCH(18); break;
    case 34: SW_TRI_LAUNCH(34); break;
    default: SW_TRI_LAUNCH(0); break;
    }
#undef SW_TRI_LAUNCH
}

// ILU application out = U^-1 L^-1 in (row-parallel gathers, per-column
// products; on periodic grids the products read the packed triangles)
template <typename TI, typename TIn, int WM>
static void st_ilu(const Problem *P, const TIn *in, TI *out, const SState *ss, int skip, cudaStream_t s) {
    const Dev &D = P->dev;
    // host code: D.walls here, never the device-only walls_of
    const bool tri = !D.walls && ((const Streamed *)P->streamed)->ltri;
    const int ng = D.ngroups;
    for (int c = 0; c < ng; ++c) {
        const int per = P->goff_h[c + 1] - P->goff_h[c];
        const long long rows = (long long)per * D.P;
        const int gb = (int)((rows + NTHREADS - 1) / NTHREADS);
        const int pb = (per * 32 + NTHREADS - 1) / NTHREADS;
        launch_gather<TI, TIn, true, WM>(D, c, gb, in, out, ss, skip, s);
        if (tri) launch_product_tri<TI>(P, c, false, out, ss, skip, s);
        else sk_ilu_product<TI, WM><<<pb, NTHREADS, 0, s>>>(D, c, out, 0, ss, skip);
    }
    for (int c = ng - 1; c >= 0; --c) {
        const int per = P->goff_h[c + 1] - P->goff_h[c];
        const long long rows = (long long)per * D.P;
        const int gb = (int)((rows + NTHREADS - 1) / NTHREADS);
        const int pb = (per * 32 + NTHREADS - 1) / NTHREADS;
        if (c < ng - 1) launch_gather<TI, TI, false, WM>(D, c, gb, out, out, ss, skip, s);
        if (tri) launch_product_tri<TI>(P, c, true, out, ss, skip, s);
        else sk_ilu_product<TI, WM><<<pb, NTHREADS, 0, s>>>(D, c, out, 1, ss, skip);
    }
}

// The restart length's Arnoldi steps; every kernel reads only problem-owned
// buffers, so the sequence is captured once per problem and replayed.
template <typename TI, int WM>
static long long enqueue_cycle(const Problem *P, TI *V, TI *tw, SState *ss, double *partB, const CtlArgs &c,
                               cudaStream_t s) {
    const Dev &D = P->dev;
    const Streamed *S = (const Streamed *)P->streamed;
    const Tiling &tl = S->tl;
    const long long m = D.m;
    const size_t smI = tile_smem<TI>(D, tl);
    long long n = 0;
    for (int j = 0; j < P->params.restart; ++j) {
        TI *w = V + (size_t)(j + 1) * m;
        if (S->col) launch_col<TI>(P, V, j, ss, tw, s);
        else sk_apply_vj<TI, WM><<<tl.ntiles, NTHREADS, smI, s>>>(D, tl, V, j, ss, tw);
        st_ilu<TI, TI, WM>(P, tw, w, ss, 1, s);
        const int nb1 = launch_cgs<TI, 1>(V, j, w, m, ss, partB, s);
        sk_ctl_h<1><<<1, NTHREADS, 0, s>>>(partB, nb1, j, ss);
        const int nb2 = launch_cgs<TI, 2>(V, j, w, m, ss, partB, s);
        sk_ctl_h<2><<<1, NTHREADS, 0, s>>>(partB, nb2, j, ss);
        const int nb3 = launch_cgs<TI, 3>(V, j, w, m, ss, partB, s);
        sk_ctl_givens<<<1, NTHREADS, 0, s>>>(partB, nb3, j, ss, c);
        n += 6 + 4 * D.ngroups;   // operator, 4 ngroups - 1 ILU launches, 3 passes, 3 control kernels
    }
    return n;
}

template <typename TI, int WM>
static int build_cycle_graph(Problem *P, TI *V, TI *tw, const CtlArgs &c) {
    Streamed *S = (Streamed *)P->streamed;
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "capture stream");
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    long long n = 0;
    if (e == cudaSuccess) {
        n = enqueue_cycle<TI, WM>(P, V, tw, S->ss, S->partB, c, cs);
        e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&S->cycle, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        S->cycle = nullptr;
        return cuda_fail(e, "restart-cycle graph");
    }
    S->cycle_kernels = n;
    return SW_OK;
}

template <typename TI, int WM>
static int st_solve(Problem *P, const SolveArgs &A, cudaStream_t s) {
    Streamed *S = (Streamed *)P->streamed;
    const Dev &D = P->dev;
    const long long m = D.m;
    const Tiling &tl = S->tl;
    const size_t smI = tile_smem<TI>(D, tl), smD = tile_smem<double>(D, tl);
    SState *ss = S->ss;
    TI *V = reinterpret_cast<TI *>(A.V);
    TI *tw = reinterpret_cast<TI *>(A.t);
    const int k = A.k, mr = A.restart;
    CtlArgs c{A.tol, A.inner_rtol, (double)m, k, mr, A.max_restarts, A.guess_mode, A.cm, (int)sizeof(TI)};
    const int gc = (D.ncol + NTHREADS - 1) / NTHREADS;
    long long launches = 0;
    // a1: geometry of the stage pair
    sk_geometry<<<gc, NTHREADS, 0, s>>>(D, A.eta_prev, A.eta_cur);
    // reference norms ||b|| and ||M^-1 b||
    st_ilu<TI, double, WM>(P, A.b, tw, ss, 0, s);
    sk_norms_b<TI><<<SNB, NTHREADS, 0, s>>>(A.b, tw, m, S->partB);
    sk_ctl_bnorm<<<1, NTHREADS, 0, s>>>(S->partB, SNB, ss, c);
    launches += 2 + 4 * D.ngroups;   // geometry, 4 ngroups - 1 ILU launches, norms, control
    // a7-a10: guess
    const int upd = A.pending;
    if (A.guess_mode == SW_GUESS_RRF) {
        for (int cc = 0; cc < k; ++cc) {
            RrfCol rc{};
            for (int r = 0; r < A.ring_Ke; ++r) rc.w[r] = A.omega_rrf[r * k + cc];
            rc.Ke = A.ring_Ke;
            rc.K = A.ring_K;
            rc.newest = A.ring_newest;
            double *Ync = A.Ynew + (size_t)cc * m;
            sk_rrf_y<<<SNB, NTHREADS, 0, s>>>(A.ring, rc, Ync, m);
            ++launches;
            if (!A.Vq) {
                sk_apply_w<WM><<<tl.ntiles, NTHREADS, smD, s>>>(D, tl, Ync, A.xprev, 0.0, 0.0, 0, A.Wm + (size_t)cc * m);
                ++launches;
            }
        }
    } else if (upd || A.guess_mode == SW_GUESS_EWMA) {
        for (int cc = 0; cc < k; ++cc) {
            const double *Yc = A.Yold + (size_t)cc * m;
            double *Ync = A.Ynew + (size_t)cc * m;
            if (upd) { sk_ynew<<<SNB, NTHREADS, 0, s>>>(Yc, A.xprev, A.decay, A.omega[cc], Ync, m); ++launches; }
            if (A.guess_mode == SW_GUESS_EWMA && !A.Vq) {
                sk_apply_w<WM><<<tl.ntiles, NTHREADS, smD, s>>>(D, tl, Yc, A.xprev, A.decay, A.omega[cc], upd,
                                                                 A.Wm + (size_t)cc * m);
                ++launches;
            }
        }
    }
    const double *Ycur = (A.pending || A.guess_mode == SW_GUESS_RRF) ? A.Ynew : A.Yold;
    const bool orth = A.Vq && (A.guess_mode == SW_GUESS_EWMA || A.guess_mode == SW_GUESS_RRF);
    if (orth) {
        // the optional QR step of Algorithms 3 and 4: CholeskyQR2 of Y, V = Y R^-1, then W = A V
        sk_gram<<<SNB, NTHREADS, 0, s>>>(Ycur, A.b, m, k, ss, 0, S->partB);
        sk_ctl_chol1<<<1, NTHREADS, 0, s>>>(S->partB, SNB, ss, c, m, upd, 1);
        sk_gram<<<SNB, NTHREADS, 0, s>>>(Ycur, A.b, m, k, ss, 1, S->partB);
        sk_ctl_chol2<<<1, NTHREADS, 0, s>>>(S->partB, SNB, ss, c);
        sk_orth_v<<<SNB, NTHREADS, 0, s>>>(Ycur, ss, k, A.Vq, m);
        for (int cc = 0; cc < k; ++cc)
            sk_apply_w<WM><<<tl.ntiles, NTHREADS, smD, s>>>(D, tl, A.Vq + (size_t)cc * m, A.xprev, 0.0, 0.0, 0,
                                                             A.Wm + (size_t)cc * m);
        launches += 5 + k;
        Ycur = A.Vq;
    }
    if (A.guess_mode == SW_GUESS_EWMA || A.guess_mode == SW_GUESS_RRF) {
        sk_gram<<<SNB, NTHREADS, 0, s>>>(A.Wm, A.b, m, k, ss, 0, S->partB);
        sk_ctl_chol1<<<1, NTHREADS, 0, s>>>(S->partB, SNB, ss, c, m, orth ? 0 : upd, orth ? 0 : 1);
        sk_gram<<<SNB, NTHREADS, 0, s>>>(A.Wm, A.b, m, k, ss, 1, S->partB);
        sk_ctl_chol2<<<1, NTHREADS, 0, s>>>(S->partB, SNB, ss, c);
        launches += 4;
    }
    sk_x0<<<SNB, NTHREADS, 0, s>>>(Ycur, A.xprev, ss, k, A.guess_mode, A.x, m);
    sk_ctl_guess_cost<<<1, 32, 0, s>>>(ss, c, upd, A.ring_Ke);
    launches += 2;
    if (A.guess_only) {
        sk_ctl_final<<<1, NTHREADS, 0, s>>>(S->partA, S->nbA, ss, c, A.stats, 1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "streamed guess launch");
        P->launches += launches + 1;
        return SW_OK;
    }
    // restarted GMRES: one host synchronisation per cycle
    for (int cycle = 0; cycle <= A.max_restarts + 1; ++cycle) {
        sk_apply_resid<WM><<<S->nbA, NTHREADS, smD, s>>>(D, tl, A.x, A.b, A.r, S->partA, ss, 1);
        st_ilu<TI, double, WM>(P, A.r, V, ss, 0, s);
        sk_norm<TI><<<SNB, NTHREADS, 0, s>>>(V, m, S->partB, ss);
        sk_ctl_cycle<<<1, NTHREADS, 0, s>>>(S->partA, S->nbA, S->partB, SNB, ss, c, cycle);
        cudaError_t e = cudaMemcpyAsync(S->h_done, &ss->done, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "streamed cycle");
        launches += 2 + 4 * D.ngroups;   // residual, 4 ngroups - 1 ILU launches, norm, control
        if (*S->h_done) break;
        // the Arnoldi steps of the cycle: one graph launch (the kernels of the
        // steps after the stop test return at once)
        if (!S->cycle) {
            // the Arnoldi steps use only the per-problem fields of the control arguments
            CtlArgs cg = c;
            cg.guess_mode = 0;
            cg.tol = 0.0;
            cg.inner_rtol = 0.0;
            int rc = build_cycle_graph<TI, WM>(P, V, tw, cg);
            if (rc != SW_OK) return rc;
        }
        e = cudaGraphLaunch(S->cycle, s);
        if (e != cudaSuccess) return cuda_fail(e, "restart-cycle graph launch");
        launches += S->cycle_kernels;
        sk_ctl_y<<<1, 32, 0, s>>>(ss, c);
        sk_update_x<TI><<<SNB, NTHREADS, 0, s>>>(A.x, V, m, ss);
        launches += 2;
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "streamed cycle launch");
    }
    // true residual ||b - A x|| / ||b|| in FP64; the solution is kept for the next guess
    sk_final_x<<<SNB, NTHREADS, 0, s>>>(A.x, A.xprev, A.ring_store, m, ss);
    sk_apply_resid<WM><<<S->nbA, NTHREADS, smD, s>>>(D, tl, A.x, A.b, A.r, S->partA, ss, 0);
    sk_ctl_final<<<1, NTHREADS, 0, s>>>(S->partA, S->nbA, ss, c, A.stats, 0);
    launches += 3;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "streamed final launch");
    P->launches += launches;
    return SW_OK;
}

int solve_streamed(Problem *P, const SolveArgs &A, cudaStream_t s) {
    const bool f32 = P->params.precision == SW_PRECISION_MIXED;
    if (P->dev.walls) return f32 ? st_solve<float, 1>(P, A, s) : st_solve<double, 1>(P, A, s);
    return f32 ? st_solve<float, 0>(P, A, s) : st_solve<double, 0>(P, A, s);
}

}  // namespace sw

// ---- profiling aid: the hot kernels of an Arnoldi step, timed alone --------

namespace sw {

// Time one class of launches: flush L2 (write `flush`), record, launch, record;
// reps times after one untimed round; returns the mean in microseconds.
template <class Launch>
static double time_launches(cudaStream_t s, void *flush, size_t flush_bytes, int reps, Launch launch) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return -1.0;
    double tot = 0.0;
    for (int r = 0; r <= reps; ++r) {
        cudaMemsetAsync(flush, r & 0xff, flush_bytes, s);
        cudaEventRecord(a, s);
        launch();
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess) { tot = -1.0; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (r > 0) tot += ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return tot < 0.0 ? -1.0 : 1e3 * tot / reps;
}

template <typename TI, int WM>
static int profile_streamed(Problem *P, int reps, double *us, int n) {
    Streamed *S = (Streamed *)P->streamed;
    const Dev &D = P->dev;
    const long long m = D.m;
    TI *V = P->params.precision == SW_PRECISION_MIXED ? (TI *)P->d_V32 : (TI *)P->d_V;
    TI *tw = (TI *)(P->d_work + m);
    TI *w = V + (size_t)11 * m;
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "profiling stream");
    // control state of a running cycle: every kernel does its work
    SState saved, run;
    e = cudaMemcpy(&saved, S->ss, sizeof(SState), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { cudaStreamDestroy(s); return cuda_fail(e, "profiling state"); }
    run = saved;
    run.stop = 0;
    run.done = 0;
    for (int i = 0; i <= MAX_RESTART; ++i) run.scale[i] = 1.0;
    for (int i = 0; i < MAX_RESTART; ++i) { run.hs[i] = 0.0; run.hs32[i] = 0.f; }
    e = cudaMemcpy(S->ss, &run, sizeof(SState), cudaMemcpyHostToDevice);
    const size_t fb = (size_t)256 << 20;
    void *flush = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&flush, fb);
    if (e != cudaSuccess) { cudaStreamDestroy(s); return cuda_fail(e, "profiling set-up"); }
    const Tiling &tl = S->tl;
    const size_t smI = tile_smem<TI>(D, tl);
    const int ng = D.ngroups;
    double t[8];
    t[0] = time_launches(s, flush, fb, reps, [&] {
        if (S->col) launch_col<TI>(P, V, 0, S->ss, tw, s);
        else sk_apply_vj<TI, WM><<<tl.ntiles, NTHREADS, smI, s>>>(D, tl, V, 0, S->ss, tw);
    });
    const bool tri = !D.walls && S->ltri;
    t[1] = time_launches(s, flush, fb, reps, [&] {
        for (int c = 0; c < ng; ++c) {
            const long long rows = (long long)(P->goff_h[c + 1] - P->goff_h[c]) * D.P;
            launch_gather<TI, TI, true, WM>(D, c, (int)((rows + NTHREADS - 1) / NTHREADS), tw, w, S->ss, 0, s);
        }
    });
    t[2] = time_launches(s, flush, fb, reps, [&] {
        for (int up = 0; up < 2; ++up)
            for (int c = 0; c < ng; ++c) {
                const int per = P->goff_h[c + 1] - P->goff_h[c];
                if (tri) launch_product_tri<TI>(P, c, up != 0, w, S->ss, 0, s);
                else sk_ilu_product<TI, WM><<<(per * 32 + NTHREADS - 1) / NTHREADS, NTHREADS, 0, s>>>(D, c, w, up, S->ss, 0);
            }
    });
    t[3] = time_launches(s, flush, fb, reps, [&] {
        for (int c = ng - 2; c >= 0; --c) {
            const long long rows = (long long)(P->goff_h[c + 1] - P->goff_h[c]) * D.P;
            launch_gather<TI, TI, false, WM>(D, c, (int)((rows + NTHREADS - 1) / NTHREADS), w, w, S->ss, 0, s);
        }
    });
    t[4] = time_launches(s, flush, fb, reps, [&] { launch_cgs<TI, 1>(V, 10, w, m, S->ss, S->partB, s); });
    t[5] = time_launches(s, flush, fb, reps, [&] { launch_cgs<TI, 2>(V, 10, w, m, S->ss, S->partB, s); });
    t[6] = time_launches(s, flush, fb, reps, [&] { launch_cgs<TI, 3>(V, 10, w, m, S->ss, S->partB, s); });
    t[7] = time_launches(s, flush, fb, reps, [&] { st_ilu<TI, TI, WM>(P, tw, w, S->ss, 0, s); });
    e = cudaStreamSynchronize(s);
    cudaFree(flush);
    cudaError_t e2 = cudaMemcpy(S->ss, &saved, sizeof(SState), cudaMemcpyHostToDevice);
    cudaStreamDestroy(s);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "profiling");
    for (int i = 0; i < n && i < 8; ++i) us[i] = t[i];
    return SW_OK;
}

}  // namespace sw

using namespace sw;

extern "C" int sw_profile_kernels(sw_problem *pp, int reps, double *us, int n) {
    Problem *P = (Problem *)pp;
    if (!P || !us || n < 1 || reps < 1) { set_error("bad argument"); return SW_ERR_BAD_ARG; }
    if (P->exec != SW_EXEC_STREAMED || !P->streamed) {
        set_error("kernel profiling needs a problem on the streamed executor");
        return SW_ERR_BAD_ARG;
    }
    if (P->n_solves < 1) { set_error("kernel profiling needs one solve first"); return SW_ERR_BAD_ARG; }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "profiling sync");
    const bool f32 = P->params.precision == SW_PRECISION_MIXED;
    if (P->dev.walls) return f32 ? profile_streamed<float, 1>(P, reps, us, n) : profile_streamed<double, 1>(P, reps, us, n);
    return f32 ? profile_streamed<float, 0>(P, reps, us, n) : profile_streamed<double, 0>(P, reps, us, n);
}

extern "C" int sw_autotuned_apply(sw_problem *pp, int *column_form, int *tile_x, int *tile_y) {
    Problem *P = (Problem *)pp;
    if (!P || !column_form || !tile_x || !tile_y) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    if (P->exec != SW_EXEC_STREAMED || !P->streamed) { set_error("not on the streamed executor"); return SW_ERR_BAD_ARG; }
    Streamed *S = (Streamed *)P->streamed;
    *column_form = S->col ? 1 : 0;
    *tile_x = S->col ? (P->dev.three_d ? ColShape<true>::CX : ColShape<false>::CX) : S->tl.TX;
    *tile_y = S->col ? (P->dev.three_d ? ColShape<true>::CY : ColShape<false>::CY) : S->tl.TY;
    return SW_OK;
}

extern "C" int sw_set_apply_form(sw_problem *pp, int column_form) {
    Problem *P = (Problem *)pp;
    if (!P || (column_form != 0 && column_form != 1)) { set_error("bad argument"); return SW_ERR_BAD_ARG; }
    if (P->exec != SW_EXEC_STREAMED || !P->streamed) { set_error("not on the streamed executor"); return SW_ERR_BAD_ARG; }
    Streamed *S = (Streamed *)P->streamed;
    if (column_form) {
        const bool f32 = P->params.precision == SW_PRECISION_MIXED;
        const void *k = nullptr;
        int grid = 0;
        size_t smem = 0;
        const bool ok = !P->dev.walls && (f32 ? col_launch_shape<float>(P->dev, &k, &grid, &smem)
                                              : col_launch_shape<double>(P->dev, &k, &grid, &smem));
        if (!ok) { set_error("the column-marching operator does not serve this grid"); return SW_ERR_BAD_ARG; }
        cudaError_t e = ensure_smem((const void *)k, (size_t)(int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "column apply attribute");
    }
    S->col = column_form != 0;
    if (S->cycle) {   // the restart cycle is captured again at the next solve
        cudaGraphExecDestroy(S->cycle);
        S->cycle = nullptr;
    }
    return SW_OK;
}
