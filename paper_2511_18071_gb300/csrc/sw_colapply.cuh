// Column-marching form of the matrix-free operator y = A(eta^(i-1), eta^(i)) p
// (Eq. 16-18) for periodic grids with a compile-time number of levels P
// (the streamed executor's large problems).
//
// One thread per column of a CX x CY tile.  The tile and its three-column halo
// are staged in shared memory plane by plane (coalesced rows along x); each
// thread keeps its own column's P values in registers.  It then marches up
// its column: at level m it forms D_x p and D_xx p (and D_y p, D_yy p) from
// the six neighbours in shared memory, and finishes every row whose sigma
// window (compile-time: clamp(l - 3, 0, P - 7)) ends at m.  The sigma
// derivatives are taken along the column from registers, with the sigma
// weights as constant-memory operands; the mixed derivatives D_x D_sigma p
// are formed as D_sigma (D_x p), the same tensor-product stencil applied in
// the other order (equal in exact arithmetic, different rounding), so a level
// needs twelve shared-memory loads and the tile one staging pass.  The row
// formulas follow apply_tile_t (sw_device.cuh) term by term.
#pragma once
#include "sw_device.cuh"

namespace sw {

// The sigma weights of the column form live in constant memory, one table per
// precision and number of levels: on the uniform sigma grid they depend on P
// alone, so every problem with P levels writes the same values (at set-up,
// before the first launch that reads them; colapply_set_weights).  With the
// level and window position known at compile time, the multiply-adds take
// them as constant-bank operands instead of loading them from shared memory.
// Layout per P: first derivative P x W, then second derivative P x W.
__constant__ float c_colw32[2 * (10 + 18 + 34) * W];
__constant__ double c_colw64[2 * (10 + 18 + 34) * W];

template <int P>
__host__ __device__ constexpr int colw_off() { return P == 10 ? 0 : (P == 18 ? 2 * 10 * W : 2 * (10 + 18) * W); }

template <typename T, int P>
__device__ __forceinline__ T colw(int d, int l, int k) {
    if constexpr (sizeof(T) == 8) return c_colw64[colw_off<P>() + d * P * W + l * W + k];
    else return c_colw32[colw_off<P>() + d * P * W + l * W + k];
}

// The x and y weights of a problem, passed by value as a kernel argument (and
// by value on to the tile routine: no address of it is ever taken, which would
// make the compiler copy it to local memory): kernel arguments sit in a
// constant bank, so the multiply-adds read them as operands.
template <typename T>
struct ColXY {
    T wx1[W], wx2[W], wy1[W], wy2[W];
};

template <bool TD> struct ColShape;
template <> struct ColShape<true> { static constexpr int CX = 32, CY = 8; };    // 3-D: 32 x 8 columns
template <> struct ColShape<false> { static constexpr int CX = 256, CY = 1; };  // 2-D: 256 columns

template <typename T, int P, bool TD>
struct ColGeom {
    static constexpr int CX = ColShape<TD>::CX, CY = ColShape<TD>::CY;
    static constexpr int HX = CX + 2 * HALF, HY = TD ? CY + 2 * HALF : 1;
    static constexpr int HW = HX * HY;
    // halo positions a row needs: three rows above and below the tile (interior
    // x only) and three columns left and right of it (interior y only); the
    // corners are never read.  At most one per thread.
    static constexpr int NHALO = TD ? 2 * HALF * CX + 2 * HALF * CY : 2 * HALF;
    static_assert(NHALO <= CX * CY, "one halo column per thread");
    static constexpr size_t smem() { return (size_t)HW * P * sizeof(T); }
};

// whether the column-marching operator serves this grid
__host__ __device__ inline bool colapply_ok(const Dev &D, int P) {
    if (D.walls || (P != 10 && P != 18 && P != 34)) return false;
    if (D.three_d) return D.nx % ColShape<true>::CX == 0 && D.ny % ColShape<true>::CY == 0;
    return D.nx % ColShape<false>::CX == 0;
}

template <typename T, int P, bool TD, class Loader, class Store>
__device__ inline void col_apply_tile(const Dev &D, const ColXY<T> xy, int tile, unsigned char *smem, Loader &ld,
                                      Store &st) {
    using G = ColGeom<T, P, TD>;
    constexpr int CX = G::CX, CY = G::CY, HX = G::HX, HW = G::HW;
    T *sp = reinterpret_cast<T *>(smem);
    const int tid = threadIdx.x;
    const int ntx = D.nx / CX;
    const int tx0 = (tile % ntx) * CX, ty0 = (tile / ntx) * CY;
    const int n = D.ncol;
    // positions of this thread: its own column, then at most one halo column
    const int txo = tid % CX, tyo = tid / CX;
    const int own = (tyo + (TD ? HALF : 0)) * HX + txo + HALF;
    const int gxo = tx0 + txo, gyo = ty0 + tyo;
    const int gco = gyo * D.nx + gxo;
    int hpos = -1, hcol = -1;
    if (tid < G::NHALO) {
        int a, b;
        if (TD) {
            if (tid < 2 * HALF * CX) {          // rows 0..2 and CY+3..CY+5, x inside the tile
                const int r = tid / CX;
                a = HALF + tid % CX;
                b = r < HALF ? r : r + CY;
            } else {                            // columns 0..2 and CX+3..CX+5, y inside the tile
                const int mq = tid - 2 * HALF * CX, e = mq % (2 * HALF);
                b = HALF + mq / (2 * HALF);
                a = e < HALF ? e : CX + e;
            }
        } else {
            b = 0;
            a = tid < HALF ? tid : CX + tid;
        }
        hpos = b * HX + a;
        const int gx = wrapi(tx0 + a - HALF, D.nx);
        const int gy = TD ? wrapi(ty0 + b - HALF, D.ny) : 0;
        hcol = gy * D.nx + gx;
    }
    // stage p
    T pc[P], ph[P];
#pragma unroll
    for (int l = 0; l < P; ++l) {
        pc[l] = ld((long long)l * n + gco);
        if (hpos >= 0) ph[l] = ld((long long)l * n + hcol);
    }
#pragma unroll
    for (int l = 0; l < P; ++l) {
        sp[l * HW + own] = pc[l];
        if (hpos >= 0) sp[l * HW + hpos] = ph[l];
    }
    __syncthreads();
    // the column's transform coefficients
    const T *cc = Prec<T>::cc(D);
    const T ap0 = cc[CC_AP0 * n + gco], ap1 = cc[CC_AP1 * n + gco];
    const T axp0 = cc[CC_AXP0 * n + gco], axp1 = cc[CC_AXP1 * n + gco];
    const T bp0 = cc[CC_BP0 * n + gco], bp1 = cc[CC_BP1 * n + gco];
    const T ef = cc[CC_EF * n + gco];
    const T gs = cc[CC_GS * n + gco], gxc = cc[CC_GX * n + gco];
    T gyc = T(0), ay0 = T(0), ay1 = T(0), ayy0 = T(0), ayy1 = T(0), by0 = T(0), by1 = T(0);
    if (TD) {
        gyc = cc[CC_GY * n + gco];
        ay0 = cc[CC_AY0 * n + gco];
        ay1 = cc[CC_AY1 * n + gco];
        ayy0 = cc[CC_AYY0 * n + gco];
        ayy1 = cc[CC_AYY1 * n + gco];
        by0 = cc[CC_BY0 * n + gco];
        by1 = cc[CC_BY1 * n + gco];
    }
    const T inv_nzm1 = T(1) / T(D.nz - 1);
    constexpr int LAST = P - W;
    // Level by level, upwards: D_x p and D_xx p (and y) at level m from the
    // six neighbours in shared memory; a row l is finished as soon as the
    // last level of its sigma window is in, its mixed derivatives taken as
    // D_sigma (D_x p) along the column (the tensor-product stencils commute).
    T px[P] = {}, py[P] = {}, pxx[P] = {}, pyy[P] = {};
    auto finish = [&](int l) {
        const int s0 = l - HALF < 0 ? 0 : (l - HALF > LAST ? LAST : l - HALF);
        T y;
        if (l == P - 1) {
            y = pc[l];
        } else if (l == 0) {
            T q1 = T(0);
            constexpr int s1 = 1 - HALF < 0 ? 0 : (1 - HALF > LAST ? LAST : 1 - HALF);
#pragma unroll
            for (int k = 0; k < W; ++k) q1 += colw<T, P>(0, 1, k) * pc[s1 + k];
            y = gs * q1 + gxc * px[1];
            if (TD) y += gyc * py[1];
        } else {
            const T sg = T(l - 1) * inv_nzm1;
            const T aa = ap0 - sg * ap1;
            const T bb = bp0 - sg * bp1;
            const T ax = axp0 - sg * axp1 - aa * ap1;
            const T c_xs = aa + bb;
            T c_ss = aa * bb + ef;
            const T c_s = ax - bb * ap1;
            T ql = T(0), pxs = T(0), pss = T(0);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                ql += colw<T, P>(0, l, k) * pc[s0 + k];
                pxs += colw<T, P>(0, l, k) * px[s0 + k];
                pss += colw<T, P>(1, l, k) * pc[s0 + k];
            }
            y = pxx[l] + c_xs * pxs + c_s * ql;
            if (TD) {
                const T ay = ay0 - sg * ay1;
                const T by = by0 - sg * by1;
                const T ayy = ayy0 - sg * ayy1 - ay * ay1;
                c_ss += ay * by;
                const T c_ys = ay + by;
                const T c_sy = ayy - by * ay1;
                T pys = T(0);
#pragma unroll
                for (int k = 0; k < W; ++k) pys += colw<T, P>(0, l, k) * py[s0 + k];
                y += pyy[l] + c_ys * pys + c_sy * ql;
            }
            y += c_ss * pss;
        }
        st((long long)l * n + gco, y);
    };
#pragma unroll
    for (int mlev = 0; mlev < P; ++mlev) {
        const T *pl = sp + mlev * HW + own;
        T a1 = T(0), a2 = T(0), b1 = T(0), b2 = T(0);
#pragma unroll
        for (int t = -HALF; t <= HALF; ++t) {
            const T vx = t == 0 ? pc[mlev] : pl[t];
            a1 += xy.wx1[t + HALF] * vx;
            a2 += xy.wx2[t + HALF] * vx;
            if (TD) {
                const T vy = t == 0 ? pc[mlev] : pl[t * HX];
                b1 += xy.wy1[t + HALF] * vy;
                b2 += xy.wy2[t + HALF] * vy;
            }
        }
        px[mlev] = a1;
        pxx[mlev] = a2;
        py[mlev] = b1;
        pyy[mlev] = b2;
        // rows whose window ends at this level: the surface row at once, the
        // ghost row with D_x p of level 1, rows 1..3 (window 0..6) at level 6,
        // interior rows l at l + 3, rows P-4..P-2 (window P-7..P-1) at the top
        if (mlev == 0) finish(P - 1);
        if (mlev == 1) finish(0);
        if (mlev == W - 1) {
#pragma unroll
            for (int l = 1; l <= HALF; ++l) finish(l);
        }
        if (mlev >= W && mlev <= P - 2) finish(mlev - HALF);
        if (mlev == P - 1) {
#pragma unroll
            for (int l = P - 1 - HALF; l <= P - 2; ++l) finish(l);
        }
    }
    __syncthreads();
}

}  // namespace sw
