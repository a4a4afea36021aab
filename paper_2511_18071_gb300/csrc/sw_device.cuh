// Device building blocks of the solver: column geometry, the matrix-free
// mixed-stage operator, the colour-ordered ILU(0) sweeps and grid reductions.
//
// FP64 on this GPU issues one warp instruction per ~32 ns per SM sub-partition
// whatever the number of active lanes, so the code below counts FP64 warp
// instructions rather than lanes: sums over many values are done with a
// reduce-scatter across lanes (about one add per value per warp) instead of a
// shuffle tree per value (five adds per value).
#pragma once
#include <cooperative_groups.h>

#include "sw_internal.cuh"

namespace sw {
namespace cg = cooperative_groups;

constexpr int NTHREADS = 256;
constexpr int NWARPS = NTHREADS / 32;
constexpr int NCC = 19;   // per-column coefficients written by the geometry step
constexpr int PART_STRIDE = 160;  // values per block in the partial-sum buffer

// Column coefficient slots (each an array of ncol doubles in Dev::gp).
enum {
    CC_F = 0,      // 1/d at stage i-1
    CC_E,          // 1/d at stage i
    CC_EF,         // e f
    CC_AP0,        // h_x f           (sigma_x^(i-1) = AP0 - sigma AP1)
    CC_AP1,        // d_x^(i-1) f
    CC_AXP0,       // h_xx f          (d sigma_x^(i-1)/d chi = AXP0 - sigma AXP1 - sigma_x AP1)
    CC_AXP1,       // d_xx^(i-1) f
    CC_BP0,        // h_x e           (sigma_x^(i) = BP0 - sigma BP1)
    CC_BP1,        // d_x^(i) e
    CC_GS,         // ghost row: coefficient of D_sigma p at the bed
    CC_GX,         // ghost row: coefficient of D_chi p at the bed
    CC_GY,         // ghost row: coefficient of D_gamma p at the bed
    CC_AY0, CC_AY1, CC_AYY0, CC_AYY1, CC_BY0, CC_BY1,  // y counterparts (3-D)
    CC_GN          // ghost row: -1/|(h_x, h_y, 1)|, the vertical component of the unit normal
};

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Walls: first column of the x window of an unknown of the linear system at
// column ix (ghost columns included), and of surface data / velocities at the
// physical column ixp (1..nx-2).  ixp of a ghost column is its wall column.
__device__ __forceinline__ int xwin_field(const Dev &D, int ix) { return min(max(ix - HALF, 0), D.nx - W); }
__device__ __forceinline__ int phys_col(const Dev &D, int ix) { return min(max(ix, 1), D.nx - 2); }
__device__ __forceinline__ int xwin_phys(const Dev &D, int ixp) { return min(max(ixp - HALF, 1), D.nx - 1 - W); }

// ---------------------------------------------------------------------------
// a1: geometry.  For eta^(i-1) and eta^(i): d = h + eta, its surface
// derivatives with the fixed 7-point operators (Sec. 3), and the per-column
// factors of sigma_x, sigma_y and 1/d used by every row (Eq. 13b-13d).
// ---------------------------------------------------------------------------
// Coefficients of column c (ghost columns of a walled grid take their wall
// column's); out[k] is coefficient k of the CC_* list.
__device__ inline void column_coefs(const Dev &D, const double *eta_prev, const double *eta_cur, int c,
                                    double (&out)[NCC]) {
    // x window: centred and periodic, or (walls, 2-D) over the physical
    // columns; a ghost column takes the coefficients of its wall column
    int ix = c % D.nx;
    const int iy = c / D.nx;
    int xs0 = ix - HALF;
    const double *w1 = D.wx1, *w2 = D.wx2;
    if (D.walls) {
        ix = phys_col(D, ix);
        xs0 = xwin_phys(D, ix);
        w1 = D.wxo1 + (ix - xs0) * W;
        w2 = D.wxo2 + (ix - xs0) * W;
    }
    const int ce = iy * D.nx + ix;   // column the coefficients are evaluated at
    double dp1 = 0, dp2 = 0, dc1 = 0, dpy1 = 0, dpy2 = 0, dcy1 = 0;
#pragma unroll
    for (int t = -HALF; t <= HALF; ++t) {
        int gx = xs0 + t + HALF;
        if (!D.walls) gx = wrapi(gx, D.nx);
        int cx = iy * D.nx + gx;
        double vp = D.h[cx] + eta_prev[cx];
        double vc = D.h[cx] + eta_cur[cx];
        dp1 += w1[t + HALF] * vp;
        dp2 += w2[t + HALF] * vp;
        dc1 += w1[t + HALF] * vc;
        if (D.three_d) {
            int cy = wrapi(iy + t, D.ny) * D.nx + ix;
            double wp = D.h[cy] + eta_prev[cy];
            double wc = D.h[cy] + eta_cur[cy];
            dpy1 += D.wy1[t + HALF] * wp;
            dpy2 += D.wy2[t + HALF] * wp;
            dcy1 += D.wy1[t + HALF] * wc;
        }
    }
    double dp = D.h[ce] + eta_prev[ce], dcu = D.h[ce] + eta_cur[ce];
    double f = 1.0 / dp, e = 1.0 / dcu;
    double hx = D.hx[ce], hy = D.three_d ? D.hy[ce] : 0.0;
    const double hxx = D.hxx[ce], hyy = D.three_d ? D.hyy[ce] : 0.0;
    out[CC_F] = f;
    out[CC_E] = e;
    out[CC_EF] = e * f;
    out[CC_AP0] = hx * f;
    out[CC_AP1] = dp1 * f;
    out[CC_AXP0] = hxx * f;
    out[CC_AXP1] = dp2 * f;
    out[CC_BP0] = hx * e;
    out[CC_BP1] = dc1 * e;
    // ghost row n . grad^(i-1) p at sigma = 0 with n = -(h_x, h_y, 1)/|(h_x, h_y, 1)|
    double nrm = 1.0 / sqrt(1.0 + hx * hx + hy * hy);
    out[CC_GS] = -nrm * (hx * hx * f + hy * hy * f + f);
    out[CC_GX] = -nrm * hx;
    out[CC_GY] = -nrm * hy;
    out[CC_GN] = -nrm;
    out[CC_AY0] = hy * f;
    out[CC_AY1] = dpy1 * f;
    out[CC_AYY0] = hyy * f;
    out[CC_AYY1] = dpy2 * f;
    out[CC_BY0] = hy * e;
    out[CC_BY1] = dcy1 * e;
}

__device__ inline void geometry_columns(const Dev &D, const double *eta_prev, const double *eta_cur, int tid,
                                        int nth) {
    double *cc = D.gp;
    const int n = D.ncol;
    for (int c = tid; c < n; c += nth) {
        double v[NCC];
        column_coefs(D, eta_prev, eta_cur, c, v);
        const int nc = D.three_d ? NCC : CC_GN + 1;
        for (int k = 0; k < nc; ++k) cc[k * n + c] = v[k];
        if (D.gp32)
            for (int k = 0; k < nc; ++k) D.gp32[k * n + c] = (float)v[k];
    }
}

// Weights and per-column coefficients in the arithmetic precision of the caller.
template <typename T> struct Prec;
template <> struct Prec<double> {
    __device__ static const double *wxo1(const Dev &D) { return D.wxo1; }
    __device__ static const double *wxo2(const Dev &D) { return D.wxo2; }
    __device__ static const double *wx1(const Dev &D) { return D.wx1; }
    __device__ static const double *wx2(const Dev &D) { return D.wx2; }
    __device__ static const double *wy1(const Dev &D) { return D.wy1; }
    __device__ static const double *wy2(const Dev &D) { return D.wy2; }
    __device__ static const double *ws1(const Dev &D) { return D.ws1; }
    __device__ static const double *ws2(const Dev &D) { return D.ws2; }
    __device__ static const double *cc(const Dev &D) { return D.gp; }
};
template <> struct Prec<float> {
    __device__ static const float *wxo1(const Dev &D) { return D.w32 + 4 * W + 2 * D.P * W; }
    __device__ static const float *wxo2(const Dev &D) { return D.w32 + 4 * W + 2 * D.P * W + W * W; }
    __device__ static const float *wx1(const Dev &D) { return D.w32; }
    __device__ static const float *wx2(const Dev &D) { return D.w32 + W; }
    __device__ static const float *wy1(const Dev &D) { return D.w32 + 2 * W; }
    __device__ static const float *wy2(const Dev &D) { return D.w32 + 3 * W; }
    __device__ static const float *ws1(const Dev &D) { return D.w32 + 4 * W; }
    __device__ static const float *ws2(const Dev &D) { return D.w32 + 4 * W + D.P * W; }
    __device__ static const float *cc(const Dev &D) { return D.gp32; }
};

// ---------------------------------------------------------------------------
// a2: matrix-free operator y = A(eta^(i-1), eta^(i)) p (Eq. 16-18).
// One tile = TX x TY columns, all levels.  p and q = D_sigma p are staged in
// shared memory for the tile plus a 3-column halo, so each q value is computed
// once and reused by the 7 rows that need it for the mixed derivative
// D_chi D_sigma.  Interior rows:
//   p_xx + p_yy + (a+b) p_xs + (a'+b') p_ys + (a b + a' b' + e f) p_ss
//        + (a_x + b a_s + a'_y + b' a'_s) p_s
// with a = sigma_x^(i-1), b = sigma_x^(i) (the chain rule applied to the
// push-forward of Eq. 9b); ghost rows the Neumann condition of Eq. (17) at the
// bed; surface rows the identity (p = 0 on the free surface).
// ---------------------------------------------------------------------------
struct Tiling {
    int TX, TY, HX, HY, HW, ntx, nty, ntiles;
};

template <typename T, bool WALLS, int TD, class Loader, class Store>
__device__ inline void apply_tile_t(const Dev &D, const Tiling &tl, int tile, T *sp, T *sq, Loader &ld, Store &st) {
    const int P = D.P, HX = tl.HX, HY = tl.HY, HW = tl.HW;
    const bool td = TD == 0 ? D.three_d != 0 : TD == 2;
    const int tx0 = (tile % tl.ntx) * tl.TX;
    const int ty0 = (tile / tl.ntx) * tl.TY;
    const int tid = threadIdx.x;
    // stage p on tile + halo
    for (int idx = tid; idx < P * HW; idx += blockDim.x) {
        int l = idx / HW, r = idx - l * HW;
        int a = r % HX, b = r / HX;
        bool hxo = a < HALF || a >= HX - HALF;
        bool hyo = td && (b < HALF || b >= HY - HALF);
        T v = T(0);
        int gx = tx0 + a - HALF;
        if (WALLS) {
            // no wrap: the shifted windows next to a wall never reach outside [0, nx)
            if (gx >= 0 && gx < D.nx) v = ld((long long)l * D.ncol + gx);
        } else if (!(hxo && hyo)) {
            gx = wrapi(gx, D.nx);
            int gy = td ? wrapi(ty0 + b - HALF, D.ny) : 0;
            v = ld((long long)l * D.ncol + gy * D.nx + gx);
        }
        sp[idx] = v;
    }
    __syncthreads();
    // q = D_sigma p on tile + halo
    const T *ws1 = Prec<T>::ws1(D), *ws2 = Prec<T>::ws2(D);
    const T *wx1 = Prec<T>::wx1(D), *wx2 = Prec<T>::wx2(D), *wy1 = Prec<T>::wy1(D), *wy2 = Prec<T>::wy2(D);
    for (int idx = tid; idx < P * HW; idx += blockDim.x) {
        int l = idx / HW, r = idx - l * HW;
        const T *w1 = ws1 + l * W;
        int base = (D.win[l] + 1) * HW + r;
        T s = T(0);
#pragma unroll
        for (int k = 0; k < W; ++k) s += w1[k] * sp[base + k * HW];
        sq[idx] = s;
    }
    __syncthreads();
    const int n = D.ncol;
    const T inv_nzm1 = T(1) / T(D.nz - 1);
    const T *cc = Prec<T>::cc(D);
    for (int idx = tid; idx < P * tl.TX * tl.TY; idx += blockDim.x) {
        int l = idx / (tl.TX * tl.TY), r = idx - l * (tl.TX * tl.TY);
        int a = r % tl.TX + HALF, b = td ? r / tl.TX + HALF : 0;
        int gx = tx0 + a - HALF, gy = td ? ty0 + b - HALF : 0;
        int c = gy * D.nx + gx;
        int hr = b * HX + a;
        long long node = (long long)l * n + c;
        // x window of the row: positions t = 0..6 at shared-memory offsets
        // x0 + t from the row's column, weights of the evaluation point
        int x0 = -HALF;
        const T *wa1 = wx1, *wa2 = wx2;
        if (WALLS) {
            const int ixe = phys_col(D, gx);          // a ghost row evaluates at its wall column
            const int xs = xwin_field(D, ixe);
            x0 = xs - gx;
            wa1 = Prec<T>::wxo1(D) + (ixe - xs) * W;
            wa2 = Prec<T>::wxo2(D) + (ixe - xs) * W;
        }
        T y;
        if (l == P - 1) {
            y = sp[l * HW + hr];
        } else if (WALLS && (gx == 0 || gx == D.nx - 1)) {
            // wall row (walls of Sec. 5.2, ghost nodes of Sec. 3): n . grad^(i-1) p at the wall
            // node (iw, j) = +-(D_chi p + sigma_x^(i-1) D_sigma p); the ghost column holds the
            // coefficients of its wall column
            const int dw = gx == 0 ? 1 : -1;          // shared-memory offset of the wall column
            T sg = T(l - 1) * inv_nzm1;
            T aa = cc[CC_AP0 * n + c] - sg * cc[CC_AP1 * n + c];
            const T *pl = sp + l * HW + hr + x0;
            T px = T(0);
#pragma unroll
            for (int t = 0; t < W; ++t) px += wa1[t] * pl[t];
            y = px + aa * sq[l * HW + hr + dw];
            if (gx == 0) y = -y;
        } else if (l == 0) {
            // ghost row at the bed (level index 1)
            T px = T(0), py = T(0);
#pragma unroll
            for (int t = -HALF; t <= HALF; ++t) {
                px += wa1[t + HALF] * sp[HW + hr + x0 + HALF + t];
                if (td) py += wy1[t + HALF] * sp[HW + hr + t * HX];
            }
            y = cc[CC_GS * n + c] * sq[HW + hr] + cc[CC_GX * n + c] * px;
            if (td) y += cc[CC_GY * n + c] * py;
        } else {
            T sg = T(l - 1) * inv_nzm1;
            T ap1 = cc[CC_AP1 * n + c];
            T aa = cc[CC_AP0 * n + c] - sg * ap1;
            T bb = cc[CC_BP0 * n + c] - sg * cc[CC_BP1 * n + c];
            T ax = cc[CC_AXP0 * n + c] - sg * cc[CC_AXP1 * n + c] - aa * ap1;
            T c_xs = aa + bb;
            T c_ss = aa * bb + cc[CC_EF * n + c];
            T c_s = ax - bb * ap1;
            const T *pl = sp + l * HW + hr;
            const T *ql = sq + l * HW + hr;
            T pxx = T(0), pxs = T(0);
#pragma unroll
            for (int t = -HALF; t <= HALF; ++t) {
                pxx += wa2[t + HALF] * pl[x0 + HALF + t];
                pxs += wa1[t + HALF] * ql[x0 + HALF + t];
            }
            const T *w2 = ws2 + l * W;
            const T *pc = sp + (D.win[l] + 1) * HW + hr;
            T pss = T(0);
#pragma unroll
            for (int k = 0; k < W; ++k) pss += w2[k] * pc[k * HW];
            y = pxx + c_xs * pxs + c_s * ql[0];
            if (td) {
                T ay1 = cc[CC_AY1 * n + c];
                T ay = cc[CC_AY0 * n + c] - sg * ay1;
                T by = cc[CC_BY0 * n + c] - sg * cc[CC_BY1 * n + c];
                T ayy = cc[CC_AYY0 * n + c] - sg * cc[CC_AYY1 * n + c] - ay * ay1;
                c_ss += ay * by;
                T c_ys = ay + by;
                T c_sy = ayy - by * ay1;
                T pyy = T(0), pys = T(0);
#pragma unroll
                for (int t = -HALF; t <= HALF; ++t) {
                    pyy += wy2[t + HALF] * pl[t * HX];
                    pys += wy1[t + HALF] * ql[t * HX];
                }
                y += pyy + c_ys * pys + c_sy * ql[0];
            }
            y += c_ss * pss;
        }
        st(node, y);
    }
    __syncthreads();
}

// Problem class a kernel is compiled for (its "mode" WM), so that a kernel
// instantiated for one class carries no code for the others:
//   bits 0-1, walls: 0 periodic grids only, 1 walls only, 2 decided per problem
//            at run time (batches mixing both);
//   bits 2-3, dimension: 0 decided per problem, 1 two-dimensional only (the
//            CROSS2D and BOX2D preconditioner layouts), 2 three-dimensional only.
constexpr int WM_PERIODIC = 0, WM_WALLS = 1, WM_ANYWALL = 2, WM_2D = 4, WM_3D = 8;
template <int WM>
__device__ __forceinline__ bool walls_of(const Dev &D) { return (WM & 3) == 2 ? D.walls != 0 : (WM & 3) == 1; }
template <int WM> constexpr int dim_of() { return (WM >> 2) & 3; }

template <typename T, int WM = 2, class Loader, class Store>
__device__ inline void apply_tile(const Dev &D, const Tiling &tl, int tile, T *sp, T *sq, Loader &ld, Store &st) {
    if (walls_of<WM>(D)) apply_tile_t<T, true, 1>(D, tl, tile, sp, sq, ld, st);
    else apply_tile_t<T, false, dim_of<WM>()>(D, tl, tile, sp, sq, ld, st);
}

// ---------------------------------------------------------------------------
// a3: preconditioner sweeps.  Rank order = column group, column, level.  A
// warp owns one column; lane l holds levels l-1 and l+31.  The forward sweep
// of group c first subtracts the couplings to columns of earlier groups
// (final already), then applies the inverse of the column's unit-lower block.
// The backward sweep mirrors it with the upper factor and later groups.  In
// place on `out`.
// ---------------------------------------------------------------------------
// Column groups: periodic grids have four equal colours (closed form); with
// walls the offsets come from the device table.
template <bool WALLS>
__device__ __forceinline__ int group_off(const Dev &D, int c) { return WALLS ? D.goff[c] : c * (D.ncol >> 2); }
template <bool WALLS>
__device__ __forceinline__ int group_size_t(const Dev &D, int c) {
    return WALLS ? D.goff[c + 1] - D.goff[c] : (D.ncol >> 2);
}
template <int WM = 2>
__device__ __forceinline__ int group_size(const Dev &D, int c) {
    return walls_of<WM>(D) ? group_size_t<true>(D, c) : group_size_t<false>(D, c);
}

template <bool WALLS>
__device__ __forceinline__ int col_of(const Dev &D, int c, int q) {
    if (WALLS) return D.gcol[D.goff[c] + q];
    if (!D.three_d) return c + 4 * q;
    int per_row = D.nx >> 2;
    int iy = q / per_row;
    int ix = ((c - iy) & 3) + 4 * (q - iy * per_row);
    return iy * D.nx + ix;
}

// Neighbour (column, level) of slot s for a row at (ix, iy, j); returns false
// for the in-column sigma slots.
__device__ __forceinline__ bool off_slot(const Dev &D, int s, int ix, int iy, int j, int &col, int &lev) {
    int ox = 0, oy = 0;
    int w0 = D.win[j + 1];
    switch (D.layout) {
    case CROSS2D:
        if (s >= 6) return false;
        ox = s < 3 ? s - 3 : s - 2; lev = j; break;
    case BOX2D:
        ox = s / 7 - 3; if (ox == 0) return false; lev = w0 + s % 7; break;
    case CROSS3D:
        if (s >= 12) return false;
        if (s < 6) ox = s < 3 ? s - 3 : s - 2; else { int u = s - 6; oy = u < 3 ? u - 3 : u - 2; }
        lev = j; break;
    default:
        if (s < 49) { ox = s / 7 - 3; if (ox == 0) return false; lev = w0 + s % 7; }
        else { int u = (s - 49) / 7; oy = u < 3 ? u - 3 : u - 2; lev = w0 + (s - 49) % 7; }
    }
    int gx = wrapi(ix + ox, D.nx);
    int gy = D.three_d ? wrapi(iy + oy, D.ny) : 0;
    col = gy * D.nx + gx;
    return true;
}

template <typename T>
__device__ __forceinline__ const T *lu_ptr(const Dev &D);
template <> __device__ __forceinline__ const double *lu_ptr<double>(const Dev &D) { return D.lu64; }
template <> __device__ __forceinline__ const float *lu_ptr<float>(const Dev &D) { return D.lu32; }
template <typename T>
__device__ __forceinline__ const T *udinv_ptr(const Dev &D);
template <> __device__ __forceinline__ const double *udinv_ptr<double>(const Dev &D) { return D.udinv64; }
template <> __device__ __forceinline__ const float *udinv_ptr<float>(const Dev &D) { return D.udinv32; }

__device__ __forceinline__ int colour_of(const Dev &D, int col) {
    int ix = col % D.nx, iy = col / D.nx;
    return (ix + iy) & 3;
}

// Off-column slots of each layout, enumerated at compile time: i -> (slot,
// dx, dy, window offset kk or -1 for "same level").
template <int L> struct Off;
template <> struct Off<CROSS2D> {
    static constexpr int N = 6;
    __device__ static constexpr int slot(int i) { return i; }
    __device__ static constexpr int ox(int i) { return i < 3 ? i - 3 : i - 2; }
    __device__ static constexpr int oy(int) { return 0; }
    __device__ static constexpr int kk(int) { return -1; }
};
template <> struct Off<BOX2D> {
    static constexpr int N = 42;
    __device__ static constexpr int ox(int i) { return (i / 7) < 3 ? (i / 7) - 3 : (i / 7) - 2; }
    __device__ static constexpr int oy(int) { return 0; }
    __device__ static constexpr int kk(int i) { return i % 7; }
    __device__ static constexpr int slot(int i) { return (ox(i) + 3) * 7 + i % 7; }
};
template <> struct Off<CROSS3D> {
    static constexpr int N = 12;
    __device__ static constexpr int slot(int i) { return i; }
    __device__ static constexpr int ox(int i) { return i < 6 ? (i < 3 ? i - 3 : i - 2) : 0; }
    __device__ static constexpr int oy(int i) { return i < 6 ? 0 : ((i - 6) < 3 ? (i - 6) - 3 : (i - 6) - 2); }
    __device__ static constexpr int kk(int) { return -1; }
};
template <> struct Off<BOX3D> {
    static constexpr int N = 84;
    __device__ static constexpr int ox(int i) { return i < 42 ? ((i / 7) < 3 ? (i / 7) - 3 : (i / 7) - 2) : 0; }
    __device__ static constexpr int oy(int i) {
        return i < 42 ? 0 : (((i - 42) / 7) < 3 ? ((i - 42) / 7) - 3 : ((i - 42) / 7) - 2);
    }
    __device__ static constexpr int kk(int i) { return i < 42 ? i % 7 : (i - 42) % 7; }
    __device__ static constexpr int slot(int i) { return i < 42 ? (ox(i) + 3) * 7 + i % 7 : 49 + ((i - 42) / 7) * 7 + (i - 42) % 7; }
};

// Device row index of the factors: group, level, column within the group.
template <bool WALLS>
__device__ __forceinline__ long long fac_row(const Dev &D, int c, int q, int j) {
    return (long long)group_off<WALLS>(D, c) * D.P + (long long)(j + 1) * group_size_t<WALLS>(D, c) + q;
}

// Walls (2-D): sum over the off-column slots of row (ix, j) whose column lies in
// an earlier (LOWER) or later group.  Slots follow the x positions t of the
// row's (possibly shifted) window; the own column sits at position o.
template <typename T, bool LOWER>
__device__ __forceinline__ T off_column_sum_walls(const Dev &D, const T *lu, const T *vals, int c, int ix, int j,
                                                  long long r) {
    const long long m = D.m;
    const int xs = xwin_field(D, ix), o = ix - xs;
    const int w0 = D.win[j + 1];
    T acc = T(0);
#pragma unroll
    for (int t = 0; t < W; ++t) {
        if (t == o) continue;
        const int nc = xs + t;
        const int g = D.grp[nc];
        if (LOWER ? (g >= c) : (g <= c)) continue;
        if (D.layout == CROSS2D) {
            const int s = t < o ? t : t - 1;
            acc += lu[(long long)s * m + r] * vals[(long long)(j + 1) * D.ncol + nc];
        } else {
#pragma unroll
            for (int kk = 0; kk < W; ++kk)
                acc += lu[(long long)(t * 7 + kk) * m + r] * vals[(long long)(w0 + kk + 1) * D.ncol + nc];
        }
    }
    return acc;
}

// sum over the off-column slots whose neighbour colour satisfies pick(colour)
// CC >= 0 fixes the colour at compile time: the slot selection is then static
// and every remaining load is unconditional.  With the colour known only at
// run time the slots go in chunks (the seven levels of one neighbour column in
// the box patterns, all slots of a cross pattern) whose loads are all issued
// before the chunk's multiply-adds, so they are in flight together instead of
// one slot's pair at a time.  The products are added in slot order either way.
template <int L, typename T, bool LOWER, int CC = -1>
__device__ __forceinline__ T off_column_sum(const Dev &D, const T *lu, const T *vals, int c, int ix, int iy, int j,
                                            long long r) {
    constexpr int N = Off<L>::N;
    constexpr int CH = (L == BOX2D || L == BOX3D) ? 7 : N;
    const long long m = D.m;
    const int w0 = D.win[j + 1];
    const int cc = CC >= 0 ? CC : c;
    T acc = T(0);
    if constexpr (CC >= 0) {
        // static selection: one straight run of unconditional loads and adds
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const int ox = Off<L>::ox(i), oy = Off<L>::oy(i);
            const int nc = (cc + ox + oy) & 3;
            if (LOWER ? (nc >= cc) : (nc <= cc)) continue;
            const int lev = Off<L>::kk(i) < 0 ? j : w0 + Off<L>::kk(i);
            const int gx = wrapi(ix + ox, D.nx);
            const int gy = (L == CROSS3D || L == BOX3D) ? wrapi(iy + oy, D.ny) : 0;
            acc += lu[(long long)Off<L>::slot(i) * m + r] * vals[(long long)(lev + 1) * D.ncol + gy * D.nx + gx];
        }
    } else {
#pragma unroll
        for (int i0 = 0; i0 < N; i0 += CH) {
            T a[CH], b[CH];
            bool on[CH];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int i = i0 + u;
                const int ox = Off<L>::ox(i), oy = Off<L>::oy(i);
                const int nc = (cc + ox + oy) & 3;
                on[u] = LOWER ? (nc < cc) : (nc > cc);
                a[u] = T(0);
                b[u] = T(0);
                if (on[u]) {
                    const int lev = Off<L>::kk(i) < 0 ? j : w0 + Off<L>::kk(i);
                    const int gx = wrapi(ix + ox, D.nx);
                    const int gy = (L == CROSS3D || L == BOX3D) ? wrapi(iy + oy, D.ny) : 0;
                    a[u] = lu[(long long)Off<L>::slot(i) * m + r];
                    b[u] = vals[(long long)(lev + 1) * D.ncol + gy * D.nx + gx];
                }
            }
#pragma unroll
            for (int u = 0; u < CH; ++u)
                if (on[u]) acc += a[u] * b[u];
        }
    }
    return acc;
}

template <typename T>
__device__ __forceinline__ const T *linv_ptr(const Dev &D);
template <> __device__ __forceinline__ const double *linv_ptr<double>(const Dev &D) { return D.linv64; }
template <> __device__ __forceinline__ const float *linv_ptr<float>(const Dev &D) { return D.linv32; }
template <typename T>
__device__ __forceinline__ const T *uinv_ptr(const Dev &D);
template <> __device__ __forceinline__ const double *uinv_ptr<double>(const Dev &D) { return D.uinv64; }
template <> __device__ __forceinline__ const float *uinv_ptr<float>(const Dev &D) { return D.uinv32; }

// y = B g for the column's P x P block inverse B (transposed storage bt[a2 * P + a]),
// g held one level per lane (two slots per lane when P > 32).
template <typename T>
__device__ __forceinline__ void column_block_product_two(const T *bt, const T (&g)[2], T (&y)[2], int P, int lane);
template <typename T>
__device__ __forceinline__ void column_block_product(const T *bt, const T (&g)[2], T (&y)[2], int P, int lane) {
    if (P > 32) {
        column_block_product_two<T>(bt, g, y, P, lane);
        return;
    }
    // One level per lane.  Predicated-off FP64 instructions still take their
    // issue slots on this GPU, so the second half (levels 32..63) is not
    // issued at all here: half the multiply-adds of the general form.
    // The block's rows are loaded eight at a time before they are used, so a
    // warp has eight independent loads in flight instead of one.
    T a0 = T(0), a1 = T(0);
    const bool on = lane < P;
    for (int a2 = 0; a2 < P; a2 += 8) {
        T b8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) b8[u] = (on && a2 + u < P) ? bt[(a2 + u) * P + lane] : T(0);
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            if (a2 + u >= P) break;
            const T g0 = __shfl_sync(0xffffffffu, g[0], a2 + u);
            a0 += b8[u] * g0;
            if (a2 + u + 1 < P) {
                const T g1 = __shfl_sync(0xffffffffu, g[0], a2 + u + 1);
                a1 += b8[u + 1] * g1;
            }
        }
    }
    y[0] = a0 + a1;
    y[1] = T(0);
}
template <typename T>
__device__ __forceinline__ void column_block_product_two(const T *bt, const T (&g)[2], T (&y)[2], int P, int lane) {
    // two levels per lane (lane and lane + 32); rows loaded eight at a time
    // as in the one-level form, even rows summed in a0 and odd rows in a1
    T a0[2] = {T(0), T(0)}, a1[2] = {T(0), T(0)};
    const int a_h[2] = {lane, lane + 32};
    for (int a2 = 0; a2 < P; a2 += 8) {
        T b8[2][8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int h = 0; h < 2; ++h) b8[h][u] = (a_h[h] < P && a2 + u < P) ? bt[(a2 + u) * P + a_h[h]] : T(0);
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            if (a2 + u >= P) break;
            const int r0 = a2 + u, r1 = a2 + u + 1;
            const T g0 = __shfl_sync(0xffffffffu, (r0 >> 5) ? g[1] : g[0], r0 & 31);
            const T g1 = __shfl_sync(0xffffffffu, (r1 < P && (r1 >> 5)) ? g[1] : g[0], r1 & 31);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (a_h[h] < P) {
                    a0[h] += b8[h][u] * g0;
                    if (r1 < P) a1[h] += b8[h][u + 1] * g1;
                }
            }
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) y[h] = a0[h] + a1[h];
}

// forward (lower) sweep of one column of colour c; in -> out
template <int L, typename T, bool LOWER, bool WALLS>
__device__ __forceinline__ T off_sum(const Dev &D, const T *lu, const T *vals, int c, int ix, int iy, int j,
                                     long long r) {
    if (WALLS) return off_column_sum_walls<T, LOWER>(D, lu, vals, c, ix, j, r);
    return off_column_sum<L, T, LOWER>(D, lu, vals, c, ix, iy, j, r);
}

template <int L, typename T, typename TI, bool WALLS>
__device__ inline void ilu_fwd_column_t(const Dev &D, int c, int q, const TI *in, T *out, int lane) {
    const T *lu = lu_ptr<T>(D);
    const int col = col_of<WALLS>(D, c, q);
    const int ix = col % D.nx, iy = col / D.nx;
    const long long cr = (long long)group_off<WALLS>(D, c) + q;
    T g[2], y[2];
    const int jl[2] = {lane - 1, lane + 31};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j = jl[h];
        g[h] = T(0);
        if (j >= D.nz) continue;
        g[h] = T(in[(long long)(j + 1) * D.ncol + col]) -
               off_sum<L, T, true, WALLS>(D, lu, out, c, ix, iy, j, fac_row<WALLS>(D, c, q, j));
    }
    // in-column part: y = (unit lower block)^-1 g
    column_block_product<T>(linv_ptr<T>(D) + cr * D.P * D.P, g, y, D.P, lane);
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (jl[h] < D.nz) out[(long long)(jl[h] + 1) * D.ncol + col] = y[h];
}

// backward (upper) sweep of one column of colour c; in place on out
template <int L, typename T, bool WALLS>
__device__ inline void ilu_bwd_column_t(const Dev &D, int c, int q, T *out, int lane) {
    const T *lu = lu_ptr<T>(D);
    const int col = col_of<WALLS>(D, c, q);
    const int ix = col % D.nx, iy = col / D.nx;
    const long long cr = (long long)group_off<WALLS>(D, c) + q;
    T g[2], x[2];
    const int jl[2] = {lane - 1, lane + 31};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j = jl[h];
        g[h] = T(0);
        if (j >= D.nz) continue;
        g[h] = out[(long long)(j + 1) * D.ncol + col] -
               off_sum<L, T, false, WALLS>(D, lu, out, c, ix, iy, j, fac_row<WALLS>(D, c, q, j));
    }
    __syncwarp();
    // in-column part: x = (upper block)^-1 g
    column_block_product<T>(uinv_ptr<T>(D) + cr * D.P * D.P, g, x, D.P, lane);
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (jl[h] < D.nz) out[(long long)(jl[h] + 1) * D.ncol + col] = x[h];
}

// Two-phase sweep of one colour for large problems.  Phase 1, one thread per
// row (consecutive threads take consecutive columns of one level, so factor
// reads are coalesced): g = rhs - (couplings to the other colours), stored in
// place.  Phase 2, one warp per column: the in-column block product.
template <int L, typename T, typename TI, bool LOWER, bool WALLS>
__device__ inline void ilu_gather_row_t(const Dev &D, int c, long long row, const TI *in, T *out) {
    const int per = group_size_t<WALLS>(D, c);
    const int q = (int)(row % per), j = (int)(row / per) - 1;
    const int col = col_of<WALLS>(D, c, q);
    const int ix = col % D.nx, iy = col / D.nx;
    const long long node = (long long)(j + 1) * D.ncol + col;
    const T rhs = LOWER ? T(in[node]) : out[node];
    out[node] = rhs - off_sum<L, T, LOWER, WALLS>(D, lu_ptr<T>(D), out, c, ix, iy, j, fac_row<WALLS>(D, c, q, j));
}
// Periodic grids, colour CC known at compile time (row-parallel gather of the streamed executor).
template <int L, typename T, typename TI, bool LOWER, int CC>
__device__ inline void ilu_gather_row_cc(const Dev &D, long long row, const TI *in, T *out) {
    const int per = D.ncol >> 2;
    const int q = (int)(row % per), j = (int)(row / per) - 1;
    const int col = col_of<false>(D, CC, q);
    const int ix = col % D.nx, iy = col / D.nx;
    const long long node = (long long)(j + 1) * D.ncol + col;
    const T rhs = LOWER ? T(in[node]) : out[node];
    out[node] = rhs - off_column_sum<L, T, LOWER, CC>(D, lu_ptr<T>(D), out, CC, ix, iy, j, fac_row<false>(D, CC, q, j));
}

template <typename T, typename TI, bool LOWER, int WM = 2>
__device__ inline void ilu_gather_row(const Dev &D, int c, long long row, const TI *in, T *out) {
    if (walls_of<WM>(D)) {
        if (D.layout == CROSS2D) ilu_gather_row_t<CROSS2D, T, TI, LOWER, true>(D, c, row, in, out);
        else ilu_gather_row_t<BOX2D, T, TI, LOWER, true>(D, c, row, in, out);
        return;
    }
    if constexpr (dim_of<WM>() != 2) {
        if (D.layout == CROSS2D) { ilu_gather_row_t<CROSS2D, T, TI, LOWER, false>(D, c, row, in, out); return; }
        if (D.layout == BOX2D) { ilu_gather_row_t<BOX2D, T, TI, LOWER, false>(D, c, row, in, out); return; }
    }
    if constexpr (dim_of<WM>() != 1) {
        if (D.layout == CROSS3D) ilu_gather_row_t<CROSS3D, T, TI, LOWER, false>(D, c, row, in, out);
        else ilu_gather_row_t<BOX3D, T, TI, LOWER, false>(D, c, row, in, out);
    }
}
template <typename T, int WM = 2>
__device__ inline void ilu_column_product(const Dev &D, int c, int q, T *out, int lane, bool upper) {
    const bool wl = walls_of<WM>(D);
    const int col = wl ? col_of<true>(D, c, q) : col_of<false>(D, c, q);
    const long long cr = (long long)(wl ? group_off<true>(D, c) : group_off<false>(D, c)) + q;
    T g[2], y[2];
    const int jl[2] = {lane - 1, lane + 31};
#pragma unroll
    for (int h = 0; h < 2; ++h) g[h] = jl[h] < D.nz ? out[(long long)(jl[h] + 1) * D.ncol + col] : T(0);
    __syncwarp();
    const T *blk = (upper ? uinv_ptr<T>(D) : linv_ptr<T>(D)) + cr * D.P * D.P;
    column_block_product<T>(blk, g, y, D.P, lane);
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (jl[h] < D.nz) out[(long long)(jl[h] + 1) * D.ncol + col] = y[h];
}

// runtime dispatch on the layout
template <typename T, typename TI, int WM = 2>
__device__ inline void ilu_fwd_column(const Dev &D, int c, int q, const TI *in, T *out, int lane) {
    if (walls_of<WM>(D)) {
        if (D.layout == CROSS2D) ilu_fwd_column_t<CROSS2D, T, TI, true>(D, c, q, in, out, lane);
        else ilu_fwd_column_t<BOX2D, T, TI, true>(D, c, q, in, out, lane);
        return;
    }
    if constexpr (dim_of<WM>() != 2) {
        if (D.layout == CROSS2D) { ilu_fwd_column_t<CROSS2D, T, TI, false>(D, c, q, in, out, lane); return; }
        if (D.layout == BOX2D) { ilu_fwd_column_t<BOX2D, T, TI, false>(D, c, q, in, out, lane); return; }
    }
    if constexpr (dim_of<WM>() != 1) {
        if (D.layout == CROSS3D) ilu_fwd_column_t<CROSS3D, T, TI, false>(D, c, q, in, out, lane);
        else ilu_fwd_column_t<BOX3D, T, TI, false>(D, c, q, in, out, lane);
    }
}
template <typename T, int WM = 2>
__device__ inline void ilu_bwd_column(const Dev &D, int c, int q, T *out, int lane) {
    if (walls_of<WM>(D)) {
        if (D.layout == CROSS2D) ilu_bwd_column_t<CROSS2D, T, true>(D, c, q, out, lane);
        else ilu_bwd_column_t<BOX2D, T, true>(D, c, q, out, lane);
        return;
    }
    if constexpr (dim_of<WM>() != 2) {
        if (D.layout == CROSS2D) { ilu_bwd_column_t<CROSS2D, T, false>(D, c, q, out, lane); return; }
        if (D.layout == BOX2D) { ilu_bwd_column_t<BOX2D, T, false>(D, c, q, out, lane); return; }
    }
    if constexpr (dim_of<WM>() != 1) {
        if (D.layout == CROSS3D) ilu_bwd_column_t<CROSS3D, T, false>(D, c, q, out, lane);
        else ilu_bwd_column_t<BOX3D, T, false>(D, c, q, out, lane);
    }
}

// ---------------------------------------------------------------------------
// Reductions.  Each thread holds up to N partial sums; the block reduces them
// with a reduce-scatter inside each warp (lane i ends with the warp's sum of
// value i), then across warps through shared memory, and writes one partial
// per value and block to part[v * nblocks + block].
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void warp_reduce_scatter(double (&v)[N], int lane) {
    static_assert(N == 32, "reduce-scatter over 32 values");
    // after the step with offset o a lane keeps the values whose bit o matches its lane bit
#pragma unroll
    for (int o = 16, cnt = 16; o >= 1; o >>= 1, cnt >>= 1) {
        bool upper = lane & o;
#pragma unroll
        for (int i = 0; i < cnt; ++i) {
            // pair (i, i + cnt): keep i if lower half, i + cnt if upper half
            double send = upper ? v[i] : v[i + cnt];
            double keep = upper ? v[i + cnt] : v[i];
            double recv = __shfl_xor_sync(0xffffffffu, send, o);
            v[i] = keep + recv;
        }
    }
    // v[0] of lane l now holds the warp sum of value l: at the step with offset
    // o the kept index gains bit o exactly when lane bit o is set.
}

// Block-reduce n <= 32 values (v[i], i >= n ignored) into part[v * nb + blockIdx.x].
// Warps that hold no data (active == false) contribute zeros without FP64 work.
__device__ inline void block_partials32(double (&v)[32], int n, double *red, double *part, int nb,
                                        bool active = true, int off = -1) {
    if (off < 0) off = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (!active) {
        red[warp * 32 + lane] = 0.0;
    } else if (n <= 4) {
        red[warp * 32 + lane] = 0.0;
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i >= n) break;
            double s = v[i];
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) red[warp * 32 + i] = s;
        }
    } else {
        warp_reduce_scatter<32>(v, lane);
        red[warp * 32 + lane] = v[0];
    }
    __syncthreads();
    if (warp == 0) {
        double s = 0.0;
        if (lane < n)
            for (int w = 0; w < NWARPS; ++w) s += red[w * 32 + lane];
        if (lane < n) part[lane * nb + off] = s;
    }
    __syncthreads();
}

// After a grid barrier: every block sums value i over the blocks into out[i]
// (n <= 32).  Lane i of warp w adds the partials of blocks w, w + 8, ...; all
// loads are issued before the adds, then the warps are combined.
constexpr int GATHER_PER_WARP = 20;   // supports up to 160 blocks
__device__ inline void gather_partials(const double *part, int n, int nb, double *out, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double t[GATHER_PER_WARP];
#pragma unroll
    for (int u = 0; u < GATHER_PER_WARP; ++u) {
        const int b = warp + NWARPS * u;
        t[u] = (b < nb && lane < n) ? part[lane * nb + b] : 0.0;
    }
    double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
#pragma unroll
    for (int u = 0; u < GATHER_PER_WARP; u += 4) {
        a += t[u];
        b += t[u + 1];
        c += t[u + 2];
        d += t[u + 3];
    }
    red[warp * 32 + lane] = (a + b) + (c + d);
    __syncthreads();
    if (warp == 0) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NWARPS; ++w) s += red[w * 32 + lane];
        if (lane < n) out[lane] = s;
    }
    __syncthreads();
}

}  // namespace sw
