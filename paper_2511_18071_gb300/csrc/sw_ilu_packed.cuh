// In-column half of the ILU(0) colour sweeps (Sec. 3: forward substitution
// with L, backward with U, in the four-colour column order) for periodic
// grids on the streamed executor, with the column blocks stored packed.
//
// After the row-parallel gathers of a colour (g = rhs - couplings to the
// other colours), every column of the colour needs y = B g, B the inverse of
// the column's unit lower (forward) or upper (backward) diagonal P x P block.
// Those inverses are triangular, so only their triangles are stored
// ("packed": P (P + 1) / 2 values per column, padded to a multiple of four so
// every column starts 16 bytes apart), half the bytes of the dense form that
// the persistent and batch kernels read.
//
// Packed layout of column cr (transposed blocks, bt[a2][i] = B[i][a2]):
//   lower: row a2 holds i = a2 .. P-1 at offL(a2) + i - a2, offL(a2) = a2 P - a2 (a2 - 1) / 2
//   upper: row a2 holds i = 0 .. a2   at offU(a2) + i,      offU(a2) = a2 (a2 + 1) / 2
// Row a2 is one contiguous run, so the lanes that need it read consecutive
// addresses.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sw_device.cuh"

namespace sw {

// packed values per column, padded so that every column starts 16 bytes apart
__host__ __device__ inline int tri_stride(int P) { return ((P * (P + 1) / 2) + 3) & ~3; }

// dense transposed inverse blocks -> packed triangles (set-up, once)
template <typename T>
__global__ void sk_pack_tri(const T *linv, const T *uinv, int P, long long ncol, T *ltri, T *utri) {
    const int tp = tri_stride(P);
    const long long total = ncol * (long long)P * P;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long cr = e / ((long long)P * P);
        const int rem = (int)(e - cr * P * P), a2 = rem / P, i = rem % P;
        const T v_l = linv[e], v_u = uinv[e];
        if (i >= a2) ltri[cr * tp + a2 * P - a2 * (a2 - 1) / 2 + (i - a2)] = v_l;
        if (i <= a2) utri[cr * tp + a2 * (a2 + 1) / 2 + i] = v_u;
    }
}

// offset of row r within a packed block and whether level i takes part in it
template <bool LOWER>
__device__ __forceinline__ int tri_next(int off, int r, int P) { return off + (LOWER ? P - r : r + 1); }
template <bool LOWER>
__device__ __forceinline__ bool tri_has(int i, int r, int P) { return LOWER ? (i >= r && i < P) : (i <= r); }
template <bool LOWER>
__device__ __forceinline__ int tri_at(int off, int i, int r) { return off + (LOWER ? i - r : i); }

// y = B g for one column, one warp: lane holds levels lane and lane + 32 of g
// (and of y).  The block's rows are loaded eight at a time before they are
// used, so a warp has eight independent loads in flight; lanes outside a
// row's triangle load nothing.
template <typename T, bool LOWER>
__device__ __forceinline__ void tri_product(const T *B, const T (&g)[2], T (&y)[2], int P, int lane) {
    T a0[2] = {T(0), T(0)}, a1[2] = {T(0), T(0)};   // [level half]: even and odd rows summed apart
    const int i0 = lane, i1 = lane + 32;
    int off = 0;
    for (int r0 = 0; r0 < P; r0 += 8) {
        T b0[8], b1[8];
        int o = off;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int r = r0 + u;
            b0[u] = (r < P && tri_has<LOWER>(i0, r, P)) ? B[tri_at<LOWER>(o, i0, r)] : T(0);
            b1[u] = (P > 32 && r < P && tri_has<LOWER>(i1, r, P)) ? B[tri_at<LOWER>(o, i1, r)] : T(0);
            if (r < P) o = tri_next<LOWER>(o, r, P);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int r = r0 + u;
            if (r >= P) break;
            const T gr = __shfl_sync(0xffffffffu, (r >> 5) ? g[1] : g[0], r & 31);
            if (u & 1) a1[0] += b0[u] * gr; else a0[0] += b0[u] * gr;
            if (P > 32) { if (u & 1) a1[1] += b1[u] * gr; else a0[1] += b1[u] * gr; }
        }
        off = o;
    }
    y[0] = a0[0] + a1[0];
    y[1] = a0[1] + a1[1];
}

// The same product with the number of levels PC known at compile time (10,
// 18 and 34 levels: nz = 9, 17, 33): the triangle's row offsets and the
// lanes of each row are constants, every load of the block is issued before
// the first multiply-add, and no index arithmetic is left at run time.
template <typename T, bool LOWER, int PC>
__device__ __forceinline__ void tri_product_fixed(const T *B, const T (&g)[2], T (&y)[2], int lane) {
    constexpr int NH = PC > 32 ? 2 : 1;
    T b[NH][PC];
#pragma unroll
    for (int h = 0; h < NH; ++h) {
        const int i = lane + 32 * h;
        int o = 0;
#pragma unroll
        for (int r = 0; r < PC; ++r) {
            b[h][r] = tri_has<LOWER>(i, r, PC) ? B[tri_at<LOWER>(o, i, r)] : T(0);
            o = tri_next<LOWER>(o, r, PC);
        }
    }
    T a0[NH], a1[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) a0[h] = a1[h] = T(0);
#pragma unroll
    for (int r = 0; r < PC; ++r) {
        const T gr = __shfl_sync(0xffffffffu, g[r >> 5], r & 31);
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            if (r & 1) a1[h] += b[h][r] * gr;
            else a0[h] += b[h][r] * gr;
        }
    }
    y[0] = a0[0] + a1[0];
    y[1] = NH > 1 ? a0[NH - 1] + a1[NH - 1] : T(0);
}

// In-column products of colour c (forward: LOWER, backward: upper), in place
// on out, one warp per column of the colour; tri holds the colour-ordered
// packed blocks (column rank c (ncol / 4) + q).  PC > 0: the number of levels
// at compile time (must equal D.P); PC = 0: any number of levels.
template <typename T, bool LOWER, int PC, class State>
__global__ void __launch_bounds__(NTHREADS) sk_ilu_product_tri(Dev D, int c, const T *tri, T *out, const State *ss,
                                                                 int skip) {
    if (skip && (ss->stop || ss->done)) return;
    const int lane = threadIdx.x & 31;
    const int per = D.ncol >> 2;
    const int tp = tri_stride(D.P);
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < per; q += nw) {
        const int col = col_of<false>(D, c, q);
        const long long cr = (long long)c * per + q;
        T g[2], y[2];
        const int lev[2] = {lane, lane + 32};   // level index j + 1 of the node
#pragma unroll
        for (int h = 0; h < 2; ++h) g[h] = lev[h] < D.P ? out[(long long)lev[h] * D.ncol + col] : T(0);
        __syncwarp();
        if constexpr (PC > 0) tri_product_fixed<T, LOWER, PC>(tri + cr * tp, g, y, lane);
        else tri_product<T, LOWER>(tri + cr * tp, g, y, D.P, lane);
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (lev[h] < D.P) out[(long long)lev[h] * D.ncol + col] = y[h];
    }
}

}  // namespace sw
