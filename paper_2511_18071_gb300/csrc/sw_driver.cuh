// Device arithmetic of the stage driver (Algorithm 1, Eq. 14-17), shared by
// the single-problem and the batched kernels.
#pragma once
#include "sw_device.cuh"

namespace sw {

struct RK {
    double alpha, beta, dt, g, rho;
};

// LSERK45: 2N-storage fourth-order five-stage scheme (Carpenter & Kennedy 1994).
static const double LS_A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                               -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
static const double LS_B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                               1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                               2277821191437.0 / 14882151754819.0};
// abscissae c_i: stage i (1-based) evaluates at t_n + c_i dt
static const double LS_C[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                               2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

// Device pointers of one problem's stage-driver state.
struct DrvPtrs {
    double *u, *v, *w, *eta, *eta_new, *Keta, *Ku, *Kv, *Kw, *feta, *G, *rhs, *p;
    RK rk;
};

// D_chi of a node field.  With walls, `field` selects the window of an unknown
// of the linear system (ghost columns included); otherwise the window of the
// velocities and of G over the physical columns.
__device__ __forceinline__ double d1x(const Dev &D, const double *f, int col, int j, bool field) {
    int ix = col % D.nx, iy = col / D.nx;
    const double *row = f + (long long)(j + 1) * D.ncol + iy * D.nx;
    double s = 0.0;
    if (D.walls) {
        const int xe = field ? ix : phys_col(D, ix);
        const int xs = field ? xwin_field(D, xe) : xwin_phys(D, xe);
        const double *w = D.wxo1 + (xe - xs) * W;
#pragma unroll
        for (int t = 0; t < W; ++t) s += w[t] * row[xs + t];
        return s;
    }
#pragma unroll
    for (int t = -HALF; t <= HALF; ++t) s += D.wx1[t + HALF] * row[wrapi(ix + t, D.nx)];
    return s;
}
__device__ __forceinline__ bool wall_ghost(const Dev &D, int col) {
    return D.walls && (col == 0 || col == D.nx - 1);
}
__device__ __forceinline__ double d1y(const Dev &D, const double *f, int col, int j) {
    if (!D.three_d) return 0.0;
    int ix = col % D.nx, iy = col / D.nx;
    const double *pl = f + (long long)(j + 1) * D.ncol + ix;
    double s = 0.0;
#pragma unroll
    for (int t = -HALF; t <= HALF; ++t) s += D.wy1[t + HALF] * pl[(long long)wrapi(iy + t, D.ny) * D.nx];
    return s;
}
__device__ __forceinline__ double d1s(const Dev &D, const double *f, int col, int j) {
    const double *w = D.ws1 + (j + 1) * W;
    int w0 = D.win[j + 1];
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < W; ++k) s += w[k] * f[(long long)(w0 + k + 1) * D.ncol + col];
    return s;
}

// f_eta (Eq. 14b), K_eta and eta^(i) at column c.
__device__ inline void feta_at(const Dev &D, const DrvPtrs &q, int c) {
    int ix = c % D.nx, iy = c / D.nx;
    double ex = 0.0, ey = 0.0;
    if (D.walls) {
        const int xe = phys_col(D, ix), xs = xwin_phys(D, xe);
        const double *w = D.wxo1 + (xe - xs) * W;
#pragma unroll
        for (int t = 0; t < W; ++t) ex += w[t] * q.eta[xs + t];
    } else {
#pragma unroll
        for (int t = -HALF; t <= HALF; ++t) {
            ex += D.wx1[t + HALF] * q.eta[iy * D.nx + wrapi(ix + t, D.nx)];
            if (D.three_d) ey += D.wy1[t + HALF] * q.eta[wrapi(iy + t, D.ny) * D.nx + ix];
        }
    }
    long long s = (long long)D.nz * D.ncol + c;   // surface node (level nz-1)
    double f = q.w[s] - q.u[s] * ex - (D.three_d ? q.v[s] * ey : 0.0);
    if (wall_ghost(D, c)) f = 0.0;                // no flow in the ghost columns
    q.feta[c] = f;
    double K = q.rk.alpha * q.Keta[c] + q.rk.dt * f;
    q.Keta[c] = K;
    q.eta_new[c] = q.eta[c] + q.rk.beta * K;
}

// (u . grad^(i-1)) phi and D_sigma phi at one node.
__device__ __forceinline__ void advect(const Dev &D, const DrvPtrs &q, const double *phi, int col, int j,
                                       long long node, double sx, double sy, double f, double &adv, double &ps) {
    ps = d1s(D, phi, col, j);
    double gx = d1x(D, phi, col, j, false) + sx * ps;
    double gy = D.three_d ? d1y(D, phi, col, j) + sy * ps : 0.0;
    double gz = f * ps;
    adv = q.u[node] * gx + (D.three_d ? q.v[node] * gy : 0.0) + q.w[node] * gz;
}

// G field of the right-hand side (three components) at one node.
__device__ inline void rhs_g_at(const Dev &D, const DrvPtrs &q, long long node) {
    int j = (int)(node / D.ncol) - 1;
    int col = (int)(node % D.ncol);
    const int n = D.ncol;
    const double *cc = D.gp;
    const RK &rk = q.rk;
    double sg = (double)j / (D.nz - 1);
    double f = cc[CC_F * n + col];
    double sx = cc[CC_AP0 * n + col] - sg * cc[CC_AP1 * n + col];
    double sy = D.three_d ? cc[CC_AY0 * n + col] - sg * cc[CC_AY1 * n + col] : 0.0;
    double c1 = rk.rho / (rk.beta * rk.dt), c2 = rk.rho * rk.alpha / rk.dt;
    double mov = rk.rho * sg * f * q.feta[col];
    const double *comp[3] = {q.u, q.v, q.w};
    const double *Kc[3] = {q.Ku, q.Kv, q.Kw};
    for (int d = 0; d < 3; ++d) {
        if (d == 1 && !D.three_d) { q.G[D.m + node] = 0.0; continue; }
        double adv, ps;
        advect(D, q, comp[d], col, j, node, sx, sy, f, adv, ps);
        double Fd = d == 2 ? -rk.rho * rk.g : 0.0;
        q.G[(long long)d * D.m + node] = c1 * comp[d][node] + c2 * Kc[d][node] + Fd - rk.rho * adv + mov * ps;
    }
}

// b = grad^(i) . G (interior), n . G (ghost), 0 (surface) at one node.
__device__ inline void rhs_div_at(const Dev &D, const DrvPtrs &q, long long node) {
    int j = (int)(node / D.ncol) - 1;
    int col = (int)(node % D.ncol);
    const int n = D.ncol;
    const double *cc = D.gp;
    const double *Gu = q.G, *Gv = q.G + D.m, *Gw = q.G + 2 * D.m;
    if (j == D.nz - 1) { q.rhs[node] = 0.0; return; }
    if (wall_ghost(D, col)) {
        // wall row: n . G at the wall node, n = (-1, 0) at x = 0 and (1, 0) at x = lx
        const int iw = col == 0 ? 1 : D.nx - 2;
        const double g = Gu[(long long)(j + 1) * D.ncol + iw];
        q.rhs[node] = col == 0 ? -g : g;
        return;
    }
    if (j == -1) {
        long long nb = (long long)D.ncol + col;   // bed node, level 0
        q.rhs[node] = cc[CC_GX * n + col] * Gu[nb] + (D.three_d ? cc[CC_GY * n + col] * Gv[nb] : 0.0) +
                      cc[CC_GN * n + col] * Gw[nb];
        return;
    }
    double sg = (double)j / (D.nz - 1);
    double e = cc[CC_E * n + col];
    double bx = cc[CC_BP0 * n + col] - sg * cc[CC_BP1 * n + col];
    double val = d1x(D, Gu, col, j, false) + bx * d1s(D, Gu, col, j) + e * d1s(D, Gw, col, j);
    if (D.three_d) {
        double by = cc[CC_BY0 * n + col] - sg * cc[CC_BY1 * n + col];
        val += d1y(D, Gv, col, j) + by * d1s(D, Gv, col, j);
    }
    q.rhs[node] = val;
}

// K_u <- alpha K_u + dt f_u (Eq. 14a with grad^(i-1) of Algorithm 1) at one node.
__device__ inline void fu_at(const Dev &D, const DrvPtrs &q, long long node) {
    int j = (int)(node / D.ncol) - 1;
    int col = (int)(node % D.ncol);
    const int n = D.ncol;
    const double *cc = D.gp;
    const RK &rk = q.rk;
    double sg = (double)j / (D.nz - 1);
    double f = cc[CC_F * n + col];
    double sx = cc[CC_AP0 * n + col] - sg * cc[CC_AP1 * n + col];
    double sy = D.three_d ? cc[CC_AY0 * n + col] - sg * cc[CC_AY1 * n + col] : 0.0;
    double pss = d1s(D, q.p, col, j);
    double gp[3] = {d1x(D, q.p, col, j, true) + sx * pss, D.three_d ? d1y(D, q.p, col, j) + sy * pss : 0.0, f * pss};
    const bool ghost = wall_ghost(D, col);
    double mov = sg * f * q.feta[col];
    const double *comp[3] = {q.u, q.v, q.w};
    double *Kc[3] = {q.Ku, q.Kv, q.Kw};
    for (int d = 0; d < 3; ++d) {
        if (d == 1 && !D.three_d) continue;
        double adv, ps;
        advect(D, q, comp[d], col, j, node, sx, sy, f, adv, ps);
        double Fd = d == 2 ? -rk.g : 0.0;
        double fu = -gp[d] / rk.rho + Fd - adv + mov * ps;
        if (ghost) fu = 0.0;
        Kc[d][node] = rk.alpha * Kc[d][node] + rk.dt * fu;
    }
}

// u^(i) = u + beta K_u at one node.
__device__ inline void update_at(const Dev &D, const DrvPtrs &q, long long node) {
    q.u[node] += q.rk.beta * q.Ku[node];
    q.w[node] += q.rk.beta * q.Kw[node];
    if (D.three_d) q.v[node] += q.rk.beta * q.Kv[node];
}

// Generation and absorption zones (Sec. 5.2), applied after a stage at its end
// time: phi <- Gamma phi + (1 - Gamma) phi_target for eta, then u and w
// (2-D), with Gamma(xi) = 1 - (exp(xi^3.5) - 1)/(e - 1) of Engsig-Karup,
// Bingham & Lindberg (2009).  Generation target: the incident linear wave
// eta = a cos(k x - omega t), u = a omega cosh(k(z+h0))/sinh(k h0) cos(.),
// w = a omega sinh(k(z+h0))/sinh(k h0) sin(.), at z = sigma d - h with the
// relaxed eta; absorption target: still water.
struct RelaxArgs {
    double gen_x0, gen_x1, abs_x0, abs_x1;
    double amp, k, omega, depth, t;
};

__device__ __forceinline__ double relax_weight(double xi) {
    if (xi <= 0.0) return 1.0;
    if (xi >= 1.0) return 0.0;
    return 1.0 - (exp(pow(xi, 3.5)) - 1.0) / (2.718281828459045 - 1.0);
}

__device__ inline void relax_column(const Dev &D, const DrvPtrs &q, const RelaxArgs &ra, int c) {
    if (wall_ghost(D, c)) return;
    const double x = D.walls ? (c - 1) * D.dx : c * D.dx;
    double gam;
    bool gen;
    if (ra.gen_x1 > ra.gen_x0 && x >= ra.gen_x0 && x <= ra.gen_x1) {
        gam = relax_weight((ra.gen_x1 - x) / (ra.gen_x1 - ra.gen_x0));
        gen = true;
    } else if (ra.abs_x1 > ra.abs_x0 && x >= ra.abs_x0 && x <= ra.abs_x1) {
        gam = relax_weight((x - ra.abs_x0) / (ra.abs_x1 - ra.abs_x0));
        gen = false;
    } else {
        return;
    }
    const double th = ra.k * x - ra.omega * ra.t;
    const double eta_t = gen ? ra.amp * cos(th) : 0.0;
    const double eta = gam * q.eta[c] + (1.0 - gam) * eta_t;
    q.eta[c] = eta;
    const double h = D.h[c], d = h + eta;
    const double sh = sinh(ra.k * ra.depth);
    const double ct = cos(th), st = sin(th);
    for (int j = -1; j < D.nz; ++j) {
        const long long node = (long long)(j + 1) * D.ncol + c;
        const double z = ((double)j / (double)(D.nz - 1)) * d - h;
        double ut = 0.0, wt = 0.0;
        if (gen) {
            ut = ra.amp * ra.omega * cosh(ra.k * (z + ra.depth)) / sh * ct;
            wt = ra.amp * ra.omega * sinh(ra.k * (z + ra.depth)) / sh * st;
        }
        q.u[node] = gam * q.u[node] + (1.0 - gam) * ut;
        q.w[node] = gam * q.w[node] + (1.0 - gam) * wt;
    }
}

}  // namespace sw
