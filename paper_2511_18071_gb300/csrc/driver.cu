// Stage driver: Algorithm 1 with the low-storage Runge-Kutta update of Eq. (15)
// and the LSERK45 coefficients of Carpenter & Kennedy (1994) (Sec. 5).
// Inviscid, F = (0, 0, -rho g), total pressure with p = 0 on the free surface.
//
// One stage i:
//   f_eta (Eq. 14b) at stage i-1, K_eta <- alpha_i K_eta + dt f_eta, eta^(i) = eta + beta_i K_eta;
//   right-hand side of Eq. (16)-(17) for the pair (eta^(i-1), eta^(i)):
//     G = rho/(beta_i dt) u + rho alpha_i/dt K_u + F - rho (u . grad^(i-1)) u
//         + rho (sigma/d^(i-1)) (D_tau eta^(i-1)) D_sigma u,
//     interior rows grad^(i) . G, ghost rows n . G at the bed, surface rows 0;
//   the Poisson solve A(eta^(i-1), eta^(i)) p = b (Algorithm 2);
//   f_u (Eq. 14a) with grad^(i-1), K_u <- alpha_i K_u + dt f_u, u^(i) = u + beta_i K_u.
#include <cstring>
#include <utility>

#include "sw_device.cuh"

namespace sw {

int solve_device(Problem *P, const double *ep, const double *ec, const double *b, double *x, cudaStream_t s);

struct RK {
    double alpha, beta, dt, g, rho;
};

// LSERK45: 2N-storage fourth-order five-stage scheme (Carpenter & Kennedy 1994).
static const double LS_A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                               -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
static const double LS_B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                               1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                               2277821191437.0 / 14882151754819.0};

__device__ __forceinline__ double d1x(const Dev &D, const double *f, int col, int j) {
    int ix = col % D.nx, iy = col / D.nx;
    const double *row = f + (long long)(j + 1) * D.ncol + iy * D.nx;
    double s = 0.0;
#pragma unroll
    for (int t = -HALF; t <= HALF; ++t) s += D.wx1[t + HALF] * row[wrapi(ix + t, D.nx)];
    return s;
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

// f_eta, K_eta and eta^(i) per column.
__global__ void feta_kernel(Dev D, const double *u, const double *v, const double *w, const double *eta,
                            double *Keta, double *eta_new, double *feta, RK rk) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D.ncol) return;
    int ix = c % D.nx, iy = c / D.nx;
    double ex = 0.0, ey = 0.0;
#pragma unroll
    for (int t = -HALF; t <= HALF; ++t) {
        ex += D.wx1[t + HALF] * eta[iy * D.nx + wrapi(ix + t, D.nx)];
        if (D.three_d) ey += D.wy1[t + HALF] * eta[wrapi(iy + t, D.ny) * D.nx + ix];
    }
    long long s = (long long)D.nz * D.ncol + c;   // surface node (level nz-1)
    double f = w[s] - u[s] * ex - (D.three_d ? v[s] * ey : 0.0);
    feta[c] = f;
    double K = rk.alpha * Keta[c] + rk.dt * f;
    Keta[c] = K;
    eta_new[c] = eta[c] + rk.beta * K;
}

// (u . grad^(i-1)) phi and D_sigma phi at one node.
__device__ __forceinline__ void advect(const Dev &D, const double *u, const double *v, const double *w,
                                       const double *phi, int col, int j, long long node, double sx, double sy,
                                       double f, double &adv, double &ps) {
    ps = d1s(D, phi, col, j);
    double gx = d1x(D, phi, col, j) + sx * ps;
    double gy = D.three_d ? d1y(D, phi, col, j) + sy * ps : 0.0;
    double gz = f * ps;
    adv = u[node] * gx + (D.three_d ? v[node] * gy : 0.0) + w[node] * gz;
}

// G field of the right-hand side at every node (three components).
__global__ void rhs_g_kernel(Dev D, const double *u, const double *v, const double *w, const double *Ku,
                             const double *Kv, const double *Kw, const double *feta, double *G, RK rk) {
    long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (node >= D.m) return;
    int j = (int)(node / D.ncol) - 1;
    int col = (int)(node % D.ncol);
    const int n = D.ncol;
    const double *cc = D.gp;
    double sg = (double)j / (D.nz - 1);
    double f = cc[CC_F * n + col];
    double sx = cc[CC_AP0 * n + col] - sg * cc[CC_AP1 * n + col];
    double sy = D.three_d ? cc[CC_AY0 * n + col] - sg * cc[CC_AY1 * n + col] : 0.0;
    double c1 = rk.rho / (rk.beta * rk.dt), c2 = rk.rho * rk.alpha / rk.dt;
    double mov = rk.rho * sg * f * feta[col];
    const double *comp[3] = {u, v, w};
    const double *Kc[3] = {Ku, Kv, Kw};
    for (int d = 0; d < 3; ++d) {
        if (d == 1 && !D.three_d) { G[D.m + node] = 0.0; continue; }
        double adv, ps;
        advect(D, u, v, w, comp[d], col, j, node, sx, sy, f, adv, ps);
        double Fd = d == 2 ? -rk.rho * rk.g : 0.0;
        G[(long long)d * D.m + node] = c1 * comp[d][node] + c2 * Kc[d][node] + Fd - rk.rho * adv + mov * ps;
    }
}

// b = grad^(i) . G (interior), n . G (ghost), 0 (surface).
__global__ void rhs_div_kernel(Dev D, const double *G, double *b) {
    long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (node >= D.m) return;
    int j = (int)(node / D.ncol) - 1;
    int col = (int)(node % D.ncol);
    const int n = D.ncol;
    const double *cc = D.gp;
    const double *Gu = G, *Gv = G + D.m, *Gw = G + 2 * D.m;
    if (j == D.nz - 1) { b[node] = 0.0; return; }
    if (j == -1) {
        long long nb = (long long)D.ncol + col;   // bed node, level 0
        b[node] = cc[CC_GX * n + col] * Gu[nb] + (D.three_d ? cc[CC_GY * n + col] * Gv[nb] : 0.0) +
                  cc[CC_GN * n + col] * Gw[nb];
        return;
    }
    double sg = (double)j / (D.nz - 1);
    double e = cc[CC_E * n + col];
    double bx = cc[CC_BP0 * n + col] - sg * cc[CC_BP1 * n + col];
    double val = d1x(D, Gu, col, j) + bx * d1s(D, Gu, col, j) + e * d1s(D, Gw, col, j);
    if (D.three_d) {
        double by = cc[CC_BY0 * n + col] - sg * cc[CC_BY1 * n + col];
        val += d1y(D, Gv, col, j) + by * d1s(D, Gv, col, j);
    }
    b[node] = val;
}

// K_u <- alpha K_u + dt f_u (Eq. 14a with grad^(i-1) of Algorithm 1).
__global__ void fu_kernel(Dev D, const double *u, const double *v, const double *w, const double *p,
                          const double *feta, double *Ku, double *Kv, double *Kw, RK rk) {
    long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (node >= D.m) return;
    int j = (int)(node / D.ncol) - 1;
    int col = (int)(node % D.ncol);
    const int n = D.ncol;
    const double *cc = D.gp;
    double sg = (double)j / (D.nz - 1);
    double f = cc[CC_F * n + col];
    double sx = cc[CC_AP0 * n + col] - sg * cc[CC_AP1 * n + col];
    double sy = D.three_d ? cc[CC_AY0 * n + col] - sg * cc[CC_AY1 * n + col] : 0.0;
    double pss = d1s(D, p, col, j);
    double gp[3] = {d1x(D, p, col, j) + sx * pss, D.three_d ? d1y(D, p, col, j) + sy * pss : 0.0, f * pss};
    double mov = sg * f * feta[col];
    const double *comp[3] = {u, v, w};
    double *Kc[3] = {Ku, Kv, Kw};
    for (int d = 0; d < 3; ++d) {
        if (d == 1 && !D.three_d) continue;
        double adv, ps;
        advect(D, u, v, w, comp[d], col, j, node, sx, sy, f, adv, ps);
        double Fd = d == 2 ? -rk.g : 0.0;
        double fu = -gp[d] / rk.rho + Fd - adv + mov * ps;
        Kc[d][node] = rk.alpha * Kc[d][node] + rk.dt * fu;
    }
}

__global__ void update_kernel(Dev D, double *u, double *v, double *w, const double *Ku, const double *Kv,
                              const double *Kw, double beta) {
    long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (node >= D.m) return;
    u[node] += beta * Ku[node];
    w[node] += beta * Kw[node];
    if (D.three_d) v[node] += beta * Kv[node];
}

__global__ void geometry_only_kernel(Dev D, const double *ep, const double *ec) {
    geometry_columns(D, ep, ec, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

static int ensure_state(Problem *P) {
    if (P->d_u) return SW_OK;
    const long long m = P->m;
    const int n = P->ncol;
    auto al = [&](double **p, size_t cnt) -> int {
        cudaError_t e = cudaMalloc((void **)p, cnt * sizeof(double));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        P->allocs.push_back(*p);
        e = cudaMemset(*p, 0, cnt * sizeof(double));
        return e == cudaSuccess ? SW_OK : cuda_fail(e, "cudaMemset");
    };
    int rc;
    if ((rc = al(&P->d_u, m)) || (rc = al(&P->d_v, m)) || (rc = al(&P->d_w, m)) || (rc = al(&P->d_eta, n)) ||
        (rc = al(&P->d_Ku, m)) || (rc = al(&P->d_Kv, m)) || (rc = al(&P->d_Kw, m)) || (rc = al(&P->d_Keta, n)) ||
        (rc = al(&P->d_p, m)) || (rc = al(&P->d_rhs, m)) || (rc = al(&P->d_eta_new, n)) ||
        (rc = al(&P->d_feta, n)) || (rc = al(&P->d_drv, 3 * (size_t)m)))
        return rc;
    return SW_OK;
}

}  // namespace sw

using namespace sw;

extern "C" int sw_set_physics(sw_problem *pp, const sw_physics *ph) {
    Problem *P = (Problem *)pp;
    if (!P || !ph || !(ph->dt > 0) || !(ph->rho > 0)) { set_error("bad physics"); return SW_ERR_BAD_ARG; }
    P->phys = *ph;
    return SW_OK;
}

extern "C" int sw_set_state(sw_problem *pp, const double *u, const double *v, const double *w, const double *eta,
                            void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !u || !w || !eta || (P->dev.three_d && !v)) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    int rc = ensure_state(P);
    if (rc != SW_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t mb = P->m * sizeof(double), nb = P->ncol * sizeof(double);
    cudaError_t e = cudaMemcpyAsync(P->d_u, u, mb, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->d_w, w, mb, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && v) e = cudaMemcpyAsync(P->d_v, v, mb, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->d_eta, eta, nb, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->d_Ku, 0, mb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->d_Kv, 0, mb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->d_Kw, 0, mb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->d_Keta, 0, nb, s);
    if (e != cudaSuccess) return cuda_fail(e, "set state");
    P->stage = 0;
    P->has_state = true;
    P->last_stream = s;
    return SW_OK;
}

extern "C" int sw_get_state(sw_problem *pp, double *u, double *v, double *w, double *eta, double *p,
                            void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !P->has_state) { set_error("no state loaded"); return SW_ERR_BAD_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t mb = P->m * sizeof(double), nb = P->ncol * sizeof(double);
    cudaError_t e = cudaSuccess;
    if (u) e = cudaMemcpyAsync(u, P->d_u, mb, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && v && P->dev.three_d) e = cudaMemcpyAsync(v, P->d_v, mb, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && w) e = cudaMemcpyAsync(w, P->d_w, mb, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && eta) e = cudaMemcpyAsync(eta, P->d_eta, nb, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && p) e = cudaMemcpyAsync(p, P->d_p, mb, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "get state");
    P->last_stream = s;
    return SW_OK;
}

extern "C" int sw_advance_stage(sw_problem *pp, void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !P->has_state || !(P->phys.dt > 0)) { set_error("state or physics not set"); return SW_ERR_BAD_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const int i = P->stage;
    RK rk{LS_A[i], LS_B[i], P->phys.dt, P->phys.g, P->phys.rho};
    const Dev &D = P->dev;
    const int T = 256;
    const int gc = (P->ncol + T - 1) / T;
    const int gm = (int)((P->m + T - 1) / T);
    feta_kernel<<<gc, T, 0, s>>>(D, P->d_u, P->d_v, P->d_w, P->d_eta, P->d_Keta, P->d_eta_new, P->d_feta, rk);
    geometry_only_kernel<<<gc, T, 0, s>>>(D, P->d_eta, P->d_eta_new);
    rhs_g_kernel<<<gm, T, 0, s>>>(D, P->d_u, P->d_v, P->d_w, P->d_Ku, P->d_Kv, P->d_Kw, P->d_feta, P->d_drv, rk);
    rhs_div_kernel<<<gm, T, 0, s>>>(D, P->d_drv, P->d_rhs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "stage launch");
    int rc = solve_device(P, P->d_eta, P->d_eta_new, P->d_rhs, P->d_p, s);
    if (rc != SW_OK) return rc;
    // the solve recomputed the same geometry pair; f_u uses its stage i-1 half
    fu_kernel<<<gm, T, 0, s>>>(D, P->d_u, P->d_v, P->d_w, P->d_p, P->d_feta, P->d_Ku, P->d_Kv, P->d_Kw, rk);
    update_kernel<<<gm, T, 0, s>>>(D, P->d_u, P->d_v, P->d_w, P->d_Ku, P->d_Kv, P->d_Kw, rk.beta);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "stage launch");
    // eta^(i) becomes the state; the buffer of eta^(i-1) is kept for sw_get_last_system
    std::swap(P->d_eta, P->d_eta_new);
    P->launches += 6;
    P->stage = (P->stage + 1) % 5;
    P->last_stream = s;
    return SW_OK;
}

extern "C" int sw_get_last_system(sw_problem *pp, double *ep, double *ec, double *b, void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !P->has_state) { set_error("no state loaded"); return SW_ERR_BAD_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nb = P->ncol * sizeof(double);
    cudaError_t e = cudaSuccess;
    if (ep) e = cudaMemcpyAsync(ep, P->d_eta_new, nb, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && ec) e = cudaMemcpyAsync(ec, P->d_eta, nb, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && b) e = cudaMemcpyAsync(b, P->d_rhs, P->m * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "get last system");
    return SW_OK;
}
