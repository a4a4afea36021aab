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
#include <cmath>
#include <cstring>
#include <utility>

#include "sw_driver.cuh"

namespace sw {

int solve_device(Problem *P, const double *ep, const double *ec, const double *b, double *x, cudaStream_t s);

__global__ void feta_kernel(Dev D, DrvPtrs q) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < D.ncol) feta_at(D, q, c);
}
__global__ void geometry_only_kernel(Dev D, const double *ep, const double *ec) {
    geometry_columns(D, ep, ec, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}
__global__ void rhs_g_kernel(Dev D, DrvPtrs q) {
    long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (node < D.m) rhs_g_at(D, q, node);
}
__global__ void rhs_div_kernel(Dev D, DrvPtrs q) {
    long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (node < D.m) rhs_div_at(D, q, node);
}
__global__ void fu_kernel(Dev D, DrvPtrs q) {
    long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (node < D.m) fu_at(D, q, node);
}
__global__ void update_kernel(Dev D, DrvPtrs q) {
    long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (node < D.m) update_at(D, q, node);
}
__global__ void relax_kernel(Dev D, DrvPtrs q, RelaxArgs ra) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < D.ncol) relax_column(D, q, ra, c);
}

// Wavenumber of the linear dispersion relation omega^2 = g k tanh(k h) by
// Newton's method from the deep-water value (the residual is increasing and
// concave in k, so the iteration converges monotonically).
static double dispersion_k(double omega, double depth, double g) {
    double k = omega * omega / g;
    for (int it = 0; it < 100; ++it) {
        const double th = std::tanh(k * depth);
        const double F = g * k * th - omega * omega;
        const double dF = g * th + g * k * depth * (1.0 - th * th);
        const double dk = F / dF;
        k -= dk;
        if (std::fabs(dk) <= 1e-15 * k) break;
    }
    return k;
}

DrvPtrs driver_ptrs(Problem *P) {
    const int i = P->stage;
    DrvPtrs q;
    q.u = P->d_u; q.v = P->d_v; q.w = P->d_w; q.eta = P->d_eta; q.eta_new = P->d_eta_new;
    q.Keta = P->d_Keta; q.Ku = P->d_Ku; q.Kv = P->d_Kv; q.Kw = P->d_Kw; q.feta = P->d_feta;
    q.G = P->d_drv; q.rhs = P->d_rhs; q.p = P->d_p;
    q.rk = RK{LS_A[i], LS_B[i], P->phys.dt, P->phys.g, P->phys.rho};
    return q;
}

int ensure_state(Problem *P) {
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
    P->step_index = 0;
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
    const Dev &D = P->dev;
    DrvPtrs q = driver_ptrs(P);
    const int T = 256;
    const int gc = (P->ncol + T - 1) / T;
    const int gm = (int)((P->m + T - 1) / T);
    feta_kernel<<<gc, T, 0, s>>>(D, q);
    geometry_only_kernel<<<gc, T, 0, s>>>(D, P->d_eta, P->d_eta_new);
    rhs_g_kernel<<<gm, T, 0, s>>>(D, q);
    rhs_div_kernel<<<gm, T, 0, s>>>(D, q);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "stage launch");
    int rc = solve_device(P, P->d_eta, P->d_eta_new, P->d_rhs, P->d_p, s);
    if (rc != SW_OK) return rc;
    // the solve recomputed the same geometry pair; f_u uses its stage i-1 half
    fu_kernel<<<gm, T, 0, s>>>(D, q);
    update_kernel<<<gm, T, 0, s>>>(D, q);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "stage launch");
    // eta^(i) becomes the state; the buffer of eta^(i-1) is kept for sw_get_last_system
    std::swap(P->d_eta, P->d_eta_new);
    P->launches += 6;
    if (P->relax_on) {
        // generation/absorption zones at the stage's end time t_n + c_(i+1) dt (t_n + dt after stage 5)
        const double c_next = P->stage < 4 ? LS_C[P->stage + 1] : 1.0;
        const double t = ((double)P->step_index + c_next) * P->phys.dt;
        const sw_relaxation &rl = P->relax;
        const double pi = 3.14159265358979323846;
        double ramp = 1.0;
        if (rl.ramp_time > 0.0 && t < rl.ramp_time) ramp = 0.5 * (1.0 - std::cos(pi * t / rl.ramp_time));
        RelaxArgs ra{rl.gen_x0, rl.gen_x1, rl.abs_x0, rl.abs_x1, 0.5 * rl.height * ramp, P->relax_k,
                     2.0 * pi / rl.period, rl.depth, t};
        DrvPtrs q2 = driver_ptrs(P);   // q2.eta is eta^(i) after the swap
        relax_kernel<<<gc, T, 0, s>>>(D, q2, ra);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "relaxation launch");
        P->launches += 1;
    }
    if (P->stage == 4) P->step_index++;
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

extern "C" int sw_set_relaxation(sw_problem *pp, const sw_relaxation *rl) {
    Problem *P = (Problem *)pp;
    if (!P) { set_error("null problem"); return SW_ERR_BAD_ARG; }
    if (!rl) { P->relax_on = false; return SW_OK; }
    if (P->dev.three_d) { set_error("relaxation zones: 2-D problems only"); return SW_ERR_BAD_ARG; }
    const bool gen = rl->gen_x1 > rl->gen_x0;
    if (gen && (!(rl->period > 0) || !(rl->height >= 0) || !(rl->depth > 0) || !(rl->g > 0))) {
        set_error("relaxation zones: generation needs period > 0, height >= 0, depth > 0, g > 0");
        return SW_ERR_BAD_ARG;
    }
    P->relax = *rl;
    P->relax_k = gen ? dispersion_k(2.0 * 3.14159265358979323846 / rl->period, rl->depth, rl->g) : 0.0;
    P->relax_on = true;
    return SW_OK;
}

extern "C" int sw_set_step(sw_problem *pp, long long n_steps) {
    Problem *P = (Problem *)pp;
    if (!P || n_steps < 0) { set_error("bad argument"); return SW_ERR_BAD_ARG; }
    P->step_index = n_steps;
    P->stage = 0;
    return SW_OK;
}
