// The Poisson solve of one Runge-Kutta stage as one persistent cooperative
// kernel (Algorithm 2 with the EWMA subspace of Algorithm 4, then restarted
// GMRES left-preconditioned with the fixed ILU(0) factors, Sec. 3 and 4).
// All control flow stays on the device: every block runs the same loop, the
// decisions (convergence, breakdown, restarts) are made on values that every
// block reduces identically, and grid barriers separate the phases.
#include <cmath>
#include <cstring>

#include "sw_solve.cuh"

namespace sw {

// ---------------------------------------------------------------------------
// The persistent solve kernel (solve_kernel.cu), one variant per inner
// precision and problem class, each compiled on its own.
// ---------------------------------------------------------------------------
constexpr size_t SMEM_FIXED = (sizeof(SmemFixed) + 255) & ~size_t(255);

const void *solve_kernel_f64_p2();   // FP64, periodic, 2-D
const void *solve_kernel_f64_p3();   // FP64, periodic, 3-D
const void *solve_kernel_f64_w2();   // FP64, walls (2-D)
const void *solve_kernel_f32_p2();   // FP32 inner cycles
const void *solve_kernel_f32_p3();
const void *solve_kernel_f32_w2();

static const void *solve_kernel_for(const Problem *P) {
    const bool f32 = P->params.precision == SW_PRECISION_MIXED;
    if (P->dev.walls) return f32 ? solve_kernel_f32_w2() : solve_kernel_f64_w2();
    if (P->dev.three_d) return f32 ? solve_kernel_f32_p3() : solve_kernel_f64_p3();
    return f32 ? solve_kernel_f32_p2() : solve_kernel_f64_p2();
}

// ---------------------------------------------------------------------------
// Standalone kernels for the per-step entry points.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NTHREADS) geometry_kernel(Dev D, const double *ep, const double *ec) {
    geometry_columns(D, ep, ec, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void __launch_bounds__(NTHREADS) apply_kernel(Dev D, Tiling tl, const double *x, double *y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *sp = reinterpret_cast<double *>(smem_raw);
    double *sq = sp + (size_t)D.P * tl.HW;
    LdVec<double, double> ld{x, 1.0};
    StVec<double, double> st{y};
    for (int tile = blockIdx.x; tile < tl.ntiles; tile += gridDim.x) apply_tile<double>(D, tl, tile, sp, sq, ld, st);
}

__global__ void __launch_bounds__(NTHREADS) ilu_fwd_kernel(Dev D, int c, const double *in, double *out) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int q = gw; q < group_size(D, c); q += nw) ilu_fwd_column<double, double>(D, c, q, in, out, lane);
}

struct SketchUpd {
    double om[MAX_K];
};

// out = r Y + x omega^T (Algorithm 4), column c at offset c m; Y in the
// problem's sketch precision, out in FP64.
template <typename TY>
__global__ void __launch_bounds__(NTHREADS) sketch_update_kernel(const TY *Y, double *out, const double *x,
                                                                 SketchUpd u, int k, long long m, double rho,
                                                                 int apply) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m; p += (long long)gridDim.x * blockDim.x) {
        const double xp = x[p];
        for (int c = 0; c < k; ++c) {
            const TY yv = Y[(size_t)c * m + p];
            out[(size_t)c * m + p] = apply ? (double)TY(TY(rho) * yv + TY(u.om[c]) * TY(xp)) : (double)yv;
        }
    }
}

// FP64 sketch into the problem's sketch precision.
template <typename TY>
__global__ void __launch_bounds__(NTHREADS) sketch_store_kernel(const double *in, TY *Y, long long n) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
        Y[p] = TY(in[p]);
}

__global__ void __launch_bounds__(NTHREADS) ilu_bwd_kernel(Dev D, int c, double *out) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int q = gw; q < group_size(D, c); q += nw) ilu_bwd_column<double>(D, c, q, out, lane);
}

// ---------------------------------------------------------------------------
// Launch configuration.
// ---------------------------------------------------------------------------
static Tiling make_tiling(const Dev &D) {
    Tiling t{};
    if (!D.three_d) {
        // enough tiles to spread over the SMs, at most 64 columns per tile
        int TX = 64;
        while (TX > 4 && (D.nx % TX != 0 || D.nx / TX < 304)) TX >>= 1;
        t.TX = TX; t.TY = 1;
    } else {
        int TX = 16, TY = 8;
        while ((size_t)(TX + 6) * (TY + 6) * D.P * 2 * sizeof(double) > 150 * 1024 && TX > 4) {
            if (TX > TY) TX >>= 1; else TY >>= 1;
        }
        while (D.nx % TX) TX >>= 1;
        while (D.ny % TY) TY >>= 1;
        t.TX = TX; t.TY = TY;
    }
    t.HX = t.TX + 2 * HALF;
    t.HY = D.three_d ? t.TY + 2 * HALF : 1;
    t.HW = t.HX * t.HY;
    t.ntx = D.nx / t.TX;
    t.nty = D.three_d ? D.ny / t.TY : 1;
    t.ntiles = t.ntx * t.nty;
    return t;
}

static size_t solve_smem(const Dev &D, const Tiling &t) {
    return SMEM_FIXED + 2 * (size_t)D.P * t.HW * sizeof(double);
}

static bool mixed(const Problem *P) { return P->params.precision == SW_PRECISION_MIXED; }

int setup_streamed(Problem *P);                                   // streamed.cu
int solve_streamed(Problem *P, const SolveArgs &A, cudaStream_t s);  // streamed.cu
int setup_resident(Problem *P);                                   // resident.cu
bool resident_fits(const Problem *P, int nsm, int *C_out, size_t *smem_out);   // resident.cu
int solve_resident(Problem *P, const SolveArgs &A, cudaStream_t s);  // resident.cu

int setup_solver_launch(Problem *P) {
    int ex = P->params.executor;
    if (ex == SW_EXEC_AUTO) {
        // small periodic 2-D FP64 problems: resident; otherwise by size
        int nsm = 0, C = 0;
        size_t rs = 0;
        cudaError_t e0 = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P->device);
        if (e0 != cudaSuccess) return cuda_fail(e0, "SM count");
        if (resident_fits(P, nsm, &C, &rs)) ex = SW_EXEC_RESIDENT;
        else ex = P->m >= SW_EXEC_STREAMED_MIN ? SW_EXEC_STREAMED : SW_EXEC_PERSISTENT;
    }
    P->exec = ex;
    if (ex == SW_EXEC_STREAMED) {
        int rc = setup_streamed(P);
        if (rc != SW_OK) return rc;
    }
    if (ex == SW_EXEC_RESIDENT) {
        int rc = setup_resident(P);
        if (rc != SW_OK) return rc;
    }
    Tiling t = make_tiling(P->dev);
    size_t smem = solve_smem(P->dev, t);
    const void *kern = solve_kernel_for(P);
    cudaError_t e = ensure_smem((const void *)kern, (size_t)(int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "solve_kernel smem attribute");
    e = ensure_smem((const void *)apply_kernel, (size_t)(int)(2 * (size_t)P->dev.P * t.HW * sizeof(double)));
    if (e != cudaSuccess) return cuda_fail(e, "apply_kernel smem attribute");
    int nsm = 0, per = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P->device);
    if (e != cudaSuccess) return cuda_fail(e, "SM count");
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NTHREADS, smem);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    if (per < 1) { set_error("solve kernel does not fit on an SM"); return SW_ERR_BAD_ARG; }
    // one block per SM; the cross-block gathers are sized for at most 160 blocks
    P->nblocks = nsm < NWARPS * GATHER_PER_WARP ? nsm : NWARPS * GATHER_PER_WARP;
    P->nthreads = NTHREADS;
    P->smem = smem;
    return SW_OK;
}

static Tiling tiling_of(const Problem *P) { return make_tiling(P->dev); }

// Fold the recorded event pairs into the running total.
static int flush_timing(Problem *P) {
    for (int i = 0; i < P->ev_used; ++i) {
        cudaError_t e = cudaEventSynchronize(P->ev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "event sync");
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, P->ev[2 * i], P->ev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "event time");
        P->timed_ms += ms;
        P->n_timed++;
    }
    P->ev_used = 0;
    return SW_OK;
}

// Arguments of one solve of problem P; the FP32 inner form stores its Krylov,
// sketch and W vectors as floats in the same buffers.
SolveArgs make_args(Problem *P, const double *ep, const double *ec, const double *b, double *x, int guess_only) {
    const sw_params &pr = P->params;
    SolveArgs A{};
    A.eta_prev = ep; A.eta_cur = ec; A.b = b; A.x = x;
    A.V = mixed(P) ? (void *)P->d_V32 : (void *)P->d_V;
    A.r = P->d_work; A.t = (void *)(P->d_work + P->m);
    A.Yold = P->d_Y[P->ybuf]; A.Ynew = P->d_Y[P->ybuf ^ 1];
    A.Wm = P->d_W; A.xprev = P->d_xprev; A.part = P->d_part; A.stats = (DevStats *)P->d_stats;
    A.Vq = P->params.orthonormalize ? P->d_Q : nullptr;
    A.tl = tiling_of(P);
    A.restart = pr.restart; A.max_restarts = pr.max_restarts; A.k = pr.k; A.nb = P->nblocks;
    A.tol = pr.tol; A.decay = pr.decay; A.guess_only = guess_only;
    // FP32 inner cycles run like FP64 ones (to the restart length or the
    // global target); the FP64 residual at each restart does the refinement
    A.inner_rtol = 0.0;
    int mode = pr.guess;
    if ((mode == SW_GUESS_EWMA || mode == SW_GUESS_RRF) && P->n_solves < pr.n_init_solves) mode = SW_GUESS_PREVIOUS;
    if (mode == SW_GUESS_RRF && P->n_solves == 0) mode = SW_GUESS_PREVIOUS;
    if (guess_only) mode = pr.guess == SW_GUESS_RRF && P->n_solves > 0 ? SW_GUESS_RRF : SW_GUESS_EWMA;
    A.guess_mode = mode;
    A.cm = P->cost;
    A.pending = P->pending ? 1 : 0;
    if (A.pending) sw_draw_omega(pr.seed, P->n_solves - 1, pr.k, A.omega);
    if (pr.guess == SW_GUESS_RRF) {
        const int K = pr.history;
        A.ring = P->d_X;
        A.ring_K = K;
        A.ring_store = guess_only ? nullptr : P->d_X + (size_t)(P->n_solves % K) * P->m;
        A.ring_Ke = (int)(P->n_solves < K ? P->n_solves : K);
        A.ring_newest = (int)((P->n_solves + K - 1) % K);
        if (mode == SW_GUESS_RRF) {
            // Omega of this solve: K x k, entry (r, c) at r k + c; k_e = min(k, K_e) columns
            double om[SW_RRF_MAX_HISTORY * MAX_K];
            sw_draw_omega(pr.seed, P->n_solves, K * pr.k, om);
            A.k = pr.k < A.ring_Ke ? pr.k : A.ring_Ke;
            for (int r = 0; r < K; ++r)
                for (int c = 0; c < A.k; ++c) A.omega_rrf[r * A.k + c] = om[r * pr.k + c];
        }
    }
    return A;
}

// Bookkeeping after a solve of P was enqueued.
void after_solve(Problem *P, const SolveArgs &A, int guess_only) {
    if (A.pending) P->ybuf ^= 1;
    P->pending = false;
    if (!guess_only) {
        P->n_solves++;
        P->pending = P->params.guess == SW_GUESS_EWMA;
    }
}

static int launch_solve(Problem *P, const double *ep, const double *ec, const double *b, double *x,
                        cudaStream_t s, int guess_only) {
    SolveArgs A = make_args(P, ep, ec, b, x, guess_only);
    Dev D = P->dev;
    void *args[] = {&D, &A};
    cudaError_t e = cudaSuccess;
    int evi = -1;
    if (P->timing) {
        if (P->ev_used * 2 + 2 > (int)P->ev.size()) {
            int rc = flush_timing(P);
            if (rc != SW_OK) return rc;
        }
        evi = P->ev_used++;
        e = cudaEventRecord(P->ev[2 * evi], s);
        if (e != cudaSuccess) return cuda_fail(e, "event record");
    }
    if (P->exec == SW_EXEC_STREAMED) {
        int rc = solve_streamed(P, A, s);
        if (rc != SW_OK) return rc;
    } else if (P->exec == SW_EXEC_RESIDENT) {
        int rc = solve_resident(P, A, s);
        if (rc != SW_OK) return rc;
    } else {
        const void *kern = solve_kernel_for(P);
        e = cudaLaunchCooperativeKernel(kern, P->nblocks, NTHREADS, args, P->smem, s);
        if (e != cudaSuccess) return cuda_fail(e, "solve launch");
        P->launches++;
    }
    if (evi >= 0) {
        e = cudaEventRecord(P->ev[2 * evi + 1], s);
        if (e != cudaSuccess) return cuda_fail(e, "event record");
    }
    after_solve(P, A, guess_only);
    P->last_stream = s;
    return SW_OK;
}

int solve_device(Problem *P, const double *ep, const double *ec, const double *b, double *x, cudaStream_t s) {
    return launch_solve(P, ep, ec, b, x, s, 0);
}

int read_stats(Problem *P, DevStats *out) {
    cudaError_t e = cudaStreamSynchronize(P->last_stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream sync");
    e = cudaMemcpy(out, P->d_stats, sizeof(DevStats), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "stats copy");
    return SW_OK;
}

}  // namespace sw

using namespace sw;

extern "C" int sw_solve_poisson(sw_problem *pp, const double *ep, const double *ec, const double *b, double *x,
                                void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !ep || !ec || !b || !x) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    return solve_device(P, ep, ec, b, x, (cudaStream_t)stream);
}

extern "C" int sw_solve_poisson_host(sw_problem *pp, const double *hep, const double *hec, const double *hb,
                                     double *hx, void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !hep || !hec || !hb || !hx) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    double *db = P->d_host_io, *dx = db + P->m, *dep = dx + P->m, *dec = dep + P->ncol;
    cudaError_t e = cudaMemcpyAsync(db, hb, P->m * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dep, hep, P->ncol * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dec, hec, P->ncol * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    int rc = solve_device(P, dep, dec, db, dx, s);
    if (rc != SW_OK) return rc;
    e = cudaMemcpyAsync(hx, dx, P->m * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    DevStats st;
    rc = read_stats(P, &st);
    if (rc != SW_OK) return rc;
    return st.status;
}

extern "C" int sw_get_stats(sw_problem *pp, sw_stats *out) {
    Problem *P = (Problem *)pp;
    if (!P || !out) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    DevStats st;
    std::memset(&st, 0, sizeof(st));
    if (P->n_solves > 0) {
        int rc = read_stats(P, &st);
        if (rc != SW_OK) return rc;
    }
    out->iterations = st.iterations;
    out->restarts = st.restarts;
    out->converged = st.converged;
    out->status = P->n_solves > 0 ? st.status : SW_OK;
    out->res0 = st.res0;
    out->res_final = st.res_final;
    out->true_res = st.true_res;
    out->guess_res = st.guess_res;
    out->n_solves = P->n_solves;
    out->total_iterations = st.total_iterations;
    out->launches = P->launches;
    out->model_flops = st.model_flops;
    out->model_bytes = st.model_bytes;
    out->executor = P->exec;
    return SW_OK;
}

extern "C" int sw_get_phase_times(sw_problem *pp, double *us, int n) {
    Problem *P = (Problem *)pp;
    if (!P || !us || n < 1) { set_error("bad argument"); return SW_ERR_BAD_ARG; }
    DevStats st;
    std::memset(&st, 0, sizeof(st));
    if (P->n_solves > 0) {
        int rc = read_stats(P, &st);
        if (rc != SW_OK) return rc;
    }
    for (int i = 0; i < n && i < 16; ++i) us[i] = i < PH_COUNT ? st.phase_ns[i] * 1e-3 : 0.0;
    return SW_OK;
}

extern "C" int sw_enable_timing(sw_problem *pp, int on) {
    Problem *P = (Problem *)pp;
    if (!P) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    if (on && P->ev.empty()) {
        P->ev.resize(512);
        for (auto &ev : P->ev) {
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return cuda_fail(e, "event create");
        }
    }
    if (P->timing && !on) {
        int rc = flush_timing(P);
        if (rc != SW_OK) return rc;
    }
    P->timing = on != 0;
    P->timed_ms = 0.0;
    P->n_timed = 0;
    P->ev_used = 0;
    return SW_OK;
}

extern "C" int sw_get_solve_time(sw_problem *pp, double *total_ms, long long *n_timed) {
    Problem *P = (Problem *)pp;
    if (!P || !total_ms || !n_timed) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    int rc = flush_timing(P);
    if (rc != SW_OK) return rc;
    *total_ms = P->timed_ms;
    *n_timed = P->n_timed;
    return SW_OK;
}

extern "C" int sw_apply_operator(sw_problem *pp, const double *ep, const double *ec, const double *x, double *y,
                                 void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !ep || !ec || !x || !y) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    Tiling tl = tiling_of(P);
    int gb = (P->ncol + NTHREADS - 1) / NTHREADS;
    geometry_kernel<<<gb, NTHREADS, 0, s>>>(P->dev, ep, ec);
    apply_kernel<<<tl.ntiles, NTHREADS, 2 * (size_t)P->dev.P * tl.HW * sizeof(double), s>>>(P->dev, tl, x, y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "apply launch");
    P->launches += 2;
    P->last_stream = s;
    return SW_OK;
}

extern "C" int sw_apply_preconditioner(sw_problem *pp, const double *v, double *out, void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !v || !out || v == out) { set_error("bad argument"); return SW_ERR_BAD_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const Dev &D = P->dev;
    for (int c = 0; c < D.ngroups; ++c) {
        int blocks = ((P->goff_h[c + 1] - P->goff_h[c]) * 32 + NTHREADS - 1) / NTHREADS;
        ilu_fwd_kernel<<<blocks, NTHREADS, 0, s>>>(D, c, v, out);
    }
    for (int c = D.ngroups - 1; c >= 0; --c) {
        int blocks = ((P->goff_h[c + 1] - P->goff_h[c]) * 32 + NTHREADS - 1) / NTHREADS;
        ilu_bwd_kernel<<<blocks, NTHREADS, 0, s>>>(D, c, out);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "preconditioner launch");
    P->launches += 2 * D.ngroups;
    P->last_stream = s;
    return SW_OK;
}

extern "C" int sw_subspace_guess(sw_problem *pp, const double *ep, const double *ec, const double *b, double *x0,
                                 void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !ep || !ec || !b || !x0) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    return launch_solve(P, ep, ec, b, x0, (cudaStream_t)stream, 1);
}

extern "C" int sw_get_sketch(sw_problem *pp, double *Y, void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !Y) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    // The update with the newest solution is applied lazily at the start of
    // the next solve; apply it here on the copy when one is pending.
    cudaStream_t s = (cudaStream_t)stream;
    SketchUpd u{};
    if (P->pending) sw_draw_omega(P->params.seed, P->n_solves - 1, P->params.k, u.om);
    int blocks = (int)((P->m + NTHREADS - 1) / NTHREADS);
    if (blocks > 4096) blocks = 4096;
    sketch_update_kernel<double><<<blocks, NTHREADS, 0, s>>>(P->d_Y[P->ybuf], Y, P->d_xprev, u, P->params.k, P->m,
                                                             P->params.decay, P->pending);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "sketch launch");
    P->launches++;
    P->last_stream = s;
    return SW_OK;
}

extern "C" int sw_set_sketch(sw_problem *pp, const double *Y, long long n_solves, void *stream) {
    Problem *P = (Problem *)pp;
    if (!P || !Y || n_solves < 0) { set_error("bad argument"); return SW_ERR_BAD_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = (long long)P->params.k * P->m;
    int blocks = (int)((n + NTHREADS - 1) / NTHREADS);
    if (blocks > 4096) blocks = 4096;
    sketch_store_kernel<double><<<blocks, NTHREADS, 0, s>>>(Y, P->d_Y[P->ybuf], n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "sketch launch");
    P->launches++;
    // the loaded sketch is complete: no update pending; later draws continue at n_solves
    P->n_solves = n_solves;
    P->pending = false;
    P->last_stream = s;
    return SW_OK;
}
