// Operator apply y = A(eta_prev, eta_cur) x for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: code running under a memory budget
// that forbids new device allocations, code inside a pre-planned memory pool,
// or a host framework that hands over only the buffers it owns.  For them this
// entry point keeps its scratch (finite-difference weights, bathymetry
// derivatives and the per-column geometry coefficients) in one file-scope
// static device array instead of problem-owned allocations.  The caller passes
// the depth, both surfaces, x and y as device pointers; nothing is allocated.
//
// The array holds at most SW_NOALLOC_MAX_COLUMNS columns (65,536, about
// 12.6 MB); every GPU that loads the library keeps it until the process exits.
// On the first call on a device (with that device current) the host resolves
// the array's device address with cudaGetSymbolAddress and sets the kernel
// attributes; that first call should come before any stream capture.  The
// weights travel to the device as a kernel argument, so a call issues kernel
// launches only.  All calls share the one array and every call rewrites
// everything it reads, so nothing needs clearing between calls, but two calls
// that overlap on the GPU (different streams, or different host threads) race
// on it.
#include <cmath>
#include <cstring>
#include <mutex>

#include "sw_device.cuh"

#define SW_NOALLOC_MAX_COLUMNS 65536

namespace sw {
namespace {

constexpr int NA_WEIGHTS = 4 * W + 2 * MAX_LEVELS * W;     // 924 doubles
constexpr int NA_HEAD = 1024;                              // weights region (doubles)
constexpr int NA_WIN = 32;                                 // 64 ints
constexpr int NA_COLS = SW_NOALLOC_MAX_COLUMNS;
constexpr int NA_HDERIV = 4;                               // h_x, h_y, h_xx, h_yy
constexpr int NA_CC = 20;                                  // per-column coefficients (NCC used)
constexpr size_t NA_TOTAL = NA_HEAD + NA_WIN + (size_t)(NA_HDERIV + NA_CC) * NA_COLS;

static_assert(NA_WEIGHTS <= NA_HEAD, "weights region");
static_assert(NCC <= NA_CC, "coefficient region");

static __device__ __align__(256) double g_noalloc_scratch[NA_TOTAL];

// Host-side copy of the array's device address, per device, set once under
// the mutex.
constexpr int NA_MAX_DEVICES = 64;
double *g_dev_ptr[NA_MAX_DEVICES] = {};
std::mutex g_setup_mutex;

// Weights and sigma windows of one call, passed by value (7.6 KB of kernel
// arguments) to the kernel that installs them in the array.
struct NaHead {
    double w[NA_WEIGHTS];
    int win[MAX_LEVELS];
};

__global__ void na_install_kernel(NaHead hd, double *base) {
    for (int i = threadIdx.x; i < NA_WEIGHTS; i += blockDim.x) base[i] = hd.w[i];
    int *win = reinterpret_cast<int *>(base + NA_HEAD);
    for (int i = threadIdx.x; i < MAX_LEVELS; i += blockDim.x) win[i] = hd.win[i];
}

struct NaLoad {
    const double *v;
    __device__ double operator()(long long i) const { return v[i]; }
};
struct NaStore {
    double *y;
    __device__ void operator()(long long i, double v) const { y[i] = v; }
};

__global__ void na_hderiv_kernel(Dev D, double *hx, double *hy, double *hxx, double *hyy) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D.ncol) return;
    int ix = c % D.nx, iy = c / D.nx;
    double s1 = 0, s2 = 0, t1 = 0, t2 = 0;
#pragma unroll
    for (int t = -HALF; t <= HALF; ++t) {
        double vx = D.h[iy * D.nx + wrapi(ix + t, D.nx)];
        s1 += D.wx1[t + HALF] * vx;
        s2 += D.wx2[t + HALF] * vx;
        if (D.three_d) {
            double vy = D.h[wrapi(iy + t, D.ny) * D.nx + ix];
            t1 += D.wy1[t + HALF] * vy;
            t2 += D.wy2[t + HALF] * vy;
        }
    }
    hx[c] = s1;
    hxx[c] = s2;
    hy[c] = t1;
    hyy[c] = t2;
}

__global__ void na_geometry_kernel(Dev D, const double *ep, const double *ec) {
    geometry_columns(D, ep, ec, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void __launch_bounds__(NTHREADS) na_apply_kernel(Dev D, Tiling tl, const double *x, double *y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *sp = reinterpret_cast<double *>(smem_raw);
    double *sq = sp + (size_t)D.P * tl.HW;
    NaLoad ld{x};
    NaStore st{y};
    for (int tile = blockIdx.x; tile < tl.ntiles; tile += gridDim.x) apply_tile<double>(D, tl, tile, sp, sq, ld, st);
}

Tiling na_tiling(const Dev &D) {
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

// First call on a device: resolve the array's address and set the kernel's
// shared-memory limit (neither allocates).
int na_setup(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= NA_MAX_DEVICES) { set_error("device index out of range"); return SW_ERR_BAD_ARG; }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
        e = ensure_smem((const void *)na_apply_kernel, (size_t)200 * 1024);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        g_dev_ptr[dev] = (double *)p;
    }
    *out = g_dev_ptr[dev];
    return SW_OK;
}

}  // namespace
}  // namespace sw

using namespace sw;

extern "C" int sw_apply_operator_noalloc(const sw_grid *grid, const double *d_h, const double *d_eta_prev,
                                         const double *d_eta_cur, const double *d_x, double *d_y, void *stream) {
    if (!grid || !d_h || !d_eta_prev || !d_eta_cur || !d_x || !d_y) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    const sw_grid g = *grid;
    const bool three_d = g.ny > 1;
    if (g.nx < 8 || g.nx % 4 != 0 || g.ny < 1 || (three_d && (g.ny < 8 || g.ny % 4 != 0)) || g.nz < W ||
        g.nz + 1 > MAX_LEVELS || !(g.lx > 0) || (three_d && !(g.ly > 0))) {
        set_error("grid: need nx (and ny in 3-D) multiples of 4 and >= 8, 7 <= nz <= 63, positive lengths");
        return SW_ERR_BAD_ARG;
    }
    if (g.walls) {
        set_error("sw_apply_operator_noalloc: periodic grids only");
        return SW_ERR_BAD_ARG;
    }
    if ((long long)g.nx * g.ny > SW_NOALLOC_MAX_COLUMNS) {
        set_error("sw_apply_operator_noalloc: nx*ny exceeds the static scratch limit of 65536 columns");
        return SW_ERR_BAD_ARG;
    }
    double *base = nullptr;
    int rc = na_setup(&base);
    if (rc != SW_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int P = g.nz + 1;
    const int ncol = g.nx * g.ny;
    // weights and sigma windows (the same host builder as sw_create_problem),
    // installed by a kernel that receives them by value
    NaHead hd;
    std::memset(&hd, 0, sizeof(hd));
    {
        const sw_grid gp = {g.nx, g.ny, g.nz, g.lx, three_d ? g.ly : 0.0, 0};
        grid_weights(gp, hd.w, hd.w + W, hd.w + 2 * W, hd.w + 3 * W, hd.w + 4 * W, hd.w + 4 * W + P * W, hd.win);
    }
    na_install_kernel<<<1, 256, 0, s>>>(hd, base);
    double *hder = base + NA_HEAD + NA_WIN;
    double *cc = hder + (size_t)NA_HDERIV * NA_COLS;
    Dev D{};
    D.nx = g.nx; D.ny = g.ny; D.nz = g.nz; D.P = P; D.ncol = ncol; D.three_d = three_d;
    D.layout = 0; D.nslot = 0; D.m = (long long)ncol * P;
    D.dx = g.lx / g.nx; D.dy = three_d ? g.ly / g.ny : 1.0;
    D.wx1 = base; D.wx2 = base + W; D.wy1 = base + 2 * W; D.wy2 = base + 3 * W;
    D.ws1 = base + 4 * W; D.ws2 = base + 4 * W + P * W;
    D.win = reinterpret_cast<const int *>(base + NA_HEAD);
    D.h = d_h;
    D.hx = hder; D.hy = hder + NA_COLS; D.hxx = hder + 2 * NA_COLS; D.hyy = hder + 3 * NA_COLS;
    D.gp = cc;   // coefficient c of column col at cc[c * ncol + col]
    const int T = 256;
    const int gc = (ncol + T - 1) / T;
    na_hderiv_kernel<<<gc, T, 0, s>>>(D, (double *)D.hx, (double *)D.hy, (double *)D.hxx, (double *)D.hyy);
    na_geometry_kernel<<<gc, T, 0, s>>>(D, d_eta_prev, d_eta_cur);
    Tiling tl = na_tiling(D);
    size_t smem = 2 * (size_t)P * tl.HW * sizeof(double);
    na_apply_kernel<<<tl.ntiles, NTHREADS, smem, s>>>(D, tl, d_x, d_y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "noalloc apply launch");
    return SW_OK;
}
