// Host-side set-up of a problem: finite-difference weights, the still-water
// operator in slot form, its ILU(0) factorisation in the column-group
// ordering, and the device allocations.
//
// Preconditioner (Sec. 3 and Sec. 5): one incomplete LU factorisation of the
// operator built for the still-water state eta = 0, computed once and reused
// for every stage.  Variant ILU(0): fill restricted to the sparsity pattern of
// that operator.  Ordering: column group first, then the column, then the level
// from the ghost level up.  Periodic grids use the colours (ix + iy) mod 4:
// with nx, ny multiples of four, columns of one colour never share a 7-point
// stencil, which lets the device sweep all columns of a colour at once.  With
// walls, the six columns next to the walls (whose rows reach 7 columns
// inwards) form three more groups after the four colours.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <thread>

#include "sw_internal.cuh"

namespace sw {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
int cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return SW_ERR_CUDA;
}

cudaError_t ensure_smem(const void *kern, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> set_to;   // (device, kernel) -> limit set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t &cur = set_to[{dev, kern}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

// Derivative weights at z from the Lagrange basis polynomials through nodes
// x[0..6]: the d-th derivative of l_i at z is d! times the coefficient of
// (x - z)^d in prod_{q != i} (x - x_q) / prod_{q != i} (x_i - x_q).
void lagrange_weights(const long double *x, long double z, double *w1, double *w2) {
    for (int i = 0; i < W; ++i) {
        long double c[W] = {1.0L};  // coefficients in powers of t = x - z
        int deg = 0;
        long double den = 1.0L;
        for (int q = 0; q < W; ++q) {
            if (q == i) continue;
            long double r = x[q] - z;  // factor (t - r)
            for (int p = deg + 1; p >= 1; --p) c[p] = c[p - 1] - r * c[p];
            c[0] = -r * c[0];
            ++deg;
            den *= (x[i] - x[q]);
        }
        w1[i] = (double)(c[1] / den);
        w2[i] = (double)(2.0L * c[2] / den);
    }
}

int sigma_window(int nz, int j) {
    int s = j - HALF;
    if (s < -1) s = -1;
    if (s > nz - W) s = nz - W;
    return s;
}

void grid_weights(const sw_grid &g, double *wx1, double *wx2, double *wy1, double *wy2, double *ws1, double *ws2,
                  int *win) {
    const double dx = g.walls ? g.lx / (g.nx - 3) : g.lx / g.nx;
    const double dy = g.ny > 1 ? g.ly / g.ny : 1.0;
    long double xs[W];
    for (int t = 0; t < W; ++t) xs[t] = (long double)(t - HALF) * (long double)dx;
    lagrange_weights(xs, 0.0L, wx1, wx2);
    for (int t = 0; t < W; ++t) xs[t] = (long double)(t - HALF) * (long double)dy;
    lagrange_weights(xs, 0.0L, wy1, wy2);
    for (int j = -1; j < g.nz; ++j) {
        const int s0 = sigma_window(g.nz, j);
        win[j + 1] = s0;
        for (int k = 0; k < W; ++k) xs[k] = (long double)(s0 + k) / (long double)(g.nz - 1);
        lagrange_weights(xs, (long double)j / (long double)(g.nz - 1), ws1 + (j + 1) * W, ws2 + (j + 1) * W);
    }
}

namespace {

struct Host {
    int nx, ny, nz, P, ncol, layout, nslot, three_d, walls;
    long long m;
    double dx, dy;
    double wx1[W], wx2[W], wy1[W], wy2[W];
    double wxo1[W][W], wxo2[W][W];  // walls: weights at node o of a window of 7 equispaced nodes
    std::vector<double> ws1, ws2;   // P x W
    std::vector<int> win;           // P
    std::vector<double> h, hx, hy, hxx, hyy;
    // column groups of the factorisation order (see build_groups)
    int ngroups = 4;
    std::vector<int> goff, gcol, colrank;
    std::vector<unsigned char> grp;

    // Periodic: colour (ix + iy) mod 4, columns in index order within a colour.
    // Walls: the rows of columns 0-2 and nx-3..nx-1 reach 7 columns inwards, so
    // those six columns form three groups {0, nx-1}, {1, nx-2}, {2, nx-3} after
    // the four colours ix mod 4 of columns 3..nx-4.  No two columns of one group
    // share a row's x window.
    void build_groups() {
        gcol.clear();
        ngroups = walls ? 7 : 4;
        goff.assign(ngroups + 1, 0);
        grp.assign(ncol, 0);
        for (int c = 0; c < 4; ++c) {
            goff[c] = (int)gcol.size();
            if (walls) {
                for (int ix = 3; ix <= nx - 4; ++ix)
                    if (ix % 4 == c) gcol.push_back(ix);
            } else {
                for (int iy = 0; iy < ny; ++iy)
                    for (int ix = 0; ix < nx; ++ix)
                        if (((ix + iy) & 3) == c) gcol.push_back(iy * nx + ix);
            }
        }
        if (walls)
            for (int e = 0; e < 3; ++e) {
                goff[4 + e] = (int)gcol.size();
                gcol.push_back(e);
                gcol.push_back(nx - 1 - e);
            }
        goff[ngroups] = (int)gcol.size();
        colrank.assign(ncol, 0);
        for (int g = 0; g < ngroups; ++g)
            for (int r = goff[g]; r < goff[g + 1]; ++r) {
                colrank[gcol[r]] = r;
                grp[gcol[r]] = (unsigned char)g;
            }
    }
    long long rank_of(int ix, int iy, int j) const { return (long long)colrank[iy * nx + ix] * P + (j + 1); }
    void node_of_rank(long long r, int &ix, int &iy, int &j) const {
        const int col = gcol[r / P];
        j = (int)(r % P) - 1;
        ix = col % nx;
        iy = col / nx;
    }
    int wrapx(int i) const { i %= nx; return i < 0 ? i + nx : i; }
    int wrapy(int i) const { i %= ny; return i < 0 ? i + ny : i; }
    // x window of the unknowns at column ix: first column (walls) and position of ix in it
    int xs(int ix) const { return walls ? std::min(std::max(ix - HALF, 0), nx - W) : ix - HALF; }
    int own_pos(int ix) const { return ix - xs(ix); }
    int xcol(int ix, int t) const { return walls ? xs(ix) + t : wrapx(ix - HALF + t); }
    const double *xw1(int ix) const { return walls ? wxo1[own_pos(ix)] : wx1; }
    const double *xw2(int ix) const { return walls ? wxo2[own_pos(ix)] : wx2; }
    bool ghost_col(int ix) const { return walls && (ix == 0 || ix == nx - 1); }

    // neighbour of slot s for row (ix, iy, j)
    void slot_nb(int s, int ix, int iy, int j, int &nx_, int &ny_, int &lev) const {
        static const int off[6] = {-3, -2, -1, 1, 2, 3};
        int ox = 0, oy = 0;
        int w0 = win[j + 1];
        const int o = own_pos(ix);
        switch (layout) {
        case CROSS2D:
            if (s < 6) { nx_ = xcol(ix, s < o ? s : s + 1); lev = j; } else { nx_ = ix; lev = w0 + (s - 6); }
            ny_ = 0;
            return;
        case BOX2D:
            nx_ = xcol(ix, s / 7); lev = w0 + s % 7; ny_ = 0;
            return;
        case CROSS3D:
            if (s < 6) { ox = off[s]; lev = j; }
            else if (s < 12) { oy = off[s - 6]; lev = j; }
            else { lev = w0 + (s - 12); }
            break;
        default:
            if (s < 49) { ox = s / 7 - 3; lev = w0 + s % 7; }
            else { oy = off[(s - 49) / 7]; lev = w0 + (s - 49) % 7; }
        }
        nx_ = wrapx(ix + ox);
        ny_ = ny > 1 ? wrapy(iy + oy) : 0;
    }
    // structural pattern of the still-water operator in row (ix, j)
    bool in_pattern(int s, int ix, int j) const {
        const int o = three_d ? HALF : own_pos(ix);
        if (j == nz - 1) return s == own_slot(layout, W - 1, o);
        if (ghost_col(ix)) {
            // wall row: x window at the row's level, and (box) the wall column's sigma window
            const int kkj = j - win[j + 1];
            if (layout == CROSS2D) return s < 6 || s == 6 + kkj;
            const int tw = (ix == 0 ? 1 : nx - 2) - xs(ix);
            return s % 7 == kkj || s / 7 == tw;
        }
        if (j == -1) {
            int ss = own_slot(layout, 0, o);
            if (s >= ss && s < ss + W) return true;
            if (layout == CROSS2D || layout == CROSS3D) return false;
            // box: horizontal entries at the bed level (window offset 1)
            if (layout == BOX2D) return s % 7 == 1;
            return (s < 49 ? s % 7 : (s - 49) % 7) == 1;
        }
        return true;
    }
    // slot of row (ix, iy, j) that refers to node (bx, by, lev), or -1
    int find_slot(int ix, int iy, int j, int bx, int by, int lev) const {
        int kk = lev - win[j + 1];
        auto xoff = [](int o) { return o < 0 ? o + 3 : o + 2; };  // -3..-1,1..3 -> 0..5
        if (!three_d) {
            int t;
            if (walls) {
                t = bx - xs(ix);
            } else {
                int dxo = bx - ix;
                if (dxo > nx / 2) dxo -= nx;
                if (dxo < -nx / 2) dxo += nx;
                t = dxo + HALF;
            }
            const int o = own_pos(ix);
            if (t < 0 || t >= W) return -1;
            if (layout == CROSS2D) {
                if (t == o) return (kk >= 0 && kk < W) ? 6 + kk : -1;
                return lev == j ? (t < o ? t : t - 1) : -1;
            }
            return (kk >= 0 && kk < W) ? t * 7 + kk : -1;
        }
        int dxo = bx - ix, dyo = by - iy;
        if (dxo > nx / 2) dxo -= nx;
        if (dxo < -nx / 2) dxo += nx;
        if (dyo > ny / 2) dyo -= ny;
        if (dyo < -ny / 2) dyo += ny;
        switch (layout) {
        case CROSS3D:
            if (dxo == 0 && dyo == 0) return (kk >= 0 && kk < W) ? 12 + kk : -1;
            if (lev != j) return -1;
            if (dyo == 0 && dxo >= -3 && dxo <= 3) return xoff(dxo);
            if (dxo == 0 && dyo >= -3 && dyo <= 3) return 6 + xoff(dyo);
            return -1;
        default:
            if (kk < 0 || kk >= W) return -1;
            if (dyo == 0 && dxo >= -3 && dxo <= 3) return (dxo + 3) * 7 + kk;
            if (dxo == 0 && dyo >= -3 && dyo <= 3) return 49 + xoff(dyo) * 7 + kk;
            return -1;
        }
    }

    // Row of the still-water operator (eta = 0, d = h) in slot form,
    // following Eq. (16)-(18) with the push-forward of Eq. (9b) and (13b-13d);
    // with walls, the ghost-column rows are the wall conditions of Sec. 3.
    void a0_row(int ix, int iy, int j, double *v) const {
        for (int s = 0; s < nslot; ++s) v[s] = 0.0;
        int c = iy * nx + ix;
        const int o = three_d ? HALF : own_pos(ix);
        if (j == nz - 1) { v[own_slot(layout, W - 1, o)] = 1.0; return; }
        bool box = layout == BOX2D || layout == BOX3D;
        if (ghost_col(ix)) {
            // n . grad p at the wall node (iw, j), n = (-1, 0) at x = 0 and (1, 0) at x = lx
            const int iw = ix == 0 ? 1 : nx - 2;
            const double nxs = ix == 0 ? -1.0 : 1.0;
            const double *w1x = xw1(iw);
            for (int t = 0; t < W; ++t) v[find_slot(ix, iy, j, xcol(iw, t), 0, j)] += nxs * w1x[t];
            if (box) {
                const double sg = (double)j / (nz - 1);
                const double a = (hx[iw] - sg * hx[iw]) / h[iw];   // sigma_x at still water
                for (int kk = 0; kk < W; ++kk)
                    v[find_slot(ix, iy, j, iw, 0, win[j + 1] + kk)] += nxs * a * ws1[(j + 1) * W + kk];
            }
            return;
        }
        double d = h[c], f = 1.0 / d;
        double gx = hx[c], gy = three_d ? hy[c] : 0.0;
        const double *w1x = xw1(ix), *w2x = xw2(ix);
        if (j == -1) {
            double nrm = 1.0 / std::sqrt(1.0 + gx * gx + gy * gy);
            double a0 = gx * f, a0y = gy * f;
            double cs = -nrm * (gx * a0 + gy * a0y + f);
            const double *w1 = &ws1[1 * W];   // sigma weights of level 0
            for (int kk = 0; kk < W; ++kk) v[own_slot(layout, kk, o)] += cs * w1[kk];
            if (box) {
                for (int t = 0; t < W; ++t) {
                    if (t == o) {
                        v[own_slot(layout, 1, o)] += -nrm * gx * w1x[t] - nrm * gy * (three_d ? wy1[t] : 0.0);
                        continue;
                    }
                    int s = find_slot(ix, iy, j, xcol(ix, t), iy, 0);
                    v[s] += -nrm * gx * w1x[t];
                    if (three_d) {
                        int s2 = find_slot(ix, iy, j, ix, wrapy(iy + t - HALF), 0);
                        v[s2] += -nrm * gy * wy1[t];
                    }
                }
            }
            return;
        }
        double sg = (double)j / (nz - 1);
        const double *w1 = &ws1[(j + 1) * W];
        const double *w2 = &ws2[(j + 1) * W];
        int w0 = win[j + 1];
        double a = (gx - sg * hx[c]) * f;           // sigma_x (both stages equal at rest)
        double as = -hx[c] * f;
        double ax = (hxx[c] - sg * hxx[c] - a * hx[c]) * f;
        double ay = 0, ays = 0, ayy = 0;
        if (three_d) {
            ay = (gy - sg * hy[c]) * f;
            ays = -hy[c] * f;
            ayy = (hyy[c] - sg * hyy[c] - ay * hy[c]) * f;
        }
        double c_ss = a * a + ay * ay + f * f;
        double c_s = ax + a * as + ayy + ay * ays;
        for (int t = 0; t < W; ++t) {
            int s = find_slot(ix, iy, j, xcol(ix, t), iy, j);
            v[s] += w2x[t];
            if (three_d) {
                int s2 = find_slot(ix, iy, j, ix, wrapy(iy + t - HALF), j);
                v[s2] += wy2[t];
            }
        }
        for (int kk = 0; kk < W; ++kk) v[own_slot(layout, kk, o)] += c_ss * w2[kk] + c_s * w1[kk];
        if (box) {
            for (int t = 0; t < W; ++t)
                for (int kk = 0; kk < W; ++kk) {
                    int s = find_slot(ix, iy, j, xcol(ix, t), iy, w0 + kk);
                    v[s] += 2.0 * a * w1x[t] * w1[kk];
                    if (three_d) {
                        int s2 = find_slot(ix, iy, j, ix, wrapy(iy + t - HALF), w0 + kk);
                        v[s2] += 2.0 * ay * wy1[t] * w1[kk];
                    }
                }
        }
    }
};

// ILU(0), row by row in rank order (IKJ form): for each row i and each entry
// k < i of its pattern in increasing order, l_ik = a_ik / u_kk, then
// a_ij -= l_ik u_kj for every j > k present in both row k and row i.
// Rows of one column are consecutive ranks and only reference earlier groups
// or the same column, so the columns of one group are factorised in parallel.
static void factorise_column(const Host &H, int c, int q, std::vector<double> &lu, std::vector<double> &udinv,
                             std::vector<double> &v, std::vector<std::pair<long long, int>> &lower, int &status) {
    const int ns = H.nslot;
    for (int a = 0; a < H.P; ++a) {
        const long long i = ((long long)H.goff[c] + q) * H.P + a;
        int ix, iy, j;
        H.node_of_rank(i, ix, iy, j);
        H.a0_row(ix, iy, j, v.data());
        lower.clear();
        for (int s = 0; s < ns; ++s) {
            if (!H.in_pattern(s, ix, j)) { v[s] = 0.0; continue; }
            int bx, by, bl;
            H.slot_nb(s, ix, iy, j, bx, by, bl);
            long long k = H.rank_of(bx, by, bl);
            if (k < i) lower.push_back({k, s});
        }
        std::sort(lower.begin(), lower.end());
        for (auto &ks : lower) {
            const long long k = ks.first;
            const int s = ks.second;
            const double l = v[s] * udinv[k];
            v[s] = l;
            int kx, ky, kj;
            H.node_of_rank(k, kx, ky, kj);
            const double *rowk = &lu[(size_t)k * ns];
            for (int s2 = 0; s2 < ns; ++s2) {
                if (!H.in_pattern(s2, kx, kj)) continue;
                int bx, by, bl;
                H.slot_nb(s2, kx, ky, kj, bx, by, bl);
                if (H.rank_of(bx, by, bl) <= k) continue;
                int s3 = H.find_slot(ix, iy, j, bx, by, bl);
                if (s3 < 0 || !H.in_pattern(s3, ix, j)) continue;
                v[s3] -= l * rowk[s2];
            }
        }
        const double ud = v[own_slot(H.layout, j - H.win[j + 1], H.three_d ? HALF : H.own_pos(ix))];
        if (ud == 0.0 || !std::isfinite(ud)) { status = SW_ERR_SINGULAR_PRECOND; return; }
        udinv[i] = 1.0 / ud;
        std::copy(v.begin(), v.end(), lu.begin() + (size_t)i * ns);
    }
}

static int factorise(const Host &H, std::vector<double> &lu, std::vector<double> &udinv) {
    const int ns = H.nslot;
    const long long m = H.m;
    lu.assign((size_t)m * ns, 0.0);   // row-major during the factorisation
    udinv.assign((size_t)m, 0.0);
    unsigned hw = std::thread::hardware_concurrency();
    int nt = (int)std::max(1u, std::min(hw ? hw : 1u, 32u));
    if (m < 20000) nt = 1;
    std::vector<int> status(nt, SW_OK);
    for (int c = 0; c < H.ngroups; ++c) {
        const int per = H.goff[c + 1] - H.goff[c];
        auto work = [&](int t) {
            std::vector<double> v(ns);
            std::vector<std::pair<long long, int>> lower;
            for (int q = t; q < per && status[t] == SW_OK; q += nt) factorise_column(H, c, q, lu, udinv, v, lower, status[t]);
        };
        if (nt == 1) {
            work(0);
        } else {
            std::vector<std::thread> th;
            for (int t = 0; t < nt; ++t) th.emplace_back(work, t);
            for (auto &x : th) x.join();
        }
        for (int t = 0; t < nt; ++t)
            if (status[t] != SW_OK) return status[t];
    }
    return SW_OK;
}

}  // namespace

static int dalloc(Problem *P, void **ptr, size_t bytes) {
    cudaError_t e = cudaMalloc(ptr, bytes ? bytes : 16);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    P->allocs.push_back(*ptr);
    e = cudaMemset(*ptr, 0, bytes ? bytes : 16);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
    return SW_OK;
}

int setup_solver_launch(Problem *P);  // solver.cu

}  // namespace sw

using namespace sw;

extern "C" const char *sw_last_error(void) { return g_err.c_str(); }

extern "C" int sw_create_problem(const sw_grid *grid, const sw_params *params, const double *h_depth,
                                 sw_problem **out) {
    if (!grid || !params || !h_depth || !out) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    *out = nullptr;
    const sw_grid g = *grid;
    const sw_params p = *params;
    bool three_d = g.ny > 1;
    if (g.nx < 8 || g.nx % 4 != 0 || g.ny < 1 || (three_d && (g.ny < 8 || g.ny % 4 != 0)) || g.nz < W ||
        g.nz + 1 > MAX_LEVELS || !(g.lx > 0) || (three_d && !(g.ly > 0))) {
        set_error("grid: need nx (and ny in 3-D) multiples of 4 and >= 8, 7 <= nz <= 63, positive lengths");
        return SW_ERR_BAD_ARG;
    }
    if (g.walls != 0 && (g.walls != 1 || three_d || g.nx < 16)) {
        set_error("grid: walls need a 2-D grid with nx >= 16");
        return SW_ERR_BAD_ARG;
    }
    if (p.orthonormalize != 0 && p.orthonormalize != 1) {
        set_error("params: orthonormalize must be 0 or 1");
        return SW_ERR_BAD_ARG;
    }
    if (p.guess == SW_GUESS_RRF && (p.history < p.k || p.history > SW_RRF_MAX_HISTORY)) {
        set_error("params: the range finder needs k <= history <= 16");
        return SW_ERR_BAD_ARG;
    }
    if (p.restart < 1 || p.restart > MAX_RESTART || p.max_restarts < 0 || !(p.tol > 0) || p.guess < 0 ||
        p.guess > 3 || p.k < 1 || p.k > MAX_K || !(p.decay > 0) || p.decay > 1 || p.n_init_solves < 0 ||
        (p.precision != SW_PRECISION_FP64 && p.precision != SW_PRECISION_MIXED) || p.executor < 0 ||
        p.executor > SW_EXEC_RESIDENT) {
        set_error("params: restart 1..32, k 1..16, decay in (0,1], tol > 0, known guess/precision/executor");
        return SW_ERR_BAD_ARG;
    }
    Host H;
    H.nx = g.nx; H.ny = g.ny; H.nz = g.nz; H.P = g.nz + 1; H.ncol = g.nx * g.ny;
    H.three_d = three_d;
    H.walls = g.walls;
    H.m = (long long)H.ncol * H.P;
    H.dx = H.walls ? g.lx / (g.nx - 3) : g.lx / g.nx;
    H.dy = three_d ? g.ly / g.ny : 1.0;
    bool flat = true;
    H.h.assign(h_depth, h_depth + H.ncol);
    for (int c = 0; c < H.ncol; ++c) {
        if (!(H.h[c] > 0) || !std::isfinite(H.h[c])) { set_error("depth must be positive"); return SW_ERR_BAD_ARG; }
        if (H.h[c] != H.h[0]) flat = false;
    }
    H.layout = three_d ? (flat ? CROSS3D : BOX3D) : (flat ? CROSS2D : BOX2D);
    H.nslot = layout_nslot(H.layout);
    {
        H.ws1.resize(H.P * W); H.ws2.resize(H.P * W); H.win.resize(H.P);
        grid_weights(g, H.wx1, H.wx2, H.wy1, H.wy2, H.ws1.data(), H.ws2.data(), H.win.data());
        // walls: every evaluation point o of a window of 7 equispaced nodes
        long double xs[W];
        for (int t = 0; t < W; ++t) xs[t] = (long double)t * (long double)H.dx;
        for (int o = 0; o < W; ++o) lagrange_weights(xs, (long double)o * (long double)H.dx, H.wxo1[o], H.wxo2[o]);
    }
    // surface-grid derivatives of the bathymetry (D_chi, D_gamma of Sec. 3);
    // with walls over the physical columns, a ghost column taking its wall column's
    H.hx.assign(H.ncol, 0.0); H.hy.assign(H.ncol, 0.0); H.hxx.assign(H.ncol, 0.0); H.hyy.assign(H.ncol, 0.0);
    for (int iy = 0; iy < g.ny; ++iy)
        for (int ix = 0; ix < g.nx; ++ix) {
            double s1 = 0, s2 = 0, t1 = 0, t2 = 0;
            int xe = ix, x0 = ix - HALF;
            const double *w1 = H.wx1, *w2 = H.wx2;
            if (H.walls) {
                xe = std::min(std::max(ix, 1), g.nx - 2);
                x0 = std::min(std::max(xe - HALF, 1), g.nx - 1 - W);
                w1 = H.wxo1[xe - x0];
                w2 = H.wxo2[xe - x0];
            }
            for (int t = -HALF; t <= HALF; ++t) {
                double vx = H.h[iy * g.nx + H.wrapx(x0 + HALF + t)];
                s1 += w1[t + HALF] * vx;
                s2 += w2[t + HALF] * vx;
                if (three_d) {
                    double vy = H.h[H.wrapy(iy + t) * g.nx + ix];
                    t1 += H.wy1[t + HALF] * vy;
                    t2 += H.wy2[t + HALF] * vy;
                }
            }
            int c = iy * g.nx + ix;
            H.hx[c] = s1; H.hxx[c] = s2; H.hy[c] = t1; H.hyy[c] = t2;
        }
    H.build_groups();
    std::vector<double> lu_rows, udinv;
    int st = factorise(H, lu_rows, udinv);
    if (st != SW_OK) { set_error("zero pivot in ILU(0)"); return st; }
    // In-column blocks: rows of one column are consecutive ranks, so the
    // column's part of L (unit lower) and U (upper) are P x P blocks; their
    // inverses turn the in-column recurrences into small dense products.
    std::vector<double> linv((size_t)H.ncol * H.P * H.P, 0.0), uinv((size_t)H.ncol * H.P * H.P, 0.0);
    {
        const int Pl = H.P, ns = H.nslot;
        std::vector<double> Lb(Pl * Pl), Ub(Pl * Pl), X(Pl * Pl);
        for (long long cr = 0; cr < H.ncol; ++cr) {
            std::fill(Lb.begin(), Lb.end(), 0.0);
            std::fill(Ub.begin(), Ub.end(), 0.0);
            const int col = H.gcol[cr];
            const int cix = col % H.nx, o = H.three_d ? HALF : H.own_pos(cix);
            for (int a = 0; a < Pl; ++a) {
                int j = a - 1;
                long long r = cr * Pl + a;
                int w0 = H.win[j + 1];
                Lb[a * Pl + a] = 1.0;
                for (int kk = 0; kk < W; ++kk) {
                    int lev = w0 + kk, b = lev + 1;
                    const int so = own_slot(H.layout, kk, o);
                    double v = lu_rows[(size_t)r * ns + so];
                    if (!H.in_pattern(so, cix, j)) continue;
                    if (b < a) Lb[a * Pl + b] = v;
                    else Ub[a * Pl + b] = v;
                }
            }
            // L^-1 by forward substitution, column by column
            std::fill(X.begin(), X.end(), 0.0);
            for (int c = 0; c < Pl; ++c) {
                for (int a = 0; a < Pl; ++a) {
                    double sum = a == c ? 1.0 : 0.0;
                    for (int b = 0; b < a; ++b) sum -= Lb[a * Pl + b] * X[b * Pl + c];
                    X[a * Pl + c] = sum;
                }
            }
            for (int a = 0; a < Pl; ++a)
                for (int c = 0; c < Pl; ++c) linv[((size_t)cr * Pl + c) * Pl + a] = X[a * Pl + c];
            // U^-1 by backward substitution
            std::fill(X.begin(), X.end(), 0.0);
            for (int c = 0; c < Pl; ++c) {
                for (int a = Pl - 1; a >= 0; --a) {
                    double sum = a == c ? 1.0 : 0.0;
                    for (int b = a + 1; b < Pl; ++b) sum -= Ub[a * Pl + b] * X[b * Pl + c];
                    X[a * Pl + c] = sum / Ub[a * Pl + a];
                }
            }
            for (int a = 0; a < Pl; ++a)
                for (int c = 0; c < Pl; ++c) uinv[((size_t)cr * Pl + c) * Pl + a] = X[a * Pl + c];
        }
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    Problem *P = new (std::nothrow) Problem();
    if (!P) { set_error("out of host memory"); return SW_ERR_BAD_ARG; }
    P->grid = g; P->params = p; P->device = dev;
    P->phys.g = 9.81; P->phys.rho = 1000.0; P->phys.dt = 0.0;
    P->m = H.m; P->ncol = H.ncol; P->P = H.P;
    const long long m = H.m;
    const int ns = H.nslot;
    int rc = SW_OK;
#define ALLOC(ptr, bytes) do { if ((rc = dalloc(P, (void **)&(ptr), (bytes))) != SW_OK) { sw_destroy_problem((sw_problem *)P); return rc; } } while (0)
    // weights: wx1, wx2, wy1, wy2, ws1 (P*7), ws2 (P*7), wxo1 (7*7), wxo2 (7*7)
    const size_t wxo_at = 4 * W + 2 * (size_t)H.P * W;
    std::vector<double> wts(wxo_at + 2 * W * W);
    for (int o = 0; o < W; ++o)
        for (int t = 0; t < W; ++t) {
            wts[wxo_at + o * W + t] = H.wxo1[o][t];
            wts[wxo_at + W * W + o * W + t] = H.wxo2[o][t];
        }
    std::copy(H.wx1, H.wx1 + W, wts.begin());
    std::copy(H.wx2, H.wx2 + W, wts.begin() + W);
    std::copy(H.wy1, H.wy1 + W, wts.begin() + 2 * W);
    std::copy(H.wy2, H.wy2 + W, wts.begin() + 3 * W);
    std::copy(H.ws1.begin(), H.ws1.end(), wts.begin() + 4 * W);
    std::copy(H.ws2.begin(), H.ws2.end(), wts.begin() + 4 * W + H.P * W);
    ALLOC(P->d_weights, wts.size() * sizeof(double));
    ALLOC(P->d_win, H.P * sizeof(int));
    ALLOC(P->d_hcols, 5 * (size_t)H.ncol * sizeof(double));
    ALLOC(P->d_geom, 20 * (size_t)H.ncol * sizeof(double));
    ALLOC(P->d_geom32, 20 * (size_t)H.ncol * sizeof(float));
    ALLOC(P->d_weights32, wts.size() * sizeof(float));
    ALLOC(P->d_lu64, (size_t)m * ns * sizeof(double));
    ALLOC(P->d_udinv64, (size_t)m * sizeof(double));
    ALLOC(P->d_lu32, (size_t)m * ns * sizeof(float));
    ALLOC(P->d_udinv32, (size_t)m * sizeof(float));
    ALLOC(P->d_linv64, linv.size() * sizeof(double));
    ALLOC(P->d_uinv64, uinv.size() * sizeof(double));
    ALLOC(P->d_linv32, linv.size() * sizeof(float));
    ALLOC(P->d_uinv32, uinv.size() * sizeof(float));
    ALLOC(P->d_V, (size_t)(p.restart + 1) * m * sizeof(double));
    if (p.precision == SW_PRECISION_MIXED) ALLOC(P->d_V32, (size_t)(p.restart + 1) * m * sizeof(float));
    ALLOC(P->d_work, 6 * (size_t)m * sizeof(double));
    ALLOC(P->d_Y[0], (size_t)p.k * m * sizeof(double));
    ALLOC(P->d_Y[1], (size_t)p.k * m * sizeof(double));
    ALLOC(P->d_W, (size_t)p.k * m * sizeof(double));
    ALLOC(P->d_xprev, (size_t)m * sizeof(double));
    if (p.guess == SW_GUESS_RRF) ALLOC(P->d_X, (size_t)p.history * m * sizeof(double));
    if (p.orthonormalize) ALLOC(P->d_Q, (size_t)p.k * m * sizeof(double));
    ALLOC(P->d_omega, MAX_K * sizeof(double));
    ALLOC(P->d_stats, sizeof(DevStats));
    ALLOC(P->d_host_io, (3 * (size_t)m + 2 * (size_t)H.ncol) * sizeof(double));
    ALLOC(P->d_gcol, (size_t)H.ncol * sizeof(int));
    ALLOC(P->d_grp, (size_t)H.ncol);
    ALLOC(P->d_goff, (MAX_GROUPS + 1) * sizeof(int));
    e = cudaMemcpy(P->d_weights, wts.data(), wts.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->d_gcol, H.gcol.data(), H.ncol * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->d_grp, H.grp.data(), H.ncol, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->d_goff, H.goff.data(), H.goff.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->d_win, H.win.data(), H.P * sizeof(int), cudaMemcpyHostToDevice);
    {
        std::vector<float> w32(wts.begin(), wts.end());
        if (e == cudaSuccess)
            e = cudaMemcpy(P->d_weights32, w32.data(), w32.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    std::vector<double> hc(5 * (size_t)H.ncol);
    std::copy(H.h.begin(), H.h.end(), hc.begin());
    std::copy(H.hx.begin(), H.hx.end(), hc.begin() + H.ncol);
    std::copy(H.hy.begin(), H.hy.end(), hc.begin() + 2 * H.ncol);
    std::copy(H.hxx.begin(), H.hxx.end(), hc.begin() + 3 * H.ncol);
    std::copy(H.hyy.begin(), H.hyy.end(), hc.begin() + 4 * H.ncol);
    if (e == cudaSuccess) e = cudaMemcpy(P->d_hcols, hc.data(), hc.size() * sizeof(double), cudaMemcpyHostToDevice);
    // factors slot-major on the device, rows ordered group, level, column:
    // lu[s * m + goff[c] * P + (j + 1) * size(c) + q] for rank (goff[c] + q) * P + j + 1
    {
        std::vector<double> t((size_t)m * ns);
        std::vector<float> t32((size_t)m * ns);
        for (long long i = 0; i < m; ++i) {
            const long long cr = i / H.P, a = i % H.P;
            const int c = H.grp[H.gcol[cr]];
            const long long per = H.goff[c + 1] - H.goff[c], q = cr - H.goff[c];
            const long long i2 = (long long)H.goff[c] * H.P + a * per + q;
            for (int s = 0; s < ns; ++s) {
                double v = lu_rows[(size_t)i * ns + s];
                t[(size_t)s * m + i2] = v;
                t32[(size_t)s * m + i2] = (float)v;
            }
        }
        if (e == cudaSuccess) e = cudaMemcpy(P->d_lu64, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(P->d_lu32, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice);
        std::vector<float> u32(udinv.size());
        for (size_t i = 0; i < udinv.size(); ++i) u32[i] = (float)udinv[i];
        if (e == cudaSuccess) e = cudaMemcpy(P->d_udinv64, udinv.data(), m * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(P->d_udinv32, u32.data(), m * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(P->d_linv64, linv.data(), linv.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(P->d_uinv64, uinv.data(), uinv.size() * sizeof(double), cudaMemcpyHostToDevice);
        std::vector<float> f32(linv.size());
        for (size_t i = 0; i < linv.size(); ++i) f32[i] = (float)linv[i];
        if (e == cudaSuccess) e = cudaMemcpy(P->d_linv32, f32.data(), f32.size() * sizeof(float), cudaMemcpyHostToDevice);
        for (size_t i = 0; i < uinv.size(); ++i) f32[i] = (float)uinv[i];
        if (e == cudaSuccess) e = cudaMemcpy(P->d_uinv32, f32.data(), f32.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) { sw_destroy_problem((sw_problem *)P); return cuda_fail(e, "upload"); }
    Dev &D = P->dev;
    D.nx = g.nx; D.ny = g.ny; D.nz = g.nz; D.P = H.P; D.ncol = H.ncol; D.three_d = three_d;
    D.layout = H.layout; D.nslot = ns; D.m = m; D.dx = H.dx; D.dy = H.dy;
    D.walls = H.walls;
    D.ngroups = H.ngroups;
    for (int c = 0; c <= H.ngroups; ++c) P->goff_h[c] = H.goff[c];
    D.goff = P->d_goff;
    D.gcol = P->d_gcol;
    D.grp = P->d_grp;
    D.wxo1 = P->d_weights + wxo_at;
    D.wxo2 = P->d_weights + wxo_at + W * W;
    D.wx1 = P->d_weights; D.wx2 = P->d_weights + W; D.wy1 = P->d_weights + 2 * W; D.wy2 = P->d_weights + 3 * W;
    D.ws1 = P->d_weights + 4 * W; D.ws2 = P->d_weights + 4 * W + H.P * W;
    D.win = P->d_win;
    D.h = P->d_hcols; D.hx = P->d_hcols + H.ncol; D.hy = P->d_hcols + 2 * H.ncol;
    D.hxx = P->d_hcols + 3 * H.ncol; D.hyy = P->d_hcols + 4 * H.ncol;
    D.gp = P->d_geom;
    D.gp32 = P->d_geom32;
    D.w32 = P->d_weights32;
    D.lu64 = P->d_lu64; D.lu32 = P->d_lu32; D.udinv64 = P->d_udinv64; D.udinv32 = P->d_udinv32;
    D.linv64 = P->d_linv64; D.uinv64 = P->d_uinv64; D.linv32 = P->d_linv32; D.uinv32 = P->d_uinv32;
    // algorithmic cost per point: 7-point sums counted as 7 fused multiply-adds (14 flops)
    {
        double fA = three_d ? 123.0 : 76.0;
        double bA = 16.0 + 8.0 * (three_d ? 18.0 : 12.0) / H.P;
        P->cost.fA = fA;
        P->cost.bA = bA;
        P->cost.fM = 2.0 * ns - 1.0;
        P->cost.bM = (ns + 1.0) * 8.0 + 32.0;
    }
    rc = setup_solver_launch(P);
    if (rc != SW_OK) { sw_destroy_problem((sw_problem *)P); return rc; }
    ALLOC(P->d_part, (size_t)P->nblocks * 2 * 160 * sizeof(double) + 8192);
    ALLOC(P->d_sync, 256);
#undef ALLOC
    *out = (sw_problem *)P;
    return SW_OK;
}

namespace sw {
void destroy_streamed(Problem *P);   // streamed.cu
void destroy_resident(Problem *P);   // resident.cu
}

extern "C" int sw_destroy_problem(sw_problem *pp) {
    Problem *P = (Problem *)pp;
    if (!P) return SW_OK;
    destroy_streamed(P);
    destroy_resident(P);
    for (auto ev : P->ev) cudaEventDestroy(ev);
    for (void *a : P->allocs) cudaFree(a);
    delete P;
    return SW_OK;
}

extern "C" int sw_problem_size(const sw_problem *pp, long long *m) {
    if (!pp || !m) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    *m = ((const Problem *)pp)->m;
    return SW_OK;
}

// Gaussian sketch vectors: SplitMix64 (Steele, Lea & Flood 2014) as a
// counter-based generator, two outputs per value through Box-Muller.
static uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + i * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

extern "C" int sw_draw_omega(uint64_t seed, long long solve_index, int k, double *h_omega) {
    if (!h_omega || k < 1 || solve_index < 0) { set_error("bad argument"); return SW_ERR_BAD_ARG; }
    const double inv53 = 1.0 / 9007199254740992.0;
    const double two_pi = 6.283185307179586476925286766559;
    for (int c = 0; c < k; ++c) {
        uint64_t base = 2 * ((uint64_t)solve_index * (uint64_t)k + (uint64_t)c) + 1;
        double u1 = ((double)(splitmix64_at(seed, base) >> 11) + 1.0) * inv53;
        double u2 = (double)(splitmix64_at(seed, base + 1) >> 11) * inv53;
        double r = std::sqrt(-2.0 * std::log(u1));
        double th = two_pi * u2;
        h_omega[c] = r * std::cos(th);
    }
    return SW_OK;
}
