// Batches of independent problems (many wave simulations of uneven sizes):
// one launch per stage step for all of them.  The Poisson solves run one
// thread block per problem (block barriers instead of grid barriers), handed
// out largest first through an atomic counter; the stage-driver steps run as
// one 2-D grid over (problem, node).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <utility>

#include "sw_batch.cuh"
#include "sw_driver.cuh"

namespace sw {

SolveArgs make_args(Problem *P, const double *ep, const double *ec, const double *b, double *x, int guess_only);
void after_solve(Problem *P, const SolveArgs &A, int guess_only);
DrvPtrs driver_ptrs(Problem *P);
int ensure_state(Problem *P);

struct DrvItem {
    Dev D;
    DrvPtrs q;
    const double *ep, *ec;
};

__global__ void feta_batch(const DrvItem *it) {
    const DrvItem &d = it[blockIdx.y];
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < d.D.ncol) feta_at(d.D, d.q, c);
}
__global__ void geometry_batch(const DrvItem *it) {
    const DrvItem &d = it[blockIdx.y];
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < d.D.ncol) geometry_columns(d.D, d.ep, d.ec, c, d.D.ncol);
}
__global__ void rhs_g_batch(const DrvItem *it) {
    const DrvItem &d = it[blockIdx.y];
    long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (node < d.D.m) rhs_g_at(d.D, d.q, node);
}
__global__ void rhs_div_batch(const DrvItem *it) {
    const DrvItem &d = it[blockIdx.y];
    long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (node < d.D.m) rhs_div_at(d.D, d.q, node);
}
__global__ void fu_batch(const DrvItem *it) {
    const DrvItem &d = it[blockIdx.y];
    long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (node < d.D.m) fu_at(d.D, d.q, node);
}
__global__ void update_batch(const DrvItem *it) {
    const DrvItem &d = it[blockIdx.y];
    long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (node < d.D.m) update_at(d.D, d.q, node);
}

// Tiles of a member's operator apply: TX columns (all levels) per tile in
// 2-D, the largest width up to TX that divides nx.
static Tiling batch_tiling(const Dev &D, int TXmax = 16) {
    Tiling t{};
    if (!D.three_d) {
        int TX = TXmax;
        while (D.nx % TX) TX >>= 1;
        t.TX = TX;
        t.TY = 1;
    } else {
        int TX = 8, TY = 4;
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

constexpr int TILE_CANDIDATES[4] = {8, 16, 32, 64};

// The operator apply of every member at once, one block per member: the
// measurement of the tile autotuner (the Arnoldi step's apply, in the inner
// precision, from the first Krylov vector into the scratch vector).
template <typename TC>
__global__ void __launch_bounds__(NTHREADS) batch_apply_kernel(const BatchItem *items, int n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int i = blockIdx.x;
    if (i >= n) return;
    const Dev D = items[i].D;
    const Tiling tl = items[i].A.tl;
    LdVec<TC, TC> ld{reinterpret_cast<const TC *>(items[i].A.V), TC(1)};
    StVec<TC, TC> st{reinterpret_cast<TC *>(items[i].A.t)};
    BlockTeam tm;
    team_apply<BlockTeam, TC, BATCH_WM>(tm, D, tl, smem_raw, ld, st);
}

struct Batch {
    std::vector<Problem *> probs;   // largest first
    std::vector<int> order;         // probs[i] is the caller's problem order[i]
    int n = 0;
    bool mixed = false;
    BatchItem *d_items = nullptr;
    DrvItem *d_drv = nullptr;
    int *d_counter = nullptr;
    BatchItem *h_items[2] = {nullptr, nullptr};
    DrvItem *h_drv[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int slot = 0;
    size_t smem = 0;
    int nblocks = 0;
    int cluster = 1;                // blocks per member (1: one block, no cluster)
    int cluster_grid = 0;           // blocks of the cluster launch
    int split = 0;                  // > 0: the split largest members on clusters, the rest on blocks
    int split_bgrid = 0;            // blocks of the single-block launch of a split
    cudaStream_t side = nullptr;    // stream of the single-block launch of a split
    cudaEvent_t fork = nullptr, join = nullptr;
    int nsm = 0;
    int tile_tx = 16;               // tile width of the members' operator applies (autotuned)
    float tile_us[4] = {0, 0, 0, 0};   // the autotuner's time per candidate (0: not admissible)
    int max_ncol = 0;
    long long max_m = 0;
};

static void free_batch(Batch *B) {
    if (!B) return;
    cudaFree(B->d_items);
    cudaFree(B->d_drv);
    cudaFree(B->d_counter);
    if (B->side) cudaStreamDestroy(B->side);
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->join) cudaEventDestroy(B->join);
    for (int i = 0; i < 2; ++i) {
        if (B->h_items[i]) cudaFreeHost(B->h_items[i]);
        if (B->h_drv[i]) cudaFreeHost(B->h_drv[i]);
        if (B->ev[i]) cudaEventDestroy(B->ev[i]);
    }
    delete B;
}

// Wait until the staging slot is free, fill it with fill(items, drv), copy it up.
template <class Fill>
static int upload(Batch *B, cudaStream_t s, bool with_drv, Fill fill) {
    const int sl = B->slot;
    cudaError_t e = cudaEventSynchronize(B->ev[sl]);
    if (e != cudaSuccess) return cuda_fail(e, "batch staging wait");
    fill(B->h_items[sl], B->h_drv[sl]);
    e = cudaMemcpyAsync(B->d_items, B->h_items[sl], B->n * sizeof(BatchItem), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && with_drv)
        e = cudaMemcpyAsync(B->d_drv, B->h_drv[sl], B->n * sizeof(DrvItem), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(B->ev[sl], s);
    if (e != cudaSuccess) return cuda_fail(e, "batch staging copy");
    B->slot ^= 1;
    return SW_OK;
}

static const void *cluster_kern(bool mixed) { return mixed ? batch_kernel_cluster_f32() : batch_kernel_cluster_f64(); }
static const void *block_kern(bool mixed) { return mixed ? batch_kernel_block_f32() : batch_kernel_block_f64(); }

// Cluster of cs blocks per member: the largest number of clusters the device
// can hold at once (0 when it cannot place one).
static int cluster_capacity(Batch *B, int cs) {
    const void *kern = cluster_kern(B->mixed);
    cudaError_t e = ensure_smem((const void *)kern, (size_t)(int)B->smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return 0; }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(NTHREADS, 1, 1);
    cfg.dynamicSmemBytes = B->smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    e = cudaOccupancyMaxActiveClusters(&nc, kern, &cfg);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return 0; }
    return nc;
}

static cudaError_t launch_clusters(Batch *B, BatchItem *items, int n, int *counter, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(NTHREADS, 1, 1);
    cfg.dynamicSmemBytes = B->smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = B->cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void *args[] = {&items, &n, &counter};
    return cudaLaunchKernelExC(&cfg, cluster_kern(B->mixed), args);
}

static cudaError_t launch_blocks(Batch *B, BatchItem *items, int n, int *counter, int grid, cudaStream_t s) {
    void *args[] = {&items, &n, &counter};
    return cudaLaunchKernel(block_kern(B->mixed), dim3(grid), dim3(NTHREADS), args, B->smem, s);
}

static int launch_batch_solve(Batch *B, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(B->d_counter, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "batch counter");
    if (B->split > 0) {
        // the cluster launch goes first, so that its clusters find whole
        // groups of free SMs; the single-block launch runs beside it on the
        // side stream and takes the remaining SMs
        e = cudaEventRecord(B->fork, s);
        if (e == cudaSuccess) e = launch_clusters(B, B->d_items, B->split, B->d_counter, B->cluster_grid, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(B->side, B->fork, 0);
        if (e == cudaSuccess)
            e = launch_blocks(B, B->d_items + B->split, B->n - B->split, B->d_counter + 1, B->split_bgrid, B->side);
        if (e == cudaSuccess) e = cudaEventRecord(B->join, B->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, B->join, 0);
        if (e != cudaSuccess) return cuda_fail(e, "batch split launch");
        return SW_OK;
    }
    if (B->cluster > 1) {
        e = launch_clusters(B, B->d_items, B->n, B->d_counter, B->cluster_grid, s);
        if (e != cudaSuccess) return cuda_fail(e, "batch cluster launch");
        return SW_OK;
    }
    e = launch_blocks(B, B->d_items, B->n, B->d_counter, B->nblocks, s);
    if (e != cudaSuccess) return cuda_fail(e, "batch solve launch");
    return SW_OK;
}

// Split: the n_big largest members on clusters of cs blocks, the others one
// block each, the two launches side by side.  Each big member gets a cluster
// of its own where the device can place that many next to at least one
// single block; the single blocks take the remaining SMs.
static int set_split(Batch *B, int n_big, int cs) {
    if (n_big < 1 || n_big >= B->n) { set_error("split: between 1 and n - 1 members on clusters"); return SW_ERR_BAD_ARG; }
    const int cap = cluster_capacity(B, cs);
    if (cap < 1) { set_error("the device cannot place a cluster of that size for this batch"); return SW_ERR_BAD_ARG; }
    int ncl = std::min(n_big, cap);
    if (ncl * cs >= B->nsm) ncl = std::max(1, (B->nsm - 1) / cs);
    B->cluster = cs;
    B->cluster_grid = ncl * cs;
    B->split = n_big;
    B->split_bgrid = std::max(1, std::min(B->n - n_big, B->nsm - ncl * cs));
    return SW_OK;
}

// Tile autotuner: time the batched operator apply (all members, one block
// each, the inner precision) for every candidate tile width and keep the
// fastest for the members' applies.  Set-up only (synchronous).
static int tune_batch_tiles(Batch *B) {
    const void *kern = B->mixed ? (const void *)batch_apply_kernel<float> : (const void *)batch_apply_kernel<double>;
    cudaError_t e = ensure_smem(kern, B->smem);
    if (e != cudaSuccess) return cuda_fail(e, "batch autotuner attribute");
    std::vector<BatchItem> items(B->n);
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best = 0.f;
    for (int ci = 0; ci < 4 && e == cudaSuccess; ++ci) {
        for (int i = 0; i < B->n; ++i) {
            Problem *P = B->probs[i];
            items[i].D = P->dev;
            items[i].A = make_args(P, nullptr, nullptr, nullptr, nullptr, 0);
            items[i].A.tl = batch_tiling(P->dev, TILE_CANDIDATES[ci]);
        }
        e = cudaMemcpy(B->d_items, items.data(), B->n * sizeof(BatchItem), cudaMemcpyHostToDevice);
        void *args[] = {&B->d_items, &B->n};
        for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
            if (r == 1) e = cudaEventRecord(a, 0);
            if (e == cudaSuccess) e = cudaLaunchKernel(kern, dim3(B->n), dim3(NTHREADS), args, B->smem, 0);
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess) break;
        B->tile_us[ci] = ms * 1e3f / 3.f;
        if (ci == 0 || B->tile_us[ci] < best) { best = B->tile_us[ci]; B->tile_tx = TILE_CANDIDATES[ci]; }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_fail(e, "batch tile autotuner");
    return SW_OK;
}

}  // namespace sw

using namespace sw;

extern "C" int sw_create_batch(sw_problem *const *problems, int n, sw_batch **out) {
    if (!problems || n < 1 || n > 65535 || !out) { set_error("bad argument"); return SW_ERR_BAD_ARG; }
    *out = nullptr;
    Batch *B = new Batch();
    B->n = n;
    B->order.resize(n);
    std::iota(B->order.begin(), B->order.end(), 0);
    for (int i = 0; i < n; ++i)
        if (!problems[i]) { delete B; set_error("null problem"); return SW_ERR_BAD_ARG; }
    std::stable_sort(B->order.begin(), B->order.end(), [&](int a, int b) {
        return ((Problem *)problems[a])->m > ((Problem *)problems[b])->m;
    });
    size_t tiles = 0;
    for (int i = 0; i < n; ++i) {
        Problem *P = (Problem *)problems[B->order[i]];
        if (P->dev.three_d) { delete B; set_error("a batch holds two-dimensional problems"); return SW_ERR_BAD_ARG; }
        B->probs.push_back(P);
        bool mx = P->params.precision == SW_PRECISION_MIXED;
        if (i == 0) B->mixed = mx;
        if (mx != B->mixed) { delete B; set_error("a batch needs one precision"); return SW_ERR_BAD_ARG; }
        Tiling t = batch_tiling(P->dev, TILE_CANDIDATES[3]);
        tiles = std::max(tiles, 2 * (size_t)P->dev.P * t.HW * sizeof(double));
        B->max_ncol = std::max(B->max_ncol, P->ncol);
        B->max_m = std::max(B->max_m, P->m);
    }
    B->smem = BSMEM_FIXED + tiles;
    const void *kern = block_kern(B->mixed);
    cudaError_t e = ensure_smem((const void *)kern, (size_t)(int)B->smem);
    int nsm = 0, per = 0, dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NTHREADS, B->smem);
    if (e == cudaSuccess && per < 1) { free_batch(B); set_error("batch kernel does not fit"); return SW_ERR_BAD_ARG; }
    B->nblocks = std::min(n, nsm * per);
    B->nsm = nsm;
    if (e == cudaSuccess) e = cudaMalloc(&B->d_items, n * sizeof(BatchItem));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_drv, n * sizeof(DrvItem));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_counter, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->join, cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaMallocHost(&B->h_items[i], n * sizeof(BatchItem));
        if (e == cudaSuccess) e = cudaMallocHost(&B->h_drv[i], n * sizeof(DrvItem));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) { free_batch(B); return cuda_fail(e, "batch set-up"); }
    {
        const int rc = tune_batch_tiles(B);
        if (rc != SW_OK) { free_batch(B); return rc; }
    }
    // default launch: the shape with the shortest modelled makespan, a
    // member's time taken as its unknowns over (SMs x efficiency) of its team.
    // Efficiencies of an SM in a cluster of cs blocks against one block alone,
    // measured on GB300 on the 2,048 x 33 members of the 512-member batch
    // (precision form): 0.88 (2), 0.85 (4), 0.7 (8), 0.48 (16).  Candidates:
    // one block for every member (makespan: the larger of the even share and
    // the largest member), clusters of cs for every member (the share over the
    // efficiency, or the largest member on its cluster), and splits with each
    // of the n_big largest members on a cluster of its own.  The largest
    // member's time counts twice: single members of a size class took up to
    // 2.5x their class's mean iterations per solve on that batch.
    {
        const double eff[5] = {1.0, 0.88, 0.85, 0.7, 0.48};
        std::vector<double> mm(n), tail(n + 1, 0.0);
        for (int i = 0; i < n; ++i) mm[i] = (double)B->probs[i]->m;
        for (int i = n - 1; i >= 0; --i) tail[i] = tail[i + 1] + mm[i];
        double best = std::max(tail[0] / nsm, 2.0 * mm[0]);
        int best_cs = 1, best_nb = 0;
        for (int lg = 1; lg <= 4; ++lg) {
            const int cs = 1 << lg;
            if (cluster_capacity(B, cs) < 1) continue;
            const double t_all = std::max(tail[0] / (nsm * eff[lg]), 2.0 * mm[0] / (cs * eff[lg]));
            if (t_all < best) { best = t_all; best_cs = cs; best_nb = n; }
            for (int nb = 1; nb < n && (nb + 1) * cs < nsm; ++nb) {
                const double t_big = 2.0 * mm[0] / (cs * eff[lg]);
                const double t_small = std::max(tail[nb] / (nsm - nb * cs), 2.0 * mm[nb]);
                const double t = std::max(t_big, t_small);
                if (t < best * 0.999) { best = t; best_cs = cs; best_nb = nb; }
            }
        }
        if (best_nb == n) {
            const int nc = cluster_capacity(B, best_cs);
            B->cluster = best_cs;
            B->cluster_grid = std::min(B->n, nc) * best_cs;
        } else if (best_nb > 0) {
            (void)set_split(B, best_nb, best_cs);
        }
        set_error("");
    }
    *out = (sw_batch *)B;
    return SW_OK;
}

extern "C" int sw_batch_set_cluster(sw_batch *bb, int blocks_per_member) {
    Batch *B = (Batch *)bb;
    if (!B || blocks_per_member < 1 || blocks_per_member > MAX_CLUSTER ||
        (blocks_per_member & (blocks_per_member - 1)) != 0) {
        set_error("blocks per member: 1, 2, 4, 8 or 16");
        return SW_ERR_BAD_ARG;
    }
    B->split = 0;
    if (blocks_per_member == 1) { B->cluster = 1; return SW_OK; }
    const int nc = cluster_capacity(B, blocks_per_member);
    if (nc < 1) { set_error("the device cannot place a cluster of that size for this batch"); return SW_ERR_BAD_ARG; }
    B->cluster = blocks_per_member;
    B->cluster_grid = std::min(B->n, nc) * blocks_per_member;
    return SW_OK;
}

extern "C" int sw_batch_set_split(sw_batch *bb, int n_big, int blocks_per_member) {
    Batch *B = (Batch *)bb;
    if (!B || blocks_per_member < 2 || blocks_per_member > MAX_CLUSTER ||
        (blocks_per_member & (blocks_per_member - 1)) != 0) {
        set_error("split: blocks per member 2, 4, 8 or 16");
        return SW_ERR_BAD_ARG;
    }
    return set_split(B, n_big, blocks_per_member);
}

extern "C" int sw_batch_get_launch(sw_batch *bb, int *n_big, int *blocks_per_member, int *cluster_blocks,
                                   int *single_blocks) {
    Batch *B = (Batch *)bb;
    if (!B || !n_big || !blocks_per_member || !cluster_blocks || !single_blocks) {
        set_error("null argument");
        return SW_ERR_BAD_ARG;
    }
    if (B->split > 0) {
        *n_big = B->split; *blocks_per_member = B->cluster;
        *cluster_blocks = B->cluster_grid; *single_blocks = B->split_bgrid;
    } else if (B->cluster > 1) {
        *n_big = B->n; *blocks_per_member = B->cluster; *cluster_blocks = B->cluster_grid; *single_blocks = 0;
    } else {
        *n_big = 0; *blocks_per_member = 1; *cluster_blocks = 0; *single_blocks = B->nblocks;
    }
    return SW_OK;
}

extern "C" int sw_batch_autotuned_tile(sw_batch *bb, int *tile_x, double *us, int n) {
    Batch *B = (Batch *)bb;
    if (!B || !tile_x || (n > 0 && !us)) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    *tile_x = B->tile_tx;
    for (int i = 0; i < n; ++i) us[i] = i < 4 ? (double)B->tile_us[i] : 0.0;
    return SW_OK;
}

extern "C" int sw_destroy_batch(sw_batch *bb) {
    Batch *B = (Batch *)bb;
    if (B) cudaDeviceSynchronize();
    free_batch(B);
    return SW_OK;
}

extern "C" int sw_batch_solve(sw_batch *bb, const double *const *d_eta_prev, const double *const *d_eta_cur,
                              const double *const *d_b, double *const *d_x, void *stream) {
    Batch *B = (Batch *)bb;
    if (!B || !d_eta_prev || !d_eta_cur || !d_b || !d_x) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    for (int i = 0; i < B->n; ++i)
        if (!d_eta_prev[i] || !d_eta_cur[i] || !d_b[i] || !d_x[i]) { set_error("null pointer in batch"); return SW_ERR_BAD_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<SolveArgs> args(B->n);
    int rc = upload(B, s, false, [&](BatchItem *items, DrvItem *) {
        for (int i = 0; i < B->n; ++i) {
            Problem *P = B->probs[i];
            const int o = B->order[i];
            args[i] = make_args(P, d_eta_prev[o], d_eta_cur[o], d_b[o], d_x[o], 0);
            args[i].tl = batch_tiling(P->dev, B->tile_tx);
            items[i].D = P->dev;
            items[i].A = args[i];
        }
    });
    if (rc != SW_OK) return rc;
    rc = launch_batch_solve(B, s);
    if (rc != SW_OK) return rc;
    for (int i = 0; i < B->n; ++i) {
        after_solve(B->probs[i], args[i], 0);
        B->probs[i]->launches++;
        B->probs[i]->last_stream = s;
    }
    return SW_OK;
}

extern "C" int sw_batch_advance_stage(sw_batch *bb, void *stream) {
    Batch *B = (Batch *)bb;
    if (!B) { set_error("null argument"); return SW_ERR_BAD_ARG; }
    for (Problem *P : B->probs)
        if (!P->has_state || !(P->phys.dt > 0)) { set_error("state or physics not set in a batch member"); return SW_ERR_BAD_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<SolveArgs> args(B->n);
    int rc = upload(B, s, true, [&](BatchItem *items, DrvItem *drv) {
        for (int i = 0; i < B->n; ++i) {
            Problem *P = B->probs[i];
            drv[i].D = P->dev;
            drv[i].q = driver_ptrs(P);
            drv[i].ep = P->d_eta;
            drv[i].ec = P->d_eta_new;
            args[i] = make_args(P, P->d_eta, P->d_eta_new, P->d_rhs, P->d_p, 0);
            args[i].tl = batch_tiling(P->dev, B->tile_tx);
            items[i].D = P->dev;
            items[i].A = args[i];
        }
    });
    if (rc != SW_OK) return rc;
    const int T = 256;
    dim3 gc((B->max_ncol + T - 1) / T, B->n), gm((unsigned)((B->max_m + T - 1) / T), B->n);
    feta_batch<<<gc, T, 0, s>>>(B->d_drv);
    geometry_batch<<<gc, T, 0, s>>>(B->d_drv);
    rhs_g_batch<<<gm, T, 0, s>>>(B->d_drv);
    rhs_div_batch<<<gm, T, 0, s>>>(B->d_drv);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "batch stage launch");
    rc = launch_batch_solve(B, s);
    if (rc != SW_OK) return rc;
    fu_batch<<<gm, T, 0, s>>>(B->d_drv);
    update_batch<<<gm, T, 0, s>>>(B->d_drv);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "batch stage launch");
    for (int i = 0; i < B->n; ++i) {
        Problem *P = B->probs[i];
        after_solve(P, args[i], 0);
        std::swap(P->d_eta, P->d_eta_new);
        P->stage = (P->stage + 1) % 5;
        P->launches++;
        P->last_stream = s;
    }
    // the six driver launches and the solve launch serve the whole batch; they
    // are counted once, on the first member
    B->probs[0]->launches += 6;
    return SW_OK;
}
