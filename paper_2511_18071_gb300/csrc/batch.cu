// Batches of independent problems (many wave simulations of uneven sizes):
// one launch per stage step for all of them.  The Poisson solves run one
// thread block per problem (block barriers instead of grid barriers), handed
// out largest first through an atomic counter; the stage-driver steps run as
// one 2-D grid over (problem, node).
#include <algorithm>
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

// Tiles for a block team: wide enough that one pass gives every thread a row.
static Tiling batch_tiling(const Dev &D) {
    Tiling t{};
    if (!D.three_d) {
        int TX = 16;
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
    int max_ncol = 0;
    long long max_m = 0;
};

static void free_batch(Batch *B) {
    if (!B) return;
    cudaFree(B->d_items);
    cudaFree(B->d_drv);
    cudaFree(B->d_counter);
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

static int launch_batch_solve(Batch *B, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(B->d_counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "batch counter");
    if (B->cluster > 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(B->cluster_grid, 1, 1);
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
        void *args[] = {&B->d_items, &B->n, &B->d_counter};
        e = cudaLaunchKernelExC(&cfg, cluster_kern(B->mixed), args);
        if (e != cudaSuccess) return cuda_fail(e, "batch cluster launch");
        return SW_OK;
    }
    void *args[] = {&B->d_items, &B->n, &B->d_counter};
    e = cudaLaunchKernel(block_kern(B->mixed), dim3(B->nblocks), dim3(NTHREADS), args, B->smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "batch solve launch");
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
        Tiling t = batch_tiling(P->dev);
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
    if (e == cudaSuccess) e = cudaMalloc(&B->d_items, n * sizeof(BatchItem));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_drv, n * sizeof(DrvItem));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_counter, sizeof(int));
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaMallocHost(&B->h_items[i], n * sizeof(BatchItem));
        if (e == cudaSuccess) e = cudaMallocHost(&B->h_drv[i], n * sizeof(DrvItem));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) { free_batch(B); return cuda_fail(e, "batch set-up"); }
    // default: members of a few thousand unknowns or more get a 16-block
    // cluster (one block per member was 7.7x slower on 128 uneven members of
    // 1,280-69,632 unknowns); the largest cluster the device can place
    long long total = 0;
    for (Problem *P : B->probs) total += P->m;
    if (total / n >= 4096) {
        for (int cs = MAX_CLUSTER; cs >= 4; cs >>= 1) {
            const int nc = cluster_capacity(B, cs);
            if (nc >= 1) {
                B->cluster = cs;
                B->cluster_grid = std::min(B->n, nc) * cs;
                break;
            }
        }
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
    if (blocks_per_member == 1) { B->cluster = 1; return SW_OK; }
    const int nc = cluster_capacity(B, blocks_per_member);
    if (nc < 1) { set_error("the device cannot place a cluster of that size for this batch"); return SW_ERR_BAD_ARG; }
    B->cluster = blocks_per_member;
    B->cluster_grid = std::min(B->n, nc) * blocks_per_member;
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
            args[i].tl = batch_tiling(P->dev);
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
            args[i].tl = batch_tiling(P->dev);
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
