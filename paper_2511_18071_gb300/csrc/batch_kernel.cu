// One variant of the batch solve kernel: the Poisson solves of many
// independent two-dimensional problems in one launch, members handed out
// largest first through an atomic counter.  The build compiles this file once
// per variant with
//   SW_TI      - inner precision of the GMRES cycles (double or float);
//   SW_CLUSTER - 0: one thread block per member; 1: one thread-block cluster
//                per member (cluster barriers, partial sums through
//                distributed shared memory);
//   SW_NAME    - name of the function that returns the kernel's address.
// Members may mix periodic and walled grids (decided per member).
#include "sw_batch.cuh"

#if !defined(SW_TI) || !defined(SW_CLUSTER) || !defined(SW_NAME)
#error "batch_kernel.cu is compiled once per variant with SW_TI, SW_CLUSTER and SW_NAME defined"
#endif

namespace sw {

template <typename TI>
__global__ void __launch_bounds__(NTHREADS, 1) batch_solve_kernel(const BatchItem *items, int n, int *counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemFixed &S = *reinterpret_cast<SmemFixed *>(smem_raw);
    __shared__ int idx;
    for (;;) {
        if (threadIdx.x == 0) idx = atomicAdd(counter, 1);
        __syncthreads();
        const int i = idx;
        __syncthreads();
        if (i >= n) break;
        const Dev D = items[i].D;
        const SolveArgs A = items[i].A;
        BlockTeam tm;
        double ph[PH_COUNT];   // per-phase device time of this member's solve (thread 0)
        for (int q = 0; q < PH_COUNT; ++q) ph[q] = 0.0;
        solve_body<BlockTeam, TI, BATCH_WM>(tm, D, A, S, smem_raw + BSMEM_FIXED, ph);
        __syncthreads();
    }
}

// The cluster's first block takes the next member from the counter and the
// others read its index through distributed shared memory.  Large members get
// several SMs.
template <typename TI>
__global__ void __launch_bounds__(NTHREADS, 1) batch_solve_cluster_kernel(const BatchItem *items, int n, int *counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemFixed &S = *reinterpret_cast<SmemFixed *>(smem_raw);
    __shared__ int idx;
    cg::cluster_group cl = cg::this_cluster();
    for (;;) {
        if (cl.block_rank() == 0 && threadIdx.x == 0) idx = atomicAdd(counter, 1);
        cl.sync();
        const int i = *cl.map_shared_rank(&idx, 0);
        cl.sync();
        if (i >= n) break;
        const Dev D = items[i].D;
        const SolveArgs A = items[i].A;
        ClusterTeam tm(S.xchg);
        double ph[PH_COUNT];
        for (int q = 0; q < PH_COUNT; ++q) ph[q] = 0.0;
        solve_body<ClusterTeam, TI, BATCH_WM>(tm, D, A, S, smem_raw + BSMEM_FIXED, ph);
        cl.sync();
    }
}

#if SW_CLUSTER
const void *SW_NAME() { return (const void *)batch_solve_cluster_kernel<SW_TI>; }
#else
const void *SW_NAME() { return (const void *)batch_solve_kernel<SW_TI>; }
#endif

}  // namespace sw
