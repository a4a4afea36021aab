// One variant of the persistent solve kernel (the Poisson solve of one stage,
// Algorithm 2 with the subspace guess, then restarted GMRES left-preconditioned
// with the fixed ILU(0) factors, Sec. 3 and 4), compiled on its own so that
// the variants build in parallel.  The build compiles this file once per
// variant with
//   SW_TI   - inner precision of the GMRES cycles (double or float);
//   SW_WM   - problem class (walls and dimension, see sw_device.cuh);
//   SW_NAME - name of the function that returns the kernel's address.
#include "sw_solve.cuh"

#if !defined(SW_TI) || !defined(SW_WM) || !defined(SW_NAME)
#error "solve_kernel.cu is compiled once per variant with SW_TI, SW_WM and SW_NAME defined"
#endif

namespace sw {

constexpr size_t SMEM_FIXED_K = (sizeof(SmemFixed) + 255) & ~size_t(255);

template <typename TI, int WM>
__global__ void __launch_bounds__(NTHREADS, 1) solve_kernel(Dev D, SolveArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemFixed &S = *reinterpret_cast<SmemFixed *>(smem_raw);
    GridTeam tm(A.part, A.nb);
    double ph[PH_COUNT];
    for (int i = 0; i < PH_COUNT; ++i) ph[i] = 0.0;
    solve_body<GridTeam, TI, WM>(tm, D, A, S, smem_raw + SMEM_FIXED_K, ph);
}

const void *SW_NAME() { return (const void *)solve_kernel<SW_TI, SW_WM>; }

}  // namespace sw
