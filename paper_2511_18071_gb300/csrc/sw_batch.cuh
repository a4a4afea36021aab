// Shared definitions of the batch form (batch.cu and the batch kernel variants).
#pragma once
#include "sw_solve.cuh"

namespace sw {

// batch members: any mix of periodic and walled two-dimensional grids
constexpr int BATCH_WM = WM_ANYWALL | WM_2D;

constexpr size_t BSMEM_FIXED = (sizeof(SmemFixed) + 255) & ~size_t(255);

struct BatchItem {
    Dev D;
    SolveArgs A;
};

const void *batch_kernel_block_f64();
const void *batch_kernel_block_f32();
const void *batch_kernel_cluster_f64();
const void *batch_kernel_cluster_f32();

}  // namespace sw
