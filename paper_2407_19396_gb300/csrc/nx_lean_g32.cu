// nx_lean_g32.cu -- the lean step kernels with 32 lanes per env, one per family
// (see nx_step_kernel: FAM >= 0).
#include <cuda_runtime.h>
#include <stdint.h>

#include "navixgb.h"
#include "nx_internal.h"
#include "nx_step.cuh"

using namespace nxk;

int nx_lean_occupancy_g32(int family, int threads, int smem, int* err)
{
    NX_DISPATCH_FAM(32, family, occupancy_t, threads, smem, err)
}

int nx_lean_launch_g32(int family, const nx_kparams& p, int grid, int smem, cudaStream_t st)
{
    NX_DISPATCH_FAM(32, family, launch_t, p, grid, smem, st)
}
