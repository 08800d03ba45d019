// nx_kernels_full.cu -- instantiates the step kernel with the fully observable
// views (symbolic, categorical and RGB of the whole grid, Table 4), used only
// by calls that request them.
#include <cuda_runtime.h>
#include <stdint.h>

#include "navixgb.h"
#include "nx_internal.h"
#include "nx_step.cuh"

using namespace nxk;

int nx_kernel_max_ctas_full(const nx_launch_shape& s, int threads, int smem, int* err)
{
    NX_DISPATCH_G(s.group_lanes, s.rgb, true, occupancy_t, threads, smem, err)
}

int nx_launch_step_kernel_full(const nx_launch_shape& s, const nx_kparams& p, int grid, int smem, cudaStream_t st)
{
    NX_DISPATCH_G(s.group_lanes, s.rgb, true, launch_t, p, grid, smem, st)
}
