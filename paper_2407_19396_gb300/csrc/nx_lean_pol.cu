// nx_lean_pol.cu -- the lean fused-policy step kernels (one lane per env,
// 128 envs per block), one per family and one for any family (see
// nx_step_kernel: FAM >= 0 with POL).
#include <cuda_runtime.h>
#include <stdint.h>

#include "navixgb.h"
#include "nx_internal.h"
#include "nx_step.cuh"

using namespace nxk;

int nx_lean_pol_occupancy(int family, int threads, int smem, int agents, int* err)
{
    NX_DISPATCH_POL_FAM(family, policy_occupancy, threads, smem, agents, err)
}

int nx_lean_pol_launch(int family, const nx_kparams& p, int grid, int smem, cudaStream_t st)
{
    NX_DISPATCH_POL_FAM(family, launch_policy_t, p, grid, smem, st)
}
