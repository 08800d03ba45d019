// nx_kernels.cu -- instantiates the step kernel without the fully observable
// views (the hot path), the small bookkeeping kernels and the host-side
// launch helpers.
#include <cuda_runtime.h>
#include <stdint.h>

#include "navixgb.h"
#include "nx_internal.h"
#include "nx_step.cuh"

using namespace nxk;

namespace {

// Sets the per-call fields of request 0 (arguments by value, so the update is
// stream-ordered and needs no host buffer).  gstep_mode: 0 keeps the
// random-action step counter, 1 restarts it at 0, 2 takes v.gstep.
__global__ void nx_configure_kernel(nx_req* r, nx_req v, int gstep_mode)
{
    if (gstep_mode == 0) v.gstep = r->gstep;
    if (gstep_mode == 1) v.gstep = 0u;
    *r = v;
}

__global__ void nx_set_steps_kernel(nx_req* r, int steps) { r->steps = steps; }

// Moves every request's counters past the launch that just ran.
__global__ void nx_advance_kernel(nx_req* reqs, int n_reqs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_reqs) {
        const int s = reqs[i].steps;
        reqs[i].gstep += (uint32_t)s;
        reqs[i].call_step += (uint32_t)s;
    }
}

}  // namespace


int nx_shape_supported(const nx_launch_shape& s)
{
    if (s.policy && (s.group_lanes != 1 || s.envs_per_cta != nxp::kRows || s.rgb || s.full)) return 0;
    const int G = s.group_lanes;
    if (G != 1 && G != 2 && G != 4 && G != 8 && G != 16 && G != 32) return 0;
    if (s.envs_per_cta < 1 || s.envs_per_cta * G > kMaxThreads) return 0;
    if ((s.envs_per_cta * G) % 32 != 0) return 0;
    return 1;
}

int nx_lean_supported(const nx_launch_shape& s)
{
    const int G = s.group_lanes;
    return (G == 1 || G == 4 || G == 8 || G == 16 || G == 32) && !s.rgb && !s.full && (!s.policy || G == 1);
}

// dynamic shared memory of a launch with env slots of cell_stride bytes
static int smem_for_stride(const nx_launch_shape& s, int cell_stride)
{
    const int E = s.envs_per_cta;
    const int epw = 32 / s.group_lanes, warps = E * s.group_lanes / 32;
    const int whalf = (s.phases > 1 && s.group_lanes < 16) ? (epw + 1) / 2 : epw;  // as nx_step_kernel
    // one lane per env pads its grid region with guard bytes (see nx_step_kernel)
    const int grid_bytes = align16(s.group_lanes == 1 ? E * cell_stride + 2 * kGridGuard : E * cell_stride);
    int b = grid_bytes + warps * align16(whalf * NX_OBS_SYM_BYTES + 16);
    if (s.policy) b = policy_smem_offset(grid_bytes, warps * align16(whalf * NX_OBS_SYM_BYTES + 16)) +
                      nxp::kATileBytes + s.policy_agents * nxp::kImageBytes;
    if (s.rgb) b += align16(E * 49 * 2) + align16(E * s.rgb_full_side * s.rgb_full_side * 2);
    return b;
}

int nx_kernel_smem_bytes(const nx_launch_shape& s, int max_side)
{
    return smem_for_stride(s, nx_slot_stride(s, max_side));
}

int nx_kernel_max_ctas(const nx_launch_shape& s, int max_side, int* err)
{
    const int smem = nx_kernel_smem_bytes(s, max_side);
    const int threads = s.envs_per_cta * s.group_lanes;
    if (s.full) return nx_kernel_max_ctas_full(s, threads, smem, err);
    if (s.policy)
        return s.lean_family >= 0 ? nx_lean_pol_occupancy(s.lean_family, threads, smem, s.policy_agents, err)
                                  : policy_occupancy(threads, smem, s.policy_agents, err);
    if (s.lean_family >= 0) {
        if (!nx_lean_supported(s)) return -1;
        switch (s.group_lanes) {
        case 1: return nx_lean_occupancy_g1(s.lean_family, threads, smem, err);
        case 4: return nx_lean_occupancy_g4(s.lean_family, threads, smem, err);
        case 8: return nx_lean_occupancy_g8(s.lean_family, threads, smem, err);
        case 16: return nx_lean_occupancy_g16(s.lean_family, threads, smem, err);
        default: return nx_lean_occupancy_g32(s.lean_family, threads, smem, err);
        }
    }
    NX_DISPATCH_G(s.group_lanes, s.rgb, false, occupancy_t, threads, smem, err)
}

int nx_launch_step_kernel(const nx_launch_shape& s, const nx_kparams& p, int grid, void* stream)
{
    const int smem = smem_for_stride(s, p.cell_stride);
    cudaStream_t st = (cudaStream_t)stream;
    if (s.full) return nx_launch_step_kernel_full(s, p, grid, smem, st);
    if (s.policy)
        return s.lean_family >= 0 ? nx_lean_pol_launch(s.lean_family, p, grid, smem, st)
                                  : launch_t<1, false, false, true>(p, grid, smem, st);
    if (s.lean_family >= 0) {
        if (!nx_lean_supported(s)) return -1;
        switch (s.group_lanes) {
        case 1: return nx_lean_launch_g1(s.lean_family, p, grid, smem, st);
        case 4: return nx_lean_launch_g4(s.lean_family, p, grid, smem, st);
        case 8: return nx_lean_launch_g8(s.lean_family, p, grid, smem, st);
        case 16: return nx_lean_launch_g16(s.lean_family, p, grid, smem, st);
        default: return nx_lean_launch_g32(s.lean_family, p, grid, smem, st);
        }
    }
    NX_DISPATCH_G(s.group_lanes, s.rgb, false, launch_t, p, grid, smem, st)
}

int nx_launch_configure(nx_req* r, const nx_req& v, int gstep_mode, void* stream)
{
    nx_configure_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(r, v, gstep_mode);
    return (int)cudaGetLastError();
}

int nx_launch_set_steps(nx_req* r, int steps, void* stream)
{
    nx_set_steps_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(r, steps);
    return (int)cudaGetLastError();
}

int nx_launch_advance(nx_req* reqs, int n_reqs, void* stream)
{
    if (n_reqs <= 0) return 0;
    nx_advance_kernel<<<(n_reqs + 127) / 128, 128, 0, (cudaStream_t)stream>>>(reqs, n_reqs);
    return (int)cudaGetLastError();
}
