// nx_static.cu -- nx_rollout_noalloc: a rollout entry point that allocates no
// memory at all.
//
// Some callers cannot call cudaMalloc: a process where another runtime has
// already reserved nearly all device memory up front (a framework that
// preallocates its pool, a serving engine holding a fixed cache), or a
// latency-sensitive loop that must not hit cudaMalloc's implicit device
// synchronisation.  For them this entry point keeps every byte of scratch the
// step kernel needs (the env state, the work list, the request record and the
// flags) in one file-scope device array of fixed size, which every GPU that
// loads the library holds until the process exits.  The caller still passes
// the action input and the output buffers.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <string>

#include "navixgb.h"
#include "nx_internal.h"
#include "nx_runtime.h"
#include "nx_trace.h"

namespace {

// The whole scratch: [request record][flags][work list][agent blocks][grids].
__device__ __align__(256) static uint8_t g_noalloc_scratch[NX_NOALLOC_SCRATCH_BYTES];

constexpr size_t kReqOff = 0;
constexpr size_t kCtlOff = 256;
constexpr size_t kItemsOff = 512;
constexpr int kLanes = 8;
constexpr int kEnvsPerCta = 32;
constexpr int kStepsPerLaunch = 128;

// Fills the work list (runs of kEnvsPerCta consecutive envs) and clears the
// flags, so nothing from an earlier call leaks into this one.
__global__ void nx_noalloc_setup_kernel(uint8_t* scratch, int n_envs, int family, int size, int max_steps)
{
    nx_ctl* ctl = reinterpret_cast<nx_ctl*>(scratch + kCtlOff);
    nx_item* items = reinterpret_cast<nx_item*>(scratch + kItemsOff);
    const int n_items = (n_envs + kEnvsPerCta - 1) / kEnvsPerCta;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) ctl->flags = 0u;
    if (i < n_items) {
        nx_item it;
        memset(&it, 0, sizeof it);
        it.env_begin = (uint32_t)(i * kEnvsPerCta);
        it.n_envs = (uint32_t)min(kEnvsPerCta, n_envs - i * kEnvsPerCta);
        it.grid_offset = (uint32_t)(i * kEnvsPerCta) * (uint32_t)(3 * size * size);
        it.req = 0;
        it.local_begin = it.env_begin;
        it.max_steps = (uint16_t)max_steps;
        it.family = (uint8_t)family;
        it.size = (uint8_t)size;
        items[i] = it;
    }
}

// Device address of the array in the current device's context.  In host
// code the array's name is only a host-side stand-in, so its device address
// is looked up, with the device current, on every call: a host-side lookup,
// and never stale, also after cudaDeviceReset gave the device a new context
// (and the array possibly a new address).  The first lookup on a device may
// load the library's device code, which is why the first call on a device
// must come before any stream capture.
nx_status device_scratch(uint8_t** out)
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return nx_cuda_fail(nullptr, (int)e, "cudaGetSymbolAddress of the scratch array");
    }
    *out = (uint8_t*)p;
    return NX_OK;
}

// Bytes of the array one call uses.
size_t scratch_needed(int32_t size, int32_t n_envs)
{
    if (size < NX_MIN_SIZE || size > NX_MAX_SIZE || n_envs < 1) return 0;
    const size_t n_items = ((size_t)n_envs + kEnvsPerCta - 1) / kEnvsPerCta;
    const size_t agents_off = (kItemsOff + n_items * sizeof(nx_item) + 255) & ~(size_t)255;
    const size_t grids_off = (agents_off + (size_t)n_envs * sizeof(nx_agent) + 255) & ~(size_t)255;
    return grids_off + (size_t)n_envs * 3 * (size_t)size * (size_t)size;
}

}  // namespace

nx_status nx_rollout_noalloc(int32_t family, int32_t size, int32_t n_envs, uint64_t seed, int32_t n_steps,
                             int32_t act_mode, const int8_t* d_actions_TN, const nx_out* traj, void* cuda_stream)
{
    nx_range range("nx_rollout_noalloc");
    if (family < NX_EMPTY || family >= NX_N_FAMILIES) return nx_fail(nullptr, NX_E_INVAL, "unknown family");
    if (size < NX_MIN_SIZE || size > NX_MAX_SIZE) return nx_fail(nullptr, NX_E_INVAL, "grid size must be in 5..19");
    if (nx_max_variant(family, size) < 0) return nx_fail(nullptr, NX_E_INVAL, "the family has no grid of this size");
    if (n_envs < 1) return nx_fail(nullptr, NX_E_INVAL, "n_envs must be >= 1");
    if (n_steps < 0) return nx_fail(nullptr, NX_E_INVAL, "n_steps must be >= 0");
    if (act_mode != NX_ACT_RANDOM && act_mode != NX_ACT_BUFFER) return nx_fail(nullptr, NX_E_INVAL, "unknown act_mode");
    if (act_mode == NX_ACT_BUFFER && !d_actions_TN) return nx_fail(nullptr, NX_E_INVAL, "NX_ACT_BUFFER needs actions");
    if (traj && (traj->obs_rgb || traj->obs_full || traj->obs_cat || traj->obs_cat_fp || traj->obs_rgb_full ||
                 traj->mission || traj->action))
        return nx_fail(nullptr, NX_E_INVAL,
                       "nx_rollout_noalloc writes obs_sym, reward, terminated and truncated only (the other outputs must be NULL)");
    const size_t need = scratch_needed(size, n_envs);
    if (need > (size_t)NX_NOALLOC_SCRATCH_BYTES) {
        return nx_fail(nullptr, NX_E_INVAL,
                       "nx_rollout_noalloc: n_envs x (3 size^2 + 32) bytes of state exceed the fixed scratch of " +
                           std::to_string((size_t)NX_NOALLOC_SCRATCH_BYTES) + " bytes (this call needs " +
                           std::to_string(need) + ")");
    }
    uint8_t* scratch = nullptr;
    nx_status st = device_scratch(&scratch);
    if (st != NX_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    const int n_items = (n_envs + kEnvsPerCta - 1) / kEnvsPerCta;
    const size_t agents_off = (kItemsOff + (size_t)n_items * sizeof(nx_item) + 255) & ~(size_t)255;
    const size_t grids_off = (agents_off + (size_t)n_envs * sizeof(nx_agent) + 255) & ~(size_t)255;
    const int max_steps = nx_default_max_steps(family, size);
    const nx_launch_shape shape{kLanes, kEnvsPerCta, 0};
    const int cell_stride = nx_slot_stride(shape, size);
    int err = 0;
    const int per_sm = nx_kernel_max_ctas(shape, size, &err);
    if (err) return nx_cuda_fail(nullptr, err, "occupancy query");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return nx_fail(nullptr, NX_E_CUDA, "device query failed");
    const int grid = n_items < per_sm * sms ? n_items : per_sm * sms;

    nx_req* req = reinterpret_cast<nx_req*>(scratch + kReqOff);
    nx_kparams p;
    memset(&p, 0, sizeof p);
    p.items = reinterpret_cast<const nx_item*>(scratch + kItemsOff);
    p.n_items = n_items;
    p.agents = reinterpret_cast<nx_agent*>(scratch + agents_off);
    p.grids = scratch + grids_off;
    p.reqs = req;
    p.ctl = reinterpret_cast<nx_ctl*>(scratch + kCtlOff);
    p.atlas = nullptr;
    p.cell_stride = cell_stride;
    p.envs_per_cta = kEnvsPerCta;

    nx_noalloc_setup_kernel<<<(n_items + 127) / 128, 128, 0, s>>>(scratch, n_envs, family, size, max_steps);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return nx_cuda_fail(nullptr, (int)e, "noalloc setup launch");

    nx_options o;
    nx_options_default(&o);
    nx_req r;
    memset(&r, 0, sizeof r);
    r.seed = seed;
    r.n_envs = (uint32_t)n_envs;
    r.reward_mode = (uint32_t)o.reward_mode;
    r.lava_reward = o.lava_reward;
    r.n_balls = o.n_balls;
    r.key_base = 0;
    r.depth = 1;
    r.act_mode = NX_ACT_RANDOM;
    // reset every env to episode 0 without emitting the reset observation
    int rc = nx_launch_configure(req, r, 1, s);
    if (rc) return nx_cuda_fail(nullptr, rc, "noalloc configure");
    p.reset_all = 1;
    p.launch_steps = 0;
    rc = nx_launch_step_kernel(shape, p, grid, s);
    if (rc) return nx_cuda_fail(nullptr, rc, "noalloc reset launch");
    if (n_steps == 0) return NX_OK;

    // the steps, in chunks of kStepsPerLaunch
    r.act_mode = act_mode;
    r.actions = d_actions_TN;
    r.depth = (traj && traj->depth > 0) ? traj->depth : 1;
    r.obs_sym = traj ? traj->obs_sym : nullptr;
    r.reward = traj ? traj->reward : nullptr;
    r.terminated = traj ? traj->terminated : nullptr;
    r.truncated = traj ? traj->truncated : nullptr;
    r.steps = kStepsPerLaunch;
    rc = nx_launch_configure(req, r, 0, s);
    if (rc) return nx_cuda_fail(nullptr, rc, "noalloc configure");
    p.reset_all = 0;
    for (int t0 = 0; t0 < n_steps; t0 += kStepsPerLaunch) {
        const int c = n_steps - t0 < kStepsPerLaunch ? n_steps - t0 : kStepsPerLaunch;
        if (c != kStepsPerLaunch) {
            rc = nx_launch_set_steps(req, c, s);
            if (rc) return nx_cuda_fail(nullptr, rc, "noalloc set steps");
        }
        p.launch_steps = c;
        rc = nx_launch_step_kernel(shape, p, grid, s);
        if (rc) return nx_cuda_fail(nullptr, rc, "noalloc step launch");
        rc = nx_launch_advance(req, 1, s);
        if (rc) return nx_cuda_fail(nullptr, rc, "noalloc advance launch");
    }
    return NX_OK;
}
