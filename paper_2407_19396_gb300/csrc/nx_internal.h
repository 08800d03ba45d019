// nx_internal.h -- data layout shared by the host runtime and the kernels of
// libnavixgb (never exposed through the C ABI).
//
// HBM layout of one context (all 256-byte aligned, one allocation each):
//   agents   nx_agent[n_envs]        32 B per env, the documented snapshot block
//   grids    uint8[pool]             per env three planes (entity, colour,
//                                    state) of size*size bytes, row-major
//   items    nx_item[n_items]        work list: runs of <= envs_per_cta
//                                    consecutive envs sharing a descriptor
//   reqs     nx_req[n_reqs]          per request: key, step counters, outputs
//   ctl      nx_ctl                  sticky flags
//   atlas    uint8[397 * 3072]       sprite atlas (RGB only)
#pragma once
#include <stdint.h>

#define NX_ALIGN16 __attribute__((aligned(16)))

// One env's persistent state (exactly the 32-byte agent block of the
// snapshot format in navixgb.h).
struct NX_ALIGN16 nx_agent {
    uint8_t x, y, dir, carry_ent;
    uint8_t carry_col, done, invalid, n_balls;
    uint16_t t, max_steps;
    uint32_t episode;
    uint8_t ball_x[4];
    uint8_t ball_y[4];
    uint8_t family, size;
    uint8_t mission;       // GoToDoor: colour of the target door; 255 otherwise
    uint8_t reserved;
    uint32_t grid_offset;  // the low 32 bits of the env's byte offset in the grid pool
};
static_assert(sizeof(nx_agent) == 32, "agent block is 32 bytes");

// A run of consecutive envs with one descriptor, processed by one CTA.
struct NX_ALIGN16 nx_item {
    uint32_t env_begin;    // first env (index into agents)
    uint32_t n_envs;       // number of envs (<= envs_per_cta)
    uint64_t grid_offset;  // byte offset of env_begin's planes in the grid pool (pools may exceed 4 GiB)
    uint32_t req;          // request record index
    uint32_t local_begin;  // index of env_begin within its request (keys, output rows)
    uint16_t max_steps;
    uint8_t family, size;
    uint32_t variant;      // rivers of a crossing family, 0 otherwise
};
static_assert(sizeof(nx_item) == 32, "item is 32 bytes");

// Per request (a context is one request; the server has one per admitted
// request).  The kernels read it at item start; the advance kernel moves the
// counters after each launch.
struct NX_ALIGN16 nx_req {
    uint64_t seed;
    uint32_t gstep;       // step word of random-action draws at the next step
    uint32_t call_step;   // steps already done in the current call (output slot, action row)
    int32_t steps;        // steps each launch runs for this request (<= launch steps)
    int32_t depth;        // output time slots
    uint32_t n_envs;      // envs of the request (output row stride)
    int32_t act_mode;     // NX_ACT_*
    const int8_t* actions;  // [*, n_envs]
    uint8_t* obs_sym;       // [depth, n_envs, 147]
    uint8_t* obs_rgb;       // [depth, n_envs, 150528]
    float* reward;          // [depth, n_envs]
    uint8_t* terminated;
    uint8_t* truncated;
    float* returns;         // [n_envs] running sum of rewards (may be NULL)
    uint64_t* digest;       // [n_envs] running output digest (may be NULL)
    uint32_t* episodes;     // [n_envs] finished-episode counter (may be NULL)
    uint32_t reward_mode;
    float lava_reward;
    int32_t n_balls;      // Dynamic-Obstacles balls placed at every reset
    uint32_t key_base;    // draw-counter env index of the request's env 0
    uint8_t* obs_full;    // [depth, n_envs, full_side, full_side, 3] (may be NULL)
    uint8_t* obs_cat;     // [depth, n_envs, full_side, full_side]
    uint8_t* obs_cat_fp;  // [depth, n_envs, 7, 7]
    uint8_t* obs_rgb_full;  // [depth, n_envs, 32 full_side, 32 full_side, 3]
    uint8_t* mission;     // [depth, n_envs] (may be NULL)
    int32_t full_side;
    float action_cost;    // Table 5 shaping terms
    float time_cost;
    int8_t* action_out;   // [depth, n_envs] the action of every step (may be NULL)
    const uint8_t* policy;  // NX_ACT_POLICY: per-agent weight images (nxp::kImageBytes each)
    uint32_t policy_epa;  // envs per agent
    int32_t shift1, shift2;
    uint32_t epsilon;     // exploration threshold on a 32-bit draw
};

struct NX_ALIGN16 nx_ctl {
    uint32_t flags;  // bit 0 invalid action seen, bit 1 bounds check
    uint32_t pad[3];
};

enum { NX_FLAG_INVALID_ACTION = 1u, NX_FLAG_BOUNDS = 2u, NX_FLAG_WAIT_TIMEOUT = 4u };

// Launch arguments of the step kernel.
struct nx_kparams {
    const nx_item* items;
    int32_t n_items;
    int32_t launch_steps;  // upper bound of steps per item in this launch
    nx_agent* agents;
    uint8_t* grids;
    nx_req* reqs;
    nx_ctl* ctl;
    const uint8_t* atlas;
    int32_t cell_stride;   // smem bytes per env slot (nx_slot_stride of the launch shape and its reference side)
    // nonzero: each work item's slots are sized for its own grid side (an
    // item of a grid larger than the reference side holds fewer envs, so
    // that its slots fit the block's region of envs_per_cta * cell_stride)
    int32_t envs_per_cta;
    int32_t reset_all;     // 1: start every env at episode 0 and emit its observation (no steps)
    int32_t phases;        // symbolic staging parts per step (1 or 2)
    int32_t rgb_full_side; // side of the smem full-view tile buffer (0: none)
    int32_t policy_agents; // fused policy: weight sets per 128-env block (1, 2, 4 or 8)
    int32_t item_strides;
};

// Host-side launch helpers implemented in nx_kernels.cu.
struct nx_launch_shape {
    int group_lanes;
    int envs_per_cta;
    int rgb;
    int phases = 1;  // the symbolic outputs of a CTA are staged and stored in this many parts (1 or 2)
    int rgb_full_side = 0;  // reserve smem for full-view RGB tile ids of this grid side
    bool full = false;      // the instantiation that writes the fully observable views
    bool policy = false;    // the fused-policy instantiation (1 lane, 128 envs per CTA)
    int lean_family = -1;   // >= 0: the lean instantiation for this family, NX_N_FAMILIES: any family
    int policy_agents = 1;  // the fused policy's weight sets per block (shared memory, tensor memory)
};
// Shared-memory bytes per env grid for grids of up to max_cells cells: a
// whole number of 4-byte words, and an odd one, so that the grids of the 32
// envs a warp steps one lane each start in 32 different banks.
#ifdef __CUDACC__
#define NX_HD __host__ __device__
#else
#define NX_HD
#endif
NX_HD inline int nx_cell_stride(int max_cells)
{
    const int s = (max_cells + 3) & ~3;
    return ((s >> 2) & 1) ? s : s + 4;
}
// Groups of 8 or more lanes keep NX_VIEW_PAD wall cells around each grid in
// shared memory (the view reaches six cells ahead), narrower ones pack it.
#define NX_VIEW_PAD 6
// Bytes per env slot of a launch shape for grids of side up to max_side
// (nx_kparams::cell_stride).
NX_HD inline int nx_side_stride(int group_lanes, int side)
{
    const int w = group_lanes >= 8 ? side + 2 * NX_VIEW_PAD : side;
    return nx_cell_stride(w * w);
}
inline int nx_slot_stride(const nx_launch_shape& s, int max_side) { return nx_side_stride(s.group_lanes, max_side); }
// Envs per work item for grids of side `side` in a launch whose blocks hold
// envs_per_cta slots sized for `ref_side`: all of them for grids up to the
// reference side, as many as fit the same region for larger ones.
inline int nx_item_envs(const nx_launch_shape& s, int ref_side, int side)
{
    if (side <= ref_side) return s.envs_per_cta;
    const int n = s.envs_per_cta * nx_slot_stride(s, ref_side) / nx_slot_stride(s, side);
    return n < 1 ? 1 : n;
}
int nx_kernel_smem_bytes(const nx_launch_shape& s, int max_side);
int nx_kernel_max_ctas(const nx_launch_shape& s, int max_side, int* err);  // resident CTAs on the device
int nx_launch_step_kernel(const nx_launch_shape& s, const nx_kparams& p, int grid, void* stream);
int nx_launch_advance(nx_req* reqs, int n_reqs, void* stream);
int nx_launch_configure(nx_req* r, const nx_req& v, int gstep_mode, void* stream);
int nx_launch_set_steps(nx_req* r, int steps, void* stream);
int nx_shape_supported(const nx_launch_shape& s);
// Whether a shape has lean instantiations (random actions, no action output
// or digest, Markov reward, symbolic outputs only; one per family and one for
// any family).
int nx_lean_supported(const nx_launch_shape& s);
#ifdef __CUDACC__
int nx_kernel_max_ctas_full(const nx_launch_shape& s, int threads, int smem, int* err);
int nx_launch_step_kernel_full(const nx_launch_shape& s, const nx_kparams& p, int grid, int smem, cudaStream_t st);
// the lean instantiations, one translation unit per lane count
#define NX_LEAN_DECL(G_)                                                                                   \
    int nx_lean_occupancy_g##G_(int family, int threads, int smem, int* err);                              \
    int nx_lean_launch_g##G_(int family, const nx_kparams& p, int grid, int smem, cudaStream_t st);
NX_LEAN_DECL(1)
NX_LEAN_DECL(4)
NX_LEAN_DECL(8)
NX_LEAN_DECL(16)
NX_LEAN_DECL(32)
#undef NX_LEAN_DECL
int nx_lean_pol_occupancy(int family, int threads, int smem, int agents, int* err);
int nx_lean_pol_launch(int family, const nx_kparams& p, int grid, int smem, cudaStream_t st);
#endif
