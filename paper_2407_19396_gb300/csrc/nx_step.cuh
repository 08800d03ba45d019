// nx_step.cuh -- the fused, persistent MiniGrid step kernel of libnavixgb
// (template; instantiated by nx_kernels.cu without and by nx_kernels_full.cu
// with the fully observable views, so the hot path carries none of their code).
//
// One CTA processes one work item at a time (a run of <= envs_per_cta
// consecutive envs that share a descriptor); a group of G lanes owns one env.
// Per item: the envs' three int8 planes are packed into one byte per cell in
// shared memory, then `steps` steps run back to back with the grid and the
// agent state on chip, and the state is written back at the end.  Per step:
//   draws (Philox, lanes in parallel) -> autoreset or transition + rules +
//   reward/termination/truncation -> egocentric view + occlusion (ballots
//   build the 49-bit transparency mask, a 32 KB table gives each row) ->
//   147 symbolic bytes staged per warp in smem (co-aligned with the
//   destination) and stored with 16-byte vectors -> with RGB, one CTA barrier
//   and 16-byte streaming stores of the atlas tiles (L2-resident atlas).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "navixgb.h"
#include "nx_device.cuh"
#include "nx_internal.h"
#include "nx_policy.cuh"

namespace nxk {

using namespace nxd;

// Guard bytes before and after the grid region of one-lane-per-env blocks:
// their view gather reads every view cell without a bounds test, up to six
// rows and six columns beyond a grid (at most 6 * 19 + 6 bytes before or
// after it); reads that land in a neighbour's grid or a guard are replaced by
// walls.
constexpr int kGridGuard = 128;
// Groups of 8 or more lanes keep this many wall cells around each grid in
// shared memory (row stride S + 2 kViewPad): the view reaches six cells
// ahead and three to the side, so every read of the view or of the forward
// cell lands in the env's slot, and beyond the grid it reads a wall.
constexpr int kViewPad = NX_VIEW_PAD;
constexpr int kMaxThreads = 256;

__host__ __device__ __forceinline__ int align16(int v) { return (v + 15) & ~15; }

// 64-bit FNV-style running digest over 32-bit words
__device__ __forceinline__ uint64_t digest_word(uint64_t h, uint32_t w) { return (h ^ (uint64_t)w) * 0x100000001B3ull; }

// One Dynamic-Obstacles ball's move (reading R12): to a uniformly drawn empty
// cell of its 8-neighbourhood that is not the agent's cell, with draw db.
// Balls lie in the grid's interior (placed there, they only ever move to
// empty cells, and the kernel checks every agent block it loads), so the
// eight neighbours are read without a bounds test and the candidate mask,
// the drawn candidate and the move are computed without a branch.
template <int G>
__device__ __forceinline__ void move_ball(const Grp<G>& grp, uint8_t* g, int S, int W, AgentReg& a, int b, uint32_t db,
                                          nx_ctl* ctl)
{
    const int bx = ball_x(a, b), by = ball_y(a, b);
    const uint8_t* c = g + by * W + bx;
    // bit j: neighbour j of the 3x3 block in row-major order without the centre
    uint32_t cand = (uint32_t)(c[-W - 1] == C_EMPTY) | ((uint32_t)(c[-W] == C_EMPTY) << 1) |
                    ((uint32_t)(c[-W + 1] == C_EMPTY) << 2) | ((uint32_t)(c[-1] == C_EMPTY) << 3) |
                    ((uint32_t)(c[1] == C_EMPTY) << 4) | ((uint32_t)(c[W - 1] == C_EMPTY) << 5) |
                    ((uint32_t)(c[W] == C_EMPTY) << 6) | ((uint32_t)(c[W + 1] == C_EMPTY) << 7);
    // the agent's cell, when it is a neighbour, is no candidate (it is never the ball's own cell)
    const int ox = a.x - bx + 1, oy = a.y - by + 1, ao = oy * 3 + ox;
    const bool adj = (unsigned)ox < 3u && (unsigned)oy < 3u;
    cand &= adj ? ~(1u << (ao - (ao > 4 ? 1 : 0))) : 0xFFFFFFFFu;
    const int cnt = __popc(cand);
    const bool moved = cnt > 0;
    const int jj = nth_set_bit(cand, bounded(db, (uint32_t)cnt)) & 7;  // 0..7 (any value when nothing is free)
    // neighbour jj's offsets plus one, two bits each: dx + 1 = 0,1,2,0,2,0,1,2 and dy + 1 = 0,0,0,1,1,2,2,2
    const int nx = bx + (int)((0x9224u >> (2 * jj)) & 3u) - 1, ny = by + (int)((0xA940u >> (2 * jj)) & 3u) - 1;
    if (G == 1) {
        if (moved && NX_DCHECK(ctl, (unsigned)nx < (unsigned)S && (unsigned)ny < (unsigned)S)) {
            g[by * W + bx] = (uint8_t)C_EMPTY;
            g[ny * W + nx] = (uint8_t)C_BALL_BLUE;
        }
    } else if (moved) {
        grp.sync();
        if (grp.lane == 0 && NX_DCHECK(ctl, (unsigned)nx < (unsigned)S && (unsigned)ny < (unsigned)S)) {
            g[by * W + bx] = (uint8_t)C_EMPTY;
            g[ny * W + nx] = (uint8_t)C_BALL_BLUE;
        }
        grp.sync();
    }
    set_ball(a, b, moved ? nx : bx, moved ? ny : by);
}

// Intervention (rotate / forward / pickup / drop / toggle / done), the
// Dynamic-Obstacles transition, then time, truncation, reward and termination.
// The balls' draws: d[b] for groups of several lanes (drawn in parallel by
// the caller); one lane per env draws each ball's inside the ball loop,
// which is not unrolled (a smaller loop body: the unrolled loop's code
// missed the instruction cache).
template <int G>
__device__ __forceinline__ void env_step(const Grp<G>& grp, uint8_t* g, int S, int W, int family, int max_steps, AgentReg& a,
                                         int action, const uint32_t (&d)[8], uint32_t reward_mode, float lava_reward,
                                         float action_cost, float time_cost, float& reward, int& term, int& trunc,
                                         nx_ctl* ctl, uint64_t seed, uint32_t key)
{
    // transition system: each ball, in index order, moves (move_ball)
    if (family == NX_DYNOBS) {
        if constexpr (G == 1) {
            const uint32_t episode = a.episode, t = (uint32_t)a.t;
#pragma unroll 1
            for (int b = 0; b < a.nb; ++b)
                move_ball(grp, g, S, W, a, b, draw(seed, key, episode, t, PURPOSE_BALL, (uint32_t)b), ctl);
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (b >= a.nb) break;
                move_ball(grp, g, S, W, a, b, d[b], ctl);
            }
        }
    }
    // intervention system, written as selects so that envs of one warp taking
    // different actions do not serialise on branches; the forward cell's kind
    // is tested as one bit against constant kind masks.  An out-of-range
    // action is a no-op that sets the sticky invalid flag (published to the
    // device flags when the work item ends).
    const int n_act = family == NX_DYNOBS ? 3 : 7;
    a.invalid |= (unsigned)action > 6u ? 1 : 0;
    const int act = (unsigned)action < (unsigned)n_act ? action : 7;  // 7: no-op
    const int fxd = (a.dir == 0) - (a.dir == 2), fyd = (a.dir == 1) - (a.dir == 3);
    const int fx = a.x + fxd, fy = a.y + fyd;
    // (with a wall margin, W > S, a cell beyond the grid reads as a wall)
    const bool in = W > S || ((unsigned)fx < (unsigned)S && (unsigned)fy < (unsigned)S);
    const int fi = fy * W + fx;
    const uint32_t fc = in ? (uint32_t)g[fi] : (uint32_t)C_WALL;
    const uint32_t fcol = cell_col(fc), kb = 1u << cell_kind(fc);
    constexpr uint32_t kDoors = (1u << K_DOOR_OPEN) | (1u << K_DOOR_CLOSED) | (1u << K_DOOR_LOCKED);
    // a ball is not walkable, so moving and being hit exclude each other
    const bool move = act == 2 && (kb & NX_WALKABLE_KINDS);
    const bool hit = act == 2 && family == NX_DYNOBS && (kb & (1u << K_BALL));
    const bool pick = act == 3 && a.carry == 0u && (kb & ((1u << K_KEY) | (1u << K_BALL)));
    const bool drop = act == 4 && a.carry != 0u && fc == C_EMPTY;  // a cell outside the grid reads as wall
    const bool unlock = act == 5 && (kb & (1u << K_DOOR_LOCKED)) && a.carry == make_code(K_KEY, fcol);
    const bool open_ = act == 5 && (kb & (1u << K_DOOR_CLOSED));
    const bool close_ = act == 5 && (kb & (1u << K_DOOR_OPEN));
    // on_door_done (Tables 5, 6): GoToDoor's done action facing a door of the
    // mission's colour completes the task; done does nothing elsewhere
    const bool door_done = act == 6 && family == NX_GOTODOOR && (kb & kDoors) && fcol == a.mission;
    const bool goal = (move && (kb & (1u << K_GOAL))) || door_done, lava = move && (kb & (1u << K_LAVA));
    a.dir = (a.dir + (act == 1 ? 1 : 0) + (act == 0 ? 3 : 0)) & 3;
    a.x = move ? fx : a.x;
    a.y = move ? fy : a.y;
    const bool write = pick || drop || unlock || open_ || close_;
    const uint32_t wcode = pick ? (uint32_t)C_EMPTY
                                : drop ? a.carry : (close_ ? make_code(K_DOOR_CLOSED, fcol) : make_code(K_DOOR_OPEN, fcol));
    a.carry = pick ? fc : (drop ? 0u : a.carry);
    if (write) {
        grp.sync();
        if (grp.lane == 0 && NX_DCHECK(ctl, (unsigned)fx < (unsigned)S && (unsigned)fy < (unsigned)S)) g[fi] = (uint8_t)wcode;
        grp.sync();
    }
    // time and truncation; reward and termination on the goal / lava / hit events
    a.t += 1;
    trunc = a.t >= max_steps;
    // (selects; only MiniGrid's success reward, a rare event, takes a branch)
    float rgoal = 1.0f;
    if (goal && reward_mode == NX_REWARD_MINIGRID)
        rgoal = __fsub_rn(1.0f, __fdiv_rn(__fmul_rn(0.9f, (float)a.t), (float)max_steps));
    reward = goal ? rgoal : (lava ? lava_reward : (hit ? -1.0f : 0.0f));
    term = (goal || lava || hit) ? 1 : 0;
    // the shaping terms of Table 5: action_cost for every action but done
    // (0..5), then time_cost (subtracting 0 leaves a reward unchanged)
    reward = __fsub_rn(reward, (unsigned)action < 6u ? action_cost : 0.0f);
    reward = __fsub_rn(reward, time_cost);
    a.done = term || trunc;
}

// CTA-wide copy from shared to global memory; src and dst are congruent
// modulo 16, the body moves in 16-byte vectors.
__device__ __forceinline__ void coop_copy(uint8_t* dst, const uint8_t* src, int nbytes, int tid, int nthreads)
{
    const int head = min(nbytes, (int)((16u - ((uint32_t)(uintptr_t)dst & 15u)) & 15u));
    const int body = (nbytes - head) & ~15;
    const int tail = nbytes - head - body;
    for (int i = tid; i < head; i += nthreads) dst[i] = src[i];
    const uint4* s4 = reinterpret_cast<const uint4*>(src + head);
    uint4* d4 = reinterpret_cast<uint4*>(dst + head);
    for (int i = tid; i < body / 16; i += nthreads) d4[i] = s4[i];
    for (int i = tid; i < tail; i += nthreads) dst[head + body + i] = src[head + body + i];
}

// Bulk (TMA) copy of a staged block from shared to global memory: the
// writing lanes fence their generic-proxy stores (bulk_fence_smem) and meet
// at a warp barrier, one lane issues the copy; before the buffer is written
// again that lane waits until the copy has read it, and before the block's
// work item ends until every copy has completed.
__device__ __forceinline__ void bulk_fence_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_copy_s2g(void* gdst, const void* ssrc, uint32_t bytes)
{
    const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(ssrc));
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(s), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Writes n envs' 224x224x3 images: 16-byte chunk r of an image is pixel row
// r / 42, bytes 16 (r % 42) .. of it, i.e. view column (r % 42) / 6, part
// (r % 42) % 6 of that tile's 96-byte row.
__device__ __forceinline__ void coop_rgb(uint8_t* dst, const uint16_t* tiles, const uint8_t* atlas, int n, int tid,
                                         int nthreads)
{
    constexpr int kChunks = NX_OBS_RGB_BYTES / 16;  // 9408
    for (int e = 0; e < n; ++e) {
        uint4* d4 = reinterpret_cast<uint4*>(dst + (size_t)e * NX_OBS_RGB_BYTES);
        const uint16_t* te = tiles + e * 49;
#pragma unroll 4
        for (int r = tid; r < kChunks; r += nthreads) {
            const int row = r / 42, c16 = r - row * 42;
            const int vx = c16 / 6, part = c16 - vx * 6;
            const int vy = row >> 5, ty = row & 31;
            const uint32_t tile = te[vy * 7 + vx];
            const uint4* src = reinterpret_cast<const uint4*>(atlas + (size_t)tile * 3072u + ty * 96 + part * 16);
            __stcs(d4 + r, __ldg(src));
        }
    }
}

// The same for the fully observable RGB view: F x F tiles per env.
__device__ __forceinline__ void coop_rgb_full(uint8_t* dst, const uint16_t* tiles, const uint8_t* atlas, int n, int F,
                                              int tid, int nthreads)
{
    const int per_row = 6 * F;  // 16-byte chunks per pixel row
    const int chunks = 32 * F * per_row;
    for (int e = 0; e < n; ++e) {
        uint4* d4 = reinterpret_cast<uint4*>(dst + (size_t)e * chunks * 16);
        const uint16_t* te = tiles + e * F * F;
#pragma unroll 4
        for (int r = tid; r < chunks; r += nthreads) {
            const int row = r / per_row, c16 = r - row * per_row;
            const int tx = c16 / 6, part = c16 - tx * 6;
            const int ty = row >> 5, py = row & 31;
            const uint32_t tile = te[ty * F + tx];
            const uint4* src = reinterpret_cast<const uint4*>(atlas + (size_t)tile * 3072u + py * 96 + part * 16);
            __stcs(d4 + r, __ldg(src));
        }
    }
}

// Byte offset of the fused policy's shared memory (the A tile, then the
// agent's weight image) after the grids and the staging.
__host__ __device__ __forceinline__ int policy_smem_offset(int grid_bytes, int staging_bytes)
{
    return (grid_bytes + staging_bytes + 127) & ~127;
}

// FAM >= 0 is a lean instantiation, for requests of the common kind: no
// digest, the Markov reward, symbolic outputs only, and (except the fused
// policy) random actions without an action output.  FAM < NX_N_FAMILIES:
// every work item of the launch has family FAM, so the compiler also drops
// the other families' generators and rules (the paper's implementation
// likewise compiles one program per environment); FAM = NX_N_FAMILIES: items
// of any family.  The host launches them only for such calls.
template <int G, bool RGB, bool FULL, bool POL = false, int FAM = -1>
__global__ void __launch_bounds__(kMaxThreads, 2) nx_step_kernel(const nx_kparams p)
{
    static_assert(!POL || (G == 1 && !RGB && !FULL), "the fused policy runs one lane per env");
    constexpr bool kLean = FAM >= 0, kLeanRandom = kLean && !POL;
    // The lean random-action kernels run only for calls that ask for the
    // symbolic view, the reward and both flags and for no mission (the host
    // checks it; the server gives each request a place for them), so their
    // stores need no test
    constexpr bool kOuts = kLeanRandom;
    // the fused policy with several weight sets per block (fewer than 128 envs
    // per set) runs in the general instantiation; the lean ones hold one set
    constexpr bool kMultiPol = POL && !kLean;
    static_assert(!kLean || (!RGB && !FULL && FAM <= NX_N_FAMILIES), "lean: symbolic outputs only");
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ __align__(8) uint64_t s_mbar;  // fused policy: MMA completion
    __shared__ uint32_t s_tmem;               // fused policy: tensor-memory base address
    __shared__ uint32_t s_dec[256];  // cell code -> observation triple
    // the occlusion table in shared memory for groups of 8 or more lanes (the
    // narrow groups run many more envs per block, whose grids need the space)
    constexpr bool kSmemOcc = G >= 8;
    // narrow groups (at least 8 envs per warp) store their staged symbolic
    // records with bulk copies; wider ones with the warp's vector copy
    constexpr bool kBulk = G <= 4;
    __shared__ __align__(16) uint16_t s_occ[kSmemOcc ? (1 << 14) : 8];
    // the lean kernels of groups of 8 or more lanes draw the random actions of
    // up to kActChunk steps ahead, one per lane and step, into shared memory
    // (a byte per env and step), so the step loop reads its action with one
    // load instead of a shuffle and a branch every G steps
    constexpr bool kPreAct = kLeanRandom && G >= 8;
    constexpr int kActChunk = kPreAct ? 128 : (1 << 30);
    __shared__ uint8_t s_act[kPreAct ? (kMaxThreads / G) * kActChunk : 1];
    const int E = p.envs_per_cta;
    // groups of 16 or more lanes stage at most two records per warp: always
    // in one part (the host sizes the staging the same way)
    const int phases = (G < 16 && p.phases > 1) ? 2 : 1;
    const int tid = threadIdx.x, nthreads = blockDim.x, lane32 = tid & 31, warp = tid >> 5;
    constexpr int epw = 32 / G;                         // envs per warp
    const int whalf = (epw + phases - 1) / phases;      // envs staged per part
    const int wbytes = align16(whalf * NX_OBS_SYM_BYTES + 16);
    const int wenv0 = warp * epw;                       // the warp's first env slot
    // One lane per env reads its view cells without bounds tests
    // (render_view), so guards pad its grid region on both sides.
    constexpr bool kGuard = G == 1;
    const int cs = p.cell_stride;  // bytes per env slot of the reference side (the block's grid region)
    const int grid_bytes = align16(kGuard ? E * cs + 2 * kGridGuard : E * cs);  // the staging after it is 16-aligned
    uint8_t* sgrid = smem + (kGuard ? kGridGuard : 0);
    uint8_t* wstage = smem + grid_bytes + warp * wbytes;
    uint16_t* stiles = reinterpret_cast<uint16_t*>(smem + grid_bytes + (nthreads >> 5) * wbytes);
    const int FR = p.rgb_full_side;  // full-view RGB tile buffer: E x FR x FR ids after the egocentric ones
    uint16_t* sfull = reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(stiles) + align16(E * 49 * 2));
    const int gi = tid / G;
    const Grp<G> grp(tid);
    constexpr int kPad = G >= 8 ? kViewPad : 0;
    // fused policy: the A tile of the 128 envs' rows, then the agent's weights
    uint8_t* sA = smem + policy_smem_offset(grid_bytes, (nthreads >> 5) * wbytes);
    uint8_t* sW = sA + nxp::kATileBytes;
    uint32_t tmem = 0, phase = 0;
    bool pol_ok = true;
    int pol_agents = 1;  // fused policy: weight sets of the current item
    nxp::PolRows pol_rows{1, 0, 0, 1};
    if constexpr (POL) {
        // 64 tensor-memory columns: the 128 x 64 f32 accumulator of a layer
        if (warp == 0) {
            // 64 columns per weight set of the block (a power of two, <= 512)
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(nxp::smem_u32(&s_tmem)),
                         "r"(64u * (uint32_t)p.policy_agents));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        }
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(nxp::smem_u32(&s_mbar)));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tmem = s_tmem;
    }
    for (int i = tid; i < 256; i += nthreads) s_dec[i] = cell_triple((uint32_t)i);
    if constexpr (kSmemOcc)
        for (int i = tid; i < (1 << 14) / 8; i += nthreads)
            reinterpret_cast<uint4*>(s_occ)[i] = __ldg(reinterpret_cast<const uint4*>(occ_table.v) + i);

    for (int it = blockIdx.x; it < p.n_items; it += gridDim.x) {
        const nx_item item = p.items[it];
        const nx_req* rq = p.reqs + item.req;
        const uint64_t seed = rq->seed;
        const uint32_t gstep0 = rq->gstep, call0 = rq->call_step;
        const int steps = p.reset_all ? 0 : min(rq->steps, p.launch_steps);
        const int depth = rq->depth > 0 ? rq->depth : 1;
        const uint32_t nreq = rq->n_envs;
        const int act_mode = rq->act_mode;
        const int8_t* actions = rq->actions;
        uint8_t* obs_sym = rq->obs_sym;
        uint8_t* obs_rgb = RGB ? rq->obs_rgb : nullptr;
        float* out_reward = rq->reward;
        uint8_t* out_term = rq->terminated;
        uint8_t* out_trunc = rq->truncated;
        uint8_t* out_mission = rq->mission;
        int8_t* out_action = kLeanRandom ? nullptr : rq->action_out;
        const uint32_t reward_mode = kLean ? (uint32_t)NX_REWARD_MARKOV : rq->reward_mode;
        const float lava_reward = rq->lava_reward;
        const float action_cost = rq->action_cost, time_cost = rq->time_cost;
        const int n_balls = rq->n_balls;
        float* returns = rq->returns;
        uint64_t* digest = kLean ? nullptr : rq->digest;
        uint32_t* episodes = rq->episodes;
        // the fully observable views exist only in the FULL instantiations
        uint8_t* obs_full = FULL ? rq->obs_full : nullptr;
        uint8_t* obs_cat = FULL ? rq->obs_cat : nullptr;
        uint8_t* obs_cat_fp = FULL ? rq->obs_cat_fp : nullptr;
        uint8_t* obs_rgb_full = (FULL && RGB && FR > 0) ? rq->obs_rgb_full : nullptr;
        const int F = FULL ? rq->full_side : 0;

        const int n = (int)item.n_envs, S = item.size, HW = S * S, variant = (int)item.variant;
        const int W = S + 2 * kPad;                                 // row stride of the env's grid in its slot
        const int ics = p.item_strides ? nx_side_stride(G, S) : cs;  // this item's bytes per env slot
        uint8_t* mygrid = sgrid + gi * ics + kPad * (W + 1);        // cell (0, 0)
        const int family = (kLean && FAM < NX_N_FAMILIES) ? FAM : (int)item.family;
        const int max_steps = item.max_steps;
        const bool active = gi < n;
        const uint32_t local = item.local_begin + (uint32_t)gi;
        const uint32_t key = rq->key_base + local;  // env index in the draw counters
        const uint32_t env = item.env_begin + (uint32_t)gi;
        AgentReg a;
        float ret = 0.0f;
        uint64_t dig = 0;
        uint32_t eps = 0;

        if constexpr (kPad > 0) {
            // every slot starts as walls (the margins stay so)
            constexpr uint32_t kWall4 = C_WALL * 0x01010101u;
            for (int i = tid; i < n * ics / 4; i += nthreads) reinterpret_cast<uint32_t*>(sgrid)[i] = kWall4;
            __syncthreads();
        }
        // i / HW and c / S by multiply-high with ceil(2^32 / d): exact for
        // i < 2^32 / d, far above the n * HW <= 256 * 361 cells of an item
        const uint32_t inv_hw = 0xFFFFFFFFu / (uint32_t)HW + 1u, inv_s = 0xFFFFFFFFu / (uint32_t)S + 1u;
        if (!p.reset_all) {
            const uint8_t* src = p.grids + item.grid_offset;
            // U cells per thread and round, their three global loads issued
            // before any is used (one dependent round trip per cell made the
            // loads of the larger grids latency-bound)
            const int nhw = n * HW;
            constexpr int U = 4;
            for (int i0 = tid; i0 < nhw; i0 += U * nthreads) {
                uint32_t pe[U], pc[U], ps[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = i0 + u * nthreads;
                    const int e = (int)__umulhi((uint32_t)i, inv_hw), c = i - e * HW;
                    const uint8_t* b = src + (size_t)e * 3 * HW + c;
                    const bool ok = i < nhw;
                    pe[u] = ok ? (uint32_t)b[0] : 0u;
                    pc[u] = ok ? (uint32_t)b[HW] : 0u;
                    ps[u] = ok ? (uint32_t)b[2 * HW] : 0u;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = i0 + u * nthreads;
                    if (i < nhw) {
                        const int e = (int)__umulhi((uint32_t)i, inv_hw), c = i - e * HW;
                        int si = e * ics + c;  // a packed grid: row stride S
                        if constexpr (kPad > 0) {
                            const int y = (int)__umulhi((uint32_t)c, inv_s), x = c - y * S;
                            si = e * ics + (y + kPad) * W + x + kPad;
                        }
                        sgrid[si] = (uint8_t)pack_cell(pe[u], pc[u], ps[u]);
                    }
                }
            }
            if (active) {
                load_agent(p.agents + env, a);
                if (!agent_in_range(a, S)) {
                    // only a block corrupted in device memory gets here: flag
                    // it (nx_sync: NX_E_DEVICE_CHECK) and continue the env from
                    // a safe pose instead of indexing outside its grid
                    if (grp.lane == 0) atomicOr(&p.ctl->flags, (unsigned)NX_FLAG_BOUNDS);
                    a.x = 1;
                    a.y = 1;
                    a.dir = 0;
                    a.nb = 0;
                }
            }
        }
        if (active) {
            if (returns) ret = returns[local];
            if (digest) dig = digest[local];
            if (episodes) eps = episodes[local];
        }
        __syncthreads();

        if constexpr (POL) {
            // the item's weight set, and every env's current view as its input row
            // the weight sets of the item's envs (one, or with fewer than 128
            // envs per set those of each aligned group of envs_per_agent)
            const uint32_t epa = rq->policy_epa;
            const uint32_t agent = (rq->key_base + item.local_begin) / epa;
            pol_agents = epa < (uint32_t)nxp::kRows ? (int)((item.n_envs + epa - 1) / epa) : 1;
            pol_rows = nxp::pol_rows(pol_agents, (int)epa);
            const uint4* src = reinterpret_cast<const uint4*>(rq->policy + (size_t)agent * nxp::kImageBytes);
            for (int i = tid; i < pol_agents * (nxp::kImageBytes / 16); i += nthreads)
                reinterpret_cast<uint4*>(sW)[i] = src[i];
            if (active) {
                ViewOut<G> v0;
                render_view<G>(grp, mygrid, S, W, a, s_dec, nullptr, v0, nullptr);
                nxp::store_obs_row(sA, tid, v0.sw);
            } else {
                nxp::store_zero_row(sA, tid);
            }
            if (steps > 0) nxp::policy_issue_first<kMultiPol>(sA, sW, tmem, &s_mbar, pol_agents);
        }

        // steps == 0 with reset_all: one emission of the episode-0 start state
        const int emissions = p.reset_all ? 1 : steps;
        const bool rnd = kLeanRandom || act_mode == NX_ACT_RANDOM;
        const uint32_t n_act = family == NX_DYNOBS ? 3u : 7u;
        uint32_t slot = call0 % (uint32_t)depth;
        // this env's row of the output ring (slot * n_envs + local), advanced
        // by one add per step
        size_t o = (size_t)slot * nreq + local;
        uint32_t my_draw = 0;  // G > 1 (unless kPreAct): this lane's random-action draw for step s0 + lane
        for (int s0 = 0; s0 < emissions; s0 += kActChunk) {
        if constexpr (kPreAct) {
            // the actions of steps s0 .. s0 + kActChunk - 1, drawn by the group's lanes
            const int cnt = min(kActChunk, steps - s0);
            if (active)
                for (int j = grp.lane; j < cnt; j += G)
                    s_act[gi * kActChunk + j] = (uint8_t)bounded(
                        draw(seed, key, 0xFFFFFFFFu, gstep0 + (uint32_t)(s0 + j), PURPOSE_ACTION, 0u), n_act);
            grp.sync();
        }
        const int s_end = min(emissions, s0 + kActChunk);
        for (int s = s0; s < s_end; ++s) {
            const size_t row0 = o - (size_t)gi;  // the item's first env in this slot
            uint8_t* sym_dst = (kOuts || obs_sym) ? obs_sym + row0 * NX_OBS_SYM_BYTES : nullptr;
            ViewOut<G> vo;
            float reward = 0.0f;
            int term = 0, trunc = 0;
            int pol_act = 0;  // fused policy: the greedy action of every env (all threads take part)
            if constexpr (POL)
                pol_act = nxp::policy_finish<kMultiPol>(sA, sW, tmem, &s_mbar, phase, (int)n_act, rq->shift1,
                                                        rq->shift2, pol_ok, pol_rows);
            if (!kPreAct && G > 1 && rnd && (s % G) == 0) {
                // the random actions of the next G steps depend only on the step
                // counter, so the group's lanes draw them in parallel
                my_draw = (s + grp.lane < steps) ? draw(seed, key, 0xFFFFFFFFu, gstep0 + (uint32_t)(s + grp.lane),
                                                        PURPOSE_ACTION, 0u)
                                                 : 0u;
            }
            // Episode starts (every env on a reset launch; autoreset after a
            // terminal or truncated step).  Groups of 8 or more lanes lay out
            // their own env; narrower groups hand every starting env of the
            // warp to all 32 lanes, one env after another, so one resetting env
            // never runs its layout generation serially while the rest of its
            // warp waits.
            const bool starts = active && (p.reset_all || a.done);
            if constexpr (G >= 8) {
                if (starts) {
                    // (out of line: the rare path's code stays out of the step loop)
                    const uint32_t ep = p.reset_all ? 0u : a.episode + 1u;
                    const uint4 r = reset_layout_grp<G, FAM>(grp, mygrid, S, W, family, n_balls, variant, seed, key, ep);
                    if (!(r.y & 0x100u) && grp.lane == 0) atomicOr(&p.ctl->flags, (unsigned)NX_FLAG_BOUNDS);
                    unpack_reset(r, ep, p.reset_all != 0, a);
                }
            } else {
                unsigned lead = __ballot_sync(0xFFFFFFFFu, starts && grp.lane == 0);
                while (lead) {
                    const int L = __ffs(lead) - 1;
                    lead &= lead - 1u;
                    const uint32_t ep = __shfl_sync(0xFFFFFFFFu, p.reset_all ? 0u : a.episode + 1u, L);
                    const uint32_t k = __shfl_sync(0xFFFFFFFFu, key, L);
                    const int owner = ((tid & ~31) + L) / G;  // group (env slot) of lane L
                    const uint4 r = reset_layout_warp<FAM>(sgrid + owner * ics, S, family, n_balls, variant, seed, k, ep);
                    if (!(r.y & 0x100u) && (tid & 31) == 0) atomicOr(&p.ctl->flags, (unsigned)NX_FLAG_BOUNDS);
                    if (gi == owner) unpack_reset(r, ep, p.reset_all != 0, a);
                }
                __syncwarp();
            }
            // (NX_DEBUG: the output row lies inside the caller's [depth, n_envs] buffers)
            const bool row_ok = NX_DCHECK(p.ctl, !active || o < (size_t)depth * nreq);
            if (active && row_ok) {
                // the step's action (an env that starts an episode ignores it)
                int action;
                if (POL) {
                    // exploration: with a draw below epsilon, the uniform random action
                    const uint32_t eps_t = rq->epsilon;
                    const uint32_t coin =
                        eps_t ? draw(seed, key, 0xFFFFFFFEu, gstep0 + (uint32_t)s, PURPOSE_EXPLORE, 0u) : 0xFFFFFFFFu;
                    action = coin < eps_t
                                 ? bounded(draw(seed, key, 0xFFFFFFFFu, gstep0 + (uint32_t)s, PURPOSE_ACTION, 0u), n_act)
                                 : pol_act;
                } else if (kPreAct) {
                    action = s_act[gi * kActChunk + (s - s0)];
                } else if (rnd) {
                    const uint32_t x = G > 1 ? grp.shfl(my_draw, s % G)
                                             : draw(seed, key, 0xFFFFFFFFu, gstep0 + (uint32_t)s, PURPOSE_ACTION, 0u);
                    action = bounded(x, n_act);
                } else {
                    action = actions[(size_t)(call0 + (uint32_t)s) * nreq + local];
                }
                if (out_action) out_action[o] = (int8_t)action;
                if (starts) {
                    // the new episode's start: reward padding 0, the action is ignored
                } else {
                    uint32_t d[8];
                    if (G > 1 && family == NX_DYNOBS) {  // (one lane per env draws inside env_step)
                        const uint32_t episode = a.episode, t = (uint32_t)a.t;
                        group_draws(grp, a.nb, d, [&](uint32_t k) -> uint32_t {
                            return draw(seed, key, episode, t, PURPOSE_BALL, k);
                        });
                    }
                    env_step(grp, mygrid, S, W, family, max_steps, a, action, d, reward_mode, lava_reward, action_cost,
                             time_cost, reward, term, trunc, p.ctl, seed, key);
                }
                // (every grid write above -- a reset, a ball move, the action's
                // write -- ends with a group barrier, so the view sees it)
                render_view<G>(grp, mygrid, S, W, a, s_dec, kSmemOcc ? s_occ : nullptr, vo,
                            RGB && obs_rgb ? stiles + gi * 49 : nullptr);
                if constexpr (POL) nxp::store_obs_row(sA, tid, vo.sw);  // the next step's policy input
                if constexpr (FULL) if (obs_full || obs_cat || obs_rgb_full) {
                    // fully observable views: every cell's triple, the agent's
                    // cell holding (agent, red, direction), zero beyond the grid;
                    // for the RGB view, the cell's tile (the agent facing its
                    // direction) goes to shared memory for the gather below
                    uint8_t* fo = obs_full ? obs_full + o * (size_t)(F * F * 3) : nullptr;
                    uint8_t* co = obs_cat ? obs_cat + o * (size_t)(F * F) : nullptr;
                    for (int c = grp.lane; c < F * F; c += G) {
                        const int y = c / F, x = c - y * F;
                        uint32_t tri = 0;
                        const bool agent_cell = x == a.x && y == a.y;
                        if (x < S && y < S) tri = agent_cell ? (10u | ((uint32_t)a.dir << 16)) : s_dec[mygrid[y * W + x]];
                        if (fo) {
                            fo[3 * c] = (uint8_t)tri;
                            fo[3 * c + 1] = (uint8_t)(tri >> 8);
                            fo[3 * c + 2] = (uint8_t)(tri >> 16);
                        }
                        if (co) co[c] = (uint8_t)tri;
                        if (RGB && obs_rgb_full && c < FR * FR) {
                            uint32_t tile = 0;
                            if (x < S && y < S)
                                tile = agent_cell ? 397u + (uint32_t)a.dir
                                                  : 1u + 18u * (tri & 0xFFu) + 3u * ((tri >> 8) & 0xFFu) + (tri >> 16);
                            sfull[gi * FR * FR + c] = (uint16_t)(tile < (uint32_t)NX_ATLAS_TILES ? tile : 0u);
                        }
                    }
                }
                {
                    // every lane of the group stores the same values (one
                    // transaction); absent outputs are skipped
                    if (kOuts || out_reward) out_reward[o] = reward;
                    if (kOuts || out_term) out_term[o] = (uint8_t)term;
                    if (kOuts || out_trunc) out_trunc[o] = (uint8_t)trunc;
                    if (!kOuts && out_mission) out_mission[o] = (uint8_t)a.mission;
                    ret += reward;
                    eps += (uint32_t)(term || trunc);
                }
                // Groups of 8 or more lanes (at most 4 envs per warp) write each
                // cell's three bytes straight to global memory (measured faster
                // than staging there); the staged path below serves the narrow
                // groups and the outputs that read the staged record (digest,
                // the categorical first-person view).
                if (G >= 8 && !digest && !(FULL && obs_cat_fp) && (kOuts || obs_sym))
                    write_view(grp, vo, obs_sym + o * NX_OBS_SYM_BYTES);
            }
            // fused policy: the next step's first layer runs during the stores
            if constexpr (POL)
                if (s + 1 < emissions) nxp::policy_issue_first<kMultiPol>(sA, sW, tmem, &s_mbar, pol_agents);
            if (G >= 8 && !digest && !(FULL && obs_cat_fp)) {
                // (stored above)
            } else {
            // Each warp stages the symbolic outputs of its own envs (placed at
            // the same address modulo 16 as their destination) and stores them
            // with 16-byte vectors, in `phases` parts; warps never wait for
            // each other here.
            for (int ph = 0; ph < phases; ++ph) {
                const int lo = wenv0 + ph * whalf, hi = min(n, min(wenv0 + epw, lo + whalf));
                // (NX_DEBUG: the warp's block of rows lies inside the caller's buffer)
                const bool blk_ok = NX_DCHECK(p.ctl, hi <= lo || row0 + (size_t)hi <= (size_t)depth * nreq);
                uint8_t* dst = (sym_dst && blk_ok) ? sym_dst + (size_t)lo * NX_OBS_SYM_BYTES : nullptr;
                uint8_t* stage = wstage + ((uint32_t)(uintptr_t)dst & 15u);
                if constexpr (kBulk) {
                    // the previous bulk copy out of this buffer must have read it
                    if (lane32 == 0) bulk_wait_read();
                    __syncwarp();
                }
                if (active && gi >= lo && gi < hi) {
                    uint8_t* my_sym = stage + (gi - lo) * NX_OBS_SYM_BYTES;
                    write_view(grp, vo, my_sym);
                    if (FULL && obs_cat_fp && row_ok) {
                        // categorical_first_person: the entity bytes of the staged view
                        grp.sync();
                        uint8_t* cf = obs_cat_fp + o * 49;
                        for (int c = grp.lane; c < 49; c += G) cf[c] = my_sym[3 * c];
                    }
                    if (digest) {
                        grp.sync();
                        if (grp.lane == 0) {
#pragma unroll 7
                            for (int c = 0; c < 49; ++c)
                                dig = digest_word(dig, (uint32_t)my_sym[3 * c] | ((uint32_t)my_sym[3 * c + 1] << 8) |
                                                           ((uint32_t)my_sym[3 * c + 2] << 16));
                            dig = digest_word(dig, __float_as_uint(reward));
                            dig = digest_word(dig, (uint32_t)term | ((uint32_t)trunc << 8));
                        }
                    }
                }
                if constexpr (kBulk) {
                    // the 16-byte-aligned body goes by one bulk copy, the
                    // ragged head and tail by plain stores
                    bulk_fence_smem();
                    __syncwarp();
                    if (dst && hi > lo) {
                        const int nbytes = (hi - lo) * NX_OBS_SYM_BYTES;
                        const int head = min(nbytes, (int)((16u - ((uint32_t)(uintptr_t)dst & 15u)) & 15u));
                        const int body = (nbytes - head) & ~15;
                        const int tail = nbytes - head - body;
                        if (lane32 < head) dst[lane32] = stage[lane32];
                        if (lane32 < tail) dst[head + body + lane32] = stage[head + body + lane32];
                        if (lane32 == 0 && body > 0) bulk_copy_s2g(dst + head, stage + head, (uint32_t)body);
                    }
                } else if constexpr (G >= 16) {
                    // at most two records (294 bytes): one pass of the warp, no loops
                    __syncwarp();
                    if (dst && hi > lo) {
                        const int nbytes = (hi - lo) * NX_OBS_SYM_BYTES;
                        const int head = min(nbytes, (int)((16u - ((uint32_t)(uintptr_t)dst & 15u)) & 15u));
                        const int body = (nbytes - head) & ~15;
                        const int tail = nbytes - head - body;
                        if (lane32 < head) dst[lane32] = stage[lane32];
                        if (lane32 < (body >> 4))
                            reinterpret_cast<uint4*>(dst + head)[lane32] = reinterpret_cast<const uint4*>(stage + head)[lane32];
                        if (lane32 < tail) dst[head + body + lane32] = stage[head + body + lane32];
                    }
                    __syncwarp();
                } else {
                    __syncwarp();
                    if (dst && hi > lo) coop_copy(dst, stage, (hi - lo) * NX_OBS_SYM_BYTES, lane32, 32);
                    __syncwarp();
                }
            }
            }
            // (NX_DEBUG: the item's image rows lie inside the caller's buffers)
            if (RGB && (obs_rgb || obs_rgb_full) && NX_DCHECK(p.ctl, row0 + (size_t)n <= (size_t)depth * nreq)) {
                __syncthreads();
                if (obs_rgb) coop_rgb(obs_rgb + row0 * NX_OBS_RGB_BYTES, stiles, p.atlas, n, tid, nthreads);
                if (FULL && obs_rgb_full)
                    coop_rgb_full(obs_rgb_full + row0 * (size_t)(3072 * FR * FR), sfull, p.atlas, n, FR, tid, nthreads);
                __syncthreads();
            }
            const bool wrap = slot + 1u == (uint32_t)depth;
            slot = wrap ? 0u : slot + 1u;
            o = wrap ? (size_t)local : o + nreq;
        }
        }

        if (kBulk && lane32 == 0) bulk_wait_all();  // every record of this item is in global memory
        // write the state back (the grids are written back by every thread of
        // the CTA, so all groups' last smem writes must be visible first)
        __syncthreads();
        if (active && grp.lane == 0) {
            if (a.invalid) atomicOr(&p.ctl->flags, (unsigned)NX_FLAG_INVALID_ACTION);
            store_agent(p.agents + env, a, item, (uint32_t)(item.grid_offset + (uint64_t)(gi * 3 * HW)));
            if (returns) returns[local] = ret;
            if (digest) digest[local] = dig;
            if (episodes) episodes[local] = eps;
        }
        {
            uint8_t* dst = p.grids + item.grid_offset;
            for (int i = tid; i < n * HW; i += nthreads) {
                const int e = (int)__umulhi((uint32_t)i, inv_hw), c = i - e * HW;
                int si = e * ics + c;
                if constexpr (kPad > 0) {
                    const int y = (int)__umulhi((uint32_t)c, inv_s), x = c - y * S;
                    si = e * ics + (y + kPad) * W + x + kPad;
                }
                const uint32_t code = sgrid[si];
                uint8_t* b = dst + (size_t)e * 3 * HW;
                b[c] = (uint8_t)cell_ent(code);
                b[HW + c] = (uint8_t)cell_col(code);
                b[2 * HW + c] = (uint8_t)cell_st(code);
            }
        }
        __syncthreads();
    }
    if constexpr (POL) {
        // every MMA has completed (each was waited for): free the tensor memory
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64u * (uint32_t)p.policy_agents));
        if (!pol_ok) atomicOr(&p.ctl->flags, (unsigned)NX_FLAG_WAIT_TIMEOUT);
    }
}


// The dynamic shared-memory limit is raised once per shape by
// nx_kernel_max_ctas (outside any stream capture); launches only launch.
template <int G, bool RGB, bool FULL, bool POL = false, int FAM = -1>
int launch_t(const nx_kparams& p, int grid, int smem, cudaStream_t st)
{
    nx_step_kernel<G, RGB, FULL, POL, FAM><<<grid, p.envs_per_cta * G, smem, st>>>(p);
    return (int)cudaGetLastError();
}

// The dynamic shared-memory limit is a per-kernel attribute shared by every
// context in the process, so it is always raised to the most the device
// allows next to the kernel's static shared memory (never lowered to one
// context's need).
template <int G, bool RGB, bool FULL, bool POL = false, int FAM = -1>
int occupancy_t(int threads, int smem, int* err)
{
    auto k = nx_step_kernel<G, RGB, FULL, POL, FAM>;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
    const int dyn_max = e == cudaSuccess ? optin - (int)fa.sharedSizeBytes : 0;  // static + dynamic <= opt-in limit
    if (e == cudaSuccess && smem > dyn_max) {
        *err = 0;
        return 0;
    }
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    int blocks = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, threads, smem);
    *err = (int)e;
    return blocks;
}

// Resident blocks per SM of the fused-policy instantiation, from its shared
// memory, registers and threads and the SM's 512 tensor-memory columns (64
// per weight set of a block).  The occupancy API reports one block for this kernel (it does
// not size the tensor memory a kernel allocates at run time), while the
// launch itself fits as many blocks as the resources allow; a block whose
// allocation found the columns taken would wait for them, never fail.
template <int FAM>
int launch_policy_t(const nx_kparams& p, int grid, int smem, cudaStream_t st)
{
    return launch_t<1, false, false, true, FAM>(p, grid, smem, st);
}

template <int FAM = -1>
int policy_occupancy(int threads, int smem, int agents, int* err)
{
    auto k = nx_step_kernel<1, false, false, true, FAM>;
    int dev = 0, optin = 0, smem_sm = 0, reserved = 0, regs_sm = 0, threads_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
    *err = (int)e;
    if (e != cudaSuccess) return 0;
    const int dyn_max = optin - (int)fa.sharedSizeBytes;
    if (smem > dyn_max) return 0;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    *err = (int)e;
    if (e != cudaSuccess) return 0;
    const int regs_block = ((fa.numRegs * 32 + 255) & ~255) * (threads / 32);  // per-warp allocation granule 256
    int n = smem_sm / (smem + (int)fa.sharedSizeBytes + reserved);
    n = std::min(n, regs_sm / std::max(regs_block, 1));
    n = std::min(n, threads_sm / threads);
    n = std::min(n, 512 / (64 * std::max(agents, 1)));
    return std::max(n, 0);
}

#define NX_DISPATCH_G(G_, RGB_, FULL_, FN, ...)                                                   \
    switch (G_) {                                                                                 \
    case 1: return RGB_ ? FN<1, true, FULL_>(__VA_ARGS__) : FN<1, false, FULL_>(__VA_ARGS__);    \
    case 2: return RGB_ ? FN<2, true, FULL_>(__VA_ARGS__) : FN<2, false, FULL_>(__VA_ARGS__);    \
    case 4: return RGB_ ? FN<4, true, FULL_>(__VA_ARGS__) : FN<4, false, FULL_>(__VA_ARGS__);    \
    case 8: return RGB_ ? FN<8, true, FULL_>(__VA_ARGS__) : FN<8, false, FULL_>(__VA_ARGS__);    \
    case 16: return RGB_ ? FN<16, true, FULL_>(__VA_ARGS__) : FN<16, false, FULL_>(__VA_ARGS__); \
    case 32: return RGB_ ? FN<32, true, FULL_>(__VA_ARGS__) : FN<32, false, FULL_>(__VA_ARGS__); \
    default: return -1;                                                                           \
    }

// The lean instantiations of one lane count, by family.
#define NX_DISPATCH_FAM(G_, FAM_, FN, ...)                                   \
    switch (FAM_) {                                                         \
    case 0: return FN<G_, false, false, false, 0>(__VA_ARGS__);             \
    case 1: return FN<G_, false, false, false, 1>(__VA_ARGS__);             \
    case 2: return FN<G_, false, false, false, 2>(__VA_ARGS__);             \
    case 3: return FN<G_, false, false, false, 3>(__VA_ARGS__);             \
    case 4: return FN<G_, false, false, false, 4>(__VA_ARGS__);             \
    case 5: return FN<G_, false, false, false, 5>(__VA_ARGS__);             \
    case 6: return FN<G_, false, false, false, 6>(__VA_ARGS__);             \
    case 7: return FN<G_, false, false, false, 7>(__VA_ARGS__);             \
    case 8: return FN<G_, false, false, false, 8>(__VA_ARGS__);             \
    case 9: return FN<G_, false, false, false, 9>(__VA_ARGS__);             \
    case 10: return FN<G_, false, false, false, 10>(__VA_ARGS__);           \
    case 11: return FN<G_, false, false, false, 11>(__VA_ARGS__);           \
    default: return -1;                                                     \
    }
static_assert(NX_N_FAMILIES == 11, "NX_DISPATCH_FAM lists every family, then any family (11)");

// The lean fused-policy instantiations, by family.
#define NX_DISPATCH_POL_FAM(FAM_, FN, ...)                             \
    switch (FAM_) {                                                    \
    case 0: return FN<0>(__VA_ARGS__);                                 \
    case 1: return FN<1>(__VA_ARGS__);                                 \
    case 2: return FN<2>(__VA_ARGS__);                                 \
    case 3: return FN<3>(__VA_ARGS__);                                 \
    case 4: return FN<4>(__VA_ARGS__);                                 \
    case 5: return FN<5>(__VA_ARGS__);                                 \
    case 6: return FN<6>(__VA_ARGS__);                                 \
    case 7: return FN<7>(__VA_ARGS__);                                 \
    case 8: return FN<8>(__VA_ARGS__);                                 \
    case 9: return FN<9>(__VA_ARGS__);                                 \
    case 10: return FN<10>(__VA_ARGS__);                               \
    case 11: return FN<11>(__VA_ARGS__);                               \
    default: return -1;                                                \
    }

}  // namespace nxk
