// nx_capi.cu -- host runtime behind the C ABI of include/navixgb.h: contexts
// (device state pool, work list), graph-captured persistent chunks, the
// per-family comparison form, the launch-shape autotuner, host-buffer
// rollouts with overlapped copies, snapshots and error reporting.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "navixgb.h"
#include "nx_internal.h"
#include "nx_runtime.h"
#include "nx_policy.cuh"
#include "nx_trace.h"

// ---------------------------------------------------------------------------
// errors

static thread_local std::string g_create_error;

const char* nx_status_str(nx_status s)
{
    switch (s) {
    case NX_OK: return "ok";
    case NX_PENDING: return "pending";
    case NX_E_INVAL: return "invalid argument";
    case NX_E_NOMEM: return "out of memory";
    case NX_E_CUDA: return "CUDA error";
    case NX_E_TIMEOUT: return "timeout";
    case NX_E_DEVICE_CHECK: return "device check failed";
    case NX_E_BUDGET: return "request exceeds the HBM budget";
    case NX_E_STATE: return "call out of order";
    case NX_E_CANCELED: return "request canceled";
    default: return "unknown status";
    }
}

const char* nx_last_error(const nx_env* env)
{
    if (!env) return g_create_error.c_str();
    return env->last_error.c_str();
}

nx_status nx_fail(nx_env* env, nx_status s, const std::string& msg)
{
    if (env)
        env->last_error = msg;
    else
        g_create_error = msg;
    return s;
}

nx_status nx_cuda_fail(nx_env* env, int err, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString((cudaError_t)err);
    return nx_fail(env, err == cudaErrorMemoryAllocation ? NX_E_NOMEM : NX_E_CUDA, m);
}

#define NX_CK(env, call, what)                                  \
    do {                                                        \
        int e_ = (int)(call);                                   \
        if (e_ != 0) return nx_cuda_fail((env), e_, (what));    \
    } while (0)

// ---------------------------------------------------------------------------
// device memory

void* nx_dev_alloc(nx_env* env, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (env->opt.alloc) {
        p = env->opt.alloc(bytes, env->opt.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        env->allocs.push_back(p);
        env->device_bytes += bytes;
    }
    return p;
}

void nx_dev_free(nx_env* env, void* p)
{
    if (!p) return;
    auto it = std::find(env->allocs.begin(), env->allocs.end(), p);
    if (it == env->allocs.end()) return;
    env->allocs.erase(it);
    if (env->opt.free)
        env->opt.free(p, env->opt.alloc_user);
    else
        cudaFree(p);
}

void nx_dev_free_all(nx_env* env)
{
    for (void* p : env->allocs) {
        if (env->opt.free)
            env->opt.free(p, env->opt.alloc_user);
        else
            cudaFree(p);
    }
    env->allocs.clear();
}

// ---------------------------------------------------------------------------
// options and creation

void nx_options_default(nx_options* o)
{
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->obs_flags = NX_OBS_SYM;
    o->reward_mode = NX_REWARD_MARKOV;
    o->lava_reward = 0.0f;
    o->n_balls = 4;
    o->steps_per_launch = 128;
    o->autotune = 1;
}

int nx_default_max_steps(int family, int size)
{
    switch (family) {
    case NX_DOORKEY: return 10 * size * size;
    case NX_FOURROOMS: return 100;
    case NX_GOTODOOR: return 5 * size * size;
    case NX_KEYCORRIDOR: {
        const int s = (size - 1) / 3 + 1;  // room side
        return 30 * s * s;
    }
    default: return 4 * size * size;
    }
}

int32_t nx_max_variant(int32_t family, int32_t size)
{
    if (size < NX_MIN_SIZE || size > NX_MAX_SIZE) return 0;
    if (family == NX_DISTSHIFT) return 1;
    if (family == NX_KEYCORRIDOR) return (size >= 7 && size % 3 == 1) ? 2 : -1;
    if (family != NX_LAVA_CROSSING && family != NX_SIMPLE_CROSSING) return 0;
    return 2 * ((size - 3) / 2);  // rows and columns 2, 4, .., size - 3
}

static nx_status validate_desc(const nx_desc& d, int n_balls, std::string* why)
{
    if (d.family < NX_EMPTY || d.family >= NX_N_FAMILIES) {
        *why = "unknown family";
        return NX_E_INVAL;
    }
    if (d.variant < 0 || d.variant > nx_max_variant(d.family, d.height)) {
        *why = "variant out of range for this family and size (see nx_max_variant)";
        return NX_E_INVAL;
    }
    if (d.height != d.width) {
        *why = "grids must be square (height == width)";
        return NX_E_INVAL;
    }
    if (d.height < NX_MIN_SIZE || d.height > NX_MAX_SIZE) {
        *why = "grid size must be in 5..19";
        return NX_E_INVAL;
    }
    if (d.max_steps > 65535) {
        *why = "max_steps must be <= 65535";
        return NX_E_INVAL;
    }
    if (d.family == NX_DYNOBS && (n_balls < 0 || n_balls > NX_MAX_BALLS)) {
        *why = "n_balls must be in 0..4";
        return NX_E_INVAL;
    }
    return NX_OK;
}

// Splits the env list into runs of equal descriptors and runs into items:
// envs_per_cta envs each, or fewer for grids larger than ref_side (their
// slots are larger, the block's grid region the same; nx_item_envs).
std::vector<nx_item> nx_build_items(const nx_env* env, const nx_launch_shape& s, int ref_side)
{
    std::vector<nx_item> items;
    const int n = env->n_envs;
    int i = 0;
    while (i < n) {
        int j = i;
        const nx_desc& d = env->descs[i];
        while (j < n && env->descs[j].family == d.family && env->descs[j].height == d.height &&
               env->descs[j].max_steps == d.max_steps && env->descs[j].variant == d.variant)
            ++j;
        const int E = nx_item_envs(s, ref_side, d.height);
        for (int b = i; b < j; b += E) {
            nx_item it;
            memset(&it, 0, sizeof it);
            it.env_begin = (uint32_t)b;
            it.n_envs = (uint32_t)std::min(E, j - b);
            it.grid_offset = env->grid_offset[b];
            it.req = 0;
            it.local_begin = (uint32_t)b;
            it.max_steps = (uint16_t)d.max_steps;
            it.family = (uint8_t)d.family;
            it.size = (uint8_t)d.height;
            it.variant = (uint32_t)d.variant;
            items.push_back(it);
        }
        i = j;
    }
    return items;
}

static nx_status create_common(nx_env** out, std::vector<nx_desc>&& descs, uint64_t seed, const nx_options* opts,
                               void* stream)
{
    if (!out) return nx_fail(nullptr, NX_E_INVAL, "env pointer is NULL");
    *out = nullptr;
    nx_options o;
    if (opts)
        o = *opts;
    else
        nx_options_default(&o);
    if (o.obs_flags & ~(uint32_t)(NX_OBS_SYM | NX_OBS_RGB | NX_OBS_RGB_FULL))
        return nx_fail(nullptr, NX_E_INVAL, "unknown obs flag");
    if ((o.obs_flags & (NX_OBS_RGB | NX_OBS_RGB_FULL)) && !o.atlas)
        return nx_fail(nullptr, NX_E_INVAL, "NX_OBS_RGB / NX_OBS_RGB_FULL need opts.atlas");
    if (o.steps_per_launch <= 0) o.steps_per_launch = 128;
    if (o.steps_per_launch > 1024) return nx_fail(nullptr, NX_E_INVAL, "steps_per_launch must be <= 1024");
    if (o.reward_mode != NX_REWARD_MARKOV && o.reward_mode != NX_REWARD_MINIGRID)
        return nx_fail(nullptr, NX_E_INVAL, "unknown reward mode");
    if ((o.alloc == nullptr) != (o.free == nullptr))
        return nx_fail(nullptr, NX_E_INVAL, "alloc and free callbacks go together");
    if (o.group_lanes || o.envs_per_cta) {
        nx_launch_shape s{o.group_lanes, o.envs_per_cta, 0};
        if (!o.group_lanes || !o.envs_per_cta || !nx_shape_supported(s))
            return nx_fail(nullptr, NX_E_INVAL, "unsupported group_lanes / envs_per_cta");
    }
    std::string why;
    for (auto& d : descs) {
        if (d.max_steps <= 0) d.max_steps = nx_default_max_steps(d.family, d.height);
        if (validate_desc(d, o.n_balls, &why) != NX_OK) return nx_fail(nullptr, NX_E_INVAL, why);
    }

    nx_env* env = new (std::nothrow) nx_env();
    if (!env) return nx_fail(nullptr, NX_E_NOMEM, "host allocation failed");
    env->opt = o;
    env->seed = seed;
    env->stream = (cudaStream_t)stream;
    env->n_envs = (int)descs.size();
    env->descs = std::move(descs);
    env->rgb = (o.obs_flags & (NX_OBS_RGB | NX_OBS_RGB_FULL)) != 0;
    env->rgb_full = (o.obs_flags & NX_OBS_RGB_FULL) != 0;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&env->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        nx_status s = nx_fail(nullptr, NX_E_CUDA, "no CUDA device available");
        delete env;
        return s;
    }
    env->device = dev;

    // grid pool layout and families
    size_t off = 0;
    bool seen[NX_N_FAMILIES] = {};
    env->grid_offset.resize(env->n_envs);
    for (int i = 0; i < env->n_envs; ++i) {
        const int S = env->descs[i].height;
        env->grid_offset[i] = off;
        off += (size_t)3 * S * S;
        env->max_side = std::max(env->max_side, S);
        seen[env->descs[i].family] = true;
    }
    env->grid_pool = off;
    env->grid_side = o.grid_side > 0 ? std::min(std::max((int)o.grid_side, (int)NX_MIN_SIZE), env->max_side) : env->max_side;
    env->n_families = 0;
    for (bool b : seen) env->n_families += b ? 1 : 0;
    env->lean_family = env->n_families == 1 ? (int)env->descs[0].family : NX_N_FAMILIES;

    env->d_agents = (nx_agent*)nx_dev_alloc(env, sizeof(nx_agent) * (size_t)env->n_envs);
    env->d_grids = (uint8_t*)nx_dev_alloc(env, env->grid_pool);
    env->d_req = (nx_req*)nx_dev_alloc(env, sizeof(nx_req));
    env->d_ctl = (nx_ctl*)nx_dev_alloc(env, sizeof(nx_ctl));
    if (!env->d_agents || !env->d_grids || !env->d_req || !env->d_ctl) {
        nx_dev_free_all(env);
        delete env;
        return nx_fail(nullptr, NX_E_NOMEM, "device allocation of the state pool failed");
    }
    if (env->rgb) {
        env->d_atlas = (uint8_t*)nx_dev_alloc(env, NX_ATLAS_BYTES);
        if (!env->d_atlas) {
            nx_dev_free_all(env);
            delete env;
            return nx_fail(nullptr, NX_E_NOMEM, "device allocation of the atlas failed");
        }
    }
    cudaError_t e = cudaSuccess;
    if (env->rgb) e = cudaMemcpyAsync(env->d_atlas, o.atlas, NX_ATLAS_BYTES, cudaMemcpyHostToDevice, env->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(env->d_ctl, 0, sizeof(nx_ctl), env->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(env->d_req, 0, sizeof(nx_req), env->stream);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&env->capture_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&env->copy_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        nx_dev_free_all(env);
        if (env->capture_stream) cudaStreamDestroy(env->capture_stream);
        delete env;
        return nx_fail(nullptr, NX_E_CUDA, std::string("context setup: ") + cudaGetErrorString(e));
    }
    env->req_host.seed = seed;
    env->req_host.n_envs = (uint32_t)env->n_envs;
    env->req_host.reward_mode = (uint32_t)o.reward_mode;
    env->req_host.lava_reward = o.lava_reward;
    env->req_host.action_cost = o.action_cost;
    env->req_host.time_cost = o.time_cost;
    env->req_host.n_balls = o.n_balls;
    env->req_host.key_base = o.env_index_base;

    // default launch shape (replaced by the autotuner when enabled)
    nx_launch_shape s{8, 32, env->rgb ? 1 : 0, 1, env->rgb_full ? env->max_side : 0};
    if (o.group_lanes)
        s = nx_launch_shape{o.group_lanes, o.envs_per_cta, env->rgb ? 1 : 0, o.staging == NX_STAGE_HALF ? 2 : 1,
                            env->rgb_full ? env->max_side : 0};
    nx_status st = nx_apply_shape(env, s);
    if (st != NX_OK) {
        std::string m = env->last_error;
        nx_destroy(env);
        return nx_fail(nullptr, st, m);
    }
    env->tuned = (o.group_lanes != 0) || !o.autotune;
    *out = env;
    return NX_OK;
}

nx_status nx_create(nx_env** env, int32_t family, int32_t size, int32_t n_envs, uint64_t seed, const nx_options* opts,
                    void* cuda_stream)
{
    if (n_envs < 1) return nx_fail(nullptr, NX_E_INVAL, "n_envs must be >= 1");
    std::vector<nx_desc> d((size_t)n_envs, nx_desc{family, size, size, 0, opts ? opts->variant : 0});
    return create_common(env, std::move(d), seed, opts, cuda_stream);
}

nx_status nx_create_mixed(nx_env** env, const nx_desc* host_descs, int32_t n_envs, uint64_t seed,
                          const nx_options* opts, void* cuda_stream)
{
    if (n_envs < 1 || !host_descs) return nx_fail(nullptr, NX_E_INVAL, "need n_envs >= 1 descriptors");
    std::vector<nx_desc> d(host_descs, host_descs + n_envs);
    return create_common(env, std::move(d), seed, opts, cuda_stream);
}

// ---------------------------------------------------------------------------
// launch shapes

nx_status nx_apply_shape(nx_env* env, const nx_launch_shape& s)
{
    if (!nx_shape_supported(s)) return nx_fail(env, NX_E_INVAL, "unsupported launch shape");
    int err = 0;
    const int per_sm = nx_kernel_max_ctas(s, env->grid_side, &err);
    if (err) return nx_cuda_fail(env, err, "occupancy query");
    if (per_sm < 1) return nx_fail(env, NX_E_INVAL, "launch shape does not fit on an SM");
    std::vector<nx_item> items = nx_build_items(env, s, env->grid_side);
    // family-ordered copy for the per-family form
    std::vector<nx_item> fam;
    std::vector<int> fam_begin(NX_N_FAMILIES + 1, 0);
    for (int f = 0; f < NX_N_FAMILIES; ++f) {
        fam_begin[f] = (int)fam.size();
        for (auto& it : items)
            if (it.family == f) fam.push_back(it);
    }
    fam_begin[NX_N_FAMILIES] = (int)fam.size();
    const size_t bytes = sizeof(nx_item) * items.size();
    if (bytes > env->items_capacity) {
        // the previous list stays allocated until the context goes away (small)
        env->d_items = (nx_item*)nx_dev_alloc(env, bytes);
        env->d_items_fam = (nx_item*)nx_dev_alloc(env, bytes);
        if (!env->d_items || !env->d_items_fam) return nx_fail(env, NX_E_NOMEM, "work list allocation failed");
        env->items_capacity = bytes;
    }
    NX_CK(env, cudaMemcpyAsync(env->d_items, items.data(), bytes, cudaMemcpyHostToDevice, env->stream), "work list upload");
    NX_CK(env, cudaMemcpyAsync(env->d_items_fam, fam.data(), bytes, cudaMemcpyHostToDevice, env->stream),
          "work list upload");
    // the host vectors must outlive the asynchronous copies from pageable memory
    NX_CK(env, cudaStreamSynchronize(env->stream), "work list upload");
    env->shape = s;
    env->per_sm_full = 0;  // recomputed for the new shape on first use
    env->per_sm_lean = 0;
    env->n_items = (int)items.size();
    env->fam_begin = fam_begin;
    env->grid_ctas = std::min(env->n_items, per_sm * env->sm_count);
    env->per_sm = per_sm;
    nx_drop_graphs(env);
    return NX_OK;
}

void nx_drop_graphs(nx_env* env)
{
    for (auto& g : env->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    env->graphs.clear();
}

nx_kparams nx_params(const nx_env* env, int launch_steps, int reset_all)
{
    nx_kparams p;
    memset(&p, 0, sizeof p);
    p.items = env->d_items;
    p.n_items = env->n_items;
    p.launch_steps = launch_steps;
    p.agents = env->d_agents;
    p.grids = env->d_grids;
    p.reqs = env->d_req;
    p.ctl = env->d_ctl;
    p.atlas = env->d_atlas;
    p.cell_stride = nx_slot_stride(env->shape, env->grid_side);
    p.item_strides = env->grid_side < env->max_side ? 1 : 0;
    p.envs_per_cta = env->shape.envs_per_cta;
    p.reset_all = reset_all;
    p.phases = env->shape.phases;
    p.rgb_full_side = env->shape.rgb_full_side;
    return p;
}

// Event pair around one step-kernel launch while profiling (never inside a
// stream capture: graph launches are bracketed from outside).
static nx_status prof_mark(nx_env* env, bool begin)
{
    if (!env->profiling) return NX_OK;
    if (begin && env->prof_used + 2 > env->prof_events.size()) {
        for (int k = 0; k < 2; ++k) {
            cudaEvent_t e;
            NX_CK(env, cudaEventCreate(&e), "profile event");
            env->prof_events.push_back(e);
        }
    }
    NX_CK(env, cudaEventRecord(env->prof_events[env->prof_used], env->stream), "profile event");
    env->prof_used += 1;
    return NX_OK;
}

// The fused-policy launch shape: 1 lane per env, 128 envs per block; its lean
// instantiation (the context's family or any family) with the Markov reward.
static nx_launch_shape policy_shape(const nx_env* env, int agents)
{
    nx_launch_shape ps{1, nxp::kRows, 0, 1, 0, false, true};
    // the lean instantiations hold one weight set per block
    if (agents == 1 && env->lean_family >= 0 && env->req_host.reward_mode == NX_REWARD_MARKOV)
        ps.lean_family = env->lean_family;
    ps.policy_agents = agents;
    return ps;
}

// The lean instantiation of the context's shape (for its one family, or for
// any family; the Markov reward; see nx_step_kernel), with its grid; false
// where there is none.  Its
// occupancy query (which sets a kernel attribute) runs on first use, outside
// any stream capture.
static bool lean_shape(const nx_env* env, nx_launch_shape* s, int* grid)
{
    if (env->lean_family < 0 || env->req_host.reward_mode != NX_REWARD_MARKOV) return false;
    nx_launch_shape ls = env->shape;
    ls.lean_family = env->lean_family;
    if (!nx_lean_supported(ls)) return false;
    if (env->per_sm_lean == 0) {
        int err = 0;
        const int n = nx_kernel_max_ctas(ls, env->grid_side, &err);
        if (err) cudaGetLastError();
        env->per_sm_lean = (!err && n >= 1) ? n : -1;  // the general kernel serves where it is unavailable
    }
    if (env->per_sm_lean < 1) return false;
    *s = ls;
    *grid = std::min(env->n_items, env->per_sm_lean * env->sm_count);
    return true;
}

// Whether a random-action call's outputs suit the lean kernels, which store
// the symbolic view, the reward and both flags without testing for them and
// write no mission and no action.
static bool lean_outputs(const nx_out* o)
{
    return o && o->obs_sym && o->reward && o->terminated && o->truncated && !o->mission && !o->action;
}

// Launch shape and grid of a call: the plain instantiation, its lean form
// (lean: a call with random actions and no action output), or (full) the
// one that also writes the fully observable views.
static nx_status shape_for(nx_env* env, bool full, nx_launch_shape* s, int* grid, bool policy = false,
                           bool lean = false)
{
    if (policy) {
        *s = policy_shape(env, env->policy_agents);
        *grid = std::min(env->n_items_pol, env->per_sm_pol * env->sm_count);
        return NX_OK;
    }
    *s = env->shape;
    *grid = env->grid_ctas;
    if (!full && lean) lean_shape(env, s, grid);
    if (!full) return NX_OK;
    s->full = true;
    if (env->per_sm_full <= 0) {
        int err = 0;
        env->per_sm_full = nx_kernel_max_ctas(*s, env->grid_side, &err);
        if (err) return nx_cuda_fail(env, err, "occupancy query");
        if (env->per_sm_full < 1) return nx_fail(env, NX_E_INVAL, "launch shape does not fit on an SM");
    }
    *grid = std::min(env->n_items, env->per_sm_full * env->sm_count);
    return NX_OK;
}

static nx_status launch_chunk(nx_env* env, int steps, cudaStream_t st, bool full, bool policy = false,
                              bool lean = false)
{
    nx_launch_shape s;
    int grid = 0;
    nx_status ss = shape_for(env, full, &s, &grid, policy, lean);
    if (ss != NX_OK) return ss;
    nx_kparams p = nx_params(env, steps, 0);
    if (policy) {
        p.items = env->d_items_pol;
        p.n_items = env->n_items_pol;
        p.envs_per_cta = nxp::kRows;
        p.cell_stride = nx_slot_stride(s, env->max_side);
        p.item_strides = 0;  // the policy's work list: 128 envs per item, uniform slots
        p.policy_agents = env->policy_agents;
        p.phases = 1;
        p.rgb_full_side = 0;
    }
    NX_CK(env, nx_launch_step_kernel(s, p, grid, st), "step kernel launch");
    NX_CK(env, nx_launch_advance(env->d_req, 1, st), "advance launch");
    return NX_OK;
}

// A direct (uncaptured) chunk launch on the context stream, counted and timed.
static nx_status launch_chunk_direct(nx_env* env, int steps, bool full, bool policy = false, bool lean = false)
{
    nx_range range("nx_chunk");
    nx_status st = prof_mark(env, true);
    if (st == NX_OK) st = launch_chunk(env, steps, env->stream, full, policy, lean);
    if (st == NX_OK) st = prof_mark(env, false);
    env->n_step_launches += 1;
    env->n_all_launches += 2;
    return st;
}

// Replays (capturing on first use) the graph {step kernel of `steps` steps;
// counter advance}.  The graph reads every per-call argument from the
// device-side request record, so one graph serves every call.
static nx_status launch_chunk_graph(nx_env* env, int steps, bool full, bool policy = false, bool lean = false)
{
    nx_range range("nx_chunk");
    nx_graph* g = nullptr;
    for (auto& c : env->graphs)
        if (c.steps == steps && c.full == full && c.policy == policy && c.lean == lean) g = &c;
    if (!g) {
        nx_graph ng;
        ng.steps = steps;
        ng.full = full;
        ng.policy = policy;
        ng.lean = lean;
        if (full || lean) {  // the occupancy query sets a kernel attribute: keep it out of the capture
            nx_launch_shape s;
            int grid = 0;
            nx_status ss = shape_for(env, full, &s, &grid, false, lean);
            if (ss != NX_OK) return ss;
        }
        cudaGraph_t graph = nullptr;
        NX_CK(env, cudaStreamBeginCapture(env->capture_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        nx_status st = launch_chunk(env, steps, env->capture_stream, full, policy, lean);
        cudaError_t e = cudaStreamEndCapture(env->capture_stream, &graph);
        if (st != NX_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        NX_CK(env, e, "end capture");
        e = cudaGraphInstantiate(&ng.exec, graph, 0);
        cudaGraphDestroy(graph);
        NX_CK(env, e, "graph instantiate");
        env->graphs.push_back(ng);
        g = &env->graphs.back();
    }
    nx_status st = prof_mark(env, true);
    if (st != NX_OK) return st;
    NX_CK(env, cudaGraphLaunch(g->exec, env->stream), "graph launch");
    env->n_step_launches += 1;
    env->n_all_launches += 2;
    return prof_mark(env, false);
}

// ---------------------------------------------------------------------------
// reset / step / rollout

static nx_req call_req(const nx_env* env, int steps, int act_mode, const int8_t* actions, const nx_out* out)
{
    nx_req r = env->req_host;
    r.gstep = 0;
    r.call_step = 0;
    r.steps = steps;
    r.depth = (out && out->depth > 0) ? out->depth : 1;
    r.act_mode = act_mode;
    r.actions = actions;
    r.obs_sym = out ? out->obs_sym : nullptr;
    r.obs_rgb = (out && env->rgb) ? out->obs_rgb : nullptr;
    r.reward = out ? out->reward : nullptr;
    r.terminated = out ? out->terminated : nullptr;
    r.truncated = out ? out->truncated : nullptr;
    r.returns = nullptr;
    r.digest = nullptr;
    r.episodes = nullptr;
    r.obs_full = out ? out->obs_full : nullptr;
    r.obs_cat = out ? out->obs_cat : nullptr;
    r.obs_cat_fp = out ? out->obs_cat_fp : nullptr;
    r.obs_rgb_full = (out && env->rgb_full) ? out->obs_rgb_full : nullptr;
    r.mission = out ? out->mission : nullptr;
    r.action_out = out ? out->action : nullptr;
    if (act_mode == NX_ACT_POLICY) {
        r.policy = env->d_policy;
        r.policy_epa = env->policy_epa;
        r.shift1 = env->policy_shift1;
        r.shift2 = env->policy_shift2;
        r.epsilon = env->policy_eps;
    }
    r.full_side = (out && out->full_side > 0) ? out->full_side : env->max_side;
    return r;
}

static bool wants_full(const nx_out* out)
{
    return out && (out->obs_full || out->obs_cat || out->obs_cat_fp || out->obs_rgb_full);
}

static nx_status check_out(nx_env* env, const nx_out* out)
{
    if (out && out->obs_rgb && !env->rgb) return nx_fail(env, NX_E_INVAL, "obs_rgb given but NX_OBS_RGB was not enabled");
    if (out && (out->obs_full || out->obs_cat) && out->full_side > 0 && out->full_side < env->max_side)
        return nx_fail(env, NX_E_INVAL, "full_side is smaller than the largest grid");
    if (out && (out->full_side < 0 || out->full_side > 255)) return nx_fail(env, NX_E_INVAL, "full_side must be 0..255");
    if (out && out->obs_rgb_full && !env->rgb_full)
        return nx_fail(env, NX_E_INVAL, "obs_rgb_full given but NX_OBS_RGB_FULL was not enabled");
    if (out && out->obs_rgb_full && out->full_side != 0 && out->full_side != env->max_side)
        return nx_fail(env, NX_E_INVAL, "obs_rgb_full needs full_side equal to the largest grid size");
    return NX_OK;
}

nx_status nx_reset(nx_env* env, const nx_out* out)
{
    nx_range range("nx_reset");
    if (!env) return nx_fail(nullptr, NX_E_INVAL, "env is NULL");
    nx_status st = check_out(env, out);
    if (st != NX_OK) return st;
    nx_req r = call_req(env, 0, NX_ACT_RANDOM, nullptr, out);
    NX_CK(env, nx_launch_configure(env->d_req, r, 1, env->stream), "configure");
    nx_kparams p = nx_params(env, 0, 1);
    nx_launch_shape sh;
    int grid = 0;
    st = shape_for(env, wants_full(out), &sh, &grid);
    if (st != NX_OK) return st;
    NX_CK(env, nx_launch_step_kernel(sh, p, grid, env->stream), "reset kernel launch");
    env->n_all_launches += 2;
    env->was_reset = true;
    return NX_OK;
}

static nx_status rollout_impl(nx_env* env, int32_t n_steps, int32_t act_mode, const int8_t* d_actions,
                              const nx_out* traj, bool per_family)
{
    nx_range range(per_family ? "nx_rollout_per_family" : "nx_rollout");
    if (!env) return nx_fail(nullptr, NX_E_INVAL, "env is NULL");
    if (!env->was_reset) return nx_fail(env, NX_E_STATE, "nx_reset must come first");
    if (n_steps < 0) return nx_fail(env, NX_E_INVAL, "n_steps must be >= 0");
    if (act_mode != NX_ACT_RANDOM && act_mode != NX_ACT_BUFFER && act_mode != NX_ACT_POLICY)
        return nx_fail(env, NX_E_INVAL, "unknown act_mode");
    if (act_mode == NX_ACT_BUFFER && !d_actions) return nx_fail(env, NX_E_INVAL, "NX_ACT_BUFFER needs actions");
    const bool policy = act_mode == NX_ACT_POLICY;
    if (policy) {
        if (!env->d_policy) return nx_fail(env, NX_E_STATE, "NX_ACT_POLICY needs nx_set_policy first");
        if (per_family) return nx_fail(env, NX_E_INVAL, "the per-family form has no fused policy");
        if (traj && (traj->obs_rgb || traj->obs_rgb_full || wants_full(traj)))
            return nx_fail(env, NX_E_INVAL, "policy rollouts write the symbolic outputs only");
    }
    nx_status st = check_out(env, traj);
    if (st != NX_OK) return st;
    if (n_steps == 0) return NX_OK;
    if (!env->tuned && !policy) {
        st = nx_autotune(env);
        if (st != NX_OK) return st;
    }
    const int C = per_family ? 1 : env->opt.steps_per_launch;
    const bool full = wants_full(traj);
    nx_launch_shape fsh;
    int fgrid = 0;
    st = shape_for(env, full, &fsh, &fgrid);
    if (st != NX_OK) return st;
    nx_req r = call_req(env, C, act_mode, d_actions, traj);
    NX_CK(env, nx_launch_configure(env->d_req, r, 0, env->stream), "configure");
    env->n_all_launches += 1;
    if (per_family) {
        for (int t = 0; t < n_steps; ++t) {
            for (int f = 0; f < NX_N_FAMILIES; ++f) {
                const int b = env->fam_begin[f], e = env->fam_begin[f + 1];
                if (e == b) continue;
                nx_kparams p = nx_params(env, 1, 0);
                p.items = env->d_items_fam + b;
                p.n_items = e - b;
                const int grid = std::min(e - b, (full ? env->per_sm_full : env->per_sm) * env->sm_count);
                st = prof_mark(env, true);
                if (st != NX_OK) return st;
                NX_CK(env, nx_launch_step_kernel(fsh, p, grid, env->stream), "per-family launch");
                st = prof_mark(env, false);
                if (st != NX_OK) return st;
                env->n_step_launches += 1;
                env->n_all_launches += 1;
            }
            NX_CK(env, nx_launch_advance(env->d_req, 1, env->stream), "advance launch");
            env->n_all_launches += 1;
        }
        return NX_OK;
    }
    // random actions with the lean kernels' outputs (lean_outputs) run the
    // lean kernel where the context has one (the Markov reward)
    const bool lean = act_mode == NX_ACT_RANDOM && lean_outputs(traj);
    const int nfull = n_steps / C, rem = n_steps % C;
    for (int k = 0; k < nfull; ++k) {
        st = launch_chunk_graph(env, C, full, policy, lean);
        if (st != NX_OK) return st;
    }
    if (rem) {
        NX_CK(env, nx_launch_set_steps(env->d_req, rem, env->stream), "set steps");
        env->n_all_launches += 1;
        st = launch_chunk_direct(env, rem, full, policy, lean);
        if (st != NX_OK) return st;
    }
    return NX_OK;
}

// ---------------------------------------------------------------------------
// fused policy: weight images in the tensor-core operand layout (bf16, see
// nx_policy.cuh), a 128-env work list whose items never split a weight set.

nx_status nx_set_policy(nx_env* env, const nx_policy* pol)
{
    if (!env || !pol) return nx_fail(env, NX_E_INVAL, "NULL argument");
    if (pol->n_agents < 1 || pol->envs_per_agent < 1) return nx_fail(env, NX_E_INVAL, "n_agents and envs_per_agent >= 1");
    if (!pol->w1 || !pol->b1 || !pol->w2 || !pol->b2 || !pol->w3 || !pol->b3)
        return nx_fail(env, NX_E_INVAL, "policy weights missing");
    if (pol->shift1 < 0 || pol->shift1 > 24 || pol->shift2 < 0 || pol->shift2 > 24)
        return nx_fail(env, NX_E_INVAL, "shifts must be 0..24");
    const uint64_t base = env->opt.env_index_base;
    const uint64_t epa = (uint64_t)pol->envs_per_agent;
    if ((base + (uint64_t)env->n_envs - 1) / epa >= (uint64_t)pol->n_agents)
        return nx_fail(env, NX_E_INVAL, "the weight sets do not cover every env");
    const int A = pol->n_agents;
    auto bias_ok = [](const int32_t* b, size_t n) {
        for (size_t i = 0; i < n; ++i)
            if (b[i] > (1 << 22) || b[i] < -(1 << 22)) return false;
        return true;
    };
    if (!bias_ok(pol->b1, (size_t)A * 64) || !bias_ok(pol->b2, (size_t)A * 64) || !bias_ok(pol->b3, (size_t)A * 7))
        return nx_fail(env, NX_E_INVAL, "biases must lie in [-2^22, 2^22]");
    // a block of 128 envs holds one weight set, or 128 / envs_per_agent of them
    if (epa < (uint64_t)nxp::kRows && (epa < 16 || nxp::kRows % epa != 0))
        return nx_fail(env, NX_E_INVAL, "envs_per_agent must be 16, 32, 64 or at least 128");
    const int agents = epa < (uint64_t)nxp::kRows ? (int)(nxp::kRows / epa) : 1;
    std::vector<nx_item> items = nx_build_items(env, nx_launch_shape{1, nxp::kRows, 0}, env->max_side);
    for (const nx_item& it : items) {
        const uint64_t first = base + it.local_begin, last = first + it.n_envs - 1;
        if (epa >= (uint64_t)nxp::kRows ? first / epa != last / epa : first % epa != 0)
            return nx_fail(env, NX_E_INVAL, "a weight set boundary splits a 128-env block of the work list");
    }
    const nx_launch_shape ps = policy_shape(env, agents);
    int err = 0;
    const int per_sm = nx_kernel_max_ctas(ps, env->max_side, &err);
    if (err) return nx_cuda_fail(env, err, "occupancy query");
    if (per_sm < 1) return nx_fail(env, NX_E_INVAL, "the fused policy does not fit on an SM with these grids");
    // weight images: bf16 bits of int8 values (exact); biases of layers 1, 2 as
    // f32 times 2^-shift (exact for |b| <= 2^22), of layer 3 as int32
    std::vector<uint8_t> img((size_t)A * nxp::kImageBytes, 0);
    auto bf16 = [](int v) -> uint16_t {
        float f = (float)v;
        uint32_t u;
        memcpy(&u, &f, 4);
        return (uint16_t)(u >> 16);  // exact: |v| <= 128 has at most 8 significant bits
    };
    for (int a = 0; a < A; ++a) {
        uint8_t* im = img.data() + (size_t)a * nxp::kImageBytes;
        auto put = [&](int region, int n, int k, int v) {
            const uint16_t b = bf16(v);
            memcpy(im + region + nxp::tile_offset(n, k), &b, 2);
        };
        for (int n = 0; n < 64; ++n)
            for (int k = 0; k < 64; ++k) {
                put(nxp::kW1, n, k, k < nxp::kIn ? pol->w1[((size_t)a * 64 + n) * 49 + k] : 0);
                put(nxp::kW2, n, k, pol->w2[((size_t)a * 64 + n) * 64 + k]);
                if (n < 16) put(nxp::kW3, n, k, n < 7 ? pol->w3[((size_t)a * 7 + n) * 64 + k] : 0);
            }
        for (int j = 0; j < 64; ++j) {
            const float s1 = std::ldexp((float)pol->b1[(size_t)a * 64 + j], -pol->shift1);
            const float s2 = std::ldexp((float)pol->b2[(size_t)a * 64 + j], -pol->shift2);
            memcpy(im + nxp::kB1 + 4 * j, &s1, 4);
            memcpy(im + nxp::kB2 + 4 * j, &s2, 4);
        }
        memcpy(im + nxp::kB3, pol->b3 + (size_t)a * 7, 7 * 4);
    }
    NX_CK(env, cudaStreamSynchronize(env->stream), "policy upload");  // the previous images are no longer read
    if (env->d_policy) nx_dev_free(env, env->d_policy);
    if (env->d_items_pol) nx_dev_free(env, env->d_items_pol);
    env->d_policy = nullptr;
    env->d_items_pol = nullptr;
    env->d_policy = (uint8_t*)nx_dev_alloc(env, img.size());
    env->d_items_pol = (nx_item*)nx_dev_alloc(env, items.size() * sizeof(nx_item));
    if (!env->d_policy || !env->d_items_pol) return nx_fail(env, NX_E_NOMEM, "policy allocation failed");
    env->policy_host = std::move(img);
    env->items_pol = std::move(items);
    NX_CK(env, cudaMemcpyAsync(env->d_policy, env->policy_host.data(), env->policy_host.size(), cudaMemcpyHostToDevice,
                               env->stream), "policy upload");
    NX_CK(env, cudaMemcpyAsync(env->d_items_pol, env->items_pol.data(), env->items_pol.size() * sizeof(nx_item),
                               cudaMemcpyHostToDevice, env->stream), "policy work list upload");
    env->n_items_pol = (int)env->items_pol.size();
    env->per_sm_pol = per_sm;
    env->policy_agents = agents;
    env->policy_epa = (uint32_t)epa;
    env->policy_shift1 = pol->shift1;
    env->policy_shift2 = pol->shift2;
    env->policy_eps = pol->epsilon;
    return NX_OK;
}

nx_status nx_step(nx_env* env, const int8_t* d_actions, const nx_out* out)
{
    return rollout_impl(env, 1, d_actions ? NX_ACT_BUFFER : NX_ACT_RANDOM, d_actions, out, false);
}

nx_status nx_rollout(nx_env* env, int32_t n_steps, int32_t act_mode, const int8_t* d_actions_TN, const nx_out* traj)
{
    return rollout_impl(env, n_steps, act_mode, d_actions_TN, traj, false);
}

nx_status nx_rollout_per_family(nx_env* env, int32_t n_steps, int32_t act_mode, const int8_t* d_actions_TN,
                                const nx_out* traj)
{
    return rollout_impl(env, n_steps, act_mode, d_actions_TN, traj, true);
}

// ---------------------------------------------------------------------------
// host-buffer rollout: chunk k computes into device buffer k % 2 while the
// copy stream drains buffer (k - 1) % 2 into the host arrays.

nx_status nx_rollout_host(nx_env* env, int32_t n_steps, int32_t act_mode, const int8_t* h_actions, const nx_out* h)
{
    nx_range range("nx_rollout_host");
    if (!env) return nx_fail(nullptr, NX_E_INVAL, "env is NULL");
    if (!env->was_reset) return nx_fail(env, NX_E_STATE, "nx_reset must come first");
    if (n_steps < 0) return nx_fail(env, NX_E_INVAL, "n_steps must be >= 0");
    if (act_mode != NX_ACT_RANDOM && act_mode != NX_ACT_BUFFER) return nx_fail(env, NX_E_INVAL, "unknown act_mode");
    if (act_mode == NX_ACT_BUFFER && !h_actions) return nx_fail(env, NX_E_INVAL, "NX_ACT_BUFFER needs actions");
    nx_status st = check_out(env, h);
    if (st != NX_OK) return st;
    if (h && (h->obs_full || h->obs_cat || h->obs_cat_fp || h->obs_rgb_full || h->action))
        return nx_fail(env, NX_E_INVAL, "the fully observable views and the actions are device outputs only");
    if (n_steps == 0) return NX_OK;
    if (!env->tuned) {
        st = nx_autotune(env);
        if (st != NX_OK) return st;
    }
    const int C = env->opt.steps_per_launch;
    const size_t N = (size_t)env->n_envs;
    const bool want_sym = h && h->obs_sym, want_rgb = h && h->obs_rgb, want_r = h && h->reward,
               want_te = h && h->terminated, want_tr = h && h->truncated, want_m = h && h->mission;
    const size_t per_step = N * ((want_sym ? NX_OBS_SYM_BYTES : 0) + (want_rgb ? NX_OBS_RGB_BYTES : 0) +
                                 (want_r ? 4 : 0) + (want_te ? 1 : 0) + (want_tr ? 1 : 0) + (want_m ? 1 : 0)) +
                            (act_mode == NX_ACT_BUFFER ? N : 0) + 256 * 7;
    const size_t need = per_step * (size_t)C;
    if (need > env->host_chunk_bytes) {
        for (int b = 0; b < 2; ++b) {
            env->host_chunk[b] = (uint8_t*)nx_dev_alloc(env, need);
            if (!env->host_chunk[b]) return nx_fail(env, NX_E_NOMEM, "host-rollout staging allocation failed");
        }
        env->host_chunk_bytes = need;
        for (int b = 0; b < 2; ++b) {
            if (!env->ev_done[b]) NX_CK(env, cudaEventCreateWithFlags(&env->ev_done[b], cudaEventDisableTiming), "event");
            if (!env->ev_copied[b])
                NX_CK(env, cudaEventCreateWithFlags(&env->ev_copied[b], cudaEventDisableTiming), "event");
        }
    }
    for (int b = 0; b < 2; ++b)
        if (!env->ev_done[b]) {
            NX_CK(env, cudaEventCreateWithFlags(&env->ev_done[b], cudaEventDisableTiming), "event");
            NX_CK(env, cudaEventCreateWithFlags(&env->ev_copied[b], cudaEventDisableTiming), "event");
        }
    // host outputs form a ring of D time slots: step i goes to slot i % D
    // (D <= 0 or D >= n_steps: every step has its own slot)
    const int D = (h && h->depth > 0 && h->depth < n_steps) ? h->depth : n_steps;
    bool used[2] = {false, false};
    for (int t0 = 0, k = 0; t0 < n_steps; t0 += C, ++k) {
        const int b = k & 1;
        const int Ck = std::min(C, n_steps - t0);
        if (used[b]) NX_CK(env, cudaStreamWaitEvent(env->stream, env->ev_copied[b], 0), "wait copy");
        uint8_t* p = env->host_chunk[b];
        auto take = [&](size_t bytes) {
            uint8_t* q = p;
            p += (bytes + 255) & ~(size_t)255;
            return q;
        };
        nx_out d;
        memset(&d, 0, sizeof d);
        d.depth = Ck;
        if (want_sym) d.obs_sym = take((size_t)Ck * N * NX_OBS_SYM_BYTES);
        if (want_rgb) d.obs_rgb = take((size_t)Ck * N * NX_OBS_RGB_BYTES);
        if (want_r) d.reward = (float*)take((size_t)Ck * N * 4);
        if (want_te) d.terminated = take((size_t)Ck * N);
        if (want_tr) d.truncated = take((size_t)Ck * N);
        if (want_m) d.mission = take((size_t)Ck * N);
        int8_t* dact = nullptr;
        if (act_mode == NX_ACT_BUFFER) {
            dact = (int8_t*)take((size_t)Ck * N);
            NX_CK(env, cudaMemcpyAsync(dact, h_actions + (size_t)t0 * N, (size_t)Ck * N, cudaMemcpyHostToDevice, env->stream),
                  "actions upload");
        }
        nx_req r = call_req(env, Ck, act_mode, dact, &d);
        NX_CK(env, nx_launch_configure(env->d_req, r, 0, env->stream), "configure");
        env->n_all_launches += 1;
        st = launch_chunk_direct(env, Ck, false, false, act_mode == NX_ACT_RANDOM && lean_outputs(&d));
        if (st != NX_OK) return st;
        NX_CK(env, cudaEventRecord(env->ev_done[b], env->stream), "record");
        NX_CK(env, cudaStreamWaitEvent(env->copy_stream, env->ev_done[b], 0), "wait compute");
        // only the chunk's last min(Ck, D) steps survive in a ring of D
        // slots (a chunk longer than the ring overwrites its own first
        // steps); they go to host slots (t0 + skip) % D onwards, in two
        // copies where they wrap around the end of the ring, never more
        // than D slots in all
        const int keep = std::min(Ck, D), skip = Ck - keep;
        const int s0 = (t0 + skip) % D, first = std::min(keep, D - s0);
        auto copy_back = [&](void* host, const void* dev, size_t step_bytes) -> cudaError_t {
            const uint8_t* src = (const uint8_t*)dev + (size_t)skip * step_bytes;
            cudaError_t e = cudaMemcpyAsync((uint8_t*)host + (size_t)s0 * step_bytes, src, (size_t)first * step_bytes,
                                            cudaMemcpyDeviceToHost, env->copy_stream);
            if (e == cudaSuccess && first < keep)
                e = cudaMemcpyAsync(host, src + (size_t)first * step_bytes, (size_t)(keep - first) * step_bytes,
                                    cudaMemcpyDeviceToHost, env->copy_stream);
            return e;
        };
        if (want_sym) NX_CK(env, copy_back(h->obs_sym, d.obs_sym, N * NX_OBS_SYM_BYTES), "copy back");
        if (want_rgb) NX_CK(env, copy_back(h->obs_rgb, d.obs_rgb, N * NX_OBS_RGB_BYTES), "copy back");
        if (want_r) NX_CK(env, copy_back(h->reward, d.reward, N * 4), "copy back");
        if (want_te) NX_CK(env, copy_back(h->terminated, d.terminated, N), "copy back");
        if (want_tr) NX_CK(env, copy_back(h->truncated, d.truncated, N), "copy back");
        if (want_m) NX_CK(env, copy_back(h->mission, d.mission, N), "copy back");
        NX_CK(env, cudaEventRecord(env->ev_copied[b], env->copy_stream), "record");
        used[b] = true;
    }
    NX_CK(env, cudaStreamSynchronize(env->copy_stream), "copy stream");
    NX_CK(env, cudaStreamSynchronize(env->stream), "stream");
    return NX_OK;
}

// ---------------------------------------------------------------------------
// autotuner: times every supported shape on a scratch copy of the state and
// keeps the fastest.  Results never depend on the shape (each env's
// arithmetic is independent of where it runs), only the speed does.

nx_status nx_autotune(nx_env* env)
{
    nx_range range("nx_autotune");
    env->tuned = true;
    // (2 lanes per env, never the fastest in any measured workload and the
    // slowest to try, stays available as an explicit shape only)
    const int lanes[5] = {1, 4, 8, 16, 32};
    const int threads[4] = {32, 64, 128, 256};
    const size_t N = (size_t)env->n_envs;
    // scratch: state copy + one output slot
    nx_agent* sa = (nx_agent*)nx_dev_alloc(env, sizeof(nx_agent) * N);
    uint8_t* sg = (uint8_t*)nx_dev_alloc(env, env->grid_pool);
    nx_req* sr = (nx_req*)nx_dev_alloc(env, sizeof(nx_req));
    uint8_t* so = (uint8_t*)nx_dev_alloc(env, N * NX_OBS_SYM_BYTES + 16);
    uint8_t* srgb = env->rgb ? (uint8_t*)nx_dev_alloc(env, N * NX_OBS_RGB_BYTES) : nullptr;
    float* srew = (float*)nx_dev_alloc(env, N * 4);
    uint8_t* sflag = (uint8_t*)nx_dev_alloc(env, N * 2);
    if (!sa || !sg || !sr || !so || !srew || !sflag || (env->rgb && !srgb))
        return nx_fail(env, NX_E_NOMEM, "autotune scratch allocation failed");
    // 64-step trials (32-step ones could not separate shapes 1-2 % apart)
    const int T = std::min(env->opt.steps_per_launch, 64);
    nx_out o;
    memset(&o, 0, sizeof o);
    o.obs_sym = so;
    o.obs_rgb = srgb;
    o.reward = srew;
    o.terminated = sflag;
    o.truncated = sflag + N;
    o.depth = 1;
    nx_req r = call_req(env, T, NX_ACT_RANDOM, nullptr, &o);
    cudaEvent_t e0, e1;
    NX_CK(env, cudaEventCreate(&e0), "event");
    NX_CK(env, cudaEventCreate(&e1), "event");
    const nx_launch_shape orig = env->shape;
    nx_launch_shape best = orig;
    int best_side = env->grid_side;
    float best_ms = 1e30f;
    // slot sides to try: the largest grid's (every item holds envs_per_cta
    // envs), and the next largest side of the batch (items of the largest
    // grids hold fewer envs, every block needs less shared memory); an
    // explicit nx_options.grid_side is kept
    std::vector<int> sides{env->max_side};
    if (env->opt.grid_side <= 0) {
        int next = 0;
        for (const nx_desc& d : env->descs)
            if (d.height < env->max_side) next = std::max(next, d.height);
        if (next > 0) sides.push_back(next);
    } else {
        sides[0] = env->grid_side;
    }
    for (int side : sides)
    for (int G : lanes)
        for (int th : threads)
            for (int ph = 1; ph <= 2; ++ph) {
            nx_launch_shape s{G, th / G, env->rgb ? 1 : 0, ph, env->rgb_full ? env->max_side : 0};
            if (!nx_shape_supported(s)) continue;
            env->grid_side = side;
            if (nx_apply_shape(env, s) != NX_OK) {
                cudaGetLastError();
                continue;
            }
            // time the kernel these calls will run: the lean one where the
            // context has it (the timing request has random actions)
            nx_launch_shape ls = s;
            int lgrid = env->grid_ctas;
            lean_shape(env, &ls, &lgrid);
            nx_kparams p = nx_params(env, T, 0);
            p.phases = s.phases;
            p.agents = sa;
            p.grids = sg;
            p.reqs = sr;
            float ms_min = 1e30f;
            bool ok = true;
            for (int rep = 0; rep < 4 && ok; ++rep) {
                ok = cudaMemcpyAsync(sa, env->d_agents, sizeof(nx_agent) * N, cudaMemcpyDeviceToDevice, env->stream) == cudaSuccess &&
                     cudaMemcpyAsync(sg, env->d_grids, env->grid_pool, cudaMemcpyDeviceToDevice, env->stream) == cudaSuccess &&
                     nx_launch_configure(sr, r, 1, env->stream) == 0 && cudaEventRecord(e0, env->stream) == cudaSuccess &&
                     nx_launch_step_kernel(ls, p, lgrid, env->stream) == 0 &&
                     cudaEventRecord(e1, env->stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
                float ms = 0;
                if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && rep > 0) ms_min = std::min(ms_min, ms);
            }
            if (!ok) {
                cudaGetLastError();
                continue;
            }
            if (ms_min < best_ms) {
                best_ms = ms_min;
                best = s;
                best_side = side;
            }
            env->tune_log.push_back(nx_tune_entry{s.group_lanes, s.envs_per_cta, ms_min});
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(env->stream);
    for (void* q : {(void*)sa, (void*)sg, (void*)sr, (void*)so, (void*)srgb, (void*)srew, (void*)sflag}) nx_dev_free(env, q);
    env->grid_side = best_side;
    return nx_apply_shape(env, best);
}

// ---------------------------------------------------------------------------
// snapshots, flags, sync, info, destroy

size_t nx_state_bytes(const nx_env* env)
{
    if (!env) return 0;
    return 64 + sizeof(nx_agent) * (size_t)env->n_envs + env->grid_pool;
}

nx_status nx_get_state(nx_env* env, void* host_buf, size_t bytes)
{
    if (!env || !host_buf) return nx_fail(env, NX_E_INVAL, "NULL argument");
    if (bytes < nx_state_bytes(env)) return nx_fail(env, NX_E_INVAL, "buffer smaller than nx_state_bytes()");
    uint8_t* b = (uint8_t*)host_buf;
    memset(b, 0, 64);
    memcpy(b, "NXST", 4);
    const uint32_t ver = 1, n = (uint32_t)env->n_envs;
    uint32_t gstep = 0;
    const uint64_t pool = env->grid_pool, seed = env->seed;
    NX_CK(env, cudaMemcpyAsync(&gstep, &env->d_req->gstep, 4, cudaMemcpyDeviceToHost, env->stream), "snapshot");
    NX_CK(env, cudaMemcpyAsync(b + 64, env->d_agents, sizeof(nx_agent) * n, cudaMemcpyDeviceToHost, env->stream), "snapshot");
    NX_CK(env, cudaMemcpyAsync(b + 64 + sizeof(nx_agent) * n, env->d_grids, env->grid_pool, cudaMemcpyDeviceToHost, env->stream),
          "snapshot");
    NX_CK(env, cudaStreamSynchronize(env->stream), "snapshot");
    memcpy(b + 4, &ver, 4);
    memcpy(b + 8, &n, 4);
    memcpy(b + 12, &gstep, 4);
    memcpy(b + 16, &pool, 8);
    memcpy(b + 24, &seed, 8);
    return NX_OK;
}

nx_status nx_set_state(nx_env* env, const void* host_buf, size_t bytes)
{
    if (!env || !host_buf) return nx_fail(env, NX_E_INVAL, "NULL argument");
    if (bytes < nx_state_bytes(env)) return nx_fail(env, NX_E_INVAL, "buffer smaller than nx_state_bytes()");
    const uint8_t* b = (const uint8_t*)host_buf;
    uint32_t ver, n, gstep;
    uint64_t pool;
    memcpy(&ver, b + 4, 4);
    memcpy(&n, b + 8, 4);
    memcpy(&gstep, b + 12, 4);
    memcpy(&pool, b + 16, 8);
    if (memcmp(b, "NXST", 4) != 0 || ver != 1 || n != (uint32_t)env->n_envs || pool != env->grid_pool)
        return nx_fail(env, NX_E_INVAL, "snapshot does not match this context");
    const nx_agent* ag = (const nx_agent*)(b + 64);
    const uint8_t* pool_b = b + 64 + sizeof(nx_agent) * n;
    for (uint32_t i = 0; i < n; ++i) {
        const nx_desc& d = env->descs[i];
        const nx_agent& a = ag[i];
        const int S = d.height;
        if (a.family != d.family || a.size != S || a.grid_offset != (uint32_t)env->grid_offset[i] ||
            a.max_steps != d.max_steps)
            return nx_fail(env, NX_E_INVAL, "snapshot descriptors differ from this context");
        // every index the kernels derive from the snapshot must stay inside the grid
        bool ok = a.x < S && a.y < S && a.dir < 4 && a.done <= 1 && a.invalid <= 1 && a.n_balls <= NX_MAX_BALLS &&
                  a.carry_ent <= 10 && a.carry_col <= 5 && (d.family == NX_DYNOBS || a.n_balls == 0) &&
                  (d.family == NX_GOTODOOR ? a.mission <= 5 : a.mission == NX_NO_MISSION);
        // balls lie in the interior: placed there, they only move to empty cells
        for (int k = 0; ok && k < a.n_balls; ++k)
            ok = a.ball_x[k] >= 1 && a.ball_x[k] <= S - 2 && a.ball_y[k] >= 1 && a.ball_y[k] <= S - 2;
        const uint8_t* g = pool_b + env->grid_offset[i];
        for (int c = 0; ok && c < S * S; ++c) ok = g[c] <= 10 && g[S * S + c] <= 5 && g[2 * S * S + c] <= 2;
        if (!ok) return nx_fail(env, NX_E_INVAL, "snapshot holds out-of-range state");
    }
    // the staging copy keeps the upload asynchronous-safe for pageable memory
    std::vector<uint8_t> tmp(b + 64, b + 64 + sizeof(nx_agent) * n + env->grid_pool);
    NX_CK(env, cudaMemcpyAsync(env->d_agents, tmp.data(), sizeof(nx_agent) * n, cudaMemcpyHostToDevice, env->stream), "restore");
    NX_CK(env, cudaMemcpyAsync(env->d_grids, tmp.data() + sizeof(nx_agent) * n, env->grid_pool, cudaMemcpyHostToDevice,
                               env->stream), "restore");
    nx_req r = call_req(env, 0, NX_ACT_RANDOM, nullptr, nullptr);
    r.gstep = gstep;
    NX_CK(env, nx_launch_configure(env->d_req, r, 2, env->stream), "restore");
    NX_CK(env, cudaStreamSynchronize(env->stream), "restore");
    env->was_reset = true;
    return NX_OK;
}

nx_status nx_device_flags(nx_env* env, uint32_t* flags)
{
    if (!env || !flags) return nx_fail(env, NX_E_INVAL, "NULL argument");
    uint32_t f = 0;
    NX_CK(env, cudaMemcpyAsync(&f, &env->d_ctl->flags, 4, cudaMemcpyDeviceToHost, env->stream), "flags");
    NX_CK(env, cudaStreamSynchronize(env->stream), "flags");
    *flags = f;
    return NX_OK;
}

nx_status nx_sync(nx_env* env, double timeout_s)
{
    if (!env) return nx_fail(nullptr, NX_E_INVAL, "env is NULL");
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(env->stream);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return nx_cuda_fail(env, e, "stream");
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (timeout_s > 0 && el > timeout_s) return nx_fail(env, NX_E_TIMEOUT, "stream did not finish in time");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    uint32_t f = 0;
    nx_status st = nx_device_flags(env, &f);
    if (st != NX_OK) return st;
    if (f & NX_FLAG_BOUNDS) return nx_fail(env, NX_E_DEVICE_CHECK, "a device bounds check fired");
    return NX_OK;
}

nx_status nx_get_info(const nx_env* env, nx_info* info)
{
    if (!env || !info) return NX_E_INVAL;
    memset(info, 0, sizeof *info);
    info->group_lanes = env->shape.group_lanes;
    info->envs_per_cta = env->shape.envs_per_cta;
    info->staging = env->shape.phases > 1 ? NX_STAGE_HALF : NX_STAGE_FULL;
    info->n_items = env->n_items;
    info->grid_ctas = env->grid_ctas;
    info->smem_bytes = nx_kernel_smem_bytes(env->shape, env->grid_side);
    info->grid_side = env->grid_side;
    info->steps_per_launch = env->opt.steps_per_launch;
    info->n_envs = env->n_envs;
    info->n_families = env->n_families;
    info->state_bytes = nx_state_bytes(env);
    info->device_bytes = env->device_bytes;
    if (env->d_policy) {
        const nx_launch_shape ps = policy_shape(env, env->policy_agents);
        info->policy_items = env->n_items_pol;
        info->policy_ctas_per_sm = env->per_sm_pol;
        info->policy_grid_ctas = std::min(env->n_items_pol, env->per_sm_pol * env->sm_count);
        info->policy_smem_bytes = nx_kernel_smem_bytes(ps, env->max_side);
    }
    nx_launch_shape ls;
    int lgrid = 0;
    info->lean_family = -1;
    if (lean_shape(env, &ls, &lgrid)) {
        info->lean_family = ls.lean_family;
        info->lean_grid_ctas = lgrid;
    }
    return NX_OK;
}

nx_status nx_profile_begin(nx_env* env)
{
    if (!env) return nx_fail(nullptr, NX_E_INVAL, "env is NULL");
    env->profiling = true;
    env->prof_used = 0;
    return NX_OK;
}

nx_status nx_profile_end(nx_env* env, double* kernel_ms, int64_t* step_launches)
{
    if (!env) return nx_fail(nullptr, NX_E_INVAL, "env is NULL");
    env->profiling = false;
    NX_CK(env, cudaStreamSynchronize(env->stream), "profile sync");
    double total = 0.0;
    for (size_t i = 0; i + 1 < env->prof_used; i += 2) {
        float ms = 0.0f;
        NX_CK(env, cudaEventElapsedTime(&ms, env->prof_events[i], env->prof_events[i + 1]), "profile elapsed");
        total += ms;
    }
    if (kernel_ms) *kernel_ms = total;
    if (step_launches) *step_launches = (int64_t)(env->prof_used / 2);
    env->prof_used = 0;
    return NX_OK;
}

nx_status nx_launch_counts(const nx_env* env, int64_t* step_launches, int64_t* all_launches)
{
    if (!env) return NX_E_INVAL;
    if (step_launches) *step_launches = env->n_step_launches;
    if (all_launches) *all_launches = env->n_all_launches;
    return NX_OK;
}

void nx_destroy(nx_env* env)
{
    if (!env) return;
    cudaStreamSynchronize(env->stream);
    nx_drop_graphs(env);
    for (int b = 0; b < 2; ++b) {
        if (env->ev_done[b]) cudaEventDestroy(env->ev_done[b]);
        if (env->ev_copied[b]) cudaEventDestroy(env->ev_copied[b]);
    }
    if (env->copy_stream) {
        cudaStreamSynchronize(env->copy_stream);
        cudaStreamDestroy(env->copy_stream);
    }
    if (env->capture_stream) cudaStreamDestroy(env->capture_stream);
    for (cudaEvent_t e : env->prof_events) cudaEventDestroy(e);
    nx_dev_free_all(env);
    delete env;
}
