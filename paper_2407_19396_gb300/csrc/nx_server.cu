// nx_server.cu -- continuous batching of rollout requests (config C5).
//
// A worker thread owns the GPU.  Requests wait in a FIFO queue and are
// admitted, strictly in arrival order, as soon as their device memory fits in
// the budget (one pool allocated up front, carved first-fit) and a request
// record is free.  Every chunk launch runs the persistent step kernel over
// the work items of *all* admitted requests; each request record carries its
// own seed, step counter and step count for the chunk, so a request advances
// exactly as it would alone.  The host queues chunk k+1 (uploads, kernel,
// result copies of the requests it finishes, an event) before it retires
// chunk k, so the GPU is never idle while requests are waiting.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "navixgb.h"
#include "nx_internal.h"
#include "nx_runtime.h"
#include "nx_trace.h"

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

// First-fit allocator over [0, cap) with coalescing frees (offsets only).
struct RangeAlloc {
    std::map<size_t, size_t> free_;  // offset -> length
    size_t cap = 0, used = 0, peak = 0;
    void init(size_t c)
    {
        cap = c;
        free_.clear();
        free_[0] = c;
        used = peak = 0;
    }
    bool alloc(size_t len, size_t* off)
    {
        len = up256(len);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                *off = it->first;
                const size_t rest = it->second - len, o = it->first + len;
                free_.erase(it);
                if (rest) free_[o] = rest;
                used += len;
                peak = std::max(peak, used);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t len)
    {
        len = up256(len);
        used -= len;
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

// Per-request device block: [agents][grids][step][returns][digest][episodes][obs];
// `step` takes each step's reward and flags (the lean kernels store them
// unconditionally; the server returns per-env returns instead).
struct Layout {
    size_t agents, grids, step, returns, digest, episodes, obs, total, tail;  // tail = bytes from `returns` to the end
    static Layout of(int n, int S)
    {
        Layout l;
        l.agents = 0;
        l.grids = up256((size_t)n * sizeof(nx_agent));
        l.step = l.grids + up256((size_t)n * 3 * S * S);
        l.returns = l.step + up256((size_t)n * 4) + up256((size_t)n * 2);
        l.digest = l.returns + up256((size_t)n * 4);
        l.episodes = l.digest + up256((size_t)n * 8);
        l.obs = l.episodes + up256((size_t)n * 4);
        l.total = l.obs + up256((size_t)n * NX_OBS_SYM_BYTES);
        l.tail = l.total - l.returns;
        return l;
    }
};

struct SReq {
    nx_request r{};
    int max_steps = 0;
    Layout lay{};
    size_t dev_off = 0, host_off = 0;
    int slot = -1;
    int launched = 0;  // steps enqueued so far
    bool admitted = false, reset_done = false;
    bool cancel = false;  // nx_cancel on an admitted request: no further chunk
    nvtxRangeId_t range = 0;  // NVTX range from admission to retirement
    nx_result res{};
    bool finished = false;
};

// One block of a chunk's batched clears and result copies: bytes from src
// (or zeros when src is NULL) to dst; every block is 256-byte aligned and a
// whole number of 256-byte units (the request layout pads every part).
struct BlockCopy {
    const uint8_t* src;
    uint8_t* dst;
    uint64_t bytes;
};

// All of a chunk's blocks in one launch: blockIdx.y picks the block, the x
// dimension strides its 16-byte words.  The result copies write the pinned
// host staging through its device mapping (SM stores over the host link run
// at the copy engines' rate), so a chunk that finishes many requests needs
// one launch instead of one copy per request, and the clears of the
// accumulators of its new requests one launch instead of one memset each.
__global__ void nx_block_copy_kernel(const BlockCopy* blocks)
{
    const BlockCopy b = blocks[blockIdx.y];
    const uint64_t n = b.bytes / 16, stride = (uint64_t)gridDim.x * blockDim.x;
    uint4* d = reinterpret_cast<uint4*>(b.dst);
    if (b.src) {
        const uint4* src = reinterpret_cast<const uint4*>(b.src);
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) d[i] = src[i];
    } else {
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) d[i] = make_uint4(0u, 0u, 0u, 0u);
    }
}

struct Chunk {
    cudaEvent_t ev = nullptr;
    std::vector<uint64_t> finishing;
    bool valid = false;
};

uint64_t fold(uint64_t h, uint32_t w) { return (h ^ (uint64_t)w) * 0x100000001B3ull; }

}  // namespace

struct nx_server {
    nx_options opt{};
    cudaStream_t stream = nullptr;
    size_t budget = 0;
    int device = 0;
    int sm_count = 0;
    nx_launch_shape shape{1, 128, 0, 2};  // measured best for the serving mix
    int cell_stride = 0, per_sm = 0, chunk = 128;
    int per_sm_lean = 0;  // the lean kernel for several families (chunks without a digest), 0: none
    // Requests of at most small_envs envs run with 16 lanes per env on a second
    // stream, beside the one-lane launch of the larger ones: at one lane per
    // env a small request's step is one long dependent chain (about 9 us),
    // which would set the floor of every chunk.  0: one shape for all.
    nx_launch_shape small{16, 8, 0, 1};
    int small_envs = 0, cell_stride_small = 0, per_sm_small = 0, per_sm_small_lean = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    int max_slots = 4096;
    size_t max_items = 0;

    uint8_t* d_pool = nullptr;
    uint8_t* h_pool = nullptr;  // pinned result staging
    RangeAlloc dev_alloc, host_alloc;
    nx_req* d_reqs = nullptr;
    nx_req* h_reqs[2] = {nullptr, nullptr};
    nx_item* d_items = nullptr;  // [2 staging buffers][2 * max_items]
    nx_item* h_items[2] = {nullptr, nullptr};
    // batched clears and result copies: [2 staging buffers][2 * max_slots]
    BlockCopy* d_blocks = nullptr;
    BlockCopy* h_blocks[2] = {nullptr, nullptr};
    uint8_t* h_pool_dev = nullptr;  // the pinned staging as the device addresses it
    nx_ctl* d_ctl = nullptr;
    Chunk chunks[2];

    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> waiting;
    std::unordered_map<uint64_t, SReq> reqs;
    std::vector<uint64_t> active;
    std::vector<int> free_slots;
    bool stop = false;
    nx_status fatal = NX_OK;
    std::string fatal_msg;
    uint64_t next_ticket = 1;
    nx_server_stats stats{};
    double busy_since = -1.0;
};

namespace {

void set_fatal(nx_server* s, nx_status st, const std::string& msg)
{
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal == NX_OK) {
        s->fatal = st;
        s->fatal_msg = msg;
    }
}

#define SRV_CK(call, what)                                                                               \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) {                                                                         \
            set_fatal(s, NX_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e_));                  \
            return false;                                                                                \
        }                                                                                                \
    } while (0)

nx_req record_of(const nx_server* s, const SReq& q, int steps)
{
    nx_req r;
    memset(&r, 0, sizeof r);
    uint8_t* base = s->d_pool + q.dev_off;
    r.seed = q.r.seed;
    r.gstep = (uint32_t)q.launched;
    r.call_step = 0;
    r.steps = steps;
    r.depth = 1;
    r.n_envs = (uint32_t)q.r.n_envs;
    r.act_mode = NX_ACT_RANDOM;
    r.obs_sym = base + q.lay.obs;
    r.reward = (float*)(base + q.lay.step);
    r.terminated = base + q.lay.step + up256((size_t)q.r.n_envs * 4);
    r.truncated = r.terminated + q.r.n_envs;
    r.returns = (float*)(base + q.lay.returns);
    r.digest = (q.r.flags & NX_REQ_DIGEST) ? (uint64_t*)(base + q.lay.digest) : nullptr;
    r.episodes = (uint32_t*)(base + q.lay.episodes);
    r.reward_mode = (uint32_t)s->opt.reward_mode;
    r.lava_reward = s->opt.lava_reward;
    r.action_cost = s->opt.action_cost;
    r.time_cost = s->opt.time_cost;
    r.n_balls = s->opt.n_balls;
    r.key_base = 0;
    return r;
}

// The launch shape of a request's work items.
const nx_launch_shape& shape_of_req(const nx_server* s, const nx_request& r)
{
    return r.n_envs <= s->small_envs ? s->small : s->shape;
}

void items_of(const nx_server* s, const SReq& q, std::vector<nx_item>& out)
{
    const int E = shape_of_req(s, q.r).envs_per_cta, n = q.r.n_envs, S = q.r.size;
    const uint32_t agent0 = (uint32_t)((q.dev_off + q.lay.agents) / sizeof(nx_agent));
    for (int b = 0; b < n; b += E) {
        nx_item it;
        memset(&it, 0, sizeof it);
        it.env_begin = agent0 + (uint32_t)b;
        it.n_envs = (uint32_t)std::min(E, n - b);
        it.grid_offset = (uint64_t)(q.dev_off + q.lay.grids + (size_t)b * 3 * S * S);
        it.req = (uint32_t)q.slot;
        it.local_begin = (uint32_t)b;
        it.max_steps = (uint16_t)q.max_steps;
        it.family = (uint8_t)q.r.family;
        it.size = (uint8_t)S;
        it.variant = (uint32_t)q.r.variant;
        out.push_back(it);
    }
}

// Copies a finished request's results into the caller's buffers and releases
// its memory (the chunk that produced them has completed).
void retire(nx_server* s, uint64_t t)
{
    std::unique_lock<std::mutex> lk(s->mu);
    SReq& q = s->reqs.at(t);
    const int n = q.r.n_envs;
    const uint8_t* h = s->h_pool + q.host_off;  // same relative layout as the device tail
    const float* ret = (const float*)h;
    const uint64_t* dig = (const uint64_t*)(h + (q.lay.digest - q.lay.returns));
    const uint32_t* eps = (const uint32_t*)(h + (q.lay.episodes - q.lay.returns));
    const uint8_t* obs = h + (q.lay.obs - q.lay.returns);
    const bool canceled = q.cancel;
    lk.unlock();
    uint64_t d = 0;
    uint32_t e = 0;
    if (!canceled) {
        if (q.r.returns) memcpy(q.r.returns, ret, (size_t)n * 4);
        if (q.r.final_obs) memcpy(q.r.final_obs, obs, (size_t)n * NX_OBS_SYM_BYTES);
        const bool with_digest = (q.r.flags & NX_REQ_DIGEST) != 0;
        for (int i = 0; i < n; ++i) {
            if (with_digest) {
                d = fold(d, (uint32_t)dig[i]);
                d = fold(d, (uint32_t)(dig[i] >> 32));
            }
            e += eps[i];
        }
    }
    lk.lock();
    q.res.digest = d;
    q.res.episodes = e;
    q.res.env_steps = (uint64_t)n * (uint64_t)q.launched;  // the steps that ran
    q.res.status = canceled ? NX_E_CANCELED : NX_OK;
    q.res.t_done = now_s();
    nvtxRangeEnd(q.range);
    q.finished = true;
    s->dev_alloc.release(q.dev_off, q.lay.total);
    s->host_alloc.release(q.host_off, q.lay.tail);
    s->free_slots.push_back(q.slot);
    s->stats.finished += canceled ? 0 : 1;
    s->stats.canceled += canceled ? 1 : 0;
    s->stats.env_steps += q.res.env_steps;
    s->stats.in_use_bytes = s->dev_alloc.used;
    s->cv_done.notify_all();
}

// Launches the blocks [first, first + n) of buffer `cur` (already uploaded).
bool launch_blocks(nx_server* s, int cur, size_t first, size_t n, uint64_t max_bytes)
{
    if (n == 0) return true;
    const unsigned threads = 256;
    const uint64_t per_x = (uint64_t)threads * 16 * 4;  // four 16-byte words per thread and pass
    const unsigned gx = (unsigned)std::min<uint64_t>(128, std::max<uint64_t>(1, (max_bytes + per_x - 1) / per_x));
    nx_block_copy_kernel<<<dim3(gx, (unsigned)n), threads, 0, s->stream>>>(s->d_blocks + (size_t)cur * 2 * s->max_slots +
                                                                            first);
    SRV_CK(cudaGetLastError(), "block copy launch");
    return true;
}

bool wait_chunk(nx_server* s, Chunk& c)
{
    if (!c.valid) return true;
    SRV_CK(cudaEventSynchronize(c.ev), "chunk completion");
    for (uint64_t t : c.finishing) retire(s, t);
    c.finishing.clear();
    c.valid = false;
    return true;
}

// One iteration: admit, reset the newcomers and launch the next chunk into
// staging buffer `cur`, then retire the previous chunk (buffer cur ^ 1) while
// the new one runs.  Returns false on a fatal CUDA error.
bool iterate(nx_server* s, int& cur, bool* idle)
{
    nx_range range("nx_server_iteration");
    std::vector<uint64_t> fresh;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        while (!s->stop && !s->waiting.empty() && !s->free_slots.empty()) {
            const uint64_t t = s->waiting.front();
            SReq& q = s->reqs.at(t);
            size_t doff, hoff;
            if (!s->dev_alloc.alloc(q.lay.total, &doff)) break;
            if (!s->host_alloc.alloc(q.lay.tail, &hoff)) {
                s->dev_alloc.release(doff, q.lay.total);
                break;
            }
            s->waiting.pop_front();
            q.dev_off = doff;
            q.host_off = hoff;
            q.slot = s->free_slots.back();
            s->free_slots.pop_back();
            q.admitted = true;
            q.res.t_start = now_s();
            q.range = nvtxRangeStartA("nx_request");
            s->active.push_back(t);
            fresh.push_back(t);
        }
        s->stats.in_use_bytes = s->dev_alloc.used;
        s->stats.peak_bytes = s->dev_alloc.peak;
        *idle = s->active.empty();
        if (*idle && s->busy_since >= 0) {
            s->stats.busy_s += now_s() - s->busy_since;
            s->busy_since = -1.0;
        } else if (!*idle && s->busy_since < 0) {
            s->busy_since = now_s();
        }
    }
    if (*idle) return wait_chunk(s, s->chunks[0]) && wait_chunk(s, s->chunks[1]);

    Chunk& c = s->chunks[cur];
    if (!wait_chunk(s, c)) return false;  // normally retired already by the previous iteration
    nx_req* hr = s->h_reqs[cur];
    nx_item* hi = s->h_items[cur];
    std::vector<nx_item> reset_items, step_items, reset_small, step_small;
    std::vector<uint64_t> finishing, still;
    // element addresses of the request map never move, but lookups must not
    // race with nx_submit's insertions: take the pointers under the lock
    std::vector<const SReq*> fresh_q, finishing_q;
    int launch_steps = 0;
    bool digest_reset = false, digest_step = false;  // some request of the launch wants its digest
    bool digest_reset_s = false, digest_step_s = false;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (uint64_t t : fresh) {
            fresh_q.push_back(&s->reqs.at(t));
            const nx_request& r = fresh_q.back()->r;
            const bool sm = r.n_envs <= s->small_envs;
            items_of(s, *fresh_q.back(), sm ? reset_small : reset_items);
            (sm ? digest_reset_s : digest_reset) |= (r.flags & NX_REQ_DIGEST) != 0;
        }
        for (uint64_t t : s->active) {
            SReq& q = s->reqs.at(t);
            if (q.cancel) {
                // withdrawn: no steps in this chunk (a request admitted in this
                // very iteration still has its reset items, which read this
                // record); its memory is released when this chunk, queued
                // behind every earlier use, completes
                hr[q.slot] = record_of(s, q, 0);
                finishing.push_back(t);
                continue;
            }
            const int k = std::min(s->chunk, q.r.horizon - q.launched);
            hr[q.slot] = record_of(s, q, k);
            const bool sm = q.r.n_envs <= s->small_envs;
            items_of(s, q, sm ? step_small : step_items);
            (sm ? digest_step_s : digest_step) |= (q.r.flags & NX_REQ_DIGEST) != 0;
            launch_steps = std::max(launch_steps, k);
            q.launched += k;
            if (q.launched >= q.r.horizon) {
                finishing.push_back(t);
                finishing_q.push_back(&q);
            } else {
                still.push_back(t);
            }
        }
        s->active = still;
        s->stats.chunks += 1;
    }
    const size_t nr = reset_items.size(), ns = step_items.size(), nrs = reset_small.size(), nss = step_small.size();
    if (nr + ns + nrs + nss > 2 * s->max_items) {
        set_fatal(s, NX_E_INVAL, "work list larger than the server's capacity");
        return false;
    }
    // the new requests' accumulator clears, then the finished requests' result copies
    BlockCopy* hb = s->h_blocks[cur];
    size_t n_clear = 0, n_copy = 0;
    uint64_t max_clear = 0, max_copy = 0;
    for (const SReq* qp : fresh_q) {
        const SReq& q = *qp;
        hb[n_clear++] = BlockCopy{nullptr, s->d_pool + q.dev_off + q.lay.returns, (uint64_t)(q.lay.obs - q.lay.returns)};
        max_clear = std::max<uint64_t>(max_clear, q.lay.obs - q.lay.returns);
    }
    if (s->h_pool_dev)
        for (const SReq* qp : finishing_q) {
            const SReq& q = *qp;
            hb[n_clear + n_copy++] = BlockCopy{s->d_pool + q.dev_off + q.lay.returns, s->h_pool_dev + q.host_off,
                                               (uint64_t)q.lay.tail};
            max_copy = std::max<uint64_t>(max_copy, q.lay.tail);
        }
    if (n_clear + n_copy)
        SRV_CK(cudaMemcpyAsync(s->d_blocks + (size_t)cur * 2 * s->max_slots, hb, (n_clear + n_copy) * sizeof(BlockCopy),
                               cudaMemcpyHostToDevice, s->stream),
               "block list upload");
    memcpy(hi, reset_items.data(), nr * sizeof(nx_item));
    memcpy(hi + nr, step_items.data(), ns * sizeof(nx_item));
    memcpy(hi + nr + ns, reset_small.data(), nrs * sizeof(nx_item));
    memcpy(hi + nr + ns + nrs, step_small.data(), nss * sizeof(nx_item));
    nx_item* di = s->d_items + (size_t)cur * 2 * s->max_items;
    SRV_CK(cudaMemcpyAsync(di, hi, (nr + ns + nrs + nss) * sizeof(nx_item), cudaMemcpyHostToDevice, s->stream),
           "item upload");
    SRV_CK(cudaMemcpyAsync(s->d_reqs, hr, sizeof(nx_req) * (size_t)s->max_slots, cudaMemcpyHostToDevice, s->stream),
           "record upload");
    nx_kparams p;
    memset(&p, 0, sizeof p);
    p.agents = (nx_agent*)s->d_pool;
    p.grids = s->d_pool;
    p.reqs = s->d_reqs;
    p.ctl = s->d_ctl;
    p.cell_stride = s->cell_stride;
    p.envs_per_cta = s->shape.envs_per_cta;
    p.phases = s->shape.phases;
    // launches whose requests want no digest run the lean kernel (random
    // actions, no action output, the server's Markov reward, any family)
    auto shape_of = [&](bool small, bool digest, int n, int* grid) {
        nx_launch_shape sh = small ? s->small : s->shape;
        int per_sm = small ? s->per_sm_small : s->per_sm;
        const int per_sm_lean = small ? s->per_sm_small_lean : s->per_sm_lean;
        if (!digest && per_sm_lean > 0) {
            sh.lean_family = NX_N_FAMILIES;
            per_sm = per_sm_lean;
        }
        *grid = std::min(n, per_sm * s->sm_count);
        return sh;
    };
    int grid = 0;
    if (!launch_blocks(s, cur, 0, n_clear, max_clear)) return false;  // the new requests' accumulators
    if (nrs + nss) {
        // the small requests' launches on the side stream, after the uploads
        SRV_CK(cudaEventRecord(s->fork_ev, s->stream), "fork");
        SRV_CK(cudaStreamWaitEvent(s->side, s->fork_ev, 0), "fork");
        nx_kparams ps = p;
        ps.cell_stride = s->cell_stride_small;
        ps.envs_per_cta = s->small.envs_per_cta;
        ps.phases = s->small.phases;
        if (nrs) {
            ps.items = di + nr + ns;
            ps.n_items = (int)nrs;
            ps.reset_all = 1;
            ps.launch_steps = 0;
            const nx_launch_shape sh = shape_of(true, digest_reset_s, (int)nrs, &grid);
            int rc = nx_launch_step_kernel(sh, ps, grid, s->side);
            if (rc) SRV_CK((cudaError_t)rc, "reset launch");
        }
        if (nss) {
            ps.items = di + nr + ns + nrs;
            ps.n_items = (int)nss;
            ps.reset_all = 0;
            ps.launch_steps = launch_steps;
            const nx_launch_shape sh = shape_of(true, digest_step_s, (int)nss, &grid);
            int rc = nx_launch_step_kernel(sh, ps, grid, s->side);
            if (rc) SRV_CK((cudaError_t)rc, "step launch");
        }
        SRV_CK(cudaEventRecord(s->join_ev, s->side), "join");
    }
    if (nr) {
        p.items = di;
        p.n_items = (int)nr;
        p.reset_all = 1;
        p.launch_steps = 0;
        const nx_launch_shape sh = shape_of(false, digest_reset, (int)nr, &grid);
        int rc = nx_launch_step_kernel(sh, p, grid, s->stream);
        if (rc) SRV_CK((cudaError_t)rc, "reset launch");
    }
    if (ns) {
        p.items = di + nr;
        p.n_items = (int)ns;
        p.reset_all = 0;
        p.launch_steps = launch_steps;
        const nx_launch_shape sh = shape_of(false, digest_step, (int)ns, &grid);
        int rc = nx_launch_step_kernel(sh, p, grid, s->stream);
        if (rc) SRV_CK((cudaError_t)rc, "step launch");
    }
    if (nrs + nss) SRV_CK(cudaStreamWaitEvent(s->stream, s->join_ev, 0), "join");
    // the results of the requests this chunk finishes (withdrawn ones copy
    // nothing back), into the pinned staging
    if (s->h_pool_dev) {
        if (!launch_blocks(s, cur, n_clear, n_copy, max_copy)) return false;
    } else {
        for (const SReq* qp : finishing_q) {
            const SReq& q = *qp;
            SRV_CK(cudaMemcpyAsync(s->h_pool + q.host_off, s->d_pool + q.dev_off + q.lay.returns, q.lay.tail,
                                   cudaMemcpyDeviceToHost, s->stream),
                   "result copy");
        }
    }
    SRV_CK(cudaEventRecord(c.ev, s->stream), "chunk event");
    c.finishing = finishing;
    c.valid = true;
    cur ^= 1;
    // the previous chunk finishes while this one is queued behind it
    return wait_chunk(s, s->chunks[cur]);
}

void worker_main(nx_server* s)
{
    int cur = 0;
    if (cudaSetDevice(s->device) != cudaSuccess) set_fatal(s, NX_E_CUDA, "worker cannot select the device");
    for (;;) {
        bool idle = false;
        bool ok = iterate(s, cur, &idle);
        std::unique_lock<std::mutex> lk(s->mu);
        if (!ok || s->fatal != NX_OK) break;
        if (s->stop && s->active.empty()) break;
        if (idle) s->cv_work.wait_for(lk, std::chrono::milliseconds(2), [&] { return s->stop || !s->waiting.empty(); });
    }
    // drain what is in flight, then fail whatever cannot finish
    wait_chunk(s, s->chunks[0]);
    wait_chunk(s, s->chunks[1]);
    std::lock_guard<std::mutex> lk(s->mu);
    const nx_status st = s->fatal != NX_OK ? s->fatal : NX_E_STATE;
    for (auto& kv : s->reqs) {
        if (!kv.second.finished) {
            kv.second.finished = true;
            kv.second.res.status = st;
            kv.second.res.t_done = now_s();
        }
    }
    s->waiting.clear();
    s->active.clear();
    s->cv_done.notify_all();
}

}  // namespace

nx_status nx_server_create(nx_server** out, size_t budget, const nx_options* opts, void* cuda_stream)
{
    if (!out) return nx_fail(nullptr, NX_E_INVAL, "server pointer is NULL");
    *out = nullptr;
    nx_options o;
    if (opts)
        o = *opts;
    else
        nx_options_default(&o);
    if (budget < (1u << 20) || budget > ((size_t)1 << 40)) return nx_fail(nullptr, NX_E_INVAL, "budget must be 1 MiB..1 TiB");
    if (o.obs_flags != NX_OBS_SYM) return nx_fail(nullptr, NX_E_INVAL, "the server produces symbolic observations only");
    if (o.steps_per_launch <= 0) o.steps_per_launch = 128;
    if (o.steps_per_launch > 1024) return nx_fail(nullptr, NX_E_INVAL, "steps_per_launch must be <= 1024");
    if (o.n_balls < 0 || o.n_balls > NX_MAX_BALLS) return nx_fail(nullptr, NX_E_INVAL, "n_balls must be in 0..4");
    nx_server* s = new (std::nothrow) nx_server();
    if (!s) return nx_fail(nullptr, NX_E_NOMEM, "host allocation failed");
    s->opt = o;
    s->stream = (cudaStream_t)cuda_stream;
    s->budget = budget;
    s->chunk = o.steps_per_launch;
    if (o.group_lanes) s->shape = nx_launch_shape{o.group_lanes, o.envs_per_cta, 0, o.staging == NX_STAGE_FULL ? 1 : 2};
    if (!nx_shape_supported(s->shape)) {
        delete s;
        return nx_fail(nullptr, NX_E_INVAL, "unsupported launch shape");
    }
    s->cell_stride = nx_slot_stride(s->shape, NX_MAX_SIZE);
    int dev = 0, err = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return nx_fail(nullptr, NX_E_CUDA, "no CUDA device available");
    }
    s->device = dev;
    s->per_sm = nx_kernel_max_ctas(s->shape, NX_MAX_SIZE, &err);
    if (err || s->per_sm < 1) {
        delete s;
        return nx_fail(nullptr, NX_E_CUDA, "occupancy query failed");
    }
    {
        nx_launch_shape ls = s->shape;
        ls.lean_family = NX_N_FAMILIES;
        if (nx_lean_supported(ls) && o.reward_mode == NX_REWARD_MARKOV) {
            int lerr = 0;
            const int n = nx_kernel_max_ctas(ls, NX_MAX_SIZE, &lerr);
            if (lerr) cudaGetLastError();
            s->per_sm_lean = (!lerr && n >= 1) ? n : 0;  // else every chunk runs the general kernel
        }
    }
    if (!o.group_lanes) {
        // the small requests' shape, on its own stream (none if it cannot run)
        int serr = 0;
        s->cell_stride_small = nx_slot_stride(s->small, NX_MAX_SIZE);
        s->per_sm_small = nx_kernel_max_ctas(s->small, NX_MAX_SIZE, &serr);
        if (!serr && s->per_sm_small >= 1) {
            nx_launch_shape ls = s->small;
            ls.lean_family = NX_N_FAMILIES;
            if (o.reward_mode == NX_REWARD_MARKOV) {
                const int n = nx_kernel_max_ctas(ls, NX_MAX_SIZE, &serr);
                s->per_sm_small_lean = (!serr && n >= 1) ? n : 0;
                serr = 0;
            }
        }
        if (!serr && s->per_sm_small >= 1 &&
            cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&s->fork_ev, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&s->join_ev, cudaEventDisableTiming) == cudaSuccess)
            s->small_envs = 64;
        cudaGetLastError();
    }
    // the smallest request (1 env of 5x5) needs about 1.8 KB: bound the work list by that
    s->max_items = std::min<size_t>(budget / 1536 + 1, (size_t)1 << 20);
    // pinned result staging (returns, digests, episodes, final views: 163
    // bytes per env in flight), at most 1 GiB whatever the budget
    const size_t host_cap = std::min(budget / 4, (size_t)1 << 30) + (1u << 20);
    cudaError_t e = cudaMalloc(&s->d_pool, budget);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_reqs, sizeof(nx_req) * (size_t)s->max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_items, sizeof(nx_item) * s->max_items * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_ctl, sizeof(nx_ctl));
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_pool, host_cap);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_blocks, sizeof(BlockCopy) * 2 * (size_t)s->max_slots * 2);
    if (e == cudaSuccess && cudaHostGetDevicePointer((void**)&s->h_pool_dev, s->h_pool, 0) != cudaSuccess) {
        cudaGetLastError();  // no device mapping of pinned memory: one copy per finished request
        s->h_pool_dev = nullptr;
    }
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaMallocHost(&s->h_reqs[b], sizeof(nx_req) * (size_t)s->max_slots);
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_items[b], sizeof(nx_item) * 2 * s->max_items);
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_blocks[b], sizeof(BlockCopy) * 2 * (size_t)s->max_slots);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->chunks[b].ev, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_ctl, 0, sizeof(nx_ctl), s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        std::string m = std::string("server setup: ") + cudaGetErrorString(e);
        nx_server_destroy(s);
        return nx_fail(nullptr, e == cudaErrorMemoryAllocation ? NX_E_NOMEM : NX_E_CUDA, m);
    }
    for (int b = 0; b < 2; ++b) memset(s->h_reqs[b], 0, sizeof(nx_req) * (size_t)s->max_slots);
    s->dev_alloc.init(budget);
    s->host_alloc.init(host_cap);
    for (int i = s->max_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->stats.budget_bytes = budget;
    s->worker = std::thread(worker_main, s);
    *out = s;
    return NX_OK;
}

nx_status nx_submit(nx_server* s, const nx_request* r, uint64_t* ticket)
{
    if (!s || !r || !ticket) return nx_fail(nullptr, NX_E_INVAL, "NULL argument");
    if (r->family < NX_EMPTY || r->family >= NX_N_FAMILIES || r->size < NX_MIN_SIZE || r->size > NX_MAX_SIZE ||
        r->n_envs < 1 || r->horizon < 1 || r->variant < 0 || r->variant > nx_max_variant(r->family, r->size) ||
        (r->flags & ~NX_REQ_DIGEST) != 0)
        return nx_fail(nullptr, NX_E_INVAL,
                       "request: known family, size 5..19, n_envs >= 1, horizon >= 1, variant <= nx_max_variant, "
                       "flags NX_REQ_DIGEST or 0");
    SReq q;
    q.r = *r;
    q.max_steps = nx_default_max_steps(r->family, r->size);
    q.lay = Layout::of(r->n_envs, r->size);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal != NX_OK) return nx_fail(nullptr, s->fatal, s->fatal_msg);
    if (s->stop) return nx_fail(nullptr, NX_E_STATE, "server is shutting down");
    if (up256(q.lay.total) > s->budget || up256(q.lay.tail) > s->host_alloc.cap ||
        (size_t)((r->n_envs + shape_of_req(s, *r).envs_per_cta - 1) / shape_of_req(s, *r).envs_per_cta) * 2 >
            s->max_items) {
        s->stats.rejected += 1;
        return nx_fail(nullptr, NX_E_BUDGET, "request needs " + std::to_string(q.lay.total) +
                                                 " bytes, more than the whole budget of " + std::to_string(s->budget));
    }
    const uint64_t t = s->next_ticket++;
    q.res.status = NX_PENDING;
    q.res.t_submit = now_s();
    s->reqs.emplace(t, q);
    s->waiting.push_back(t);
    s->stats.submitted += 1;
    *ticket = t;
    s->cv_work.notify_one();
    return NX_OK;
}

nx_status nx_poll(nx_server* s, uint64_t ticket, nx_result* res)
{
    if (!s) return nx_fail(nullptr, NX_E_INVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return nx_fail(nullptr, NX_E_INVAL, "unknown ticket");
    if (!it->second.finished) return NX_PENDING;
    if (res) *res = it->second.res;
    return it->second.res.status == NX_OK ? NX_OK : it->second.res.status;
}

nx_status nx_wait(nx_server* s, uint64_t ticket, nx_result* res, double timeout_s)
{
    if (!s) return nx_fail(nullptr, NX_E_INVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return nx_fail(nullptr, NX_E_INVAL, "unknown ticket");
    // an element's address survives insertions (an iterator may not), and the
    // lock is released while waiting
    const SReq* q = &it->second;
    auto done = [&] { return q->finished; };
    if (timeout_s > 0) {
        if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done))
            return nx_fail(nullptr, NX_E_TIMEOUT, "request did not finish in time");
    } else {
        s->cv_done.wait(lk, done);
    }
    if (res) *res = q->res;
    return q->res.status;
}

nx_status nx_cancel(nx_server* s, uint64_t ticket)
{
    if (!s) return nx_fail(nullptr, NX_E_INVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return nx_fail(nullptr, NX_E_INVAL, "unknown ticket");
    SReq& q = it->second;
    if (q.finished || q.cancel || (q.admitted && q.launched >= q.r.horizon))
        return nx_fail(nullptr, NX_E_STATE, "the request has finished or its last chunk is on the GPU");
    if (!q.admitted) {
        // still queued: nothing of it ever reached the GPU
        s->waiting.erase(std::find(s->waiting.begin(), s->waiting.end(), ticket));
        q.finished = true;
        q.res.status = NX_E_CANCELED;
        q.res.t_done = now_s();
        s->stats.canceled += 1;
        s->cv_done.notify_all();
        s->cv_work.notify_one();
        return NX_OK;
    }
    q.cancel = true;
    return NX_OK;
}

nx_status nx_server_get_stats(nx_server* s, nx_server_stats* st)
{
    if (!s || !st) return nx_fail(nullptr, NX_E_INVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->stats;
    if (s->busy_since >= 0) st->busy_s += now_s() - s->busy_since;
    return NX_OK;
}

void nx_server_destroy(nx_server* s)
{
    if (!s) return;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
            // queued requests are dropped; admitted ones finish
            for (uint64_t t : s->waiting) {
                s->reqs.at(t).finished = true;
                s->reqs.at(t).res.status = NX_E_STATE;
            }
            s->waiting.clear();
        }
        s->cv_work.notify_all();
        s->worker.join();
    }
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->side) cudaStreamSynchronize(s->side);
    if (s->side) cudaStreamDestroy(s->side);
    if (s->fork_ev) cudaEventDestroy(s->fork_ev);
    if (s->join_ev) cudaEventDestroy(s->join_ev);
    for (int b = 0; b < 2; ++b) {
        if (s->chunks[b].ev) cudaEventDestroy(s->chunks[b].ev);
        if (s->h_reqs[b]) cudaFreeHost(s->h_reqs[b]);
        if (s->h_items[b]) cudaFreeHost(s->h_items[b]);
        if (s->h_blocks[b]) cudaFreeHost(s->h_blocks[b]);
    }
    if (s->h_pool) cudaFreeHost(s->h_pool);
    if (s->d_pool) cudaFree(s->d_pool);
    if (s->d_reqs) cudaFree(s->d_reqs);
    if (s->d_items) cudaFree(s->d_items);
    if (s->d_blocks) cudaFree(s->d_blocks);
    if (s->d_ctl) cudaFree(s->d_ctl);
    delete s;
}
