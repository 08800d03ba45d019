// nx_device.cuh -- device-side building blocks of the fused MiniGrid step
// (NAVIX, arXiv 2407.19396): counter-based draws, packed cells, the family
// layout generators, the intervention/transition rules and the egocentric
// view with occlusion.  Every function works for a *group* of G lanes
// (G = 1, 2, 4, 8, 16 or 32) that owns one environment: cell-parallel work
// is split over the lanes, per-env scalar work is repeated by every lane
// (so no broadcast is needed), and shared-memory writes are done by lane 0
// followed by a group barrier.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "navixgb.h"
#include "nx_internal.h"

namespace nxd {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), word 0 only.  Ten
// rounds: two 32x32 multiplications (0xD2511F53 on word 0, 0xCD9E8D57 on
// word 2), the high halves mixed with the other words and the key; the key is
// advanced by the Weyl constants after each round.
__device__ __forceinline__ uint32_t philox_word0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                 uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c0;
}

enum { PURPOSE_LAYOUT = 1u, PURPOSE_BALL = 2u, PURPOSE_ACTION = 3u, PURPOSE_EXPLORE = 4u };

__device__ __forceinline__ uint32_t draw(uint64_t seed, uint32_t env, uint32_t episode, uint32_t step,
                                         uint32_t purpose, uint32_t k)
{
    return philox_word0(env, episode, step, (purpose << 24) | k, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// bounded draw in [0, n): (x * n) >> 32
__device__ __forceinline__ int bounded(uint32_t x, uint32_t n) { return (int)__umulhi(x, n); }

// ---------------------------------------------------------------------------
// Packed cell code (one byte in shared memory): bits 0-2 colour, bits 3-6
// kind, bit 7 set when the cell blocks sight.  The kind is the entity code
// except for doors: 4 open, 11 closed, 12 locked.
enum : uint32_t {
    K_EMPTY = 1, K_WALL = 2, K_FLOOR = 3, K_DOOR_OPEN = 4, K_KEY = 5, K_BALL = 6, K_BOX = 7, K_GOAL = 8,
    K_LAVA = 9, K_DOOR_CLOSED = 11, K_DOOR_LOCKED = 12
};
constexpr uint32_t OPAQUE = 0x80u;
__host__ __device__ constexpr uint32_t make_code(uint32_t kind, uint32_t col)
{
    return (kind << 3) | (col & 7u) | ((kind == K_WALL || kind >= K_DOOR_CLOSED) ? OPAQUE : 0u);
}
enum : uint32_t {
    C_EMPTY = make_code(K_EMPTY, 0),
    C_WALL = make_code(K_WALL, 5),
    C_GOAL = make_code(K_GOAL, 1),
    C_LAVA = make_code(K_LAVA, 0),
    C_BALL_BLUE = make_code(K_BALL, 2),
    C_KEY_YELLOW = make_code(K_KEY, 4),
    C_DOOR_LOCKED_YELLOW = make_code(K_DOOR_LOCKED, 4)
};
// kinds the agent can enter: empty, floor, open door, goal, lava
#define NX_WALKABLE_KINDS ((1u << 1) | (1u << 3) | (1u << 4) | (1u << 8) | (1u << 9))

__device__ __forceinline__ uint32_t pack_cell(uint32_t ent, uint32_t col, uint32_t st)
{
    uint32_t kind = ent & 15u;
    if (ent == 4u) kind = st == 0u ? K_DOOR_OPEN : (st == 1u ? K_DOOR_CLOSED : K_DOOR_LOCKED);
    return make_code(kind, col);
}
__device__ __forceinline__ uint32_t cell_kind(uint32_t code) { return (code >> 3) & 15u; }
__device__ __forceinline__ uint32_t cell_col(uint32_t code) { return code & 7u; }
__device__ __forceinline__ uint32_t cell_ent(uint32_t code)
{
    const uint32_t k = cell_kind(code);
    return k >= 11u ? 4u : k;
}
__device__ __forceinline__ uint32_t cell_st(uint32_t code)
{
    const uint32_t k = cell_kind(code);
    return k >= 11u ? k - 10u : 0u;
}
__device__ __forceinline__ bool walkable(uint32_t code) { return (NX_WALKABLE_KINDS >> cell_kind(code)) & 1u; }
// the observation triple (ent | col << 8 | st << 16) of a code
__device__ __forceinline__ uint32_t cell_triple(uint32_t code)
{
    return cell_ent(code) | (cell_col(code) << 8) | (cell_st(code) << 16);
}

// ---------------------------------------------------------------------------
// A group of G lanes of one warp owning one environment.
template <int G>
struct Grp {
    int lane;       // 0..G-1
    int base;       // first lane of the group within the warp
    unsigned mask;  // the group's lanes
    __device__ __forceinline__ explicit Grp(int tid)
    {
        lane = tid % G;
        base = (tid & 31) - lane;
        mask = G == 32 ? 0xFFFFFFFFu : (((1u << G) - 1u) << base);
    }
    __device__ __forceinline__ uint32_t ballot(bool p) const
    {
        if (G == 1) return p ? 1u : 0u;
        const uint32_t b = __ballot_sync(mask, p);
        return G == 32 ? b : (b >> base) & ((1u << G) - 1u);
    }
    template <class T>
    __device__ __forceinline__ T shfl(T v, int src) const
    {
        if (G == 1) return v;
        return __shfl_sync(mask, v, base + src);
    }
    __device__ __forceinline__ void sync() const
    {
        if (G > 1) __syncwarp(mask);
    }
};

// Draws k = 0..n-1 (n <= 8) of one counter family, computed in parallel over
// the group's lanes and shared with every lane.
template <int G, class F>
__device__ __forceinline__ void group_draws(const Grp<G>& grp, int n, uint32_t (&d)[8], F counter_draw)
{
#pragma unroll
    for (int k0 = 0; k0 < 8; k0 += G) {
        if (k0 < n) {
            const int k = k0 + grp.lane;
            const uint32_t v = k < n ? counter_draw((uint32_t)k) : 0u;
#pragma unroll
            for (int j = 0; j < G && k0 + j < 8; ++j) d[k0 + j] = grp.shfl(v, j);
        }
    }
}

// Position of the (k+1)-th set bit of b (k < popc(b)): halving search on
// the bit counts of the low halves.
__device__ __forceinline__ int nth_set_bit(uint32_t b, int k)
{
    int pos = 0;
#pragma unroll
    for (int sh = 16; sh >= 1; sh >>= 1) {
        const int c = __popc(b & ((1u << sh) - 1u));
        const bool up = k >= c;
        k -= up ? c : 0;
        b = up ? (b >> sh) : b;
        pos += up ? sh : 0;
    }
    return pos;
}

// Number of empty cells in the rectangle [x0,x1] x [y0,y1] not counting cell
// index `skip` (-1 for none).
template <int G>
__device__ int count_free(const Grp<G>& grp, const uint8_t* g, int W, int x0, int x1, int y0, int y1, int skip)
{
    // lane l visits rectangle positions r = l, l + G, ..; its column and row
    // advance by G mod w and G / w per round (one wrap at most), no division
    const int w = x1 - x0 + 1, n = w * (y1 - y0 + 1);
    const int dy = G / w, dx = G - dy * w;
    int ry = grp.lane / w, rx = grp.lane - ry * w;
    int total = 0;
    for (int r0 = 0; r0 < n; r0 += G) {
        const bool in = r0 + grp.lane < n;
        const int ci = in ? (y0 + ry) * W + x0 + rx : 0;  // lanes past the end read cell 0
        const bool f = in && g[ci] == C_EMPTY && ci != skip;
        total += __popc(grp.ballot(f));
        rx += dx;
        ry += dy;
        if (rx >= w) {
            rx -= w;
            ry += 1;
        }
    }
    return total;
}

// Cell index of the k-th empty cell of the rectangle in row-major order (y
// outer, x inner), not counting `skip`; -1 if there is none.
template <int G>
__device__ int kth_free(const Grp<G>& grp, const uint8_t* g, int W, int x0, int x1, int y0, int y1, int skip, int k)
{
    const int w = x1 - x0 + 1, n = w * (y1 - y0 + 1);
    const int dy = G / w, dx = G - dy * w;
    int ry = grp.lane / w, rx = grp.lane - ry * w;
    for (int r0 = 0; r0 < n; r0 += G) {
        const bool in = r0 + grp.lane < n;
        const int ci = in ? (y0 + ry) * W + x0 + rx : 0;  // lanes past the end read cell 0
        const bool f = in && g[ci] == C_EMPTY && ci != skip;
        const uint32_t b = grp.ballot(f);
        const int cnt = __popc(b);
        if (k < cnt) return grp.shfl(ci, nth_set_bit(b, k));
        k -= cnt;
        rx += dx;
        ry += dy;
        if (rx >= w) {
            rx -= w;
            ry += 1;
        }
    }
    return -1;
}

// The k-th free interior cell of a FourRooms-S grid (reading R18, rows
// outer) before its goal is placed, in closed form: the walls x = m and
// y = m (m = S / 2) leave S - 3 cells in every other interior row, plus the
// gap (m, gy0) in the upper half and (m, gy1) in the lower one; row m holds
// only its gaps (gx2, m) and (gx3, m).  Returns x | y << 8.
__device__ __forceinline__ uint32_t fourrooms_kth(int S, int m, int gy0, int gy1, int gx2, int gx3, int k)
{
    const int w = S - 3;                 // cells of a row without a gap
    const int upper = (m - 1) * w + 1;   // cells of rows 1 .. m-1 (one gap)
    int y0 = 1, gy = gy0;                // the half holding k: first row, gap row
    if (k >= upper + 2) {
        k -= upper + 2;
        y0 = m + 1;
        gy = gy1;
    } else if (k >= upper) {
        return (uint32_t)(k == upper ? gx2 : gx3) | ((uint32_t)m << 8);
    }
    const int before = (gy - y0) * w;    // cells of the half's rows above its gap row
    if (k >= before && k < before + w + 1)  // the gap row: x = 1 .. S-2 without a hole
        return (uint32_t)(1 + k - before) | ((uint32_t)gy << 8);
    const int kk = k < before ? k : k - 1;  // (past the gap row, one cell fewer per row index)
    const int r = kk / w, j = kk - r * w;
    const int x = j < m - 1 ? 1 + j : j + 2;  // skip the wall column x = m
    return (uint32_t)x | ((uint32_t)(y0 + r) << 8);
}

// ---------------------------------------------------------------------------
// Per-env registers (every lane of the group holds the same copy).
struct AgentReg {
    int x, y, dir;
    uint32_t carry;  // packed code of the carried object, 0 = nothing
    int done, invalid, t;
    uint32_t episode;
    uint32_t mission;  // GoToDoor target colour, NX_NO_MISSION otherwise
    int nb;
    uint32_t bxp, byp;  // ball b's column / row in byte b (two registers for the four balls)
};

__device__ __forceinline__ int ball_x(const AgentReg& a, int b) { return (int)((a.bxp >> (8 * b)) & 0xFFu); }
__device__ __forceinline__ int ball_y(const AgentReg& a, int b) { return (int)((a.byp >> (8 * b)) & 0xFFu); }
__device__ __forceinline__ void set_ball(AgentReg& a, int b, int x, int y)
{
    const uint32_t m = ~(0xFFu << (8 * b));
    a.bxp = (a.bxp & m) | ((uint32_t)x << (8 * b));
    a.byp = (a.byp & m) | ((uint32_t)y << (8 * b));
}

__device__ __forceinline__ void load_agent(const nx_agent* src, AgentReg& a)
{
    const uint4 w0 = reinterpret_cast<const uint4*>(src)[0];
    const uint4 w1 = reinterpret_cast<const uint4*>(src)[1];
    a.x = w0.x & 0xFF;
    a.y = (w0.x >> 8) & 0xFF;
    a.dir = (w0.x >> 16) & 0xFF;
    const uint32_t ce = w0.x >> 24, cc = w0.y & 0xFF;
    a.carry = ce ? pack_cell(ce, cc, 0) : 0u;
    a.done = (w0.y >> 8) & 0xFF;
    a.invalid = (w0.y >> 16) & 0xFF;
    a.nb = (w0.y >> 24) & 0xFF;
    a.t = w0.z & 0xFFFF;
    a.episode = w0.w;
    a.mission = (w1.z >> 16) & 0xFF;
    a.bxp = w1.x;
    a.byp = w1.y;
}

// Writes the agent block; the descriptor fields (max_steps, family, size,
// grid offset) are rewritten from the item so the block stays self-describing.
__device__ __forceinline__ void store_agent(nx_agent* dst, const AgentReg& a, const nx_item& it, uint32_t grid_offset)
{
    uint4 w0, w1;
    const uint32_t ce = a.carry ? cell_ent(a.carry) : 0u, cc = a.carry ? cell_col(a.carry) : 0u;
    w0.x = (uint32_t)a.x | ((uint32_t)a.y << 8) | ((uint32_t)a.dir << 16) | (ce << 24);
    w0.y = cc | ((uint32_t)a.done << 8) | ((uint32_t)a.invalid << 16) | ((uint32_t)a.nb << 24);
    w0.z = (uint32_t)a.t | ((uint32_t)it.max_steps << 16);
    w0.w = a.episode;
    w1.x = a.bxp;
    w1.y = a.byp;
    w1.z = (uint32_t)it.family | ((uint32_t)it.size << 8) | (a.mission << 16);
    w1.w = grid_offset;
    reinterpret_cast<uint4*>(dst)[0] = w0;
    reinterpret_cast<uint4*>(dst)[1] = w1;
}

// Whether every index a step derives from the agent block stays inside an
// S x S grid: the agent's cell and direction, and each ball's cell, which
// lies in the interior (1..S-2), so that its whole 8-neighbourhood is in the
// grid.  Blocks written by the kernels and by nx_set_state (which validates
// the same) always pass; the step kernel checks each block it loads, so that
// a block corrupted in device memory can never make a step index outside
// its env's grid.
__device__ __forceinline__ bool agent_in_range(const AgentReg& a, int S)
{
    bool ok = (unsigned)a.x < (unsigned)S && (unsigned)a.y < (unsigned)S && (unsigned)a.dir < 4u && (unsigned)a.nb <= 4u;
#pragma unroll
    for (int b = 0; b < 4; ++b)
        ok = ok && (b >= a.nb || ((unsigned)(ball_x(a, b) - 1) < (unsigned)(S - 2) &&
                                  (unsigned)(ball_y(a, b) - 1) < (unsigned)(S - 2)));
    return ok;
}

// Device checks of the NX_DEBUG build (explicit bounds tests before grid
// writes and output stores; a failed test sets NX_FLAG_BOUNDS, which nx_sync
// reports as NX_E_DEVICE_CHECK, and skips the access -- nothing traps).  The
// release build compiles them out.
#ifdef NX_DEBUG
#define NX_DCHECK(ctl, cond) ((cond) ? true : (atomicOr(&(ctl)->flags, (unsigned)NX_FLAG_BOUNDS), false))
#else
#define NX_DCHECK(ctl, cond) true
#endif

// L7 crossings: N rivers of lava or wall (see reset_layout), kept out of line
// to hold down the step kernel's registers.  Its shuffles run on registers:
// an array indexed by a loop counter would sit in local memory and be charged
// to the calling kernel's stack frame.
template <int G>
__device__ __noinline__ void crossing_layout(const Grp<G>& grp, uint8_t* g, int S, int W, int family, int variant,
                                             uint64_t seed, uint32_t key_env, uint32_t episode)
{
    const int HW = S * S;
    // rivers: a partial Fisher-Yates choice among rows then columns 2, 4, ..
    // S-3 (at most 16 candidates for S <= 19), one byte each in two 64-bit
    // words: the row y for a horizontal river, 0x80 | x for a vertical one;
    // the choice is kept as row/column bitmasks, so their sorted order is the
    // bit order
    uint64_t ck[2] = {0ull, 0ull};  // constant indexes only after unrolling
    auto get = [&](int i) -> uint32_t {
        const uint64_t w = i < 8 ? ck[0] : ck[1];
        return (uint32_t)(w >> (8 * (i & 7))) & 0xFFu;
    };
    auto put = [&](int i, uint32_t v) {
        const int sh = 8 * (i & 7);
        const uint64_t cleared = ((i < 8 ? ck[0] : ck[1]) & ~(0xFFull << sh)) | ((uint64_t)v << sh);
        if (i < 8)
            ck[0] = cleared;
        else
            ck[1] = cleared;
    };
    int m = 0;
    for (int y = 2; y <= S - 3; y += 2) put(m++, (uint32_t)y);           // horizontal: the row
    for (int x = 2; x <= S - 3; x += 2) put(m++, 0x80u | (uint32_t)x);   // vertical: 0x80 | the column
    uint32_t k = 0;
    for (int i = 0; i < variant; ++i) {
        const int j = i + bounded(draw(seed, key_env, episode, 0u, PURPOSE_LAYOUT, k++), (uint32_t)(m - i));
        const uint32_t ti = get(i), tj = get(j);
        put(i, tj);
        put(j, ti);
    }
    uint32_t hmask = 0, vmask = 0;
    for (int i = 0; i < variant; ++i) {
        const uint32_t c = get(i);
        if (c & 0x80u)
            vmask |= 1u << (c & 0x7Fu);
        else
            hmask |= 1u << c;
    }
    const uint32_t obst = family == NX_LAVA_CROSSING ? (uint32_t)C_LAVA : (uint32_t)C_WALL;
    grp.sync();
    for (int c = grp.lane; c < HW; c += G) {
        const int y = c / S, x = c - y * S;
        if (x >= 1 && y >= 1 && x <= S - 2 && y <= S - 2 && (((hmask >> y) | (vmask >> x)) & 1u))
            g[y * W + x] = (uint8_t)obst;
    }
    // order of crossings: east moves (vertical rivers) first, then south
    // moves, shuffled by Fisher-Yates from the last position down; bit i of
    // `east` is set when move i goes east
    const int nv = __popc(vmask), nh = __popc(hmask), L = nv + nh;
    uint32_t east = (1u << nv) - 1u;
    for (int i = L - 1; i >= 1; --i) {
        const int j = bounded(draw(seed, key_env, episode, 0u, PURPOSE_LAYOUT, k++), (uint32_t)(i + 1));
        if (((east >> i) ^ (east >> j)) & 1u) east ^= (1u << i) | (1u << j);
    }
    // walk the rooms from the top-left one; each move opens one cell of
    // the river it crosses, drawn within the current room's span
    int x_lo = 0, y_lo = 0;                 // the current room's west / north bounds
    uint32_t vrest = vmask, hrest = hmask;  // rivers not yet crossed, east / south of the room
    grp.sync();
    for (int i = 0; i < L; ++i) {
        const int x_hi = vrest ? __ffs(vrest) - 1 : S - 1;
        const int y_hi = hrest ? __ffs(hrest) - 1 : S - 1;
        if ((east >> i) & 1u) {
            const int y = y_lo + 1 + bounded(draw(seed, key_env, episode, 0u, PURPOSE_LAYOUT, k++),
                                             (uint32_t)(y_hi - y_lo - 1));
            if (grp.lane == 0) g[y * W + x_hi] = (uint8_t)C_EMPTY;
            x_lo = x_hi;
            vrest &= vrest - 1u;
        } else {
            const int x = x_lo + 1 + bounded(draw(seed, key_env, episode, 0u, PURPOSE_LAYOUT, k++),
                                             (uint32_t)(x_hi - x_lo - 1));
            if (grp.lane == 0) g[y_hi * W + x] = (uint8_t)C_EMPTY;
            y_lo = y_hi;
            hrest &= hrest - 1u;
        }
    }
}

// L10 KeyCorridor S{s}R{R} (variant R - 1): a 3 x R block of rooms of side s
// sharing walls in the S x S grid, S = 3(s-1)+1; rows from H - 1 = (s-1)R on
// are wall (cells outside a grid read as wall, so views and rules are those
// of the H x S grid).  The middle column of rooms is one open corridor; each
// side room has a door in its corridor wall; the goal's room is locked and the
// key of its colour lies in a room on the other side.  Draw k: 0..2R-1 the
// door rows (left rooms top to bottom, then right), 2R..4R-1 their colours,
// then the goal's side and room row, the key's room row, the goal cell, the
// key cell and the agent's corridor cell and direction; the rooms and the
// corridor are empty when their cells are drawn, so the k-th free cell is a
// closed form (row-major).  Out of line like the crossings; returns the
// agent as x | y << 8 | dir << 16.
template <int G>
__device__ __noinline__ uint32_t keycorridor_layout(const Grp<G>& grp, uint8_t* g, int S, int W, int variant,
                                                    uint64_t seed, uint32_t key_env, uint32_t episode)
{
    const int s = (S - 1) / 3 + 1, R = variant + 1, H = (s - 1) * R + 1, xl = s - 1, xr = 2 * (s - 1), w = s - 2;
    auto dr = [&](int k) { return draw(seed, key_env, episode, 0u, PURPOSE_LAYOUT, (uint32_t)k); };
    for (int c = grp.lane; c < S * S; c += G) {
        const int y = c / S, x = c - y * S;
        bool wall = y >= H - 1 || y == 0 || x == 0 || x == S - 1 || x == xl || x == xr;
        if (y % (s - 1) == 0 && !(x > xl && x < xr)) wall = true;
        g[y * W + x] = (uint8_t)(wall ? C_WALL : C_EMPTY);
    }
    const int gside = bounded(dr(4 * R), 2u), grow = bounded(dr(4 * R + 1), (uint32_t)R);
    const int krow = bounded(dr(4 * R + 2), (uint32_t)R);
    grp.sync();
    for (int j = grp.lane; j < 2 * R; j += G) {  // door j: side j / R, room row j % R
        const int side = j >= R, row = j - side * R;
        const int y = row * (s - 1) + 1 + bounded(dr(j), (uint32_t)w);
        const uint32_t c = bounded(dr(2 * R + j), 6u);
        g[y * W + (side ? xr : xl)] = (uint8_t)make_code((side == gside && row == grow) ? K_DOOR_LOCKED : K_DOOR_CLOSED, c);
    }
    if (grp.lane == 0) {
        const uint32_t lock_col = bounded(dr(2 * R + gside * R + grow), 6u);
        const int gi = bounded(dr(4 * R + 3), (uint32_t)(w * w)), ki = bounded(dr(4 * R + 4), (uint32_t)(w * w));
        const int gx0 = gside == 0 ? 1 : xr + 1, kx0 = gside == 0 ? xr + 1 : 1;
        g[(grow * (s - 1) + 1 + gi / w) * W + gx0 + gi % w] = (uint8_t)C_GOAL;
        g[(krow * (s - 1) + 1 + ki / w) * W + kx0 + ki % w] = (uint8_t)make_code(K_KEY, lock_col);
    }
    const int ai = bounded(dr(4 * R + 5), (uint32_t)(w * (H - 2)));
    const int ax = xl + 1 + ai % w, ay = 1 + ai / w;
    return (uint32_t)ax | ((uint32_t)ay << 8) | ((uint32_t)bounded(dr(4 * R + 6), 4u) << 16);
}

// ---------------------------------------------------------------------------
// Layout generators of the Table 8 families.  Draw k of a reset is
// draw(seed, env, episode, 0, PURPOSE_LAYOUT, k); the k-th free cell is
// counted row-major; the agent is never stored in the grid.  Cell (x, y) is
// g[y W + x]: W = S for a packed grid, larger with a wall margin around it
// (the margin is never written).
// Returns false (and leaves a partial layout) only if a free-cell choice found
// no cell, which cannot happen for sizes 5..19; the caller raises a flag.
template <int G>
__device__ __forceinline__ bool reset_layout(const Grp<G>& grp, uint8_t* g, int S, int W, int family, int n_balls,
                                             int variant, uint64_t seed, uint32_t key_env, uint32_t episode, AgentReg& a)
{
    // empty cells (a packed grid four at a time: its slot is a whole number
    // of words at least S * S bytes long), then the four border lines of walls
    const int HW = S * S;
    constexpr uint32_t kEmpty4 = C_EMPTY * 0x01010101u;
    if (W == S) {
        for (int c4 = grp.lane; c4 < (HW + 3) / 4; c4 += G) reinterpret_cast<uint32_t*>(g)[c4] = kEmpty4;
    } else {
        for (int y = 0; y < S; ++y)
            for (int x = grp.lane; x < S; x += G) g[y * W + x] = (uint8_t)C_EMPTY;
    }
    grp.sync();
    for (int i = grp.lane; i < S; i += G) {
        g[i] = (uint8_t)C_WALL;
        g[(S - 1) * W + i] = (uint8_t)C_WALL;
        g[i * W] = (uint8_t)C_WALL;
        g[i * W + S - 1] = (uint8_t)C_WALL;
    }
    a.x = 1;
    a.y = 1;
    a.dir = 0;
    a.carry = 0;
    a.done = 0;
    a.t = 0;
    a.episode = episode;
    a.mission = NX_NO_MISSION;
    a.nb = 0;
    a.bxp = 0u;
    a.byp = 0u;
    uint32_t d[8];
    const int n_draws = family == NX_DOORKEY ? 5 : family == NX_FOURROOMS ? 7 : family == NX_LAVAGAP ? 2
                        : family == NX_EMPTY_RANDOM ? 2
                        : family == NX_GOTODOOR ? 8 : 0;
    group_draws(grp, n_draws, d,
                [&](uint32_t k) { return draw(seed, key_env, episode, 0u, PURPOSE_LAYOUT, k); });
    grp.sync();
    const int goal = family == NX_DISTSHIFT ? W + (S - 2) : (S - 2) * W + (S - 2);
    if (family != NX_FOURROOMS && family != NX_GOTODOOR && family != NX_KEYCORRIDOR) {
        if (grp.lane == 0) g[goal] = (uint8_t)C_GOAL;
    }
    if (family == NX_DOORKEY) {
        const int xw = 2 + bounded(d[0], (uint32_t)(S - 4));
        const int door_y = 1 + bounded(d[1], (uint32_t)(S - 3));
        for (int y = 1 + grp.lane; y <= S - 2; y += G)
            g[y * W + xw] = (uint8_t)(y == door_y ? C_DOOR_LOCKED_YELLOW : C_WALL);
        // the region left of the wall, x 1..xw-1 by y 1..S-2, is all empty:
        // its k-th cell row-major is (1 + k % w, 1 + k / w); the key's list
        // is the same without the agent's cell
        const int w = xw - 1, n = w * (S - 2);
        const int ka = bounded(d[2], (uint32_t)n);
        int kk = bounded(d[4], (uint32_t)(n - 1));
        kk += kk >= ka ? 1 : 0;
        const int ay = ka / w, ky = kk / w;
        a.x = 1 + ka - ay * w;
        a.y = 1 + ay;
        a.dir = bounded(d[3], 4u);
        grp.sync();
        if (grp.lane == 0) g[(1 + ky) * W + 1 + kk - ky * w] = (uint8_t)C_KEY_YELLOW;
    } else if (family == NX_FOURROOMS) {
        const int m = S / 2;
        for (int i = grp.lane; i < S; i += G) {
            g[i * W + m] = (uint8_t)C_WALL;
            g[m * W + i] = (uint8_t)C_WALL;
        }
        const int gy0 = 1 + bounded(d[0], (uint32_t)(m - 1)), gy1 = m + 1 + bounded(d[1], (uint32_t)(S - 2 - m));
        const int gx2 = 1 + bounded(d[2], (uint32_t)(m - 1)), gx3 = m + 1 + bounded(d[3], (uint32_t)(S - 2 - m));
        // goal and agent by the closed-form k-th free cell; the agent's list
        // is the same without the goal's cell
        const int n = (S - 3) * (S - 3) + 4;
        const int kg = bounded(d[4], (uint32_t)n);
        int ka = bounded(d[5], (uint32_t)(n - 1));
        ka += ka >= kg ? 1 : 0;
        const uint32_t gc = fourrooms_kth(S, m, gy0, gy1, gx2, gx3, kg);
        const uint32_t ac = fourrooms_kth(S, m, gy0, gy1, gx2, gx3, ka);
        grp.sync();
        if (grp.lane == 0) {
            g[gy0 * W + m] = (uint8_t)C_EMPTY;
            g[gy1 * W + m] = (uint8_t)C_EMPTY;
            g[m * W + gx2] = (uint8_t)C_EMPTY;
            g[m * W + gx3] = (uint8_t)C_EMPTY;
            g[(gc >> 8) * W + (gc & 0xFFu)] = (uint8_t)C_GOAL;
        }
        a.x = (int)(ac & 0xFFu);
        a.y = (int)(ac >> 8);
        a.dir = bounded(d[6], 4u);
    } else if (family == NX_LAVAGAP) {
        const int xl = 2 + bounded(d[0], (uint32_t)(S - 4));
        const int gap = 1 + bounded(d[1], (uint32_t)(S - 2));
        for (int y = 1 + grp.lane; y <= S - 2; y += G)
            if (y != gap) g[y * W + xl] = (uint8_t)C_LAVA;
    } else if (family == NX_EMPTY_RANDOM) {
        // the interior without the goal, its last cell row-major: the k-th
        // cell is (1 + k % (S-2), 1 + k / (S-2))
        const int w = S - 2, ka = bounded(d[0], (uint32_t)(w * w - 1)), ay = ka / w;
        a.x = 1 + ka - ay * w;
        a.y = 1 + ay;
        a.dir = bounded(d[1], 4u);
    } else if (family == NX_GOTODOOR) {
        // L8: one closed door on each wall (top, bottom, left, right) at drawn
        // positions 1..S-2; their colours are the first four of a partial
        // Fisher-Yates shuffle of the six colours (nibble i of perm holds the
        // colour at position i); draws 8..10 pick the target door, the agent's
        // interior cell (row-major; the interior is all empty) and direction
        uint32_t perm = 0x543210u;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int j = i + bounded(d[4 + i], (uint32_t)(6 - i));
            const uint32_t ci = (perm >> (4 * i)) & 15u, cj = (perm >> (4 * j)) & 15u;
            perm = (perm & ~((15u << (4 * i)) | (15u << (4 * j)))) | (cj << (4 * i)) | (ci << (4 * j));
        }
        if (grp.lane == 0) {
            g[1 + bounded(d[0], (uint32_t)(S - 2))] = (uint8_t)make_code(K_DOOR_CLOSED, perm & 15u);
            g[(S - 1) * W + 1 + bounded(d[1], (uint32_t)(S - 2))] = (uint8_t)make_code(K_DOOR_CLOSED, (perm >> 4) & 15u);
            g[(1 + bounded(d[2], (uint32_t)(S - 2))) * W] = (uint8_t)make_code(K_DOOR_CLOSED, (perm >> 8) & 15u);
            g[(1 + bounded(d[3], (uint32_t)(S - 2))) * W + S - 1] =
                (uint8_t)make_code(K_DOOR_CLOSED, (perm >> 12) & 15u);
        }
        group_draws(grp, 3, d,
                    [&](uint32_t k) { return draw(seed, key_env, episode, 0u, PURPOSE_LAYOUT, 8u + k); });
        a.mission = (perm >> (4 * bounded(d[0], 4u))) & 15u;
        const int w = S - 2, ac = bounded(d[1], (uint32_t)(w * w));
        a.y = 1 + ac / w;
        a.x = 1 + (ac - (a.y - 1) * w);
        a.dir = bounded(d[2], 4u);
    } else if (family == NX_DISTSHIFT) {
        // L9: lava over columns 2..S-3 of row 1 and of row 3 (variant 0) or
        // S-2 (variant 1); the goal is at (S-2, 1); no draws
        const int r2 = variant == 0 ? 3 : S - 2;
        for (int x = 2 + grp.lane; x <= S - 3; x += G) {
            g[W + x] = (uint8_t)C_LAVA;
            g[r2 * W + x] = (uint8_t)C_LAVA;
        }
    } else if (family == NX_KEYCORRIDOR) {
        const uint32_t ag = keycorridor_layout(grp, g, S, W, variant, seed, key_env, episode);
        a.x = ag & 0xFF;
        a.y = (ag >> 8) & 0xFF;
        a.dir = ag >> 16;
    } else if (family == NX_LAVA_CROSSING || family == NX_SIMPLE_CROSSING) {
        crossing_layout(grp, g, S, W, family, variant, seed, key_env, episode);
    } else if (family == NX_DYNOBS) {
        grp.sync();
        const int agent = 1 * W + 1;
        a.nb = n_balls;
        // ball b's column / row go to byte b of px / py and its draw k = b is
        // taken in the loop, so that no array is indexed by the loop counter
        // (that would move the draws to local memory)
        uint32_t px = 0, py = 0;
        for (int b = 0; b < n_balls; ++b) {
            const uint32_t db = draw(seed, key_env, episode, 0u, PURPOSE_LAYOUT, (uint32_t)b);
            const int n = count_free(grp, g, W, 1, S - 2, 1, S - 2, agent);
            const int bc = kth_free(grp, g, W, 1, S - 2, 1, S - 2, agent, bounded(db, (uint32_t)n));
            if (bc < 0) return false;
            grp.sync();
            if (grp.lane == 0) g[bc] = (uint8_t)C_BALL_BLUE;
            grp.sync();
            const int by = bc / W;
            px |= (uint32_t)(bc - by * W) << (8 * b);
            py |= (uint32_t)by << (8 * b);
        }
        a.bxp = px;
        a.byp = py;
    }
    grp.sync();
    return true;
}

// The same generator run by a whole warp for one env, kept out of line: it is
// the rare path of narrow groups, and inlining it would raise the register
// allocation of the whole step kernel.  0 <= FAM < NX_N_FAMILIES fixes the
// family (the lean step kernels of one family).  The new agent comes back in
// registers (a reference argument would put it on the caller's stack):
// x | y << 8 | dir << 16 | mission << 24, n_balls | ok << 8, then the balls'
// columns and rows one byte each.
// The same for the group of G >= 8 lanes that owns the env, likewise out of
// line: inlined into the step loop, the rare path's code cost the loop's
// scheduling more than the call costs.
template <int G, int FAM>
__device__ __noinline__ uint4 reset_layout_grp(const Grp<G> grp, uint8_t* g, int S, int W, int family, int n_balls,
                                               int variant, uint64_t seed, uint32_t key_env, uint32_t episode)
{
    AgentReg a;
    const bool ok = reset_layout(grp, g, S, W, (FAM >= 0 && FAM < NX_N_FAMILIES) ? FAM : family, n_balls, variant, seed,
                                 key_env, episode, a);
    uint4 r;
    r.x = (uint32_t)a.x | ((uint32_t)a.y << 8) | ((uint32_t)a.dir << 16) | (a.mission << 24);
    r.y = (uint32_t)a.nb | (ok ? 0x100u : 0u);
    r.z = a.bxp;
    r.w = a.byp;
    return r;
}

// The new episode's start from a packed reset (reset_layout_warp /
// reset_layout_grp); the invalid-action flag is sticky except on a reset
// launch.
__device__ __forceinline__ void unpack_reset(const uint4 r, uint32_t episode, bool reset_all, AgentReg& a)
{
    a.x = (int)(r.x & 0xFFu);
    a.y = (int)((r.x >> 8) & 0xFFu);
    a.dir = (int)((r.x >> 16) & 0xFFu);
    a.mission = r.x >> 24;
    a.nb = (int)(r.y & 0xFFu);
    a.carry = 0u;
    a.done = 0;
    a.t = 0;
    a.episode = episode;
    a.invalid = reset_all ? 0 : a.invalid;
    a.bxp = r.z;
    a.byp = r.w;
}

template <int FAM>
__device__ __noinline__ uint4 reset_layout_warp(uint8_t* g, int S, int family, int n_balls, int variant, uint64_t seed,
                                                uint32_t key_env, uint32_t episode)
{
    AgentReg a;
    const bool ok = reset_layout(Grp<32>((int)(threadIdx.x & 31u)), g, S, S,
                                 (FAM >= 0 && FAM < NX_N_FAMILIES) ? FAM : family, n_balls, variant, seed, key_env,
                                 episode, a);
    uint4 r;
    r.x = (uint32_t)a.x | ((uint32_t)a.y << 8) | ((uint32_t)a.dir << 16) | (a.mission << 24);
    r.y = (uint32_t)a.nb | (ok ? 0x100u : 0u);
    r.z = a.bxp;
    r.w = a.byp;
    return r;
}

// ---------------------------------------------------------------------------
// Occlusion of the 7x7 view (bit c = vy * 7 + vx of a 49-bit mask).  Rows are
// processed from the agent's row (vy = 6) outward.  Within a row, light
// spreads first toward +vx, then toward -vx, through transparent cells (a lit
// opaque cell is visible but passes nothing on); every lit transparent cell
// also lights the two cells ahead of it and of its neighbour in that pass,
// which seeds the next row.  occ_row() evaluates one row with prefix fills by
// doubling shifts; occ_table holds it for all 2^7 seeds x 2^7 transparency
// patterns (visible row in bits 0-6, next seed in bits 7-13), built by the
// compiler, so a row costs one cached load.
__host__ __device__ constexpr uint32_t occ_row(uint32_t seed, uint32_t t)
{
    uint32_t m = seed;
    const uint32_t p1 = t & 0x3Fu, p2 = p1 & (p1 >> 1), p4 = p2 & (p2 >> 2);  // toward +vx
    m |= (m & p1) << 1;
    m |= (m & p2) << 2;
    m |= (m & p4) << 4;
    m &= 0x7Fu;
    const uint32_t fa = m & p1;
    uint32_t up = fa | (fa << 1);
    const uint32_t q1 = t & 0x7Eu, q2 = q1 & (q1 << 1), q4 = q2 & (q2 << 2);  // toward -vx
    m |= (m & q1) >> 1;
    m |= (m & q2) >> 2;
    m |= (m & q4) >> 4;
    const uint32_t ba = m & q1;
    up |= ba | (ba >> 1);
    return m | ((up & 0x7Fu) << 7);
}

struct OccTable {
    uint16_t v[1 << 14];
};
constexpr OccTable make_occ_table()
{
    OccTable t{};
    for (uint32_t i = 0; i < (1u << 14); ++i) t.v[i] = (uint16_t)occ_row(i >> 7, i & 0x7Fu);
    return t;
}
__device__ const OccTable occ_table = make_occ_table();

// The same row by carries.  Adding (seed & p) to p sends a carry from every
// lit transparent cell up through the run of transparent cells above it to
// the first opaque (or edge) cell; the bits the addition changes are that run
// and its stopping cell -- the forward fill -- except for seeds inside the
// run, which the OR puts back.  The backward fill is the forward fill of the
// bit-reversed row.  About half the operations of occ_row's doubling shifts;
// carry_rows_agree() checks the two against each other for every input.
struct RevSwap {  // 32-bit reversal by swapping halves, bytes, nibbles, pairs, bits
    __host__ __device__ static constexpr uint32_t apply(uint32_t x)
    {
        x = ((x >> 1) & 0x55555555u) | ((x & 0x55555555u) << 1);
        x = ((x >> 2) & 0x33333333u) | ((x & 0x33333333u) << 2);
        x = ((x >> 4) & 0x0F0F0F0Fu) | ((x & 0x0F0F0F0Fu) << 4);
        x = ((x >> 8) & 0x00FF00FFu) | ((x & 0x00FF00FFu) << 8);
        return (x >> 16) | (x << 16);
    }
};
#ifdef __CUDACC__
struct RevBrev {
    __device__ static __forceinline__ uint32_t apply(uint32_t x) { return __brev(x); }
};
#endif
// The row's visible cells and the next row's seed, both 7-bit: the one-lane
// view keeps them apart, which saves packing and unpacking them per row.
struct OccRow {
    uint32_t vis, next;
};
template <class Rev>
__host__ __device__ constexpr OccRow occ_row_carry2(uint32_t seed, uint32_t t)
{
    const uint32_t p1 = t & 0x3Fu, q1 = t & 0x7Eu;  // may pass light toward +vx / -vx
    uint32_t m = seed | ((p1 + (seed & p1)) ^ p1);
    const uint32_t fa = m & p1;
    const uint32_t rq = Rev::apply(q1);
    uint32_t r = Rev::apply(m);
    r |= (rq + (r & rq)) ^ rq;  // rq's top bit (q1's bit 0) is clear: no carry leaves the word
    m = Rev::apply(r);
    const uint32_t ba = m & q1;
    return OccRow{m, fa | (fa << 1) | ba | (ba >> 1)};
}
template <class Rev>
__host__ __device__ constexpr uint32_t occ_row_carry(uint32_t seed, uint32_t t)
{
    const OccRow o = occ_row_carry2<Rev>(seed, t);
    return o.vis | (o.next << 7);
}
constexpr bool carry_rows_agree()
{
    for (uint32_t i = 0; i < (1u << 14); ++i) {
        const OccRow o = occ_row_carry2<RevSwap>(i >> 7, i & 0x7Fu);
        // both parts stay within 7 bits, so their packed form is occ_row's
        if (o.vis > 0x7Fu || o.next > 0x7Fu || (o.vis | (o.next << 7)) != occ_row(i >> 7, i & 0x7Fu)) return false;
    }
    return true;
}
static_assert(carry_rows_agree(), "the carry form of an occlusion row equals the doubling-shift form");

// Groups of two or more lanes (the ballot-assembled 49-bit mask of
// transparent cells, bit c = vy * 7 + vx): rows are looked up in `tab` (the
// table staged in shared memory by groups of eight or more lanes), or in the
// global table (L1-cached) when tab is null, all seven without a branch (a
// zero seed gives a zero row and a zero seed).  One lane per env evaluates
// each row in its carry form instead (render_view), which measures faster
// there than either table: a lane per env is bound by issue and by the
// latency of the chain.
template <int G>
__device__ __forceinline__ uint64_t occlusion(uint64_t tmask, const uint16_t* tab)
{
    static_assert(G > 1, "one lane per env evaluates the rows in render_view");
    uint64_t vis = 0;
    uint32_t seed = 1u << 3;
#pragma unroll
    for (int j = 6; j >= 0; --j) {
        const uint32_t t = (uint32_t)(tmask >> (7 * j)) & 0x7Fu;
        const uint32_t e = tab ? (uint32_t)tab[(seed << 7) | t] : (uint32_t)__ldg(&occ_table.v[(seed << 7) | t]);
        vis |= (uint64_t)(e & 0x7Fu) << (7 * j);
        seed = e >> 7;
    }
    return vis;
}

// Geometry of one env's view for one step: view cell (vx, vy) shows world
// cell pos + (6 - vy) F + (vx - 3) R (F the facing direction, R its
// right-hand side, y growing downward), i.e. linear index
// idx0 + vx dR - vy dF for row stride W; it lies inside the grid iff bit vx
// of colmask and bit vy of rowmask are set (outside cells read as a grey
// wall).
struct ViewGeom {
    int idx0, dR, dF;
    uint32_t colmask, rowmask;
};

__device__ __forceinline__ uint32_t bit_range(int lo, int hi)  // bits lo..hi of 0..6 (empty if lo > hi)
{
    lo = max(lo, 0);
    hi = min(hi, 6);
    return lo > hi ? 0u : ((2u << hi) - (1u << lo));
}

__device__ __forceinline__ ViewGeom view_geom(const AgentReg& a, int S, int W)
{
    const int fx = (a.dir == 0) - (a.dir == 2), fy = (a.dir == 1) - (a.dir == 3);
    const int rx = -fy, ry = fx;
    ViewGeom g;
    g.dF = fy * W + fx;
    g.dR = ry * W + rx;
    g.idx0 = a.y * W + a.x + 6 * g.dF - 3 * g.dR;
    // along R: coordinate a_r + (vx - 3) * sign(R)
    const int ar = rx != 0 ? a.x : a.y, sr = rx + ry;
    g.colmask = sr > 0 ? bit_range(3 - ar, 3 + (S - 1 - ar)) : bit_range(3 - (S - 1 - ar), 3 + ar);
    // along F: forward distance d = 6 - vy, coordinate a_f + d * sign(F)
    const int af = fx != 0 ? a.x : a.y, sf = fx + fy;
    const int dmax = sf > 0 ? S - 1 - af : af;
    g.rowmask = bit_range(6 - dmax, 6);
    return g;
}

// Atlas tile of a view cell from its triple: 0 unseen; 1 + 18 ent + 3 col +
// st when visible; + 198 for the agent's own cell.
__device__ __forceinline__ uint32_t tile_of_triple(bool visible, bool agent_cell, uint32_t tri)
{
    if (!visible) return 0u;
    const uint32_t t = 1u + 18u * (tri & 0xFFu) + 3u * ((tri >> 8) & 0xFFu) + (tri >> 16) + (agent_cell ? 198u : 0u);
    return t < (uint32_t)NX_ATLAS_TILES ? t : 0u;
}

// Egocentric view of one env: render_view computes it into registers (and,
// if `tiles` is non-null, writes the 49 atlas tile indices); write_view then
// stores the 147 symbolic bytes (row-major [vy][vx][ent, col, st], unseen
// cells 0) at `sym`.  `dec` maps a cell code to its observation triple.
//
// G >= 8: one view row per 8 lanes -- in round k, lane l holds cell
// (vx, vy) = (l % 8, k G/8 + l / 8) (lanes with vx = 7 or vy > 6 idle), so a
// round's ballot carries whole rows at byte offsets; the occlusion reads
// and writes those bytes and a lane's visibility bit is bit l of its round.
// G = 2, 4: lane l owns cells c = l, l + G, ...; a ballot per round assembles
// the 49-bit transparency mask.  Each lane stores its cells' three bytes.
// G = 1: the 49 codes are packed four per register, the transparency mask is
// gathered four cells at a time from the opaque bits, and the byte stream is
// stored as 36 funnel-shifted 32-bit words plus three single bytes.
template <int G>
struct ViewOut {
    uint32_t tri[(49 + G - 1) / G];
};
template <>
struct ViewOut<1> {
    uint32_t sw[37];  // stream words of the 147-byte record
};

// Byte masks of a 7-bit row mask m: spread_bits_lo sets byte i to 0xFF iff
// bit i of m is set (i = 0..3), spread_bits_hi byte i iff bit i + 4 is (byte
// 3 stays 0).  The multiply copies m four times, seven bits apart, so that
// bit i of m lands on bit 8 i + 7 (resp. bit i + 4 on 8 i + 7) with no two
// copies overlapping; the byte permute's sign-replicating selectors then fill
// each byte with its top bit.
__device__ __forceinline__ uint32_t sign_fill_bytes(uint32_t x)
{
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(0u), "n"(0xBA98));
    return r;
}
// a * b + c as one multiply-add.  Where the bytes of a * b and c never
// overlap the sum is their OR; written this way, the one-lane view's byte
// packing runs on the multiply-add pipe instead of adding shifts and ORs to
// the integer pipe, which the one-lane kernels keep the busiest (measured 3 %
// faster on the mixed batch).
__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}
__device__ __forceinline__ uint32_t spread_bits_lo(uint32_t m) { return sign_fill_bytes(m * 0x10204080u); }
__device__ __forceinline__ uint32_t spread_bits_hi(uint32_t m) { return sign_fill_bytes(m * 0x01020408u); }

// Groups of 8 or more lanes read a grid with a wall margin of at least six
// cells on every side (row stride W >= S + 12): every cell of the view, and of
// the idle lanes' positions (one row behind the agent, four columns to its
// right), lies in the margin or the grid, so they read without an in-grid
// test.  Narrower groups read a packed grid (W = S) with the masks.
template <int G>
__device__ __forceinline__ void render_view(const Grp<G>& grp, const uint8_t* g, int S, int W, const AgentReg& a,
                                            const uint32_t* dec, const uint16_t* occ, ViewOut<G>& out, uint16_t* tiles)
{
    const ViewGeom v = view_geom(a, S, W);
    if constexpr (G == 1) {
        // Strided gather: cell (vx, vy) is read at g[idx0 + vx dR - vy dF]
        // without a bounds test (guard bytes around the grid region keep every
        // read inside shared memory).  View row vy is held in two words,
        // row[2 vy] (cells 0-3) and row[2 vy + 1] (cells 4-6, byte 3 spare),
        // so that the row's in-grid walls, its transparency bits and, after
        // the occlusion pass, its visibility each take a few word operations.
        constexpr uint32_t kWall4 = C_WALL * 0x01010101u;
        const uint8_t* p0 = g + v.idx0;
        const uint32_t cm0 = spread_bits_lo(v.colmask), cm1 = spread_bits_hi(v.colmask);  // in-grid columns
        uint32_t row[14], trow[7];
#pragma unroll
        for (int vy = 0; vy < 7; ++vy) {
            uint32_t w0 = 0, w1 = 0;
#pragma unroll
            for (int vx = 0; vx < 7; ++vx) {
                if (vy == 6 && vx == 3) continue;  // the agent's cell
                const uint32_t b = p0[vx * v.dR - vy * v.dF];
                if (vx < 4) w0 = mad_lo(b, 1u << (8 * vx), w0);  // w0 |= b << 8 vx
                else w1 = mad_lo(b, 1u << (8 * (vx - 4)), w1);
            }
            // cells outside the grid read as grey walls
            const uint32_t rin = 0u - ((v.rowmask >> vy) & 1u);
            const uint32_t k0 = cm0 & rin, k1 = cm1 & rin;
            w0 = (w0 & k0) | (kWall4 & ~k0);
            w1 = (w1 & k1) | (kWall4 & ~k1);
            if (vy == 6)  // the agent's cell (3, 6): what it carries, else empty
                w0 = (w0 & 0x00FFFFFFu) | ((a.carry ? a.carry : (uint32_t)C_EMPTY) << 24);
            row[2 * vy] = w0;
            row[2 * vy + 1] = w1;
            // transparency bit vx = inverted top bit of cell vx's code: the
            // inverted top bits sit at bits 0, 8, 16, 24 (cells 0-3) and 4,
            // 12, 20 (cells 4-6); one multiply gathers them to bits 24-30
            // (the partial products never overlap, so nothing carries)
            const uint32_t x = ((~w0 >> 7) & 0x01010101u) | ((~w1 >> 3) & 0x00101010u);
            trow[vy] = (x * 0x01020408u) >> 24;
        }
        // occlusion: rows from the agent's (6) outward; an unseen cell's code
        // becomes 0, whose triple is (0, 0, 0) (a seen cell's code is never 0)
        uint32_t seed = 1u << 3;
#pragma unroll
        for (int vy = 6; vy >= 0; --vy) {
            const OccRow e = occ_row_carry2<RevBrev>(seed, trow[vy]);
            row[2 * vy] &= spread_bits_lo(e.vis);
            row[2 * vy + 1] &= spread_bits_hi(e.vis);
            seed = e.next;
        }
        uint32_t tri[49];
#pragma unroll
        for (int c = 0; c < 49; ++c) {
            const int vy = c / 7, vx = c % 7;
            const uint32_t code = (row[2 * vy + (vx >> 2)] >> (8 * (vx & 3))) & 0xFFu;
            tri[c] = dec[code];
            if (tiles) tiles[c] = (uint16_t)tile_of_triple(code != 0u, c == 45, tri[c]);
        }
#pragma unroll
        for (int m = 0; m < 12; ++m) {
            // (triples are 24-bit: tri[4m] | tri[4m+1] << 24, and so on)
            out.sw[3 * m] = mad_lo(tri[4 * m + 1], 1u << 24, tri[4 * m]);
            out.sw[3 * m + 1] = mad_lo(tri[4 * m + 2], 1u << 16, tri[4 * m + 1] >> 8);
            out.sw[3 * m + 2] = mad_lo(tri[4 * m + 3], 1u << 8, tri[4 * m + 2] >> 16);
        }
        out.sw[36] = tri[48];
    } else if constexpr (G >= 8) {
        constexpr int RPK = G / 8, K = (7 + RPK - 1) / RPK;  // view rows per round, rounds
        static_assert(K == (49 + G - 1) / G, "ViewOut holds one triple per round");
        const int vx = grp.lane & 7, r0 = grp.lane >> 3;
        const uint32_t carried = a.carry ? a.carry : (uint32_t)C_EMPTY;
        uint32_t code[K], tw[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int vy = k * RPK + r0;
            const bool cell = vx < 7 && vy < 7;
            // cells beyond the grid read the wall margin; the agent's cell
            // (3, 6) shows what it carries
            const uint32_t ld = g[v.idx0 + vx * v.dR - vy * v.dF];
            const uint32_t cd = (vy == 6 && vx == 3) ? carried : ld;
            code[k] = cd;
            tw[k] = grp.ballot(cell && !(cd & OPAQUE));  // row k RPK + r: bits 8 r .. 8 r + 6
        }
        // rows from the agent's (6) to the farthest (0), as in occlusion()
        uint32_t vw[K];
#pragma unroll
        for (int k = 0; k < K; ++k) vw[k] = 0u;
        uint32_t seed = 1u << 3;
#pragma unroll
        for (int j = 6; j >= 0; --j) {
            const int k = j / RPK, sh = 8 * (j % RPK);
            const uint32_t t = (tw[k] >> sh) & 0x7Fu;
            const uint32_t e = occ ? (uint32_t)occ[(seed << 7) | t] : (uint32_t)__ldg(&occ_table.v[(seed << 7) | t]);
            vw[k] |= (e & 0x7Fu) << sh;
            seed = e >> 7;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int vy = k * RPK + r0;
            const bool vb = (vw[k] >> grp.lane) & 1u;  // only cells have their bit set
            out.tri[k] = vb ? dec[code[k]] : 0u;
            if (tiles && vx < 7 && vy < 7)
                tiles[vy * 7 + vx] = (uint16_t)tile_of_triple(vb, vy == 6 && vx == 3, out.tri[k]);
        }
    } else {
        constexpr int K = (49 + G - 1) / G;
        uint32_t code[K];
        uint64_t tmask = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int c = k * G + grp.lane;
            const int vy = (c * 37) >> 8, vx = c - 7 * vy;  // c / 7 and c % 7 for c < 56
            // the in-grid test and the agent's cell (c = 45) as selects
            const bool in = c < 49 && ((v.colmask >> vx) & (v.rowmask >> vy) & 1u);
            const uint32_t ld = in ? (uint32_t)g[v.idx0 + vx * v.dR - vy * v.dF] : (uint32_t)C_WALL;
            const uint32_t cd = c == 45 ? (a.carry ? a.carry : (uint32_t)C_EMPTY) : ld;
            code[k] = cd;
            const uint32_t bits = grp.ballot(c < 49 && !(cd & OPAQUE));
            tmask |= (uint64_t)bits << (k * G);
        }
        const uint64_t vis = occlusion<G>(tmask, occ);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int c = k * G + grp.lane;
            const bool vb = c < 49 && ((vis >> c) & 1ull);
            out.tri[k] = vb ? dec[code[k]] : 0u;
            if (tiles && c < 49) tiles[c] = (uint16_t)tile_of_triple(vb, c == 45, out.tri[k]);
        }
    }
}

template <int G>
__device__ __forceinline__ void write_view(const Grp<G>& grp, const ViewOut<G>& out, uint8_t* sym)
{
    if constexpr (G == 1) {
        const uint32_t head = (4u - ((uint32_t)(uintptr_t)sym & 3u)) & 3u;  // bytes before the first aligned word
#pragma unroll
        for (uint32_t i = 0; i < 3; ++i)
            if (i < head) sym[i] = (uint8_t)(out.sw[0] >> (8 * i));
        uint32_t* wd = reinterpret_cast<uint32_t*>(sym + head);
#pragma unroll
        for (int i = 0; i < 36; ++i) wd[i] = __funnelshift_r(out.sw[i], out.sw[i + 1], 8 * head);
#pragma unroll
        for (uint32_t i = 0; i < 3; ++i)
            if (i >= head) sym[144 + i] = (uint8_t)(out.sw[36] >> (8 * i));
    } else if constexpr (G >= 8) {
        constexpr int RPK = G / 8, K = (7 + RPK - 1) / RPK;
        const int vx = grp.lane & 7, r0 = grp.lane >> 3;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int vy = k * RPK + r0, c = vy * 7 + vx;
            if (vx < 7 && vy < 7) {
                const uint32_t tri = out.tri[k];
                sym[3 * c + 0] = (uint8_t)tri;
                sym[3 * c + 1] = (uint8_t)(tri >> 8);
                sym[3 * c + 2] = (uint8_t)(tri >> 16);
            }
        }
    } else {
        constexpr int K = (49 + G - 1) / G;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int c = k * G + grp.lane;
            if (c < 49) {
                const uint32_t tri = out.tri[k];
                sym[3 * c + 0] = (uint8_t)tri;
                sym[3 * c + 1] = (uint8_t)(tri >> 8);
                sym[3 * c + 2] = (uint8_t)(tri >> 16);
            }
        }
    }
}

}  // namespace nxd
