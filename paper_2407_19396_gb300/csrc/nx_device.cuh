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

enum { PURPOSE_LAYOUT = 1u, PURPOSE_BALL = 2u, PURPOSE_ACTION = 3u };

__device__ __forceinline__ uint32_t draw(uint64_t seed, uint32_t env, uint32_t episode, uint32_t step,
                                         uint32_t purpose, uint32_t k)
{
    return philox_word0(env, episode, step, (purpose << 24) | k, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// bounded draw in [0, n): (x * n) >> 32
__device__ __forceinline__ int bounded(uint32_t x, uint32_t n) { return (int)__umulhi(x, n); }

// ---------------------------------------------------------------------------
// Packed cell code (one byte in shared memory): (kind << 3) | colour, where
// kind is the entity code except for doors: 4 open, 11 closed, 12 locked.
enum : uint32_t {
    K_EMPTY = 1, K_WALL = 2, K_FLOOR = 3, K_DOOR_OPEN = 4, K_KEY = 5, K_BALL = 6, K_BOX = 7, K_GOAL = 8,
    K_LAVA = 9, K_DOOR_CLOSED = 11, K_DOOR_LOCKED = 12
};
enum : uint32_t {
    C_EMPTY = (K_EMPTY << 3),
    C_WALL = (K_WALL << 3) | 5u,
    C_GOAL = (K_GOAL << 3) | 1u,
    C_LAVA = (K_LAVA << 3),
    C_BALL_BLUE = (K_BALL << 3) | 2u,
    C_KEY_YELLOW = (K_KEY << 3) | 4u,
    C_DOOR_LOCKED_YELLOW = (K_DOOR_LOCKED << 3) | 4u
};
// kinds that let light through: all but wall (2), closed (11) and locked (12) doors
#define NX_TRANSPARENT_KINDS 0x7FBu
// kinds the agent can enter: empty, floor, open door, goal, lava
#define NX_WALKABLE_KINDS ((1u << 1) | (1u << 3) | (1u << 4) | (1u << 8) | (1u << 9))

__device__ __forceinline__ uint32_t pack_cell(uint32_t ent, uint32_t col, uint32_t st)
{
    uint32_t kind = ent;
    if (ent == 4u) kind = st == 0u ? K_DOOR_OPEN : (st == 1u ? K_DOOR_CLOSED : K_DOOR_LOCKED);
    return (kind << 3) | (col & 7u);
}
__device__ __forceinline__ uint32_t cell_kind(uint32_t code) { return code >> 3; }
__device__ __forceinline__ uint32_t cell_col(uint32_t code) { return code & 7u; }
__device__ __forceinline__ uint32_t cell_ent(uint32_t code)
{
    const uint32_t k = code >> 3;
    return k >= 11u ? 4u : k;
}
__device__ __forceinline__ uint32_t cell_st(uint32_t code)
{
    const uint32_t k = code >> 3;
    return k >= 11u ? k - 10u : 0u;
}
__device__ __forceinline__ bool transparent(uint32_t code) { return (NX_TRANSPARENT_KINDS >> (code >> 3)) & 1u; }
__device__ __forceinline__ bool walkable(uint32_t code) { return (NX_WALKABLE_KINDS >> (code >> 3)) & 1u; }

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

// Number of empty cells in the rectangle [x0,x1] x [y0,y1] not counting cell
// index `skip` (-1 for none).
template <int G>
__device__ int count_free(const Grp<G>& grp, const uint8_t* g, int W, int x0, int x1, int y0, int y1, int skip)
{
    const int w = x1 - x0 + 1, n = w * (y1 - y0 + 1);
    int total = 0;
    for (int r0 = 0; r0 < n; r0 += G) {
        const int r = r0 + grp.lane;
        bool f = false;
        if (r < n) {
            const int yy = y0 + r / w, xx = x0 + r % w, ci = yy * W + xx;
            f = g[ci] == C_EMPTY && ci != skip;
        }
        total += __popc(grp.ballot(f));
    }
    return total;
}

// Cell index of the k-th empty cell of the rectangle in row-major order (y
// outer, x inner), not counting `skip`; -1 if there is none.
template <int G>
__device__ int kth_free(const Grp<G>& grp, const uint8_t* g, int W, int x0, int x1, int y0, int y1, int skip, int k)
{
    const int w = x1 - x0 + 1, n = w * (y1 - y0 + 1);
    for (int r0 = 0; r0 < n; r0 += G) {
        const int r = r0 + grp.lane;
        bool f = false;
        int ci = 0;
        if (r < n) {
            const int yy = y0 + r / w, xx = x0 + r % w;
            ci = yy * W + xx;
            f = g[ci] == C_EMPTY && ci != skip;
        }
        uint32_t b = grp.ballot(f);
        const int cnt = __popc(b);
        if (k < cnt) {
            for (int i = 0; i < k; ++i) b &= b - 1u;
            return grp.shfl(ci, __ffs(b) - 1);
        }
        k -= cnt;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// Per-env registers (every lane of the group holds the same copy).
struct AgentReg {
    int x, y, dir;
    uint32_t carry;  // packed code of the carried object, 0 = nothing
    int done, invalid, t;
    uint32_t episode;
    int nb;
    int bx[4], by[4];
};

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
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        a.bx[b] = (w1.x >> (8 * b)) & 0xFF;
        a.by[b] = (w1.y >> (8 * b)) & 0xFF;
    }
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
    w1.x = 0;
    w1.y = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        w1.x |= (uint32_t)a.bx[b] << (8 * b);
        w1.y |= (uint32_t)a.by[b] << (8 * b);
    }
    w1.z = (uint32_t)it.family | ((uint32_t)it.size << 8);
    w1.w = grid_offset;
    reinterpret_cast<uint4*>(dst)[0] = w0;
    reinterpret_cast<uint4*>(dst)[1] = w1;
}

// ---------------------------------------------------------------------------
// Layout generators of the Table 8 families.  Draw k of a reset is
// draw(seed, env, episode, 0, PURPOSE_LAYOUT, k); the k-th free cell is
// counted row-major; the agent is never stored in the grid.
// Returns false (and leaves a partial layout) only if a free-cell choice found
// no cell, which cannot happen for sizes 5..19; the caller raises a flag.
template <int G>
__device__ bool reset_layout(const Grp<G>& grp, uint8_t* g, int S, int family, int n_balls, uint64_t seed,
                             uint32_t key_env, uint32_t episode, AgentReg& a)
{
    const int HW = S * S;
    for (int c = grp.lane; c < HW; c += G) {
        const int y = c / S, x = c - y * S;
        const bool border = x == 0 || y == 0 || x == S - 1 || y == S - 1;
        g[c] = (uint8_t)(border ? C_WALL : C_EMPTY);
    }
    a.x = 1;
    a.y = 1;
    a.dir = 0;
    a.carry = 0;
    a.done = 0;
    a.t = 0;
    a.episode = episode;
    a.nb = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        a.bx[b] = 0;
        a.by[b] = 0;
    }
    uint32_t d[8];
    const int n_draws = family == NX_DOORKEY ? 5 : family == NX_FOURROOMS ? 7 : family == NX_LAVAGAP ? 2
                        : family == NX_DYNOBS ? n_balls : 0;
    group_draws(grp, n_draws, d,
                [&](uint32_t k) { return draw(seed, key_env, episode, 0u, PURPOSE_LAYOUT, k); });
    grp.sync();
    const int goal = (S - 2) * S + (S - 2);
    if (family != NX_FOURROOMS) {
        if (grp.lane == 0) g[goal] = (uint8_t)C_GOAL;
    }
    if (family == NX_DOORKEY) {
        const int xw = 2 + bounded(d[0], (uint32_t)(S - 4));
        const int door_y = 1 + bounded(d[1], (uint32_t)(S - 3));
        for (int y = 1 + grp.lane; y <= S - 2; y += G)
            g[y * S + xw] = (uint8_t)(y == door_y ? C_DOOR_LOCKED_YELLOW : C_WALL);
        grp.sync();
        const int n = count_free(grp, g, S, 1, xw - 1, 1, S - 2, -1);
        const int ac = kth_free(grp, g, S, 1, xw - 1, 1, S - 2, -1, bounded(d[2], (uint32_t)n));
        const int kc = kth_free(grp, g, S, 1, xw - 1, 1, S - 2, ac, bounded(d[4], (uint32_t)(n - 1)));
        if (ac < 0 || kc < 0) return false;
        a.x = ac % S;
        a.y = ac / S;
        a.dir = bounded(d[3], 4u);
        grp.sync();
        if (grp.lane == 0) g[kc] = (uint8_t)C_KEY_YELLOW;
    } else if (family == NX_FOURROOMS) {
        const int m = S / 2;
        for (int i = grp.lane; i < S; i += G) {
            g[i * S + m] = (uint8_t)C_WALL;
            g[m * S + i] = (uint8_t)C_WALL;
        }
        grp.sync();
        if (grp.lane == 0) {
            g[(1 + bounded(d[0], (uint32_t)(m - 1))) * S + m] = (uint8_t)C_EMPTY;
            g[(m + 1 + bounded(d[1], (uint32_t)(S - 2 - m))) * S + m] = (uint8_t)C_EMPTY;
            g[m * S + 1 + bounded(d[2], (uint32_t)(m - 1))] = (uint8_t)C_EMPTY;
            g[m * S + m + 1 + bounded(d[3], (uint32_t)(S - 2 - m))] = (uint8_t)C_EMPTY;
        }
        grp.sync();
        const int n = count_free(grp, g, S, 1, S - 2, 1, S - 2, -1);
        const int gc = kth_free(grp, g, S, 1, S - 2, 1, S - 2, -1, bounded(d[4], (uint32_t)n));
        if (gc < 0) return false;
        grp.sync();
        if (grp.lane == 0) g[gc] = (uint8_t)C_GOAL;
        grp.sync();
        const int ac = kth_free(grp, g, S, 1, S - 2, 1, S - 2, -1, bounded(d[5], (uint32_t)(n - 1)));
        if (ac < 0) return false;
        a.x = ac % S;
        a.y = ac / S;
        a.dir = bounded(d[6], 4u);
    } else if (family == NX_LAVAGAP) {
        const int xl = 2 + bounded(d[0], (uint32_t)(S - 4));
        const int gap = 1 + bounded(d[1], (uint32_t)(S - 2));
        for (int y = 1 + grp.lane; y <= S - 2; y += G)
            if (y != gap) g[y * S + xl] = (uint8_t)C_LAVA;
    } else if (family == NX_DYNOBS) {
        grp.sync();
        const int agent = 1 * S + 1;
        a.nb = n_balls;
        for (int b = 0; b < n_balls; ++b) {
            const int n = count_free(grp, g, S, 1, S - 2, 1, S - 2, agent);
            const int bc = kth_free(grp, g, S, 1, S - 2, 1, S - 2, agent, bounded(d[b], (uint32_t)n));
            if (bc < 0) return false;
            grp.sync();
            if (grp.lane == 0) g[bc] = (uint8_t)C_BALL_BLUE;
            grp.sync();
            a.bx[b] = bc % S;
            a.by[b] = bc / S;
        }
    }
    grp.sync();
    return true;
}

// ---------------------------------------------------------------------------
// Occlusion of the 7x7 view (bit c = vy * 7 + vx of a 49-bit mask).  Rows are
// processed from the agent's row (vy = 6) outward.  Within a row, light
// spreads first toward +vx, then toward -vx, through transparent cells (a lit
// opaque cell is visible but passes nothing on); every lit transparent cell
// also lights the two cells ahead of it and of its neighbour in that pass,
// which seeds the next row.  Each pass is a prefix fill done with doubling
// shifts (propagate masks of length 1, 2, 4).
__device__ __forceinline__ uint64_t occlusion(uint64_t tmask)
{
    uint64_t vis = 0;
    uint32_t seed = 1u << 3;
#pragma unroll
    for (int j = 6; j >= 0; --j) {
        const uint32_t t = (uint32_t)(tmask >> (7 * j)) & 0x7Fu;
        uint32_t m = seed;
        // toward +vx: a lit cell i <= 5 that is transparent lights i + 1
        const uint32_t p1 = t & 0x3Fu;
        const uint32_t p2 = p1 & (p1 >> 1);
        const uint32_t p4 = p2 & (p2 >> 2);
        m |= (m & p1) << 1;
        m |= (m & p2) << 2;
        m |= (m & p4) << 4;
        m &= 0x7Fu;
        const uint32_t fa = m & p1;
        uint32_t up = fa | (fa << 1);
        // toward -vx: a lit cell i >= 1 that is transparent lights i - 1
        const uint32_t q1 = t & 0x7Eu;
        const uint32_t q2 = q1 & (q1 << 1);
        const uint32_t q4 = q2 & (q2 << 2);
        m |= (m & q1) >> 1;
        m |= (m & q2) >> 2;
        m |= (m & q4) >> 4;
        const uint32_t ba = m & q1;
        up |= ba | (ba >> 1);
        vis |= (uint64_t)m << (7 * j);
        seed = up & 0x7Fu;
    }
    return vis;
}

// Atlas tile of a view cell: 0 unseen; 1 + 18 ent + 3 col + st when visible;
// + 198 for the agent's own cell.
__device__ __forceinline__ uint32_t tile_of(bool visible, bool agent_cell, uint32_t code)
{
    if (!visible) return 0u;
    const uint32_t t = 1u + 18u * cell_ent(code) + 3u * cell_col(code) + cell_st(code) + (agent_cell ? 198u : 0u);
    return t < (uint32_t)NX_ATLAS_TILES ? t : 0u;  // codes outside the tables cannot index past the atlas
}

// Egocentric view of one env: cell (vx, vy) shows world cell
// pos + (6 - vy) F + (vx - 3) R (F facing, R its right-hand direction);
// outside the grid reads as a grey wall; the agent's cell shows what it
// carries.  Writes the 147 symbolic bytes (row-major [vy][vx][ent, col, st])
// to `sym` and, if `tiles` is non-null, the 49 atlas tile indices.
template <int G>
__device__ __forceinline__ void render_view(const Grp<G>& grp, const uint8_t* g, int S, const AgentReg& a,
                                            uint8_t* sym, uint16_t* tiles)
{
    constexpr int K = (49 + G - 1) / G;
    const int fx = (a.dir == 0) - (a.dir == 2), fy = (a.dir == 1) - (a.dir == 3);
    const int rx = -fy, ry = fx;  // right-hand direction = facing rotated clockwise (y grows downward)
    uint32_t code[K];
    uint64_t tmask = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int c = k * G + grp.lane;
        uint32_t cd = 0;
        if (c < 49) {
            const int vy = c / 7, vx = c - 7 * vy;
            if (c == 45) {
                cd = a.carry ? a.carry : (uint32_t)C_EMPTY;
            } else {
                const int x = a.x + (6 - vy) * fx + (vx - 3) * rx;
                const int y = a.y + (6 - vy) * fy + (vx - 3) * ry;
                cd = ((unsigned)x < (unsigned)S && (unsigned)y < (unsigned)S) ? (uint32_t)g[y * S + x]
                                                                              : (uint32_t)C_WALL;
            }
        }
        code[k] = cd;
        const uint32_t bits = grp.ballot(c < 49 && transparent(cd));
        tmask |= (uint64_t)bits << (k * G);
    }
    const uint64_t vis = occlusion(tmask);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int c = k * G + grp.lane;
        if (c < 49) {
            const bool v = (vis >> c) & 1ull;
            const uint32_t cd = code[k];
            sym[3 * c + 0] = v ? (uint8_t)cell_ent(cd) : (uint8_t)0;
            sym[3 * c + 1] = v ? (uint8_t)cell_col(cd) : (uint8_t)0;
            sym[3 * c + 2] = v ? (uint8_t)cell_st(cd) : (uint8_t)0;
            if (tiles) tiles[c] = (uint16_t)tile_of(v, c == 45, cd);
        }
    }
}

}  // namespace nxd
