/*
 * navix_oracle.c -- plain CPU oracle of the batched MiniGrid step of NAVIX
 * (arXiv 2407.19396).  TEST INFRASTRUCTURE ONLY: see navix_oracle.h.
 *
 * Everything here is written as the literal sequence of steps, one env at a
 * time, with no blocking, fusion or bit tricks, so that a reader can check it
 * against the paper's systems (Table 3, Appendix A) and the readings stated
 * beside each function.
 */
#include "navix_oracle.h"

#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Randomness (reading R1).  The paper draws its randomness from JAX keys
 * (reset(key), Section 3.2.2; key splitting, Code 1 and Code 3).  Here every
 * draw is a counter-based Philox4x32-10 value: key = (seed lo, seed hi),
 * counter = (env index, episode, step, purpose << 24 | draw), word 0.
 * Philox4x32-10 as defined by Salmon et al., "Parallel Random Numbers: As
 * Easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 multiplications by
 * 0xD2511F53 and 0xCD9E8D57, with the key bumped by the Weyl constants
 * 0x9E3779B9 / 0xBB67AE85 between rounds. */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0;
    c[1] = n1;
    c[2] = n2;
    c[3] = n3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = c[3];
}

/* Bounded draw in [0, n): multiply-shift (Lemire), no rejection (R1). */
uint32_t orc_bounded(uint32_t x, uint32_t n) { return (uint32_t)(((uint64_t)x * (uint64_t)n) >> 32); }

uint32_t orc_draw(uint64_t seed, uint32_t env_index, uint32_t episode, uint32_t step, uint32_t purpose, uint32_t draw)
{
    uint32_t ctr[4] = {env_index, episode, step, (purpose << 24) | draw};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[0];
}

enum { PURPOSE_LAYOUT = 1, PURPOSE_BALL = 2, PURPOSE_ACTION = 3, PURPOSE_EXPLORE = 4 };

/* ------------------------------------------------------------------------ */
/* Cells (reading R5): the grid stores (entity, colour, state) per cell. */
static int idx(const orc_env* e, int x, int y) { return y * e->width + x; }

static int in_grid(const orc_env* e, int x, int y) { return x >= 0 && y >= 0 && x < e->width && y < e->height; }

void orc_set_cell(orc_env* e, int32_t x, int32_t y, int32_t ent, int32_t col, int32_t st)
{
    int i = idx(e, x, y);
    e->ent[i] = (uint8_t)ent;
    e->col[i] = (uint8_t)col;
    e->st[i] = (uint8_t)st;
}

static void set_empty(orc_env* e, int x, int y) { orc_set_cell(e, x, y, ORC_EMPTYCELL, 0, 0); }

/* Reads a cell; cells outside the grid read as a grey wall (reading R4). */
static void get_cell(const orc_env* e, int x, int y, int* ent, int* col, int* st)
{
    if (!in_grid(e, x, y)) {
        *ent = ORC_WALL;
        *col = ORC_GREY;
        *st = 0;
        return;
    }
    int i = idx(e, x, y);
    *ent = e->ent[i];
    *col = e->col[i];
    *st = e->st[i];
}

static int is_empty_cell(const orc_env* e, int x, int y)
{
    if (!in_grid(e, x, y)) return 0;
    int i = idx(e, x, y);
    return e->ent[i] == ORC_EMPTYCELL && e->col[i] == 0 && e->st[i] == 0;
}

/* Walkable: empty, floor, goal, lava, or an open door (R5). */
static int walkable(int ent, int st)
{
    if (ent == ORC_EMPTYCELL || ent == ORC_FLOOR || ent == ORC_GOAL || ent == ORC_LAVA) return 1;
    if (ent == ORC_DOOR && st == ORC_OPEN) return 1;
    return 0;
}

/* Transparent: everything but walls and doors that are not open (R5). */
static int transparent(int ent, int st)
{
    if (ent == ORC_WALL) return 0;
    if (ent == ORC_DOOR && st != ORC_OPEN) return 0;
    return 1;
}

/* Directions: 0 = east (+x), 1 = south (+y), 2 = west, 3 = north. */
static const int DX[4] = {1, 0, -1, 0};
static const int DY[4] = {0, 1, 0, -1};

void orc_set_agent(orc_env* e, int32_t x, int32_t y, int32_t dir, int32_t carry_ent, int32_t carry_col)
{
    e->ax = x;
    e->ay = y;
    e->dir = dir;
    e->carry_ent = carry_ent;
    e->carry_col = carry_col;
}

/* ------------------------------------------------------------------------ */
/* Layouts (Table 8 environment families; concrete generators L1-L5). */

int32_t orc_default_max_steps(int32_t family, int32_t size)
{
    /* reading R17: Empty 4S^2 (100 at S = 5), DoorKey 10S^2 (640 at S = 8),
     * FourRooms 100, LavaGap 4S^2, Dynamic-Obstacles 4S^2; Empty-Random and the
     * crossings 4S^2; GoToDoor 5S^2; KeyCorridor 30 s^2 for room side s */
    switch (family) {
    case ORC_DOORKEY: return 10 * size * size;
    case ORC_GOTODOOR: return 5 * size * size;
    case ORC_KEYCORRIDOR: {
        int s = (size - 1) / 3 + 1; /* the room side */
        return 30 * s * s;
    }
    case ORC_FOURROOMS: return 100;
    default: return 4 * size * size;
    }
}

static void clear_grid(orc_env* e)
{
    for (int y = 0; y < e->height; y++)
        for (int x = 0; x < e->width; x++) set_empty(e, x, y);
}

static void border_walls(orc_env* e)
{
    for (int x = 0; x < e->width; x++) {
        orc_set_cell(e, x, 0, ORC_WALL, ORC_GREY, 0);
        orc_set_cell(e, x, e->height - 1, ORC_WALL, ORC_GREY, 0);
    }
    for (int y = 0; y < e->height; y++) {
        orc_set_cell(e, 0, y, ORC_WALL, ORC_GREY, 0);
        orc_set_cell(e, e->width - 1, y, ORC_WALL, ORC_GREY, 0);
    }
}

/* Counts the empty cells of the rectangle [x0,x1]x[y0,y1], not counting the
 * cell (skip_x, skip_y) (pass -1 to skip nothing). */
static int count_free(const orc_env* e, int x0, int x1, int y0, int y1, int skip_x, int skip_y)
{
    int n = 0;
    for (int y = y0; y <= y1; y++)
        for (int x = x0; x <= x1; x++)
            if (is_empty_cell(e, x, y) && !(x == skip_x && y == skip_y)) n++;
    return n;
}

/* The k-th empty cell of the rectangle in row-major order, y outer and x
 * inner (reading R18), not counting (skip_x, skip_y). */
static void kth_free(const orc_env* e, int k, int x0, int x1, int y0, int y1, int skip_x, int skip_y, int* ox,
                     int* oy)
{
    int n = 0;
    for (int y = y0; y <= y1; y++)
        for (int x = x0; x <= x1; x++) {
            if (!is_empty_cell(e, x, y) || (x == skip_x && y == skip_y)) continue;
            if (n == k) {
                *ox = x;
                *oy = y;
                return;
            }
            n++;
        }
    /* unreachable for valid k: the callers draw k in [0, count) */
    *ox = -1;
    *oy = -1;
}

static uint32_t layout_draw(const orc_env* e, uint32_t k)
{
    return orc_draw(e->seed, e->env_index, e->episode, 0, PURPOSE_LAYOUT, k);
}

/* L1 Empty-S: border walls, agent at (1,1) facing east, goal at (S-2,S-2). */
static void layout_empty(orc_env* e)
{
    orc_set_cell(e, e->width - 2, e->height - 2, ORC_GOAL, ORC_GREEN, 0);
    orc_set_agent(e, 1, 1, 0, 0, 0);
}

/* L2 DoorKey-S: a wall column at x_w in 2..W-3 with a locked yellow door at a
 * row in 1..H-3; agent and yellow key on free cells left of the wall; goal
 * at (W-2,H-2). */
static void layout_doorkey(orc_env* e)
{
    int W = e->width, H = e->height;
    orc_set_cell(e, W - 2, H - 2, ORC_GOAL, ORC_GREEN, 0);
    int xw = 2 + (int)orc_bounded(layout_draw(e, 0), (uint32_t)(W - 4));
    for (int y = 1; y <= H - 2; y++) orc_set_cell(e, xw, y, ORC_WALL, ORC_GREY, 0);
    int door_y = 1 + (int)orc_bounded(layout_draw(e, 1), (uint32_t)(H - 3));
    orc_set_cell(e, xw, door_y, ORC_DOOR, ORC_YELLOW, ORC_LOCKED);
    int n = count_free(e, 1, xw - 1, 1, H - 2, -1, -1);
    int ax, ay;
    kth_free(e, (int)orc_bounded(layout_draw(e, 2), (uint32_t)n), 1, xw - 1, 1, H - 2, -1, -1, &ax, &ay);
    int dir = (int)orc_bounded(layout_draw(e, 3), 4u);
    orc_set_agent(e, ax, ay, dir, 0, 0);
    int kx, ky;
    kth_free(e, (int)orc_bounded(layout_draw(e, 4), (uint32_t)(n - 1)), 1, xw - 1, 1, H - 2, ax, ay, &kx, &ky);
    orc_set_cell(e, kx, ky, ORC_KEY, ORC_YELLOW, 0);
}

/* L3 FourRooms-S: walls on x = m and y = m (m = S/2), one gap per half wall,
 * goal and agent on random free cells, random direction. */
static void layout_fourrooms(orc_env* e)
{
    int S = e->width, m = S / 2;
    for (int i = 0; i < S; i++) {
        orc_set_cell(e, m, i, ORC_WALL, ORC_GREY, 0);
        orc_set_cell(e, i, m, ORC_WALL, ORC_GREY, 0);
    }
    set_empty(e, m, 1 + (int)orc_bounded(layout_draw(e, 0), (uint32_t)(m - 1)));
    set_empty(e, m, m + 1 + (int)orc_bounded(layout_draw(e, 1), (uint32_t)(S - 2 - m)));
    set_empty(e, 1 + (int)orc_bounded(layout_draw(e, 2), (uint32_t)(m - 1)), m);
    set_empty(e, m + 1 + (int)orc_bounded(layout_draw(e, 3), (uint32_t)(S - 2 - m)), m);
    int n = count_free(e, 1, S - 2, 1, S - 2, -1, -1);
    int gx, gy;
    kth_free(e, (int)orc_bounded(layout_draw(e, 4), (uint32_t)n), 1, S - 2, 1, S - 2, -1, -1, &gx, &gy);
    orc_set_cell(e, gx, gy, ORC_GOAL, ORC_GREEN, 0);
    int ax, ay;
    kth_free(e, (int)orc_bounded(layout_draw(e, 5), (uint32_t)(n - 1)), 1, S - 2, 1, S - 2, -1, -1, &ax, &ay);
    int dir = (int)orc_bounded(layout_draw(e, 6), 4u);
    orc_set_agent(e, ax, ay, dir, 0, 0);
}

/* L4 LavaGap-S: agent (1,1) east, goal (S-2,S-2), a lava column at x_l in
 * 2..S-3 with one gap at a row in 1..S-2. */
static void layout_lavagap(orc_env* e)
{
    int S = e->width;
    orc_set_cell(e, S - 2, S - 2, ORC_GOAL, ORC_GREEN, 0);
    orc_set_agent(e, 1, 1, 0, 0, 0);
    int xl = 2 + (int)orc_bounded(layout_draw(e, 0), (uint32_t)(S - 4));
    int gap = 1 + (int)orc_bounded(layout_draw(e, 1), (uint32_t)(S - 2));
    for (int y = 1; y <= S - 2; y++)
        if (y != gap) orc_set_cell(e, xl, y, ORC_LAVA, 0, 0);
}

/* L5 Dynamic-Obstacles-S: agent (1,1) east, goal (S-2,S-2), n blue balls on
 * free interior cells (never the agent's cell), placed in index order. */
static void layout_dynobs(orc_env* e)
{
    int S = e->width;
    orc_set_cell(e, S - 2, S - 2, ORC_GOAL, ORC_GREEN, 0);
    orc_set_agent(e, 1, 1, 0, 0, 0);
    for (int b = 0; b < e->n_balls; b++) {
        int n = count_free(e, 1, S - 2, 1, S - 2, e->ax, e->ay);
        int bx, by;
        kth_free(e, (int)orc_bounded(layout_draw(e, (uint32_t)b), (uint32_t)n), 1, S - 2, 1, S - 2, e->ax, e->ay,
                 &bx, &by);
        orc_set_cell(e, bx, by, ORC_BALL, ORC_BLUE, 0);
        e->ball_x[b] = bx;
        e->ball_y[b] = by;
    }
}

/* L6 Empty-Random-S: Empty-S with the agent on a drawn empty interior cell
 * (never the goal), facing a drawn direction. */
static void layout_empty_random(orc_env* e)
{
    int S = e->width;
    orc_set_cell(e, S - 2, S - 2, ORC_GOAL, ORC_GREEN, 0);
    int n = count_free(e, 1, S - 2, 1, S - 2, -1, -1);
    int ax, ay;
    kth_free(e, (int)orc_bounded(layout_draw(e, 0), (uint32_t)n), 1, S - 2, 1, S - 2, -1, -1, &ax, &ay);
    orc_set_agent(e, ax, ay, (int)orc_bounded(layout_draw(e, 1), 4u), 0, 0);
}

/* L9 DistShift-S, variant v (0: DistShift1, 1: DistShift2): agent (1,1)
 * east, goal (S-2, 1); lava on row 1 and on row 3 (v = 0) or row S-2 (v = 1),
 * each over the columns 2..S-3.  No draws: the two variants are the fixed
 * train / test layouts of a distribution shift. */
static void layout_distshift(orc_env* e)
{
    int S = e->width;
    orc_set_cell(e, S - 2, 1, ORC_GOAL, ORC_GREEN, 0);
    orc_set_agent(e, 1, 1, 0, 0, 0);
    int r2 = e->variant == 0 ? 3 : S - 2;
    for (int x = 2; x <= S - 3; x++) {
        orc_set_cell(e, x, 1, ORC_LAVA, 0, 0);
        orc_set_cell(e, x, r2, ORC_LAVA, 0, 0);
    }
}

/* L10 KeyCorridor S{s}R{R} (Table 8; variant R - 1): a 3 x R block of rooms
 * of side s sharing their walls, held in the S x S grid with S = 3(s-1)+1.
 * The rooms span rows 0..H-1 with H = (s-1)R+1; every row below is wall
 * (the views treat cells outside a grid as wall, so views and rules are those
 * of the H x S grid).  The middle column of rooms is one corridor: the walls
 * between its rooms are open.  Every side room has a door in the wall it
 * shares with the corridor; the room holding the goal has a locked door and
 * the key of that door's colour lies in a side room on the other side; the
 * other doors are closed.  Draws, in order: the door rows (left rooms top to
 * bottom, then right rooms), the door colours in the same order, the goal's
 * side and room row, the key's room row, the goal cell, the key cell (free
 * interior cells of their rooms), the agent's corridor cell and direction. */
static void layout_keycorridor(orc_env* e)
{
    int S = e->width, s = (S - 1) / 3 + 1, R = e->variant + 1, H = (s - 1) * R + 1;
    int xl = s - 1, xr = 2 * (s - 1); /* the corridor's walls */
    for (int y = 0; y < S; y++)
        for (int x = 0; x < S; x++) {
            int wall = y >= H - 1 || y == 0 || x == 0 || x == S - 1 || x == xl || x == xr;
            if (y % (s - 1) == 0 && !(x > xl && x < xr)) wall = 1;
            if (wall) orc_set_cell(e, x, y, ORC_WALL, ORC_GREY, 0);
        }
    uint32_t k = 0;
    int door_y[2][3], door_c[2][3];
    for (int side = 0; side < 2; side++)
        for (int j = 0; j < R; j++) door_y[side][j] = j * (s - 1) + 1 + (int)orc_bounded(layout_draw(e, k++), (uint32_t)(s - 2));
    for (int side = 0; side < 2; side++)
        for (int j = 0; j < R; j++) door_c[side][j] = (int)orc_bounded(layout_draw(e, k++), 6u);
    int gside = (int)orc_bounded(layout_draw(e, k++), 2u);
    int grow = (int)orc_bounded(layout_draw(e, k++), (uint32_t)R);
    int krow = (int)orc_bounded(layout_draw(e, k++), (uint32_t)R);
    for (int side = 0; side < 2; side++)
        for (int j = 0; j < R; j++)
            orc_set_cell(e, side == 0 ? xl : xr, door_y[side][j], ORC_DOOR, door_c[side][j],
                         (side == gside && j == grow) ? ORC_LOCKED : ORC_CLOSED);
    /* the goal in room (gside, grow), the key in room (1 - gside, krow) */
    int gx0 = gside == 0 ? 1 : xr + 1, gy0 = grow * (s - 1) + 1;
    int n = count_free(e, gx0, gx0 + s - 3, gy0, gy0 + s - 3, -1, -1);
    int gx, gy;
    kth_free(e, (int)orc_bounded(layout_draw(e, k++), (uint32_t)n), gx0, gx0 + s - 3, gy0, gy0 + s - 3, -1, -1, &gx, &gy);
    orc_set_cell(e, gx, gy, ORC_GOAL, ORC_GREEN, 0);
    int kx0 = gside == 0 ? xr + 1 : 1, ky0 = krow * (s - 1) + 1;
    n = count_free(e, kx0, kx0 + s - 3, ky0, ky0 + s - 3, -1, -1);
    int kx, ky;
    kth_free(e, (int)orc_bounded(layout_draw(e, k++), (uint32_t)n), kx0, kx0 + s - 3, ky0, ky0 + s - 3, -1, -1, &kx, &ky);
    orc_set_cell(e, kx, ky, ORC_KEY, door_c[gside][grow], 0);
    n = count_free(e, xl + 1, xr - 1, 1, H - 2, -1, -1);
    int ax, ay;
    kth_free(e, (int)orc_bounded(layout_draw(e, k++), (uint32_t)n), xl + 1, xr - 1, 1, H - 2, -1, -1, &ax, &ay);
    orc_set_agent(e, ax, ay, (int)orc_bounded(layout_draw(e, k++), 4u), 0, 0);
}

/* Candidate rivers of an S x S crossing layout: rows 2, 4, .., S-3 (kind 0,
 * horizontal), then columns 2, 4, .., S-3 (kind 1, vertical). */
static int crossing_candidates(int S, int* kind, int* pos)
{
    int m = 0;
    for (int y = 2; y <= S - 3; y += 2) {
        kind[m] = 0;
        pos[m] = y;
        m++;
    }
    for (int x = 2; x <= S - 3; x += 2) {
        kind[m] = 1;
        pos[m] = x;
        m++;
    }
    return m;
}

int32_t orc_max_variant(int32_t family, int32_t size)
{
    if (family == ORC_DISTSHIFT) return 1;
    /* KeyCorridor exists at S = 3(s-1)+1 for room sides s = 3..7, with 1..3
     * rows of rooms; -1 marks a size the family does not have */
    if (family == ORC_KEYCORRIDOR) return (size >= 7 && size % 3 == 1) ? 2 : -1;
    if (family != ORC_LAVA_CROSSING && family != ORC_SIMPLE_CROSSING) return 0;
    int kind[ORC_MAX_SIZE * 2], pos[ORC_MAX_SIZE * 2];
    return crossing_candidates(size, kind, pos);
}

static void sort_ints(int* v, int n)
{
    for (int i = 1; i < n; i++)
        for (int j = i; j > 0 && v[j - 1] > v[j]; j--) {
            int t = v[j];
            v[j] = v[j - 1];
            v[j - 1] = t;
        }
}

/* L7 Crossings-S with N rivers (the variant) of lava or wall; agent (1,1)
 * facing east, goal (S-2,S-2).  The layout draws, in this order:
 *  1. N rivers among the candidates by a partial Fisher-Yates shuffle
 *     (step i swaps candidate i with candidate i + k(d, m - i));
 *  2. every interior cell of a chosen row or column becomes the obstacle;
 *  3. a random order of the crossings: one east move per vertical river and
 *     one south move per horizontal river, shuffled by Fisher-Yates from the
 *     last position down (position i swaps with k(d, i + 1));
 *  4. walking that order from the top-left room, each move opens one cell of
 *     the river it crosses, drawn uniformly within the current room's span;
 * so the goal is always reachable and every river has exactly one opening. */
static void layout_crossing(orc_env* e)
{
    int S = e->width, N = e->variant;
    int obst_ent = e->family == ORC_LAVA_CROSSING ? ORC_LAVA : ORC_WALL;
    int obst_col = e->family == ORC_LAVA_CROSSING ? 0 : ORC_GREY;
    int kind[ORC_MAX_SIZE * 2], pos[ORC_MAX_SIZE * 2];
    int m = crossing_candidates(S, kind, pos);
    uint32_t k = 0;
    for (int i = 0; i < N; i++) {
        int j = i + (int)orc_bounded(layout_draw(e, k++), (uint32_t)(m - i));
        int tk = kind[i], tp = pos[i];
        kind[i] = kind[j];
        pos[i] = pos[j];
        kind[j] = tk;
        pos[j] = tp;
    }
    int hs[ORC_MAX_SIZE], vs[ORC_MAX_SIZE], nh = 0, nv = 0;
    for (int i = 0; i < N; i++) {
        if (kind[i] == 0)
            hs[nh++] = pos[i];
        else
            vs[nv++] = pos[i];
    }
    sort_ints(hs, nh);
    sort_ints(vs, nv);
    for (int i = 0; i < nh; i++)
        for (int x = 1; x <= S - 2; x++) orc_set_cell(e, x, hs[i], obst_ent, obst_col, 0);
    for (int i = 0; i < nv; i++)
        for (int y = 1; y <= S - 2; y++) orc_set_cell(e, vs[i], y, obst_ent, obst_col, 0);
    int path[ORC_MAX_SIZE * 2];  /* 1 = east (cross a vertical river), 0 = south */
    int L = nv + nh;
    for (int i = 0; i < L; i++) path[i] = i < nv ? 1 : 0;
    for (int i = L - 1; i >= 1; i--) {
        int j = (int)orc_bounded(layout_draw(e, k++), (uint32_t)(i + 1));
        int t = path[i];
        path[i] = path[j];
        path[j] = t;
    }
    int xb[ORC_MAX_SIZE + 2], yb[ORC_MAX_SIZE + 2];
    xb[0] = 0;
    for (int i = 0; i < nv; i++) xb[i + 1] = vs[i];
    xb[nv + 1] = S - 1;
    yb[0] = 0;
    for (int i = 0; i < nh; i++) yb[i + 1] = hs[i];
    yb[nh + 1] = S - 1;
    int rx = 0, ry = 0;
    for (int i = 0; i < L; i++) {
        if (path[i]) {
            int x = xb[rx + 1];
            int y = yb[ry] + 1 + (int)orc_bounded(layout_draw(e, k++), (uint32_t)(yb[ry + 1] - yb[ry] - 1));
            set_empty(e, x, y);
            rx++;
        } else {
            int y = yb[ry + 1];
            int x = xb[rx] + 1 + (int)orc_bounded(layout_draw(e, k++), (uint32_t)(xb[rx + 1] - xb[rx] - 1));
            set_empty(e, x, y);
            ry++;
        }
    }
    orc_set_cell(e, S - 2, S - 2, ORC_GOAL, ORC_GREEN, 0);
    orc_set_agent(e, 1, 1, 0, 0, 0);
}

/* L8 GoToDoor-S: four closed doors, one on each side of the border (never a
 * corner), in four distinct colours; the mission is one of them; the agent
 * on a drawn empty interior cell facing a drawn direction.  Draws, in order:
 * the door positions along the top, bottom, left and right walls (each in
 * 1..S-2), the colours by a partial Fisher-Yates shuffle of the six (step i
 * swaps colour i with colour i + k(d, 6 - i)), the target door k(d, 4), the
 * agent cell k(d, n) and its direction k(d, 4). */
static void layout_gotodoor(orc_env* e)
{
    int S = e->width;
    uint32_t k = 0;
    int px[4], py[4];
    int p0 = 1 + (int)orc_bounded(layout_draw(e, k++), (uint32_t)(S - 2));
    px[0] = p0;
    py[0] = 0;
    int p1 = 1 + (int)orc_bounded(layout_draw(e, k++), (uint32_t)(S - 2));
    px[1] = p1;
    py[1] = S - 1;
    int p2 = 1 + (int)orc_bounded(layout_draw(e, k++), (uint32_t)(S - 2));
    px[2] = 0;
    py[2] = p2;
    int p3 = 1 + (int)orc_bounded(layout_draw(e, k++), (uint32_t)(S - 2));
    px[3] = S - 1;
    py[3] = p3;
    int colours[6] = {0, 1, 2, 3, 4, 5};
    for (int i = 0; i < 4; i++) {
        int j = i + (int)orc_bounded(layout_draw(e, k++), (uint32_t)(6 - i));
        int t = colours[i];
        colours[i] = colours[j];
        colours[j] = t;
    }
    for (int i = 0; i < 4; i++) orc_set_cell(e, px[i], py[i], ORC_DOOR, colours[i], ORC_CLOSED);
    e->mission = colours[(int)orc_bounded(layout_draw(e, k++), 4u)];
    int n = count_free(e, 1, S - 2, 1, S - 2, -1, -1);
    int ax, ay;
    kth_free(e, (int)orc_bounded(layout_draw(e, k++), (uint32_t)n), 1, S - 2, 1, S - 2, -1, -1, &ax, &ay);
    orc_set_agent(e, ax, ay, (int)orc_bounded(layout_draw(e, k++), 4u), 0, 0);
}

void orc_set_costs(orc_env* e, float action_cost, float time_cost)
{
    e->action_cost = action_cost;
    e->time_cost = time_cost;
}

/* reset(key) of Section 3.2.2: sample a start state for the given episode. */
void orc_reset(orc_env* e, uint32_t episode)
{
    e->episode = episode;
    e->t = 0;
    e->done = 0;
    e->mission = ORC_NO_MISSION;
    e->carry_ent = 0;
    e->carry_col = 0;
    for (int b = 0; b < ORC_MAX_BALLS; b++) {
        e->ball_x[b] = 0;
        e->ball_y[b] = 0;
    }
    memset(e->ent, 0, sizeof e->ent);
    memset(e->col, 0, sizeof e->col);
    memset(e->st, 0, sizeof e->st);
    clear_grid(e);
    border_walls(e);
    switch (e->family) {
    case ORC_EMPTY: layout_empty(e); break;
    case ORC_DOORKEY: layout_doorkey(e); break;
    case ORC_FOURROOMS: layout_fourrooms(e); break;
    case ORC_LAVAGAP: layout_lavagap(e); break;
    case ORC_DYNOBS: layout_dynobs(e); break;
    case ORC_EMPTY_RANDOM: layout_empty_random(e); break;
    case ORC_LAVA_CROSSING:
    case ORC_SIMPLE_CROSSING: layout_crossing(e); break;
    case ORC_GOTODOOR: layout_gotodoor(e); break;
    case ORC_DISTSHIFT: layout_distshift(e); break;
    case ORC_KEYCORRIDOR: layout_keycorridor(e); break;
    default: break;
    }
}

int32_t orc_env_init(orc_env* e, int32_t family, int32_t size, int32_t max_steps, int32_t n_balls, uint64_t seed,
                     uint32_t env_index, int32_t reward_mode, float lava_reward, int32_t variant)
{
    if (family < ORC_EMPTY || family >= ORC_N_FAMILIES) return -1;
    if (size < ORC_MIN_SIZE || size > ORC_MAX_SIZE) return -1;
    if (n_balls < 0 || n_balls > ORC_MAX_BALLS) return -1;
    if (variant < 0 || variant > orc_max_variant(family, size)) return -1;
    memset(e, 0, sizeof *e);
    e->family = family;
    e->height = size;
    e->width = size;
    e->max_steps = max_steps > 0 ? max_steps : orc_default_max_steps(family, size);
    e->n_balls = family == ORC_DYNOBS ? n_balls : 0;
    e->reward_mode = reward_mode;
    e->lava_reward = lava_reward;
    e->action_cost = 0.0f;
    e->time_cost = 0.0f;
    e->seed = seed;
    e->env_index = env_index;
    e->variant = variant;
    orc_reset(e, 0);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Random actions (R1 purpose 3, R13): uniform over the 7 actions, or over
 * left/right/forward in Dynamic-Obstacles. */
int32_t orc_random_action(const orc_env* e, uint32_t gstep)
{
    uint32_t n_act = e->family == ORC_DYNOBS ? 3u : 7u;
    return (int32_t)orc_bounded(orc_draw(e->seed, e->env_index, 0xFFFFFFFFu, gstep, PURPOSE_ACTION, 0), n_act);
}

/* Transition system (Table 3, Appendix A) for Dynamic-Obstacles (R12): each
 * ball, in index order, moves to a uniformly drawn empty cell of its
 * 8-neighbourhood (never the agent's cell), else stays. */
static void move_balls(orc_env* e)
{
    for (int b = 0; b < e->n_balls; b++) {
        int bx = e->ball_x[b], by = e->ball_y[b];
        int cand_x[8], cand_y[8], count = 0;
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                if (dx == 0 && dy == 0) continue;
                int x = bx + dx, y = by + dy;
                if (!is_empty_cell(e, x, y)) continue;
                if (x == e->ax && y == e->ay) continue;
                cand_x[count] = x;
                cand_y[count] = y;
                count++;
            }
        if (count == 0) continue;
        uint32_t d = orc_draw(e->seed, e->env_index, e->episode, (uint32_t)e->t, PURPOSE_BALL, (uint32_t)b);
        int k = (int)orc_bounded(d, (uint32_t)count);
        set_empty(e, bx, by);
        orc_set_cell(e, cand_x[k], cand_y[k], ORC_BALL, ORC_BLUE, 0);
        e->ball_x[b] = cand_x[k];
        e->ball_y[b] = cand_y[k];
    }
}

/* Eq. 1 (Section 3.2.1) read as MiniGrid's success reward 1 - 0.9 t / T, with
 * t already counting this step; IEEE single operations in a fixed order:
 * multiply, divide, subtract (reading R15). */
static float minigrid_goal_reward(int t, int T)
{
    volatile float num = 0.9f * (float)t;
    volatile float q = num / (float)T;
    volatile float r = 1.0f - q;
    return r;
}

/* One env step in the order of reading R2 / the step-order list:
 * autoreset, transition, intervention, reward/termination, time, truncation.
 * The observation is produced separately from the resulting state. */
void orc_step(orc_env* e, int32_t action, float* reward, uint8_t* terminated, uint8_t* truncated)
{
    /* 1. autoreset (Section 3.2.2, Code 1): the call after a terminal or
     *    truncated step returns the new episode's start with reward padding 0
     *    and ignores its action. */
    if (e->done) {
        orc_reset(e, e->episode + 1);
        *reward = 0.0f;
        *terminated = 0;
        *truncated = 0;
        return;
    }
    /* 2. transition system */
    if (e->family == ORC_DYNOBS) move_balls(e);

    /* 3. intervention system (Table 3, Appendix A, readings R7-R11, R13) */
    int goal = 0, lava = 0, hit = 0;
    int n_act = e->family == ORC_DYNOBS ? 3 : 7;
    if (action < 0 || action > ORC_DONE) {
        e->invalid_action = 1; /* executed as a no-op */
    } else if (action < n_act) {
        int fx = e->ax + DX[e->dir], fy = e->ay + DY[e->dir];
        int fent, fcol, fst;
        get_cell(e, fx, fy, &fent, &fcol, &fst);
        if (action == ORC_LEFT) {
            e->dir = (e->dir + 3) % 4;
        } else if (action == ORC_RIGHT) {
            e->dir = (e->dir + 1) % 4;
        } else if (action == ORC_FORWARD) {
            if (e->family == ORC_DYNOBS && fent == ORC_BALL) {
                hit = 1; /* hit by an obstacle: the agent does not move */
            } else if (walkable(fent, fst)) {
                e->ax = fx;
                e->ay = fy;
                if (fent == ORC_GOAL) goal = 1;
                if (fent == ORC_LAVA) lava = 1;
            }
        } else if (action == ORC_PICKUP) {
            if (e->carry_ent == 0 && (fent == ORC_KEY || fent == ORC_BALL)) {
                e->carry_ent = fent;
                e->carry_col = fcol;
                set_empty(e, fx, fy);
            }
        } else if (action == ORC_DROP) {
            if (e->carry_ent != 0 && is_empty_cell(e, fx, fy)) {
                orc_set_cell(e, fx, fy, e->carry_ent, e->carry_col, 0);
                e->carry_ent = 0;
                e->carry_col = 0;
            }
        } else if (action == ORC_TOGGLE) {
            if (fent == ORC_DOOR) {
                if (fst == ORC_LOCKED) {
                    if (e->carry_ent == ORC_KEY && e->carry_col == fcol) orc_set_cell(e, fx, fy, ORC_DOOR, fcol, ORC_OPEN);
                } else if (fst == ORC_CLOSED) {
                    orc_set_cell(e, fx, fy, ORC_DOOR, fcol, ORC_OPEN);
                } else {
                    orc_set_cell(e, fx, fy, ORC_DOOR, fcol, ORC_CLOSED);
                }
            }
        }
        else if (action == ORC_DONE) {
            /* on_door_done (Tables 5 and 6): in GoToDoor, done while facing a
             * door of the mission's colour completes the task; elsewhere done
             * has no effect (reading R21) */
            if (e->family == ORC_GOTODOOR && fent == ORC_DOOR && fcol == e->mission) goal = 1;
        }
    }

    /* 4. time and truncation (R17) */
    e->t += 1;
    int trunc = e->t >= e->max_steps;

    /* 5. reward (Table 5, Table 8 R1/R2/R3; R14, R15) and termination
     *    (Table 6: terminate when the reward event fires) */
    float r = 0.0f;
    int term = 0;
    if (goal) {
        r = e->reward_mode == ORC_REWARD_MINIGRID ? minigrid_goal_reward(e->t, e->max_steps) : 1.0f;
        term = 1;
    } else if (lava) {
        r = e->lava_reward;
        term = 1;
    } else if (hit) {
        r = -1.0f;
        term = 1;
    }
    /* the shaping terms of Table 5 (reading R22): action_cost for every
     * action but done (an action in 0..5, whether or not it changes the
     * state), then time_cost, each subtracted in single precision */
    if (action >= 0 && action < ORC_DONE) r = r - e->action_cost;
    r = r - e->time_cost;
    *reward = r;
    *terminated = (uint8_t)term;
    *truncated = (uint8_t)trunc;
    e->done = term || trunc;
}

/* ------------------------------------------------------------------------ */
/* symbolic_first_person (Table 4): a 7x7x3 egocentric view.
 * View geometry (R3, R4): output cell (vx, vy), agent at (3, 6) looking
 * toward vy = 0, right hand toward +vx; world = pos + (6 - vy) F + (vx - 3) Rt
 * with F the facing direction and Rt the direction to its right.
 * Visibility (R6): rows are processed from the agent's row outward; a visible
 * transparent cell lights its side neighbour and the two cells ahead. */
static void view_cells(const orc_env* e, int vent[7][7], int vcol[7][7], int vst[7][7])
{
    int F = e->dir, Rt = (e->dir + 1) % 4;
    for (int vy = 0; vy < 7; vy++)
        for (int vx = 0; vx < 7; vx++) {
            int x = e->ax + (6 - vy) * DX[F] + (vx - 3) * DX[Rt];
            int y = e->ay + (6 - vy) * DY[F] + (vx - 3) * DY[Rt];
            if (vx == 3 && vy == 6) {
                /* the agent's own cell shows what it carries, else empty */
                if (e->carry_ent != 0) {
                    vent[vy][vx] = e->carry_ent;
                    vcol[vy][vx] = e->carry_col;
                } else {
                    vent[vy][vx] = ORC_EMPTYCELL;
                    vcol[vy][vx] = 0;
                }
                vst[vy][vx] = 0;
            } else {
                get_cell(e, x, y, &vent[vy][vx], &vcol[vy][vx], &vst[vy][vx]);
            }
        }
}

static void visibility(int vent[7][7], int vst[7][7], int vis[7][7])
{
    memset(vis, 0, sizeof(int) * 49);
    vis[6][3] = 1;
    for (int j = 6; j >= 0; j--) {
        for (int i = 0; i <= 5; i++) {
            if (!vis[j][i]) continue;
            if (!transparent(vent[j][i], vst[j][i])) continue;
            vis[j][i + 1] = 1;
            if (j > 0) {
                vis[j - 1][i + 1] = 1;
                vis[j - 1][i] = 1;
            }
        }
        for (int i = 6; i >= 1; i--) {
            if (!vis[j][i]) continue;
            if (!transparent(vent[j][i], vst[j][i])) continue;
            vis[j][i - 1] = 1;
            if (j > 0) {
                vis[j - 1][i - 1] = 1;
                vis[j - 1][i] = 1;
            }
        }
    }
}

void orc_obs_sym(const orc_env* e, uint8_t obs[ORC_OBS_BYTES])
{
    int vent[7][7], vcol[7][7], vst[7][7], vis[7][7];
    view_cells(e, vent, vcol, vst);
    visibility(vent, vst, vis);
    for (int vy = 0; vy < 7; vy++)
        for (int vx = 0; vx < 7; vx++) {
            uint8_t* o = obs + (vy * 7 + vx) * 3;
            if (vis[vy][vx]) {
                o[0] = (uint8_t)vent[vy][vx];
                o[1] = (uint8_t)vcol[vy][vx];
                o[2] = (uint8_t)vst[vy][vx];
            } else {
                o[0] = 0;
                o[1] = 0;
                o[2] = 0;
            }
        }
}

/* rgb_first_person (Table 4; Sprite component of Table 1): each view cell
 * becomes a 32x32x3 sprite.  Sprite atlas convention (the atlas is an input,
 * 397 tiles of 32x32x3 bytes): tile 0 = unseen; a visible cell (e, c, s) uses
 * tile 1 + 18 e + 3 c + s; the agent's own cell uses the same index + 198
 * (the agent drawn over what it carries). */
int32_t orc_tile_index(int32_t visible, int32_t agent_cell, int32_t ent, int32_t col, int32_t st)
{
    if (!visible) return 0;
    int32_t t = 1 + ent * 18 + col * 3 + st;
    if (agent_cell) t += 198;
    return t;
}

void orc_obs_rgb(const orc_env* e, const uint8_t* atlas, uint8_t* img)
{
    uint8_t obs[ORC_OBS_BYTES];
    orc_obs_sym(e, obs);
    const int row_bytes = 7 * ORC_TILE * 3;
    for (int vy = 0; vy < 7; vy++)
        for (int vx = 0; vx < 7; vx++) {
            const uint8_t* o = obs + (vy * 7 + vx) * 3;
            int visible = !(o[0] == 0 && o[1] == 0 && o[2] == 0);
            int agent_cell = (vx == 3 && vy == 6);
            int tile = orc_tile_index(visible, agent_cell, o[0], o[1], o[2]);
            const uint8_t* src = atlas + (size_t)tile * ORC_TILE_BYTES;
            for (int ty = 0; ty < ORC_TILE; ty++)
                for (int tx = 0; tx < ORC_TILE; tx++)
                    for (int c = 0; c < 3; c++)
                        img[(size_t)(vy * ORC_TILE + ty) * row_bytes + (size_t)(vx * ORC_TILE + tx) * 3 + c] =
                            src[(ty * ORC_TILE + tx) * 3 + c];
        }
}

/* symbolic (Table 4): the canonical grid encoding of the whole grid; the
 * agent's cell holds (agent, red, direction) in place of what lies under it
 * (reading R19).  categorical (Table 4): the entity code of every cell, the
 * agent's cell holding the agent code (reading R20).  Cells beyond the grid
 * (up to `side`) are 0. */
void orc_obs_full(const orc_env* e, uint8_t* full, int32_t side)
{
    for (int y = 0; y < side; y++)
        for (int x = 0; x < side; x++) {
            uint8_t* o = full + ((size_t)y * side + x) * 3;
            if (x >= e->width || y >= e->height) {
                o[0] = o[1] = o[2] = 0;
            } else if (x == e->ax && y == e->ay) {
                o[0] = ORC_AGENT;
                o[1] = ORC_RED;
                o[2] = (uint8_t)e->dir;
            } else {
                int i = idx(e, x, y);
                o[0] = e->ent[i];
                o[1] = e->col[i];
                o[2] = e->st[i];
            }
        }
}

void orc_obs_cat(const orc_env* e, uint8_t* cat, int32_t side)
{
    for (int y = 0; y < side; y++)
        for (int x = 0; x < side; x++) {
            uint8_t v = 0;
            if (x < e->width && y < e->height) v = (x == e->ax && y == e->ay) ? ORC_AGENT : e->ent[idx(e, x, y)];
            cat[(size_t)y * side + x] = v;
        }
}

void orc_obs_rgb_full(const orc_env* e, const uint8_t* atlas, uint8_t* img, int32_t side)
{
    uint8_t* full = (uint8_t*)malloc((size_t)side * side * 3);
    if (!full) return;
    orc_obs_full(e, full, side);
    const size_t row_bytes = (size_t)side * ORC_TILE * 3;
    for (int y = 0; y < side; y++)
        for (int x = 0; x < side; x++) {
            const uint8_t* f = full + ((size_t)y * side + x) * 3;
            int tile;
            if (x >= e->width || y >= e->height)
                tile = 0;
            else if (f[0] == ORC_AGENT)
                tile = 397 + f[2];
            else
                tile = 1 + 18 * f[0] + 3 * f[1] + f[2];
            const uint8_t* src = atlas + (size_t)tile * ORC_TILE_BYTES;
            for (int ty = 0; ty < ORC_TILE; ty++)
                for (int tx = 0; tx < ORC_TILE; tx++)
                    for (int c = 0; c < 3; c++)
                        img[(size_t)(y * ORC_TILE + ty) * row_bytes + (size_t)(x * ORC_TILE + tx) * 3 + c] =
                            src[(ty * ORC_TILE + tx) * 3 + c];
        }
    free(full);
}

/* categorical_first_person (Table 4): the entity codes of the egocentric view */
void orc_obs_cat_fp(const orc_env* e, uint8_t cat[ORC_VIEW * ORC_VIEW])
{
    uint8_t obs[ORC_OBS_BYTES];
    orc_obs_sym(e, obs);
    for (int c = 0; c < ORC_VIEW * ORC_VIEW; c++) cat[c] = obs[3 * c];
}

/* ------------------------------------------------------------------------ */
/* Batch convenience (vmap over environments, Code 3), stepped sequentially. */
struct orc_batch {
    int32_t n;
    uint32_t gstep; /* calls to step since the batch was reset */
    orc_env* envs;
};

orc_batch* orc_batch_create(int32_t n, const int32_t* family, const int32_t* size, const int32_t* max_steps,
                            const int32_t* variant, int32_t n_balls, uint64_t seed, uint32_t env_index_base,
                            int32_t reward_mode, float lava_reward)
{
    uint32_t* idx = (uint32_t*)malloc((n > 0 ? (size_t)n : 1u) * sizeof(uint32_t));
    if (!idx) return NULL;
    for (int32_t i = 0; i < n; i++) idx[i] = env_index_base + (uint32_t)i;
    orc_batch* b =
        orc_batch_create_indexed(n, family, size, max_steps, variant, n_balls, seed, idx, reward_mode, lava_reward);
    free(idx);
    return b;
}

orc_batch* orc_batch_create_indexed(int32_t n, const int32_t* family, const int32_t* size, const int32_t* max_steps,
                                    const int32_t* variant, int32_t n_balls, uint64_t seed, const uint32_t* env_index,
                                    int32_t reward_mode, float lava_reward)
{
    if (n < 0) return NULL;
    orc_batch* b = (orc_batch*)calloc(1, sizeof *b);
    if (!b) return NULL;
    b->n = n;
    b->envs = (orc_env*)calloc(n > 0 ? (size_t)n : 1u, sizeof(orc_env));
    if (!b->envs) {
        free(b);
        return NULL;
    }
    for (int32_t i = 0; i < n; i++) {
        if (orc_env_init(&b->envs[i], family[i], size[i], max_steps ? max_steps[i] : 0, n_balls, seed,
                         env_index[i], reward_mode, lava_reward, variant ? variant[i] : 0) != 0) {
            free(b->envs);
            free(b);
            return NULL;
        }
    }
    return b;
}

void orc_batch_destroy(orc_batch* b)
{
    if (!b) return;
    free(b->envs);
    free(b);
}

void orc_batch_set_costs(orc_batch* b, float action_cost, float time_cost)
{
    for (int32_t i = 0; i < b->n; i++) orc_set_costs(&b->envs[i], action_cost, time_cost);
}

orc_env* orc_batch_env(orc_batch* b, int32_t i) { return (i >= 0 && i < b->n) ? &b->envs[i] : NULL; }

uint32_t orc_batch_gstep(const orc_batch* b) { return b->gstep; }

static void emit(orc_env* e, int32_t i, uint8_t* obs_sym, uint8_t* obs_rgb, const uint8_t* atlas)
{
    if (obs_sym) orc_obs_sym(e, obs_sym + (size_t)i * ORC_OBS_BYTES);
    if (obs_rgb && atlas) orc_obs_rgb(e, atlas, obs_rgb + (size_t)i * ORC_RGB_BYTES);
}

void orc_batch_reset(orc_batch* b, uint8_t* obs_sym, uint8_t* obs_rgb, const uint8_t* atlas, float* reward,
                     uint8_t* terminated, uint8_t* truncated)
{
    b->gstep = 0;
    for (int32_t i = 0; i < b->n; i++) {
        orc_env* e = &b->envs[i];
        e->invalid_action = 0;
        orc_reset(e, 0);
        emit(e, i, obs_sym, obs_rgb, atlas);
        if (reward) reward[i] = 0.0f;
        if (terminated) terminated[i] = 0;
        if (truncated) truncated[i] = 0;
    }
}

void orc_batch_step(orc_batch* b, const int8_t* actions, uint8_t* obs_sym, uint8_t* obs_rgb, const uint8_t* atlas,
                    float* reward, uint8_t* terminated, uint8_t* truncated)
{
    for (int32_t i = 0; i < b->n; i++) {
        orc_env* e = &b->envs[i];
        int32_t a = actions ? (int32_t)actions[i] : orc_random_action(e, b->gstep);
        float r;
        uint8_t te, tr;
        orc_step(e, a, &r, &te, &tr);
        emit(e, i, obs_sym, obs_rgb, atlas);
        if (reward) reward[i] = r;
        if (terminated) terminated[i] = te;
        if (truncated) truncated[i] = tr;
    }
    b->gstep += 1;
}

void orc_batch_rollout(orc_batch* b, int32_t T, const int8_t* actions_TN, uint8_t* obs_sym, uint8_t* obs_rgb,
                       const uint8_t* atlas, float* reward, uint8_t* terminated, uint8_t* truncated)
{
    size_t n = (size_t)b->n;
    for (int32_t t = 0; t < T; t++) {
        orc_batch_step(b, actions_TN ? actions_TN + (size_t)t * n : NULL,
                       obs_sym ? obs_sym + (size_t)t * n * ORC_OBS_BYTES : NULL,
                       obs_rgb ? obs_rgb + (size_t)t * n * ORC_RGB_BYTES : NULL, atlas,
                       reward ? reward + (size_t)t * n : NULL, terminated ? terminated + (size_t)t * n : NULL,
                       truncated ? truncated + (size_t)t * n : NULL);
    }
}

void orc_batch_obs_full(orc_batch* b, uint8_t* full, uint8_t* cat, uint8_t* cat_fp, int32_t side)
{
    for (int32_t i = 0; i < b->n; i++) {
        const orc_env* e = &b->envs[i];
        if (full) orc_obs_full(e, full + (size_t)i * side * side * 3, side);
        if (cat) orc_obs_cat(e, cat + (size_t)i * side * side, side);
        if (cat_fp) orc_obs_cat_fp(e, cat_fp + (size_t)i * ORC_VIEW * ORC_VIEW);
    }
}

void orc_batch_obs_rgb_full(orc_batch* b, const uint8_t* atlas, uint8_t* img, int32_t side)
{
    const size_t per = (size_t)side * ORC_TILE * side * ORC_TILE * 3;
    for (int32_t i = 0; i < b->n; i++) orc_obs_rgb_full(&b->envs[i], atlas, img + (size_t)i * per, side);
}

/* ------------------------------------------------------------------------ */
/* The fused rollout's policy (reading P1): the integer MLP of orc_policy,
 * evaluated literally in 64-bit integers. */
static int64_t floor_shift(int64_t v, int32_t s)
{
    /* floor(v / 2^s) for negative v as well */
    int64_t d = (int64_t)1 << s;
    int64_t q = v / d;
    if (v % d != 0 && v < 0) q -= 1;
    return q;
}

static int64_t clamp255(int64_t v) { return v < 0 ? 0 : (v > 255 ? 255 : v); }

int32_t orc_policy_greedy(const orc_policy* p, int32_t agent, const uint8_t* cat_fp, int32_t n_act)
{
    const int8_t* w1 = p->w1 + (size_t)agent * ORC_HIDDEN * ORC_POLICY_IN;
    const int32_t* b1 = p->b1 + (size_t)agent * ORC_HIDDEN;
    const int8_t* w2 = p->w2 + (size_t)agent * ORC_HIDDEN * ORC_HIDDEN;
    const int32_t* b2 = p->b2 + (size_t)agent * ORC_HIDDEN;
    const int8_t* w3 = p->w3 + (size_t)agent * 7 * ORC_HIDDEN;
    const int32_t* b3 = p->b3 + (size_t)agent * 7;
    int64_t h1[ORC_HIDDEN], h2[ORC_HIDDEN];
    for (int j = 0; j < ORC_HIDDEN; j++) {
        int64_t acc = b1[j];
        for (int k = 0; k < ORC_POLICY_IN; k++) acc += (int64_t)w1[j * ORC_POLICY_IN + k] * cat_fp[k];
        h1[j] = clamp255(floor_shift(acc, p->shift1));
    }
    for (int j = 0; j < ORC_HIDDEN; j++) {
        int64_t acc = b2[j];
        for (int i = 0; i < ORC_HIDDEN; i++) acc += (int64_t)w2[j * ORC_HIDDEN + i] * h1[i];
        h2[j] = clamp255(floor_shift(acc, p->shift2));
    }
    int32_t best = 0;
    int64_t best_z = 0;
    for (int a = 0; a < n_act; a++) {
        int64_t z = b3[a];
        for (int i = 0; i < ORC_HIDDEN; i++) z += (int64_t)w3[a * ORC_HIDDEN + i] * h2[i];
        if (a == 0 || z > best_z) {
            best = a;
            best_z = z;
        }
    }
    return best;
}

int32_t orc_policy_action(const orc_policy* p, const orc_env* e, uint32_t gstep)
{
    int32_t n_act = e->family == ORC_DYNOBS ? 3 : 7;
    uint32_t coin = orc_draw(e->seed, e->env_index, 0xFFFFFFFEu, gstep, PURPOSE_EXPLORE, 0);
    if (coin < p->epsilon) return orc_random_action(e, gstep);
    uint8_t cat[ORC_VIEW * ORC_VIEW];
    orc_obs_cat_fp(e, cat);
    return orc_policy_greedy(p, (int32_t)(e->env_index / (uint32_t)p->envs_per_agent), cat, n_act);
}

void orc_batch_rollout_policy(orc_batch* b, int32_t T, const orc_policy* p, int8_t* actions_out, uint8_t* obs_sym,
                              float* reward, uint8_t* terminated, uint8_t* truncated)
{
    size_t n = (size_t)b->n;
    for (int32_t t = 0; t < T; t++) {
        for (int32_t i = 0; i < b->n; i++) {
            orc_env* e = &b->envs[i];
            /* the action is chosen from the current state's view (an env
             * about to autoreset ignores it) */
            int32_t a = orc_policy_action(p, e, b->gstep);
            float r;
            uint8_t te, tr;
            orc_step(e, a, &r, &te, &tr);
            size_t o = (size_t)t * n + (size_t)i;
            if (actions_out) actions_out[o] = (int8_t)a;
            if (obs_sym) orc_obs_sym(e, obs_sym + o * ORC_OBS_BYTES);
            if (reward) reward[o] = r;
            if (terminated) terminated[o] = te;
            if (truncated) truncated[o] = tr;
        }
        b->gstep += 1;
    }
}
