"""An independent, deliberately different restatement of the view and the rules,
used only to pin the oracle on tiny inputs (brute force).

It shares nothing with the oracle: the egocentric view is cut out of a padded
grid and turned with ``numpy.rot90`` (instead of the oracle's per-cell
world-coordinate formula), the occlusion pass runs on a column-major
``mask[i, j]`` array, and the rules work on an immutable tuple state for a
breadth-first search.
"""
from __future__ import annotations

from collections import deque

import numpy as np

WALL = (2, 5, 0)
EMPTY = (1, 0, 0)


def egocentric_slice(ent, col, st, ax, ay, d, carry=None):
    """7x7x3 view, rows = distance ahead (row 0 farthest), agent at row 6 col 3.

    ent/col/st are [H, W] arrays (row = y).  The 7x7 window is taken in world
    coordinates so that the agent sits on the window's edge facing inward, and
    the window is then rotated counter-clockwise (dir + 1) quarter turns, which
    brings the facing direction to "up".
    """
    H, W = ent.shape
    pad = 8
    g = np.zeros((H + 2 * pad, W + 2 * pad, 3), np.int64)
    g[:, :] = WALL
    g[pad:pad + H, pad:pad + W, 0] = ent
    g[pad:pad + H, pad:pad + W, 1] = col
    g[pad:pad + H, pad:pad + W, 2] = st
    # window origin (top-left, world x/y) for each facing direction
    if d == 0:  # east: agent on the window's left edge, middle row
        x0, y0 = ax, ay - 3
    elif d == 1:  # south: agent on the top edge, middle column
        x0, y0 = ax - 3, ay
    elif d == 2:  # west: right edge
        x0, y0 = ax - 6, ay - 3
    else:  # north: bottom edge
        x0, y0 = ax - 3, ay - 6
    win = g[pad + y0:pad + y0 + 7, pad + x0:pad + x0 + 7].copy()
    win = np.rot90(win, k=(d + 1) % 4, axes=(0, 1)).copy()
    win[6, 3] = EMPTY if carry is None else (carry[0], carry[1], 0)
    return win


def occlusion(view):
    """Visibility mask [7, 7] (row, col) computed column-major as mask[i, j]."""
    def see_behind(c):
        e, _, s = (int(v) for v in c)
        if e == 2:
            return False
        if e == 4 and s != 0:
            return False
        return True

    cells = view.transpose(1, 0, 2)  # cells[i, j] = view[j, i]
    mask = np.zeros((7, 7), bool)
    mask[3, 6] = True
    for j in range(6, -1, -1):
        for i in range(0, 6):
            if mask[i, j] and see_behind(cells[i, j]):
                mask[i + 1, j] = True
                if j > 0:
                    mask[i + 1, j - 1] = True
                    mask[i, j - 1] = True
        for i in range(6, 0, -1):
            if mask[i, j] and see_behind(cells[i, j]):
                mask[i - 1, j] = True
                if j > 0:
                    mask[i - 1, j - 1] = True
                    mask[i, j - 1] = True
    return mask.T  # back to [row, col]


def observe(ent, col, st, ax, ay, d, carry=None):
    v = egocentric_slice(ent, col, st, ax, ay, d, carry)
    m = occlusion(v)
    out = np.where(m[:, :, None], v, 0)
    return out.astype(np.uint8)


# ---------------------------------------------------------------------------
# rules for breadth-first search; a state is (x, y, d, carry, cells) where
# cells is a tuple of (ent, col, st) triples, row-major.
STEP = {0: (1, 0), 1: (0, 1), 2: (-1, 0), 3: (0, -1)}


def successors(state, W, H, n_actions=6, mission=None):
    """Yield (action, next_state, event) with event in {None, 'goal', 'lava'}.

    With a mission colour, action 6 (done) facing a door of that colour is
    the goal event (GoToDoor's on_door_done)."""
    x, y, d, carry, cells = state
    dx, dy = STEP[d]
    fx, fy = x + dx, y + dy
    inside = 0 <= fx < W and 0 <= fy < H
    f = cells[fy * W + fx] if inside else WALL
    # 0 / 1: turn
    yield 0, (x, y, (d + 3) % 4, carry, cells), None
    yield 1, (x, y, (d + 1) % 4, carry, cells), None
    # 2: forward
    passable = f[0] in (1, 3, 8, 9) or (f[0] == 4 and f[2] == 0)
    if passable:
        ev = "goal" if f[0] == 8 else ("lava" if f[0] == 9 else None)
        yield 2, (fx, fy, d, carry, cells), ev
    else:
        yield 2, state, None
    # 3: pickup keys and balls with an empty hand
    if carry is None and f[0] in (5, 6):
        c = list(cells)
        c[fy * W + fx] = EMPTY
        yield 3, (x, y, d, (f[0], f[1]), tuple(c)), None
    # 4: drop onto an empty cell
    if carry is not None and inside and f == EMPTY:
        c = list(cells)
        c[fy * W + fx] = (carry[0], carry[1], 0)
        yield 4, (x, y, d, None, tuple(c)), None
    # 5: toggle a door
    if f[0] == 4:
        if f[2] == 2:
            new = 0 if (carry is not None and carry[0] == 5 and carry[1] == f[1]) else 2
        else:
            new = 1 - f[2]
        if new != f[2]:
            c = list(cells)
            c[fy * W + fx] = (4, f[1], new)
            yield 5, (x, y, d, carry, tuple(c)), None
    # 6: done, facing the mission's door
    if mission is not None and f[0] == 4 and f[1] == mission:
        yield 6, state, "goal"


def bfs_goal(start, W, H, max_depth=64, mission=None):
    """Shortest action sequence to a goal event (lava ends a path)."""
    q = deque([start])
    parent = {start: None}
    while q:
        s = q.popleft()
        depth = 0
        p = s
        while parent[p] is not None:
            depth += 1
            p = parent[p][0]
        if depth >= max_depth:
            continue
        for a, n, ev in successors(s, W, H, mission=mission):
            if ev == "goal":
                plan = [a]
                p = s
                while parent[p] is not None:
                    plan.append(parent[p][1])
                    p = parent[p][0]
                return plan[::-1]
            if ev == "lava":
                continue
            if n not in parent:
                parent[n] = (s, a)
                q.append(n)
    return None


# ---------------------------------------------------------------------------
# Counter-based draws (reading R1), restated with Python integers from the
# definition of Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds,
# each two 32x32 -> 64-bit products whose high halves are mixed with the other
# two words and the round key; the key advances by the Weyl constants.  It
# shares nothing with the oracle and is pinned by the published known-answer
# vectors (tests/golden/philox4x32_10_kat.txt).
_U32 = 0xFFFFFFFF
_MULT = (0xD2511F53, 0xCD9E8D57)
_WEYL = (0x9E3779B9, 0xBB67AE85)


def philox4x32_10(ctr, key):
    x = [int(v) & _U32 for v in ctr]
    k = [int(v) & _U32 for v in key]
    for _ in range(10):
        (hi0, lo0), (hi1, lo1) = divmod(_MULT[0] * x[0], 1 << 32), divmod(_MULT[1] * x[2], 1 << 32)
        x = [hi1 ^ x[1] ^ k[0], lo1, hi0 ^ x[3] ^ k[1], lo0]
        k = [(k[0] + _WEYL[0]) & _U32, (k[1] + _WEYL[1]) & _U32]
    return x


LAYOUT, BALL, ACTION = 1, 2, 3  # the purposes of reading R1


def draw(seed, env, episode, step, purpose, k):
    """Word 0 at counter (env, episode, step, purpose << 24 | k), key (seed lo, seed hi)."""
    return philox4x32_10([env, episode, step, (purpose << 24) | k], [seed & _U32, seed >> 32])[0]


def bounded(x, n):
    """floor(x n / 2^32): a draw in [0, n) (reading R1)."""
    return (int(x) * int(n)) >> 32


def random_action(seed, env, gstep, n_actions=7):
    """Random-action mode: the episode word is all ones, the step word the
    step count since the reset call (reading R1, purpose 3; R13)."""
    return bounded(draw(seed, env, 0xFFFFFFFF, gstep, ACTION, 0), n_actions)


# ---------------------------------------------------------------------------
# Layout generators L2, L3, L5 and the ball moves of reading R12, restated on a
# numpy grid [H, W, 3] of (entity, colour, state).  Free cells of a rectangle
# are listed by numpy.argwhere, whose order is C order over (y, x): rows
# outer, columns inner, the row-major order of reading R18.
GOAL = (8, 1, 0)
LOCKED_YELLOW_DOOR = (4, 4, 2)
YELLOW_KEY = (5, 4, 0)
BLUE_BALL = (6, 2, 0)


def walled_grid(S):
    g = np.zeros((S, S, 3), np.int64)
    g[:, :] = EMPTY
    g[0, :] = WALL
    g[-1, :] = WALL
    g[:, 0] = WALL
    g[:, -1] = WALL
    return g


def free_cells(g, x0, x1, y0, y1, skip=None):
    """Empty cells of [x0, x1] x [y0, y1] as (x, y), rows outer (reading R18)."""
    sub = g[y0:y1 + 1, x0:x1 + 1]
    mask = np.all(sub == np.array(EMPTY), axis=2)
    out = [(int(x0 + c[1]), int(y0 + c[0])) for c in np.argwhere(mask)]
    return [c for c in out if c != skip]


def doorkey_start(S, seed, env, episode):
    """L2; returns (grid, agent (x, y, dir), wall column, door (x, y), key (x, y), draws)."""
    d = [draw(seed, env, episode, 0, LAYOUT, k) for k in range(5)]
    g = walled_grid(S)
    g[S - 2, S - 2] = GOAL
    xw = 2 + bounded(d[0], S - 4)
    g[1:S - 1, xw] = WALL
    door = (xw, 1 + bounded(d[1], S - 3))
    g[door[1], door[0]] = LOCKED_YELLOW_DOOR
    cells = free_cells(g, 1, xw - 1, 1, S - 2)
    ax, ay = cells[bounded(d[2], len(cells))]
    adir = bounded(d[3], 4)
    rest = [c for c in cells if c != (ax, ay)]
    key = rest[bounded(d[4], len(rest))]
    g[key[1], key[0]] = YELLOW_KEY
    return g, (ax, ay, adir), xw, door, key, d


def fourrooms_start(S, seed, env, episode):
    """L3; returns (grid, agent (x, y, dir), goal (x, y), gaps, draws)."""
    d = [draw(seed, env, episode, 0, LAYOUT, k) for k in range(7)]
    m = S // 2
    g = walled_grid(S)
    g[:, m] = WALL
    g[m, :] = WALL
    gaps = [(m, 1 + bounded(d[0], m - 1)), (m, m + 1 + bounded(d[1], S - 2 - m)),
            (1 + bounded(d[2], m - 1), m), (m + 1 + bounded(d[3], S - 2 - m), m)]
    for x, y in gaps:
        g[y, x] = EMPTY
    cells = free_cells(g, 1, S - 2, 1, S - 2)
    goal = cells[bounded(d[4], len(cells))]
    g[goal[1], goal[0]] = GOAL
    rest = [c for c in cells if c != goal]
    ax, ay = rest[bounded(d[5], len(rest))]
    return g, (ax, ay, bounded(d[6], 4)), goal, gaps, d


def dynobs_start(S, seed, env, episode, n_balls=4):
    """L5; returns (grid, balls [(x, y)], draws)."""
    g = walled_grid(S)
    g[S - 2, S - 2] = GOAL
    balls, ds = [], []
    for b in range(n_balls):
        cells = free_cells(g, 1, S - 2, 1, S - 2, skip=(1, 1))
        ds.append(draw(seed, env, episode, 0, LAYOUT, b))
        x, y = cells[bounded(ds[-1], len(cells))]
        g[y, x] = BLUE_BALL
        balls.append((x, y))
    return g, balls, ds


# the 8-neighbourhood in reading R12's candidate order: dy outer, dx inner
NEIGHBOURS = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dx, dy) != (0, 0)]


def move_balls(g, balls, agent_xy, seed, env, episode, t):
    """R12: balls in index order, each onto a drawn free neighbour (empty, not
    the agent's cell) of the grid as the earlier balls left it.  Returns the
    new positions and, per ball, (candidates, draw)."""
    H, W = g.shape[:2]
    balls = list(balls)
    trace = []
    for b, (bx, by) in enumerate(balls):
        cand = [(bx + dx, by + dy) for dx, dy in NEIGHBOURS
                if 0 <= bx + dx < W and 0 <= by + dy < H and tuple(g[by + dy, bx + dx]) == EMPTY
                and (bx + dx, by + dy) != tuple(agent_xy)]
        x = draw(seed, env, episode, t, BALL, b)
        trace.append((cand, x))
        if not cand:
            continue
        nx_, ny_ = cand[bounded(x, len(cand))]
        g[by, bx] = EMPTY
        g[ny_, nx_] = BLUE_BALL
        balls[b] = (nx_, ny_)
    return balls, trace


# ---------------------------------------------------------------------------
# The other layout generators (L4, L6-L10), restated the same way.  Each
# consumes the layout draws k = 0, 1, 2, ... of its episode in the order its
# reading states, through a small stream object.
LAVA = (9, 0, 0)
GREY_WALL = WALL


class _Draws:
    """The layout draws of one episode, handed out in order."""

    def __init__(self, seed, env, episode):
        self.seed, self.env, self.episode, self.k = seed, env, episode, 0
        self.words = []

    def below(self, n):
        w = draw(self.seed, self.env, self.episode, 0, LAYOUT, self.k)
        self.k += 1
        self.words.append(w)
        return bounded(w, n)


def lavagap_start(S, seed, env, episode):
    """L4: a lava column at 2 + k(S - 4) with one gap at row 1 + k(S - 2)."""
    r = _Draws(seed, env, episode)
    g = walled_grid(S)
    g[S - 2, S - 2] = GOAL
    xl = 2 + r.below(S - 4)
    gap = 1 + r.below(S - 2)
    for y in range(1, S - 1):
        if y != gap:
            g[y, xl] = LAVA
    return g, (1, 1, 0)


def empty_random_start(S, seed, env, episode):
    """L6: Empty-S with the agent on the k-th free interior cell, a drawn direction."""
    r = _Draws(seed, env, episode)
    g = walled_grid(S)
    g[S - 2, S - 2] = GOAL
    cells = free_cells(g, 1, S - 2, 1, S - 2)
    ax, ay = cells[r.below(len(cells))]
    return g, (ax, ay, r.below(4))


def gotodoor_start(S, seed, env, episode):
    """L8: closed doors at drawn places on the top, bottom, left and right
    walls; colours from the first four of a partial shuffle of the six; the
    mission one of the four; the agent on a free interior cell."""
    r = _Draws(seed, env, episode)
    g = walled_grid(S)
    spots = [(1 + r.below(S - 2), 0), (1 + r.below(S - 2), S - 1), (0, 1 + r.below(S - 2)),
             (S - 1, 1 + r.below(S - 2))]
    palette = list(range(6))
    for i in range(4):
        j = i + r.below(6 - i)
        palette[i], palette[j] = palette[j], palette[i]
    for (x, y), c in zip(spots, palette[:4]):
        g[y, x] = (4, c, 1)
    mission = palette[r.below(4)]
    cells = free_cells(g, 1, S - 2, 1, S - 2)
    ax, ay = cells[r.below(len(cells))]
    return g, (ax, ay, r.below(4)), mission


def crossing_start(S, n_rivers, obstacle, seed, env, episode):
    """L7: n_rivers of the candidate rivers (rows 2, 4, .., S-3, then columns
    2, 4, .., S-3) by a partial shuffle, filled with the obstacle; the
    crossing order (east per column river, south per row river) shuffled from
    the last position down; walking it from the top-left room opens one cell
    of each river within the current room's span."""
    r = _Draws(seed, env, episode)
    g = walled_grid(S)
    cand = [("row", y) for y in range(2, S - 2, 2)] + [("col", x) for x in range(2, S - 2, 2)]
    for i in range(n_rivers):
        j = i + r.below(len(cand) - i)
        cand[i], cand[j] = cand[j], cand[i]
    rows = sorted(p for kind, p in cand[:n_rivers] if kind == "row")
    cols = sorted(p for kind, p in cand[:n_rivers] if kind == "col")
    for y in rows:
        g[y, 1:S - 1] = obstacle
    for x in cols:
        g[1:S - 1, x] = obstacle
    order = ["east"] * len(cols) + ["south"] * len(rows)
    for i in range(len(order) - 1, 0, -1):
        j = r.below(i + 1)
        order[i], order[j] = order[j], order[i]
    xs, ys = [0] + cols + [S - 1], [0] + rows + [S - 1]
    room_x = room_y = 0
    for move in order:
        if move == "east":
            room_x += 1
            g[ys[room_y] + 1 + r.below(ys[room_y + 1] - ys[room_y] - 1), xs[room_x]] = EMPTY
        else:
            room_y += 1
            g[ys[room_y], xs[room_x] + 1 + r.below(xs[room_x + 1] - xs[room_x] - 1)] = EMPTY
    g[S - 2, S - 2] = GOAL
    return g, (1, 1, 0)


def keycorridor_start(S, variant, seed, env, episode):
    """L10: a 3 x R block of rooms of side s (S = 3(s-1) + 1, R = variant + 1)
    whose middle column is an open corridor; a door per side room (rows, then
    colours, drawn left rooms first); the goal's side and room row, the key's
    room row; goal and key on free cells of their rooms (the key in a room on
    the other side, of the locked door's colour); the agent in the corridor."""
    r = _Draws(seed, env, episode)
    s, R = (S - 1) // 3 + 1, variant + 1
    H = (s - 1) * R + 1
    left, right = s - 1, 2 * (s - 1)
    g = walled_grid(S)
    g[H - 1:, :] = WALL
    g[:, left] = WALL
    g[:, right] = WALL
    for y in range(0, H, s - 1):  # the walls between rooms, open in the corridor
        g[y, :left + 1] = WALL
        g[y, right:] = WALL
    door_rows = [[j * (s - 1) + 1 + r.below(s - 2) for j in range(R)] for _ in range(2)]
    door_cols = [[r.below(6) for _ in range(R)] for _ in range(2)]
    gside, grow, krow = r.below(2), r.below(R), r.below(R)
    for side, x in ((0, left), (1, right)):
        for j in range(R):
            g[door_rows[side][j], x] = (4, door_cols[side][j], 2 if (side, j) == (gside, grow) else 1)

    def room(side, row):
        x0 = 1 if side == 0 else right + 1
        y0 = row * (s - 1) + 1
        return free_cells(g, x0, x0 + s - 3, y0, y0 + s - 3)

    cells = room(gside, grow)
    gx, gy = cells[r.below(len(cells))]
    g[gy, gx] = GOAL
    cells = room(1 - gside, krow)
    kx, ky = cells[r.below(len(cells))]
    g[ky, kx] = (5, door_cols[gside][grow], 0)
    cells = free_cells(g, left + 1, right - 1, 1, H - 2)
    ax, ay = cells[r.below(len(cells))]
    return g, (ax, ay, r.below(4))
