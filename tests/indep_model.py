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
