"""Pins of the oracle's Empty-Random and crossing layouts (Table 8 families
Empty-Random-S, LavaCrossing / SimpleCrossing S9N1-3, S11N5), CPU only.

* Empty-Random: the agent lands on every interior cell but the goal, facing
  every direction, and the rest of the room is the Empty layout;
* crossings: exactly N full rivers on even rows/columns, each with exactly one
  opening that is never on a river intersection, the goal reachable from the
  agent (an independent flood fill), every candidate river chosen over many
  episodes, and BFS-optimal plans (independent rule model) reaching the goal
  with reward 1.0 at the plan's length.
"""
from collections import deque

import numpy as np
import pytest

import oracle as O
from tests import indep_model as M


def test_empty_random_covers_cells_and_directions():
    S = 6
    cells, dirs = set(), set()
    for ep in range(600):
        e = O.Env(O.EMPTY_RANDOM, S, seed=3)
        e.reset(ep)
        ent, _, _ = e.grid()
        assert ent[S - 2, S - 2] == 8 and (ent[1:S - 1, 1:S - 1] != 2).all()
        assert (e.s.ax, e.s.ay) != (S - 2, S - 2) and ent[e.s.ay, e.s.ax] == 1
        cells.add((e.s.ax, e.s.ay))
        dirs.add(e.s.dir)
    assert len(cells) == (S - 2) ** 2 - 1 and dirs == {0, 1, 2, 3}


def _reachable(ent, start, goal, blocked=(2, 9)):
    S = ent.shape[0]
    seen = {start}
    q = deque([start])
    while q:
        x, y = q.popleft()
        if (x, y) == goal:
            return True
        for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            nx_, ny_ = x + dx, y + dy
            if 0 <= nx_ < S and 0 <= ny_ < S and (nx_, ny_) not in seen and ent[ny_, nx_] not in blocked:
                seen.add((nx_, ny_))
                q.append((nx_, ny_))
    return False


@pytest.mark.parametrize("family,obst", [(O.LAVA_CROSSING, 9), (O.SIMPLE_CROSSING, 2)])
def test_crossing_layouts_are_valid(family, obst):
    for S in (5, 7, 9, 11, 13, 19):
        for N in range(0, O.max_variant(family, S) + 1):
            for seed in range(6):
                e = O.Env(family, S, seed=seed, env_index=N, variant=N)
                ent, col, st = e.grid()
                inner = ent[1:S - 1, 1:S - 1]
                rows = [y for y in range(1, S - 1) if (ent[y, 1:S - 1] == obst).sum() >= S - 3]
                cols = [x for x in range(1, S - 1) if (ent[1:S - 1, x] == obst).sum() >= S - 3]
                # a chosen river is a full interior line except its one opening
                # (and except crossings with perpendicular rivers' openings)
                rivers = [("h", y) for y in rows] + [("v", x) for x in cols]
                assert len(rivers) == N, (S, N, seed, rivers)
                for kind, p in rivers:
                    assert p % 2 == 0 and 2 <= p <= S - 3
                n_open = 0
                for kind, p in rivers:
                    line = ent[p, 1:S - 1] if kind == "h" else ent[1:S - 1, p]
                    opens = [i + 1 for i, v in enumerate(line) if v != obst]
                    assert len(opens) == 1, (kind, p, opens)
                    o = opens[0]
                    # the opening is not on a perpendicular river
                    assert o not in (cols if kind == "h" else rows)
                    n_open += 1
                assert n_open == N
                assert (inner[(inner != obst)] == 1).sum() + (inner == 8).sum() == (inner != obst).sum()
                assert (e.s.ax, e.s.ay, e.s.dir) == (1, 1, 0) and ent[S - 2, S - 2] == 8
                assert _reachable(ent, (1, 1), (S - 2, S - 2))
                if family == O.LAVA_CROSSING and N:
                    assert (col[ent == 9] == 0).all()


def test_crossing_choices_cover_every_river_and_opening():
    S, N = 9, 2
    chosen, openings = set(), set()
    for ep in range(400):
        e = O.Env(O.SIMPLE_CROSSING, S, seed=5, variant=N)
        e.reset(ep)
        ent, _, _ = e.grid()
        for y in range(2, S - 2, 2):
            line = ent[y, 1:S - 1]
            if (line == 2).sum() >= S - 3:
                chosen.add(("h", y))
                openings.add(("h", y, int(np.argwhere(line != 2)[0][0]) + 1))
        for x in range(2, S - 2, 2):
            line = ent[1:S - 1, x]
            if (line == 2).sum() >= S - 3:
                chosen.add(("v", x))
                openings.add(("v", x, int(np.argwhere(line != 2)[0][0]) + 1))
    assert chosen == {(k, p) for k in "hv" for p in (2, 4, 6)}
    assert len(openings) >= 24


@pytest.mark.parametrize("family,size,n,seed", [(O.SIMPLE_CROSSING, 7, 2, 1), (O.LAVA_CROSSING, 7, 2, 2),
                                                (O.SIMPLE_CROSSING, 9, 3, 3), (O.EMPTY_RANDOM, 6, 0, 4)])
def test_bfs_plans_solve_new_families(family, size, n, seed):
    env = O.Env(family, size, seed=seed, variant=n)
    ent, col, st = env.grid()
    cells = tuple((int(ent[y, x]), int(col[y, x]), int(st[y, x])) for y in range(size) for x in range(size))
    plan = M.bfs_goal((env.s.ax, env.s.ay, env.s.dir, None, cells), size, size, max_depth=60)
    assert plan is not None
    c = O.Env.__new__(O.Env)
    c.s = O.OrcEnv.from_buffer_copy(bytes(env.s))
    for i, a in enumerate(plan):
        r, te, tr = c.step(a)
        if i < len(plan) - 1:
            assert (r, te) == (0.0, 0)
    assert (r, te) == (1.0, 1) and c.s.t == len(plan)


@pytest.mark.parametrize("family,size,n", [(O.EMPTY_RANDOM, 8, 0), (O.LAVA_CROSSING, 9, 1), (O.LAVA_CROSSING, 11, 5),
                                           (O.SIMPLE_CROSSING, 9, 3), (O.SIMPLE_CROSSING, 19, 9)])
def test_new_family_rollout_invariants(family, size, n):
    b = O.Batch([family] * 12, [size] * 12, seed=7, variants=[n] * 12)
    b.reset()
    for t in range(600):
        o = b.step()
        for i in range(12):
            s = b.state(i)
            ent = np.frombuffer(s["ent"], np.uint8).reshape(size, size)
            x, y = s["x"], s["y"]
            assert ent[y, x] in (1, 8, 9)
            if o["terminated"][i]:
                assert ent[y, x] in (8, 9)
                assert o["reward"][i] == (1.0 if ent[y, x] == 8 else 0.0)


def test_invalid_variants_rejected():
    with pytest.raises(ValueError):
        O.Env(O.LAVA_CROSSING, 9, variant=7)  # 6 candidate rivers at S = 9
    with pytest.raises(ValueError):
        O.Env(O.EMPTY, 9, variant=1)
    assert O.max_variant(O.SIMPLE_CROSSING, 11) == 8 and O.max_variant(O.LAVA_CROSSING, 5) == 2
