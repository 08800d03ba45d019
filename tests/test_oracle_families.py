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


# --- GoToDoor-S (Table 8; on_door_done of Tables 5 and 6) ---------------------

def _doors(ent, col, st):
    S = ent.shape[0]
    ys, xs = np.nonzero(ent == 4)
    return [(int(x), int(y), int(col[y, x]), int(st[y, x])) for x, y in zip(xs, ys)]


def test_gotodoor_layouts_are_valid():
    for S in (5, 6, 8, 11, 19):
        for seed in range(25):
            e = O.Env(O.GOTODOOR, S, seed=seed, env_index=seed)
            ent, col, st = e.grid()
            doors = _doors(ent, col, st)
            assert len(doors) == 4
            sides = set()
            for x, y, c, s in doors:
                assert s == 1  # closed
                assert (x in (0, S - 1)) != (y in (0, S - 1))  # on a wall, never a corner
                sides.add("top" if y == 0 else "bottom" if y == S - 1 else "left" if x == 0 else "right")
            assert sides == {"top", "bottom", "left", "right"}
            colours = [c for *_, c, _ in doors]
            assert len(set(colours)) == 4 and all(0 <= c <= 5 for c in colours)
            assert e.s.mission in colours
            # no goal, an empty interior, walls elsewhere on the border
            assert (ent != 8).all() and (ent[1:S - 1, 1:S - 1] == 1).all()
            border = np.ones((S, S), bool)
            border[1:S - 1, 1:S - 1] = False
            assert ((ent == 2) | (ent == 4))[border].all() and (ent == 2)[border].sum() == 4 * (S - 1) - 4
            assert 1 <= e.s.ax <= S - 2 and 1 <= e.s.ay <= S - 2 and 0 <= e.s.dir < 4
            assert e.s.max_steps == 5 * S * S


def test_gotodoor_draws_cover_their_ranges():
    S = 6
    pos = {k: set() for k in ("top", "bottom", "left", "right")}
    col_side = set()
    target_sides, agents, dirs, missions = set(), set(), set(), set()
    for ep in range(1500):
        e = O.Env(O.GOTODOOR, S, seed=11)
        e.reset(ep)
        ent, col, st = e.grid()
        for x, y, c, _ in _doors(ent, col, st):
            side = "top" if y == 0 else "bottom" if y == S - 1 else "left" if x == 0 else "right"
            pos[side].add(x if side in ("top", "bottom") else y)
            col_side.add((side, c))
            if c == e.s.mission:
                target_sides.add(side)
        agents.add((e.s.ax, e.s.ay))
        dirs.add(e.s.dir)
        missions.add(e.s.mission)
    assert all(v == set(range(1, S - 1)) for v in pos.values())
    assert len(col_side) == 24  # every colour on every side
    assert target_sides == {"top", "bottom", "left", "right"}
    assert missions == set(range(6)) and dirs == {0, 1, 2, 3} and len(agents) == (S - 2) ** 2


def _plan_to_door(env, S):
    ent, col, st = env.grid()
    cells = tuple((int(ent[y, x]), int(col[y, x]), int(st[y, x])) for y in range(S) for x in range(S))
    return M.bfs_goal((env.s.ax, env.s.ay, env.s.dir, None, cells), S, S, max_depth=40, mission=env.s.mission)


@pytest.mark.parametrize("S,seed,mode", [(5, 0, 0), (6, 1, 0), (8, 2, 1), (8, 3, 0), (11, 4, 1)])
def test_gotodoor_done_at_the_mission_door_ends_with_reward(S, seed, mode):
    env = O.Env(O.GOTODOOR, S, seed=seed, reward_mode=mode)
    plan = _plan_to_door(env, S)
    assert plan is not None and plan[-1] == 6
    T = env.s.max_steps
    for i, a in enumerate(plan):
        r, te, tr = env.step(a)
        if i < len(plan) - 1:
            assert (r, te) == (0.0, 0)
    want = 1.0 if mode == 0 else float(np.float32(1.0) - np.float32(np.float32(0.9) * np.float32(len(plan))) / np.float32(T))
    assert (te, tr) == (1, 0) and r == pytest.approx(want, abs=0) and env.s.t == len(plan)
    # the next call starts a new episode with reward padding 0
    assert env.step(2) == (0.0, 0, 0) and env.s.t == 0 and env.s.episode == 1


def test_gotodoor_done_elsewhere_does_nothing():
    S = 7
    for seed in range(30):
        env = O.Env(O.GOTODOOR, S, seed=seed)
        ent, col, st = env.grid()
        doors = {(x, y): c for x, y, c, _ in _doors(ent, col, st)}
        # walk straight ahead, saying done at every cell on the way
        for _ in range(S):
            fx = env.s.ax + (1, 0, -1, 0)[env.s.dir]
            fy = env.s.ay + (0, 1, 0, -1)[env.s.dir]
            facing = doors.get((fx, fy))
            before = (env.s.ax, env.s.ay, env.s.dir, bytes(env.s.ent))
            r, te, tr = env.step(6)
            if facing == env.s.mission:
                assert (r, te) == (1.0, 1)
                break
            assert (r, te, tr) == (0.0, 0, 0)
            assert (env.s.ax, env.s.ay, env.s.dir, bytes(env.s.ent)) == before
            env.step(2)
    # done never rewards in a family without a mission, even facing a door
    e = O.Env(O.DOORKEY, 5, seed=0)
    e.set_cell(2, 1, 4, 4, 1)
    e.set_agent(1, 1, 0)
    assert e.step(6) == (0.0, 0, 0) and e.s.mission == O.NO_MISSION


def test_gotodoor_truncates_at_5_s_squared():
    S = 5
    env = O.Env(O.GOTODOOR, S, seed=3)
    for t in range(1, 5 * S * S + 1):
        r, te, tr = env.step(0)  # turning never ends the episode
        assert (r, te) == (0.0, 0) and tr == (t == 5 * S * S)


# --- DistShift1/2 (Table 8, R2) -----------------------------------------------

@pytest.mark.parametrize("S", [5, 6, 8, 11, 19])
def test_distshift_layouts(S):
    assert O.max_variant(O.DISTSHIFT, S) == 1
    grids = []
    for v in (0, 1):
        e = O.Env(O.DISTSHIFT, S, seed=v, variant=v, env_index=3)
        ent, col, st = e.grid()
        r2 = 3 if v == 0 else S - 2
        want = np.full((S, S), 1, np.uint8)
        want[0, :] = want[-1, :] = want[:, 0] = want[:, -1] = 2
        want[1, 2:S - 2] = 9
        want[r2, 2:S - 2] = 9
        want[1, S - 2] = 8
        np.testing.assert_array_equal(ent, want)
        assert (e.s.ax, e.s.ay, e.s.dir) == (1, 1, 0)
        # no draws: every episode and seed gives the same layout
        e2 = O.Env(O.DISTSHIFT, S, seed=99, variant=v)
        e2.reset(17)
        assert bytes(e2.s.ent) == bytes(e.s.ent)
        grids.append(ent)
        # a BFS plan (independent rules; lava ends a path) reaches the goal
        cells = tuple((int(ent[y, x]), int(col[y, x]), int(st[y, x])) for y in range(S) for x in range(S))
        plan = M.bfs_goal((1, 1, 0, None, cells), S, S, max_depth=60)
        assert plan is not None
        for a in plan:
            r, te, tr = e.step(a)
        assert (r, te) == (1.0, 1) and e.s.t == len(plan)
    assert S == 5 or (grids[0] != grids[1]).any()


def test_distshift_lava_ends_with_the_lava_reward():
    e = O.Env(O.DISTSHIFT, 8, lava_reward=-1.0)
    assert e.step(2) == (-1.0, 1, 0)  # the lava cell right of the start
    e = O.Env(O.DISTSHIFT, 8)
    assert e.step(2) == (0.0, 1, 0)


# --- action_cost / time_cost (Table 5) ----------------------------------------

def test_shaping_costs_follow_table5():
    f = np.float32
    ac, tc = f(0.01), f(0.003)
    e = O.Env(O.EMPTY, 5, action_cost=float(ac), time_cost=float(tc))
    # a plain move: both costs, subtracted in order
    r, te, tr = e.step(2)
    assert np.float32(r) == (f(0.0) - ac) - tc and te == 0
    # done: only the time cost
    r, te, tr = e.step(6)
    assert np.float32(r) == f(0.0) - tc
    # out-of-range action: a no-op that is no action, only the time cost
    r, te, tr = e.step(9)
    assert np.float32(r) == f(0.0) - tc
    # reaching the goal: 1 - action_cost - time_cost
    e.step(2)
    e.step(1)
    e.step(2)
    r, te, tr = e.step(2)
    assert (e.s.ax, e.s.ay) == (3, 3) and te == 1 and np.float32(r) == (f(1.0) - ac) - tc
    # the autoreset step carries no cost (reward padding)
    assert e.step(2) == (0.0, 0, 0)
    # with zero costs nothing changes, bit for bit
    b1 = O.Batch([O.DOORKEY] * 16, [6] * 16, seed=3)
    b2 = O.Batch([O.DOORKEY] * 16, [6] * 16, seed=3, action_cost=0.0, time_cost=0.0)
    b1.reset(), b2.reset()
    o1, o2 = b1.rollout(300), b2.rollout(300)
    assert o1["reward"].tobytes() == o2["reward"].tobytes()


# --- KeyCorridor S{s}R{R} (Table 8) --------------------------------------------

KC_IDS = [(7, 0), (7, 1), (7, 2), (10, 2), (13, 2), (16, 2), (19, 0), (10, 1)]  # S3R1..S3R3, S4R3, S5R3, S6R3, ...


def _kc_geometry(S, variant):
    s = (S - 1) // 3 + 1
    R = variant + 1
    return s, R, (s - 1) * R + 1


@pytest.mark.parametrize("S,variant", KC_IDS)
def test_keycorridor_layouts(S, variant):
    s, R, H = _kc_geometry(S, variant)
    xl, xr = s - 1, 2 * (s - 1)
    for seed in range(12):
        e = O.Env(O.KEYCORRIDOR, S, seed=seed, variant=variant, env_index=seed)
        ent, col, st = e.grid()
        assert e.s.max_steps == 30 * s * s
        assert (ent[H - 1:, :] == 2).all()  # the rows below the rooms are wall
        assert (ent[:, 0] == 2).all() and (ent[:, S - 1] == 2).all() and (ent[0, :] == 2).all()
        # horizontal room walls, open inside the corridor
        for j in range(1, R):
            y = j * (s - 1)
            assert (ent[y, :xl + 1] == 2).all() and (ent[y, xr:] == 2).all() and (ent[y, xl + 1:xr] == 1).all()
        doors = _doors(ent, col, st)
        assert len(doors) == 2 * R
        locked = [d for d in doors if d[3] == 2]
        assert len(locked) == 1 and all(d[3] in (1, 2) for d in doors)
        for side_x in (xl, xr):
            for j in range(R):
                rows = [y for x, y, _, _ in doors if x == side_x and j * (s - 1) < y < (j + 1) * (s - 1)]
                assert len(rows) == 1
        # walls of the corridor hold only the doors
        for x in (xl, xr):
            for y in range(H):
                assert ent[y, x] in (2, 4)
        lx, ly, lc, _ = locked[0]
        (gy, gx), = np.argwhere(ent == 8)
        (ky, kx), = np.argwhere(ent == 5)
        assert col[ky, kx] == lc
        # the goal is in the locked door's room, the key on the other side
        assert (gx < xl) == (lx == xl) and (gy - 1) // (s - 1) == (ly - 1) // (s - 1)
        assert (kx < xl) != (gx < xl) and 0 < ky < H - 1
        # side room interiors are empty but for the goal and key
        assert xl < e.s.ax < xr and 0 < e.s.ay < H - 1 and ent[e.s.ay, e.s.ax] == 1


def test_keycorridor_draws_cover_their_ranges():
    S, variant = 10, 2
    s, R, H = _kc_geometry(S, variant)
    seen = {"door_rows": set(), "colours": set(), "goal_room": set(), "key_room": set(), "agent": set(), "dir": set()}
    for ep in range(2000):
        e = O.Env(O.KEYCORRIDOR, S, seed=4, variant=variant)
        e.reset(ep)
        ent, col, st = e.grid()
        for x, y, c, _ in _doors(ent, col, st):
            seen["door_rows"].add((x, y))
            seen["colours"].add(c)
        (gy, gx), = np.argwhere(ent == 8)
        (ky, kx), = np.argwhere(ent == 5)
        seen["goal_room"].add((gx > s, (gy - 1) // (s - 1), gx, gy))
        seen["key_room"].add((kx > s, (ky - 1) // (s - 1)))
        seen["agent"].add((e.s.ax, e.s.ay))
        seen["dir"].add(e.s.dir)
    assert len(seen["door_rows"]) == 2 * R * (s - 2)
    assert seen["colours"] == set(range(6)) and seen["dir"] == {0, 1, 2, 3}
    assert len({g[:2] for g in seen["goal_room"]}) == 2 * R and len(seen["goal_room"]) == 2 * R * (s - 2) ** 2
    assert len(seen["key_room"]) == 2 * R
    assert len(seen["agent"]) == (s - 2) * (H - 2)


@pytest.mark.parametrize("S,variant", [(7, 0), (7, 1), (10, 2)])
def test_keycorridor_views_equal_those_of_the_unpadded_grid(S, variant):
    """The square holding a non-square KeyCorridor gives the views of the
    H x S grid itself (independent window model, outside = wall), for every
    pose of the agent in the corridor."""
    s, R, H = _kc_geometry(S, variant)
    e = O.Env(O.KEYCORRIDOR, S, seed=9, variant=variant)
    ent, col, st = e.grid()
    for y in range(1, H - 1):
        for x in range(s, 2 * s - 2):
            for d in range(4):
                e.set_agent(x, y, d)
                want = M.observe(ent[:H], col[:H], st[:H], x, y, d)
                np.testing.assert_array_equal(e.obs(), want)


@pytest.mark.parametrize("S,variant,seed", [(7, 0, 0), (7, 1, 1), (7, 2, 2), (10, 1, 3)])
def test_keycorridor_bfs_plans_fetch_the_key_and_reach_the_goal(S, variant, seed):
    e = O.Env(O.KEYCORRIDOR, S, seed=seed, variant=variant)
    ent, col, st = e.grid()
    cells = tuple((int(ent[y, x]), int(col[y, x]), int(st[y, x])) for y in range(S) for x in range(S))
    plan = M.bfs_goal((e.s.ax, e.s.ay, e.s.dir, None, cells), S, S, max_depth=60)
    assert plan is not None and 3 in plan and 5 in plan  # a pickup and a toggle on the way
    for i, a in enumerate(plan):
        r, te, tr = e.step(a)
        if i < len(plan) - 1:
            assert (r, te) == (0.0, 0)
    assert (r, te) == (1.0, 1) and e.s.t == len(plan)


def test_keycorridor_sizes():
    for S in (7, 10, 13, 16, 19):
        assert O.max_variant(O.KEYCORRIDOR, S) == 2
    for S in (5, 6, 8, 9, 11, 12, 18):
        with pytest.raises(ValueError):
            O.Env(O.KEYCORRIDOR, S)
    with pytest.raises(ValueError):
        O.Env(O.KEYCORRIDOR, 7, variant=3)
