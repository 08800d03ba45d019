"""Brute-force pins of the oracle on tiny inputs, invariants and layout sweeps (CPU).

* every agent pose (position x direction x carried object) of small layouts:
  the oracle's symbolic_first_person view (Table 4) equals the independent
  window-and-rotate model of ``indep_model``;
* BFS-optimal plans found on the independent rule model, replayed through the
  oracle, reach the goal with reward exactly 1.0 at exactly the plan length
  (R1 of Table 8), and the oracle's own state graph has no shorter route;
* long random rollouts of every family keep the invariants of the entity
  rules (Tables 1-2: one agent, never inside a wall or closed door, keys and
  balls conserved, doors only unlock with a matching key);
* layout generators (Table 8 families) are valid for every size and cover
  their random choices.
"""
import ctypes
from collections import deque

import numpy as np
import pytest

import oracle as O
from tests import indep_model as M


def _clone(env: O.Env) -> O.Env:
    c = O.Env.__new__(O.Env)
    c.s = O.OrcEnv.from_buffer_copy(bytes(env.s))
    return c


def _carry(env):
    return None if env.s.carry_ent == 0 else (env.s.carry_ent, env.s.carry_col)


@pytest.mark.parametrize("family,size,seed", [(O.EMPTY, 5, 0), (O.DOORKEY, 5, 1), (O.DOORKEY, 6, 2),
                                              (O.FOURROOMS, 7, 3), (O.LAVAGAP, 6, 4), (O.DYNOBS, 6, 5),
                                              (O.FOURROOMS, 11, 6), (O.DOORKEY, 8, 7)])
def test_view_matches_independent_window_model(family, size, seed):
    base = O.Env(family, size, seed=seed)
    ent, col, st = base.grid()
    # open the door in half of the poses to exercise see-through doors too
    doors = np.argwhere(ent == 4)
    n = 0
    for variant in range(2):
        env = _clone(base)
        if variant == 1:
            for (y, x) in doors:
                env.set_cell(int(x), int(y), 4, int(col[y, x]), 0)
        e2, c2, s2 = env.grid()
        for y in range(size):
            for x in range(size):
                for d in range(4):
                    for carry in (None, (5, 4), (6, 2)):
                        env.set_agent(x, y, d, *(carry or (0, 0)))
                        want = M.observe(e2, c2, s2, x, y, d, carry)
                        np.testing.assert_array_equal(env.obs(), want, err_msg=f"pose {(x, y, d, carry)}")
                        n += 1
    assert n > 0


def test_view_all_transparent_sees_everything():
    # special case: no opaque cell in view -> all 49 cells visible
    env = O.Env(O.EMPTY, 19)
    env.set_agent(9, 12, 3)
    o = env.obs()
    assert (o[:, :, 0] != 0).all()


def test_view_facing_wall_point_blank():
    # a wall row straight ahead at distance 1 and walls all along the agent row:
    # only the agent row's reachable part and the row ahead are lit
    env = O.Env(O.EMPTY, 5)
    env.set_agent(1, 1, 3)  # face north: the border wall is ahead
    o = env.obs()
    assert (o[:5, :, 0] == 0).all()
    assert tuple(o[5, 3]) == (2, 5, 0)


def _state_key(env):
    e, c, s = env.grid()
    return (env.s.ax, env.s.ay, env.s.dir, env.s.carry_ent, env.s.carry_col, e.tobytes(), c.tobytes(), s.tobytes())


def _oracle_bfs_len(env, max_depth=40):
    """Length of the shortest goal-reaching action sequence in the oracle's own state graph."""
    start = _clone(env)
    seen = {_state_key(start)}
    q = deque([(start, 0)])
    while q:
        s, depth = q.popleft()
        if depth >= max_depth:
            continue
        for a in range(6):
            n = _clone(s)
            r, te, tr = n.step(a)
            if te and r == 1.0:
                return depth + 1
            if te:
                continue
            k = _state_key(n)
            if k not in seen:
                seen.add(k)
                q.append((n, depth + 1))
    return None


@pytest.mark.parametrize("family,size,seed", [(O.EMPTY, 5, 0), (O.EMPTY, 6, 0), (O.EMPTY, 8, 0),
                                              (O.DOORKEY, 5, 1), (O.DOORKEY, 5, 2), (O.DOORKEY, 6, 3),
                                              (O.LAVAGAP, 5, 4), (O.LAVAGAP, 6, 5), (O.FOURROOMS, 7, 6)])
def test_bfs_plans_reach_goal_with_exact_reward(family, size, seed):
    env = O.Env(family, size, seed=seed)
    ent, col, st = env.grid()
    cells = tuple((int(ent[y, x]), int(col[y, x]), int(st[y, x])) for y in range(size) for x in range(size))
    start = (env.s.ax, env.s.ay, env.s.dir, None, cells)
    plan = M.bfs_goal(start, size, size, max_depth=40)
    assert plan is not None
    if family == O.EMPTY:
        # closed form: S-3 steps east, one turn, S-3 steps south
        assert len(plan) == 2 * (size - 3) + 1
    play = _clone(env)
    for i, a in enumerate(plan):
        r, te, tr = play.step(a)
        if i < len(plan) - 1:
            assert (r, te) == (0.0, 0), f"early end at step {i}"
    assert (r, te) == (1.0, 1)
    assert play.s.t == len(plan)
    assert _oracle_bfs_len(env) == len(plan)


def _count(ent, code):
    return int((ent == code).sum())


@pytest.mark.parametrize("family,size,seed", [(O.EMPTY, 5, 10), (O.EMPTY, 16, 11), (O.DOORKEY, 5, 12),
                                              (O.DOORKEY, 8, 13), (O.DOORKEY, 16, 14), (O.FOURROOMS, 19, 15),
                                              (O.LAVAGAP, 7, 16), (O.DYNOBS, 16, 17), (O.DYNOBS, 5, 18)])
def test_random_rollout_invariants(family, size, seed):
    n_envs, T = 16, 1500
    b = O.Batch([family] * n_envs, [size] * n_envs, seed=seed)
    b.reset()
    init = []
    for i in range(n_envs):
        e = b.env(i)
        ent = np.frombuffer(bytes(e.ent), np.uint8)[: size * size].reshape(size, size)
        init.append((_count(ent, 5), _count(ent, 6)))
    prev = [b.state(i) for i in range(n_envs)]
    for t in range(T):
        o = b.step()
        for i in range(n_envs):
            s = b.state(i)
            p = prev[i]
            ent = np.frombuffer(s["ent"], np.uint8).reshape(size, size)
            col = np.frombuffer(s["col"], np.uint8).reshape(size, size)
            st = np.frombuffer(s["st"], np.uint8).reshape(size, size)
            # border walls
            assert (ent[0, :] == 2).all() and (ent[-1, :] == 2).all() and (ent[:, 0] == 2).all() and (ent[:, -1] == 2).all()
            assert not (ent == 10).any()
            # the agent stands on a walkable cell inside the grid
            x, y = s["x"], s["y"]
            assert 1 <= x <= size - 2 and 1 <= y <= size - 2
            ce, cs = ent[y, x], st[y, x]
            assert ce in (1, 3, 8, 9) or (ce == 4 and cs == 0)
            assert 0 <= s["t"] <= s["max_steps"]
            if p["done"]:
                # autoreset step
                assert s["episode"] == p["episode"] + 1 and s["t"] == 0
                assert o["reward"][i] == 0 and o["terminated"][i] == 0 and o["truncated"][i] == 0
                continue
            assert s["episode"] == p["episode"] and s["t"] == p["t"] + 1
            keys0, balls0 = init[i]
            keys = _count(ent, 5) + (1 if s["carry_ent"] == 5 else 0)
            balls = _count(ent, 6) + (1 if s["carry_ent"] == 6 else 0)
            pe = np.frombuffer(p["ent"], np.uint8).reshape(size, size)
            pk = _count(pe, 5) + (1 if p["carry_ent"] == 5 else 0)
            pb = _count(pe, 6) + (1 if p["carry_ent"] == 6 else 0)
            assert keys == pk and balls == pb
            # doors unlock only with a key of the door's colour in hand
            pst = np.frombuffer(p["st"], np.uint8).reshape(size, size)
            unlocked = (pe == 4) & (pst == 2) & (st != 2)
            if unlocked.any():
                yy, xx = np.argwhere(unlocked)[0]
                assert s["carry_ent"] == 5 and s["carry_col"] == col[yy, xx]
            # termination exactly on the reward events
            term = o["terminated"][i]
            on_goal = ent[y, x] == 8
            on_lava = ent[y, x] == 9
            hit = family == O.DYNOBS and term and not on_goal and not on_lava
            assert bool(term) == bool(on_goal or on_lava or hit)
            if on_goal:
                assert o["reward"][i] == 1.0
            if hit:
                assert o["reward"][i] == -1.0
            assert o["truncated"][i] == (1 if s["t"] >= s["max_steps"] else 0)
            # the agent cell is always visible and shows the carried object
            oc = tuple(o["obs_sym"][i, 6, 3])
            assert oc == ((s["carry_ent"], s["carry_col"], 0) if s["carry_ent"] else (1, 0, 0))
        prev = [b.state(i) for i in range(n_envs)]
        if t > 300 and family in (O.EMPTY, O.LAVAGAP):
            break


SIZES = {O.EMPTY: range(5, 20), O.DOORKEY: range(5, 20), O.FOURROOMS: range(5, 20), O.LAVAGAP: range(5, 20),
         O.DYNOBS: range(5, 20)}


@pytest.mark.parametrize("family", [O.EMPTY, O.DOORKEY, O.FOURROOMS, O.LAVAGAP, O.DYNOBS])
def test_layouts_valid_for_every_size(family):
    for size in SIZES[family]:
        for seed in range(24):
            env = O.Env(family, size, seed=seed, env_index=seed * 7 + 1)
            ent, col, st = env.grid()
            S = size
            assert (ent[0] == 2).all() and (ent[-1] == 2).all() and (ent[:, 0] == 2).all() and (ent[:, -1] == 2).all()
            x, y, d = env.s.ax, env.s.ay, env.s.dir
            assert 0 <= d < 4 and ent[y, x] == 1
            if family in (O.EMPTY, O.LAVAGAP, O.DYNOBS):
                assert (x, y, d) == (1, 1, 0)
            if family != O.FOURROOMS:
                assert ent[S - 2, S - 2] == 8 and _count(ent, 8) == 1
            if family == O.DOORKEY:
                walls = [c for c in range(2, S - 2) if (ent[1:S - 1, c] != 1).all() and (ent[1:S - 1, c] == 2).sum() == S - 3]
                assert len(walls) == 1
                xw = walls[0]
                dy = np.argwhere(ent[:, xw] == 4).ravel()
                assert len(dy) == 1 and 1 <= dy[0] <= S - 3 and (col[dy[0], xw], st[dy[0], xw]) == (4, 2)
                ky, kx = np.argwhere(ent == 5)[0]
                assert _count(ent, 5) == 1 and col[ky, kx] == 4 and kx < xw and x < xw and (kx, ky) != (x, y)
            if family == O.FOURROOMS:
                m = S // 2
                gaps_v = [r for r in range(1, S - 1) if r != m and ent[r, m] != 2]
                gaps_h = [c for c in range(1, S - 1) if c != m and ent[m, c] != 2]
                assert len(gaps_v) == 2 and len(gaps_h) == 2
                assert gaps_v[0] < m < gaps_v[1] and gaps_h[0] < m < gaps_h[1]
                assert _count(ent, 8) == 1
            if family == O.LAVAGAP:
                cols = np.argwhere((ent == 9).any(axis=0)).ravel()
                assert len(cols) == 1 and 2 <= cols[0] <= S - 3
                assert (ent[1:S - 1, cols[0]] == 9).sum() == S - 3
            if family == O.DYNOBS:
                assert _count(ent, 6) == 4 and ent[1, 1] == 1
                bx, by = list(env.s.ball_x), list(env.s.ball_y)
                assert len({(a, b) for a, b in zip(bx, by)}) == 4
                for a, b in zip(bx, by):
                    assert ent[b, a] == 6 and col[b, a] == 2


def test_layout_choices_cover_their_ranges():
    S = 8
    xs, doors, agents, dirs = set(), set(), set(), set()
    for ep in range(400):
        env = O.Env(O.DOORKEY, S, seed=1)
        env.reset(ep)
        ent, _, _ = env.grid()
        xw = [c for c in range(2, S - 2) if (ent[1:S - 1, c] == 2).sum() == S - 3][0]
        xs.add(xw)
        doors.add(int(np.argwhere(ent[:, xw] == 4)[0][0]))
        agents.add((env.s.ax, env.s.ay))
        dirs.add(env.s.dir)
    assert xs == set(range(2, S - 2)) and doors == set(range(1, S - 2)) and dirs == {0, 1, 2, 3}
    assert len(agents) >= 20
    gaps = set()
    for ep in range(300):
        env = O.Env(O.LAVAGAP, 7, seed=2)
        env.reset(ep)
        ent, _, _ = env.grid()
        c = int(np.argwhere((ent == 9).any(axis=0)).ravel()[0])
        gaps.add((c, int(np.argwhere(ent[1:6, c] != 9).ravel()[0]) + 1))
    assert gaps == {(c, g) for c in range(2, 5) for g in range(1, 6)}


def test_ball_moves_stay_on_free_neighbours():
    env = O.Env(O.DYNOBS, 8, seed=9)
    for t in range(300):
        before = list(zip(env.s.ball_x, env.s.ball_y))
        r, te, tr = env.step(0)  # turning in place: only the balls move
        after = list(zip(env.s.ball_x, env.s.ball_y))
        if env.s.t == 0:
            continue
        for (a, b), (c, d) in zip(before, after):
            assert max(abs(a - c), abs(b - d)) <= 1
            assert (c, d) != (env.s.ax, env.s.ay)
        assert len(set(after)) == 4


@pytest.mark.parametrize("size", [5, 6, 8, 16, 19])
def test_balls_never_leave_the_interior(size):
    """Balls are placed in the grid's interior and only move to empty cells,
    so every ball of every reachable state lies in 1..size-2 on both axes and
    sits on a ball cell of the grid (the step kernels read a ball's eight
    neighbours without bounds tests, and a restored state must satisfy it)."""
    n = 8
    b = O.Batch([O.DYNOBS] * n, [size] * n, seed=size)
    b.reset()
    seen_move = False
    for t in range(400):
        b.step()
        for i in range(n):
            s = b.state(i)
            ent = np.frombuffer(s["ent"], np.uint8).reshape(size, size)
            assert s["n_balls"] == 4
            for x, y in zip(s["ball_x"], s["ball_y"]):
                assert 1 <= x <= size - 2 and 1 <= y <= size - 2, (t, i, x, y)
                assert ent[y, x] == 6
            seen_move = seen_move or t > 0
    assert seen_move


@pytest.mark.parametrize("family,size,seed", [(O.DOORKEY, 8, 1), (O.FOURROOMS, 19, 2), (O.DYNOBS, 8, 3),
                                              (O.SIMPLE_CROSSING, 11, 4)])
def test_full_views_agree_with_the_grid_and_the_egocentric_view(family, size, seed):
    """symbolic / categorical (Table 4) against the grid planes, and every
    visible egocentric cell against the full view at its world position."""
    variant = 3 if family == O.SIMPLE_CROSSING else 0
    b = O.Batch([family] * 6, [size] * 6, seed=seed, variants=[variant] * 6)
    b.reset()
    for t in range(150):
        o = b.step()
        full, cat, cfp = b.full_views(size + 2)
        for i in range(6):
            s = b.state(i)
            ent = np.frombuffer(s["ent"], np.uint8).reshape(size, size)
            col = np.frombuffer(s["col"], np.uint8).reshape(size, size)
            st = np.frombuffer(s["st"], np.uint8).reshape(size, size)
            f = full[i]
            assert (f[size:, :, :] == 0).all() and (f[:, size:, :] == 0).all()
            x, y, d = s["x"], s["y"], s["dir"]
            assert tuple(f[y, x]) == (10, 0, d) and cat[i, y, x] == 10
            mask = np.ones((size, size), bool)
            mask[y, x] = False
            assert (f[:size, :size, 0][mask] == ent[mask]).all() and (f[:size, :size, 1][mask] == col[mask]).all()
            assert (f[:size, :size, 2][mask] == st[mask]).all() and (cat[i, :size, :size][mask] == ent[mask]).all()
            np.testing.assert_array_equal(cfp[i], o["obs_sym"][i][:, :, 0])
            F = [(1, 0), (0, 1), (-1, 0), (0, -1)][d]
            R = [(1, 0), (0, 1), (-1, 0), (0, -1)][(d + 1) % 4]
            for vy in range(7):
                for vx in range(7):
                    v = o["obs_sym"][i][vy, vx]
                    if (vx, vy) == (3, 6) or v[0] == 0:
                        continue
                    wx = x + (6 - vy) * F[0] + (vx - 3) * R[0]
                    wy = y + (6 - vy) * F[1] + (vx - 3) * R[1]
                    if 0 <= wx < size and 0 <= wy < size:
                        assert tuple(v) == tuple(f[wy, wx])
                    else:
                        assert tuple(v) == (2, 5, 0)


def test_egocentric_rgb_assembles_the_atlas_tiles_of_the_symbolic_view(atlas):
    """rgb_first_person (Table 4): each 32x32 block (vx, vy) of the oracle's
    224x224 view is the atlas tile of that view cell's symbolic triple: the
    unseen tile where the triple is (0, 0, 0), the agent-cell tile of what the
    agent carries (or of an empty cell) at (3, 6), the plain tile elsewhere;
    on the reset and on every step."""
    from paper_2407_19396_gb300 import inputs

    index = {atlas[k].tobytes(): k for k in range(atlas.shape[0])}
    fams, sizes = [O.DOORKEY, O.DYNOBS, O.FOURROOMS, O.LAVAGAP], [8, 6, 9, 7]
    b = O.Batch(fams, sizes, seed=9)

    def check(o):
        for i in range(len(fams)):
            for vy in range(7):
                for vx in range(7):
                    blk = o["obs_rgb"][i, 32 * vy:32 * vy + 32, 32 * vx:32 * vx + 32]
                    tile = index[np.ascontiguousarray(blk).tobytes()]
                    vis, agent, e, c, st = inputs.tile_params(tile)
                    tri = tuple(int(v) for v in o["obs_sym"][i, vy, vx])
                    if (vx, vy) == (3, 6):
                        assert vis == 1 and agent == 1 and (e, c, st) == tri
                    elif tri == (0, 0, 0):
                        assert tile == 0
                    else:
                        assert vis == 1 and agent == 0 and (e, c, st) == tri

    check(b.reset(rgb=True, atlas=atlas))
    carried = 0
    for _ in range(60):
        o = b.step(rgb=True, atlas=atlas)
        check(o)
        carried += int((o["obs_sym"][:, 6, 3, 0] != 1).sum())
    assert carried > 0  # some step shows a carried object in the agent's cell


def test_full_rgb_view_assembles_the_atlas_tiles_of_the_full_symbolic_view(atlas):
    """rgb (Table 4): each 32x32 block of the oracle's full RGB view is the atlas
    tile the atlas module assigns to that cell's triple (the agent's cell: the
    agent facing its direction; beyond the grid: the unseen tile)."""
    from paper_2407_19396_gb300 import inputs

    index = {atlas[k].tobytes(): k for k in range(atlas.shape[0])}
    b = O.Batch([O.DOORKEY, O.SIMPLE_CROSSING, O.DYNOBS], [8, 9, 6], seed=5, variants=[0, 2, 0])
    b.reset()
    for t in range(40):
        b.step()
        full, _, _ = b.full_views(10)
        img = b.rgb_full(atlas, 10)
        for i in range(3):
            for y in range(10):
                for x in range(10):
                    blk = img[i, 32 * y:32 * y + 32, 32 * x:32 * x + 32]
                    tile = index[np.ascontiguousarray(blk).tobytes()]
                    vis, agent, e, c, s = inputs.tile_params(tile)
                    f = tuple(int(v) for v in full[i, y, x])
                    if f == (0, 0, 0):
                        assert tile == 0
                    elif f[0] == 10:
                        assert agent == 2 and s == f[2]
                    else:
                        assert vis == 1 and agent == 0 and (e, c, s) == f


def _rule_state(s):
    """An oracle state dict as the independent rule model's tuple state."""
    n = s["height"] * s["width"]
    cells = tuple(zip(s["ent"][:n], s["col"][:n], s["st"][:n]))
    carry = (s["carry_ent"], s["carry_col"]) if s["carry_ent"] else None
    return (s["x"], s["y"], s["dir"], carry, cells)


LOCKSTEP = [(O.EMPTY, 6, 0), (O.DOORKEY, 5, 0), (O.DOORKEY, 8, 0), (O.FOURROOMS, 9, 0), (O.LAVAGAP, 6, 0),
            (O.EMPTY_RANDOM, 7, 0), (O.LAVA_CROSSING, 9, 2), (O.SIMPLE_CROSSING, 9, 2), (O.GOTODOOR, 6, 0),
            (O.GOTODOOR, 8, 0), (O.DISTSHIFT, 8, 1), (O.KEYCORRIDOR, 7, 0), (O.KEYCORRIDOR, 10, 1)]


@pytest.mark.parametrize("family,size,variant", LOCKSTEP)
def test_every_step_matches_the_independent_rule_model(family, size, variant):
    """Random play (every action, out-of-range ones included) of every family
    without balls, step by step: the oracle's next agent pose, carried object
    and grid equal the independent rule model's successor for the action
    taken (no successor: nothing changes), termination happens exactly on its
    goal / lava events, the reward is 1.0 on a goal and 0 otherwise, and
    truncation exactly when t reaches max_steps."""
    n, T = 12, 500
    b = O.Batch([family] * n, [size] * n, seed=100 + family, variants=[variant] * n)
    b.reset()
    acts = np.random.default_rng(200 + family).integers(0, 8, size=(T, n)).astype(np.int8)
    prev = [b.state(i) for i in range(n)]
    events = {"goal": 0, "lava": 0, "write": 0}
    for t in range(T):
        o = b.step(acts[t])
        cur = [b.state(i) for i in range(n)]
        for i in range(n):
            p, s = prev[i], cur[i]
            if p["done"]:
                continue  # the autoreset step (pinned elsewhere)
            a = int(acts[t, i])
            mission = p["mission"] if family == O.GOTODOOR else None
            before = _rule_state(p)
            want, ev = before, None
            for act, nxt, e in M.successors(before, p["width"], p["height"], mission=mission):
                if act == a:
                    want, ev = nxt, e
                    break
            assert _rule_state(s) == want, (family, t, i, a)
            assert o["terminated"][i] == (1 if ev else 0), (family, t, i, a, ev)
            assert o["reward"][i] == (1.0 if ev == "goal" else 0.0), (family, t, i, a, ev)
            assert o["truncated"][i] == (1 if s["t"] >= s["max_steps"] else 0)
            if ev:
                events[ev] += 1
            if want[4] != before[4]:
                events["write"] += 1
        prev = cur
    # the play reached the rules that change the grid (pickup, drop, toggle)
    # wherever the layout has an object to change
    if family in (O.DOORKEY, O.KEYCORRIDOR, O.GOTODOOR):
        assert events["write"] > 0, events


def _env_rule_state(e):
    ent, col, st = e.grid()
    cells = tuple(zip(ent.reshape(-1).tolist(), col.reshape(-1).tolist(), st.reshape(-1).tolist()))
    carry = (e.s.carry_ent, e.s.carry_col) if e.s.carry_ent else None
    return (e.s.ax, e.s.ay, e.s.dir, carry, cells)


@pytest.mark.parametrize("family", [O.DOORKEY, O.GOTODOOR])
def test_random_states_match_the_independent_rule_model(family):
    """Hand-built random states no generator makes -- keys, balls and doors
    of every colour and state, goals, lava and floor scattered over a 6x6
    grid, the agent carrying nothing, a key or a ball of any colour -- and
    every action from each: the oracle's next state, termination and reward
    equal the independent rule model's (a key of another colour leaves a
    locked door shut; a full hand picks up nothing; done only completes
    GoToDoor at a door of the mission's colour)."""
    rng = np.random.default_rng(300 + family)
    S = 6
    kinds = [(1, 0, 0), (1, 0, 0), (1, 0, 0), (3, 0, 0), (2, 5, 0), (8, 1, 0), (9, 0, 0)]
    seen = set()
    for trial in range(400):
        e = O.Env(family, S, seed=trial)
        e.reset()
        for y in range(1, S - 1):
            for x in range(1, S - 1):
                r = rng.random()
                if r < 0.15:
                    e.set_cell(x, y, 4, int(rng.integers(0, 6)), int(rng.integers(0, 3)))   # door
                elif r < 0.25:
                    e.set_cell(x, y, 5, int(rng.integers(0, 6)), 0)                         # key
                elif r < 0.35:
                    e.set_cell(x, y, 6, int(rng.integers(0, 6)), 0)                         # ball
                else:
                    e.set_cell(x, y, *kinds[int(rng.integers(0, len(kinds)))])
        ax, ay = int(rng.integers(1, S - 1)), int(rng.integers(1, S - 1))
        e.set_cell(ax, ay, 1, 0, 0)
        carry = [(0, 0), (5, int(rng.integers(0, 6))), (6, int(rng.integers(0, 6)))][int(rng.integers(0, 3))]
        e.set_agent(ax, ay, int(rng.integers(0, 4)), *carry)
        start = _env_rule_state(e)
        mission = e.s.mission if family == O.GOTODOOR else None
        succ = {a: (s, ev) for a, s, ev in M.successors(start, S, S, mission=mission)}
        for a in range(8):
            c = _clone(e)
            r, term, trunc = c.step(a)
            want, ev = succ.get(a, (start, None))
            assert _env_rule_state(c) == want, (family, trial, a)
            assert term == (1 if ev else 0) and r == (1.0 if ev == "goal" else 0.0), (family, trial, a, ev)
            if want != start or ev:
                seen.add(a)  # the action changed something (done: ended GoToDoor's episode)
    assert seen >= ({0, 1, 2, 3, 4, 5, 6} if family == O.GOTODOOR else {0, 1, 2, 3, 4, 5}), seen


def test_random_grids_view_matches_independent_window_model():
    """Dense random grids no generator makes -- walls, doors of every state
    (open ones see-through), keys, balls, goals, lava and floor in random
    places, 5x5 to 12x12 -- and random poses, including poses on the border
    looking out of the grid: the oracle's view equals the independent
    window-and-rotate model's, so the occlusion is pinned on many more
    opaque patterns than the layouts produce."""
    rng = np.random.default_rng(400)
    cells = [(1, 0, 0), (1, 0, 0), (1, 0, 0), (2, 5, 0), (3, 0, 0), (8, 1, 0), (9, 0, 0)]
    n = 0
    for trial in range(300):
        S = int(rng.integers(5, 13))
        e = O.Env(O.DOORKEY, S, seed=trial)
        e.reset()
        for y in range(S):
            for x in range(S):
                r = rng.random()
                if r < 0.12:
                    e.set_cell(x, y, 4, int(rng.integers(0, 6)), int(rng.integers(0, 3)))
                elif r < 0.2:
                    e.set_cell(x, y, int(rng.choice([5, 6])), int(rng.integers(0, 6)), 0)
                else:
                    e.set_cell(x, y, *cells[int(rng.integers(0, len(cells)))])
        ent, col, st = e.grid()
        for _ in range(12):
            x, y, d = int(rng.integers(0, S)), int(rng.integers(0, S)), int(rng.integers(0, 4))
            carry = [None, (5, int(rng.integers(0, 6))), (6, int(rng.integers(0, 6)))][int(rng.integers(0, 3))]
            e.set_agent(x, y, d, *(carry or (0, 0)))
            np.testing.assert_array_equal(e.obs(), M.observe(ent, col, st, x, y, d, carry),
                                          err_msg=f"trial {trial} S {S} pose {(x, y, d, carry)}")
            n += 1
    assert n == 3600
