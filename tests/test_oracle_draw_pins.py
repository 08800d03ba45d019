"""Pins of the oracle's mapping from random draws to placements (CPU only).

The paper defines start states only as samples of reset(key) (Section 3.2.2,
Code 1) and the families only by name (Table 8), so the order in which draws
pick cells (reading R18: the k-th free cell, rows outer), the ball moves of
Dynamic-Obstacles (reading R12: candidates in row-major neighbour order, balls
moved one after another on the grid the earlier ones left) and the counter of
the random actions (reading R1, purpose 3) are this project's readings.  They
are pinned here two ways:

* hand-worked examples under tests/golden/ (DoorKey-8x8, FourRooms-19x19, one
  Dynamic-Obstacles-5x5 step, the first random actions of one env, a
  GoToDoor-6x6 start with its colour shuffle and mission, a LavaCrossing-9x9
  start with its river shuffle, crossing order and openings, a KeyCorridor
  S4R2 start with its doors, locked door, goal, key and agent), whose
  every draw word and derived placement is re-derived from the independent
  restatement in tests/indep_model.py (its Philox checked against the
  published known-answer vectors) and must be reproduced by the oracle;
* sweeps comparing the oracle's start states and ball moves with the same
  independent restatement over many seeds, envs and sizes -- the start states
  of every family with draws (DoorKey, FourRooms, Dynamic-Obstacles, LavaGap,
  Empty-Random, GoToDoor with its mission, both crossings at every river
  count, KeyCorridor at every room side and row count).

tests/test_oracle_mutants.py plants the plausible mistakes (free cells scanned
column-major, balls moved on a snapshot of the grid, neighbours scanned column
first, the action counter's episode word, a short draw range, a full instead
of a partial shuffle, an off-by-one shuffle, two draws taken in the other
order) in copies of the oracle and checks that this file catches each.
"""
import os

import numpy as np
import pytest

import oracle as O

from . import indep_model as M

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    """(draw lines, expect lines) of a golden file: draw lines are
    (kind, k, word, n, bounded); expect lines are (key, ints...)."""
    draws, expects = [], []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip() if line.lstrip().startswith("#") else line.strip()
        if not line:
            continue
        f = line.split()
        if f[0] in ("draw", "move"):
            draws.append((f[0], int(f[1]), int(f[2], 16), int(f[3]), int(f[4])))
        elif f[0] == "action":
            draws.append((f[0], int(f[1]), int(f[2], 16), 7, int(f[3])))
        elif f[0] == "expect":
            expects.append((f[1], [int(v) for v in f[2:]]))
    return draws, expects


def _kat():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            v = [int(t, 16) for t in line.split()]
            yield v[0:4], v[4:6], v[6:10]


@pytest.mark.parametrize("ctr,key,out", list(_kat()))
def test_independent_philox_reproduces_published_vectors(ctr, key, out):
    assert M.philox4x32_10(ctr, key) == out


def test_independent_bounded_draw_is_floor_of_the_scaled_fraction():
    from fractions import Fraction
    for x in (0, 1, 0x7FFFFFFF, 0x80000000, 0x9F3F38EF, 0xFFFFFFFF):
        for n in (1, 2, 4, 7, 17, 260, 361):
            assert M.bounded(x, n) == int(Fraction(x * n, 1 << 32))


# --- the hand-worked examples -------------------------------------------------

def _check_draw_lines(draws, counter):
    """Every listed word is the independent Philox word of its counter, and
    every listed draw result is bounded(word, n)."""
    for kind, k, word, n, b in draws:
        assert word == counter(kind, k), (kind, k)
        assert M.bounded(word, n) == b, (kind, k)


def test_golden_doorkey8x8_seed1_env0_start():
    draws, exp = _golden("doorkey8x8_seed1_env0_start.txt")
    _check_draw_lines(draws, lambda kind, k: M.draw(1, 0, 0, 0, M.LAYOUT, k))
    exp = dict(exp)
    g, agent, xw, door, key, _ = M.doorkey_start(8, 1, 0, 0)
    assert [xw] == exp["wall_x"] and list(door) == exp["door"] and list(agent) == exp["agent"]
    assert list(key) == exp["key"]
    e = O.Env(O.DOORKEY, 8, seed=1, env_index=0)
    assert [e.s.ax, e.s.ay, e.s.dir] == exp["agent"]
    ent, col, st = e.grid()
    wx = exp["wall_x"][0]
    for y in range(1, 7):
        if [wx, y] != exp["door"]:
            assert (ent[y, wx], col[y, wx]) == (2, 5)
    dx, dy = exp["door"]
    assert (ent[dy, dx], col[dy, dx], st[dy, dx]) == (4, 4, 2)
    kx, ky = exp["key"]
    assert (ent[ky, kx], col[ky, kx]) == (5, 4)
    gx, gy = exp["goal"]
    assert ent[gy, gx] == 8
    # the whole grid equals the independent restatement's
    np.testing.assert_array_equal(np.stack([ent, col, st], -1), g)


def test_golden_fourrooms19_seed2_env0_start():
    draws, exp = _golden("fourrooms19_seed2_env0_start.txt")
    _check_draw_lines(draws, lambda kind, k: M.draw(2, 0, 0, 0, M.LAYOUT, k))
    gaps = [v for k, v in exp if k == "gap"]
    exp = dict(exp)
    g, agent, goal, igaps, _ = M.fourrooms_start(19, 2, 0, 0)
    assert [list(p) for p in igaps] == gaps and list(goal) == exp["goal"] and list(agent) == exp["agent"]
    e = O.Env(O.FOURROOMS, 19, seed=2, env_index=0)
    assert [e.s.ax, e.s.ay, e.s.dir] == exp["agent"]
    ent, col, st = e.grid()
    for x, y in gaps:
        assert ent[y, x] == 1
    assert ent[exp["goal"][1], exp["goal"][0]] == 8
    np.testing.assert_array_equal(np.stack([ent, col, st], -1), g)


def test_golden_dynobs5x5_seed0_env0_ball_step():
    draws, exp = _golden("dynobs5x5_seed0_env0_ball_step.txt")
    _check_draw_lines([d for d in draws if d[0] == "draw"], lambda kind, k: M.draw(0, 0, 0, 0, M.LAYOUT, k))
    _check_draw_lines([d for d in draws if d[0] == "move"], lambda kind, k: M.draw(0, 0, 0, 0, M.BALL, k))
    start = [v[1:] for k, v in exp if k == "start_ball"]
    after = [v[1:] for k, v in exp if k == "ball"]
    g, balls, _ = M.dynobs_start(5, 0, 0, 0)
    assert [list(b) for b in balls] == start
    new, _ = M.move_balls(g, balls, (1, 1), 0, 0, 0, 0)
    assert [list(b) for b in new] == after
    e = O.Env(O.DYNOBS, 5, seed=0, env_index=0, n_balls=4)
    assert [[e.s.ball_x[b], e.s.ball_y[b]] for b in range(4)] == start
    r, te, tr = e.step(0)
    assert (r, te, tr) == (0.0, 0, 0) and (e.s.ax, e.s.ay) == (1, 1)
    assert [[e.s.ball_x[b], e.s.ball_y[b]] for b in range(4)] == after
    ent, col, _ = e.grid()
    for x, y in after:
        assert (ent[y, x], col[y, x]) == (6, 2)
    assert int((ent == 6).sum()) == 4


def test_golden_random_actions_seed0_env3():
    draws, _ = _golden("random_actions_seed0_env3.txt")
    _check_draw_lines(draws, lambda kind, g: M.draw(0, 3, 0xFFFFFFFF, g, M.ACTION, 0))
    want = [b for _, _, _, _, b in draws]
    assert len(want) == 8
    e = O.Env(O.EMPTY, 5, seed=0, env_index=3)
    assert [e.random_action(g) for g in range(8)] == want
    # the batch rollout's random mode draws the same actions for env 3: its
    # first steps from the start state follow them
    b = O.Batch([O.EMPTY] * 4, [5] * 4, seed=0)
    b.reset()
    ref = O.Env(O.EMPTY, 5, seed=0, env_index=3)
    for a in want:
        b.step()
        ref.step(a)
    assert O.env_state(b.env(3)) == O.env_state(ref.s)


# --- sweeps against the independent restatement --------------------------------

@pytest.mark.parametrize("S", [5, 6, 8, 11, 16, 19])
def test_doorkey_starts_equal_the_independent_generator(S):
    for seed in (0, 1, 77):
        for env in range(6):
            for ep in (0, 3):
                g, agent, *_ = M.doorkey_start(S, seed, env, ep)
                e = O.Env(O.DOORKEY, S, seed=seed, env_index=env)
                e.reset(ep)
                ent, col, st = e.grid()
                np.testing.assert_array_equal(np.stack([ent, col, st], -1), g)
                assert (e.s.ax, e.s.ay, e.s.dir) == agent


@pytest.mark.parametrize("S", [7, 9, 13, 19])
def test_fourrooms_starts_equal_the_independent_generator(S):
    for seed in (0, 2, 99):
        for env in range(6):
            for ep in (0, 5):
                g, agent, *_ = M.fourrooms_start(S, seed, env, ep)
                e = O.Env(O.FOURROOMS, S, seed=seed, env_index=env)
                e.reset(ep)
                ent, col, st = e.grid()
                np.testing.assert_array_equal(np.stack([ent, col, st], -1), g)
                assert (e.s.ax, e.s.ay, e.s.dir) == agent


@pytest.mark.parametrize("S", [5, 6, 8, 16])
def test_ball_moves_equal_the_independent_transition(S):
    """Twenty steps of turning in place (the agent never moves, so only the
    balls change the grid): the oracle's balls follow reading R12 step by step."""
    for seed in (0, 3):
        for env in range(4):
            e = O.Env(O.DYNOBS, S, seed=seed, env_index=env, n_balls=4)
            g, balls, _ = M.dynobs_start(S, seed, env, 0)
            for t in range(20):
                balls, _ = M.move_balls(g, balls, (1, 1), seed, env, 0, t)
                e.step(t % 2)
                assert [(e.s.ball_x[b], e.s.ball_y[b]) for b in range(4)] == balls, (S, seed, env, t)
                ent, col, st = e.grid()
                np.testing.assert_array_equal(np.stack([ent, col, st], -1), g)


def test_random_actions_equal_the_independent_counter():
    for seed in (0, 1, 2**40 + 5):
        for env in (0, 1, 1000, 65535):
            e = O.Env(O.EMPTY, 5, seed=seed, env_index=env)
            d = O.Env(O.DYNOBS, 8, seed=seed, env_index=env)
            for g in (0, 1, 2, 127, 128, 5000):
                assert e.random_action(g) == M.random_action(seed, env, g, 7)
                assert d.random_action(g) == M.random_action(seed, env, g, 3)


def _start_of(family, S, variant, seed, env, ep):
    e = O.Env(family, S, seed=seed, env_index=env, variant=variant)
    e.reset(ep)
    ent, col, st = e.grid()
    return np.stack([ent, col, st], -1), (e.s.ax, e.s.ay, e.s.dir), e.s.mission


@pytest.mark.parametrize("S", [5, 7, 11, 19])
def test_lavagap_and_empty_random_starts_equal_the_independent_generators(S):
    for seed in (0, 4, 2**33 + 1):
        for env in range(5):
            for ep in (0, 7):
                g, agent = M.lavagap_start(S, seed, env, ep)
                got, a, _ = _start_of(O.LAVAGAP, S, 0, seed, env, ep)
                np.testing.assert_array_equal(got, g)
                assert a == agent
                g, agent = M.empty_random_start(S, seed, env, ep)
                got, a, _ = _start_of(O.EMPTY_RANDOM, S, 0, seed, env, ep)
                np.testing.assert_array_equal(got, g)
                assert a == agent


@pytest.mark.parametrize("S", [5, 6, 9, 14, 19])
def test_gotodoor_starts_and_missions_equal_the_independent_generator(S):
    for seed in (0, 8):
        for env in range(6):
            for ep in (0, 3):
                g, agent, mission = M.gotodoor_start(S, seed, env, ep)
                got, a, m = _start_of(O.GOTODOOR, S, 0, seed, env, ep)
                np.testing.assert_array_equal(got, g)
                assert a == agent and m == mission


@pytest.mark.parametrize("S", [5, 7, 9, 11, 13, 19])
def test_crossing_starts_equal_the_independent_generator(S):
    """Every river count the size allows, lava and wall rivers."""
    for n_rivers in range(O.max_variant(O.LAVA_CROSSING, S) + 1):
        for family, obstacle in ((O.LAVA_CROSSING, M.LAVA), (O.SIMPLE_CROSSING, M.WALL)):
            for seed in (0, 6):
                for env in range(3):
                    g, agent = M.crossing_start(S, n_rivers, obstacle, seed, env, 1)
                    got, a, _ = _start_of(family, S, n_rivers, seed, env, 1)
                    np.testing.assert_array_equal(got, g, err_msg=f"{family} S {S} N {n_rivers}")
                    assert a == agent


@pytest.mark.parametrize("S", [7, 10, 13, 16, 19])
def test_keycorridor_starts_equal_the_independent_generator(S):
    """Room sides 3 to 7, one to three rows of rooms."""
    for variant in range(3):
        for seed in (0, 9):
            for env in range(4):
                for ep in (0, 2):
                    g, agent = M.keycorridor_start(S, variant, seed, env, ep)
                    got, a, _ = _start_of(O.KEYCORRIDOR, S, variant, seed, env, ep)
                    np.testing.assert_array_equal(got, g, err_msg=f"S {S} R {variant + 1}")
                    assert a == agent


def test_golden_gotodoor6x6_seed0_env0_start():
    """The hand-worked GoToDoor start: door places, the colour shuffle, the
    mission and the agent, each draw re-derived independently, and the
    oracle's start state equal to them."""
    draws, exp = _golden("gotodoor6x6_seed0_env0_start.txt")
    _check_draw_lines(draws, lambda kind, k: M.draw(0, 0, 0, 0, M.LAYOUT, k))
    assert [k for _, k, *_ in draws] == list(range(11))  # every draw of the layout, in order
    exp = dict(exp)
    g, agent, mission = M.gotodoor_start(6, 0, 0, 0)
    e = O.Env(O.GOTODOOR, 6, seed=0, env_index=0)
    ent, col, st = e.grid()
    for side in ("door_top", "door_bottom", "door_left", "door_right"):
        x, y, c = exp[side]
        assert tuple(int(v) for v in g[y, x]) == (4, c, 1)
        assert (ent[y, x], col[y, x], st[y, x]) == (4, c, 1)
    assert [mission] == exp["mission"] == [e.s.mission]
    assert list(agent) == exp["agent"] == [e.s.ax, e.s.ay, e.s.dir]
    assert int((ent == 4).sum()) == 4  # no other door
    np.testing.assert_array_equal(np.stack([ent, col, st], -1), g)


def test_golden_lavacrossing9x9_n3_seed6_env0_start():
    """The hand-worked crossing start: the river shuffle, the crossing order,
    the openings and the drawn grid, each draw re-derived independently, and
    the oracle's start state equal to them."""
    draws, exp = _golden("lavacrossing9x9_n3_seed6_env0_start.txt")
    _check_draw_lines(draws, lambda kind, k: M.draw(6, 0, 0, 0, M.LAYOUT, k))
    assert [k for _, k, *_ in draws] == list(range(8))
    exp = dict(exp)
    art = [line[1:].strip() for line in open(os.path.join(GOLDEN, "lavacrossing9x9_n3_seed6_env0_start.txt"))
           if line.startswith("#   ") and set(line[1:].strip()) <= set("#~.G")]
    assert len(art) == 9
    code = {"#": 2, "~": 9, ".": 1, "G": 8}
    g, agent = M.crossing_start(9, 3, M.LAVA, 6, 0, 0)
    e = O.Env(O.LAVA_CROSSING, 9, seed=6, env_index=0, variant=3)
    ent, col, st = e.grid()
    for y in range(9):
        assert [code[ch] for ch in art[y]] == ent[y].tolist() == g[y, :, 0].tolist(), y
    openings = exp["openings"]
    for x, y in zip(openings[0::2], openings[1::2]):
        assert ent[y, x] == 1
    assert all((ent[y, 1:8] != 1).sum() == 6 for y in exp["lava_rows"])  # one opening per row river
    assert all((ent[1:8, x] != 1).sum() == 6 for x in exp["lava_cols"])
    assert list(agent) == exp["agent"] == [e.s.ax, e.s.ay, e.s.dir]
    gx, gy = exp["goal"]
    assert ent[gy, gx] == 8
    np.testing.assert_array_equal(np.stack([ent, col, st], -1), g)


def test_golden_keycorridor_s4r2_seed3_env0_start():
    """The hand-worked KeyCorridor start: door rows and colours, the locked
    door, the goal, the key of the locked door's colour on the other side and
    the agent in the corridor, each draw re-derived independently, and the
    oracle's start state equal to them."""
    name = "keycorridor_s4r2_seed3_env0_start.txt"
    draws, exp = _golden(name)
    _check_draw_lines(draws, lambda kind, k: M.draw(3, 0, 0, 0, M.LAYOUT, k))
    assert [k for _, k, *_ in draws] == list(range(15))
    doors = [v for key, v in exp if key == "door"]
    exp = dict(exp)
    art = [line[1:].strip() for line in open(os.path.join(GOLDEN, name))
           if line.startswith("#   ") and set(line[1:].strip()) <= set("#.DKG")]
    assert len(art) == 10
    code = {"#": 2, ".": 1, "D": 4, "K": 5, "G": 8}
    g, agent = M.keycorridor_start(10, 1, 3, 0, 0)
    e = O.Env(O.KEYCORRIDOR, 10, seed=3, env_index=0, variant=1)
    ent, col, st = e.grid()
    for y in range(10):
        assert [code[ch] for ch in art[y]] == ent[y].tolist() == g[y, :, 0].tolist(), y
    for x, y, c, state in doors:
        assert (ent[y, x], col[y, x], st[y, x]) == (4, c, state)
    assert sum(state == 2 for *_, state in doors) == 1
    kx, ky, kc = exp["key"]
    assert (ent[ky, kx], col[ky, kx]) == (5, kc)
    gx, gy = exp["goal"]
    assert ent[gy, gx] == 8
    assert list(agent) == exp["agent"] == [e.s.ax, e.s.ay, e.s.dir]
    np.testing.assert_array_equal(np.stack([ent, col, st], -1), g)


@pytest.mark.parametrize("S", [5, 6, 9, 14, 19])
def test_dynobs_starts_for_every_ball_count_equal_the_independent_generator(S):
    """Zero to four balls, each on the k-th free interior cell left by the
    balls before it (never the agent's cell)."""
    for n_balls in range(5):
        for seed in (0, 12):
            for env in range(4):
                for ep in (0, 6):
                    g, balls, _ = M.dynobs_start(S, seed, env, ep, n_balls=n_balls)
                    e = O.Env(O.DYNOBS, S, seed=seed, env_index=env, n_balls=n_balls)
                    e.reset(ep)
                    ent, col, st = e.grid()
                    np.testing.assert_array_equal(np.stack([ent, col, st], -1), g)
                    assert [(e.s.ball_x[b], e.s.ball_y[b]) for b in range(n_balls)] == balls
                    assert (e.s.ax, e.s.ay, e.s.dir, e.s.n_balls) == (1, 1, 0, n_balls)
