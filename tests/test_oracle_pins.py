"""Pins of the CPU oracle against facts fixed outside it (CPU only).

* Philox4x32-10 against the published known-answer vectors;
* the hand-worked Empty-5x5 reset observation (Table 4 symbolic_first_person);
* hand sequences: the shortest walk to the goal with a blocked step (reward
  R1 of Table 8, termination of Table 6), truncation at max_steps, the
  autoreset padding of Section 3.2.2 and Code 1, the key-door colour rule of
  Table 2, and Eq. 1 evaluated in IEEE single precision by numpy.
"""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert O.philox4x32_10(ctr, key) == out


def test_bounded_draw_range_and_monotone():
    for n in (1, 2, 3, 4, 7, 9, 100, 361, 4096):
        xs = [0, 1, 2**31, 2**32 - 1, 0x9E3779B9, 12345]
        for x in xs:
            assert 0 <= O.bounded(x, n) < n
        assert O.bounded(0, n) == 0
        assert O.bounded(2**32 - 1, n) == n - 1
        # monotone non-decreasing in x, and each value has a ~2^32/n pre-image
        assert O.bounded((2**32 // n) * 1, n) in (0, 1)


def test_draw_counter_layout():
    # the draw is word 0 of Philox at counter (env, episode, step, purpose<<24|draw), key (seed lo, seed hi)
    seed = 0x0123456789ABCDEF
    got = O.draw(seed, 5, 6, 7, 3, 9)
    want = O.philox4x32_10([5, 6, 7, (3 << 24) | 9], [seed & 0xFFFFFFFF, seed >> 32])[0]
    assert got == want


def test_random_actions_uniform_over_seven():
    e = O.Env(O.EMPTY, 5, seed=0)
    counts = np.bincount([e.random_action(g) for g in range(7000)], minlength=7)
    assert counts.shape == (7,) and counts.min() > 850 and counts.max() < 1150
    d = O.Env(O.DYNOBS, 8, seed=0)
    counts = np.bincount([d.random_action(g) for g in range(3000)], minlength=3)
    assert counts.shape == (3,) and counts.min() > 900


def _golden_obs(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        rows.append([[int(v) for v in cell.split(",")] for cell in line.split()])
    return np.array(rows, np.uint8)


def test_empty5_reset_observation_worked_example():
    e = O.Env(O.EMPTY, 5)
    np.testing.assert_array_equal(e.obs(), _golden_obs("empty5x5_reset_obs.txt"))


def test_shortest_walk_with_blocked_step():
    e = O.Env(O.EMPTY, 5)
    reset_obs = e.obs()
    acts = [2, 2, 2, 1, 2, 2]  # forward, forward, forward into the wall, turn right, forward, forward
    for i, a in enumerate(acts):
        r, te, tr = e.step(a)
        if i < len(acts) - 1:
            assert (r, te, tr) == (0.0, 0, 0)
    assert (r, te, tr) == (1.0, 1, 0)
    assert e.s.t == 6 and (e.s.ax, e.s.ay) == (3, 3)
    # the blocked step kept the agent at (3, 1); the turn made it face south
    # next call: autoreset with reward padding 0, the action is ignored
    r, te, tr = e.step(2)
    assert (r, te, tr) == (0.0, 0, 0)
    assert e.s.episode == 1 and e.s.t == 0
    np.testing.assert_array_equal(e.obs(), reset_obs)


def test_minigrid_reward_eq1_in_single_precision():
    e = O.Env(O.EMPTY, 5, reward_mode=1)
    for a in [2, 2, 2, 1, 2, 2]:
        r, te, tr = e.step(a)
    f = np.float32
    want = f(1.0) - (f(0.9) * f(6)) / f(100)
    assert te == 1 and np.float32(r) == want
    assert abs(r - 0.946) < 1e-6


def test_truncation_at_max_steps():
    e = O.Env(O.EMPTY, 5)
    assert e.s.max_steps == 100
    for i in range(100):
        r, te, tr = e.step(0)
        assert r == 0.0 and te == 0
        assert tr == (1 if i == 99 else 0)
    assert e.s.t == 100
    r, te, tr = e.step(0)
    assert (r, te, tr) == (0.0, 0, 0) and e.s.t == 0 and e.s.episode == 1


def test_truncation_and_termination_on_the_same_step():
    e = O.Env(O.EMPTY, 5, max_steps=5)
    for a in [2, 2, 1, 2]:
        assert e.step(a) == (0.0, 0, 0)
    assert e.step(2) == (1.0, 1, 1)


def _door_env():
    e = O.Env(O.DOORKEY, 5, seed=0)
    # hand-built: clear the interior, wall column at x = 2 with a locked yellow door at (2, 2)
    for y in range(1, 4):
        for x in range(1, 4):
            e.set_cell(x, y, 1, 0, 0)
    for y in range(1, 4):
        e.set_cell(2, y, 2, 5, 0)
    e.set_cell(2, 2, 4, 4, 2)
    e.set_cell(3, 3, 8, 1, 0)
    e.set_agent(1, 2, 0)
    return e


def test_door_key_colour_rule():
    e = _door_env()
    door = lambda: tuple(int(v[2, 2]) for v in e.grid())  # noqa: E731
    e.step(5)  # toggle without a key
    assert door() == (4, 4, 2)
    e.set_agent(1, 2, 0, 5, 0)  # carrying a red key
    e.step(5)
    assert door() == (4, 4, 2)
    e.set_agent(1, 2, 0, 5, 4)  # carrying the yellow key
    e.step(5)
    assert door() == (4, 4, 0) and e.s.carry_ent == 5 and e.s.carry_col == 4
    # the open door shows in the view, straight ahead of the agent
    assert tuple(e.obs()[5, 3]) == (4, 4, 0)
    e.step(5)
    assert door() == (4, 4, 1)
    e.step(2)  # a closed door blocks
    assert (e.s.ax, e.s.ay) == (1, 2)
    e.step(5)
    assert door() == (4, 4, 0)
    e.step(2)
    assert (e.s.ax, e.s.ay) == (2, 2)


def test_pickup_and_drop():
    e = _door_env()
    e.set_cell(1, 1, 5, 4, 0)  # key north of the agent
    e.step(0)  # face north
    assert e.s.dir == 3
    e.step(3)
    assert (e.s.carry_ent, e.s.carry_col) == (5, 4) and tuple(int(v[1, 1]) for v in e.grid()) == (1, 0, 0)
    assert tuple(e.obs()[6, 3]) == (5, 4, 0)  # the agent cell shows what is carried
    e.step(3)  # hand full: nothing
    e.step(1)  # face east: the locked door
    e.step(4)  # drop onto a door: refused
    assert e.s.carry_ent == 5
    e.step(0)
    e.step(4)  # drop north onto the empty cell
    assert e.s.carry_ent == 0 and tuple(int(v[1, 1]) for v in e.grid()) == (5, 4, 0)


def test_invalid_actions_are_noops_with_sticky_flag():
    e = O.Env(O.EMPTY, 5)
    before = (e.s.ax, e.s.ay, e.s.dir)
    r = e.step(9)
    assert r == (0.0, 0, 0) and (e.s.ax, e.s.ay, e.s.dir) == before and e.s.t == 1
    assert e.s.invalid_action == 1
    e.step(2)
    assert e.s.invalid_action == 1


def test_dynamic_obstacles_collision_and_restricted_actions():
    e = O.Env(O.DYNOBS, 5, seed=3, n_balls=1)
    # pin the ball so it cannot move: surround it with walls except the agent side
    for y in range(1, 4):
        for x in range(1, 4):
            e.set_cell(x, y, 1, 0, 0)
    e.set_cell(3, 3, 8, 1, 0)
    e.set_cell(2, 1, 6, 2, 0)
    e.s.ball_x[0], e.s.ball_y[0] = 2, 1
    for x, y in [(3, 1), (1, 2), (2, 2), (3, 2)]:
        e.set_cell(x, y, 2, 5, 0)
    e.set_agent(1, 1, 0)
    assert e.step(3) == (0.0, 0, 0)  # pickup is not in the 3-action set
    assert e.s.carry_ent == 0
    r, te, tr = e.step(2)
    assert (r, te) == (-1.0, 1) and (e.s.ax, e.s.ay) == (1, 1)


def test_lava_reward_default_zero_and_option():
    for lava, want in ((0.0, 0.0), (-1.0, -1.0)):
        e = O.Env(O.LAVAGAP, 5, seed=0, lava_reward=lava)
        # put lava right in front of the agent
        e.set_cell(2, 1, 9, 0, 0)
        r, te, tr = e.step(2)
        assert (r, te, tr) == (want, 1, 0)


def test_oracle_ctypes_structs_match_its_header(tmp_path):
    """The oracle's ctypes mirrors of orc_env and orc_policy have the size and
    field offsets of the C structs (compiled from oracle/navix_oracle.h by the
    host C compiler), so no test reads a field at the wrong place."""
    import ctypes
    import subprocess

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    classes = [(O.OrcEnv, "orc_env"), (O.OrcPolicy, "orc_policy")]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "navix_oracle.h"', "int main(void) {"]
    for c, cname in classes:
        lines.append(f'printf("{c.__name__} - %zu\\n", sizeof({cname}));')
        for field in c._fields_:
            lines.append(f'printf("{c.__name__} {field[0]} %zu\\n", offsetof({cname}, {field[0]}));')
    lines.append("return 0; }")
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(root, "oracle"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    n = 0
    for line in out.splitlines():
        name, field, value = line.split()
        c = getattr(O, name)
        got = ctypes.sizeof(c) if field == "-" else getattr(c, field).offset
        assert got == int(value), f"{name}.{field}: ctypes {got}, C {value}"
        n += 1
    assert n == sum(1 + len(c._fields_) for c, _ in classes)
