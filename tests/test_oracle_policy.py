"""Pins of the oracle's fused-rollout policy (an integer MLP from the
categorical first-person view to actions), CPU only.

* zero weights: the greedy action is the first largest bias (closed form);
* a hand-built network computing "wall in front -> turn right, else forward"
  (ReLU combinations of the front cell's entity code) drives a rollout that
  must equal a scripted agent reading the grid directly;
* the floor of the requantisation shift and the first-max tie break;
* exploration with epsilon = 2^32 - 1 reproduces the random-action rollout;
* weight sets are chosen by env index / envs_per_agent.
"""
import numpy as np
import pytest

import oracle as O

DX = (1, 0, -1, 0)
DY = (0, 1, 0, -1)


def zero_policy(A=1, epa=128, **kw):
    z = dict(w1=np.zeros((A, 64, 49)), b1=np.zeros((A, 64)), w2=np.zeros((A, 64, 64)), b2=np.zeros((A, 64)),
             w3=np.zeros((A, 7, 64)), b3=np.zeros((A, 7)), shift1=0, shift2=0, envs_per_agent=epa)
    z.update(kw)
    return z


def wall_turner():
    """Turn right when the cell in front is a wall, else go forward."""
    p = zero_policy()
    front = 5 * 7 + 3  # view (vx 3, vy 5): the cell ahead of the agent
    for j, b in enumerate((-1, -2, -3)):  # h1[j] = relu(x - 1 - j)
        p["w1"][0, j, front] = 1
        p["b1"][0, j] = b
    p["w2"][0, 0, :3] = (1, -2, 1)  # h2[0] = relu(h1[0] - 2 h1[1] + h1[2]) = [x == 2]
    p["w3"][0, 1, 0] = 10           # right: 10 [wall]
    p["b3"][0] = (-100, 0, 5, -100, -100, -100, -100)  # forward: 5
    return O.Policy(**p)


def test_zero_weights_pick_the_first_largest_bias():
    rng = np.random.default_rng(1)
    for trial in range(20):
        b3 = rng.integers(-3, 3, 7)
        pol = O.Policy(**zero_policy(b3=b3[None, :]))
        x = rng.integers(0, 11, 49)
        assert pol.greedy(0, x, 7) == int(np.argmax(b3))
        assert pol.greedy(0, x, 3) == int(np.argmax(b3[:3]))


def test_requantisation_floor_and_first_max():
    p = zero_policy()
    p["w1"][0, 0, 0] = 1
    p["w2"][0, 0, 0] = 1
    p["w3"][0, 1, 0] = 1
    p["b3"][0] = (2, 0, -9, -9, -9, -9, -9)
    p["shift1"] = 1
    pol = O.Policy(**p)
    # h = x0 >> 1; action 1 only when h > 2 (h = 2 ties with action 0, the first)
    for x0, want in ((0, 0), (4, 0), (5, 0), (6, 1), (10, 1)):
        x = np.zeros(49, np.uint8)
        x[0] = x0
        assert pol.greedy(0, x) == want, x0
    # a negative accumulator floors below zero and clamps to 0; large ones clamp to 255
    p["b1"][0, 0] = -3  # (x0 - 3) >> 1: x0 = 0 -> floor(-1.5) = -2 -> 0
    p["w3"][0, 1, 0] = -1
    p["b3"][0] = (-1, 0, -9, -9, -9, -9, -9)  # action 1 iff h == 0
    pol = O.Policy(**p)
    for x0, want in ((0, 1), (3, 1), (4, 1), (5, 0)):
        x = np.zeros(49, np.uint8)
        x[0] = x0
        assert pol.greedy(0, x) == want, x0
    p = zero_policy()
    p["b1"][0, 0] = 100000
    p["w2"][0, 0, 0] = 1
    p["w3"][0, 1, 0] = 1
    p["b3"][0] = (254, 0, -9, -9, -9, -9, -9)  # h1 = h2 = 255 after clamping: 255 > 254
    assert O.Policy(**p).greedy(0, np.zeros(49, np.uint8)) == 1
    p["b3"][0, 0] = 255
    assert O.Policy(**p).greedy(0, np.zeros(49, np.uint8)) == 0


@pytest.mark.parametrize("family,size", [(O.EMPTY, 8), (O.FOURROOMS, 11), (O.DOORKEY, 8), (O.KEYCORRIDOR, 10)])
def test_hand_built_policy_matches_a_scripted_agent(family, size):
    pol = wall_turner()
    n, T = 12, 150
    b = O.Batch([family] * n, [size] * n, seed=5)
    b.reset()
    script = O.Batch([family] * n, [size] * n, seed=5)
    script.reset()
    out = b.rollout_policy(T, pol)
    for t in range(T):
        acts = np.zeros(n, np.int8)
        for i in range(n):
            e = script.env(i)
            fx, fy = e.ax + DX[e.dir], e.ay + DY[e.dir]
            inside = 0 <= fx < e.width and 0 <= fy < e.height
            acts[i] = 1 if (not inside or e.ent[fy * e.width + fx] == 2) else 2
        o = script.step(acts)
        np.testing.assert_array_equal(out["actions"][t], acts, err_msg=f"step {t}")
        np.testing.assert_array_equal(out["obs_sym"][t], o["obs_sym"])
        np.testing.assert_array_equal(out["reward"][t], o["reward"])


def test_full_exploration_is_the_random_action_rollout():
    pol = wall_turner()
    pol = O.Policy(pol.w1, pol.b1, pol.w2, pol.b2, pol.w3, pol.b3, 0, 0, epsilon=2**32 - 1)
    descs = ([O.DOORKEY] * 6 + [O.DYNOBS] * 6, [8] * 12)
    a = O.Batch(*descs, seed=9)
    a.reset()
    r = O.Batch(*descs, seed=9)
    r.reset()
    oa = a.rollout_policy(200, pol)
    orr = r.rollout(200)
    for k in ("obs_sym", "reward", "terminated", "truncated"):
        np.testing.assert_array_equal(oa[k], orr[k], err_msg=k)
    assert (oa["actions"][:, 6:] < 3).all()


def test_weight_sets_follow_env_index():
    p = zero_policy(A=3, epa=4)
    p["b3"] = np.full((3, 7), -5)
    for agent, act in enumerate((3, 5, 1)):
        p["b3"][agent, act] = 0
    pol = O.Policy(**p)
    b = O.Batch([O.EMPTY] * 12, [6] * 12, seed=2)
    b.reset()
    acts = b.rollout_policy(3, pol)["actions"]
    assert (acts == np.array([3] * 4 + [5] * 4 + [1] * 4, np.int8)).all()
