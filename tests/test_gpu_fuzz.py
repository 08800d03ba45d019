"""Randomised parity sweep: seeded random batches -- families, sizes and
variants per env in random order, ragged env counts -- in random launch
shapes, chunk lengths, slot sizes, output rings, reward settings and action
sources, each run through the C-ABI binding and by the oracle on the same
inputs and compared byte for byte at every step kept and in the final state.

Each case draws its configuration from its own seed, so a failure names a
configuration that reproduces on its own.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2407_19396_gb300 import inputs  # noqa: E402
from tests.gpu_util import assert_outputs_equal, assert_states_equal, oracle_batch_for, to_np  # noqa: E402

pytestmark = pytest.mark.gpu

N_FAMILIES = 11
# (lanes per env, envs per block, staging parts); (0, 0, 0) lets the library choose
SHAPES = [(0, 0, 0), (1, 32, 1), (1, 64, 2), (1, 128, 1), (2, 64, 1), (4, 16, 1), (4, 64, 2), (8, 16, 1),
          (8, 32, 2), (16, 4, 1), (16, 8, 1), (32, 2, 1), (32, 4, 2)]
N_CASES = 96


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2407_19396_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def valid_sizes(family):
    return [s for s in range(5, 20) if O.max_variant(family, s) >= 0]


def draw_case(i):
    """The configuration of case i, from its own seed."""
    rng = np.random.default_rng(7000 + i)
    k = int(rng.integers(1, 5))
    fams = rng.choice(N_FAMILIES, size=k, replace=False)
    parts = []
    for f in fams:
        f = int(f)
        s = int(rng.choice(valid_sizes(f)))
        v = int(rng.integers(0, O.max_variant(f, s) + 1))
        ms = int(rng.integers(3, 60)) if rng.random() < 0.3 else 0
        parts.append((f, s, ms, v))
    n = int(rng.integers(1, 16)) if rng.random() < 0.25 else int(rng.integers(16, 1200))
    descs = [parts[int(j)] for j in rng.integers(0, k, size=n)]  # families interleaved env by env
    lanes, envs, staging = SHAPES[int(rng.integers(0, len(SHAPES)))]
    max_side = max(p[1] for p in parts)
    T = int(rng.integers(20, 500))
    return dict(
        descs=descs, seed=int(rng.integers(0, 2**31)), lanes=lanes, envs=envs, staging=staging,
        grid_side=int(rng.integers(5, max_side + 1)) if rng.random() < 0.3 else 0,
        spl=int(rng.choice([1, 7, 64, 128])), T=T,
        depth=T if rng.random() < 0.5 else int(rng.integers(1, T + 1)),
        reward_mode=int(rng.integers(0, 2)), lava_reward=float(rng.choice([0.0, -1.0, -0.5])),
        action_cost=float(rng.choice([0.0, 0.0125])), time_cost=float(rng.choice([0.0, 0.004])),
        n_balls=int(rng.integers(0, 5)), buffered=bool(rng.random() < 0.4), action=bool(rng.random() < 0.3),
    )


def oracle_steps(ob, T, acts, missions):
    """The oracle's T steps one by one, with each step's missions when asked."""
    keys = ("obs_sym", "reward", "terminated", "truncated")
    outs = {k: [] for k in keys + ("mission",)}
    for t in range(T):
        o = ob.step(None if acts is None else acts[t])
        for k in keys:
            outs[k].append(o[k])
        if missions:
            outs["mission"].append(ob.missions())
    return {k: np.stack(v) for k, v in outs.items() if v}


def ring_of(full, T, depth):
    """Steps T - depth .. T - 1 of a [T, ...] array at their ring slots (step t in slot t % depth)."""
    out = np.empty((depth,) + full.shape[1:], full.dtype)
    for t in range(T - depth, T):
        out[t % depth] = full[t]
    return out


@pytest.mark.parametrize("case", range(N_CASES))
def test_random_configuration_matches_the_oracle(case):
    from paper_2407_19396_gb300 import navixgb as nx

    c = draw_case(case)
    descs, T, depth, n = c["descs"], c["T"], c["depth"], len(c["descs"])
    kw = dict(reward_mode=c["reward_mode"], lava_reward=c["lava_reward"], action_cost=c["action_cost"],
              time_cost=c["time_cost"], n_balls=c["n_balls"])
    what = f"case {case}: {c}"
    acts = inputs.random_actions(c["seed"] & 0xFFFF, (T, n), n_actions=7, invalid_fraction=0.02) if c["buffered"] else None
    env = nx.Env(descs=descs, seed=c["seed"], autotune=False, group_lanes=c["lanes"], envs_per_cta=c["envs"],
                 staging=c["staging"], grid_side=c["grid_side"], steps_per_launch=c["spl"], action=c["action"], **kw)
    try:
        r0 = env.reset()
        out = env.rollout(T, depth=depth, actions=None if acts is None else torch.from_numpy(acts).cuda())
        torch.cuda.synchronize()
        missions = env.want_mission
        ob = oracle_batch_for(descs, c["seed"], **kw)
        o0 = ob.reset()
        if missions:
            o0["mission"] = ob.missions()
        keys = ("obs_sym", "reward", "terminated", "truncated") + (("mission",) if missions else ())
        assert_outputs_equal(r0, o0, keys=keys, what=f"reset, {what}")
        oo = oracle_steps(ob, T, acts, missions)
        ring = {k: ring_of(v, T, depth) for k, v in oo.items()}
        assert_outputs_equal(out, ring, keys=keys, what=f"rollout, {what}")
        if c["action"] and acts is not None:
            np.testing.assert_array_equal(to_np(out["action"]), ring_of(acts, T, depth), err_msg=f"actions, {what}")
        assert_states_equal(env.state()["envs"], ob, what=what)
        assert env.flags() & ~1 == 0, what  # no bounds or wait flag; bit 0 only for invalid buffered actions
        if acts is None:
            assert env.flags() == 0, what
    finally:
        env.close()


def test_the_cases_cover_the_axes():
    """The drawn configurations reach every family, the one-lane and the
    wide-group paths, the lean and the general kernels (action output or the
    MiniGrid reward), buffered and random actions, short rings and slots
    below the largest grid."""
    cs = [draw_case(i) for i in range(N_CASES)]
    fams = {d[0] for c in cs for d in c["descs"]}
    assert len(fams) >= 10
    assert any(c["lanes"] == 1 for c in cs) and any(c["lanes"] >= 8 for c in cs)
    assert any(c["action"] or c["reward_mode"] == 1 for c in cs)
    assert any(not c["action"] and c["reward_mode"] == 0 for c in cs)
    assert any(c["buffered"] for c in cs) and any(not c["buffered"] for c in cs)
    assert any(c["depth"] < c["T"] for c in cs) and any(c["grid_side"] > 0 for c in cs)
    assert any(c["spl"] == 1 for c in cs) and any(len(c["descs"]) < 8 for c in cs)


OPTIONAL = ("obs_sym", "reward", "terminated", "truncated")


def draw_output_case(i):
    """Case i of the output sweep: a random subset of the outputs (any may be
    absent), the fully observable views, and at small sizes the RGB views."""
    rng = np.random.default_rng(8000 + i)
    rgb = bool(rng.random() < 0.25)
    rgb_full = rgb and bool(rng.random() < 0.5)
    k = int(rng.integers(1, 4))
    parts = []
    for f in rng.choice(N_FAMILIES, size=k, replace=False):
        f = int(f)
        sizes = [s for s in valid_sizes(f) if not rgb or s <= 11] or [min(valid_sizes(f))]
        s = int(rng.choice(sizes))
        parts.append((f, s, 0, int(rng.integers(0, O.max_variant(f, s) + 1))))
    n = int(rng.integers(1, 24 if rgb else 300))
    T = int(rng.integers(5, 30 if rgb else 200))
    shapes = [(0, 0, 0), (1, 64, 1), (16, 8, 1), (32, 4, 1)] if rgb else SHAPES
    lanes, envs, staging = shapes[int(rng.integers(0, len(shapes)))]
    want = {key: bool(rng.random() < 0.7) for key in OPTIONAL}
    if rng.random() < 0.1:  # none of the four (the rollout only advances the state, or writes other views)
        want = dict.fromkeys(OPTIONAL, False)
    want.update(mission=bool(rng.random() < 0.5), action=bool(rng.random() < 0.3), obs_full=bool(rng.random() < 0.3),
                obs_cat=bool(rng.random() < 0.3), obs_cat_fp=bool(rng.random() < 0.3), obs_rgb=rgb and bool(rng.random() < 0.8),
                obs_rgb_full=rgb_full)
    return dict(descs=[parts[int(j)] for j in rng.integers(0, k, size=n)], seed=int(rng.integers(0, 2**31)),
                lanes=lanes, envs=envs, staging=staging, spl=int(rng.choice([1, 7, 64, 128])), T=T,
                depth=T if rng.random() < 0.5 else int(rng.integers(1, T + 1)), reward_mode=int(rng.integers(0, 2)),
                buffered=bool(rng.random() < 0.4), want=want, rgb=rgb)


@pytest.mark.parametrize("case", range(32))
def test_random_output_subsets_match_the_oracle(case):
    from paper_2407_19396_gb300 import navixgb as nx

    c = draw_output_case(case)
    descs, T, depth, n, want = c["descs"], c["T"], c["depth"], len(c["descs"]), c["want"]
    what = f"case {case}: {dict(c, descs=sorted(set(descs)), n=n)}"
    atlas = inputs.atlas() if c["rgb"] else None
    acts = inputs.random_actions(c["seed"] & 0xFFFF, (T, n), n_actions=7, invalid_fraction=0.02) if c["buffered"] else None
    env = nx.Env(descs=descs, seed=c["seed"], autotune=False, group_lanes=c["lanes"], envs_per_cta=c["envs"],
                 staging=c["staging"], steps_per_launch=c["spl"], reward_mode=c["reward_mode"],
                 obs_sym=want["obs_sym"], obs_rgb=want["obs_rgb"] or want["obs_rgb_full"], atlas=atlas,
                 obs_full=want["obs_full"], obs_cat=want["obs_cat"], obs_cat_fp=want["obs_cat_fp"],
                 obs_rgb_full=want["obs_rgb_full"], mission=want["mission"], action=want["action"])
    try:
        env.reset()
        out = env.alloc_out(depth)
        for key in ("reward", "terminated", "truncated", "obs_rgb"):
            if not want[key]:
                out[key] = None
        g = env.rollout(T, depth=depth, out=out, actions=None if acts is None else torch.from_numpy(acts).cuda())
        torch.cuda.synchronize()
        ob = oracle_batch_for(descs, c["seed"], reward_mode=c["reward_mode"])
        ob.reset()
        side = env.side
        steps = {key: [] for key in want}
        for t in range(T):
            o = ob.step(None if acts is None else acts[t], rgb=want["obs_rgb"], atlas=atlas)
            for key in ("obs_sym", "reward", "terminated", "truncated", "obs_rgb"):
                if want[key]:
                    steps[key].append(o[key])
            if want["obs_full"] or want["obs_cat"] or want["obs_cat_fp"]:
                f, cat, cfp = ob.full_views(side)
                steps["obs_full"].append(f)
                steps["obs_cat"].append(cat)
                steps["obs_cat_fp"].append(cfp)
            if want["obs_rgb_full"]:
                steps["obs_rgb_full"].append(ob.rgb_full(atlas, side))
            if want["mission"]:
                steps["mission"].append(ob.missions())
            if want["action"] and acts is not None:
                steps["action"].append(acts[t])
        present = [key for key in want if want[key] and steps[key]]
        exp = {key: ring_of(np.stack(steps[key]), T, depth) for key in present}
        assert_outputs_equal(g, exp, keys=tuple(present), what=what)
        for key in want:
            if not want[key]:
                assert g.get(key) is None, f"{what}: {key} was not asked for"
        assert_states_equal(env.state()["envs"], ob, what=what)
        assert env.flags() & ~1 == 0, what  # no bounds or wait flag; bit 0 only for invalid buffered actions
    finally:
        env.close()


def test_the_output_cases_cover_every_output():
    cs = [draw_output_case(i) for i in range(32)]
    for key in cs[0]["want"]:
        assert any(c["want"][key] for c in cs), key
        if key not in ("obs_rgb", "obs_rgb_full"):
            assert any(not c["want"][key] for c in cs), key
    assert any(not any(c["want"][k] for k in OPTIONAL) for c in cs)  # a rollout with none of the four
