"""GPU parity: the CUDA path (through the C-ABI binding) against the CPU oracle,
byte for byte, on the same seeded inputs.

The environment is all integer work plus float32 rewards computed in a fixed
operation order, so every comparison is exact (tolerance 0): observations,
rewards, termination/truncation flags and the full state snapshot.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2407_19396_gb300 import inputs  # noqa: E402
from tests.gpu_util import (STATE_KEYS, assert_outputs_equal, assert_states_equal, mixed_descs,  # noqa: E402
                            oracle_batch_for, to_np)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2407_19396_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def nxmod():
    from paper_2407_19396_gb300 import navixgb as nx

    return nx


ALL_FAMILIES = [(O.EMPTY, 5, 0), (O.EMPTY, 8, 0), (O.EMPTY, 16, 0), (O.DOORKEY, 5, 0), (O.DOORKEY, 8, 0),
                (O.DOORKEY, 16, 0), (O.FOURROOMS, 19, 0), (O.FOURROOMS, 9, 0), (O.LAVAGAP, 5, 0), (O.LAVAGAP, 7, 0),
                (O.DYNOBS, 5, 0), (O.DYNOBS, 16, 0), (O.DOORKEY, 19, 0), (O.EMPTY, 19, 0), (O.LAVAGAP, 13, 0),
                (O.EMPTY_RANDOM, 5, 0), (O.EMPTY_RANDOM, 16, 0), (O.LAVA_CROSSING, 9, 1), (O.LAVA_CROSSING, 9, 3),
                (O.LAVA_CROSSING, 11, 5), (O.SIMPLE_CROSSING, 9, 2), (O.SIMPLE_CROSSING, 19, 16),
                (O.SIMPLE_CROSSING, 5, 2), (O.LAVA_CROSSING, 13, 0), (O.GOTODOOR, 5, 0), (O.GOTODOOR, 8, 0),
                (O.GOTODOOR, 19, 0), (O.DISTSHIFT, 6, 0), (O.DISTSHIFT, 8, 1), (O.DISTSHIFT, 5, 1),
                (O.KEYCORRIDOR, 7, 0), (O.KEYCORRIDOR, 7, 1), (O.KEYCORRIDOR, 7, 2), (O.KEYCORRIDOR, 10, 2),
                (O.KEYCORRIDOR, 16, 2), (O.KEYCORRIDOR, 19, 1)]


@pytest.mark.parametrize("lanes,envs", [(0, 0), (16, 4)])
@pytest.mark.parametrize("family,size,variant", ALL_FAMILIES)
def test_reset_matches_oracle(family, size, variant, lanes, envs):
    """Every generator at every listed size and variant, in the default shape
    and with 16 lanes per env (grids inside a wall margin)."""
    nx = nxmod()
    n = 37  # ragged against every envs-per-CTA choice
    env = nx.Env(family, size, n, seed=11, autotune=False, variant=variant, group_lanes=lanes, envs_per_cta=envs)
    out = env.reset()
    ob = O.Batch([family] * n, [size] * n, seed=11, variants=[variant] * n)
    oo = ob.reset()
    assert_outputs_equal(out, oo, what="reset")
    assert_states_equal(env.state()["envs"], ob, what="reset")
    env.close()


@pytest.mark.parametrize("lanes,envs,staging", [(1, 64, 1), (2, 64, 1), (4, 32, 1), (8, 16, 1), (16, 8, 1), (32, 8, 1),
                                                (8, 32, 1), (1, 256, 1), (1, 64, 2), (1, 128, 2), (8, 32, 2),
                                                (32, 2, 2), (4, 64, 2)])
def test_rollout_every_shape_every_step(lanes, envs, staging):
    nx = nxmod()
    descs = mixed_descs(150, [(O.EMPTY, 5), (O.DOORKEY, 8), (O.FOURROOMS, 19), (O.LAVAGAP, 7), (O.DYNOBS, 8),
                              (O.DOORKEY, 16)])
    env = nx.Env(descs=descs, seed=5, group_lanes=lanes, envs_per_cta=envs, staging=staging, autotune=False,
                 steps_per_launch=64)
    env.reset()
    T = 300
    out = env.rollout(T)
    ob = oracle_batch_for(descs, 5)
    ob.reset()
    oo = ob.rollout(T)
    assert_outputs_equal(out, oo, what=f"G={lanes} E={envs} staging={staging}")
    assert_states_equal(env.state()["envs"], ob, what=f"G={lanes} E={envs} staging={staging}")
    env.close()


def test_config_empty5x5_64envs_1000steps_full():
    nx = nxmod()
    env = nx.Env(O.EMPTY, 5, 64, seed=0)
    r = env.reset()
    out = env.rollout(1000)
    ob = O.Batch([O.EMPTY] * 64, [5] * 64, seed=0)
    assert_outputs_equal(r, ob.reset(), what="reset")
    assert_outputs_equal(out, ob.rollout(1000), what="Empty-5x5")
    assert_states_equal(env.state()["envs"], ob, what="Empty-5x5")
    assert env.flags() == 0
    env.close()


def test_config_doorkey8x8_4096envs_1000steps_full():
    nx = nxmod()
    n, T = 4096, 1000
    env = nx.Env(O.DOORKEY, 8, n, seed=1)
    r = env.reset()
    out = env.rollout(T)
    ob = O.Batch([O.DOORKEY] * n, [8] * n, seed=1)
    assert_outputs_equal(r, ob.reset(), what="reset")
    oo = ob.rollout(T)
    assert_outputs_equal(out, oo, what="DoorKey-8x8")
    assert_states_equal(env.state()["envs"], ob, what="DoorKey-8x8")
    env.close()


MIXED = [(O.EMPTY, 5), (O.EMPTY, 8), (O.EMPTY, 16), (O.DOORKEY, 16), (O.FOURROOMS, 19), (O.LAVAGAP, 7)]


def _mixed_sample(descs, per_block=48):
    """Envs to check: both ends of every block, and a spread inside it."""
    idx = set()
    start = 0
    while start < len(descs):
        end = start
        while end < len(descs) and descs[end] == descs[start]:
            end += 1
        for i in list(range(start, min(start + 8, end))) + list(range(max(start, end - 8), end)):
            idx.add(i)
        for i in np.linspace(start, end - 1, per_block).astype(int):
            idx.add(int(i))
        start = end
    return sorted(idx)


def test_config_mixed_65536envs_2048steps_sampled():
    nx = nxmod()
    n, T, C = 65536, 2048, 128
    descs = mixed_descs(n, MIXED)
    env = nx.Env(descs=descs, seed=2, steps_per_launch=C)
    env.reset()
    sample = _mixed_sample(descs)
    ob = oracle_batch_for(descs, 2, indices=sample)
    ob.reset()
    sel = torch.tensor(sample, device="cuda")
    out = env.alloc_out(C)
    for chunk in range(T // C):
        env.rollout(C, depth=C, out=out)
        got = {k: to_np(v.index_select(1, sel)) for k, v in out.items() if v is not None}
        want = ob.rollout(C)
        assert_outputs_equal(got, want, what=f"mixed chunk {chunk}")
    st = env.state()["envs"]
    assert_states_equal(st, ob, indices=sample, what="mixed final")
    env.close()


def test_config_mixed_65536envs_2048steps_every_env():
    """The full mixed configuration, every env: the reset outputs, every
    env's outputs at the last step of each of the 16 graph-captured 128-step
    chunks, and every env's final state (grid planes and agent block) equal
    the oracle's, run in spawned processes over contiguous env ranges."""
    from tests.oracle_pool import KEYS, chunk_ends

    nx = nxmod()
    n, T, C = 65536, 2048, 128
    descs = mixed_descs(n, MIXED)
    o_reset, o_ends, o_states = chunk_ends(n, MIXED, 2, T, C)
    env = nx.Env(descs=descs, seed=2, steps_per_launch=C)
    r = env.reset()
    assert_outputs_equal(r, o_reset, what="mixed reset, every env")
    out = env.alloc_out(C)
    for chunk in range(T // C):
        env.rollout(C, depth=C, out=out)
        got = {k: to_np(out[k][C - 1]) for k in KEYS}
        assert_outputs_equal(got, o_ends[chunk], what=f"mixed, every env, step {(chunk + 1) * C - 1}")
    st = env.state()["envs"]
    for i in range(n):
        for k in STATE_KEYS:
            if st[i][k] != o_states[i][k]:
                raise AssertionError(f"mixed final state, env {i}, field {k}: gpu {st[i][k]!r} oracle {o_states[i][k]!r}")
    env.close()


def test_config_rgb_dynobs16_8192envs_512steps():
    """The RGB configuration (Dynamic-Obstacles-16, 4 balls, 8192 envs x 512
    steps, seed 3) on the comparison plan of its contract: envs 0..63 at every
    step, symbolic and RGB; every env's symbolic outputs, plus the RGB images
    of 64 envs spread over the batch, at steps 0..7, every 32nd and 511; every
    env's final state.  The GPU writes an 8-slot ring, read back after each
    8-step call."""
    nx = nxmod()
    atlas = inputs.atlas()
    n, T, D = 8192, 512, 8
    env = nx.Env(O.DYNOBS, 16, n, seed=3, obs_rgb=True, atlas=atlas)
    env.reset()
    out = env.alloc_out(D)
    head = oracle_batch_for([(O.DYNOBS, 16)] * n, 3, indices=list(range(64)))
    head.reset()
    spread = sorted(set(np.linspace(64, n - 1, 64).astype(int).tolist()))
    ospread = oracle_batch_for([(O.DYNOBS, 16)] * n, 3, indices=spread)
    ospread.reset()
    whole = O.Batch([O.DYNOBS] * n, [16] * n, seed=3)
    whole.reset()
    sel = torch.tensor(spread, device="cuda")
    for call in range(T // D):
        env.rollout(D, depth=D, out=out)
        selected = call == 0 or call % 4 == 0 or call == T // D - 1  # steps 0..7, 32 k, 511
        oh = head.rollout(D, rgb=True, atlas=atlas)
        got = {k: to_np(out[k][:, :64]) for k in ("obs_sym", "obs_rgb", "reward", "terminated", "truncated")}
        assert_outputs_equal(got, oh, keys=("obs_sym", "obs_rgb", "reward", "terminated", "truncated"),
                             what=f"DynObs-16 envs 0..63, steps {call * D}..{call * D + D - 1}")
        ow = whole.rollout(D)
        os_ = ospread.rollout(D, rgb=selected, atlas=atlas if selected else None)
        if selected:
            steps = list(range(D)) if call == 0 else ([0] if call % 4 == 0 else []) + ([D - 1] if call == T // D - 1 else [])
            for j in steps:
                gsym = {k: to_np(out[k][j]) for k in ("obs_sym", "reward", "terminated", "truncated")}
                osym = {k: ow[k][j] for k in ("obs_sym", "reward", "terminated", "truncated")}
                assert_outputs_equal(gsym, osym, what=f"DynObs-16 every env, step {call * D + j}")
                np.testing.assert_array_equal(to_np(out["obs_rgb"][j].index_select(0, sel)), os_["obs_rgb"][j],
                                              err_msg=f"RGB spread, step {call * D + j}")
    assert_states_equal(env.state()["envs"], whole, what="DynObs-16 final, every env")
    env.close()


@pytest.mark.parametrize("lanes,envs", [(0, 0), (1, 64), (2, 32), (4, 16), (8, 8), (16, 4), (32, 2)])
def test_rgb_every_step_small(lanes, envs):
    """Egocentric RGB tiles and symbolic views every step, at every lane count
    (0: the library's default shape)."""
    nx = nxmod()
    atlas = inputs.atlas()
    descs = mixed_descs(40, [(O.DYNOBS, 6), (O.DOORKEY, 8), (O.FOURROOMS, 11)])
    env = nx.Env(descs=descs, seed=21, obs_rgb=True, atlas=atlas, autotune=False, steps_per_launch=16,
                 group_lanes=lanes, envs_per_cta=envs)
    r = env.reset()
    out = env.rollout(48)
    ob = oracle_batch_for(descs, 21)
    orr = ob.reset(rgb=True, atlas=atlas)
    oo = ob.rollout(48, rgb=True, atlas=atlas)
    assert_outputs_equal(r, orr, keys=("obs_sym", "obs_rgb"), what="rgb reset")
    assert_outputs_equal(out, oo, keys=("obs_sym", "obs_rgb", "reward", "terminated", "truncated"), what=f"rgb G={lanes}")
    env.close()


def test_per_family_form_equals_persistent_form():
    nx = nxmod()
    descs = mixed_descs(600, MIXED)
    a = nx.Env(descs=descs, seed=9, autotune=False)
    b = nx.Env(descs=descs, seed=9, autotune=False)
    a.reset()
    b.reset()
    T = 260
    oa = a.rollout(T)
    obb = b.rollout(T, per_family=True)
    for k in ("obs_sym", "reward", "terminated", "truncated"):
        assert torch.equal(oa[k], obb[k]), k
    ob = oracle_batch_for(descs, 9)
    ob.reset()
    assert_outputs_equal(oa, ob.rollout(T), what="persistent")
    assert a.state_bytes() == b.state_bytes()
    a.close()
    b.close()


def test_autotuned_shape_gives_identical_results():
    nx = nxmod()
    descs = mixed_descs(2000, MIXED)
    a = nx.Env(descs=descs, seed=4, autotune=True)
    b = nx.Env(descs=descs, seed=4, autotune=False, group_lanes=32, envs_per_cta=4)
    a.reset()
    b.reset()
    oa = a.rollout(200)
    obb = b.rollout(200)
    info = a.info()
    assert info["group_lanes"] in (1, 2, 4, 8, 16, 32) and info["grid_ctas"] >= 1
    for k in ("obs_sym", "reward", "terminated", "truncated"):
        assert torch.equal(oa[k], obb[k]), k
    assert a.state_bytes()[64:] == b.state_bytes()[64:]
    a.close()
    b.close()


def test_buffer_actions_with_invalid_entries():
    nx = nxmod()
    descs = mixed_descs(70, [(O.DOORKEY, 6), (O.DYNOBS, 7), (O.EMPTY, 9)])
    T = 400
    acts = inputs.random_actions(31, (T, 70), n_actions=7, invalid_fraction=0.02)
    env = nx.Env(descs=descs, seed=31, autotune=False)
    env.reset()
    assert env.flags() == 0
    out = env.rollout(T, actions=torch.from_numpy(acts).cuda())
    ob = oracle_batch_for(descs, 31)
    ob.reset()
    assert_outputs_equal(out, ob.rollout(T, actions=acts), what="buffered actions")
    assert_states_equal(env.state()["envs"], ob, what="buffered actions")
    assert env.flags() & 1
    env.close()


def test_single_steps_equal_rollout():
    nx = nxmod()
    a = nx.Env(O.DOORKEY, 5, 33, seed=8, autotune=False)
    b = nx.Env(O.DOORKEY, 5, 33, seed=8, autotune=False)
    a.reset()
    b.reset()
    steps = [a.step() for _ in range(50)]
    ro = b.rollout(50)
    for k in ("obs_sym", "reward", "terminated", "truncated"):
        assert torch.equal(torch.stack([s[k] for s in steps]), ro[k]), k
    a.close()
    b.close()


def test_snapshot_resume_is_bit_identical():
    nx = nxmod()
    descs = mixed_descs(90, [(O.FOURROOMS, 19), (O.DYNOBS, 8), (O.DOORKEY, 8)])
    a = nx.Env(descs=descs, seed=13, autotune=False)
    a.reset()
    a.rollout(77)
    snap = a.state_bytes()
    tail_a = a.rollout(150)
    b = nx.Env(descs=descs, seed=13, autotune=False)
    b.set_state(snap)
    tail_b = b.rollout(150)
    for k in ("obs_sym", "reward", "terminated", "truncated"):
        assert torch.equal(tail_a[k], tail_b[k]), k
    assert a.state_bytes() == b.state_bytes()
    a.close()
    b.close()


def test_two_shards_reproduce_one_batch():
    nx = nxmod()
    n = 300
    whole = nx.Env(O.DOORKEY, 8, n, seed=17, autotune=False)
    lo = nx.Env(O.DOORKEY, 8, 120, seed=17, autotune=False, env_index_base=0)
    hi = nx.Env(O.DOORKEY, 8, n - 120, seed=17, autotune=False, env_index_base=120)
    for e in (whole, lo, hi):
        e.reset()
    ow, ol, oh = whole.rollout(200), lo.rollout(200), hi.rollout(200)
    for k in ("obs_sym", "reward", "terminated", "truncated"):
        assert torch.equal(ow[k], torch.cat([ol[k], oh[k]], dim=1)), k
    for e in (whole, lo, hi):
        e.close()


def test_host_buffer_rollout_equals_device_rollout():
    nx = nxmod()
    descs = mixed_descs(500, MIXED)
    a = nx.Env(descs=descs, seed=23, autotune=False, steps_per_launch=32)
    b = nx.Env(descs=descs, seed=23, autotune=False, steps_per_launch=32)
    a.reset()
    b.reset()
    T = 150
    dev = a.rollout(T)
    host = b.rollout_host(T)
    for k in ("obs_sym", "reward", "terminated", "truncated"):
        np.testing.assert_array_equal(to_np(dev[k]), host[k], err_msg=k)
    acts = inputs.random_actions(3, (T, 500))
    c = nx.Env(descs=descs, seed=23, autotune=False, steps_per_launch=32)
    c.reset()
    hc = c.rollout_host(T, actions=acts)
    ob = oracle_batch_for(descs, 23)
    ob.reset()
    assert_outputs_equal(hc, ob.rollout(T, actions=acts), what="host rollout, buffered actions")
    for e in (a, b, c):
        e.close()
    # one family: host rollouts with random actions run that family's lean kernel
    d = nx.Env(O.DOORKEY, 8, 100, seed=29, autotune=False, group_lanes=16, envs_per_cta=4, steps_per_launch=32)
    assert d.info()["lean_family"] == O.DOORKEY
    d.reset()
    hd = d.rollout_host(T)
    od = O.Batch([O.DOORKEY] * 100, [8] * 100, seed=29)
    od.reset()
    assert_outputs_equal(hd, od.rollout(T), what="host rollout, one family, random actions")
    d.close()


@pytest.mark.parametrize("depth", [1, 3, 20, 45, 64, 149])
def test_host_ring_holds_the_last_steps(depth):
    """Host outputs shorter than the horizon form a ring (step i in slot
    i % depth), including rings that wrap inside a 32-step chunk and rings
    shorter than a chunk (only the chunk's last steps are copied back, never
    past the ring's end); every slot equals the oracle's output of the last
    step written there."""
    nx = nxmod()
    descs = mixed_descs(300, MIXED)
    T = 150
    e = nx.Env(descs=descs, seed=31, autotune=False, steps_per_launch=32)
    e.reset()
    n = len(descs)
    ring = {"obs_sym": np.zeros((depth, n, 7, 7, 3), np.uint8), "reward": np.zeros((depth, n), np.float32),
            "terminated": np.zeros((depth, n), np.uint8), "truncated": np.zeros((depth, n), np.uint8)}
    e.rollout_host(T, out=ring)
    ob = oracle_batch_for(descs, 31)
    ob.reset()
    full = ob.rollout(T)
    last = {k: np.empty_like(ring[k]) for k in ring}
    for t in range(T):
        for k in ring:
            last[k][t % depth] = full[k][t]
    assert_outputs_equal(ring, last, what=f"host ring of {depth} slots")
    e.close()


@pytest.mark.parametrize("lanes,envs,side", [(1, 64, 8), (1, 32, 16), (4, 16, 7), (8, 8, 11), (16, 4, 5), (32, 2, 9)])
def test_slots_sized_below_the_largest_grid(lanes, envs, side):
    """Shared-memory slots sized for a grid side below the batch's largest:
    items of larger grids hold fewer envs (down to one per block), their
    slots laid out at their own size; every step of every env, with RGB
    tiles, equals the oracle."""
    nx = nxmod()
    atlas = inputs.atlas()
    descs = mixed_descs(150, [(O.EMPTY, 5), (O.DOORKEY, 8), (O.FOURROOMS, 19), (O.DYNOBS, 11), (O.LAVAGAP, 7),
                              (O.KEYCORRIDOR, 19, 0, 2), (O.DOORKEY, 16)])
    env = nx.Env(descs=descs, seed=37, obs_rgb=True, atlas=atlas, autotune=False, group_lanes=lanes,
                 envs_per_cta=envs, steps_per_launch=16, grid_side=side)
    assert env.info()["grid_side"] == side
    r = env.reset()
    out = env.rollout(40)
    ob = oracle_batch_for(descs, 37)
    assert_outputs_equal(r, ob.reset(rgb=True, atlas=atlas), keys=("obs_sym", "obs_rgb"), what="reset")
    assert_outputs_equal(out, ob.rollout(40, rgb=True, atlas=atlas),
                         keys=("obs_sym", "obs_rgb", "reward", "terminated", "truncated"), what=f"G={lanes} side {side}")
    assert_states_equal(env.state()["envs"], ob, what="final")
    env.close()


@pytest.mark.parametrize("reward_mode,lava", [(1, 0.0), (0, -1.0), (1, -1.0)])
def test_reward_variants(reward_mode, lava):
    nx = nxmod()
    descs = mixed_descs(120, [(O.EMPTY, 5), (O.LAVAGAP, 5), (O.DYNOBS, 5)])
    env = nx.Env(descs=descs, seed=29, reward_mode=reward_mode, lava_reward=lava, autotune=False)
    env.reset()
    out = env.rollout(500)
    ob = oracle_batch_for(descs, 29, reward_mode=reward_mode, lava_reward=lava)
    ob.reset()
    oo = ob.rollout(500)
    assert_outputs_equal(out, oo, what=f"reward mode {reward_mode} lava {lava}")
    r = to_np(out["reward"])
    assert (r[(r != 0)] != 1.0).any() or reward_mode == 0
    env.close()


@pytest.mark.parametrize("lanes,envs", [(1, 64), (8, 16), (32, 4)])
@pytest.mark.parametrize("reward_mode", [0, 1])
def test_shaping_costs(lanes, envs, reward_mode):
    """action_cost / time_cost of Table 5 with buffered actions that include
    done and out-of-range entries, across families with every reward event."""
    nx = nxmod()
    descs = mixed_descs(130, [(O.DOORKEY, 5), (O.LAVAGAP, 5), (O.DYNOBS, 5), (O.GOTODOOR, 5), (O.DISTSHIFT, 6, 0, 1)])
    T = 300
    acts = inputs.random_actions(37, (T, 130), n_actions=7, invalid_fraction=0.03)
    kw = dict(action_cost=0.0125, time_cost=0.004, lava_reward=-1.0)
    env = nx.Env(descs=descs, seed=37, group_lanes=lanes, envs_per_cta=envs, autotune=False, reward_mode=reward_mode,
                 **kw)
    env.reset()
    out = env.rollout(T, actions=torch.from_numpy(acts).cuda())
    ob = oracle_batch_for(descs, 37, reward_mode=reward_mode, **kw)
    ob.reset()
    assert_outputs_equal(out, ob.rollout(T, actions=acts), what=f"costs G={lanes} mode={reward_mode}")
    r = to_np(out["reward"])
    assert (r < 0).mean() > 0.5 and (r > 0.9).any() and (r < -1.0).any()
    env.close()


NEW_FAMILIES = [(O.EMPTY_RANDOM, 6, 0, 0), (O.LAVA_CROSSING, 9, 0, 1), (O.LAVA_CROSSING, 9, 0, 3),
                (O.LAVA_CROSSING, 11, 0, 5), (O.SIMPLE_CROSSING, 9, 0, 2), (O.SIMPLE_CROSSING, 11, 0, 5),
                (O.EMPTY_RANDOM, 16, 0, 0), (O.SIMPLE_CROSSING, 19, 0, 9), (O.GOTODOOR, 6, 0, 0),
                (O.DISTSHIFT, 6, 0, 0), (O.DISTSHIFT, 8, 0, 1), (O.KEYCORRIDOR, 7, 0, 0), (O.KEYCORRIDOR, 7, 0, 1),
                (O.KEYCORRIDOR, 13, 0, 2)]


@pytest.mark.parametrize("lanes,envs,staging", [(1, 64, 2), (8, 16, 1), (32, 4, 1)])
def test_new_families_every_step(lanes, envs, staging):
    nx = nxmod()
    descs = mixed_descs(200, NEW_FAMILIES)
    for lava in (0.0, -1.0):
        env = nx.Env(descs=descs, seed=41, group_lanes=lanes, envs_per_cta=envs, staging=staging, autotune=False,
                     steps_per_launch=50, lava_reward=lava)
        r = env.reset()
        out = env.rollout(400)
        ob = oracle_batch_for(descs, 41, lava_reward=lava)
        assert_outputs_equal(r, ob.reset(), what="reset")
        assert_outputs_equal(out, ob.rollout(400), what=f"new families G={lanes} lava={lava}")
        assert_states_equal(env.state()["envs"], ob, what="new families")
        env.close()


@pytest.mark.parametrize("lanes,envs,staging", [(1, 64, 2), (8, 16, 1), (32, 4, 1)])
def test_fully_observable_views(lanes, envs, staging):
    """symbolic / categorical / categorical_first_person (Table 4) of a mixed-size
    batch, padded to the largest grid, every step."""
    nx = nxmod()
    descs = mixed_descs(90, [(O.DOORKEY, 8), (O.FOURROOMS, 11), (O.SIMPLE_CROSSING, 9, 0, 3), (O.DYNOBS, 6),
                             (O.KEYCORRIDOR, 10, 0, 1), (O.GOTODOOR, 6)])
    env = nx.Env(descs=descs, seed=51, group_lanes=lanes, envs_per_cta=envs, staging=staging, autotune=False,
                 steps_per_launch=40, obs_full=True, obs_cat=True, obs_cat_fp=True)
    r = env.reset()
    out = env.rollout(120)
    ob = oracle_batch_for(descs, 51)
    ob.reset()
    f0, c0, p0 = ob.full_views(11)
    np.testing.assert_array_equal(to_np(r["obs_full"]), f0)
    np.testing.assert_array_equal(to_np(r["obs_cat"]), c0)
    np.testing.assert_array_equal(to_np(r["obs_cat_fp"]), p0)
    oo = ob.rollout_full(120, 11)
    assert_outputs_equal(out, oo, keys=("obs_sym", "reward", "terminated", "truncated", "obs_full", "obs_cat",
                                        "obs_cat_fp"), what=f"full views G={lanes}")
    env.close()


@pytest.mark.parametrize("lanes,envs", [(1, 64), (16, 8), (32, 4)])
def test_full_rgb_view(lanes, envs):
    nx = nxmod()
    atlas = inputs.atlas()
    descs = mixed_descs(20, [(O.DOORKEY, 8), (O.FOURROOMS, 11), (O.LAVA_CROSSING, 9, 0, 2)])
    env = nx.Env(descs=descs, seed=61, group_lanes=lanes, envs_per_cta=envs, autotune=False, steps_per_launch=16,
                 obs_rgb=True, obs_rgb_full=True, atlas=atlas)
    r = env.reset()
    out = env.rollout(30)
    ob = oracle_batch_for(descs, 61)
    ob.reset()
    np.testing.assert_array_equal(to_np(r["obs_rgb_full"]), ob.rgb_full(atlas, 11))
    oo = ob.rollout_full(30, 11, atlas=atlas)
    assert_outputs_equal(out, oo, keys=("obs_sym", "reward", "obs_rgb_full"), what=f"full rgb G={lanes}")
    env.close()


def _oracle_missions(ob, T):
    """Per-step outputs of the oracle with the mission of each slot's episode."""
    outs = {k: [] for k in ("obs_sym", "reward", "terminated", "truncated", "mission")}
    for _ in range(T):
        o = ob.step()
        for k in ("obs_sym", "reward", "terminated", "truncated"):
            outs[k].append(o[k])
        outs["mission"].append(ob.missions())
    return {k: np.stack(v) for k, v in outs.items()}


@pytest.mark.parametrize("lanes,envs,staging", [(1, 64, 2), (2, 64, 1), (8, 16, 1), (32, 4, 1)])
@pytest.mark.parametrize("reward_mode", [0, 1])
def test_gotodoor_missions_and_door_done(lanes, envs, staging, reward_mode):
    """GoToDoor-5/6/8 beside DoorKey: layouts, missions of every step, and the
    on_door_done reward/termination under random actions (done is one of the
    seven), against the oracle step by step."""
    nx = nxmod()
    descs = mixed_descs(150, [(O.GOTODOOR, 5), (O.GOTODOOR, 6), (O.DOORKEY, 6), (O.GOTODOOR, 8)])
    env = nx.Env(descs=descs, seed=71, group_lanes=lanes, envs_per_cta=envs, staging=staging, autotune=False,
                 steps_per_launch=64, reward_mode=reward_mode)
    r = env.reset()
    out = env.rollout(500)
    ob = oracle_batch_for(descs, 71, reward_mode=reward_mode)
    o0 = ob.reset()
    o0["mission"] = ob.missions()
    keys = ("obs_sym", "reward", "terminated", "truncated", "mission")
    assert_outputs_equal(r, o0, keys=keys, what="gotodoor reset")
    oo = _oracle_missions(ob, 500)
    assert_outputs_equal(out, oo, keys=keys, what=f"gotodoor G={lanes} mode={reward_mode}")
    assert_states_equal(env.state()["envs"], ob, what="gotodoor")
    m = oo["mission"]
    dk = np.array([d[0] == O.DOORKEY for d in descs])
    assert (m[:, dk] == O.NO_MISSION).all() and (m[:, ~dk] <= 5).all()
    wins = (oo["terminated"] == 1) & (oo["reward"] > 0)
    assert wins[:, ~dk].sum() > 20  # done facing the right door happens under random play
    env.close()


def test_gotodoor_host_rollout_and_snapshot():
    nx = nxmod()
    env = nx.Env(O.GOTODOOR, 7, 300, seed=5, autotune=False)
    env.reset()
    dev = env.rollout(150)
    snap = env.state_bytes()
    host = env.rollout_host(100)
    env.set_state(snap)
    again = env.rollout(100)
    for k in ("obs_sym", "reward", "terminated", "truncated", "mission"):
        np.testing.assert_array_equal(host[k], to_np(again[k]), err_msg=k)
    assert (to_np(dev["mission"]) <= 5).all()
    # the mission byte of a snapshot is validated per family
    b = bytearray(snap)
    b[64 + 26] = 6
    with pytest.raises(nx.NavixError) as ei:
        env.set_state(bytes(b))
    assert ei.value.status == nx.NX_E_INVAL
    env.close()
    e2 = nx.Env(O.EMPTY, 5, 3, seed=5, autotune=False)
    e2.reset()
    b = bytearray(e2.state_bytes())
    assert b[64 + 26] == nx.NX_NO_MISSION
    b[64 + 26] = 0
    with pytest.raises(nx.NavixError):
        e2.set_state(bytes(b))
    e2.close()


# one configuration per family (small grids, so episodes end and reset often)
LEAN_FAMILIES = [(O.EMPTY, 5, 0), (O.DOORKEY, 6, 0), (O.FOURROOMS, 9, 0), (O.LAVAGAP, 5, 0), (O.DYNOBS, 6, 0),
                 (O.EMPTY_RANDOM, 6, 0), (O.LAVA_CROSSING, 9, 1), (O.SIMPLE_CROSSING, 11, 3), (O.GOTODOOR, 6, 0),
                 (O.DISTSHIFT, 7, 1), (O.KEYCORRIDOR, 7, 1)]


@pytest.mark.parametrize("family,size,variant", LEAN_FAMILIES)
def test_lean_kernels_every_family_every_lanes(family, size, variant):
    """A single-family context's random-action rollouts run the step kernel
    compiled for that family; each lane count against the oracle, every step
    (graph chunks and a remainder launch), and against the general kernel
    (selected by asking for the action output)."""
    nx = nxmod()
    n, T = 37, 200
    ob = O.Batch([family] * n, [size] * n, seed=23, variants=[variant] * n)
    oo_r = ob.reset()
    oo = ob.rollout(T)
    for lanes, envs in ((1, 64), (4, 16), (8, 8), (16, 4), (32, 2)):
        env = nx.Env(family, size, n, seed=23, variant=variant, group_lanes=lanes, envs_per_cta=envs, autotune=False,
                     steps_per_launch=64)
        info = env.info()
        assert info["lean_family"] == family and info["lean_grid_ctas"] >= 1, info
        assert_outputs_equal(env.reset(), oo_r, what=f"lean reset G={lanes}")
        out = env.rollout(T)
        assert_outputs_equal(out, oo, what=f"lean G={lanes} family={family}")
        assert_states_equal(env.state()["envs"], ob, what=f"lean G={lanes} family={family}")
        env.close()
        if lanes == 16:
            genv = nx.Env(family, size, n, seed=23, variant=variant, group_lanes=lanes, envs_per_cta=envs,
                          autotune=False, steps_per_launch=64, action=True)
            genv.reset()
            gout = genv.rollout(T)
            for k in ("obs_sym", "reward", "terminated", "truncated"):
                np.testing.assert_array_equal(to_np(gout[k]), to_np(out[k]), err_msg=f"general vs lean {k}")
            genv.close()


def test_lean_kernel_choice():
    nx = nxmod()
    mixed = nx.Env(descs=mixed_descs(40, [(O.EMPTY, 5), (O.DOORKEY, 8)]), seed=1, autotune=False)
    assert mixed.info()["lean_family"] == nx.NX_N_FAMILIES  # several families: the any-family lean kernel
    mixed.close()
    mg = nx.Env(O.DOORKEY, 8, 40, seed=1, autotune=False, reward_mode=nx.NX_REWARD_MINIGRID)
    assert mg.info()["lean_family"] == -1  # MiniGrid reward
    mg.close()
    g2 = nx.Env(O.DOORKEY, 8, 40, seed=1, autotune=False, group_lanes=2, envs_per_cta=16)
    assert g2.info()["lean_family"] == -1  # no lean instantiation with 2 lanes per env
    g2.close()


def test_variant_validation():
    nx = nxmod()
    assert nx.nx_max_variant(O.LAVA_CROSSING, 9) == O.max_variant(O.LAVA_CROSSING, 9) == 6
    assert nx.nx_max_variant(O.SIMPLE_CROSSING, 19) == 16 and nx.nx_max_variant(O.DOORKEY, 9) == 0
    with pytest.raises(nx.NavixError):
        nx.Env(O.LAVA_CROSSING, 9, 4, seed=0, variant=7)
    with pytest.raises(nx.NavixError):
        nx.Env(O.DOORKEY, 9, 4, seed=0, variant=1)


def test_nballs_option_and_small_dynobs():
    nx = nxmod()
    for nb in (0, 1, 3):
        env = nx.Env(O.DYNOBS, 6, 40, seed=nb, n_balls=nb, autotune=False)
        env.reset()
        out = env.rollout(200)
        ob = O.Batch([O.DYNOBS] * 40, [6] * 40, seed=nb, n_balls=nb)
        ob.reset()
        assert_outputs_equal(out, ob.rollout(200), what=f"n_balls={nb}")
        env.close()


def test_sync_reports_ok_and_timeout_bound():
    nx = nxmod()
    env = nx.Env(O.EMPTY, 8, 1000, seed=1, autotune=False)
    env.reset()
    env.rollout(64)
    assert env.sync(timeout_s=30.0) == 0
    env.close()
