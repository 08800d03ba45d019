"""Edge cases and error paths of the C ABI on the GPU (exact comparisons with
the oracle where outputs are produced)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from tests.gpu_util import assert_outputs_equal, assert_states_equal, mixed_descs, oracle_batch_for, to_np  # noqa: E402

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


def test_single_env_every_family():
    nx = nxmod()
    for fam, size, var in [(O.EMPTY, 5, 0), (O.DOORKEY, 19, 0), (O.FOURROOMS, 5, 0), (O.DYNOBS, 19, 0),
                           (O.LAVA_CROSSING, 19, 16), (O.EMPTY_RANDOM, 19, 0)]:
        env = nx.Env(fam, size, 1, seed=77, variant=var)
        env.reset()
        out = env.rollout(300)
        ob = O.Batch([fam], [size], seed=77, variants=[var])
        ob.reset()
        assert_outputs_equal(out, ob.rollout(300), what=f"single env family {fam}")
        env.close()


@pytest.mark.parametrize("spl", [1, 7, 1024])
def test_steps_per_launch_extremes_and_ring_wrap(spl):
    nx = nxmod()
    descs = mixed_descs(70, [(O.DOORKEY, 6), (O.LAVAGAP, 5)])
    env = nx.Env(descs=descs, seed=8, steps_per_launch=spl, autotune=False)
    env.reset()
    T, D = 1100, 3
    out = env.rollout(T, depth=D)
    ob = oracle_batch_for(descs, 8)
    ob.reset()
    oo = ob.rollout(T)
    # slot i % D holds step i: the ring keeps the last D steps
    slots = [(T - D + i) % D for i in range(D)]
    got = {k: to_np(out[k])[slots] for k in ("obs_sym", "reward", "terminated", "truncated")}
    want = {k: oo[k][T - D:] for k in ("obs_sym", "reward", "terminated", "truncated")}
    assert_outputs_equal(got, want, what=f"steps_per_launch={spl}")
    assert_states_equal(env.state()["envs"], ob, what=f"steps_per_launch={spl}")
    env.close()


def test_many_more_envs_than_resident_ctas():
    nx = nxmod()
    n = 200_000
    env = nx.Env(O.EMPTY, 5, n, seed=12, group_lanes=32, envs_per_cta=8, autotune=False)
    env.reset()
    out = env.rollout(12)
    sample = sorted(set([0, 1, 2, n // 3, n // 2, n - 2, n - 1] + list(range(1000, n, 9973))))
    ob = O.Batch([O.EMPTY] * len(sample), [5] * len(sample), seed=12, env_indices=sample)
    ob.reset()
    oo = ob.rollout(12)
    got = {k: to_np(out[k])[:, sample] for k in ("obs_sym", "reward", "terminated", "truncated")}
    assert_outputs_equal(got, oo, what="200k envs")
    env.close()


def test_paper_batch_scale_sampled():
    """The paper's batch-mode scale: Empty-8x8, 2^21 envs (autotuned shape,
    the lean kernel), a 1-slot output ring; after 40 steps the last step's
    outputs of sampled envs equal the oracle's."""
    nx = nxmod()
    n, T = 1 << 21, 40
    env = nx.Env(O.EMPTY, 8, n, seed=6)
    env.reset()
    out = env.rollout(T, depth=1)
    sample = sorted(set([0, 1, 31, 32, n // 2, n - 33, n - 1] + list(range(777, n, 65537))))
    idx = torch.tensor(sample, device="cuda")
    got = {k: out[k].index_select(1, idx).cpu().numpy() for k in ("obs_sym", "reward", "terminated", "truncated")}
    ob = O.Batch([O.EMPTY] * len(sample), [8] * len(sample), seed=6, env_indices=sample)
    ob.reset()
    oo = ob.rollout(T)
    want = {k: oo[k][T - 1:] for k in ("obs_sym", "reward", "terminated", "truncated")}
    assert_outputs_equal(got, want, what="2^21 envs, last step")
    env.close()


def test_state_pool_beyond_4_gib():
    """4,000,000 FourRooms-19x19 envs: a 4.33 GB grid pool, so the envs past
    index 3,965,000 have their planes beyond the first 4 GiB (64-bit work
    item offsets); sampled envs on both sides of that mark, after 6 steps
    with a 1-slot ring, equal the oracle."""
    nx = nxmod()
    n, T = 4_000_000, 6
    assert n * 3 * 19 * 19 > 1 << 32
    env = nx.Env(O.FOURROOMS, 19, n, seed=15, autotune=False, group_lanes=1, envs_per_cta=64)
    env.reset()
    out = env.rollout(T, depth=1)
    edge = (1 << 32) // (3 * 19 * 19)
    sample = sorted(set([0, 1, edge - 2, edge - 1, edge, edge + 1, n - 2, n - 1] + list(range(12345, n, 333331))))
    idx = torch.tensor(sample, device="cuda")
    got = {k: out[k].index_select(1, idx).cpu().numpy() for k in ("obs_sym", "reward", "terminated", "truncated")}
    del out
    ob = O.Batch([O.FOURROOMS] * len(sample), [19] * len(sample), seed=15, env_indices=sample)
    ob.reset()
    oo = ob.rollout(T)
    want = {k: oo[k][T - 1:] for k in ("obs_sym", "reward", "terminated", "truncated")}
    assert_outputs_equal(got, want, what="4M FourRooms-19 envs, last step")
    env.close()


def test_server_places_requests_beyond_4_gib():
    """A 16 GiB serving budget: a blocker request of 3.4 M FourRooms-19x19
    envs (about 4.4 GB) takes the start of the pool, so the next request's
    block lies past the first 4 GiB; its result equals the oracle's, and the
    blocker is then withdrawn."""
    from tests.gpu_util import oracle_request

    nx = nxmod()
    srv = nx.Server(budget_bytes=16 << 30, steps_per_launch=64)
    blocker = srv.submit(O.FOURROOMS, 19, 3_400_000, 100000, 21, digest=False)
    small = srv.submit(O.DOORKEY, 9, 300, 77, 22)
    res = srv.wait(small, timeout_s=300.0)
    want = oracle_request(O.DOORKEY, 9, 300, 77, 22)
    np.testing.assert_array_equal(res["returns"], want["returns"])
    np.testing.assert_array_equal(res["final_obs"], want["final_obs"])
    assert res["digest"] == want["digest"] and res["episodes"] == want["episodes"]
    assert srv.stats()["peak_bytes"] > (4 << 30)
    srv.cancel(blocker)
    with pytest.raises(nx.NavixError) as ei:
        srv.wait(blocker, timeout_s=300.0)
    assert ei.value.status == nx.NX_E_CANCELED
    assert srv.stats()["in_use_bytes"] == 0
    srv.close()


@pytest.mark.parametrize("lanes,envs", [(1, 64), (16, 4)])
def test_tiny_max_steps_truncate_every_few_steps(lanes, envs):
    """max_steps 1, 2 and 3 (a truncation on every step or every few, so an
    autoreset every other call) beside a long horizon, several families, and
    one family alone (its lean kernel); every step against the oracle."""
    nx = nxmod()
    descs = mixed_descs(60, [(O.DOORKEY, 8, 1), (O.FOURROOMS, 9, 2), (O.DYNOBS, 6, 3), (O.LAVAGAP, 7, 1000),
                             (O.KEYCORRIDOR, 7, 2, 1)])
    for d in (descs, [(O.DOORKEY, 8, 2)] * 37):
        env = nx.Env(descs=d, seed=44, group_lanes=lanes, envs_per_cta=envs, autotune=False, steps_per_launch=16)
        env.reset()
        out = env.rollout(100)
        ob = oracle_batch_for(d, 44)
        ob.reset()
        oo = ob.rollout(100)
        assert_outputs_equal(out, oo, what=f"tiny max_steps G={lanes}")
        assert_states_equal(env.state()["envs"], ob, what=f"tiny max_steps G={lanes}")
        assert oo["truncated"].sum() > 0
        env.close()


def test_reset_twice_restarts_everything():
    nx = nxmod()
    env = nx.Env(O.FOURROOMS, 11, 50, seed=3, autotune=False)
    r1 = env.reset()
    a = env.rollout(90)
    r1 = {k: v.clone() if v is not None else None for k, v in r1.items()}
    a = {k: v.clone() if v is not None else None for k, v in a.items()}
    r2 = env.reset()
    b = env.rollout(90)
    for k in ("obs_sym", "reward", "terminated", "truncated"):
        assert torch.equal(r1[k], r2[k]) and torch.equal(a[k], b[k]), k
    env.close()


def test_calls_out_of_order_and_bad_arguments():
    nx = nxmod()
    env = nx.Env(O.EMPTY, 5, 4, seed=0, autotune=False)
    with pytest.raises(nx.NavixError) as ei:
        env.rollout(3)  # before nx_reset
    assert ei.value.status == nx.NX_E_STATE
    env.reset()
    out = env.alloc_out(3)
    s = env.out_struct(out, 3)
    with pytest.raises(nx.NavixError) as ei:
        nx.nx_rollout(env.h, 3, 7, None, s)  # unknown action source
    assert ei.value.status == nx.NX_E_INVAL
    with pytest.raises(nx.NavixError) as ei:
        nx.nx_rollout(env.h, 3, nx.NX_ACT_BUFFER, None, s)  # buffered actions without a buffer
    assert ei.value.status == nx.NX_E_INVAL
    with pytest.raises(nx.NavixError) as ei:
        nx.nx_rollout(env.h, -1, nx.NX_ACT_RANDOM, None, s)
    assert ei.value.status == nx.NX_E_INVAL
    fake_rgb = torch.empty(16, dtype=torch.uint8, device="cuda")
    s.obs_rgb = fake_rgb.data_ptr()
    with pytest.raises(nx.NavixError) as ei:
        nx.nx_rollout(env.h, 3, nx.NX_ACT_RANDOM, None, s)  # RGB was not enabled at creation
    assert ei.value.status == nx.NX_E_INVAL
    s.obs_rgb = None
    s.obs_full = fake_rgb.data_ptr()
    s.full_side = 3
    with pytest.raises(nx.NavixError) as ei:
        nx.nx_rollout(env.h, 3, nx.NX_ACT_RANDOM, None, s)  # full views narrower than the grid
    assert ei.value.status == nx.NX_E_INVAL
    assert nx.nx_rollout(env.h, 0, nx.NX_ACT_RANDOM, None, None) == 0  # zero steps is a no-op
    assert env.sync(timeout_s=10.0) == 0
    env.close()


def test_corrupt_snapshots_are_rejected():
    nx = nxmod()
    env = nx.Env(O.DOORKEY, 6, 5, seed=1, autotune=False)
    env.reset()
    env.rollout(20)
    good = env.state_bytes()
    before = env.state_bytes()

    def corrupt(fn):
        b = bytearray(good)
        fn(b)
        with pytest.raises(nx.NavixError) as ei:
            env.set_state(bytes(b))
        assert ei.value.status == nx.NX_E_INVAL

    corrupt(lambda b: b.__setitem__(0, ord("X")))               # magic
    corrupt(lambda b: b.__setitem__(8, 9))                      # env count
    corrupt(lambda b: b.__setitem__(64 + 0, 200))               # agent x outside the grid
    corrupt(lambda b: b.__setitem__(64 + 2, 7))                 # direction
    corrupt(lambda b: b.__setitem__(64 + 5 * 32 + 3 * 36, 77))  # a grid cell's entity code
    with pytest.raises(nx.NavixError):
        env.set_state(good[:100])                                # too short
    assert env.state_bytes() == before                           # nothing was applied
    env.set_state(good)
    env.close()


def test_dynamic_obstacles_snapshot_balls_stay_in_the_interior():
    """A restored Dynamic-Obstacles env must hold its balls in the grid's
    interior (reset places them there and they only move to empty cells):
    a ball on the border wall is refused, and a valid snapshot resumes the
    oracle's trajectory exactly."""
    nx = nxmod()
    n, S = 6, 7
    env = nx.Env(O.DYNOBS, S, n, seed=3, autotune=False)
    env.reset()
    env.rollout(25)
    good = env.state_bytes()
    st = nx.parse_state(good)
    for e in st["envs"]:
        assert e["n_balls"] == 4
        assert all(1 <= v <= S - 2 for v in e["ball_x"] + e["ball_y"])
    for field_off, bad in ((16, 0), (16, S - 1), (20, 0), (20, S - 1)):  # ball 0's column / row
        b = bytearray(good)
        b[64 + 2 * 32 + field_off] = bad  # env 2's agent block
        with pytest.raises(nx.NavixError) as ei:
            env.set_state(bytes(b))
        assert ei.value.status == nx.NX_E_INVAL
    env.set_state(good)
    out = env.rollout(40)
    ob = O.Batch([O.DYNOBS] * n, [S] * n, seed=3)
    ob.reset()
    ob.rollout(25)
    oo = ob.rollout(40)
    assert_outputs_equal({k: to_np(out[k]) for k in ("obs_sym", "reward", "terminated", "truncated")}, oo,
                         what="Dynamic-Obstacles after a restore")
    env.close()


def test_snapshot_of_one_context_rejected_by_another_shape():
    nx = nxmod()
    a = nx.Env(O.DOORKEY, 6, 5, seed=1, autotune=False)
    b = nx.Env(O.DOORKEY, 7, 5, seed=1, autotune=False)
    a.reset()
    b.reset()
    with pytest.raises(nx.NavixError):
        b.set_state(a.state_bytes())
    a.close()
    b.close()


def test_binding_refuses_bad_output_buffers_before_any_launch():
    """Output buffers too small, of another element type, non-contiguous or
    in the wrong memory are refused by the binding (ValueError) before the
    library sees a pointer; the context's state is untouched and the next
    call with good buffers runs normally."""
    nx = nxmod()
    n = 40
    env = nx.Env(O.DOORKEY, 8, n, seed=3, autotune=False, obs_full=True)
    env.reset()
    snap = env.state_bytes()
    good = env.alloc_out(16)
    bads = [dict(good, obs_sym=good["obs_sym"][:8]),                                    # 8 slots for a 16-step ring
            dict(good, reward=torch.empty((16, n), dtype=torch.uint8, device="cuda")),  # 1-byte rewards
            dict(good, terminated=torch.empty((n, 16), dtype=torch.uint8, device="cuda").t()),  # not contiguous
            dict(good, truncated=torch.empty((16, n), dtype=torch.uint8)),              # host memory
            dict(good, obs_full=torch.empty((16, n, 7, 7, 3), dtype=torch.uint8, device="cuda"))]  # side 7, not 8
    for b in bads:
        with pytest.raises(ValueError):
            env.rollout(16, out=b)
    with pytest.raises(ValueError):
        env.step(out=dict(env.alloc_out(), obs_sym=torch.empty((n - 1, 7, 7, 3), dtype=torch.uint8, device="cuda")))
    with pytest.raises(ValueError):
        env.rollout_host(16, out={"obs_sym": np.zeros((16, n, 7, 7, 3), np.uint8), "reward": np.zeros((16, n), np.float64),
                                  "terminated": None, "truncated": None, "mission": None})
    torch.cuda.synchronize()
    assert env.state_bytes() == snap
    out = env.rollout(16, out=good)
    ob = oracle_batch_for([(O.DOORKEY, 8)] * n, 3)
    ob.reset()
    assert_outputs_equal(out, ob.rollout(16), what="after the refused calls")
    env.close()
