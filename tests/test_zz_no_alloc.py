"""The allocation-free rollout entry point, nx_rollout_noalloc, against the
regular entry points.

nx_rollout_noalloc serves callers whose process cannot call cudaMalloc (the
device memory is already held by another runtime's pool, or the loop cannot
afford cudaMalloc's implicit synchronisation): it keeps its scratch in one
fixed device array inside the library.  Two calls in a row, with different
families, sizes and action sources, must each give exactly the outputs of
nx_create + nx_reset + nx_rollout (every comparison in this suite is exact).
This file is collected last so that a failure here never hides the others.
"""
import pytest

torch = pytest.importorskip("torch")

from paper_2407_19396_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2407_19396_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def _regular(nx, family, size, n, seed, T, actions):
    env = nx.Env(family, size, n, seed=seed, autotune=False)
    env.reset()
    out = env.rollout(T, actions=actions)
    torch.cuda.synchronize()
    env.close()
    return out


def _regular_ring(nx, family, size, n, seed, T, actions, depth):
    env = nx.Env(family, size, n, seed=seed, autotune=False)
    env.reset()
    out = env.rollout(T, actions=actions, depth=depth)
    torch.cuda.synchronize()
    env.close()
    return out


def _noalloc(nx, family, size, n, seed, T, actions, depth=None):
    D = depth or T
    env_like = {"obs_sym": torch.empty((D, n, 7, 7, 3), dtype=torch.uint8, device="cuda"),
                "reward": torch.empty((D, n), dtype=torch.float32, device="cuda"),
                "terminated": torch.empty((D, n), dtype=torch.uint8, device="cuda"),
                "truncated": torch.empty((D, n), dtype=torch.uint8, device="cuda")}
    o = nx.nx_out()
    o.obs_sym = env_like["obs_sym"].data_ptr()
    o.obs_rgb = None
    o.reward = env_like["reward"].data_ptr()
    o.terminated = env_like["terminated"].data_ptr()
    o.truncated = env_like["truncated"].data_ptr()
    o.depth = D
    mode = nx.NX_ACT_RANDOM if actions is None else nx.NX_ACT_BUFFER
    ptr = None if actions is None else actions.data_ptr()
    nx.nx_rollout_noalloc(family, size, n, seed, T, mode, ptr, o, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return env_like


def test_noalloc_rollout_matches_regular_entry_points_twice_in_a_row():
    from paper_2407_19396_gb300 import navixgb as nx

    calls = [
        (nx.NX_DOORKEY, 8, 500, 41, 300, None),
        (nx.NX_DYNOBS, 6, 200, 42, 150,
         torch.from_numpy(inputs.random_actions(42, (150, 200), n_actions=3)).cuda()),
    ]
    for family, size, n, seed, T, acts in calls:
        got = _noalloc(nx, family, size, n, seed, T, acts)
        want = _regular(nx, family, size, n, seed, T, acts)
        for k in ("obs_sym", "reward", "terminated", "truncated"):
            assert torch.equal(got[k], want[k]), f"family {family}: {k} differs"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2407_19396_gb300 import navixgb as nx

    limit = nx.lib()  # noqa: F841  (loads the library)
    with pytest.raises(nx.NavixError) as ei:
        nx.nx_rollout_noalloc(nx.NX_FOURROOMS, 19, 8192, 0, 1, nx.NX_ACT_RANDOM, None, None, 0)
    assert ei.value.status == nx.NX_E_INVAL
    assert "fixed scratch" in str(ei.value)


def test_noalloc_at_its_size_limit_and_with_an_output_ring():
    """3757 FourRooms-19x19 envs fill the scratch array to within a few
    hundred bytes (3758 no longer fit); a ring shorter than the horizon keeps
    step i in slot i % depth.  Both equal the regular entry points exactly."""
    from paper_2407_19396_gb300 import navixgb as nx

    got = _noalloc(nx, nx.NX_FOURROOMS, 19, 3757, 7, 130, None)
    want = _regular(nx, nx.NX_FOURROOMS, 19, 3757, 7, 130, None)
    for k in ("obs_sym", "reward", "terminated", "truncated"):
        assert torch.equal(got[k], want[k]), f"FourRooms-19 at the limit: {k} differs"
    with pytest.raises(nx.NavixError) as ei:
        nx.nx_rollout_noalloc(nx.NX_FOURROOMS, 19, 3758, 7, 1, nx.NX_ACT_RANDOM, None, None, 0)
    assert ei.value.status == nx.NX_E_INVAL and "fixed scratch" in str(ei.value)
    got = _noalloc(nx, nx.NX_LAVAGAP, 7, 300, 9, 150, None, depth=64)
    want = _regular_ring(nx, nx.NX_LAVAGAP, 7, 300, 9, 150, None, 64)
    for k in ("obs_sym", "reward", "terminated", "truncated"):
        assert torch.equal(got[k], want[k]), f"64-slot ring: {k} differs"


def test_noalloc_against_the_oracle_and_degenerate_calls():
    """The outputs equal the CPU oracle's; a call with no outputs, a call of
    zero steps and a call asking for an output it does not write behave as
    documented, and the next call is unaffected."""
    import numpy as np

    import oracle as O
    from paper_2407_19396_gb300 import navixgb as nx

    s = torch.cuda.current_stream().cuda_stream
    nx.nx_rollout_noalloc(nx.NX_DOORKEY, 8, 100, 3, 40, nx.NX_ACT_RANDOM, None, None, s)  # no outputs
    nx.nx_rollout_noalloc(nx.NX_DOORKEY, 8, 100, 3, 0, nx.NX_ACT_RANDOM, None, None, s)  # reset only
    o = nx.nx_out()
    extra = torch.empty((4, 37), dtype=torch.uint8, device="cuda")
    o.mission = extra.data_ptr()
    o.depth = 4
    with pytest.raises(nx.NavixError) as ei:
        nx.nx_rollout_noalloc(nx.NX_DOORKEY, 5, 37, 3, 4, nx.NX_ACT_RANDOM, None, o, s)
    assert ei.value.status == nx.NX_E_INVAL
    T = 90
    got = _noalloc(nx, nx.NX_DOORKEY, 5, 37, 3, T, None)
    b = O.Batch([O.DOORKEY] * 37, [5] * 37, seed=3)
    b.reset()
    want = b.rollout(T)
    for k in ("obs_sym", "reward", "terminated", "truncated"):
        np.testing.assert_array_equal(got[k].cpu().numpy(), want[k], err_msg=k)


@pytest.mark.parametrize("case", range(16))
def test_noalloc_random_configurations_against_the_oracle(case):
    """Seeded random calls -- any family at a random size, 1 to 600 envs, 1
    to 300 steps, an output ring or not, random or buffered actions -- each
    equal to the oracle at every kept step."""
    import numpy as np

    import oracle as O
    from paper_2407_19396_gb300 import navixgb as nx

    rng = np.random.default_rng(9700 + case)
    f = int(rng.integers(0, 11))
    size = int(rng.choice([s for s in range(5, 20) if O.max_variant(f, s) >= 0]))
    n, T = int(rng.integers(1, 601)), int(rng.integers(1, 301))
    depth = T if rng.random() < 0.5 else int(rng.integers(1, T + 1))
    seed = int(rng.integers(0, 2**31))
    acts = (inputs.random_actions(seed & 0xFFFF, (T, n), n_actions=7, invalid_fraction=0.02)
            if rng.random() < 0.4 else None)
    got = _noalloc(nx, f, size, n, seed, T, None if acts is None else torch.from_numpy(acts).cuda(), depth)
    b = O.Batch([f] * n, [size] * n, seed=seed)
    b.reset()
    want = b.rollout(T, actions=acts)
    for k in ("obs_sym", "reward", "terminated", "truncated"):
        ring = np.empty((depth,) + want[k].shape[1:], want[k].dtype)
        for t in range(T - depth, T):
            ring[t % depth] = want[k][t]
        np.testing.assert_array_equal(got[k].cpu().numpy(), ring, err_msg=f"case {case} family {f} size {size} "
                                                                             f"n {n} T {T} depth {depth} {k}")
