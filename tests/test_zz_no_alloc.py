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


def _noalloc(nx, family, size, n, seed, T, actions):
    env_like = {"obs_sym": torch.empty((T, n, 7, 7, 3), dtype=torch.uint8, device="cuda"),
                "reward": torch.empty((T, n), dtype=torch.float32, device="cuda"),
                "terminated": torch.empty((T, n), dtype=torch.uint8, device="cuda"),
                "truncated": torch.empty((T, n), dtype=torch.uint8, device="cuda")}
    o = nx.nx_out()
    o.obs_sym = env_like["obs_sym"].data_ptr()
    o.obs_rgb = None
    o.reward = env_like["reward"].data_ptr()
    o.terminated = env_like["terminated"].data_ptr()
    o.truncated = env_like["truncated"].data_ptr()
    o.depth = T
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
