"""The fused policy + environment rollout (tensor-core policy inside the step
kernel) against the oracle's integer MLP, every step, element by element."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from tests.gpu_util import assert_outputs_equal, assert_states_equal, mixed_descs, oracle_batch_for, to_np  # noqa: E402
from tests.test_oracle_policy import wall_turner  # noqa: E402

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


def random_policy(A, seed, wmax=12, bmax=300, shift1=3, shift2=6, epsilon=0, epa=128):
    rng = np.random.default_rng(seed)
    w = dict(w1=rng.integers(-wmax, wmax + 1, (A, 64, 49)), b1=rng.integers(-bmax, bmax + 1, (A, 64)),
             w2=rng.integers(-wmax, wmax + 1, (A, 64, 64)), b2=rng.integers(-bmax, bmax + 1, (A, 64)),
             w3=rng.integers(-wmax, wmax + 1, (A, 7, 64)), b3=rng.integers(-bmax, bmax + 1, (A, 7)))
    return O.Policy(**w, shift1=shift1, shift2=shift2, epsilon=epsilon, envs_per_agent=epa)


def gpu_env_with(nx, descs, seed, pol, **kw):
    env = nx.Env(descs=descs, seed=seed, autotune=False, action=True, **kw)
    env.set_policy(pol.w1, pol.b1, pol.w2, pol.b2, pol.w3, pol.b3, pol.shift1, pol.shift2, pol.epsilon,
                   pol.envs_per_agent)
    return env


KEYS = ("obs_sym", "reward", "terminated", "truncated", "action")


@pytest.mark.parametrize("parts,A,epa,eps,T", [
    ([(O.DOORKEY, 8)], 2, 128, 0, 300),
    ([(O.DYNOBS, 6)], 1, 256, 2**30, 260),
    ([(O.EMPTY, 5), (O.FOURROOMS, 11)], 4, 128, 2**28, 300),
    ([(O.KEYCORRIDOR, 10, 0, 2), (O.LAVA_CROSSING, 9, 0, 2)], 2, 256, 0, 200),
    # several weight sets per 128-env block: the PPO pattern of many agents x 16 envs
    ([(O.DOORKEY, 8)], 16, 16, 0, 200),
    ([(O.EMPTY, 5), (O.FOURROOMS, 11)], 8, 32, 2**28, 200),
    ([(O.DYNOBS, 6)], 4, 64, 0, 200),
    ([(O.EMPTY, 6)], 11, 16, 2**30, 150),  # a ragged last block: 176 envs, 3 of 8 sets in it
])
def test_policy_rollout_matches_the_oracle(parts, A, epa, eps, T):
    nx = nxmod()
    descs = mixed_descs(A * epa, parts)
    pol = random_policy(A, seed=len(parts) + A, epsilon=eps, epa=epa)
    env = gpu_env_with(nx, descs, 23, pol)
    env.reset()
    out = env.rollout(T, policy=True)
    ob = oracle_batch_for(descs, 23)
    ob.reset()
    oo = ob.rollout_policy(T, pol)
    oo["action"] = oo.pop("actions")
    assert_outputs_equal(out, oo, keys=KEYS, what="policy rollout")
    assert_states_equal(env.state()["envs"], ob, what="policy rollout")
    acts = oo["action"]
    assert len(np.unique(acts)) >= 3  # the random weights do not collapse to one action
    assert env.flags() & 4 == 0       # no bounded wait gave up
    env.close()


def test_policy_workload_full_size_sampled():
    """The benchmark's policy workload at full size -- Empty-8x8, 32,768 envs =
    256 agents x 128 envs, the seeded weights, shifts 3 and 6, exploration
    1/16 -- for 200 steps; envs sampled across the agents (first, last and
    interior ones) against the oracle, every step."""
    from paper_2407_19396_gb300 import inputs

    nx = nxmod()
    n, A, epa, T = 32768, 256, 128, 200
    pw = inputs.policy_weights(5, A)
    env = nx.Env(O.EMPTY, 8, n, seed=5, action=True)
    env.set_policy(pw["w1"], pw["b1"], pw["w2"], pw["b2"], pw["w3"], pw["b3"], 3, 6, 1 << 28, epa)
    env.reset()
    out = env.rollout(T, policy=True)
    sample = sorted(set([0, 1, 127, 128, 255, 16383, 16384, n - 129, n - 2, n - 1] + list(range(300, n, 1031))))
    idx = torch.tensor(sample, device="cuda")
    got = {k: out[k].index_select(1, idx).cpu().numpy() for k in KEYS}
    pol = O.Policy(**pw, shift1=3, shift2=6, epsilon=1 << 28, envs_per_agent=epa)
    ob = O.Batch([O.EMPTY] * len(sample), [8] * len(sample), seed=5, env_indices=sample)
    ob.reset()
    oo = ob.rollout_policy(T, pol)
    oo["action"] = oo.pop("actions")
    assert_outputs_equal(got, oo, keys=KEYS, what="policy workload, sampled")
    assert env.flags() & 4 == 0
    env.close()


def test_hand_built_policy_on_the_gpu():
    nx = nxmod()
    pol = wall_turner()
    descs = [(O.FOURROOMS, 13)] * 128
    env = gpu_env_with(nx, descs, 4, pol)
    env.reset()
    out = env.rollout(150, policy=True)
    ob = oracle_batch_for(descs, 4)
    ob.reset()
    oo = ob.rollout_policy(150, pol)
    oo["action"] = oo.pop("actions")
    assert_outputs_equal(out, oo, keys=KEYS, what="wall turner")
    assert set(np.unique(to_np(out["action"]))) <= {1, 2}
    env.close()


def test_policy_then_random_then_policy_continue_one_trajectory():
    nx = nxmod()
    descs = [(O.DOORKEY, 6)] * 128
    pol = random_policy(1, seed=8, epsilon=2**29)
    env = gpu_env_with(nx, descs, 6, pol)
    env.reset()
    a = env.rollout(70, policy=True)
    b = env.rollout(50)
    c = env.rollout(90, policy=True)
    ob = oracle_batch_for(descs, 6)
    ob.reset()
    oa = ob.rollout_policy(70, pol)
    obb = ob.rollout(50)
    oc = ob.rollout_policy(90, pol)
    for got, want in ((a, oa), (b, obb), (c, oc)):
        assert_outputs_equal(got, want, what="interleaved policy / random")
    # the action output of the random-action rollout is the counter hash's draw
    g0 = 70
    ra = to_np(b["action"])
    for i in (0, 17, 127):
        e = O.Env(O.DOORKEY, 6, seed=6, env_index=i)
        assert [e.random_action(g0 + t) for t in range(50)] == list(ra[:, i])
    env.close()


def test_policy_validation():
    nx = nxmod()
    pol = random_policy(2, seed=1, epa=128)
    # a 128-env block of the work list straddling two weight sets
    env = nx.Env(descs=[(O.DOORKEY, 6)] * 100 + [(O.EMPTY, 6)] * 156, seed=0, autotune=False)
    with pytest.raises(nx.NavixError) as ei:
        env.set_policy(pol.w1, pol.b1, pol.w2, pol.b2, pol.w3, pol.b3, 3, 6, 0, 128)
    assert ei.value.status == nx.NX_E_INVAL
    env.close()
    # envs per weight set below 128 must divide the block and be >= 16, and the
    # blocks must start at a weight-set boundary
    p16 = random_policy(16, seed=2, epa=16)
    env = nx.Env(O.DOORKEY, 6, 256, seed=0, autotune=False)
    for epa in (8, 48, 100):
        with pytest.raises(nx.NavixError) as ei:
            env.set_policy(p16.w1, p16.b1, p16.w2, p16.b2, p16.w3, p16.b3, 3, 6, 0, epa)
        assert ei.value.status == nx.NX_E_INVAL
    env.close()
    env = nx.Env(descs=[(O.DOORKEY, 6)] * 40 + [(O.EMPTY, 6)] * 216, seed=0, autotune=False)
    with pytest.raises(nx.NavixError) as ei:
        env.set_policy(p16.w1, p16.b1, p16.w2, p16.b2, p16.w3, p16.b3, 3, 6, 0, 16)  # a block starts at env 40
    assert ei.value.status == nx.NX_E_INVAL
    env.close()
    env = nx.Env(O.DOORKEY, 6, 256, seed=0, autotune=False)
    env.reset()
    with pytest.raises(nx.NavixError) as ei:
        env.rollout(3, policy=True)  # no policy yet
    assert ei.value.status == nx.NX_E_STATE
    big = pol.b1.copy()
    big[0, 0] = 1 << 23
    for args in ((pol.w1, big, pol.w2, pol.b2, pol.w3, pol.b3, 3, 6, 0, 128),   # bias out of range
                 (pol.w1, pol.b1, pol.w2, pol.b2, pol.w3, pol.b3, 25, 6, 0, 128),  # shift out of range
                 (pol.w1[:1], pol.b1[:1], pol.w2[:1], pol.b2[:1], pol.w3[:1], pol.b3[:1], 3, 6, 0, 128)):  # too few sets
        with pytest.raises(nx.NavixError) as ei:
            env.set_policy(*args)
        assert ei.value.status == nx.NX_E_INVAL
    env.close()


def test_policy_snapshot_resume_and_shards():
    nx = nxmod()
    pol = random_policy(4, seed=12, epsilon=2**29, epa=128)
    # one context of 512 envs ...
    whole = gpu_env_with(nx, [(O.DOORKEY, 8)] * 512, 31, pol)
    whole.reset()
    a = whole.rollout(100, policy=True)
    # ... equals two shards of 256 over disjoint global env ranges, each with the whole weight table
    outs = []
    for base in (0, 256):
        sh = nx.Env(descs=[(O.DOORKEY, 8)] * 256, seed=31, autotune=False, action=True, env_index_base=base)
        sh.set_policy(pol.w1, pol.b1, pol.w2, pol.b2, pol.w3, pol.b3, pol.shift1, pol.shift2, pol.epsilon, 128)
        sh.reset()
        outs.append(sh.rollout(100, policy=True))
        sh.close()
    for k in KEYS:
        np.testing.assert_array_equal(to_np(a[k]), np.concatenate([to_np(o[k]) for o in outs], axis=1), err_msg=k)
    # a snapshot taken mid-rollout resumes the same trajectory
    snap = whole.state_bytes()
    b1 = whole.rollout(60, policy=True)
    b1 = {k: to_np(v) for k, v in b1.items() if v is not None}
    whole.set_state(snap)
    b2 = whole.rollout(60, policy=True)
    for k in KEYS:
        np.testing.assert_array_equal(b1[k], to_np(b2[k]), err_msg=k)
    whole.close()


def _policy_case(i):
    """Case i of the random sweep: a weight-set size, the agents, a family run
    layout that respects the work list's weight-set boundaries (runs of a
    multiple of envs_per_agent below 128 envs per set; runs inside one set
    from 128 on), exploration, shifts, weight ranges and reward settings."""
    rng = np.random.default_rng(9300 + i)
    epa = int(rng.choice([16, 32, 64, 128, 256]))
    A = int(rng.integers(1, max(1, 1024 // epa) + 1))
    pool = []
    for f in rng.choice(11, size=3, replace=False):
        f = int(f)
        s = int(rng.choice([x for x in range(5, 20) if O.max_variant(f, x) >= 0]))
        pool.append((f, s, 0, int(rng.integers(0, O.max_variant(f, s) + 1))))
    descs = []
    for _ in range(A):
        if epa < 128:
            descs += [pool[int(rng.integers(0, 3))]] * epa
        else:
            cuts = sorted(int(c) for c in rng.choice(np.arange(1, epa), size=int(rng.integers(0, 3)), replace=False))
            for k, (lo, hi) in enumerate(zip([0] + cuts, cuts + [epa])):
                d = pool[int(rng.integers(0, 3))]
                if k == 0 and descs and d == descs[-1]:
                    d = pool[(pool.index(d) + 1) % 3]  # equal neighbours would merge into a run across the sets
                descs += [d] * (hi - lo)
    kw = dict(reward_mode=int(rng.integers(0, 2)), action_cost=float(rng.choice([0.0, 0.0125])),
              time_cost=float(rng.choice([0.0, 0.004])), lava_reward=float(rng.choice([0.0, -1.0])))
    return dict(epa=epa, A=A, descs=descs, kw=kw, eps=int(rng.choice([0, 2**28, 2**30])),
                shift1=int(rng.integers(2, 5)), shift2=int(rng.integers(5, 8)), wmax=int(rng.choice([6, 12, 20])),
                T=int(rng.integers(50, 200)), seed=int(rng.integers(0, 2**31)))


@pytest.mark.parametrize("case", range(8))
def test_random_policy_configurations_match_the_oracle(case):
    nx = nxmod()
    c = _policy_case(case)
    what = f"case {case}: epa {c['epa']} A {c['A']} eps {c['eps']} shifts {c['shift1']},{c['shift2']} {c['kw']}"
    pol = random_policy(c["A"], seed=c["seed"] & 0xFFFF, wmax=c["wmax"], shift1=c["shift1"], shift2=c["shift2"],
                        epsilon=c["eps"], epa=c["epa"])
    env = gpu_env_with(nx, c["descs"], c["seed"], pol, **c["kw"])
    try:
        env.reset()
        out = env.rollout(c["T"], policy=True)
        ob = oracle_batch_for(c["descs"], c["seed"], **c["kw"])
        ob.reset()
        oo = ob.rollout_policy(c["T"], pol)
        oo["action"] = oo.pop("actions")
        assert_outputs_equal(out, oo, keys=KEYS, what=what)
        assert_states_equal(env.state()["envs"], ob, what=what)
        assert env.flags() & 4 == 0, what
    finally:
        env.close()
