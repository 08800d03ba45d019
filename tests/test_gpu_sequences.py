"""Randomised call sequences: one context driven through a seeded random
sequence of the C-ABI's calls -- single steps, device rollouts and host-buffer
rollouts of random lengths with output rings, random or buffered actions,
resets, and snapshots restored into a fresh context that carries on -- while
the oracle steps the same batch alongside.  Every output of every call, and
the state at the end, must equal the oracle's byte for byte: the step
counters, ring slots, episode counters and snapshots agree across calls.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2407_19396_gb300 import inputs  # noqa: E402
from tests.gpu_util import assert_outputs_equal, assert_states_equal, oracle_batch_for  # noqa: E402
from tests.test_gpu_fuzz import SHAPES, oracle_steps, ring_of  # noqa: E402

pytestmark = pytest.mark.gpu

N_CASES = 24
OPS = ("step", "rollout", "rollout_host", "snapshot", "reset")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2407_19396_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def draw_sequence(i):
    """Case i: a batch, a context configuration and a call sequence."""
    rng = np.random.default_rng(9500 + i)
    k = int(rng.integers(1, 4))
    parts = []
    for f in rng.choice(11, size=k, replace=False):
        f = int(f)
        s = int(rng.choice([x for x in range(5, 20) if O.max_variant(f, x) >= 0]))
        ms = int(rng.integers(3, 40)) if rng.random() < 0.3 else 0
        parts.append((f, s, ms, int(rng.integers(0, O.max_variant(f, s) + 1))))
    n = int(rng.integers(1, 400))
    descs = [parts[int(j)] for j in rng.integers(0, k, size=n)]
    lanes, envs, staging = SHAPES[int(rng.integers(0, len(SHAPES)))]
    kw = dict(reward_mode=int(rng.integers(0, 2)), lava_reward=float(rng.choice([0.0, -1.0])),
              action_cost=float(rng.choice([0.0, 0.0125])), time_cost=float(rng.choice([0.0, 0.004])),
              n_balls=int(rng.integers(0, 5)))
    ops = []
    for _ in range(int(rng.integers(4, 10))):
        op = OPS[int(rng.choice(len(OPS), p=[0.25, 0.3, 0.2, 0.15, 0.1]))]
        T = int(rng.integers(1, 150))
        ops.append(dict(op=op, T=T, depth=T if rng.random() < 0.5 else int(rng.integers(1, T + 1)),
                        buffered=bool(rng.random() < 0.4), aseed=int(rng.integers(0, 2**16))))
    c = dict(descs=descs, seed=int(rng.integers(0, 2**31)), lanes=lanes, envs=envs, staging=staging,
             spl=int(rng.choice([1, 7, 64, 128])), kw=kw, ops=ops)
    # a snapshot is restored into a context of its own launch shape (or an
    # autotuned one): snapshots do not depend on where the envs ran
    c["autotune"] = bool(rng.random() < 0.25)
    for op in ops:
        op["shape"] = SHAPES[int(rng.integers(0, len(SHAPES)))]
        op["autotune"] = bool(rng.random() < 0.25)
    return c


def _keys(missions):
    return ("obs_sym", "reward", "terminated", "truncated") + (("mission",) if missions else ())


@pytest.mark.parametrize("case", range(N_CASES))
def test_random_call_sequence_matches_the_oracle(case):
    from paper_2407_19396_gb300 import navixgb as nx

    c = draw_sequence(case)
    descs, n = c["descs"], len(c["descs"])

    def make(shape, autotune):
        return nx.Env(descs=descs, seed=c["seed"], autotune=autotune, group_lanes=shape[0], envs_per_cta=shape[1],
                      staging=shape[2], steps_per_launch=c["spl"], **c["kw"])

    env = make((c["lanes"], c["envs"], c["staging"]), c["autotune"])
    ob = oracle_batch_for(descs, c["seed"], **c["kw"])
    missions = env.want_mission
    keys = _keys(missions)
    try:
        r0 = env.reset()
        o0 = ob.reset()
        if missions:
            o0["mission"] = ob.missions()
        assert_outputs_equal(r0, o0, keys=keys, what=f"case {case} first reset")
        for j, op in enumerate(c["ops"]):
            what = f"case {case} call {j} {op} (n={n}, shape={c['lanes'], c['envs'], c['staging']}, spl={c['spl']})"
            T, depth = op["T"], op["depth"]
            acts = (inputs.random_actions(op["aseed"], (T, n), n_actions=7, invalid_fraction=0.02)
                    if op["buffered"] else None)
            if op["op"] == "step":
                g = env.step(None if acts is None else torch.from_numpy(acts[0]).cuda())
                oo = oracle_steps(ob, 1, None if acts is None else acts[:1], missions)
                assert_outputs_equal(g, {k: v[0] for k, v in oo.items()}, keys=keys, what=what)
            elif op["op"] == "rollout":
                g = env.rollout(T, depth=depth, actions=None if acts is None else torch.from_numpy(acts).cuda())
                oo = oracle_steps(ob, T, acts, missions)
                assert_outputs_equal(g, {k: ring_of(v, T, depth) for k, v in oo.items()}, keys=keys, what=what)
            elif op["op"] == "rollout_host":
                out = {"obs_sym": np.zeros((depth, n, 7, 7, 3), np.uint8), "reward": np.zeros((depth, n), np.float32),
                       "terminated": np.zeros((depth, n), np.uint8), "truncated": np.zeros((depth, n), np.uint8),
                       "mission": np.zeros((depth, n), np.uint8) if missions else None}
                g = env.rollout_host(T, actions=acts, out=out)
                oo = oracle_steps(ob, T, acts, missions)
                assert_outputs_equal(g, {k: ring_of(v, T, depth) for k, v in oo.items()}, keys=keys, what=what)
            elif op["op"] == "snapshot":
                snap = env.state_bytes()
                env.close()
                env = make(op["shape"], op["autotune"])
                env.set_state(snap)
                assert env.state_bytes() == snap, what
                assert_states_equal(env.state()["envs"], ob, what=what)
            else:
                g = env.reset()
                oo = ob.reset()
                if missions:
                    oo["mission"] = ob.missions()
                assert_outputs_equal(g, oo, keys=keys, what=what)
        torch.cuda.synchronize()
        assert_states_equal(env.state()["envs"], ob, what=f"case {case} final state")
        assert env.flags() & ~1 == 0, f"case {case}"
    finally:
        env.close()


def test_the_sequences_cover_every_call():
    seqs = [draw_sequence(i) for i in range(N_CASES)]
    seen = {op["op"] for s in seqs for op in s["ops"]}
    assert seen == set(OPS)
    assert sum(op["op"] == "snapshot" for s in seqs for op in s["ops"]) >= 5
    assert any(op["op"] == "rollout_host" and op["depth"] < op["T"] for s in seqs for op in s["ops"])
    assert any(s["lanes"] == 1 for s in seqs) and any(s["lanes"] >= 8 for s in seqs)
    assert any(s["autotune"] for s in seqs)
    assert any(op["op"] == "snapshot" and op["shape"] != (s["lanes"], s["envs"], s["staging"]) for s in seqs
               for op in s["ops"])


@pytest.mark.parametrize("case", range(4))
def test_two_contexts_interleaved_on_two_streams(case):
    """Two contexts of different batches and launch shapes, each on its own
    stream, issue their rollouts alternately without waiting for each other;
    each context's outputs equal the oracle's for its batch alone."""
    from paper_2407_19396_gb300 import navixgb as nx

    cfg = [draw_sequence(case), draw_sequence(case + N_CASES // 2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    envs, outs = [], [[], []]
    rng = np.random.default_rng(9900 + case)
    Ts = [[int(t) for t in rng.integers(1, 150, size=3)] for _ in range(2)]
    try:
        for c, st in zip(cfg, streams):
            with torch.cuda.stream(st):
                e = nx.Env(descs=c["descs"], seed=c["seed"], autotune=False, group_lanes=c["lanes"],
                           envs_per_cta=c["envs"], staging=c["staging"], steps_per_launch=c["spl"], **c["kw"])
                e.reset()
                envs.append(e)
        for r in range(3):
            for k in range(2):
                with torch.cuda.stream(streams[k]):
                    outs[k].append(envs[k].rollout(Ts[k][r]))
        torch.cuda.synchronize()
        for k in range(2):
            c = cfg[k]
            ob = oracle_batch_for(c["descs"], c["seed"], **c["kw"])
            ob.reset()
            for r in range(3):
                oo = oracle_steps(ob, Ts[k][r], None, False)
                assert_outputs_equal(outs[k][r], oo, what=f"case {case} context {k} rollout {r}")
            assert_states_equal(envs[k].state()["envs"], ob, what=f"case {case} context {k}")
    finally:
        for e in envs:
            e.close()
