"""Continuous-batching server (config C5) on the GPU.

Every request's result (per-env returns, final view, ended episodes, digest of
every per-step output) must be the same when it runs alone and when it shares
the GPU with other requests admitted before, with and after it, and must equal
the oracle's.  Exact comparison throughout.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from tests.gpu_util import oracle_request  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2407_19396_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def _mix(seed, n, max_envs=300, max_h=300):
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(n):
        fam = int(rng.integers(0, 5))
        size = int(rng.integers(5, 20))
        ne = int(min(max_envs, max(1, np.floor(np.exp(rng.uniform(0, np.log(max_envs + 1)))))))
        h = int(rng.integers(1, max_h + 1))
        reqs.append((fam, size, ne, h, int(rng.integers(0, 2**63))))
    return reqs


def _same(a, b):
    np.testing.assert_array_equal(a["returns"], b["returns"])
    np.testing.assert_array_equal(a["final_obs"], b["final_obs"])
    assert a["episodes"] == b["episodes"]
    assert a["digest"] == b["digest"]


def test_results_same_alone_in_the_mix_and_in_the_oracle():
    from paper_2407_19396_gb300 import navixgb as nx

    reqs = _mix(4, 36)
    srv = nx.Server(budget_bytes=256 << 20, steps_per_launch=32)
    tickets = [srv.submit(*r) for r in reqs]
    mixed = [srv.wait(t, timeout_s=120.0) for t in tickets]
    st = srv.stats()
    assert st["finished"] == len(reqs) and st["chunks"] >= 2
    srv.close()
    for r, m in zip(reqs, mixed):
        assert m["status"] == 0 and m["env_steps"] == r[2] * r[3]
        alone_srv = nx.Server(budget_bytes=64 << 20, steps_per_launch=32)
        alone = alone_srv.wait(alone_srv.submit(*r), timeout_s=120.0)
        alone_srv.close()
        _same(m, alone)
        _same(m, oracle_request(r[0], r[1], r[2], r[3], r[4]))


def test_digest_is_optional_and_changes_nothing_else():
    from paper_2407_19396_gb300 import navixgb as nx

    reqs = _mix(11, 8, max_envs=200, max_h=200)
    srv = nx.Server(budget_bytes=256 << 20, steps_per_launch=32)
    with_d = [srv.wait(srv.submit(*r), timeout_s=120.0) for r in reqs]
    without = [srv.wait(srv.submit(*r, digest=False), timeout_s=120.0) for r in reqs]
    for r, a, b in zip(reqs, with_d, without):
        np.testing.assert_array_equal(a["returns"], b["returns"])
        np.testing.assert_array_equal(a["final_obs"], b["final_obs"])
        assert a["episodes"] == b["episodes"] and b["digest"] == 0
        assert a["digest"] == oracle_request(r[0], r[1], r[2], r[3], r[4])["digest"]
    with pytest.raises(nx.NavixError):
        bad = nx.nx_request(0, 5, 1, 1, 0, 2, 1, 0, 0)  # an unknown flag bit
        nx.nx_submit(srv.h, bad)
    srv.close()


def test_requests_arriving_while_others_run_are_admitted_and_correct():
    from paper_2407_19396_gb300 import navixgb as nx
    import time

    reqs = _mix(7, 24, max_envs=400, max_h=500)
    srv = nx.Server(budget_bytes=256 << 20, steps_per_launch=16)
    tickets = []
    for i, r in enumerate(reqs):
        tickets.append(srv.submit(*r))
        if i % 4 == 3:
            time.sleep(0.002)
    res = [srv.wait(t, timeout_s=120.0) for t in tickets]
    srv.close()
    # overlap: some request started before an earlier-submitted one finished
    starts = [x["t_start"] for x in res]
    dones = [x["t_done"] for x in res]
    assert any(starts[j] < dones[i] for i in range(len(res)) for j in range(i + 1, len(res)))
    for r, m in zip(reqs, res):
        _same(m, oracle_request(r[0], r[1], r[2], r[3], r[4]))


def test_budget_admission_and_rejection():
    from paper_2407_19396_gb300 import navixgb as nx

    budget = 4 << 20  # room for about two of the requests below at a time
    srv = nx.Server(budget_bytes=budget, steps_per_launch=64)
    reqs = [(O.FOURROOMS, 19, 1200, 130, 100 + i) for i in range(5)]
    tickets = [srv.submit(*r) for r in reqs]
    res = [srv.wait(t, timeout_s=120.0) for t in tickets]
    st = srv.stats()
    assert st["peak_bytes"] <= budget and st["finished"] == 5
    # strictly first come, first served: later requests start after earlier ones
    starts = [x["t_start"] for x in res]
    assert starts == sorted(starts)
    assert max(starts) > min(x["t_done"] for x in res)  # the budget forced some to wait
    with pytest.raises(nx.NavixError) as ei:
        srv.submit(O.FOURROOMS, 19, 4096, 10, 1)
    assert ei.value.status == nx.NX_E_BUDGET
    srv.close()
    for r, m in zip(reqs[:2], res[:2]):
        _same(m, oracle_request(*r))


def test_new_families_served_like_the_oracle():
    from paper_2407_19396_gb300 import navixgb as nx

    reqs = [(O.LAVA_CROSSING, 11, 40, 120, 1, 5), (O.SIMPLE_CROSSING, 9, 17, 90, 2, 3), (O.EMPTY_RANDOM, 8, 33, 70, 3, 0),
            (O.GOTODOOR, 6, 29, 150, 4, 0), (O.DISTSHIFT, 8, 21, 100, 5, 1),
            (O.KEYCORRIDOR, 10, 19, 130, 6, 2)]
    srv = nx.Server(budget_bytes=64 << 20, steps_per_launch=32)
    tickets = [srv.submit(f, s_, n, h, seed, variant=v) for f, s_, n, h, seed, v in reqs]
    res = [srv.wait(t, timeout_s=120.0) for t in tickets]
    srv.close()
    for (f, s_, n, h, seed, v), m in zip(reqs, res):
        _same(m, oracle_request(f, s_, n, h, seed, variant=v))


def test_served_rewards_with_shaping_costs():
    from paper_2407_19396_gb300 import navixgb as nx

    kw = dict(action_cost=0.02, time_cost=0.001, lava_reward=-1.0)
    reqs = [(O.DISTSHIFT, 6, 25, 80, 7, 0), (O.GOTODOOR, 5, 31, 120, 8, 0), (O.LAVAGAP, 6, 12, 60, 9, 0)]
    srv = nx.Server(budget_bytes=64 << 20, steps_per_launch=32, **kw)
    tickets = [srv.submit(f, s_, n, h, seed, variant=v) for f, s_, n, h, seed, v in reqs]
    res = [srv.wait(t, timeout_s=120.0) for t in tickets]
    srv.close()
    for (f, s_, n, h, seed, v), m in zip(reqs, res):
        _same(m, oracle_request(f, s_, n, h, seed, variant=v, **kw))


def test_wait_timeout_is_bounded():
    from paper_2407_19396_gb300 import navixgb as nx

    srv = nx.Server(budget_bytes=64 << 20, steps_per_launch=128)
    t = srv.submit(O.DOORKEY, 16, 4000, 4000, 5)
    with pytest.raises(nx.NavixError) as ei:
        srv.wait(t, timeout_s=1e-4)
    assert ei.value.status == nx.NX_E_TIMEOUT
    r = srv.wait(t, timeout_s=300.0)
    assert r["status"] == 0
    srv.close()


def test_concurrent_submitters_and_waiters():
    """Several client threads submit while others wait (the request table is
    modified while the worker reads it); every result must still match the
    oracle."""
    import threading

    from paper_2407_19396_gb300 import navixgb as nx

    srv = nx.Server(budget_bytes=128 << 20, steps_per_launch=8)
    reqs = _mix(11, 90, max_envs=64, max_h=60)
    results = {}
    lock = threading.Lock()

    def client(part):
        mine = []
        for r in part:
            mine.append((r, srv.submit(*r)))
        for r, t in mine:
            res = srv.wait(t, timeout_s=120.0)
            with lock:
                results[r] = res

    threads = [threading.Thread(target=client, args=(reqs[i::6],)) for i in range(6)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    srv.close()
    assert len(results) == len(reqs)
    for r in reqs[:30]:
        _same(results[r], oracle_request(*r))


# (lanes per env, envs per block, staging parts); (0, 0, 0): the server's own shapes
SERVER_SHAPES = [(0, 0, 0), (1, 64, 2), (1, 128, 1), (4, 32, 1), (8, 16, 1), (16, 8, 1), (32, 4, 1)]


def _random_requests(rng, n, max_envs, max_h):
    """Requests of every family at its valid sizes and variants."""
    reqs = []
    for _ in range(n):
        f = int(rng.integers(0, 11))
        s = int(rng.choice([x for x in range(5, 20) if O.max_variant(f, x) >= 0]))
        v = int(rng.integers(0, O.max_variant(f, s) + 1))
        ne = int(min(max_envs, max(1, np.floor(np.exp(rng.uniform(0, np.log(max_envs + 1)))))))
        reqs.append((f, s, ne, int(rng.integers(1, max_h + 1)), int(rng.integers(0, 2**63)), v,
                     bool(rng.random() < 0.7)))
    return reqs


@pytest.mark.parametrize("case", range(12))
def test_random_request_mixes_match_the_oracle(case):
    """Seeded random servers (launch shape, chunk length, budget, reward mode,
    lava reward, shaping costs, balls) serving random request mixes (every
    family, size and variant, 1 to 600 envs, 1 to 300 steps, with or without
    the digest) submitted in bursts: every result equals the oracle's."""
    import time

    from paper_2407_19396_gb300 import navixgb as nx

    rng = np.random.default_rng(9100 + case)
    lanes, envs, staging = SERVER_SHAPES[int(rng.integers(0, len(SERVER_SHAPES)))]
    kw = dict(reward_mode=int(rng.integers(0, 2)), lava_reward=float(rng.choice([0.0, -1.0])),
              action_cost=float(rng.choice([0.0, 0.0125])), time_cost=float(rng.choice([0.0, 0.004])),
              n_balls=int(rng.integers(0, 5)))
    spl = int(rng.choice([1, 8, 32, 128]))
    budget = int(rng.choice([16 << 20, 64 << 20, 256 << 20]))
    reqs = _random_requests(rng, 20, 600, 300)
    what = f"case {case}: shape {(lanes, envs, staging)} spl {spl} budget {budget} {kw}"
    srv = nx.Server(budget_bytes=budget, steps_per_launch=spl, group_lanes=lanes, envs_per_cta=envs, staging=staging,
                    **kw)
    try:
        tickets = []
        for r in reqs:
            tickets.append(srv.submit(*r[:6], digest=r[6]))
            if rng.random() < 0.3:
                time.sleep(float(rng.uniform(0.0, 0.003)))
        res = [srv.wait(t, timeout_s=120.0) for t in tickets]
        assert srv.stats()["peak_bytes"] <= budget, what
    finally:
        srv.close()
    for r, m in zip(reqs, res):
        f, s, ne, h, seed, v, dig = r
        assert m["status"] == 0 and m["env_steps"] == ne * h, f"{what} {r}"
        o = oracle_request(f, s, ne, h, seed, variant=v, **kw)
        np.testing.assert_array_equal(m["returns"], o["returns"], err_msg=f"{what} {r}")
        np.testing.assert_array_equal(m["final_obs"], o["final_obs"], err_msg=f"{what} {r}")
        assert m["episodes"] == o["episodes"], f"{what} {r}"
        assert m["digest"] == (o["digest"] if dig else 0), f"{what} {r}"


@pytest.mark.parametrize("case", range(4))
def test_random_cancellations_leave_the_rest_exact(case):
    """Random requests, a random third of them withdrawn at random moments
    (queued, running or already finished): a withdrawn request reports
    NX_E_CANCELED, one that finished first refuses the withdrawal and keeps
    its result, every other result equals the oracle's, and the server
    ends with all its memory back."""
    import time

    from paper_2407_19396_gb300 import navixgb as nx

    rng = np.random.default_rng(9200 + case)
    reqs = _random_requests(rng, 30, 1000, 400)
    srv = nx.Server(budget_bytes=int(rng.choice([8 << 20, 32 << 20])), steps_per_launch=int(rng.choice([8, 32, 128])))
    try:
        tickets, canceled = [], set()
        for i, r in enumerate(reqs):
            tickets.append(srv.submit(*r[:6], digest=r[6]))
            if rng.random() < 0.3:
                time.sleep(float(rng.uniform(0.0, 0.004)))
            if i >= 2 and rng.random() < 0.35:
                j = int(rng.integers(max(0, i - 5), i + 1))  # a recent request: queued, running or done
                if j not in canceled:
                    try:
                        srv.cancel(tickets[j])
                        canceled.add(j)
                    except nx.NavixError as e:
                        assert e.status == nx.NX_E_STATE  # finished before the withdrawal
        finished = []
        for i, t in enumerate(tickets):
            if i in canceled:
                with pytest.raises(nx.NavixError) as ei:
                    srv.wait(t, timeout_s=120.0)
                assert ei.value.status == nx.NX_E_CANCELED
            else:
                finished.append((reqs[i], srv.wait(t, timeout_s=120.0)))
        st = srv.stats()
        assert st["canceled"] == len(canceled) and st["finished"] == len(finished)
        assert st["in_use_bytes"] == 0
    finally:
        srv.close()
    assert canceled
    for r, m in finished:
        f, s, ne, h, seed, v, dig = r
        o = oracle_request(f, s, ne, h, seed, variant=v)
        np.testing.assert_array_equal(m["returns"], o["returns"], err_msg=str(r))
        np.testing.assert_array_equal(m["final_obs"], o["final_obs"], err_msg=str(r))
        assert m["episodes"] == o["episodes"] and m["digest"] == (o["digest"] if dig else 0), r
