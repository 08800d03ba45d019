"""Benchmark of the batched MiniGrid step (NAVIX, arXiv 2407.19396) on GB300.

One bench step is one complete rollout of the workload's batch: every env of
the batch advances ``T`` environment steps through the fused CUDA step kernel
(action draw, autoreset, transition, rules, reward/termination, egocentric
view with occlusion, observation stores), run as graph-captured persistent
chunks.  ``value`` counts env-steps (one env advanced by one step) per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the CPU oracle on the host cores

Workloads (synthetic, seeded; no dataset exists for this path):
  mixed     65,536 envs over Empty-5/8/16, DoorKey-16, FourRooms-19,
            LavaGap-7 x 2048 steps, seed 2, 128-step chunks (default: the
            largest single-GPU configuration)
  doorkey8  DoorKey-8x8, 4096 envs x 1000 steps, seed 1
  empty5    Empty-5x5, 64 envs x 1000 steps, seed 0
  rgb       Dynamic-Obstacles-16, 4 balls, 8192 envs x 512 steps, seed 3,
            RGB 224x224x3 + symbolic observations
The other configurations, the fused policy rollouts and the serving run are
reported under ``extras`` of the same line.
Multi-GPU: every rank runs the full workload on its own env-index range
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

MIXED = [(0, 5), (0, 8), (0, 16), (1, 16), (2, 19), (3, 7)]
WORKLOADS = {
    "empty5": dict(desc="Empty-5x5, 64 envs x 1000 steps, seed 0, uniform random actions over 7, symbolic obs",
                   parts=[(0, 5)], n=64, T=1000, seed=0, rgb=False, depth=1000),
    "doorkey8": dict(desc="DoorKey-8x8, 4096 envs x 1000 steps, seed 1, uniform random actions over 7, symbolic obs",
                     parts=[(1, 8)], n=4096, T=1000, seed=1, rgb=False, depth=1000),
    "mixed": dict(desc="65,536 envs in contiguous blocks of Empty-5x5/8x8/16x16, DoorKey-16x16, FourRooms-19x19, "
                       "LavaGap-7x7 x 2048 steps, seed 2, 128-step graph chunks, symbolic obs",
                  parts=MIXED, n=65536, T=2048, seed=2, rgb=False, depth=128),
    "rgb": dict(desc="Dynamic-Obstacles-16x16, 4 balls, 8192 envs x 512 steps, seed 3, 3 random actions, "
                     "RGB 224x224x3 + symbolic obs (8-slot output ring)",
                parts=[(4, 16)], n=8192, T=512, seed=3, rgb=True, depth=8),
    "doorkey8_full": dict(desc="DoorKey-8x8, 4096 envs x 1000 steps, seed 1, symbolic + fully observable views "
                               "(symbolic 8x8x3, categorical 8x8, categorical first person 7x7)",
                          parts=[(1, 8)], n=4096, T=1000, seed=1, rgb=False, depth=1000, full=True),
    # the fused policy + environment rollout (the paper's PPO rollout pattern:
    # many agents, each stepping its own envs with its own policy weights)
    "policy": dict(desc="Empty-8x8, 32,768 envs = 256 agents x 128 envs x 1000 steps, seed 5, actions from each "
                        "agent's integer MLP policy on the tensor cores (categorical first-person view -> 64 -> 64 "
                        "-> 7, seeded int8 weights), exploration 1/16, symbolic obs",
                   parts=[(0, 8)], n=32768, T=1000, seed=5, rgb=False, depth=128, policy=True, agents=256),
    "policy_paper": dict(desc="Empty-8x8, 32,768 envs = 2048 agents x 16 envs (the paper's PPO batch) x 1000 steps, "
                              "seed 5, actions from each agent's integer MLP policy on the tensor cores (8 weight sets "
                              "per 128-env block), exploration 1/16, symbolic obs",
                         parts=[(0, 8)], n=32768, T=1000, seed=5, rgb=False, depth=128, policy=True, agents=2048),
    # the paper's own batch-mode scale: 2^21 envs of Empty-8x8 unrolled for
    # 1000 steps (its reported wall time: almost always below 1 s on an A100)
    "paper_scale": dict(desc="Empty-8x8, 2,097,152 envs x 1000 steps, seed 6, uniform random actions over 7, "
                             "symbolic obs (1-slot output ring)",
                        parts=[(0, 8)], n=1 << 21, T=1000, seed=6, rgb=False, depth=1),
    # a reduced RGB case sized for ncu captures only (about 2.5 GB written per launch)
    "rgb_small": dict(desc="Dynamic-Obstacles-16x16, 4 balls, 1024 envs x 16 steps, seed 3, RGB + symbolic, 2-slot ring",
                      parts=[(4, 16)], n=1024, T=16, seed=3, rgb=True, depth=2, steps_per_launch=16),
}
OUT_BYTES_SYM = 147 + 4 + 2  # symbolic obs + reward + two flags per env-step
OUT_BYTES_RGB = 150528


def descs_of(w, n=None):
    n = n or w["n"]
    parts = w["parts"]
    base, extra = divmod(n, len(parts))
    out = []
    for j, p in enumerate(parts):
        out += [p] * (base + (1 if j < extra else 0))
    return out


def alg_bytes(w, descs, steps_per_launch):
    """Algorithmic HBM bytes of one rollout: every env-step writes its outputs
    once; every launch reads and writes each env's state once (three planes of
    S*S bytes plus a 32-byte agent block)."""
    T = w["T"]
    n = len(descs)
    side = max(s for _, s in descs)
    per_step = OUT_BYTES_SYM + (OUT_BYTES_RGB if w["rgb"] else 0) + (side * side * 4 + 49 if w.get("full") else 0)
    state = sum(3 * s * s + 32 for _, s in descs)
    launches = -(-T // steps_per_launch)
    return n * T * per_step + 2 * state * launches


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def measured_tensor_peak():
    """Dense bf16 TFLOP/s measured on the GB300s, sustained (the policy
    kernel runs inside long rollouts), else the fallback figure."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        if d.get("bf16_tflops_sustained"):
            return float(d["bf16_tflops_sustained"]), "measured"
    return 1700.0, "fallback"


# the files that define the step kernels (host-side files do not change a
# captured kernel)
KERNEL_SOURCES = ("nx_device.cuh", "nx_internal.h", "nx_kernels.cu", "nx_kernels_full.cu", "nx_lean_g1.cu", "nx_lean_g4.cu",
                  "nx_lean_g8.cu", "nx_lean_g16.cu", "nx_lean_g32.cu", "nx_lean_pol.cu", "nx_policy.cuh", "nx_step.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2407_19396_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_field(workload, key):
    """A machine-read field of the committed ncu summary of the step kernel on
    this workload, or None when the summary is missing or the kernel sources
    changed since it was captured."""
    p = os.path.join(ROOT, "profiles", f"step_kernel_{workload}.md")
    if not os.path.exists(p):
        return None
    vals = {}
    with open(p) as f:
        for line in f:
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                v = v.strip()
                vals[k.strip()] = v[1:].split("`", 1)[0] if v.startswith("`") else v  # the quoted value
    if vals.get("kernel_source_hash") != kernel_source_hash():
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def ncu_traffic(workload):
    """Per-launch DRAM bytes of the step kernel (ncu), or None.  The RGB
    workload's launches are too large to capture; its summary holds the
    reduced capture's bytes scaled to a full launch by env-steps."""
    return profile_field(workload, "dram_bytes_per_full_launch")


def oracle_sample(w):
    """The bounded sample of a workload the CPU oracle is timed on: the whole
    batch for the small configurations; for the larger ones the first (up to)
    1024 envs of every family block, with their own global env indices (so
    the sample is a subset of the workload, keyed identically), over the first
    (up to) 512 steps.  Returns (families, sizes, env indices, steps)."""
    descs = descs_of(w)
    if len(descs) * w["T"] <= 4096 * 1000:
        return [d[0] for d in descs], [d[1] for d in descs], list(range(len(descs))), w["T"]
    idx, start = [], 0
    for p in w["parts"]:
        cnt = sum(1 for d in descs if d == p)
        idx += list(range(start, start + min(cnt, 1024)))
        start += cnt
    return [descs[i][0] for i in idx], [descs[i][1] for i in idx], idx, min(w["T"], 512)


def sample_text(w):
    fam, _, idx, T = oracle_sample(w)
    if len(idx) == w["n"] and T == w["T"]:
        return f"{len(idx)} envs x {T} steps (the full workload)"
    return (f"{len(idx)} envs (the first {len(idx) // len(w['parts'])} of each of the {len(w['parts'])} family "
            f"blocks, their own env indices) x {T} steps")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if (args.impl != "reference" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def cpu_model():
    """The host CPU's model name as lscpu prints it (None when unavailable)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
    except (OSError, subprocess.SubprocessError):
        return None
    for line in out.splitlines():
        if line.strip().lower().startswith("model name:"):
            return line.split(":", 1)[1].strip()
    return None


def cpu_oracle_rate(w, min_s=10.0):
    """Env-steps/s of the oracle on this host (single thread) on the
    workload's bounded sample (oracle_sample), repeated until at least min_s
    of work."""
    import oracle as O

    fam, siz, idx, T = oracle_sample(w)
    done, t0 = 0, time.perf_counter()
    reps = 0
    while True:
        b = O.Batch(fam, siz, seed=w["seed"], env_indices=idx)
        b.reset(sym=True)
        b.rollout(T, sym=True)
        done += len(idx) * T
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_s:
            break
    return done / el, reps, el, len(idx), T


def _oracle_range(args):
    """One worker of the all-cores oracle timing: envs [lo, hi) of the
    workload's bounded sample, rolled out until at least min_s of work."""
    w_name, lo, hi, min_s = args
    import oracle as O

    w = WORKLOADS[w_name]
    fam, siz, idx, T = oracle_sample(w)
    done, t0 = 0, time.perf_counter()
    while True:
        b = O.Batch(fam[lo:hi], siz[lo:hi], seed=w["seed"], env_indices=idx[lo:hi])
        b.reset(sym=True)
        b.rollout(T, sym=True)
        done += (hi - lo) * T
        el = time.perf_counter() - t0
        if el >= min_s:
            return done, el


def cpu_oracle_rate_all_cores(w_name, min_s=4.0):
    """Env-steps/s of the oracle on every host core: one spawned process per
    core, each on a contiguous range of the workload's bounded sample (their
    rates add, since they run at the same time)."""
    import multiprocessing as mp

    w = WORKLOADS[w_name]
    n = len(oracle_sample(w)[2])
    P = max(1, min(os.cpu_count() or 1, n))
    cuts = [n * i // P for i in range(P + 1)]
    with mp.get_context("spawn").Pool(P) as pool:
        res = pool.map(_oracle_range, [(w_name, cuts[i], cuts[i + 1], min_s) for i in range(P)])
    return sum(d / el for d, el in res), P, sum(d for d, _ in res)


def run_reference(args, w, world, rank):
    """The CPU oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return 0
    import oracle as O

    fam, siz, idx, oracle_T = oracle_sample(w)
    times = []
    for k in range(args.warmup + args.steps):
        b = O.Batch(fam, siz, seed=w["seed"], env_indices=idx)
        t0 = time.perf_counter()
        b.reset(sym=True, rgb=False)
        b.rollout(oracle_T, sym=True)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    total = sum(times)
    units = len(idx) * oracle_T * len(times)
    v = units / total
    sample = f"{sample_text(w)} per bench step (symbolic obs), {len(times)} timed steps, one thread"
    line = {
        "impl": "reference", "metric": "env steps/sec", "value": v, "unit": "env-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": w["desc"], "n_envs_per_gpu": w["n"], "sample_envs": len(idx), "sample_steps": oracle_T,
                   "env_steps_per_bench_step": len(idx) * oracle_T},
        "cpu_baseline": {"value": v, "unit": "env-steps/s", "cores": 1, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "e2e": {"value": v, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def serving_requests(seed, n):
    """The serving mix: family uniform over the five families, size uniform in
    5..19, n_envs log-uniform in 1..4096, horizon uniform in 1..512."""
    import numpy as np

    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        fam = int(rng.integers(0, 5))
        size = int(rng.integers(5, 20))
        ne = int(min(4096, max(1, np.floor(np.exp(rng.uniform(0.0, np.log(4097.0)))))))
        hz = int(rng.integers(1, 513))
        out.append((fam, size, ne, hz, int(rng.integers(0, 2**63))))
    return out


def mix_static_rate(reqs, n_envs=262144, T=512, seed=4):
    """Env-steps/s of the serving mix's envs as one static batch through the
    context API (the first n_envs envs of the requests, autotuned, random
    actions, T-step rollouts): the persistent kernel's rate on this mix of
    families and sizes, without a server."""
    import torch

    from paper_2407_19396_gb300 import navixgb as nx

    descs = []
    for fam, size, ne, _, _ in reqs:
        descs += [(fam, size)] * ne
        if len(descs) >= n_envs:
            break
    descs = descs[:n_envs]
    env = nx.Env(descs=descs, seed=seed)
    env.reset()
    out = env.alloc_out(128)
    env.rollout(T, depth=128, out=out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        env.rollout(T, depth=128, out=out)
    torch.cuda.synchronize()
    rate = len(descs) * T * 3 / (time.perf_counter() - t0)
    env.close()
    return rate, len(descs)


def cpu_oracle_serving(reqs, min_s=5.0):
    """Env-steps/s of the oracle (one thread) serving the mix's requests one
    after another, each alone (its envs reset, then stepped for its
    horizon), until at least min_s of work: the serving mix's CPU baseline."""
    import oracle as O

    done, n_req, t0 = 0, 0, time.perf_counter()
    for fam, size, ne, hz, seed in reqs:
        b = O.Batch([fam] * ne, [size] * ne, seed)
        b.reset(sym=True)
        b.rollout(hz, sym=True)
        done += ne * hz
        n_req += 1
        if time.perf_counter() - t0 >= min_s:
            break
    el = time.perf_counter() - t0
    return {"value": done / el, "unit": "env-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"the mix's first {n_req} requests, each alone for its horizon ({done} env-steps, {el:.1f} s), "
                      "one thread"}


def run_serving(mixed_capacity=None, n_req=2000, budget=16 << 30, load=0.7, seed=4, chunk=64):
    """Poisson arrivals of the serving mix; returns latency percentiles and
    throughput.  The arrival rate is `load` x the measured capacity of the
    65,536-env mixed configuration (its env-steps/s, when given), and, as a
    second run, `load` x the server's own capacity, measured first by
    submitting all the mix's requests at once.  Beside them, the mix's own
    static-batch rate (mix_static_rate) bounds what any server reaches on it."""
    import numpy as np

    from paper_2407_19396_gb300 import navixgb as nx

    reqs = serving_requests(seed, n_req)
    mean_work = sum(r[2] * r[3] for r in reqs) / len(reqs)
    static_rate, static_envs = mix_static_rate(reqs)
    srv = nx.Server(budget_bytes=budget, steps_per_launch=chunk)
    t0 = time.perf_counter()
    # the requests' outputs are per-env returns, final views and ended
    # episodes; the optional digest of every per-step output (a verification
    # aid, checked by the serving tests) is not asked for
    ts = [srv.submit(*r, digest=False) for r in reqs]
    for t in ts:
        srv.wait(t, timeout_s=600.0)
    cap = sum(r[2] * r[3] for r in reqs) / (time.perf_counter() - t0)

    def one_run(rate_basis, arrival_seed):
        lam = load * rate_basis / mean_work  # requests per second
        rng = np.random.default_rng(arrival_seed)
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=n_req))
        tickets = []
        c0 = srv.stats()["chunks"]
        start = time.perf_counter()
        for r, a in zip(reqs, arrivals):
            while time.perf_counter() - start < a:
                pass
            tickets.append(srv.submit(*r, digest=False))
        res = [srv.wait(t, timeout_s=600.0) for t in tickets]
        lat = np.array([x["t_done"] - x["t_submit"] for x in res]) * 1000.0
        first = min(x["t_submit"] for x in res)
        last = max(x["t_done"] for x in res)
        work = sum(x["env_steps"] for x in res)
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "env_steps_per_s": work / (last - first),
                "arrival_rate_per_s": lam, "offered_env_steps_per_s": load * rate_basis,
                "chunks": srv.stats()["chunks"] - c0}

    out = {"requests": n_req, "offered_load": load, "budget_bytes": budget, "steps_per_launch": chunk,
           "server_capacity_env_steps_per_s": cap,
           "server_capacity_basis": f"all {n_req} requests of the mix submitted at once",
           "mix_static_env_steps_per_s": static_rate,
           "mix_static_basis": f"the mix's first {static_envs} envs as one autotuned static batch, 512-step rollouts",
           "mix": "family U{5}, size U{5..19}, n_envs log-U[1, 4096], horizon U{1..512}, seed 4",
           "outputs": "per-env returns, final views, ended episodes (no per-step digest)"}
    if mixed_capacity:
        out.update(one_run(mixed_capacity, seed + 1), rate_basis="0.7 x the measured env-steps/s of the "
                   "65,536-env mixed configuration", mixed_capacity_env_steps_per_s=mixed_capacity)
        out["at_server_capacity"] = one_run(cap, seed + 2)
    else:
        out.update(one_run(cap, seed + 1), rate_basis="0.7 x the server's burst capacity")
    out["peak_bytes"] = srv.stats()["peak_bytes"]
    srv.close()
    out["cpu_baseline"] = cpu_oracle_serving(reqs)
    return out


POLICY_FLOPS = 2 * (64 * 64 + 64 * 64 + 16 * 64)  # per env-step on the tensor cores (K and N padded)


def set_bench_policy(env, w):
    from paper_2407_19396_gb300 import inputs

    pw = inputs.policy_weights(w["seed"], w["agents"])
    env.set_policy(pw["w1"], pw["b1"], pw["w2"], pw["b2"], pw["w3"], pw["b3"], 3, 6, 1 << 28, w["n"] // w["agents"])


def time_rollouts(env, w, out, K, W, flush, per_family=False, policy=False):
    """W untimed rollouts, then K timed ones with CUDA events on the launching
    stream; L2 is flushed between timed rollouts, outside the event windows.
    Returns (per-step ms list, kernel ms, step launches, all launches)."""
    import torch

    T, depth = w["T"], w["depth"]
    for _ in range(W):
        env.rollout(T, depth=depth, out=out, per_family=per_family, policy=policy)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    l0 = env.launch_counts()
    env.profile_begin()
    for k in range(K):
        flush.fill_(k & 0xFF)
        evs[k][0].record(st)
        env.rollout(T, depth=depth, out=out, per_family=per_family, policy=policy)
        evs[k][1].record(st)
    torch.cuda.synchronize()
    kernel_ms, kl = env.profile_end()
    l1 = env.launch_counts()
    return [a.elapsed_time(b) for a, b in evs], kernel_ms, kl, l1[1] - l0[1]


def roofline_of(w, descs, kernel_ms, k_launches, rollouts, C, peak, peak_src, workload):
    """HBM roofline of the step kernel: algorithmic bytes per launch over the
    live average launch time (CUDA events on the launching stream), with the
    committed ncu capture's DRAM bytes per launch beside it."""
    per_rollout = alg_bytes(w, descs, C)
    achieved = per_rollout * rollouts / (kernel_ms / 1000.0) / 1e9
    launches = -(-w["T"] // C)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": ncu_traffic(workload), "peak_source": peak_src,
            "algorithmic_bytes_per_launch": per_rollout / launches,
            "kernel_ms_per_launch": kernel_ms / max(k_launches, 1), "kernel": "nx_step_kernel"}


def issue_rate(workload, rate_per_gpu, clk, sms):
    """Issue rate beside the HBM fraction: the symbolic configs are bound by
    their instruction chain; warp-instructions per env-step come from the
    committed ncu capture, the peak is one warp-instruction per cycle per
    scheduler (4 per SM) at the SM clock sampled during the timed region."""
    ipe = profile_field(workload, "warp_instructions_per_env_step")
    if ipe is None or not clk.get("sm_mhz"):
        return None
    peak_ips = sms * 4 * clk["sm_mhz"] * 1e6
    return {"warp_instructions_per_env_step": ipe, "achieved": rate_per_gpu * ipe, "peak": peak_ips,
            "unit": "warp-instructions/s", "frac": rate_per_gpu * ipe / peak_ips,
            "source": "ncu smsp__inst_executed.sum of the committed capture; peak = SMs x 4 x SM clock"}


def run_e2e(nx, inputs, torch, w, descs, atlas, rank, world, steps, dist):
    """End to end through the C ABI with host buffers: every bench step copies
    that step's host actions in and every env-step's outputs (symbolic view,
    reward, both flags) back into pinned host memory.  Outputs stream through
    a pinned ring of at most 4 GiB (step i in slot i % D, D a multiple of the
    128-step chunk), so the whole horizon is copied back."""
    n, T = w["n"], w["T"]
    C = 128
    D = max(C, min(T, (4 << 30) // (n * (OUT_BYTES_SYM + 1)) // C * C))
    acts = torch.from_numpy(inputs.random_actions(w["seed"], (T, n), n_actions=3 if w["parts"][0][0] == 4 else 7))
    acts = acts.pin_memory()
    hout = {"obs_sym": torch.empty((D, n, 7, 7, 3), dtype=torch.uint8).pin_memory(),
            "reward": torch.empty((D, n), dtype=torch.float32).pin_memory(),
            "terminated": torch.empty((D, n), dtype=torch.uint8).pin_memory(),
            "truncated": torch.empty((D, n), dtype=torch.uint8).pin_memory(),
            # (the 150 KB images of an RGB workload are not brought to the host here)
            "obs_rgb": None}
    e = nx.Env(descs=descs, seed=w["seed"], obs_rgb=w["rgb"], atlas=atlas, env_index_base=rank * n)
    e.reset()
    ks = max(1, min(steps, 5))
    for _ in range(2):
        e.rollout_host(T, actions=acts.numpy(), out=hout)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    laps = []
    for _ in range(ks):
        e.rollout_host(T, actions=acts.numpy(), out=hout)
        laps.append(time.perf_counter())
    el = time.perf_counter() - t0
    laps = [1000.0 * (b - a) for a, b in zip([t0] + laps[:-1], laps)]
    if dist:
        t = torch.tensor([el], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el = float(t.item())
    e.close()
    value = world * n * T * ks / el
    link = host_link_d2h_gbs(torch)
    # the leg's ceiling: every env-step brings OUT_BYTES_SYM bytes back over
    # its GPU's host link (its 1-byte action goes the other way, concurrently)
    bound = link * 1e9 / OUT_BYTES_SYM
    return {"value": value, "unit": "env-steps/s", "h2d_bytes_per_step": T * n,
            "d2h_bytes_per_step": T * n * OUT_BYTES_SYM, "steps": ks, "horizon": T, "host_ring_steps": D,
            "rollout_ms": [round(v, 2) for v in laps],
            "host_link": {"d2h_gbs": round(link, 1), "bound_env_steps_per_s": bound * world,
                          "frac": value / (bound * world),
                          "measured": "best of 3 copies of 1 GiB from device to pinned host memory"},
            "actions": "host int8, seeded numpy draws", "call": "nx_rollout_host"}


def host_link_d2h_gbs(torch, nbytes=1 << 30, reps=3):
    """Device-to-host copy rate into pinned memory (GB/s), best of reps."""
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    d.fill_(1)
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    best = 0.0
    for _ in range(reps + 1):
        torch.cuda.synchronize()
        t = time.perf_counter()
        h.copy_(d, non_blocking=True)
        torch.cuda.synchronize()
        best = max(best, nbytes / (time.perf_counter() - t) / 1e9)
    del d, h
    return best


def run_extra(nx, inputs, name, flush, peak, peak_src, reps=5):
    """One other configuration: reps timed rollouts after one warm-up, with
    its own HBM roofline block."""
    wx = WORKLOADS[name]
    dx = descs_of(wx)
    fv = bool(wx.get("full"))
    ex = nx.Env(descs=dx, seed=wx["seed"], obs_rgb=wx["rgb"], atlas=inputs.atlas() if wx["rgb"] else None,
                obs_full=fv, obs_cat=fv, obs_cat_fp=fv)
    ex.reset()
    ox = ex.alloc_out(wx["depth"])
    ms, kms, kl, _ = time_rollouts(ex, wx, ox, reps, 1, flush)
    cx = ex.info()["steps_per_launch"]
    rec = {"workload": wx["desc"], "env_steps_per_s": len(dx) * wx["T"] * len(ms) / (sum(ms) / 1000),
           "ms_per_rollout": sum(ms) / len(ms), "timed_rollouts": len(ms),
           "roofline": roofline_of(wx, dx, kms, kl, len(ms), cx, peak, peak_src, name),
           "launch_shape": {k: ex.info()[k] for k in ("group_lanes", "envs_per_cta", "grid_ctas")}}
    ex.close()
    del ox
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="navixgb", choices=["navixgb", "reference"])
    ap.add_argument("--workload", default="mixed", choices=sorted(WORKLOADS))
    ap.add_argument("--no-extras", action="store_true", help="skip the other configs and the CPU baseline")
    ap.add_argument("--ncu-case", action="store_true", help="one rollout of the workload for an ncu capture")
    ap.add_argument("--shape", default="", help="force the launch shape as LANES,ENVS_PER_CTA[,STAGING[,GRID_SIDE]] "
                                               "(no autotuning)")
    args = ap.parse_args()
    if args.warmup < 3 and not args.ncu_case:
        args.warmup = 3
    w = WORKLOADS[args.workload]
    world, rank, local, dist = dist_setup(args)
    if args.impl == "reference":
        rc = run_reference(args, w, world, rank)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return rc

    import torch

    from paper_2407_19396_gb300 import build as nxbuild
    from paper_2407_19396_gb300 import inputs
    from paper_2407_19396_gb300 import navixgb as nx

    nxbuild.build()
    torch.cuda.set_device(local)
    n = w["n"]
    descs = descs_of(w)
    atlas = inputs.atlas() if w["rgb"] else None
    shape = {}
    if args.shape:
        vals = [int(v) for v in args.shape.split(",")]
        shape = dict(group_lanes=vals[0], envs_per_cta=vals[1], staging=vals[2] if len(vals) > 2 else 1,
                     autotune=False, grid_side=vals[3] if len(vals) > 3 else 0)
    if "steps_per_launch" in w:
        shape["steps_per_launch"] = w["steps_per_launch"]
    fv = bool(w.get("full"))
    env = nx.Env(descs=descs, seed=w["seed"], obs_rgb=w["rgb"], atlas=atlas, env_index_base=rank * n,
                 obs_full=fv, obs_cat=fv, obs_cat_fp=fv, **shape)
    env.reset()
    out = env.alloc_out(w["depth"])
    if args.ncu_case:
        if w.get("policy"):
            set_bench_policy(env, w)
        env.rollout(w["T"], depth=w["depth"], out=out, policy=bool(w.get("policy")))
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": args.workload, "info": env.info()}), flush=True)
        return 0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # 256 MiB > 129 MB L2

    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall0 = time.perf_counter()
    step_ms, kernel_ms, k_launches, all_launches = time_rollouts(env, w, out, args.steps, args.warmup, flush)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    units = world * n * w["T"] * args.steps
    value = units / (total_ms / 1000.0)

    peak, peak_src = measured_peaks()
    C = env.info()["steps_per_launch"]
    roofline = roofline_of(w, descs, kernel_ms, k_launches, args.steps, C, peak, peak_src, args.workload)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roofline["issue"] = issue_rate(args.workload, value / world, clk, sms)

    # the plain comparison form on the same envs: one single-step launch per
    # family per step (spec: the persistent graph-captured form must beat it)
    comparator = None
    if len(w["parts"]) > 1:
        ms_pf, _, _, _ = time_rollouts(env, w, out, 2, 1, flush, per_family=True)
        pf = world * n * w["T"] * len(ms_pf) / (sum(ms_pf) / 1000)
        comparator = {"per_family_env_steps_per_s": pf, "persistent_over_per_family": value / pf,
                      "form": "nx_rollout_per_family: one single-step launch per family per step, no graph",
                      "timed_rollouts": len(ms_pf)}

    e2e = run_e2e(nx, inputs, torch, w, descs, atlas, rank, world, args.steps, dist)

    line = {
        "metric": "env steps/sec", "value": value, "unit": "env-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": w["desc"], "n_envs_per_gpu": n, "env_steps_per_bench_step": n * w["T"] * world,
                   "steps_per_launch": C,
                   "launch_shape": {k: env.info()[k] for k in ("group_lanes", "envs_per_cta", "grid_ctas", "grid_side")},
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{world}"},
        "roofline": roofline, "e2e": e2e, "gpu_launches": all_launches, "clocks": clk,
        "wall_s": wall,
    }
    if comparator:
        line["comparator"] = comparator
    env.close()
    del out

    if rank == 0 and world == 1 and not args.no_extras:
        extras = {}
        for name in ("doorkey8", "rgb", "empty5", "doorkey8_full", "mixed"):
            if name != args.workload:
                extras[name] = run_extra(nx, inputs, name, flush, peak, peak_src)
        # the paper's batch-mode scale: wall time of one 1000-step rollout of 2^21 envs
        wx = WORKLOADS["paper_scale"]
        dx = descs_of(wx)
        ex = nx.Env(descs=dx, seed=wx["seed"])
        ex.reset()
        ox = ex.alloc_out(wx["depth"])
        ms, kms, kl, _ = time_rollouts(ex, wx, ox, 2, 1, flush)
        bx = alg_bytes(wx, dx, ex.info()["steps_per_launch"])
        extras["paper_scale"] = {"env_steps_per_s": len(dx) * wx["T"] * len(ms) / (sum(ms) / 1000),
                                 "rollout_ms": min(ms), "hbm_frac": bx * len(ms) / (kms / 1000) / 1e9 / peak,
                                 "launch_shape": {k: ex.info()[k] for k in ("group_lanes", "envs_per_cta", "grid_ctas")},
                                 "workload": wx["desc"]}
        ex.close()
        del ox
        # the fused policy rollouts (256 agents x 128 envs, and the paper's
        # 2048 agents x 16 envs), beside the random-action rollout of the same envs
        for key in ("policy", "policy_paper"):
            wx = WORKLOADS[key]
            dx = descs_of(wx)
            ex = nx.Env(descs=dx, seed=wx["seed"])
            ex.reset()
            set_bench_policy(ex, wx)
            ox = ex.alloc_out(wx["depth"])
            ms, kms, kl, _ = time_rollouts(ex, wx, ox, 2, 1, flush, policy=True)
            ms_r, _, _, _ = time_rollouts(ex, wx, ox, 2, 1, flush)
            rate = len(dx) * wx["T"] * len(ms) / (sum(ms) / 1000)
            kern_rate = len(dx) * wx["T"] * len(ms) / (kms / 1000)
            tf = kern_rate * POLICY_FLOPS / 1e12
            tpeak, tsrc = measured_tensor_peak()
            extras[key] = {"env_steps_per_s": rate, "random_action_env_steps_per_s":
                           len(dx) * wx["T"] * len(ms_r) / (sum(ms_r) / 1000),
                           "tensor_tflops": tf, "tensor_frac": tf / tpeak, "tensor_peak": tpeak,
                           "tensor_peak_source": tsrc, "tensor_flops_per_env_step": POLICY_FLOPS,
                           "envs_per_agent": len(dx) // wx["agents"],
                           # each weight set's MMA spans its block's 128 rows
                           "tensor_flops_issued_per_env_step": POLICY_FLOPS * max(1, 128 // (len(dx) // wx["agents"])),
                           "workload": wx["desc"]}
            ex.close()
            del ox
        line["extras"] = extras
    if rank == 0 and world == 1 and not args.no_extras:
        cap = value if args.workload == "mixed" else line.get("extras", {}).get("mixed", {}).get("env_steps_per_s")
        line.setdefault("extras", {})["serving"] = run_serving(mixed_capacity=cap)
    if rank == 0 and world == 1 and not args.no_extras:
        rate, reps, el, ne, nt = cpu_oracle_rate(w)
        line["cpu_baseline"] = {"value": rate, "unit": "env-steps/s", "cores": 1, "kind": "oracle",
                                "sample": f"{sample_text(w)} x {reps}, {el:.1f} s, one thread", "cpu_model": cpu_model()}
        arate, P, asteps = cpu_oracle_rate_all_cores(args.workload)
        line["cpu_baseline"]["all_cores"] = {
            "value": arate, "unit": "env-steps/s", "cores": P, "kind": "oracle",
            "sample": f"the same sample's envs in {P} contiguous ranges, one spawned process each, "
                      f"{asteps} env-steps in about 4 s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
