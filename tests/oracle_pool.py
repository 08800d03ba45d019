"""Oracle rollouts of contiguous env ranges in spawned worker processes, for
the full-population parity tests (test infrastructure: imports the oracle).

Workers are started with the ``spawn`` method, never forked from a process
that has already used the GPU."""
from __future__ import annotations

import multiprocessing as mp
import os

KEYS = ("obs_sym", "reward", "terminated", "truncated")


def _chunk_ends(args):
    """Envs [lo, hi) of a batch of contiguous family blocks: the reset
    outputs, the outputs of the last step of every C-step chunk, and the
    final state of every env."""
    lo, hi, n_total, parts, seed, T, C = args
    from tests.gpu_util import mixed_descs, oracle_batch_for

    descs = mixed_descs(n_total, parts)
    ob = oracle_batch_for(descs, seed, indices=list(range(lo, hi)))
    r0 = ob.reset()
    ends = []
    for _ in range(T // C):
        o = ob.rollout(C)
        ends.append({k: o[k][-1].copy() for k in KEYS})
    return lo, {k: r0[k] for k in KEYS}, ends, [ob.state(j) for j in range(hi - lo)]


def chunk_ends(n_total, parts, seed, T, C, workers=None):
    """The same over every env of the batch, split into contiguous ranges,
    one per worker; results concatenated in env order."""
    import numpy as np

    P = max(1, min(workers or (os.cpu_count() or 1), 32, n_total))
    cuts = [n_total * i // P for i in range(P + 1)]
    with mp.get_context("spawn").Pool(P) as pool:
        res = sorted(pool.map(_chunk_ends, [(cuts[i], cuts[i + 1], n_total, parts, seed, T, C) for i in range(P)]),
                     key=lambda r: r[0])
    reset = {k: np.concatenate([r[1][k] for r in res]) for k in KEYS}
    ends = [{k: np.concatenate([r[2][j][k] for r in res]) for k in KEYS} for j in range(T // C)]
    states = [s for r in res for s in r[3]]
    return reset, ends, states
