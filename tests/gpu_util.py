"""Shared helpers of the GPU parity tests: run the CUDA path through the
C-ABI binding and the oracle on the same seeded inputs, compare bytes."""
from __future__ import annotations

import numpy as np

import oracle as O

STATE_KEYS = ("x", "y", "dir", "carry_ent", "carry_col", "done", "t", "episode", "ent", "col", "st", "ball_x",
              "ball_y", "invalid", "max_steps", "height")


def to_np(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t
    return t.detach().cpu().numpy()


def first_mismatch(a, b):
    diff = np.argwhere(a != b)
    return tuple(int(v) for v in diff[0]) if len(diff) else None


def assert_outputs_equal(gpu: dict, orc: dict, keys=("obs_sym", "reward", "terminated", "truncated"), what=""):
    for k in keys:
        g, o = to_np(gpu[k]), orc[k]
        assert g.shape == o.shape, f"{what} {k}: shape {g.shape} vs {o.shape}"
        if not np.array_equal(g, o):
            idx = first_mismatch(g, o)
            raise AssertionError(f"{what} {k} differs first at index {idx}: gpu {g[idx[:2]] if g.ndim > 2 else g[idx]} "
                                 f"oracle {o[idx[:2]] if o.ndim > 2 else o[idx]}")


def assert_states_equal(gpu_envs: list, orc_batch: O.Batch, indices=None, what=""):
    idx = range(len(gpu_envs)) if indices is None else indices
    for j, i in enumerate(idx):
        g = gpu_envs[i]
        o = orc_batch.state(j)
        for k in STATE_KEYS:
            if g[k] != o[k]:
                raise AssertionError(f"{what} env {i} state field {k}: gpu {g[k]!r} oracle {o[k]!r}")


def oracle_batch_for(descs, seed, indices=None, **kw):
    fam = [d[0] for d in descs]
    siz = [d[1] for d in descs]
    ms = [(d[2] if len(d) > 2 and d[2] else O.default_max_steps(d[0], d[1])) for d in descs]
    if indices is not None:
        fam = [fam[i] for i in indices]
        siz = [siz[i] for i in indices]
        ms = [ms[i] for i in indices]
    return O.Batch(fam, siz, seed, max_steps=ms, env_indices=indices, **kw)


def mixed_descs(n_total, parts):
    """Contiguous blocks of (family, size) splitting n_total as evenly as possible (first blocks larger)."""
    k = len(parts)
    base, extra = divmod(n_total, k)
    out = []
    for j, p in enumerate(parts):
        out += [p] * (base + (1 if j < extra else 0))
    return out
