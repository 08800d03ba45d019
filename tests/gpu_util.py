"""Shared helpers of the GPU parity tests: run the CUDA path through the
C-ABI binding and the oracle on the same seeded inputs, compare bytes."""
from __future__ import annotations

import numpy as np

import oracle as O

STATE_KEYS = ("x", "y", "dir", "carry_ent", "carry_col", "done", "t", "episode", "ent", "col", "st", "ball_x",
              "ball_y", "invalid", "max_steps", "height", "family", "mission")


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
    """descs: (family, size[, max_steps[, variant]]) per env, as given to navixgb.Env."""
    fam = [d[0] for d in descs]
    siz = [d[1] for d in descs]
    ms = [(d[2] if len(d) > 2 and d[2] else O.default_max_steps(d[0], d[1])) for d in descs]
    var = [(d[3] if len(d) > 3 else 0) for d in descs]
    if indices is not None:
        fam = [fam[i] for i in indices]
        siz = [siz[i] for i in indices]
        ms = [ms[i] for i in indices]
        var = [var[i] for i in indices]
    return O.Batch(fam, siz, seed, max_steps=ms, env_indices=indices, variants=var, **kw)


def mixed_descs(n_total, parts):
    """Contiguous blocks of (family, size) splitting n_total as evenly as possible (first blocks larger)."""
    k = len(parts)
    base, extra = divmod(n_total, k)
    out = []
    for j, p in enumerate(parts):
        out += [p] * (base + (1 if j < extra else 0))
    return out


def _fold(h, w):
    return (h ^ w.astype(np.uint64)) * np.uint64(0x100000001B3)


def record_words(obs, reward, term, trunc):
    """Per env, the 51 digest words of one step record: the 49 view cells
    (ent | col << 8 | st << 16), the reward's float32 bits, term | trunc << 8."""
    n = obs.shape[0]
    c = obs.reshape(n, 49, 3).astype(np.uint32)
    cells = c[:, :, 0] | (c[:, :, 1] << 8) | (c[:, :, 2] << 16)
    rbits = np.ascontiguousarray(reward, np.float32).view(np.uint32)
    flags = term.astype(np.uint32) | (trunc.astype(np.uint32) << 8)
    return np.concatenate([cells, rbits[:, None], flags[:, None]], axis=1)


def oracle_request(family, size, n_envs, horizon, seed, variant=0, **kw):
    """What a serving request must return, computed by the oracle: per-env
    returns (float32, summed in step order), the final view, the number of
    ended episodes and the digest of the reset record plus every step record."""
    b = O.Batch([family] * n_envs, [size] * n_envs, seed, variants=[variant] * n_envs, **kw)
    r0 = b.reset()
    h = np.zeros(n_envs, np.uint64)
    with np.errstate(over="ignore"):
        for w in record_words(r0["obs_sym"], r0["reward"], r0["terminated"], r0["truncated"]).T:
            h = _fold(h, w)
        ret = np.zeros(n_envs, np.float32)
        eps = 0
        last = r0["obs_sym"]
        for t in range(horizon):
            o = b.step()
            for w in record_words(o["obs_sym"], o["reward"], o["terminated"], o["truncated"]).T:
                h = _fold(h, w)
            ret = (ret + o["reward"]).astype(np.float32)
            eps += int((o["terminated"] | o["truncated"]).sum())
            last = o["obs_sym"]
        d = np.zeros(1, np.uint64)
        for i in range(n_envs):
            d = _fold(d, np.array([int(h[i]) & 0xFFFFFFFF], np.uint64))
            d = _fold(d, np.array([int(h[i]) >> 32], np.uint64))
    return {"returns": ret, "final_obs": last, "episodes": eps, "digest": int(d[0])}
