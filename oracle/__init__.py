"""ctypes wrapper of the plain-C oracle (navix_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this module to compute expected values;
the product package never imports it.  The oracle shares no code with the CUDA
library: it has its own Philox, layouts, rules, view and visibility, all in
``navix_oracle.c``.

``NAVIX_ORACLE_SO`` names another build of the same source to load instead;
the mutation tests use it to check that the pins catch deliberately planted
mistakes in a copy of the oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "navix_oracle.c")]
_lock = threading.Lock()
_lib = None

OBS_BYTES = 7 * 7 * 3
RGB_BYTES = 224 * 224 * 3
TILE_BYTES = 32 * 32 * 3
MAX_CELLS = 19 * 19

(EMPTY, DOORKEY, FOURROOMS, LAVAGAP, DYNOBS, EMPTY_RANDOM, LAVA_CROSSING, SIMPLE_CROSSING, GOTODOOR, DISTSHIFT,
 KEYCORRIDOR) = range(11)
NO_MISSION = 255
FAMILY_NAMES = {"empty": EMPTY, "doorkey": DOORKEY, "fourrooms": FOURROOMS, "lavagap": LAVAGAP, "dynobs": DYNOBS,
                "empty_random": EMPTY_RANDOM, "lava_crossing": LAVA_CROSSING, "simple_crossing": SIMPLE_CROSSING,
                "gotodoor": GOTODOOR, "distshift": DISTSHIFT, "keycorridor": KEYCORRIDOR}


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain C11, -O2 -ffp-contract=off, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC + [os.path.join(_HERE, "navix_oracle.h")])
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-Wall", "-Wextra", "-o", tmp] + _SRC
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class OrcEnv(ctypes.Structure):
    _fields_ = [
        ("family", ctypes.c_int32), ("height", ctypes.c_int32), ("width", ctypes.c_int32),
        ("max_steps", ctypes.c_int32), ("n_balls", ctypes.c_int32), ("reward_mode", ctypes.c_int32),
        ("variant", ctypes.c_int32), ("lava_reward", ctypes.c_float), ("action_cost", ctypes.c_float),
        ("time_cost", ctypes.c_float),
        ("seed", ctypes.c_uint64), ("env_index", ctypes.c_uint32), ("episode", ctypes.c_uint32),
        ("t", ctypes.c_int32), ("ax", ctypes.c_int32), ("ay", ctypes.c_int32), ("dir", ctypes.c_int32),
        ("carry_ent", ctypes.c_int32), ("carry_col", ctypes.c_int32), ("done", ctypes.c_int32),
        ("mission", ctypes.c_int32), ("invalid_action", ctypes.c_int32),
        ("ball_x", ctypes.c_int32 * 4), ("ball_y", ctypes.c_int32 * 4),
        ("ent", ctypes.c_uint8 * MAX_CELLS), ("col", ctypes.c_uint8 * MAX_CELLS), ("st", ctypes.c_uint8 * MAX_CELLS),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(os.environ.get("NAVIX_ORACLE_SO") or build())
            P = ctypes.POINTER
            u8p, i8p, f32p, i32p = P(ctypes.c_uint8), P(ctypes.c_int8), P(ctypes.c_float), P(ctypes.c_int32)
            L.orc_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
            L.orc_bounded.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            L.orc_bounded.restype = ctypes.c_uint32
            L.orc_draw.argtypes = [ctypes.c_uint64] + [ctypes.c_uint32] * 5
            L.orc_draw.restype = ctypes.c_uint32
            L.orc_default_max_steps.argtypes = [ctypes.c_int32, ctypes.c_int32]
            L.orc_default_max_steps.restype = ctypes.c_int32
            L.orc_env_init.argtypes = [P(OrcEnv), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_float,
                                       ctypes.c_int32]
            L.orc_max_variant.argtypes = [ctypes.c_int32, ctypes.c_int32]
            L.orc_max_variant.restype = ctypes.c_int32
            L.orc_env_init.restype = ctypes.c_int32
            L.orc_reset.argtypes = [P(OrcEnv), ctypes.c_uint32]
            L.orc_random_action.argtypes = [P(OrcEnv), ctypes.c_uint32]
            L.orc_random_action.restype = ctypes.c_int32
            L.orc_step.argtypes = [P(OrcEnv), ctypes.c_int32, f32p, u8p, u8p]
            L.orc_obs_sym.argtypes = [P(OrcEnv), u8p]
            L.orc_obs_rgb.argtypes = [P(OrcEnv), u8p, u8p]
            L.orc_tile_index.argtypes = [ctypes.c_int32] * 5
            L.orc_tile_index.restype = ctypes.c_int32
            L.orc_set_cell.argtypes = [P(OrcEnv)] + [ctypes.c_int32] * 5
            L.orc_set_agent.argtypes = [P(OrcEnv)] + [ctypes.c_int32] * 5
            L.orc_batch_create.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, ctypes.c_int32, ctypes.c_uint64,
                                           ctypes.c_uint32, ctypes.c_int32, ctypes.c_float]
            L.orc_batch_create.restype = ctypes.c_void_p
            L.orc_batch_create_indexed.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, ctypes.c_int32,
                                                   ctypes.c_uint64, P(ctypes.c_uint32), ctypes.c_int32, ctypes.c_float]
            L.orc_batch_create_indexed.restype = ctypes.c_void_p
            L.orc_batch_destroy.argtypes = [ctypes.c_void_p]
            L.orc_policy_greedy.argtypes = [P(OrcPolicy), ctypes.c_int32, u8p, ctypes.c_int32]
            L.orc_policy_greedy.restype = ctypes.c_int32
            L.orc_policy_action.argtypes = [P(OrcPolicy), P(OrcEnv), ctypes.c_uint32]
            L.orc_policy_action.restype = ctypes.c_int32
            L.orc_batch_rollout_policy.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(OrcPolicy), i8p, u8p, f32p, u8p,
                                                   u8p]
            L.orc_set_costs.argtypes = [P(OrcEnv), ctypes.c_float, ctypes.c_float]
            L.orc_batch_set_costs.argtypes = [ctypes.c_void_p, ctypes.c_float, ctypes.c_float]
            L.orc_batch_env.argtypes = [ctypes.c_void_p, ctypes.c_int32]
            L.orc_batch_env.restype = P(OrcEnv)
            L.orc_batch_reset.argtypes = [ctypes.c_void_p, u8p, u8p, u8p, f32p, u8p, u8p]
            L.orc_batch_step.argtypes = [ctypes.c_void_p, i8p, u8p, u8p, u8p, f32p, u8p, u8p]
            L.orc_batch_rollout.argtypes = [ctypes.c_void_p, ctypes.c_int32, i8p, u8p, u8p, u8p, f32p, u8p, u8p]
            L.orc_obs_full.argtypes = [P(OrcEnv), u8p, ctypes.c_int32]
            L.orc_obs_cat.argtypes = [P(OrcEnv), u8p, ctypes.c_int32]
            L.orc_obs_cat_fp.argtypes = [P(OrcEnv), u8p]
            L.orc_batch_obs_full.argtypes = [ctypes.c_void_p, u8p, u8p, u8p, ctypes.c_int32]
            L.orc_obs_rgb_full.argtypes = [P(OrcEnv), u8p, u8p, ctypes.c_int32]
            L.orc_batch_obs_rgb_full.argtypes = [ctypes.c_void_p, u8p, u8p, ctypes.c_int32]
            L.orc_batch_gstep.argtypes = [ctypes.c_void_p]
            L.orc_batch_gstep.restype = ctypes.c_uint32
            _lib = L
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def bounded(x, n):
    return int(lib().orc_bounded(x, n))


def draw(seed, env_index, episode, step, purpose, d):
    return int(lib().orc_draw(seed, env_index, episode, step, purpose, d))


def default_max_steps(family, size):
    return int(lib().orc_default_max_steps(family, size))


def max_variant(family, size):
    return int(lib().orc_max_variant(family, size))


def tile_index(visible, agent_cell, ent, col, st):
    return int(lib().orc_tile_index(visible, agent_cell, ent, col, st))


class OrcPolicy(ctypes.Structure):
    _fields_ = [("n_agents", ctypes.c_int32), ("envs_per_agent", ctypes.c_int32),
                ("w1", ctypes.POINTER(ctypes.c_int8)), ("b1", ctypes.POINTER(ctypes.c_int32)),
                ("w2", ctypes.POINTER(ctypes.c_int8)), ("b2", ctypes.POINTER(ctypes.c_int32)),
                ("w3", ctypes.POINTER(ctypes.c_int8)), ("b3", ctypes.POINTER(ctypes.c_int32)),
                ("shift1", ctypes.c_int32), ("shift2", ctypes.c_int32), ("epsilon", ctypes.c_uint32)]


class Policy:
    """The fused rollout's integer MLP policy (numpy arrays kept alive here).

    w1 [A, 64, 49] int8, b1 [A, 64] int32, w2 [A, 64, 64] int8, b2 [A, 64]
    int32, w3 [A, 7, 64] int8, b3 [A, 7] int32."""

    def __init__(self, w1, b1, w2, b2, w3, b3, shift1, shift2, epsilon=0, envs_per_agent=128):
        self.w1 = np.ascontiguousarray(w1, np.int8)
        self.b1 = np.ascontiguousarray(b1, np.int32)
        self.w2 = np.ascontiguousarray(w2, np.int8)
        self.b2 = np.ascontiguousarray(b2, np.int32)
        self.w3 = np.ascontiguousarray(w3, np.int8)
        self.b3 = np.ascontiguousarray(b3, np.int32)
        A = self.w1.shape[0]
        assert self.w1.shape == (A, 64, 49) and self.w2.shape == (A, 64, 64) and self.w3.shape == (A, 7, 64)
        assert self.b1.shape == (A, 64) and self.b2.shape == (A, 64) and self.b3.shape == (A, 7)
        self.shift1, self.shift2, self.epsilon, self.envs_per_agent = int(shift1), int(shift2), int(epsilon), int(envs_per_agent)
        self.s = OrcPolicy(A, self.envs_per_agent, _ptr(self.w1, ctypes.c_int8), _ptr(self.b1, ctypes.c_int32),
                           _ptr(self.w2, ctypes.c_int8), _ptr(self.b2, ctypes.c_int32),
                           _ptr(self.w3, ctypes.c_int8), _ptr(self.b3, ctypes.c_int32),
                           self.shift1, self.shift2, self.epsilon)

    @property
    def n_agents(self):
        return self.w1.shape[0]

    def greedy(self, agent, cat_fp, n_act=7):
        c = np.ascontiguousarray(cat_fp, np.uint8).reshape(-1)
        return int(lib().orc_policy_greedy(ctypes.byref(self.s), agent, _ptr(c, ctypes.c_uint8), n_act))

    def action(self, env, gstep):
        return int(lib().orc_policy_action(ctypes.byref(self.s), ctypes.byref(env.s), gstep))


class Env:
    """One oracle environment (for hand-built states and worked examples)."""

    def __init__(self, family, size, seed=0, env_index=0, max_steps=0, n_balls=4, reward_mode=0, lava_reward=0.0,
                 variant=0, action_cost=0.0, time_cost=0.0):
        self.s = OrcEnv()
        rc = lib().orc_env_init(ctypes.byref(self.s), family, size, max_steps, n_balls, seed, env_index,
                                reward_mode, lava_reward, variant)
        if rc != 0:
            raise ValueError("invalid oracle env arguments")
        lib().orc_set_costs(ctypes.byref(self.s), action_cost, time_cost)

    def reset(self, episode=0):
        lib().orc_reset(ctypes.byref(self.s), episode)

    def step(self, action):
        r = ctypes.c_float()
        te = ctypes.c_uint8()
        tr = ctypes.c_uint8()
        lib().orc_step(ctypes.byref(self.s), int(action), ctypes.byref(r), ctypes.byref(te), ctypes.byref(tr))
        return float(r.value), int(te.value), int(tr.value)

    def random_action(self, gstep):
        return int(lib().orc_random_action(ctypes.byref(self.s), gstep))

    def obs(self):
        o = np.zeros(OBS_BYTES, np.uint8)
        lib().orc_obs_sym(ctypes.byref(self.s), _ptr(o, ctypes.c_uint8))
        return o.reshape(7, 7, 3)

    def rgb(self, atlas):
        img = np.zeros(RGB_BYTES, np.uint8)
        lib().orc_obs_rgb(ctypes.byref(self.s), _ptr(np.ascontiguousarray(atlas, np.uint8).reshape(-1), ctypes.c_uint8),
                          _ptr(img, ctypes.c_uint8))
        return img.reshape(224, 224, 3)

    def full(self, side=None):
        side = side or self.s.width
        o = np.zeros(side * side * 3, np.uint8)
        lib().orc_obs_full(ctypes.byref(self.s), _ptr(o, ctypes.c_uint8), side)
        return o.reshape(side, side, 3)

    def cat(self, side=None):
        side = side or self.s.width
        o = np.zeros(side * side, np.uint8)
        lib().orc_obs_cat(ctypes.byref(self.s), _ptr(o, ctypes.c_uint8), side)
        return o.reshape(side, side)

    def cat_fp(self):
        o = np.zeros(49, np.uint8)
        lib().orc_obs_cat_fp(ctypes.byref(self.s), _ptr(o, ctypes.c_uint8))
        return o.reshape(7, 7)

    def set_cell(self, x, y, ent, col, st):
        lib().orc_set_cell(ctypes.byref(self.s), x, y, ent, col, st)

    def set_agent(self, x, y, d, carry_ent=0, carry_col=0):
        lib().orc_set_agent(ctypes.byref(self.s), x, y, d, carry_ent, carry_col)

    def grid(self):
        """(ent, col, st) as [H, W] uint8 arrays."""
        H, W = self.s.height, self.s.width
        n = H * W
        e = np.frombuffer(bytes(self.s.ent), np.uint8)[:n].reshape(H, W).copy()
        c = np.frombuffer(bytes(self.s.col), np.uint8)[:n].reshape(H, W).copy()
        s = np.frombuffer(bytes(self.s.st), np.uint8)[:n].reshape(H, W).copy()
        return e, c, s


def env_state(s: OrcEnv) -> dict:
    """Canonical per-env state as a plain dict (the comparison format of the tests)."""
    H, W = s.height, s.width
    n = H * W
    return {
        "family": s.family, "height": H, "width": W, "max_steps": s.max_steps,
        "x": s.ax, "y": s.ay, "dir": s.dir, "carry_ent": s.carry_ent, "carry_col": s.carry_col,
        "done": s.done, "t": s.t, "episode": s.episode, "n_balls": s.n_balls, "variant": s.variant,
        "mission": s.mission,
        "ball_x": list(s.ball_x)[: s.n_balls], "ball_y": list(s.ball_y)[: s.n_balls],
        "invalid": s.invalid_action,
        "ent": bytes(s.ent)[:n], "col": bytes(s.col)[:n], "st": bytes(s.st)[:n],
    }


class Batch:
    """n oracle environments with global indices base..base+n-1 (Code 3's vmap)."""

    def __init__(self, families, sizes, seed, max_steps=None, n_balls=4, env_index_base=0, reward_mode=0,
                 lava_reward=0.0, env_indices=None, variants=None, action_cost=0.0, time_cost=0.0):
        fam = np.ascontiguousarray(families, np.int32)
        siz = np.ascontiguousarray(sizes, np.int32)
        self.n = int(fam.shape[0])
        ms = None if max_steps is None else np.ascontiguousarray(max_steps, np.int32)
        var = None if variants is None else np.ascontiguousarray(variants, np.int32)
        if env_indices is None:
            h = lib().orc_batch_create(self.n, _ptr(fam, ctypes.c_int32), _ptr(siz, ctypes.c_int32),
                                       _ptr(ms, ctypes.c_int32), _ptr(var, ctypes.c_int32), n_balls, seed,
                                       env_index_base, reward_mode, lava_reward)
        else:
            idx = np.ascontiguousarray(env_indices, np.uint32)
            assert idx.shape == (self.n,)
            h = lib().orc_batch_create_indexed(self.n, _ptr(fam, ctypes.c_int32), _ptr(siz, ctypes.c_int32),
                                               _ptr(ms, ctypes.c_int32), _ptr(var, ctypes.c_int32), n_balls, seed,
                                               _ptr(idx, ctypes.c_uint32), reward_mode, lava_reward)
        if not h:
            raise ValueError("invalid oracle batch arguments")
        self.h = h
        lib().orc_batch_set_costs(h, action_cost, time_cost)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_batch_destroy(h)
            self.h = None

    def _outs(self, lead, sym, rgb):
        n = self.n
        return {
            "obs_sym": np.zeros(lead + (n, 7, 7, 3), np.uint8) if sym else None,
            "obs_rgb": np.zeros(lead + (n, 224, 224, 3), np.uint8) if rgb else None,
            "reward": np.zeros(lead + (n,), np.float32),
            "terminated": np.zeros(lead + (n,), np.uint8),
            "truncated": np.zeros(lead + (n,), np.uint8),
        }

    def _call(self, fn, pre, o, atlas):
        at = None if atlas is None else np.ascontiguousarray(atlas, np.uint8).reshape(-1)
        fn(self.h, *pre, _ptr(o["obs_sym"], ctypes.c_uint8), _ptr(o["obs_rgb"], ctypes.c_uint8),
           _ptr(at, ctypes.c_uint8), _ptr(o["reward"], ctypes.c_float), _ptr(o["terminated"], ctypes.c_uint8),
           _ptr(o["truncated"], ctypes.c_uint8))

    def reset(self, sym=True, rgb=False, atlas=None):
        o = self._outs((), sym, rgb)
        self._call(lib().orc_batch_reset, (), o, atlas)
        return o

    def step(self, actions=None, sym=True, rgb=False, atlas=None):
        o = self._outs((), sym, rgb)
        a = None if actions is None else np.ascontiguousarray(actions, np.int8)
        self._call(lib().orc_batch_step, (_ptr(a, ctypes.c_int8),), o, atlas)
        return o

    def rollout(self, T, actions=None, sym=True, rgb=False, atlas=None):
        o = self._outs((T,), sym, rgb)
        a = None if actions is None else np.ascontiguousarray(actions, np.int8)
        self._call(lib().orc_batch_rollout, (ctypes.c_int32(T), _ptr(a, ctypes.c_int8)), o, atlas)
        return o

    def full_views(self, side):
        """Current fully observable views: (symbolic [n,side,side,3], categorical [n,side,side], cat_fp [n,7,7])."""
        full = np.zeros((self.n, side, side, 3), np.uint8)
        cat = np.zeros((self.n, side, side), np.uint8)
        cfp = np.zeros((self.n, 7, 7), np.uint8)
        lib().orc_batch_obs_full(self.h, _ptr(full, ctypes.c_uint8), _ptr(cat, ctypes.c_uint8),
                                 _ptr(cfp, ctypes.c_uint8), side)
        return full, cat, cfp

    def rgb_full(self, atlas, side):
        img = np.zeros((self.n, 32 * side, 32 * side, 3), np.uint8)
        at = np.ascontiguousarray(atlas, np.uint8).reshape(-1)
        lib().orc_batch_obs_rgb_full(self.h, _ptr(at, ctypes.c_uint8), _ptr(img, ctypes.c_uint8), side)
        return img

    def rollout_policy(self, T, policy):
        """T steps with the policy choosing each env's action from its current view."""
        o = {"actions": np.zeros((T, self.n), np.int8), "obs_sym": np.zeros((T, self.n, 7, 7, 3), np.uint8),
             "reward": np.zeros((T, self.n), np.float32), "terminated": np.zeros((T, self.n), np.uint8),
             "truncated": np.zeros((T, self.n), np.uint8)}
        lib().orc_batch_rollout_policy(self.h, T, ctypes.byref(policy.s), _ptr(o["actions"], ctypes.c_int8),
                                       _ptr(o["obs_sym"], ctypes.c_uint8), _ptr(o["reward"], ctypes.c_float),
                                       _ptr(o["terminated"], ctypes.c_uint8), _ptr(o["truncated"], ctypes.c_uint8))
        return o

    def missions(self):
        return np.array([self.env(i).mission for i in range(self.n)], np.uint8)

    def rollout_full(self, T, side, actions=None, atlas=None):
        """T steps with every output, including the fully observable views
        (and the full RGB view when an atlas is given)."""
        outs = []
        for t in range(T):
            o = self.step(None if actions is None else actions[t])
            o["obs_full"], o["obs_cat"], o["obs_cat_fp"] = self.full_views(side)
            o["mission"] = self.missions()
            if atlas is not None:
                o["obs_rgb_full"] = self.rgb_full(atlas, side)
            outs.append(o)
        return {k: np.stack([o[k] for o in outs]) for k in outs[0] if outs[0][k] is not None}

    def env(self, i) -> OrcEnv:
        return lib().orc_batch_env(self.h, i).contents

    def state(self, i) -> dict:
        return env_state(self.env(i))

    @property
    def gstep(self):
        return int(lib().orc_batch_gstep(self.h))
