"""Thin ctypes binding of libnavixgb (include/navixgb.h).

Functions keep the C names (``nx_create``, ``nx_reset``, ``nx_step``,
``nx_rollout`` ...) and only marshal arguments; every step of the
environment runs in the CUDA kernels of the library.  PyTorch provides the
device memory (its caching allocator, passed in as the library's allocator
callbacks, and output tensors) and the stream.  There is no CPU fallback: if
the library has not been built this module raises on first use.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libnavixgb.so")

NX_OK, NX_PENDING = 0, 1
NX_E_INVAL, NX_E_NOMEM, NX_E_CUDA, NX_E_TIMEOUT, NX_E_DEVICE_CHECK, NX_E_BUDGET, NX_E_STATE = -1, -2, -3, -4, -5, -6, -7
NX_E_CANCELED = -8
(NX_EMPTY, NX_DOORKEY, NX_FOURROOMS, NX_LAVAGAP, NX_DYNOBS, NX_EMPTY_RANDOM, NX_LAVA_CROSSING, NX_SIMPLE_CROSSING,
 NX_GOTODOOR, NX_DISTSHIFT, NX_KEYCORRIDOR) = range(11)
NX_N_FAMILIES = 11
NX_REQ_DIGEST = 1
NX_NO_MISSION = 255
NX_OBS_SYM, NX_OBS_RGB, NX_OBS_RGB_FULL = 1, 2, 4
NX_ACT_BUFFER, NX_ACT_RANDOM, NX_ACT_POLICY = 0, 1, 2
NX_REWARD_MARKOV, NX_REWARD_MINIGRID = 0, 1
NX_STAGE_AUTO, NX_STAGE_FULL, NX_STAGE_HALF = 0, 1, 2
OBS_SYM_BYTES, OBS_RGB_BYTES = 147, 150528
ATLAS_BYTES = 401 * 3072
AGENT_BYTES = 32
FAMILIES = {"empty": NX_EMPTY, "doorkey": NX_DOORKEY, "fourrooms": NX_FOURROOMS, "lavagap": NX_LAVAGAP,
            "dynobs": NX_DYNOBS, "empty_random": NX_EMPTY_RANDOM, "lava_crossing": NX_LAVA_CROSSING,
            "simple_crossing": NX_SIMPLE_CROSSING, "gotodoor": NX_GOTODOOR, "distshift": NX_DISTSHIFT,
            "keycorridor": NX_KEYCORRIDOR}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class nx_desc(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int32), ("height", ctypes.c_int32), ("width", ctypes.c_int32),
                ("max_steps", ctypes.c_int32), ("variant", ctypes.c_int32)]


class nx_options(ctypes.Structure):
    _fields_ = [("obs_flags", ctypes.c_uint32), ("reward_mode", ctypes.c_int32), ("lava_reward", ctypes.c_float),
                ("n_balls", ctypes.c_int32), ("steps_per_launch", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("group_lanes", ctypes.c_int32), ("envs_per_cta", ctypes.c_int32), ("staging", ctypes.c_int32),
                ("atlas", ctypes.POINTER(ctypes.c_uint8)), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_user", ctypes.c_void_p), ("env_index_base", ctypes.c_uint32), ("variant", ctypes.c_int32),
                ("action_cost", ctypes.c_float), ("time_cost", ctypes.c_float), ("grid_side", ctypes.c_int32)]


class nx_out(ctypes.Structure):
    _fields_ = [("obs_sym", ctypes.c_void_p), ("obs_rgb", ctypes.c_void_p), ("reward", ctypes.c_void_p),
                ("terminated", ctypes.c_void_p), ("truncated", ctypes.c_void_p), ("depth", ctypes.c_int32),
                ("full_side", ctypes.c_int32), ("obs_full", ctypes.c_void_p), ("obs_cat", ctypes.c_void_p),
                ("obs_cat_fp", ctypes.c_void_p), ("obs_rgb_full", ctypes.c_void_p), ("mission", ctypes.c_void_p),
                ("action", ctypes.c_void_p)]

OUT_KEYS = ("obs_sym", "obs_rgb", "reward", "terminated", "truncated", "obs_full", "obs_cat", "obs_cat_fp",
            "obs_rgb_full", "mission", "action")


def out_layout(key, side):
    """Element type and per-env shape of output `key` (side: the fully
    observable views' side, the batch's largest grid)."""
    return {"obs_sym": ("uint8", (7, 7, 3)), "obs_rgb": ("uint8", (224, 224, 3)), "reward": ("float32", ()),
            "terminated": ("uint8", ()), "truncated": ("uint8", ()), "obs_full": ("uint8", (side, side, 3)),
            "obs_cat": ("uint8", (side, side)), "obs_cat_fp": ("uint8", (7, 7)),
            "obs_rgb_full": ("uint8", (32 * side, 32 * side, 3)), "mission": ("uint8", ()),
            "action": ("int8", ())}[key]


def check_out_buffer(key, a, n, side, slots, device):
    """Refuses an output buffer the library would write outside of: it must
    be contiguous, of the output's element type, shaped [slots', n, ...] with
    slots' >= slots (or [n, ...] when slots is None), and on the device
    (device=True) or in host memory."""
    dtype, per_env = out_layout(key, side)
    shape = tuple(int(x) for x in a.shape)
    if slots is None:
        ok_shape = shape == (n,) + per_env
        want = f"[{n}, ...] = {(n,) + per_env}"
    else:
        ok_shape = len(shape) == 2 + len(per_env) and shape[0] >= slots and shape[1:] == (n,) + per_env
        want = f"[>= {slots}, {n}, ...] = {(slots, n) + per_env}"
    if not ok_shape:
        raise ValueError(f"output {key}: shape {shape}, expected {want}")
    if isinstance(a, np.ndarray):
        if device:
            raise ValueError(f"output {key}: a host array where a device tensor is needed")
        if a.dtype != np.dtype(dtype) or not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"output {key}: needs a C-contiguous {dtype} array, got {a.dtype}")
        return
    if str(a.dtype) != f"torch.{dtype}" or not a.is_contiguous():
        raise ValueError(f"output {key}: needs a contiguous torch.{dtype} tensor, got {a.dtype}")
    if bool(a.is_cuda) != device:
        raise ValueError(f"output {key}: a {'host' if a.is_cuda is False else 'device'} tensor where a "
                         f"{'device' if device else 'host'} one is needed")


class nx_policy(ctypes.Structure):
    _fields_ = [("n_agents", ctypes.c_int32), ("envs_per_agent", ctypes.c_int32),
                ("w1", ctypes.c_void_p), ("b1", ctypes.c_void_p), ("w2", ctypes.c_void_p), ("b2", ctypes.c_void_p),
                ("w3", ctypes.c_void_p), ("b3", ctypes.c_void_p), ("shift1", ctypes.c_int32),
                ("shift2", ctypes.c_int32), ("epsilon", ctypes.c_uint32)]


class nx_info(ctypes.Structure):
    _fields_ = [("group_lanes", ctypes.c_int32), ("envs_per_cta", ctypes.c_int32), ("staging", ctypes.c_int32),
                ("n_items", ctypes.c_int32), ("grid_ctas", ctypes.c_int32), ("smem_bytes", ctypes.c_int32),
                ("steps_per_launch", ctypes.c_int32), ("n_envs", ctypes.c_int32), ("n_families", ctypes.c_int32),
                ("state_bytes", ctypes.c_size_t), ("device_bytes", ctypes.c_size_t),
                ("policy_items", ctypes.c_int32), ("policy_ctas_per_sm", ctypes.c_int32),
                ("policy_grid_ctas", ctypes.c_int32), ("policy_smem_bytes", ctypes.c_int32),
                ("lean_family", ctypes.c_int32), ("lean_grid_ctas", ctypes.c_int32), ("grid_side", ctypes.c_int32)]


class nx_request(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int32), ("size", ctypes.c_int32), ("n_envs", ctypes.c_int32),
                ("horizon", ctypes.c_int32), ("variant", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("returns", ctypes.c_void_p), ("final_obs", ctypes.c_void_p)]


class nx_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("digest", ctypes.c_uint64), ("env_steps", ctypes.c_uint64),
                ("episodes", ctypes.c_uint32)]


class nx_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("finished", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("env_steps", ctypes.c_uint64), ("chunks", ctypes.c_uint64), ("busy_s", ctypes.c_double),
                ("budget_bytes", ctypes.c_size_t), ("in_use_bytes", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t), ("canceled", ctypes.c_uint64)]


# every symbol include/navixgb.h declares, with its signature
_P = ctypes.POINTER
_vp, _i32, _u32, _u64, _sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t
SIGNATURES = {
    "nx_options_default": (None, [_P(nx_options)]),
    "nx_max_variant": (_i32, [_i32, _i32]),
    "nx_create": (_i32, [_P(_vp), _i32, _i32, _i32, _u64, _P(nx_options), _vp]),
    "nx_create_mixed": (_i32, [_P(_vp), _P(nx_desc), _i32, _u64, _P(nx_options), _vp]),
    "nx_reset": (_i32, [_vp, _P(nx_out)]),
    "nx_step": (_i32, [_vp, _vp, _P(nx_out)]),
    "nx_rollout": (_i32, [_vp, _i32, _i32, _vp, _P(nx_out)]),
    "nx_rollout_per_family": (_i32, [_vp, _i32, _i32, _vp, _P(nx_out)]),
    "nx_rollout_host": (_i32, [_vp, _i32, _i32, _vp, _P(nx_out)]),
    "nx_state_bytes": (_sz, [_vp]),
    "nx_get_state": (_i32, [_vp, _vp, _sz]),
    "nx_set_state": (_i32, [_vp, _vp, _sz]),
    "nx_set_policy": (_i32, [_vp, _P(nx_policy)]),
    "nx_sync": (_i32, [_vp, ctypes.c_double]),
    "nx_device_flags": (_i32, [_vp, _P(_u32)]),
    "nx_get_info": (_i32, [_vp, _P(nx_info)]),
    "nx_rollout_noalloc": (_i32, [_i32, _i32, _i32, _u64, _i32, _i32, _vp, _P(nx_out), _vp]),
    "nx_profile_begin": (_i32, [_vp]),
    "nx_profile_end": (_i32, [_vp, _P(ctypes.c_double), _P(ctypes.c_int64)]),
    "nx_launch_counts": (_i32, [_vp, _P(ctypes.c_int64), _P(ctypes.c_int64)]),
    "nx_destroy": (None, [_vp]),
    "nx_server_create": (_i32, [_P(_vp), _sz, _P(nx_options), _vp]),
    "nx_submit": (_i32, [_vp, _P(nx_request), _P(_u64)]),
    "nx_poll": (_i32, [_vp, _u64, _P(nx_result)]),
    "nx_wait": (_i32, [_vp, _u64, _P(nx_result), ctypes.c_double]),
    "nx_cancel": (_i32, [_vp, _u64]),
    "nx_server_get_stats": (_i32, [_vp, _P(nx_server_stats)]),
    "nx_server_destroy": (None, [_vp]),
    "nx_status_str": (ctypes.c_char_p, [_i32]),
    "nx_last_error": (ctypes.c_char_p, [_vp]),
}

_lib = None
_lock = threading.Lock()


def lib():
    """Loads libnavixgb.so; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                                   "(python -c 'import __graft_entry__ as g; g.build()')")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class NavixError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def check(status, env_handle=None):
    if status < 0:
        L = lib()
        msg = L.nx_last_error(env_handle).decode() if env_handle is not None else L.nx_last_error(None).decode()
        raise NavixError(status, f"{L.nx_status_str(status).decode()}: {msg}")
    return status


# --- C-named wrappers (argument marshalling only) ---------------------------

def nx_options_default() -> nx_options:
    o = nx_options()
    lib().nx_options_default(ctypes.byref(o))
    return o


def nx_create(family, size, n_envs, seed, opts=None, stream=0):
    h = ctypes.c_void_p()
    st = lib().nx_create(ctypes.byref(h), family, size, n_envs, seed, ctypes.byref(opts) if opts else None,
                         ctypes.c_void_p(stream))
    check(st)
    return h


def nx_max_variant(family, size):
    return int(lib().nx_max_variant(family, size))


def nx_create_mixed(descs, seed, opts=None, stream=0):
    """descs: (family, size, max_steps, variant) per env."""
    arr = (nx_desc * len(descs))(*[nx_desc(int(f), int(s), int(s), int(m), int(v)) for f, s, m, v in descs])
    h = ctypes.c_void_p()
    st = lib().nx_create_mixed(ctypes.byref(h), arr, len(descs), seed, ctypes.byref(opts) if opts else None,
                               ctypes.c_void_p(stream))
    check(st)
    return h


def nx_reset(h, out):
    return check(lib().nx_reset(h, ctypes.byref(out) if out is not None else None), h)


def nx_step(h, actions_ptr, out):
    return check(lib().nx_step(h, ctypes.c_void_p(actions_ptr or None), ctypes.byref(out) if out is not None else None), h)


def nx_rollout(h, n_steps, act_mode, actions_ptr, out):
    return check(lib().nx_rollout(h, n_steps, act_mode, ctypes.c_void_p(actions_ptr or None),
                                  ctypes.byref(out) if out is not None else None), h)


def nx_set_policy(h, w1, b1, w2, b2, w3, b3, shift1, shift2, epsilon=0, envs_per_agent=128):
    """Uploads the fused policy's weights (numpy int8 / int32 arrays: w1 [A, 64, 49],
    b1 [A, 64], w2 [A, 64, 64], b2 [A, 64], w3 [A, 7, 64], b3 [A, 7])."""
    arrs = [np.ascontiguousarray(w1, np.int8), np.ascontiguousarray(b1, np.int32), np.ascontiguousarray(w2, np.int8),
            np.ascontiguousarray(b2, np.int32), np.ascontiguousarray(w3, np.int8), np.ascontiguousarray(b3, np.int32)]
    A = arrs[0].shape[0]
    if not (arrs[0].shape == (A, 64, 49) and arrs[2].shape == (A, 64, 64) and arrs[4].shape == (A, 7, 64) and
            arrs[1].shape == (A, 64) and arrs[3].shape == (A, 64) and arrs[5].shape == (A, 7)):
        raise ValueError("policy weights: w1 [A, 64, 49], b1 [A, 64], w2 [A, 64, 64], b2 [A, 64], w3 [A, 7, 64], "
                         "b3 [A, 7]")
    p = nx_policy(A, int(envs_per_agent), *[a.ctypes.data for a in arrs], int(shift1), int(shift2), int(epsilon))
    return check(lib().nx_set_policy(h, ctypes.byref(p)), h)


def nx_rollout_per_family(h, n_steps, act_mode, actions_ptr, out):
    return check(lib().nx_rollout_per_family(h, n_steps, act_mode, ctypes.c_void_p(actions_ptr or None),
                                             ctypes.byref(out) if out is not None else None), h)


def nx_rollout_host(h, n_steps, act_mode, actions_ptr, out):
    return check(lib().nx_rollout_host(h, n_steps, act_mode, ctypes.c_void_p(actions_ptr or None),
                                       ctypes.byref(out) if out is not None else None), h)


def nx_state_bytes(h):
    return int(lib().nx_state_bytes(h))


def nx_get_state(h) -> bytes:
    n = nx_state_bytes(h)
    buf = (ctypes.c_uint8 * n)()
    check(lib().nx_get_state(h, buf, n), h)
    return bytes(buf)


def nx_set_state(h, data: bytes):
    buf = (ctypes.c_uint8 * len(data)).from_buffer_copy(data)
    return check(lib().nx_set_state(h, buf, len(data)), h)


def nx_sync(h, timeout_s=0.0):
    return check(lib().nx_sync(h, timeout_s), h)


def nx_device_flags(h):
    f = ctypes.c_uint32()
    check(lib().nx_device_flags(h, ctypes.byref(f)), h)
    return int(f.value)


def nx_get_info(h) -> dict:
    i = nx_info()
    check(lib().nx_get_info(h, ctypes.byref(i)), h)
    return {k: getattr(i, k) for k, _ in nx_info._fields_}


def nx_rollout_noalloc(family, size, n_envs, seed, n_steps, act_mode, actions_ptr, out, stream=0):
    """Reset + rollout that allocates no device memory (see navixgb.h)."""
    return check(lib().nx_rollout_noalloc(family, size, n_envs, seed, n_steps, act_mode,
                                          ctypes.c_void_p(actions_ptr or None),
                                          ctypes.byref(out) if out is not None else None, ctypes.c_void_p(stream)))


def nx_profile_begin(h):
    return check(lib().nx_profile_begin(h), h)


def nx_profile_end(h):
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    check(lib().nx_profile_end(h, ctypes.byref(ms), ctypes.byref(n)), h)
    return float(ms.value), int(n.value)


def nx_launch_counts(h):
    a = ctypes.c_int64()
    b = ctypes.c_int64()
    check(lib().nx_launch_counts(h, ctypes.byref(a), ctypes.byref(b)), h)
    return int(a.value), int(b.value)


def nx_destroy(h):
    lib().nx_destroy(h)


# --- snapshot parsing (format documented in navixgb.h) -----------------------

def parse_state(data: bytes) -> dict:
    if data[:4] != b"NXST":
        raise ValueError("not a navixgb snapshot")
    n = int.from_bytes(data[8:12], "little")
    gstep = int.from_bytes(data[12:16], "little")
    pool = int.from_bytes(data[16:24], "little")
    ag = np.frombuffer(data, np.uint8, count=n * AGENT_BYTES, offset=64).reshape(n, AGENT_BYTES)
    grids = np.frombuffer(data, np.uint8, count=pool, offset=64 + n * AGENT_BYTES)
    envs = []
    off = 0  # envs are stored in order; the block holds the offset's low 32 bits
    for i in range(n):
        a = ag[i]
        size = int(a[25])
        if int(a[28:32].view(np.uint32)[0]) != off & 0xFFFFFFFF:
            raise ValueError("snapshot grid offsets out of order")
        hw = size * size
        nb = int(a[7])
        envs.append({
            "x": int(a[0]), "y": int(a[1]), "dir": int(a[2]), "carry_ent": int(a[3]), "carry_col": int(a[4]),
            "done": int(a[5]), "invalid": int(a[6]), "n_balls": nb,
            "t": int(a[8:10].view(np.uint16)[0]), "max_steps": int(a[10:12].view(np.uint16)[0]),
            "episode": int(a[12:16].view(np.uint32)[0]),
            "ball_x": [int(v) for v in a[16:16 + nb]], "ball_y": [int(v) for v in a[20:20 + nb]],
            "family": int(a[24]), "height": size, "width": size, "mission": int(a[26]),
            "ent": grids[off:off + hw].tobytes(), "col": grids[off + hw:off + 2 * hw].tobytes(),
            "st": grids[off + 2 * hw:off + 3 * hw].tobytes(),
        })
        off += 3 * hw
    return {"n": n, "gstep": gstep, "envs": envs}


# --- convenience class over torch tensors ------------------------------------

class Env:
    """A batch of environments on the current CUDA device.

    ``descs`` is a list of (family, size[, max_steps]) per env, or use
    ``family``/``size``/``n_envs`` for a uniform batch.  Outputs are torch
    tensors on the device, shaped [depth, N, ...] for rollouts and [N, ...]
    for reset/step.
    """

    def __init__(self, family=NX_EMPTY, size=5, n_envs=1, seed=0, *, descs=None, obs_sym=True, obs_rgb=False,
                 atlas=None, reward_mode=NX_REWARD_MARKOV, lava_reward=0.0, n_balls=4, steps_per_launch=128,
                 autotune=True, group_lanes=0, envs_per_cta=0, staging=0, env_index_base=0, variant=0,
                 obs_full=False, obs_cat=False, obs_cat_fp=False, obs_rgb_full=False, mission=None,
                 action_cost=0.0, time_cost=0.0, action=False, torch_allocator=True, grid_side=0):
        import torch

        self.torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("navixgb needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.current_stream(self.device)
        o = nx_options_default()
        o.obs_flags = (NX_OBS_SYM if obs_sym else 0) | (NX_OBS_RGB if obs_rgb else 0) | \
            (NX_OBS_RGB_FULL if obs_rgb_full else 0)
        o.reward_mode = reward_mode
        o.lava_reward = lava_reward
        o.action_cost = action_cost
        o.time_cost = time_cost
        o.grid_side = grid_side
        o.n_balls = n_balls
        o.steps_per_launch = steps_per_launch
        o.autotune = 1 if autotune else 0
        o.group_lanes = group_lanes
        o.envs_per_cta = envs_per_cta
        o.staging = staging
        o.env_index_base = env_index_base
        o.variant = variant
        self._atlas = None
        if obs_rgb or obs_rgb_full:
            if atlas is None:
                from . import inputs
                atlas = inputs.atlas()
            self._atlas = np.ascontiguousarray(atlas, np.uint8).reshape(-1)
            if self._atlas.size != ATLAS_BYTES:
                raise ValueError(f"the atlas holds {ATLAS_BYTES} bytes, got {self._atlas.size}")
            o.atlas = self._atlas.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        self._cbs = None
        if torch_allocator:
            dev, strm = self.device.index, self.stream.cuda_stream

            def _alloc(size, _user):
                return torch.cuda.caching_allocator_alloc(int(size), dev, strm)

            def _free(ptr, _user):
                torch.cuda.caching_allocator_delete(ptr)

            self._cbs = (ALLOC_FN(_alloc), FREE_FN(_free))
            o.alloc, o.free = self._cbs
        self.opts = o
        self.obs_sym, self.obs_rgb = obs_sym, obs_rgb
        self.want_full, self.want_cat, self.want_cat_fp = obs_full, obs_cat, obs_cat_fp
        self.want_rgb_full = obs_rgb_full
        self.want_action = action
        if descs is None:
            self.n = int(n_envs)
            self.side = int(size)
            self.h = nx_create(int(family), int(size), self.n, int(seed), o, self.stream.cuda_stream)
            fams = {int(family)}
        else:
            # each desc: (family, size[, max_steps[, variant]])
            d = [(f, s, (m[0] if len(m) > 0 else 0), (m[1] if len(m) > 1 else 0)) for f, s, *m in descs]
            self.n = len(d)
            self.side = max(x[1] for x in d)
            self.h = nx_create_mixed(d, int(seed), o, self.stream.cuda_stream)
            fams = {int(x[0]) for x in d}
        # the per-step mission output, by default only where a family has one
        self.want_mission = (NX_GOTODOOR in fams) if mission is None else bool(mission)

    def close(self):
        if getattr(self, "h", None):
            nx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def alloc_out(self, depth=None):
        torch = self.torch
        lead = () if depth is None else (depth,)
        n = self.n
        o = {
            "obs_sym": torch.empty(lead + (n, 7, 7, 3), dtype=torch.uint8, device=self.device) if self.obs_sym else None,
            "obs_rgb": torch.empty(lead + (n, 224, 224, 3), dtype=torch.uint8, device=self.device) if self.obs_rgb else None,
            "reward": torch.empty(lead + (n,), dtype=torch.float32, device=self.device),
            "terminated": torch.empty(lead + (n,), dtype=torch.uint8, device=self.device),
            "truncated": torch.empty(lead + (n,), dtype=torch.uint8, device=self.device),
        }
        F = self.side
        o["obs_full"] = torch.empty(lead + (n, F, F, 3), dtype=torch.uint8, device=self.device) if self.want_full else None
        o["obs_cat"] = torch.empty(lead + (n, F, F), dtype=torch.uint8, device=self.device) if self.want_cat else None
        o["obs_cat_fp"] = torch.empty(lead + (n, 7, 7), dtype=torch.uint8, device=self.device) if self.want_cat_fp else None
        o["obs_rgb_full"] = (torch.empty(lead + (n, 32 * F, 32 * F, 3), dtype=torch.uint8, device=self.device)
                             if self.want_rgb_full else None)
        o["mission"] = torch.empty(lead + (n,), dtype=torch.uint8, device=self.device) if self.want_mission else None
        o["action"] = torch.empty(lead + (n,), dtype=torch.int8, device=self.device) if self.want_action else None
        return o

    def out_struct(self, o, depth=None):
        """The nx_out of device buffers `o` ([n, ...] each for reset and step,
        [>= depth, n, ...] for a rollout ring of `depth` slots), each checked
        against the layout the library writes."""
        s = nx_out()
        for k in OUT_KEYS:
            t = o.get(k)
            if t is not None:
                check_out_buffer(k, t, self.n, self.side, depth, device=True)
            setattr(s, k, t.data_ptr() if t is not None else None)
        s.depth = 1 if depth is None else depth
        s.full_side = self.side
        return s

    def reset(self, out=None):
        out = out or self.alloc_out()
        nx_reset(self.h, self.out_struct(out))
        return out

    def step(self, actions=None, out=None):
        out = out or self.alloc_out()
        ptr = None
        if actions is not None:
            if not (actions.dtype == self.torch.int8 and actions.is_cuda and actions.numel() == self.n and
                    actions.is_contiguous()):
                raise ValueError(f"actions: a contiguous int8 device tensor of {self.n} entries")
            ptr = actions.data_ptr()
        nx_step(self.h, ptr, self.out_struct(out))
        return out

    def set_policy(self, w1, b1, w2, b2, w3, b3, shift1, shift2, epsilon=0, envs_per_agent=128):
        """The fused policy used by rollout(..., policy=True) (see nx_set_policy)."""
        nx_set_policy(self.h, w1, b1, w2, b2, w3, b3, shift1, shift2, epsilon, envs_per_agent)

    def rollout(self, n_steps, actions=None, depth=None, out=None, per_family=False, policy=False):
        depth = depth or n_steps
        out = out or self.alloc_out(depth)
        ptr, mode = None, (NX_ACT_POLICY if policy else NX_ACT_RANDOM)
        if actions is not None:
            if not (actions.dtype == self.torch.int8 and actions.is_cuda and tuple(actions.shape) == (n_steps, self.n)
                    and actions.is_contiguous()):
                raise ValueError(f"actions: a contiguous int8 device tensor [{n_steps}, {self.n}]")
            ptr, mode = actions.data_ptr(), NX_ACT_BUFFER
        fn = nx_rollout_per_family if per_family else nx_rollout
        fn(self.h, n_steps, mode, ptr, self.out_struct(out, depth))
        return out

    def rollout_host(self, n_steps, actions=None, out=None):
        """Host numpy in, host numpy out (pinned numpy-backed torch tensors may be passed as ``out``).
        Outputs with a leading dimension D < n_steps form a ring: step i lands in slot i % D."""
        n = self.n
        if out is None:
            out = {
                "obs_sym": np.empty((n_steps, n, 7, 7, 3), np.uint8) if self.obs_sym else None,
                "obs_rgb": np.empty((n_steps, n, 224, 224, 3), np.uint8) if self.obs_rgb else None,
                "reward": np.empty((n_steps, n), np.float32),
                "terminated": np.empty((n_steps, n), np.uint8),
                "truncated": np.empty((n_steps, n), np.uint8),
                "mission": np.empty((n_steps, n), np.uint8) if self.want_mission else None,
            }
        s = nx_out()
        depth = n_steps
        for k in ("obs_sym", "obs_rgb", "reward", "terminated", "truncated", "mission"):
            a = out.get(k)
            if a is None:
                setattr(s, k, None)
                continue
            check_out_buffer(k, a, n, self.side, 1, device=False)
            if isinstance(a, np.ndarray):
                setattr(s, k, a.ctypes.data)
            else:
                setattr(s, k, a.data_ptr())
            depth = min(depth, int(a.shape[0]))
        s.depth = depth
        ptr, mode = None, NX_ACT_RANDOM
        if actions is not None:
            a = actions if isinstance(actions, np.ndarray) else actions.numpy()
            if not (a.dtype == np.int8 and a.shape == (n_steps, n) and a.flags["C_CONTIGUOUS"]):
                raise ValueError(f"actions: a C-contiguous int8 host array [{n_steps}, {n}]")
            ptr, mode = a.ctypes.data, NX_ACT_BUFFER
        nx_rollout_host(self.h, n_steps, mode, ptr, s)
        return out

    def state(self) -> dict:
        return parse_state(nx_get_state(self.h))

    def state_bytes(self) -> bytes:
        return nx_get_state(self.h)

    def set_state(self, data: bytes):
        nx_set_state(self.h, data)

    def flags(self) -> int:
        return nx_device_flags(self.h)

    def sync(self, timeout_s=0.0):
        return nx_sync(self.h, timeout_s)

    def info(self) -> dict:
        return nx_get_info(self.h)

    def profile_begin(self):
        nx_profile_begin(self.h)

    def profile_end(self):
        """(summed step-kernel device ms, number of step-kernel launches) since profile_begin."""
        return nx_profile_end(self.h)

    def launch_counts(self):
        """(step-kernel launches, all kernel launches) so far."""
        return nx_launch_counts(self.h)


# --- serving -------------------------------------------------------------------

def _result_dict(r: nx_result) -> dict:
    return {k: getattr(r, k) for k, _ in nx_result._fields_}


def nx_server_create(budget_bytes, opts=None, stream=0):
    h = ctypes.c_void_p()
    check(lib().nx_server_create(ctypes.byref(h), budget_bytes, ctypes.byref(opts) if opts else None,
                                 ctypes.c_void_p(stream)))
    return h


def nx_submit(h, req: nx_request) -> int:
    t = ctypes.c_uint64()
    check(lib().nx_submit(h, ctypes.byref(req), ctypes.byref(t)))
    return int(t.value)


def nx_poll(h, ticket):
    r = nx_result()
    st = lib().nx_poll(h, ticket, ctypes.byref(r))
    if st == NX_PENDING:
        return None
    check(st)
    return _result_dict(r)


def nx_wait(h, ticket, timeout_s=0.0):
    r = nx_result()
    check(lib().nx_wait(h, ticket, ctypes.byref(r), timeout_s))
    return _result_dict(r)


def nx_cancel(h, ticket):
    return check(lib().nx_cancel(h, ticket))


def nx_server_get_stats(h) -> dict:
    st = nx_server_stats()
    check(lib().nx_server_get_stats(h, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in nx_server_stats._fields_}


def nx_server_destroy(h):
    lib().nx_server_destroy(h)


class Server:
    """Continuous-batching rollout server; results land in numpy arrays."""

    def __init__(self, budget_bytes=1 << 30, steps_per_launch=128, group_lanes=0, envs_per_cta=0,
                 reward_mode=NX_REWARD_MARKOV, lava_reward=0.0, n_balls=4, action_cost=0.0, time_cost=0.0,
                 stream=None, staging=0):
        o = nx_options_default()
        o.steps_per_launch = steps_per_launch
        o.group_lanes = group_lanes
        o.envs_per_cta = envs_per_cta
        o.staging = staging
        o.reward_mode = reward_mode
        o.lava_reward = lava_reward
        o.action_cost = action_cost
        o.time_cost = time_cost
        o.n_balls = n_balls
        if stream is None:
            try:
                import torch

                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        self.h = nx_server_create(budget_bytes, o, stream)
        self._bufs = {}

    def submit(self, family, size, n_envs, horizon, seed, variant=0, digest=True):
        """digest: also compute the request's digest of every per-step output."""
        ret = np.zeros(n_envs, np.float32)
        obs = np.zeros((n_envs, 7, 7, 3), np.uint8)
        r = nx_request(int(family), int(size), int(n_envs), int(horizon), int(variant),
                       NX_REQ_DIGEST if digest else 0, int(seed), ret.ctypes.data, obs.ctypes.data)
        t = nx_submit(self.h, r)
        self._bufs[t] = (ret, obs)
        return t

    def wait(self, ticket, timeout_s=0.0):
        res = nx_wait(self.h, ticket, timeout_s)
        ret, obs = self._bufs[ticket]
        res["returns"], res["final_obs"] = ret, obs
        return res

    def poll(self, ticket):
        res = nx_poll(self.h, ticket)
        if res is not None:
            ret, obs = self._bufs[ticket]
            res["returns"], res["final_obs"] = ret, obs
        return res

    def cancel(self, ticket):
        nx_cancel(self.h, ticket)

    def stats(self):
        return nx_server_get_stats(self.h)

    def close(self):
        if getattr(self, "h", None):
            nx_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
