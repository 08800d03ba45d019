"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds none of the environment's arithmetic: it only produces
*inputs* -- the sprite atlas (the image data behind the ``Sprite`` component of
the paper's Table 1, which the RGB observations of Table 4 are assembled
from) and seeded action arrays.  Both the CUDA library and the CPU oracle take
these arrays as arguments; neither generates them.

Sprite atlas convention (an interface between the atlas and the renderers):
``ATLAS_TILES`` tiles of 32x32x3 uint8, row-major pixels, RGB.

* tile 0: an unseen cell (black with a grey grid line, not highlighted);
* tile ``1 + 18*ent + 3*col + st``: a visible cell holding the symbolic triple
  (ent, col, st), ent in 0..10, col in 0..5, st in 0..2, highlighted;
* tile ``199 + 18*ent + 3*col + st``: the agent's own cell, i.e. the agent
  (a red triangle pointing up, since the view is egocentric) drawn over what
  it carries, highlighted;
* tile ``397 + dir``: the agent facing east, south, west or north on an empty
  cell, highlighted (the fully observable RGB view).

Every tile carries its own index in its bottom-right pixel, so no two tiles
are equal.

The sprite designs are this project's own (the paper's sprite files are not
available); every tile is drawn with 3x3 supersampled coverage in integer
arithmetic, so the atlas is bit-identical on every machine.
"""
from __future__ import annotations

import numpy as np

TILE = 32
TILE_BYTES = TILE * TILE * 3
N_ENT, N_COL, N_ST = 11, 6, 3
EGO_TILES = 1 + 2 * N_ENT * N_COL * N_ST  # 397
ATLAS_TILES = EGO_TILES + 4  # 401

# colour palette (index -> RGB); codes follow the colour table of the cell encoding
COLOURS = np.array(
    [[255, 0, 0], [0, 255, 0], [0, 0, 255], [112, 39, 195], [255, 255, 0], [100, 100, 100]], np.int64
)
GRID_LINE = np.array([100, 100, 100], np.int64)

_SS = 3  # supersampling factor


def _sample_coords():
    # sub-pixel centres in [0, 1): pixel p, sub-sample s -> (p + (s + 0.5)/3) / 32, kept as exact rationals
    sub = (np.arange(TILE * _SS) * 2 + 1)  # numerators over 2*3*32 = 192
    return sub  # coordinate = sub / 192


_SUB = _sample_coords()
_DEN = 2 * _SS * TILE  # 192


def _coverage(mask_fn) -> np.ndarray:
    """Integer coverage count 0..9 per pixel of a shape given as a predicate on
    integer sub-sample coordinates (x, y) in units of 1/192 of the tile."""
    ys, xs = np.meshgrid(_SUB, _SUB, indexing="ij")
    inside = mask_fn(xs, ys).astype(np.int64)
    return inside.reshape(TILE, _SS, TILE, _SS).sum(axis=(1, 3))


def _blend(img: np.ndarray, cov: np.ndarray, colour) -> None:
    c = np.asarray(colour, np.int64)
    img[:] = img + ((c[None, None, :] - img) * cov[:, :, None]) // (_SS * _SS)


def _rect(x0, y0, x1, y1):
    a, b, c, d = (int(round(v * _DEN)) for v in (x0, y0, x1, y1))
    return lambda x, y: (x >= a) & (x < c) & (y >= b) & (y < d)


def _circle(cx, cy, r):
    a, b, rr = int(round(cx * _DEN)), int(round(cy * _DEN)), int(round(r * _DEN))
    return lambda x, y: (x - a) ** 2 + (y - b) ** 2 <= rr * rr


def _triangle(p0, p1, p2):
    P = [(int(round(px * _DEN)), int(round(py * _DEN))) for px, py in (p0, p1, p2)]

    def f(x, y):
        def edge(a, b):
            return (b[0] - a[0]) * (y - a[1]) - (b[1] - a[1]) * (x - a[0])

        e0, e1, e2 = edge(P[0], P[1]), edge(P[1], P[2]), edge(P[2], P[0])
        return ((e0 >= 0) & (e1 >= 0) & (e2 >= 0)) | ((e0 <= 0) & (e1 <= 0) & (e2 <= 0))

    return f


def _base_tile() -> np.ndarray:
    img = np.zeros((TILE, TILE, 3), np.int64)
    img[0, :, :] = GRID_LINE
    img[:, 0, :] = GRID_LINE
    return img


def _draw_object(img: np.ndarray, ent: int, col: int, st: int) -> None:
    colour = COLOURS[col]
    if ent == 2:  # wall
        _blend(img, _coverage(_rect(0, 0, 1, 1)), COLOURS[col])
    elif ent == 3:  # floor
        _blend(img, _coverage(_rect(1 / 32, 1 / 32, 1, 1)), colour // 2)
    elif ent == 4:  # door: open = outline; closed = filled with a handle; locked = filled with a key hole
        if st == 0:
            outer, inner = _coverage(_rect(0.88, 0, 1, 1)), None
            _blend(img, outer, colour)
            _blend(img, _coverage(_rect(0.92, 0.04, 0.96, 0.96)), [0, 0, 0])
        else:
            _blend(img, _coverage(_rect(0, 0, 1, 1)), colour)
            _blend(img, _coverage(_rect(0.04, 0.04, 0.96, 0.96)), [0, 0, 0])
            _blend(img, _coverage(_rect(0.08, 0.08, 0.92, 0.92)), colour)
            _blend(img, _coverage(_rect(0.12, 0.12, 0.88, 0.88)), [0, 0, 0])
            if st == 1:
                _blend(img, _coverage(_circle(0.75, 0.5, 0.08)), colour)
            else:
                _blend(img, _coverage(_rect(0.52, 0.45, 0.75, 0.55)), colour)
    elif ent == 5:  # key: head ring, shaft, teeth
        _blend(img, _coverage(_rect(0.5, 0.31, 0.63, 0.88)), colour)
        _blend(img, _coverage(_rect(0.38, 0.59, 0.5, 0.66)), colour)
        _blend(img, _coverage(_rect(0.38, 0.81, 0.5, 0.88)), colour)
        _blend(img, _coverage(_circle(0.56, 0.28, 0.19)), colour)
        _blend(img, _coverage(_circle(0.56, 0.28, 0.064)), [0, 0, 0])
    elif ent == 6:  # ball
        _blend(img, _coverage(_circle(0.5, 0.5, 0.31)), colour)
    elif ent == 7:  # box: outline with a lid line
        _blend(img, _coverage(_rect(0.12, 0.12, 0.88, 0.88)), colour)
        _blend(img, _coverage(_rect(0.18, 0.18, 0.82, 0.82)), [0, 0, 0])
        _blend(img, _coverage(_rect(0.16, 0.48, 0.84, 0.52)), colour)
    elif ent == 8:  # goal
        _blend(img, _coverage(_rect(1 / 32, 1 / 32, 1, 1)), colour)
    elif ent == 9:  # lava: orange with three dark waves
        _blend(img, _coverage(_rect(1 / 32, 1 / 32, 1, 1)), [255, 128, 0])
        for k in range(3):
            y0 = 0.3 + 0.2 * k
            _blend(img, _coverage(_rect(0.1, y0, 0.9, y0 + 0.04)), [0, 0, 0])
    elif ent == 10:  # an agent code as a cell
        _draw_agent(img)
    # ent 0 (unseen) and 1 (empty): nothing drawn


def _draw_agent(img: np.ndarray, direction: int = 3) -> None:
    """A red triangle pointing east (0), south (1), west (2) or north (3)."""
    tri = {3: ((0.5, 0.12), (0.85, 0.88), (0.15, 0.88)), 1: ((0.5, 0.88), (0.15, 0.12), (0.85, 0.12)),
           0: ((0.88, 0.5), (0.12, 0.15), (0.12, 0.85)), 2: ((0.12, 0.5), (0.88, 0.85), (0.88, 0.15))}[direction]
    _blend(img, _coverage(_triangle(*tri)), [255, 0, 0])


def _highlight(img: np.ndarray) -> np.ndarray:
    return img + ((255 - img) * 3) // 10


def tile_params(t: int):
    """Inverse of the atlas convention: tile index -> (visible, agent_cell, ent, col, st);
    for the directional agent tiles, agent_cell is 2 and st holds the direction."""
    if t == 0:
        return 0, 0, 0, 0, 0
    if t >= EGO_TILES:
        return 1, 2, 10, 0, t - EGO_TILES
    agent = 1 if t >= 199 else 0
    r = t - (199 if agent else 1)
    return 1, agent, r // 18, (r % 18) // 3, r % 3


def make_atlas() -> np.ndarray:
    """The sprite atlas: uint8 [ATLAS_TILES, 32, 32, 3]."""
    atlas = np.zeros((ATLAS_TILES, TILE, TILE, 3), np.uint8)
    for t in range(ATLAS_TILES):
        visible, agent, ent, col, st = tile_params(t)
        img = _base_tile()
        if visible and agent == 2:
            _draw_agent(img, st)
            img = _highlight(img)
        elif visible:
            _draw_object(img, ent, col, st)
            if agent:
                _draw_agent(img)
            img = _highlight(img)
        # a one-pixel index mark in the bottom-right corner makes all tiles
        # distinct, so a wrong tile choice can never go unnoticed
        img[TILE - 1, TILE - 1, :] = [t & 0xFF, (t >> 8) & 0xFF, 0x5A]
        atlas[t] = np.clip(img, 0, 255).astype(np.uint8)
    return atlas


_ATLAS_CACHE = None


def atlas() -> np.ndarray:
    global _ATLAS_CACHE
    if _ATLAS_CACHE is None:
        _ATLAS_CACHE = make_atlas()
        _ATLAS_CACHE.setflags(write=False)
    return _ATLAS_CACHE


def random_actions(seed: int, shape, n_actions: int = 7, invalid_fraction: float = 0.0) -> np.ndarray:
    """Seeded int8 action array; with ``invalid_fraction`` > 0 some entries are
    out of range (negative or >= 7) to exercise the no-op + sticky-flag path."""
    rng = np.random.default_rng(seed)
    a = rng.integers(0, n_actions, size=shape, dtype=np.int64)
    if invalid_fraction > 0:
        bad = rng.random(size=shape) < invalid_fraction
        a = np.where(bad, rng.choice(np.array([-3, -1, 7, 9, 100, -128]), size=shape), a)
    return a.astype(np.int8)


def policy_weights(seed: int, n_agents: int, wmax: int = 12, bmax: int = 300) -> dict:
    """Seeded synthetic weights of the fused rollout's integer MLP policy:
    w1 [A, 64, 49], w2 [A, 64, 64], w3 [A, 7, 64] int8 uniform in
    [-wmax, wmax]; b1, b2 [A, 64], b3 [A, 7] int32 uniform in [-bmax, bmax].
    (No trained weights exist here: these stand in for a policy's parameters.)"""
    rng = np.random.default_rng(seed)
    A = int(n_agents)
    return dict(w1=rng.integers(-wmax, wmax + 1, (A, 64, 49)).astype(np.int8),
                b1=rng.integers(-bmax, bmax + 1, (A, 64)).astype(np.int32),
                w2=rng.integers(-wmax, wmax + 1, (A, 64, 64)).astype(np.int8),
                b2=rng.integers(-bmax, bmax + 1, (A, 64)).astype(np.int32),
                w3=rng.integers(-wmax, wmax + 1, (A, 7, 64)).astype(np.int8),
                b3=rng.integers(-bmax, bmax + 1, (A, 7)).astype(np.int32))
