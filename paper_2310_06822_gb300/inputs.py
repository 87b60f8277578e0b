"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module only draws numbers: sphere-union scenes, query encodings, evaluation
grids and initial network weights.  It holds none of the method's arithmetic
(no predicate, no network, no loss); both the CUDA library and the FP64 oracle
consume what it produces.

Number format (our reading; the paper is silent on it).  Every coordinate,
radius, direction, offset, half-extent, time and velocity is an integer multiple
of a power-of-two grid quantum ``2**-qexp`` (``qexp = 20`` for scenes inside
[-1, 1]^n, ``qexp = 18`` for the cascade's world coordinates), so each value is
exact in FP32 and exact as a scaled integer.  That lets the indicator of Sec. 3.1
(1 inside *and on* the surface) be decided exactly.

Query encodings (one row per query, FP32, row-major):

=========  =====  ====================================================
kind       width  row
=========  =====  ====================================================
POINT2     2      (x, y)
POINT3     3      (x, y, z)
POINT4T    4      (x, y, z, t)       sphere centre moves as c + v t
RAY3       6      (ox, oy, oz, dx, dy, dz)   half-line o + s d, s >= 0
PLANE3     4      (nx, ny, nz, off)  plane {x : n . x = off}
BOX3       6      (bx, by, bz, ex, ey, ez)   centre b, half-extents e
=========  =====  ====================================================

The paper parameterises rays by start and direction, planes by a point and a
normal and boxes by two corners (Suppl. Sec. "Parameterization"); the
encodings above carry the same information in the form the configurations
state.
"""
from __future__ import annotations

import dataclasses
import numpy as np

POINT2, POINT3, POINT4T, RAY3, PLANE3, BOX3 = range(6)
KIND_NAMES = ["point2", "point3", "point4t", "ray3", "plane3", "box3"]
ENC_WIDTH = [2, 3, 4, 6, 4, 6]
SCENE_DIM = [2, 3, 3, 3, 3, 3]


def kind_id(kind) -> int:
    if isinstance(kind, str):
        return KIND_NAMES.index(kind)
    return int(kind)


def quantize(x, qexp: int) -> np.ndarray:
    """Round to the nearest multiple of 2**-qexp (ties to even) and store as FP32."""
    q = 2.0 ** -qexp
    return (np.rint(np.asarray(x, dtype=np.float64) / q) * q).astype(np.float32)


@dataclasses.dataclass
class Scene:
    """A union of spheres (disks in 2D).  ``vel`` is set for moving spheres."""

    centres: np.ndarray  # (S, dim) float32
    radii: np.ndarray  # (S,) float32
    vel: np.ndarray | None  # (S, 3) float32 or None
    qexp: int

    @property
    def dim(self) -> int:
        return int(self.centres.shape[1])

    @property
    def n_spheres(self) -> int:
        return int(self.radii.shape[0])


def make_scene(seed: int, n_spheres: int, dim: int, r_lo: float, r_hi: float,
               moving: bool = False, qexp: int = 20, extent: float = 1.0,
               v_max: float = 0.5) -> Scene:
    """Union of ``n_spheres`` spheres: centres U[-extent, extent]^dim, radii U[r_lo, r_hi],
    velocities U[-v_max, v_max]^3 when ``moving``."""
    rng = np.random.default_rng(seed)
    c = quantize(rng.uniform(-extent, extent, size=(n_spheres, dim)), qexp)
    r = quantize(rng.uniform(r_lo, r_hi, size=n_spheres), qexp)
    v = quantize(rng.uniform(-v_max, v_max, size=(n_spheres, 3)), qexp) if moving else None
    return Scene(c, r, v, qexp)


def _unit_vectors(rng, n: int) -> np.ndarray:
    g = rng.standard_normal(size=(n, 3))
    nrm = np.linalg.norm(g, axis=1, keepdims=True)
    nrm[nrm == 0] = 1.0
    return g / nrm


def sample_queries(kind, seed: int, n: int, qexp: int = 20, *,
                   ray_radius: float = 2.0, e_lo: float = 0.01, e_hi: float = 0.5,
                   t_max: float = 1.0) -> np.ndarray:
    """Draw ``n`` queries of ``kind`` with the distributions of the configurations.

    points U[-1,1]^n; 4D points (x U[-1,1]^3, t U[0,t_max]); rays with origin uniform
    on the sphere of radius ``ray_radius`` and direction uniform on S^2; planes with a
    unit normal uniform on S^2 and offset U[-1,1]; boxes with centre U[-1,1]^3 and
    each half-extent log-uniform in [e_lo, e_hi].
    """
    k = kind_id(kind)
    rng = np.random.default_rng(seed)
    if k == POINT2:
        x = rng.uniform(-1, 1, size=(n, 2))
    elif k == POINT3:
        x = rng.uniform(-1, 1, size=(n, 3))
    elif k == POINT4T:
        x = np.concatenate([rng.uniform(-1, 1, size=(n, 3)), rng.uniform(0, t_max, size=(n, 1))], 1)
    elif k == RAY3:
        x = np.concatenate([ray_radius * _unit_vectors(rng, n), _unit_vectors(rng, n)], 1)
    elif k == PLANE3:
        x = np.concatenate([_unit_vectors(rng, n), rng.uniform(-1, 1, size=(n, 1))], 1)
    elif k == BOX3:
        e = np.exp(rng.uniform(np.log(e_lo), np.log(e_hi), size=(n, 3)))
        x = np.concatenate([rng.uniform(-1, 1, size=(n, 3)), e], 1)
    else:
        raise ValueError(f"unknown kind {kind}")
    return np.ascontiguousarray(quantize(x, qexp))


@dataclasses.dataclass
class MultiScene:
    """Objects scattered in a world: object k is a union of spheres given in world
    coordinates, with the frame centre its network was trained in and a box around it."""

    centres: np.ndarray         # (S, 3) float32, world
    radii: np.ndarray           # (S,) float32
    sphere_offsets: np.ndarray  # (K+1,) int64
    obj_centre: np.ndarray      # (K, 3) float32, world
    aabb: np.ndarray            # (K, 6) float32, min xyz / max xyz, slightly inflated
    qexp: int
    ball_radius: float

    @property
    def n_objects(self) -> int:
        return int(self.obj_centre.shape[0])

    def local_scene(self, k: int, qexp: int = 20) -> Scene:
        """Object k's spheres in its own frame (exact: both sides on the world grid)."""
        a, b = int(self.sphere_offsets[k]), int(self.sphere_offsets[k + 1])
        c = (self.centres[a:b].astype(np.float64) - self.obj_centre[k].astype(np.float64)).astype(np.float32)
        return Scene(c, self.radii[a:b].copy(), None, qexp)


def make_multi_scene(seed: int, n_objects: int, n_spheres: int, r_lo: float = 0.02, r_hi: float = 0.2,
                     world: float = 10.0, qexp: int = 18, ball_radius: float = 2.0) -> MultiScene:
    """n_objects unions of n_spheres spheres (local centres U[-1,1]^3, radii U[r_lo, r_hi])
    with world centres U[-world, world]^3, all on the 2^-qexp grid."""
    rng = np.random.default_rng(seed)
    oc = quantize(rng.uniform(-world, world, size=(n_objects, 3)), qexp)
    loc = quantize(rng.uniform(-1, 1, size=(n_objects, n_spheres, 3)), qexp)
    rad = quantize(rng.uniform(r_lo, r_hi, size=(n_objects, n_spheres)), qexp)
    cen = (oc[:, None, :].astype(np.float64) + loc.astype(np.float64)).astype(np.float32)
    lo = (cen - rad[..., None]).min(axis=1).astype(np.float64)
    hi = (cen + rad[..., None]).max(axis=1).astype(np.float64)
    pad = 1e-3 * (1.0 + np.abs(np.concatenate([lo, hi], 1)))
    box = np.concatenate([lo, hi], 1) + np.concatenate([-pad[:, :3], pad[:, 3:]], 1)
    off = np.arange(n_objects + 1, dtype=np.int64) * n_spheres
    return MultiScene(np.ascontiguousarray(cen.reshape(-1, 3)), np.ascontiguousarray(rad.reshape(-1)), off, oc,
                      np.ascontiguousarray(box.astype(np.float32)), qexp, ball_radius)


def sample_world_rays(seed: int, n: int, radius: float = 35.0, world: float = 10.0, qexp: int = 18) -> np.ndarray:
    """Rays with origin uniform on the sphere of `radius` around the world centre, aimed at
    a point uniform in [-world, world]^3 (unit direction), on the 2^-qexp grid."""
    rng = np.random.default_rng(seed)
    o = radius * _unit_vectors(rng, n)
    tgt = rng.uniform(-world, world, size=(n, 3))
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return np.ascontiguousarray(quantize(np.concatenate([o, d], 1), qexp))


def grid_points_2d(res: int = 256) -> np.ndarray:
    """Cell centres of a res x res grid over [-1,1]^2: -1 + (2i+1)/res (exact in binary)."""
    c = -1.0 + (2.0 * np.arange(res) + 1.0) / res
    yy, xx = np.meshgrid(c, c, indexing="ij")
    return np.ascontiguousarray(np.stack([xx.ravel(), yy.ravel()], 1).astype(np.float32))


def param_count(widths) -> int:
    """Flat parameter layout: for each layer l, W_l (out x in, row-major) then b_l (out)."""
    return int(sum(widths[i + 1] * (widths[i] + 1) for i in range(len(widths) - 1)))


def init_params(seed: int, widths) -> np.ndarray:
    """PyTorch-default-style initialisation: W and b uniform in +-1/sqrt(fan_in)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(len(widths) - 1):
        fan_in, fan_out = widths[i], widths[i + 1]
        bound = 1.0 / np.sqrt(fan_in)
        out.append(rng.uniform(-bound, bound, size=fan_out * fan_in))
        out.append(rng.uniform(-bound, bound, size=fan_out))
    return np.concatenate(out).astype(np.float32)


def random_bits(seed: int, n: int, p: float = 0.5) -> np.ndarray:
    """Random 0/1 labels packed 32 per uint32 word (bit i%32 of word i//32)."""
    rng = np.random.default_rng(seed)
    return pack_bits(rng.random(n) < p)


def pack_bits(b) -> np.ndarray:
    """Pack booleans 32 per uint32 word: bit i%32 of word i//32 (little-endian words)."""
    b = np.asarray(b, dtype=bool).ravel()
    pad = (-b.size) % 32
    if pad:
        b = np.concatenate([b, np.zeros(pad, dtype=bool)])
    return np.packbits(b, bitorder="little").view("<u4").astype(np.uint32)


def unpack_bits(words, n: int) -> np.ndarray:
    w = np.ascontiguousarray(np.asarray(words, dtype="<u4"))
    return np.unpackbits(w.view(np.uint8), bitorder="little")[:n].astype(bool)
