"""Pins of the oracle's canonical-ray transform (the network input of the learned-culler
cascade): the ray in the object's frame with its origin moved to where it enters the ball
of radius R around the object's centre.  The oracle replays the library's defined FP32
operation sequence; these tests tie that sequence to the geometry it stands for: hand
cases with exact answers, the real-valued root (FP64) within a first-order rounding bound,
and the invariants of an entry point (on the sphere, on the ray, entering).

Runs on CPU only.
"""
import numpy as np

from oracle import oracle as O
from paper_2310_06822_gb300 import inputs as I

U = 2.0 ** -24


def _one(o, d, c=(0.0, 0.0, 0.0), R=2.0):
    rays = np.array([list(o) + list(d)], dtype=np.float32)
    cen = np.array([c], dtype=np.float32)
    q6, met = O.canonical_ray(rays, cen, R)
    return q6[0], bool(met[0])


def test_axis_ray_through_the_centre_enters_at_minus_R():
    # w = (-35, 0, 0), d = +x: |w + s d| = 2 at s = 33, entry (-2, 0, 0), exact in FP32
    q, met = _one((-35.0, 0.0, 0.0), (1.0, 0.0, 0.0))
    assert met
    assert q.tolist() == [-2.0, 0.0, 0.0, 1.0, 0.0, 0.0]
    # the object's centre is subtracted first: same ray seen from an object at (3, -4, 5)
    q, met = _one((-32.0, -4.0, 5.0), (1.0, 0.0, 0.0), c=(3.0, -4.0, 5.0))
    assert met and q.tolist() == [-2.0, 0.0, 0.0, 1.0, 0.0, 0.0]


def test_tangent_ray_touches_at_the_foot_of_the_perpendicular():
    # distance 2 from the centre: discriminant 0, the single point (0, 2, 0)
    q, met = _one((-35.0, 2.0, 0.0), (1.0, 0.0, 0.0))
    assert met
    assert q.tolist() == [0.0, 2.0, 0.0, 1.0, 0.0, 0.0]


def test_ray_missing_the_ball_is_not_met():
    q, met = _one((-35.0, 2.5, 0.0), (1.0, 0.0, 0.0))
    assert not met and not np.any(q)
    # a zero direction meets nothing
    _, met = _one((-35.0, 0.0, 0.0), (0.0, 0.0, 0.0))
    assert not met


def test_origin_inside_the_ball_stays_put():
    # the origin is already inside: s clamps to 0 and the entry point is the origin itself
    q, met = _one((0.5, 0.0, 0.0), (0.0, 1.0, 0.0))
    assert met and q.tolist() == [0.5, 0.0, 0.0, 0.0, 1.0, 0.0]


def test_ray_pointing_away_from_the_ball_enters_behind_its_origin_is_clamped():
    # the line meets the ball only at s < 0; the half-line s >= 0 does not enter it, and the
    # transform (like the paper's half-line rays) reports the origin clamped at s = 0; stage 1
    # never passes such a pair (its box test fails first), so only the formula is pinned here
    q, met = _one((-35.0, 0.0, 0.0), (-1.0, 0.0, 0.0))
    assert met and q[:3].tolist() == [-35.0, 0.0, 0.0]


def test_fp32_sequence_tracks_the_real_root():
    """Random world rays against random object centres (the cascade's distribution): the
    FP32 entry point is within a first-order rounding bound of the FP64 root.  Each of the
    sequence's dozen correctly rounded operations perturbs s or the entry point by at most
    u = 2^-24 relative to |w| + |s d|; the root's condition number 1 + |b| / sqrt(disc)
    amplifies the discriminant's error; 16 u (|w| + |s d|) (1 + kappa) covers them."""
    ms = I.make_multi_scene(7, 64, 32)
    rays = I.sample_world_rays(8, 100_000)
    rng = np.random.default_rng(1)
    cen = ms.obj_centre[rng.integers(0, 64, len(rays))]
    q6, met = O.canonical_ray(rays, cen, 2.0)
    p, met64 = O.canonical_ray_f64(rays, cen, 2.0)
    w = rays[:, :3].astype(np.float64) - cen
    d = rays[:, 3:].astype(np.float64)
    b, dd, ww = (w * d).sum(1), (d * d).sum(1), (w * w).sum(1)
    disc = b * b - dd * (ww - 4.0)
    # the two may disagree only within rounding of tangency
    diff = met != met64
    assert np.all(np.abs(disc[diff]) <= 64 * U * dd[diff] * ww[diff])
    m = met & met64
    assert m.sum() > 1000
    s = np.maximum((-b - np.sqrt(np.maximum(disc, 0.0))) / dd, 0.0)
    kappa = np.abs(b) / np.sqrt(np.maximum(disc, 1e-300))
    bound = 16 * U * (np.linalg.norm(w, axis=1) + s * np.sqrt(dd)) * (1.0 + kappa)
    err = np.abs(q6[:, :3].astype(np.float64) - p).max(axis=1)
    assert np.all(err[m] <= bound[m])
    # directions are passed through unchanged
    assert np.array_equal(q6[m, 3:], rays[m, 3:])


def test_entry_point_invariants():
    """The FP64 root is the entry point: on the sphere |p| = R, on the ray (p - w parallel
    to d with s >= 0), and entering (p . d <= 0) for origins outside the ball; the FP32
    sequence satisfies the same to rounding."""
    ms = I.make_multi_scene(9, 16, 32)
    rays = I.sample_world_rays(10, 20_000)
    rng = np.random.default_rng(2)
    cen = ms.obj_centre[rng.integers(0, 16, len(rays))]
    p, met = O.canonical_ray_f64(rays, cen, 2.0)
    q6, met32 = O.canonical_ray(rays, cen, 2.0)
    w = rays[:, :3].astype(np.float64) - cen
    d = rays[:, 3:].astype(np.float64)
    m = met & met32
    assert m.sum() > 100
    assert np.all(np.abs(np.linalg.norm(p[m], axis=1) - 2.0) < 1e-12)
    v = p[m] - w[m]
    cross = np.cross(v, d[m])
    assert np.all(np.linalg.norm(cross, axis=1) <= 1e-12 * (1 + np.linalg.norm(w[m], axis=1)))
    assert np.all((v * d[m]).sum(1) >= -1e-12)
    assert np.all((p[m] * d[m]).sum(1) <= 1e-9)
    # FP32: on the sphere to a few units of |w| u
    r32 = np.linalg.norm(q6[m, :3].astype(np.float64), axis=1)
    assert np.all(np.abs(r32 - 2.0) <= 1e-4)
