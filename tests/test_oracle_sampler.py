"""Pins of the oracle's counter-based query sampler (Alg. 1's per-iteration Uniform
draw): the Philox4x64-10 block function against numpy's implementation of the same
published generator, and every encoding against the distribution it must follow
(uniform coordinates, uniform directions on S^2 by Archimedes' theorem, log-uniform
half-extents), exactly on the grid."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O

POINT2, POINT3, POINT4T, RAY3, PLANE3, BOX3 = range(6)
N = 200_000
Q = 2.0 ** -20


def _on_grid(x, qexp=20):
    s = np.ldexp(x.astype(np.float64), qexp)
    return np.all(s == np.round(s))


def _ks_uniform(x, lo, hi):
    return stats.kstest(x, stats.uniform(loc=lo, scale=hi - lo).cdf).pvalue


@pytest.mark.parametrize("case", range(6))
def test_philox_block_equals_numpy_generator(case):
    rng = np.random.default_rng(100 + case)
    ctr = rng.integers(1, 2 ** 63, size=4, dtype=np.uint64)
    key = rng.integers(0, 2 ** 63, size=2, dtype=np.uint64)
    if case == 0:
        ctr[:] = [1, 0, 0, 0]
        key[:] = [0, 0]
    # numpy's Philox advances its 256-bit counter before each block
    prev = ctr.copy()
    prev[0] -= np.uint64(1)
    ref = np.random.Philox(key=[int(key[0]), int(key[1])], counter=[int(c) for c in prev]).random_raw(4)
    assert np.array_equal(O.philox4x64(ctr, key), np.asarray(ref, dtype=np.uint64))


def test_stream_is_a_function_of_the_query_index():
    a = O.sample(RAY3, 1000, seed=5)
    b = O.sample(RAY3, 300, seed=5, first=700)
    assert np.array_equal(a[700:], b)
    assert np.array_equal(O.sample(BOX3, 5000, seed=9, nthreads=1), O.sample(BOX3, 5000, seed=9, nthreads=7))
    assert not np.array_equal(O.sample(POINT3, 100, seed=5), O.sample(POINT3, 100, seed=6))
    # the kind is part of the key: point and plane streams of one seed differ
    assert not np.array_equal(O.sample(POINT3, 100, seed=5)[:, 0], O.sample(PLANE3, 100, seed=5)[:, 3])


@pytest.mark.parametrize("kind", [POINT2, POINT3, POINT4T])
def test_points_uniform_on_the_grid(kind):
    q = O.sample(kind, N, seed=11)
    assert _on_grid(q)
    d = 2 if kind == POINT2 else 3
    for j in range(d):
        assert q[:, j].min() >= -1.0 and q[:, j].max() < 1.0
        assert _ks_uniform(q[:, j], -1.0, 1.0) > 1e-3
    c = np.corrcoef(q[:, :d].T)
    assert np.all(np.abs(c[np.triu_indices(d, 1)]) < 0.01)
    if kind == POINT4T:
        t = q[:, 3]
        assert t.min() >= 0.0 and t.max() < 1.0
        assert _ks_uniform(t, 0.0, 1.0) > 1e-3
        assert abs(np.corrcoef(t, q[:, 0])[0, 1]) < 0.01


def _check_directions(u, radius):
    r = np.linalg.norm(u.astype(np.float64), axis=1)
    # each component is within half a grid step, plus the FP32 normalisation error
    # (square root and division, at most 1.5 ulp of a value below 1), of the exact point
    assert np.all(np.abs(r - radius) <= math.sqrt(3) * radius * (Q / 2 + 1.5 * 2.0 ** -24))
    v = u.astype(np.float64) / radius
    # Archimedes: every coordinate of a uniform point on S^2 is uniform on [-1, 1]
    for j in range(3):
        assert _ks_uniform(v[:, j], -1.0, 1.0) > 1e-3
    assert _ks_uniform(np.arctan2(v[:, 1], v[:, 0]), -math.pi, math.pi) > 1e-3
    assert _ks_uniform(np.arctan2(v[:, 2], v[:, 0]), -math.pi, math.pi) > 1e-3


def test_rays_start_on_the_radius_two_sphere_with_uniform_directions():
    q = O.sample(RAY3, N, seed=13)
    assert _on_grid(q)
    _check_directions(q[:, :3], 2.0)
    _check_directions(q[:, 3:], 1.0)
    # origin and direction are independent
    assert abs(np.corrcoef(q[:, 2], q[:, 5])[0, 1]) < 0.01


def test_planes_have_uniform_normals_and_offsets():
    q = O.sample(PLANE3, N, seed=17)
    assert _on_grid(q)
    _check_directions(q[:, :3], 1.0)
    assert _ks_uniform(q[:, 3], -1.0, 1.0) > 1e-3


def test_box_half_extents_are_log_uniform():
    q = O.sample(BOX3, N, seed=19)
    assert _on_grid(q)
    for j in range(3):
        assert _ks_uniform(q[:, j], -1.0, 1.0) > 1e-3
        e = q[:, 3 + j].astype(np.float64)
        assert e.min() >= 0.01 - Q / 2 and e.max() <= 0.5 + Q / 2
        assert _ks_uniform(np.log(e), math.log(0.01), math.log(0.5)) > 1e-3


def test_box_half_extent_transform_against_library_exp2():
    # the half-extent of axis d reads the top 24 bits of word 1+d of block (i, 0, 0, 0)
    # under key (seed, kind); against numpy's Philox and a float64 exp2 the FP32 value is
    # within half a grid step plus the FP32 error (the rounding of x log2(50), up to
    # 2^-24 * 5.7 in the exponent, dominates: below 5e-7 relative), and on the same grid
    # point except where the exact value lies within that error of a rounding boundary
    seed, n = 23, 2000
    q = O.sample(BOX3, n, seed=seed)
    agree = 0
    for i in range(n):
        prev = [i - 1, 0, 0, 0] if i > 0 else [2 ** 64 - 1, 2 ** 64 - 1, 2 ** 64 - 1, 2 ** 64 - 1]
        w = np.random.Philox(key=[seed, BOX3], counter=prev).random_raw(4)
        for d in range(3):
            x = float(int(w[1 + d]) >> 40) * 2.0 ** -24
            e = 0.01 * np.exp2(x * math.log2(50.0))
            ref = np.rint(e / Q) * Q
            got = float(q[i, 3 + d])
            assert abs(got - e) <= Q / 2 + 5e-7 * e
            agree += got == ref
    assert agree >= 0.97 * 3 * n


def test_coarser_grid():
    q = O.sample(RAY3, 10_000, seed=29, qexp=18)
    assert _on_grid(q, 18)
    q = O.sample(POINT4T, 10_000, seed=29, qexp=18)
    assert _on_grid(q, 18) and q[:, :3].min() >= -1.0 and q[:, :3].max() < 1.0
    with pytest.raises(ValueError):
        O.sample(POINT3, 10, seed=1, qexp=21)
