"""The cascade's spatial index, host side: the 4-wide tree of object boxes that
nb_cascade_index_create builds (linear builder of the paper's BVH baseline, Sec. 4.1:
Morton order, median splits).  Structure invariants, the Morton order of the leaves, and
that walking the tree with the stage-1 slab test in float32 finds exactly the pairs of
the test against every box (the slab test is monotone under box inclusion).

Runs on CPU only (the builder is host code in the library)."""
import math

import numpy as np
import pytest

from paper_2310_06822_gb300 import inputs as I


@pytest.fixture(scope="module")
def nb():
    from paper_2310_06822_gb300 import nb as _nb
    _nb.lib()
    return _nb


def _leaves(nodes, i=0):
    """object ids in child-slot depth-first order"""
    out = []
    for c in range(4):
        ch = int(nodes[i]["child"][c])
        if ch == -2 ** 31:
            continue
        out += [-1 - ch] if ch < 0 else _leaves(nodes, ch)
    return out


def _subtree_box(nodes, aabb, i):
    ks = _leaves(nodes, i)
    return aabb[ks, :3].min(axis=0), aabb[ks, 3:].max(axis=0)


def _morton(aabb):
    c = 0.5 * (aabb[:, :3].astype(np.float64) + aabb[:, 3:].astype(np.float64))
    mn, mx = c.min(axis=0), c.max(axis=0)
    span = np.where(mx > mn, mx - mn, 1.0)
    q = np.clip(np.floor((c - mn) / span * 1024.0), 0, 1023).astype(np.int64)
    q = np.where(mx > mn, q, 0)
    code = np.zeros(len(c), dtype=np.int64)
    for bit in range(10):
        for axis in range(3):
            code |= ((q[:, axis] >> bit) & 1) << (3 * bit + 2 - axis)
    return code


def _boxes(K, seed):
    if K >= 8:
        return I.make_multi_scene(seed, K, 4).aabb.astype(np.float32)
    rng = np.random.default_rng(seed)
    lo = rng.uniform(-5, 5, size=(K, 3))
    return np.concatenate([lo, lo + rng.uniform(0.1, 3, size=(K, 3))], axis=1).astype(np.float32)


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5, 6, 17, 100, 1024, 4096])
def test_tree_structure(nb, K):
    aabb = _boxes(K, 40 + K)
    nodes, depth = nb.bvh4_build_host(aabb)
    assert len(nodes) <= max(1, K - 1)
    # every object exactly once, in Morton order of its box centre (ties by index)
    leaves = _leaves(nodes)
    assert sorted(leaves) == list(range(K))
    code = _morton(aabb)
    assert leaves == sorted(range(K), key=lambda k: (code[k], k))
    # each child box is the exact union of the object boxes below it; unused slots are empty
    for i in range(len(nodes)):
        used = 0
        for c in range(4):
            ch = int(nodes[i]["child"][c])
            if ch == -2 ** 31:
                assert np.all(nodes[i]["lo"][:, c] == 0) and np.all(nodes[i]["hi"][:, c] == 0)
                continue
            used += 1
            if ch < 0:
                lo, hi = aabb[-1 - ch, :3], aabb[-1 - ch, 3:]
            else:
                assert ch > i
                lo, hi = _subtree_box(nodes, aabb, ch)
            assert np.array_equal(nodes[i]["lo"][:, c], lo) and np.array_equal(nodes[i]["hi"][:, c], hi)
        assert used >= min(K, 2)
    # median splits four ways: depth ceil(log4 K) + at most one level
    assert depth <= max(1, math.ceil(math.log(K, 4)) + 1) if K > 1 else depth == 1


def _slab(o, d, inv, lo, hi):
    """stage 1's float32 slab test, vectorised over rays: same operations, same order"""
    f32 = np.float32
    t0 = np.zeros(len(o), dtype=f32)
    t1 = np.full(len(o), np.inf, dtype=f32)
    hit = np.ones(len(o), dtype=bool)
    with np.errstate(all="ignore"):
        for i in range(3):
            zero = d[:, i] == 0
            inside = (o[:, i] >= lo[i]) & (o[:, i] <= hi[i])
            ta = (f32(lo[i]) - o[:, i]) * inv[:, i]
            tb = (f32(hi[i]) - o[:, i]) * inv[:, i]
            sw = ta > tb
            ta, tb = np.where(sw, tb, ta), np.where(sw, ta, tb)
            hit &= np.where(zero, inside, True)
            t0 = np.where(zero, t0, np.fmax(t0, ta))
            t1 = np.where(zero, t1, np.fmin(t1, tb))
    return hit & (t0 <= t1)


def _walk(nodes, o, d, inv, i, rows, out):
    for c in range(4):
        ch = int(nodes[i]["child"][c])
        if ch == -2 ** 31 or len(rows) == 0:
            continue
        h = _slab(o[rows], d[rows], inv[rows], nodes[i]["lo"][:, c], nodes[i]["hi"][:, c])
        sub = rows[h]
        if ch < 0:
            out[-1 - ch] = sub
        else:
            _walk(nodes, o, d, inv, ch, sub, out)


def _rays(seed, n, aabb):
    r = I.sample_world_rays(seed, n).astype(np.float32)
    rng = np.random.default_rng(seed + 1)
    m = n // 8
    # axis-parallel directions (zero components) from origins on box faces and corners
    k = rng.integers(0, len(aabb), m)
    face = np.where(rng.random((m, 3)) < 0.5, aabb[k, :3], aabb[k, 3:])
    r[:m, :3] = np.where(rng.random((m, 3)) < 0.5, face, r[:m, :3])
    r[:m, 3:] = 0
    r[np.arange(m), 3 + rng.integers(0, 3, m)] = rng.choice([-1.0, 1.0], m)
    # origins inside boxes
    r[m:2 * m, :3] = 0.5 * (aabb[k, :3] + aabb[k, 3:])
    return r


@pytest.mark.parametrize("K", [1, 5, 64, 1024])
def test_walk_finds_exactly_the_pairs_of_every_box(nb, K):
    aabb = _boxes(K, 70 + K)
    nodes, _ = nb.bvh4_build_host(aabb)
    r = _rays(71 + K, 4000, aabb)
    o, d = r[:, :3], r[:, 3:]
    with np.errstate(divide="ignore"):
        inv = np.float32(1.0) / d
    brute = [np.nonzero(_slab(o, d, inv, aabb[k, :3], aabb[k, 3:]))[0] for k in range(K)]
    found = {}
    _walk(nodes, o, d, inv, 0, np.arange(len(r)), found)
    for k in range(K):
        assert np.array_equal(np.sort(found.get(k, np.array([], dtype=np.int64))), brute[k]), k
    assert sum(len(b) for b in brute) > 0


def test_builder_rejects_bad_input(nb):
    with pytest.raises(nb.NBError):
        nb.bvh4_build_host(np.zeros((0, 6), dtype=np.float32))
    bad = _boxes(5, 3)
    bad[2, 1] = np.nan
    with pytest.raises(nb.NBError):
        nb.bvh4_build_host(bad)
