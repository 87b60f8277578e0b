"""nb_label (exact labeler) against the oracle: bit-exact on every kind, ragged sizes,
tangency cases, invalid inputs, and sampled checks at full evaluation size."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_06822_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    import torch  # noqa: F401
    from paper_2310_06822_gb300 import nb as _nb
    _nb.lib()
    return _nb


def _gpu_labels(nb, scene, kind, q):
    import torch
    sh = nb.Shape(scene)
    qt = torch.as_tensor(q, device="cuda")
    bits, st = nb.label(sh, kind, qt, stats=True)
    torch.cuda.synchronize()
    return nb.bits_to_numpy(bits, q.shape[0]), st, bits


CASES = [
    (I.POINT2, 8, 0.05, 0.3), (I.POINT3, 64, 0.02, 0.2), (I.POINT4T, 48, 0.02, 0.2),
    (I.RAY3, 64, 0.02, 0.2), (I.PLANE3, 256, 0.02, 0.2), (I.BOX3, 256, 0.02, 0.2),
]


@pytest.mark.parametrize("kind,S,rlo,rhi", CASES)
@pytest.mark.parametrize("n", [1, 31, 33, 1000, 100_003])
def test_labels_bit_exact(nb, kind, S, rlo, rhi, n):
    dim = 2 if kind == I.POINT2 else 3
    sc = I.make_scene(10 + kind, S, dim, rlo, rhi, moving=(kind == I.POINT4T))
    q = I.sample_queries(kind, 20 + kind + n, n)
    y = O.label(kind, q, sc)
    g, st, bits = _gpu_labels(nb, sc, kind, q)
    assert np.array_equal(g, y.astype(bool))
    assert st["n_positive"] == int(y.sum()) and st["n_invalid"] == 0
    # bits past n in the last word are zero
    w = bits.cpu().numpy().view(np.uint32)
    if n % 32:
        assert (int(w[-1]) >> (n % 32)) == 0


def test_tangency_and_degenerate_cases(nb):
    Q = 2.0 ** -20
    g = lambda x: I.quantize(x, 20)
    sc = I.Scene(g([[0.0, 0.0, 0.0]]), g([0.5]), None, 20)
    rays = g([[-2.0, 0.5, 0.0, 1.0, 0.0, 0.0], [-2.0, 0.5 + Q, 0.0, 1.0, 0.0, 0.0], [2.0, 0.0, 0.0, 1.0, 0.0, 0.0],
              [0.25, 0.0, 0.0, 1.0, 0.0, 0.0], [0.5, 0, 0, 1, 0, 0], [-2.0, 0, 0, 0, 0, 0], [-2.0, 0.3, 0, 3.0, 0, 0]])
    assert _gpu_labels(nb, sc, I.RAY3, rays)[0].tolist() == O.label(I.RAY3, rays, sc).astype(bool).tolist()
    planes = g([[0, 0, 1, 0.5], [0, 0, 1, 0.5 + Q], [0.6, 0.8, 0, 0.5], [0.6, 0.8, 0, 0.5 + Q], [0, 0, 0, 0],
                [0, 0, 0, 0.25]])
    assert _gpu_labels(nb, sc, I.PLANE3, planes)[0].tolist() == O.label(I.PLANE3, planes, sc).astype(bool).tolist()
    sc2 = I.Scene(g([[0.0, 0.0, 0.0]]), g([5 / 16]), None, 20)
    e = 0.25
    boxes = g([[3 / 16 + e, 4 / 16 + e, e, e, e, e], [3 / 16 + e + Q, 4 / 16 + e, e, e, e, e],
               [0, 0, 0, 0, 0, 0], [0.9, 0.9, 0.9, 0.01, 0.01, 0.01]])
    assert _gpu_labels(nb, sc2, I.BOX3, boxes)[0].tolist() == [True, False, True, False]
    sc4 = I.Scene(g([[0.0, 0.0, 0.0]]), g([0.25]), g([[0.5, 0.0, 0.0]]), 20)
    pts = g([[0.5, 0, 0, 1.0], [0.5, 0, 0, 0.0], [0.75, 0, 0, 1.0], [0.75 + Q, 0, 0, 1.0]])
    assert _gpu_labels(nb, sc4, I.POINT4T, pts)[0].tolist() == [True, False, True, False]


def test_invalid_queries_are_conservative_and_counted(nb):
    sc = I.make_scene(5, 8, 3, 0.05, 0.2)
    q = I.sample_queries(I.POINT3, 6, 100)
    q[3, 0] = np.nan
    q[7, 1] = np.float32(1e-9)       # off the grid
    q[9, 2] = np.float32(1e6)        # out of range
    g, st, _ = _gpu_labels(nb, sc, I.POINT3, q)
    assert g[3] and g[7] and g[9]
    assert st["n_invalid"] == 3
    ok = np.ones(100, bool)
    ok[[3, 7, 9]] = False
    assert np.array_equal(g[ok], O.label(I.POINT3, q[ok], sc).astype(bool))


@pytest.mark.parametrize("kind,S,n", [(I.RAY3, 64, 16 << 20), (I.BOX3, 256, 64 << 20)])
def test_full_size_sampled(nb, kind, S, n):
    """Full evaluation sizes: every query labelled on the GPU, a seeded sample
    checked against the oracle, and the positive count checked against the
    sample's rate."""
    import torch
    sc = I.make_scene(1000 + kind, S, 3, 0.02, 0.2)
    q = I.sample_queries(kind, 2000 + kind, n)
    g, st, _ = _gpu_labels(nb, sc, kind, q)
    assert st["n_invalid"] == 0
    idx = np.random.default_rng(0).choice(n, size=20000, replace=False)
    idx = np.concatenate([idx, np.arange(n - 37, n)])
    y = O.label(kind, q[idx], sc)
    assert np.array_equal(g[idx], y.astype(bool))
    assert st["n_positive"] == int(g.sum())
    p = y.mean()
    assert abs(g.mean() - p) < 6 * np.sqrt(p * (1 - p) / len(idx)) + 1e-4
    del q
    torch.cuda.empty_cache()
