"""GPU query sampler (nb_sample) against the oracle's sampler: bit-exact on every
encoding, at ragged sizes, at offsets into the stream, on a coarser grid and at
large query indices."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

KINDS = range(6)


@pytest.fixture(scope="module")
def nb():
    from paper_2310_06822_gb300 import nb as _nb
    _nb.lib()
    return _nb


@pytest.mark.parametrize("kind", KINDS)
def test_sampler_bit_exact(nb, kind):
    n = 300_001
    got = nb.sample(kind, n, seed=77).cpu().numpy()
    ref = O.sample(kind, n, seed=77)
    assert got.shape == ref.shape
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n,first", [(1, 0), (255, 3), (257, 1000), (4099, 2 ** 40 + 17)])
def test_sampler_ranges(nb, kind, n, first):
    got = nb.sample(kind, n, seed=2 ** 63 + 5, first=first).cpu().numpy()
    ref = O.sample(kind, n, seed=2 ** 63 + 5, first=first)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_sampler_split_calls_and_coarse_grid(nb):
    import torch
    out = torch.full((10_000, 6), float("nan"), device="cuda")
    nb.sample(3, 3_333, seed=9, first=0, out=out[:3_333])
    nb.sample(3, 6_667, seed=9, first=3_333, out=out[3_333:])
    assert np.array_equal(out.cpu().numpy(), nb.sample(3, 10_000, seed=9).cpu().numpy())
    for kind in KINDS:
        got = nb.sample(kind, 20_000, seed=4, qexp=18).cpu().numpy()
        assert np.array_equal(got.view(np.uint32), O.sample(kind, 20_000, seed=4, qexp=18).view(np.uint32))


def test_sampler_rejects_bad_arguments(nb):
    import torch
    out = torch.empty((4, 3), device="cuda")
    with pytest.raises(nb.NBError):
        nb.sample(1, 4, seed=1, qexp=21, out=out)
    with pytest.raises(nb.NBError):
        nb.sample(9, 4, seed=1, out=out)
    nb.sample(1, 0, seed=1, out=out)  # empty range: nothing to do


def test_fresh_batches_train_like_the_pool(nb):
    """Sampling, labelling and a training step per iteration on fresh GPU batches:
    one step's gradient equals the oracle's on the same sampled batch."""
    from paper_2310_06822_gb300 import inputs as I
    widths = [6, 32, 32, 1]
    sc = I.make_scene(5, 16, 3, 0.05, 0.3)
    shape = nb.Shape(sc)
    q = nb.sample(3, 4096, seed=123, first=8192)
    bits = nb.label(shape, 3, q)
    m = nb.Model(widths)
    p0 = I.init_params(7, widths)
    m.set_params(p0)
    m.train_step(q, bits, 3.0, 1.0)
    qh = O.sample(3, 4096, seed=123, first=8192)
    y = O.label(3, qh, sc)
    assert np.array_equal(nb.bits_to_numpy(bits, 4096), y.astype(bool))
    _, g = O.loss_grad(widths, p0, qh, y, 3.0, 1.0)
    gg = m.get_grad().astype(np.float64)
    assert np.linalg.norm(gg - g) <= 1e-4 * np.linalg.norm(g)


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4, 5])
def test_paper_encoding_equals_oracle(nb, kind):
    """nb_encode_paper against the oracle's FP64 conversion: box corners exact, plane
    points within a few FP32 roundings, rays and points copied."""
    from oracle import oracle as O
    n = 20_001
    q = nb.sample(kind, n, seed=41)
    e = nb.encode_paper(kind, q).cpu().numpy().astype(np.float64)
    ref = O.paper_encoding(kind, q.cpu().numpy())
    assert e.shape == ref.shape
    if kind == 4:
        np.testing.assert_allclose(e, ref, rtol=0, atol=1e-6)  # about 7 FP32 roundings of values <= 1
        assert np.array_equal(e[:, 3:], ref[:, 3:])
    else:
        assert np.array_equal(e, ref)
    assert nb.encode_paper(kind, q[:0]).shape[0] == 0
