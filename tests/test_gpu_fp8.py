"""FP8 (E4M3) tcgen05 forward (NB_FP8) against the FP64 oracle: logits of networks at
their initial scale within 2e-2 absolute, the error of larger-scale networks stated as a
fraction of the last layer's scale, decisions bit-exact once the margin covers that error
(the band re-checked in FP32 / float-float), ragged sizes, both hidden widths, box and
plane encodings."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_06822_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NETS = [("box3", [6, 256, 256, 256, 256, 1]), ("plane3", [4, 256, 256, 256, 256, 1]),
        ("ray3", [6, 128, 128, 128, 128, 1]), ("point3", [3, 128, 128, 128, 1])]


@pytest.fixture(scope="module")
def nb():
    from paper_2310_06822_gb300 import nb as _nb
    _nb.lib()
    return _nb


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


@pytest.mark.parametrize("kind,widths", NETS)
@pytest.mark.parametrize("n", [1, 127, 129, 200_003])
def test_fp8_logits_at_initial_scale(nb, kind, widths, n):
    p = I.init_params(80 + n % 5, widths)
    m = nb.Model(widths, infer_prec="fp8")
    m.set_params(p)
    q = I.sample_queries(kind, 90 + n, n)
    z64 = O.forward(widths, p, q)
    m.tau = 0.0
    bits, z, st = m.query(_dev(q), margin=0.05, logits=True, stats=True)
    z = z.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(z))
    assert np.max(np.abs(z - z64)) <= 2e-2
    dec = nb.bits_to_numpy(bits, n)
    assert np.array_equal(dec, z64 >= 0.0)
    assert st["n_unresolved"] == 0


@pytest.mark.parametrize("kind,widths", NETS)
def test_fp8_decisions_exact_with_a_covering_margin(nb, kind, widths):
    n = 300_001
    # weights scaled up so logits span tens of units, like trained networks
    p = (I.init_params(91, widths) * 3.0).astype(np.float32)
    m = nb.Model(widths, infer_prec="fp8")
    m.set_params(p)
    q = I.sample_queries(kind, 92, n)
    z64 = O.forward(widths, p, q)
    S = O.forward_scale(widths, p, q)
    qd = _dev(q)
    _, z = m.query(qd, logits=True)
    err = np.abs(z.cpu().numpy().astype(np.float64) - z64)
    # E4M3 keeps 3 mantissa bits: the logit error is a few per cent of the last layer's scale
    assert np.max(err / S) <= 0.08
    tau = float(np.quantile(z64, 0.4))
    m.tau = tau
    margin = 2.0 * float(err.max()) + 0.05
    bits, st = m.query(qd, margin=margin, stats=True)
    dec = nb.bits_to_numpy(bits, n)
    tie = np.abs(z64 - tau) <= 1e-12 * max(1.0, abs(tau))
    assert np.array_equal(dec[~tie], (z64 >= tau)[~tie])
    assert st["n_unresolved"] <= int(tie.sum())
    assert st["n_flagged"] > 0


def test_fp8_flags_non_finite_rows(nb):
    import torch
    widths = [6, 256, 256, 256, 256, 1]
    m = nb.Model(widths, infer_prec="fp8")
    m.set_params(I.init_params(93, widths))
    m.tau = 0.0
    q = I.sample_queries("box3", 94, 1000)
    q[5, 2] = np.inf
    q[700, 0] = np.nan
    bits, st = m.query(_dev(q), margin=0.0, stats=True)
    assert st["n_nonfinite"] == 2
    dec = nb.bits_to_numpy(bits, 1000)
    assert dec[5] and dec[700]  # non-finite input: inside (conservative)


def test_fp8_equals_fp32_form_on_trained_network(nb):
    """A 6->128x4->1 ray network after 300 training steps: FP8 decisions with a margin
    covering the measured error equal the FP32 form's, both certified by the re-check."""
    import torch
    widths = [6, 128, 128, 128, 128, 1]
    sc = I.make_scene(95, 32, 3, 0.02, 0.2)
    shape = nb.Shape(sc)
    t = nb.Model(widths)
    t.set_params(I.init_params(96, widths))
    for s in range(300):
        qb = nb.sample(3, 8192, seed=97, first=s * 8192)
        t.train_step(qb, nb.label(shape, 3, qb), 1.0 + 99.0 * s / 299)
    p = t.get_params()
    n = 1 << 20
    qd = nb.sample(3, n, seed=98)
    f8 = nb.Model(widths, infer_prec="fp8")
    f8.set_params(p)
    f32 = nb.Model(widths)
    f32.set_params(p)
    _, z8 = f8.query(qd, logits=True)
    _, z32 = f32.query(qd, logits=True)
    err = float((z8 - z32).abs().max().item())
    tau = f32.calibrate(qd, nb.label(shape, 3, qd))
    f8.tau = tau
    margin = 2.0 * err + 0.05
    assert torch.equal(f8.query(qd, margin=margin), f32.query(qd, margin=1e-2))
