"""FP8 (E4M3) tcgen05 forward (NB_FP8: two-term E4M3 operands, three products per k-step,
weights streamed through shared memory) against the FP64 oracle: logits of networks at
their initial scale within 2e-2 absolute; on larger-scale and trained networks the error as
a fraction of the last layer's conditioning scale S = sum |W_L| |a_{L-1}| + |b_L| (the
stated bound for two terms: 2^-4 S); decisions bit-exact once the margin covers the error
(the band re-checked in FP32 / float-float), with the margin measured on a calibration
sample and the decisions checked on other queries; ragged sizes, both hidden widths, box
and plane encodings."""
REL_S_FP8 = 2.0 ** -4  # two-term E4M3 logits: |z8 - z64| <= 2^-4 S
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
    # two E4M3 terms keep about 8 bits: the logit error is well below a per cent of the
    # last layer's scale on these well-conditioned networks (one term was up to 8 %)
    assert np.max(err / S) <= 2.0 ** -6
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


def test_fp8_on_a_trained_box_network_against_the_oracle(nb):
    """The box configuration's network shape, 6->256x4->1, after 3,000 BF16 tensor-core
    training steps of 65,536 boxes against a 256-sphere union (logits of hundreds, the
    conditioning that made one E4M3 term miss by tens): FP8 logits within 2^-4 S of the
    FP64 oracle; the margin, 2x the largest FP8 deviation from the FP32 form on a
    calibration sample, sends a small band to the re-check; on other queries the decisions
    equal the oracle's and none is a false negative of the exact labels that the
    calibrated threshold covers."""
    import torch
    widths = [6, 256, 256, 256, 256, 1]
    sc = I.make_scene(120, 256, 3, 0.02, 0.2)
    shape = nb.Shape(sc)
    tr = nb.Model(widths, train_prec="bf16")
    tr.set_params(I.init_params(121, widths))
    T, B = 3000, 65536
    for t in range(T):
        qb = nb.sample(I.BOX3, B, seed=122, first=t * B)
        tr.train_step(qb, nb.label(shape, I.BOX3, qb), 1.0 + 99.0 * t / (T - 1))
    p = tr.get_params()
    f8 = nb.Model(widths, infer_prec="fp8")
    f8.set_params(p)
    f32 = nb.Model(widths)
    f32.set_params(p)
    # logits against the oracle on 100k queries
    qo = O.sample(I.BOX3, 100_000, 123)
    _, z8 = f8.query(_dev(qo), logits=True)
    z64 = O.forward(widths, p, qo)
    S = O.forward_scale(widths, p, qo)
    rel = np.abs(z8.cpu().numpy().astype(np.float64) - z64) / S
    assert rel.max() <= REL_S_FP8, rel.max()
    assert np.abs(z64).max() > 20.0  # a trained scale, not the initial one
    # margin from a calibration sample, threshold calibrated on the evaluation queries
    qc = nb.sample(I.BOX3, 1 << 20, seed=124)
    _, zc8 = f8.query(qc, logits=True)
    _, zc32 = f32.query(qc, logits=True)
    margin = 2.0 * float((zc8 - zc32).abs().max().item()) + 0.05
    n = 1 << 21
    qe = nb.sample(I.BOX3, n, seed=125)
    ye = nb.label(shape, I.BOX3, qe)
    tau = f32.calibrate(qe, ye)
    f8.tau = tau
    bits, st = f8.query(qe, margin=margin, stats=True)
    assert st["n_flagged"] <= 0.1 * n
    assert torch.equal(bits, f32.query(qe, margin=1e-2))
    y = nb.bits_to_numpy(ye, n)
    assert not np.any(y & ~nb.bits_to_numpy(bits, n))
    # and against the oracle itself on a slice of the evaluation queries
    qs = qe[:200_000].cpu().numpy()
    zs = O.forward(widths, p, qs)
    dec = nb.bits_to_numpy(bits, n)[:200_000]
    tie = np.abs(zs - tau) <= 1e-12 * max(1.0, abs(tau))
    assert np.array_equal(dec[~tie], (zs >= tau)[~tie])
