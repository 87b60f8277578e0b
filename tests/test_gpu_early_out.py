"""Neural early-out (Sec. 3.3): a small network trained and calibrated as a conservative
bound of the complement 1 - g runs first; where it decides 0 the answer is inside and the
late network is skipped.  Decisions against the oracle's two networks and thresholds,
FN = 0 on the calibration set, and the share of rows the early network settles."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_06822_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    from paper_2310_06822_gb300 import nb as _nb
    _nb.lib()
    return _nb


def _train(nb, model, shape, kind, steps, batch, seed, invert):
    for t in range(steps):
        q = nb.sample(kind, batch, seed=seed, first=t * batch)
        y = nb.label(shape, kind, q)
        if invert:
            y = nb.bits_not(y, batch)
        model.train_step(q, y, 1.0 + 99.0 * t / max(steps - 1, 1))


@pytest.mark.parametrize("kind,late_prec", [(1, "f16x3"), (3, "f32")])
def test_early_out_decisions_equal_oracle(nb, kind, late_prec):
    w0 = I.ENC_WIDTH[kind]
    # a few large spheres: deep interiors the early network can certify for points
    sc = I.make_scene(70 + kind, 12, 3, 0.3, 0.6)
    shape = nb.Shape(sc)
    early_w, late_w = [w0, 64, 64, 1], [w0, 128, 128, 128, 1]
    early = nb.Model(early_w)
    early.set_params(I.init_params(71, early_w))
    late = nb.Model(late_w, infer_prec=late_prec)
    late.set_params(I.init_params(72, late_w))
    _train(nb, early, shape, kind, 600, 8192, 73, invert=True)
    _train(nb, late, shape, kind, 300, 8192, 74, invert=False)
    n = 200_003
    q = nb.sample(kind, n, seed=75)
    y = nb.label(shape, kind, q)
    tau_e = early.calibrate(q, nb.bits_not(y, n))
    tau_l = late.calibrate(q, y)
    bits, st = nb.query_early_out(early, late, q, margin_early=1e-3, margin_late=0.05)
    dec = nb.bits_to_numpy(bits, n)
    yy = nb.bits_to_numpy(y, n)
    qh = q.cpu().numpy()
    ze = O.forward(early_w, early.get_params(), qh)
    zl = O.forward(late_w, late.get_params(), qh)
    # the early network decides 0 where its exact logit is below its threshold: inside
    expect = np.where(ze < tau_e, True, zl >= tau_l)
    tie = (np.abs(ze - tau_e) <= 1e-12 * max(1.0, abs(tau_e))) | (np.abs(zl - tau_l) <= 1e-12 * max(1.0, abs(tau_l)))
    assert np.array_equal(dec[~tie], expect[~tie])
    assert not np.any(yy & ~dec)  # FN = 0 on the calibration set
    # an early "inside" is never a miss on the calibration set
    assert not np.any((ze < tau_e) & ~yy)
    assert st["n_early_inside"] + st["n_late"] == n
    assert abs(st["n_early_inside"] - int(np.sum(ze < tau_e))) <= int(tie.sum())
    if kind == 1:
        assert st["n_early_inside"] > 0.02 * n, st


def test_bits_not_masks_the_tail(nb):
    import torch
    n = 1000
    b = torch.randint(-2 ** 31, 2 ** 31 - 1, (nb.n_words(n),), dtype=torch.int32, device="cuda")
    nb_ = nb.bits_not(b, n)
    x = nb.bits_to_numpy(b, n)
    assert np.array_equal(nb.bits_to_numpy(nb_, n), ~x)
    assert (nb_.cpu().numpy().view(np.uint32)[-1] >> (n % 32)) == 0
