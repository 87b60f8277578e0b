"""The thread-per-query FP32 forward (networks with input width <= 8 and stored hidden
layers <= 128 wide: the paper's own sizes, Sec. 3.4 "Architecture") against the FP64
oracle; non-finite query coordinates on every precision; and the one-pass early-out stage
for a one-hidden-layer early network (Sec. 3.3), whose settled rows carry a rigorous FP32
error bound."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_06822_gb300 import inputs as I

pytestmark = pytest.mark.gpu

REL_F32 = 1e-5  # FP32 logits: |z32 - z64| <= 1e-5 max(|z64|, S_abs)


@pytest.fixture(scope="module")
def nb():
    from paper_2310_06822_gb300 import nb as _nb
    _nb.lib()
    return _nb


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


# one hidden layer (four queries per thread), odd widths, the widest stored layer, the
# paper's sizes, a network too large for shared memory (tile kernel), and input widths that
# are not the encodings' (random rows of that width)
NETS = [
    ("point3", [3, 64, 1], "relu"),
    ("ray3", [6, 256, 1], "relu"),
    ("point2", [2, 7, 1], "relu"),
    ("point2", [2, 25, 25, 1], "relu"),
    ("point3", [3, 50, 50, 1], "sine"),
    ("point4t", [4, 75, 75, 1], "relu"),
    ("ray3", [6, 33, 97, 5, 1], "relu"),
    ("ray3", [6, 128, 128, 200, 1], "relu"),
    (8, [8, 64, 64, 64, 64, 64, 1], "relu"),
    (5, [5, 30, 1], "sine"),
    (1, [1, 9, 1], "relu"),
    (7, [7, 12, 1], "relu"),
]


def _queries(kind, seed, n):
    if isinstance(kind, int):
        return np.random.default_rng(seed).uniform(-1.0, 1.0, (n, kind)).astype(np.float32)
    return I.sample_queries(kind, seed, n)


@pytest.mark.parametrize("kind,widths,act", NETS)
@pytest.mark.parametrize("n", [1, 31, 4099])
def test_narrow_logits_within_tolerance(nb, kind, widths, act, n):
    m = nb.Model(widths, activation=act)
    p = I.init_params(300 + n, widths)
    m.set_params(p)
    q = _queries(kind, 301 + n, n)
    _, z = m.query(_dev(q), margin=0.0, logits=True)
    z = z.cpu().numpy().astype(np.float64)
    z64 = O.forward(widths, p, q, act=act)
    S = O.forward_scale(widths, p, q, act=act)
    err = np.abs(z - z64) / np.maximum(np.abs(z64), S)
    assert err.max() <= REL_F32, err.max()


@pytest.mark.parametrize("kind,widths,act", NETS)
def test_narrow_decisions_bit_exact_with_recheck(nb, kind, widths, act):
    n = 20011
    m = nb.Model(widths, activation=act)
    p = I.init_params(302, widths)
    m.set_params(p)
    q = _queries(kind, 303, n)
    z64 = O.forward(widths, p, q, act=act)
    for tau, margin in ((0.0, 1e-3), (float(np.median(z64)), 1e-3), (float(np.quantile(z64, 0.3)), 10.0)):
        m.tau = tau
        bits, st = m.query(_dev(q), margin=margin, stats=True)
        dec = nb.bits_to_numpy(bits, n)
        tie = np.abs(z64 - tau) <= 1e-12 * max(1.0, abs(tau))
        assert np.array_equal(dec[~tie], (z64 >= tau)[~tie]), (tau, margin)
        assert np.all(dec[tie])
        assert st["n_unresolved"] <= int(tie.sum())


@pytest.mark.parametrize("widths,prec", [([6, 64, 64, 1], "f32"), ([6, 256, 256, 1], "f32"), ([6, 40, 1], "f32"),
                                         ([6, 128, 128, 128, 128, 1], "f16x3"), ([3, 50, 50, 1], "f16x3"),
                                         ([6, 128, 128, 128, 128, 1], "bf16"),
                                         ([6, 256, 256, 256, 256, 1], "fp8")])
def test_non_finite_coordinates_are_decided_inside(nb, widths, prec):
    """A NaN or infinite coordinate can vanish in a ReLU (max(NaN, 0) = 0, or -inf before
    it); every form must still decide the row inside and count it as non-finite."""
    w0 = widths[0]
    m = nb.Model(widths, infer_prec=prec)
    m.set_params(I.init_params(304, widths))
    n = 1000
    q = np.random.default_rng(305).uniform(-1.0, 1.0, (n, w0)).astype(np.float32)
    bad = [3, 64, 65, 500, 999]
    q[3, 0] = np.nan
    q[64, w0 - 1] = np.inf
    q[65, 1] = -np.inf
    q[500, :] = np.nan
    q[999, 2] = np.inf
    m.tau = 1e30  # every finite row is outside
    bits, st = m.query(_dev(q), margin=0.0, stats=True)
    dec = nb.bits_to_numpy(bits, n)
    assert st["n_nonfinite"] == len(bad)
    assert np.array_equal(np.flatnonzero(dec), bad)


def _train(nb, model, shape, kind, steps, batch, seed, invert):
    for t in range(steps):
        q = nb.sample(kind, batch, seed=seed, first=t * batch)
        y = nb.label(shape, kind, q)
        if invert:
            y = nb.bits_not(y, batch)
        model.train_step(q, y, 1.0 + 99.0 * t / max(steps - 1, 1))


@pytest.mark.parametrize("kind,hidden", [(1, 128), (1, 200), (3, 128)])
def test_one_pass_early_out_against_the_oracle(nb, kind, hidden):
    """The early network w0 -> hidden -> 1 (one hidden layer, ReLU, FP32: the paper's early
    exit) settles a row when its FP32 logit plus a rigorous bound of the rounding error
    (and the margin) is below its threshold.  Settled rows must have an exact early logit
    below the threshold; every other row gets the late network's certified decision."""
    w0 = I.ENC_WIDTH[kind]
    sc = I.make_scene(306 + kind, 12, 3, 0.3, 0.6)
    shape = nb.Shape(sc)
    early_w, late_w = [w0, hidden, 1], [w0, 128, 128, 128, 1]
    early = nb.Model(early_w)
    early.set_params(I.init_params(307, early_w))
    late = nb.Model(late_w, infer_prec="f16x3")
    late.set_params(I.init_params(308, late_w))
    _train(nb, early, shape, kind, 2000, 8192, 309, invert=True)
    _train(nb, late, shape, kind, 300, 8192, 310, invert=False)
    n = 200_003
    q = nb.sample(kind, n, seed=311)
    y = nb.label(shape, kind, q)
    tau_e = early.calibrate(q, nb.bits_not(y, n))
    tau_l = late.calibrate(q, y)
    qh = q.cpu().numpy()
    ze = O.forward(early_w, early.get_params(), qh)
    zl = O.forward(late_w, late.get_params(), qh)
    yy = nb.bits_to_numpy(y, n)
    settled = {}
    for margin_e in (0.0, 1e-3, 0.5):
        bits, st = nb.query_early_out(early, late, q, margin_early=margin_e, margin_late=0.05)
        dec = nb.bits_to_numpy(bits, n)
        assert st["n_early_inside"] + st["n_late"] == n
        # rows below the early threshold by more than the margin and a slack far above the
        # FP32 error settle; rows at or above it never do
        certain = ze < tau_e - margin_e - 4e-3 * max(1.0, abs(tau_e))
        possible = ze < tau_e
        assert int(certain.sum()) <= st["n_early_inside"] <= int(possible.sum()), (
            int(certain.sum()), st, int(possible.sum()), tau_e)
        tie = np.abs(zl - tau_l) <= 1e-12 * max(1.0, abs(tau_l))
        late_dec = zl >= tau_l
        # rows the early network cannot settle get the late network's decision; a row it may
        # settle is inside either way on the calibration set (an early logit below its
        # threshold means g = 1 there, and the calibrated late network says 1 for those)
        assert np.array_equal(dec[~possible & ~tie], late_dec[~possible & ~tie])
        assert np.all(dec[possible])
        assert not np.any(yy & ~dec)  # FN = 0 on the calibration set
        settled[margin_e] = st["n_early_inside"]
    assert settled[0.0] >= settled[1e-3] >= settled[0.5]
    if kind == 1:  # points: the early network settles a share of the rows (the test is not vacuous)
        assert settled[0.0] > 0.01 * n, (settled, int((ze < tau_e).sum()), tau_e)


def test_one_pass_early_out_non_finite_rows_go_to_the_late_network(nb):
    early_w, late_w = [3, 64, 1], [3, 128, 128, 128, 1]
    early = nb.Model(early_w)
    early.set_params(I.init_params(312, early_w))
    late = nb.Model(late_w, infer_prec="f16x3")
    late.set_params(I.init_params(313, late_w))
    n = 5000
    q = I.sample_queries("point3", 314, n)
    q[7, 1] = np.nan
    q[4000, 0] = -np.inf
    early.tau = 1e30  # the early network would settle every finite row
    late.tau = 1e30   # the late network decides every finite row outside
    bits, st = nb.query_early_out(early, late, _dev(q), margin_early=0.0, margin_late=0.0)
    dec = nb.bits_to_numpy(bits, n)
    assert st["n_late"] == 2 and st["n_early_inside"] == n - 2
    assert dec.all()  # settled rows inside; the two non-finite rows inside by the late network


@pytest.mark.parametrize("widths", [[6, 50, 50, 1], [6, 64, 1]])
def test_narrow_full_size_16m_rays(nb, widths):
    """16M rays, the size and launch bench.py times for the paper's 3D-ray network (and a
    one-hidden-layer network): the thread-per-query FP32 form and the split-FP16 tensor-core
    form decide every ray alike (both certified by the re-check); sampled logits of the FP32
    form against the oracle, one by one."""
    import torch
    n = 16 << 20
    q = nb.sample(I.RAY3, n, seed=315)
    p = (I.init_params(316, widths) * 3.0).astype(np.float32)
    f32 = nb.Model(widths)
    f32.set_params(p)
    sp = nb.Model(widths, infer_prec="f16x3")
    sp.set_params(p)
    idx = np.sort(np.random.default_rng(317).choice(n, 20000, replace=False))
    qs = q[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    z64 = O.forward(widths, p, qs)
    S = O.forward_scale(widths, p, qs)
    _, z32 = f32.query(q, logits=True)
    z32s = z32.cpu().numpy()[idx].astype(np.float64)
    assert np.max(np.abs(z32s - z64) / np.maximum(np.abs(z64), S)) <= REL_F32
    del z32
    tau = float(np.quantile(z64, 0.5))
    f32.tau = tau
    sp.tau = tau
    b32, st = f32.query(q, margin=1e-3, stats=True)
    bsp = sp.query(q, margin=0.05)
    assert torch.equal(b32, bsp)
    assert st["n_unresolved"] == 0
    dec = nb.bits_to_numpy(b32, n)[idx]
    tie = np.abs(z64 - tau) <= 1e-12 * max(1.0, abs(tau))
    assert np.array_equal(dec[~tie], (z64 >= tau)[~tie])


@pytest.mark.parametrize("w0,hidden", [(3, 64), (6, 200), (2, 9)])
def test_early_settle_bound_is_sound_row_by_row(nb, w0, hidden):
    """With the late network answering 0 for every finite row, a 1 bit marks a settled row:
    each must have an exact (FP64) early logit below the early threshold, and every row
    below it by more than a small slack must be settled.  The threshold sits on the median
    logit, so half of the rows are within reach of it and many within FP32 rounding."""
    early_w, late_w = [w0, hidden, 1], [w0, 128, 128, 128, 1]
    early = nb.Model(early_w)
    p = (I.init_params(318 + w0, early_w) * 3.0).astype(np.float32)
    early.set_params(p)
    late = nb.Model(late_w, infer_prec="f16x3")
    late.set_params(I.init_params(319, late_w))
    late.tau = 1e30
    n = 300_007
    q = np.random.default_rng(320 + w0).uniform(-1.0, 1.0, (n, w0)).astype(np.float32)
    ze = O.forward(early_w, p, q)
    _, z32 = early.query(_dev(q), logits=True)
    z32 = z32.cpu().numpy()
    # thresholds: the median exact logit, and a float just above an FP32 logit (rows whose
    # FP32 value rounds across it)
    for tau_e in (float(np.median(ze)), float(np.nextafter(np.float32(np.quantile(z32, 0.6)), np.float32(np.inf)))):
        early.tau = tau_e
        for margin in (0.0, 1e-3):
            bits, st = nb.query_early_out(early, late, _dev(q), margin_early=margin, margin_late=0.0)
            settled = nb.bits_to_numpy(bits, n)
            tie = np.abs(ze - tau_e) <= 1e-12 * max(1.0, abs(tau_e))
            assert not np.any(settled & ~tie & (ze >= tau_e)), (tau_e, margin)  # sound
            S = O.forward_scale(early_w, p, q)
            clear = ze < tau_e - margin - 1e-4 * S  # far below the FP32 rounding of the logit
            assert np.all(settled[clear]), (tau_e, margin, int((clear & ~settled).sum()))
            assert st["n_early_inside"] == int(settled.sum())
