"""FP32 network path of libnb against the FP64 oracle: logits, bit-exact decisions
with the boundary re-check, calibration, one training step (loss, gradient, Adam),
checkpoint/resume, and the C1 configuration end to end."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_06822_gb300 import inputs as I

pytestmark = pytest.mark.gpu

REL_F32 = 1e-5  # FP32 logits: |z32 - z64| <= 1e-5 max(|z64|, S_abs)
REL_GRAD = 1e-4  # single-step gradients: ||g - g64|| / ||g64|| per tensor


@pytest.fixture(scope="module")
def nb():
    from paper_2310_06822_gb300 import nb as _nb
    _nb.lib()
    return _nb


def _model(nb, widths, seed, prec="f32"):
    m = nb.Model(widths, infer_prec=prec)
    p = I.init_params(seed, widths)
    m.set_params(p)
    return m, p


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


NETS = [
    ("point2", [2, 32, 32, 32, 1]),
    ("point3", [3, 128, 128, 128, 128, 1]),
    ("ray3", [6, 128, 128, 128, 128, 1]),
    ("box3", [6, 256, 256, 256, 256, 1]),
    ("point4t", [4, 64, 64, 64, 1]),
    ("ray3", [6, 50, 50, 1]),      # the paper's 3D ray network (widths not multiples of 16)
    ("point2", [2, 1]),            # a single layer
]


@pytest.mark.parametrize("kind,widths", NETS)
@pytest.mark.parametrize("n", [1, 33, 4099])
def test_fp32_logits_within_tolerance(nb, kind, widths, n):
    m, p = _model(nb, widths, 7 + n)
    q = I.sample_queries(kind, 8 + n, n)
    bits, z = m.query(_dev(q), margin=0.0, logits=True)
    z = z.cpu().numpy().astype(np.float64)
    z64 = O.forward(widths, p, q)
    S = O.forward_scale(widths, p, q)
    err = np.abs(z - z64) / np.maximum(np.abs(z64), S)
    assert err.max() <= REL_F32, err.max()


@pytest.mark.parametrize("kind,widths", NETS[:5])
def test_decisions_bit_exact_with_recheck(nb, kind, widths):
    n = 20011
    m, p = _model(nb, widths, 3)
    q = I.sample_queries(kind, 4, n)
    z64 = O.forward(widths, p, q)
    for tau in [0.0, float(np.median(z64)), float(np.float32(np.quantile(z64, 0.3)))]:
        m.tau = tau
        bits, st = m.query(_dev(q), margin=1e-3, stats=True)
        dec = nb.bits_to_numpy(bits, n)
        assert np.array_equal(dec, z64 >= tau), tau
        # a query whose logit equals tau to ~1e-12 cannot be settled by any bounded
        # evaluation (tau = the median is one query's own FP64 logit); it is decided
        # inside, which is the conservative side and agrees with z64 >= tau
        near = int(np.sum(np.abs(z64 - tau) <= 1e-12 * max(1.0, abs(tau))))
        assert st["n_unresolved"] <= near
        assert st["n_inside"] == int((z64 >= tau).sum())


def test_recheck_resolves_a_crowded_threshold(nb):
    # put tau exactly on FP32 logits so that many queries sit inside the margin band
    widths = [3, 64, 64, 1]
    m, p = _model(nb, widths, 11)
    q = I.sample_queries("point3", 12, 8192)
    _, z = m.query(_dev(q), logits=True)
    z = z.cpu().numpy()
    m.tau = float(z[100])
    bits, st = m.query(_dev(q), margin=10.0, stats=True)   # every query is re-checked
    z64 = O.forward(widths, p, q)
    assert st["n_flagged"] == 8192
    assert np.array_equal(nb.bits_to_numpy(bits, 8192), z64 >= float(z[100]))
    assert st["n_unresolved"] <= 2


def test_calibration_matches_oracle_and_has_no_fn(nb):
    widths = [6, 64, 64, 1]
    m, p = _model(nb, widths, 21)
    sc = I.make_scene(22, 32, 3, 0.05, 0.3)
    q = I.sample_queries("ray3", 23, 50_000)
    y = O.label(I.RAY3, q, sc)
    labels = _dev(I.pack_bits(y).view(np.int32))
    tau = m.calibrate(_dev(q), labels, eps=1e-5)
    z64 = O.forward(widths, p, q)
    tau_o, npos = O.calibrate(z64, y, 1e-5)
    assert npos == int(y.sum()) > 0
    assert abs(tau - tau_o) <= 1e-12 * max(1.0, abs(tau_o))
    bits = m.query(_dev(q), margin=1e-3)
    dec = nb.bits_to_numpy(bits, len(y))
    assert np.array_equal(dec, z64 >= tau)
    assert not np.any(y.astype(bool) & ~dec), "calibrated bound has a false negative"


def test_calibration_without_positives(nb):
    widths = [3, 16, 1]
    m, _ = _model(nb, widths, 1)
    q = I.sample_queries("point3", 2, 1000)
    labels = _dev(np.zeros(32, dtype=np.int32))
    assert m.calibrate(_dev(q), labels) == float("inf")
    bits = m.query(_dev(q))
    assert not nb.bits_to_numpy(bits, 1000).any()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _per_tensor(widths):
    out, off = [], 0
    for l in range(len(widths) - 1):
        nW = widths[l + 1] * widths[l]
        out.append((off, off + nW))
        out.append((off + nW, off + nW + widths[l + 1]))
        off += nW + widths[l + 1]
    return out


@pytest.mark.parametrize("kind,widths,n", [("point2", [2, 32, 32, 32, 1], 1024),
                                           ("ray3", [6, 128, 128, 128, 128, 1], 4133),
                                           ("box3", [6, 256, 256, 256, 256, 1], 1000),
                                           ("point4t", [4, 64, 64, 64, 1], 777)])
def test_train_step_gradient_loss_adam(nb, kind, widths, n):
    dim = 2 if kind == "point2" else 3
    kid = I.kind_id(kind)
    sc = I.make_scene(30, 16, dim, 0.1, 0.4, moving=(kid == I.POINT4T))
    q = I.sample_queries(kind, 31, n)
    y = O.label(kid, q, sc)
    m, p = _model(nb, widths, 32)
    st = nb.step_stats_tensor()
    alpha, beta = 17.0, 1.0
    m.train_step(_dev(q), _dev(I.pack_bits(y).view(np.int32)), alpha, beta, stats=st)
    g = m.get_grad().astype(np.float64)
    loss64, g64 = O.loss_grad(widths, p, q, y, alpha, beta)
    s = nb.read_step_stats(st)
    assert abs(s["loss"] - loss64) <= 1e-5 * abs(loss64)
    for a, b in _per_tensor(widths):
        assert _rel(g[a:b], g64[a:b]) <= REL_GRAD, (a, b, _rel(g[a:b], g64[a:b]))
    # Adam on the GPU gradient, in FP64, against the GPU's FP32 update
    th = p.astype(np.float64)
    mm, vv = np.zeros_like(th), np.zeros_like(th)
    O.adam(th, mm, vv, g, 1)
    p1 = m.get_params().astype(np.float64)
    assert np.max(np.abs(p1 - th)) <= 1e-6


def test_checkpoint_resume_is_bit_identical(nb):
    widths = [3, 32, 32, 1]
    sc = I.make_scene(40, 16, 3, 0.1, 0.3)
    qs = [I.sample_queries("point3", 41 + i, 512) for i in range(6)]
    ys = [_dev(I.pack_bits(O.label(I.POINT3, x, sc)).view(np.int32)) for x in qs]
    m, _ = _model(nb, widths, 42)
    for i in range(3):
        m.train_step(_dev(qs[i]), ys[i], 5.0)
    state = m.get_state()
    for i in range(3, 6):
        m.train_step(_dev(qs[i]), ys[i], 5.0)
    ref = m.get_params()
    m2 = nb.Model(widths)
    m2.set_state(state)
    for i in range(3, 6):
        m2.train_step(_dev(qs[i]), ys[i], 5.0)
    assert np.array_equal(m2.get_params(), ref)


def test_c1_end_to_end_zero_fn_on_grid(nb):
    """2D point, FP32: 8 disks, 2->32->32->32->1, 1000 Adam steps of 1024 points with
    the FN weight ramped 1 -> 100, calibration, 256x256 grid: FN = 0, decisions equal
    the oracle's."""
    import torch
    widths = [2, 32, 32, 32, 1]
    sc = I.make_scene(1000, 8, 2, 0.05, 0.3)
    shape = nb.Shape(sc)
    m, _ = _model(nb, widths, 1001)
    T = 1000
    pool = _dev(I.sample_queries("point2", 2000, T * 1024))
    labels = nb.label(shape, I.POINT2, pool)
    for t in range(T):
        alpha = 1.0 + 99.0 * t / (T - 1)
        m.train_step(pool[t * 1024:(t + 1) * 1024], labels[t * 32:(t + 1) * 32], alpha, 1.0)
    grid = I.grid_points_2d(256)
    gt = _dev(grid)
    yg = nb.label(shape, I.POINT2, gt)
    yo = O.label(I.POINT2, grid, sc).astype(bool)
    assert np.array_equal(nb.bits_to_numpy(yg, len(grid)), yo)
    tau = m.calibrate(gt, yg)
    bits = m.query(gt, margin=1e-3)
    dec = nb.bits_to_numpy(bits, len(grid))
    p = m.get_params()
    z64 = O.forward(widths, p, grid)
    assert np.array_equal(dec, z64 >= tau)
    assert not np.any(yo & ~dec)
    fp = int(np.sum(dec & ~yo))
    # the trained bound is much tighter than "everything inside"
    assert fp < 0.5 * int((~yo).sum()), fp
    torch.cuda.synchronize()


def test_trained_ray_network_bf16_and_f32_decisions(nb):
    """3D rays, 64 spheres, 6->128x4->1 trained briefly with the asymmetric ramp:
    BF16 logits within 2e-2 of the oracle, and decisions of both the BF16 and the
    FP32 forms equal to the oracle's after calibration (FN = 0)."""
    import torch
    widths = [6, 128, 128, 128, 128, 1]
    sc = I.make_scene(1001, 64, 3, 0.02, 0.2)
    shape = nb.Shape(sc)
    trainer, _ = _model(nb, widths, 4001)
    T, B = 400, 65536
    pool = _dev(I.sample_queries("ray3", 2018, T * B // 4))
    bits = nb.label(shape, I.RAY3, pool)
    per = pool.shape[0] // B
    for t in range(T):
        j = t % per
        trainer.train_step(pool[j * B:(j + 1) * B], bits[j * B // 32:(j + 1) * B // 32], 1.0 + 99.0 * t / (T - 1), 1.0)
    p = trainer.get_params()
    n = 200_003
    q = I.sample_queries("ray3", 2019, n)
    qd = _dev(q)
    y = O.label(I.RAY3, q, sc).astype(bool)
    yd = nb.label(shape, I.RAY3, qd)
    mb = nb.Model(widths, infer_prec="f16x3")
    mb.set_params(p)
    tau = mb.calibrate(qd, yd)
    z64 = O.forward(widths, p, q)
    bits_b, zb, st = mb.query(qd, margin=0.05, logits=True, stats=True)
    err = np.abs(zb.cpu().numpy().astype(np.float64) - z64)
    assert err.max() <= 2e-2, err.max()
    truth = z64 >= tau
    tie = np.abs(z64 - tau) <= 1e-12 * max(1.0, abs(tau))
    db = nb.bits_to_numpy(bits_b, n)
    assert np.array_equal(db[~tie], truth[~tie])
    assert not np.any(y & ~db)
    assert st["n_unresolved"] <= int(tie.sum())
    # plain single-product BF16: decisions exact with a margin above its measured error
    m16 = nb.Model(widths, infer_prec="bf16")
    m16.set_params(p)
    m16.tau = tau
    _, z16 = m16.query(qd, logits=True)
    e16 = float(np.max(np.abs(z16.cpu().numpy().astype(np.float64) - z64)))
    d16 = nb.bits_to_numpy(m16.query(qd, margin=4 * e16 + 1e-3), n)
    assert np.array_equal(d16[~tie], truth[~tie])
    mf = nb.Model(widths)
    mf.set_params(p)
    mf.tau = tau
    _, zf = mf.query(qd, logits=True)
    S = O.forward_scale(widths, p, q)
    ef = np.abs(zf.cpu().numpy().astype(np.float64) - z64) / np.maximum(np.abs(z64), S)
    assert ef.max() <= 1e-5
    # the FP32 form needs a margin above its own logit error
    m32 = float(4 * np.max(np.abs(zf.cpu().numpy().astype(np.float64) - z64))) + 1e-6
    df = nb.bits_to_numpy(mf.query(qd, margin=max(m32, 1e-3)), n)
    assert np.array_equal(df[~tie], truth[~tie])
    torch.cuda.synchronize()


def test_stepwise_schedule_training_reaches_zero_fn_windows(nb):
    """2D points, the paper's 2->25->25->1 network trained in FP32 under the stepwise
    schedule (windows of 100 steps, 2D rates): the weights grow more asymmetric while the
    training batches show false negatives, and training stops after three clean windows."""
    import torch
    widths = [2, 25, 25, 1]
    sc = I.make_scene(1100, 8, 2, 0.05, 0.3)
    shape = nb.Shape(sc)
    m, _ = _model(nb, widths, 1101)
    s = nb.Stepwise(dim=2, period=100, stop_windows=3)
    st = nb.step_stats_tensor()
    fns, stopped, B = [], False, 1024
    for t in range(6000):
        q = nb.sample(I.POINT2, B, seed=1102, first=t * B)
        m.train_step(q, nb.label(shape, I.POINT2, q), s.alpha, s.beta, stats=st)
        if (t + 1) % s.period == 0:
            fn = nb.read_step_stats(st)["fn"]
            st.zero_()
            fns.append(fn)
            if s.window(fn):
                stopped = True
                break
    assert s.adjustments >= 1 and fns[0] > 0
    assert stopped or s.adjustments >= 3, fns
    if stopped:
        assert fns[-3:] == [0, 0, 0]
    # the calibrated bound has no false negative on its calibration set
    grid = _dev(I.grid_points_2d(256))
    yg = nb.label(shape, I.POINT2, grid)
    m.calibrate(grid, yg)
    dec = nb.bits_to_numpy(m.query(grid, margin=1e-3), 65536)
    assert not np.any(nb.bits_to_numpy(yg, 65536) & ~dec)
    torch.cuda.synchronize()
