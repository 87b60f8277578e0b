"""BF16 tensor-core training step against the FP64 oracle: loss and per-tensor gradient
directions (BF16 operands, FP32 accumulation), Adam on the FP32 master weights, ragged
batches, and a short training run that ends conservative after calibration."""
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


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def _per_tensor(widths):
    out, off = [], 0
    for l in range(len(widths) - 1):
        nW = widths[l + 1] * widths[l]
        out.append((off, off + nW))
        out.append((off + nW, off + nW + widths[l + 1]))
        off += nW + widths[l + 1]
    return out


@pytest.mark.parametrize("kind,widths,n", [("ray3", [6, 128, 128, 128, 128, 1], 65536),
                                           ("ray3", [6, 128, 128, 128, 128, 1], 200_003),
                                           ("ray3", [6, 128, 128, 128, 1], 4133),
                                           ("point3", [3, 128, 128, 1], 128 * 152 * 3 + 77),
                                           ("box3", [6, 128, 128, 128, 1], 1_000_001),
                                           ("point4t", [4, 64, 64, 64, 1], 777),
                                           ("point4t", [4, 64, 64, 64, 1], 200_003),
                                           ("point3", [3, 128, 128, 1], 1),
                                           ("box3", [6, 256, 256, 256, 256, 1], 8191),
                                           ("plane3", [4, 256, 256, 1], 33)])
def test_bf16_step_gradient_direction_loss_adam(nb, kind, widths, n):
    kid = I.kind_id(kind)
    sc = I.make_scene(60, 32, 3, 0.05, 0.3, moving=(kid == I.POINT4T))
    q = I.sample_queries(kind, 61, n)
    y = O.label(kid, q, sc)
    p = I.init_params(62, widths)
    m = nb.Model(widths, infer_prec="f32", train_prec="bf16")
    m.set_params(p)
    st = nb.step_stats_tensor()
    m.train_step(_dev(q), _dev(I.pack_bits(y).view(np.int32)), 20.0, 1.0, stats=st)
    g = m.get_grad().astype(np.float64)
    loss64, g64 = O.loss_grad(widths, p, q, y, 20.0, 1.0)
    s = nb.read_step_stats(st)
    assert abs(s["loss"] - loss64) <= 2e-2 * abs(loss64)
    for a, b in _per_tensor(widths):
        if np.linalg.norm(g64[a:b]) == 0:
            continue
        cos = float(np.dot(g[a:b], g64[a:b]) / (np.linalg.norm(g[a:b]) * np.linalg.norm(g64[a:b])))
        rel = np.linalg.norm(g[a:b] - g64[a:b]) / np.linalg.norm(g64[a:b])
        assert cos >= 0.999 and rel <= 5e-2, (a, b, cos, rel)
    th = p.astype(np.float64)
    O.adam(th, np.zeros_like(th), np.zeros_like(th), g, 1)
    assert np.max(np.abs(m.get_params().astype(np.float64) - th)) <= 1e-6


def test_bf16_training_run_is_conservative_after_calibration(nb):
    """3D rays, 64 spheres, 6->128x4->1: 300 BF16 tensor-core steps of 65,536 rays, the
    split-FP16 forward for queries: FN = 0 after calibration, decisions equal the oracle's,
    and the bound is tighter than the trivial one."""
    import torch
    widths = [6, 128, 128, 128, 128, 1]
    sc = I.make_scene(1001, 64, 3, 0.02, 0.2)
    shape = nb.Shape(sc)
    m = nb.Model(widths, infer_prec="f16x3", train_prec="bf16")
    m.set_params(I.init_params(4001, widths))
    B, W, T = 65536, 8, 300
    pool = _dev(I.sample_queries("ray3", 2018, B * W))
    bits = nb.label(shape, I.RAY3, pool)
    st = nb.step_stats_tensor()
    losses = []
    for t in range(T):
        j = t % W
        m.train_step(pool[j * B:(j + 1) * B], bits[j * B // 32:(j + 1) * B // 32], 1.0 + 99.0 * t / (T - 1), 1.0,
                     stats=st)
        if t in (0, T - 1):
            losses.append(nb.read_step_stats(st)["loss"])
    n = 200_003
    q = I.sample_queries("ray3", 2019, n)
    qd = _dev(q)
    yd = nb.label(shape, I.RAY3, qd)
    y = nb.bits_to_numpy(yd, n)
    tau = m.calibrate(qd, yd)
    dec = nb.bits_to_numpy(m.query(qd, margin=0.05), n)
    z64 = O.forward(widths, m.get_params(), q)
    tie = np.abs(z64 - tau) <= 1e-12 * max(1.0, abs(tau))
    assert np.array_equal(dec[~tie], (z64 >= tau)[~tie])
    assert not np.any(y & ~dec)
    assert np.mean(dec & ~y) < 0.9 * np.mean(~y)
    torch.cuda.synchronize()


@pytest.mark.parametrize("widths,prec", [([6, 128, 128, 128, 128, 1], "bf16"), ([6, 128, 128, 128, 1], "bf16"),
                                         ([6, 128, 128, 1], "bf16"), ([6, 64, 64, 64, 1], "bf16"),
                                         ([6, 256, 256, 1], "bf16"), ([6, 32, 32, 1], "f32")])
def test_bf16_step_skips_nonfinite_rows_and_is_deterministic(nb, widths, prec):
    """Rows with a NaN or infinite coordinate give a non-finite logit: they add nothing to
    the loss or the gradient (the mean still divides by n) and are counted; the step on the
    other rows matches the oracle on those rows; two identical steps give identical bits."""
    n = 50_000
    sc = I.make_scene(63, 32, 3, 0.05, 0.3)
    q = I.sample_queries("ray3", 64, n)
    y = O.label(I.RAY3, q, sc)
    bad = np.zeros(n, dtype=bool)
    bad[np.random.default_rng(65).choice(n, 37, replace=False)] = True
    qb = q.copy()
    idx = np.nonzero(bad)[0]
    qb[idx[::2], 0] = np.nan
    qb[idx[1::2], 4] = np.inf
    p = I.init_params(66, widths)
    grads = []
    for rep in range(2):
        m = nb.Model(widths, infer_prec="f32", train_prec=prec)
        m.set_params(p)
        st = nb.step_stats_tensor()
        m.train_step(_dev(qb), _dev(I.pack_bits(y).view(np.int32)), 20.0, 1.0, stats=st)
        s = nb.read_step_stats(st)
        assert s["n_nonfinite"] == bad.sum()
        grads.append(m.get_grad())
        assert np.all(np.isfinite(grads[-1]))
    assert np.array_equal(grads[0].view(np.uint32), grads[1].view(np.uint32))
    good = ~bad
    loss64, g64 = O.loss_grad(widths, p, q[good], y[good], 20.0, 1.0)
    g64 *= good.sum() / n
    g = grads[0].astype(np.float64)
    for a, b in _per_tensor(widths):
        if np.linalg.norm(g64[a:b]) == 0:
            continue
        cos = float(np.dot(g[a:b], g64[a:b]) / (np.linalg.norm(g[a:b]) * np.linalg.norm(g64[a:b])))
        assert cos >= (0.999 if prec == "bf16" else 1 - 1e-8), (a, b, cos)
