"""Inverted bounds and the broad-phase three-way test (Sec. 4.4): a bounding network of g
and one of the complement 1 - g (the swapped-weight network with its logit negated),
each certified against its own threshold, classify every query as certainly outside,
certainly inside or neither.  Codes against the oracle's two networks and thresholds,
the calibration-set invariants, the counters, and the argument checks."""
import numpy as np
import pytest
import torch

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


def _near(z, tau):
    return np.abs(z - tau) <= 1e-12 * max(1.0, abs(tau))


@pytest.mark.parametrize("kind,outer_prec", [(1, "f16x3"), (3, "f32")])
def test_three_way_codes_equal_oracle(nb, kind, outer_prec):
    w0 = I.ENC_WIDTH[kind]
    sc = I.make_scene(80 + kind, 12, 3, 0.3, 0.6)
    shape = nb.Shape(sc)
    outer_w, inner_w = [w0, 128, 128, 128, 1], [w0, 64, 64, 1]
    outer = nb.Model(outer_w, infer_prec=outer_prec)
    outer.set_params(I.init_params(81, outer_w))
    inner = nb.Model(inner_w)
    inner.set_params(I.init_params(82, inner_w))
    _train(nb, outer, shape, kind, 300, 8192, 83, invert=False)
    _train(nb, inner, shape, kind, 600, 8192, 84, invert=True)
    n = 200_003
    q = nb.sample(kind, n, seed=85)
    y = nb.label(shape, kind, q)
    tau_o = outer.calibrate(q, y)
    tau_i = inner.calibrate(q, nb.bits_not(y, n))
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    codes = nb.query_three_way(outer, inner, q, margin_outer=0.05, margin_inner=1e-3, stats=stats)
    c = codes.cpu().numpy()
    qh = q.cpu().numpy()
    zo = O.forward(outer_w, outer.get_params(), qh)
    zi = O.forward(inner_w, inner.get_params(), qh)
    expect = O.three_way(zo, tau_o, zi, tau_i)
    tie = _near(zo, tau_o) | _near(zi, tau_i)
    assert np.array_equal(c[~tie], expect[~tie])
    yy = nb.bits_to_numpy(y, n)
    # on the calibration set: "outside" is never a hit, "inside" never a miss, no conflict
    assert not np.any((c == 0) & yy)
    assert not np.any((c == 1) & ~yy)
    st = stats.cpu().numpy()
    assert st.tolist() == [int(np.sum(c == 0)), int(np.sum(c == 1)), int(np.sum(c == 2)), 0]
    assert st[0] > 0 and st[2] > 0
    if kind == 1:
        assert st[1] > 0.02 * n, st
    # held-out queries: the same definition, conflicts allowed and counted
    m = 70_001
    q2 = nb.sample(kind, m, seed=86)
    stats.zero_()
    c2 = nb.query_three_way(outer, inner, q2, margin_outer=0.05, margin_inner=1e-3, stats=stats).cpu().numpy()
    q2h = q2.cpu().numpy()
    zo2 = O.forward(outer_w, outer.get_params(), q2h)
    zi2 = O.forward(inner_w, inner.get_params(), q2h)
    tie2 = _near(zo2, tau_o) | _near(zi2, tau_i)
    assert np.array_equal(c2[~tie2], O.three_way(zo2, tau_o, zi2, tau_i)[~tie2])
    st2 = stats.cpu().numpy()
    assert st2[:3].sum() == m
    assert abs(st2[3] - int(np.sum((zo2 < tau_o) & (zi2 < tau_i)))) <= int(tie2.sum())


def test_three_way_edge_cases(nb):
    a = nb.Model([3, 64, 64, 1])
    a.set_params(I.init_params(1, [3, 64, 64, 1]))
    b = nb.Model([3, 64, 64, 1])
    b.set_params(I.init_params(2, [3, 64, 64, 1]))
    a.tau, b.tau = 0.0, 0.0
    q = nb.sample(1, 33, seed=3)
    # empty input
    assert nb.query_three_way(a, b, q[:0]).numel() == 0
    # one query and a ragged 33: every code in {0, 1, 2}, equal to the oracle's
    for k in (1, 33):
        c = nb.query_three_way(a, b, q[:k], margin_outer=1e-3, margin_inner=1e-3).cpu().numpy()
        qh = q[:k].cpu().numpy()
        e = O.three_way(O.forward([3, 64, 64, 1], a.get_params(), qh), 0.0,
                        O.forward([3, 64, 64, 1], b.get_params(), qh), 0.0)
        assert np.array_equal(c, e)
    # differing input widths
    r = nb.Model([6, 64, 64, 1])
    with pytest.raises(nb.NBError):
        nb.query_three_way(a, r, q)
