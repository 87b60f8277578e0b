"""Pins for the FP64 / exact-integer oracle, against facts fixed by the paper and by
mathematics (closed forms, brute force in exact rationals, Monte Carlo monotonicity,
finite differences, an independent autograd, a hand-worked Adam sequence).

Runs on CPU only.
"""
from fractions import Fraction as Fr
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_06822_gb300 import inputs as I

Q = 2.0 ** -20


def g(x):
    """snap to the 2^-20 grid"""
    return I.quantize(x, 20)


def one_sphere(r, c=(0.0, 0.0, 0.0), dim=3, vel=None):
    return I.Scene(g(np.array([c[:dim]])), g(np.array([r])),
                   None if vel is None else g(np.array([vel])), 20)


# ----------------------------------------------------------------------------- closed forms
def _within(p_hat, p, n, k=5.0):
    sigma = math.sqrt(p * (1 - p) / n)
    assert abs(p_hat - p) <= k * sigma, (p_hat, p, sigma)


def test_point3_volume_fraction():
    # Sec. 3.1 indicator (inside and on the surface): P(point in ball) = (4/3 pi r^3) / 8
    r, n = 0.5, 200_000
    q = I.sample_queries("point3", 11, n)
    y = O.label(I.POINT3, q, one_sphere(r))
    _within(y.mean(), 4.0 / 3.0 * math.pi * r ** 3 / 8.0, n)


def test_point2_area_fraction():
    r, n = 0.375, 200_000
    q = I.sample_queries("point2", 12, n)
    y = O.label(I.POINT2, q, one_sphere(r, dim=2))
    _within(y.mean(), math.pi * r ** 2 / 4.0, n)


def test_ray_hit_probability():
    # origin uniform on the radius-2 sphere, direction uniform on S^2:
    # the half-line meets a centred ball of radius r iff the direction lies in the cone
    # of half-angle asin(r/2) around -o, solid-angle fraction (1 - sqrt(1 - r^2/4)) / 2
    r, n = 0.75, 200_000
    q = I.sample_queries("ray3", 13, n)
    y = O.label(I.RAY3, q, one_sphere(r))
    _within(y.mean(), (1.0 - math.sqrt(1.0 - r * r / 4.0)) / 2.0, n)


def test_plane_hit_probability():
    # unit normal, offset U[-1,1]: the plane is at distance |off| from the centre -> P = r
    r, n = 0.3, 200_000
    q = I.sample_queries("plane3", 14, n)
    y = O.label(I.PLANE3, q, one_sphere(r))
    _within(y.mean(), r, n)


def test_box_hit_probability_steiner():
    # box centres U[-1,1]^3 with fixed half-extent e: hit iff the centre lies in the
    # Minkowski sum of the cube (side a = 2e) and the ball, volume
    # a^3 + 6 a^2 r + 3 pi a r^2 + 4/3 pi r^3 (Steiner), inside [-1,1]^3 here.
    e, r, n = 0.25, 0.25, 200_000
    rng = np.random.default_rng(15)
    b = rng.uniform(-1, 1, size=(n, 3))
    q = g(np.concatenate([b, np.full((n, 3), e)], 1))
    y = O.label(I.BOX3, q, one_sphere(r))
    a = 2 * e
    vol = a ** 3 + 6 * a * a * r + 3 * math.pi * a * r * r + 4.0 / 3.0 * math.pi * r ** 3
    _within(y.mean(), vol / 8.0, n)


def test_point4t_moving_sphere_fraction():
    # a ball of radius r moving inside the cube: at every t the slice is a ball of volume
    # 4/3 pi r^3, so P = 4/3 pi r^3 / 8 whatever the velocity
    r, n = 0.5, 200_000
    q = I.sample_queries("point4t", 16, n)
    sc = one_sphere(r, c=(-0.25, 0.0, 0.125), vel=(0.5, -0.25, 0.0))
    y = O.label(I.POINT4T, q, sc)
    _within(y.mean(), 4.0 / 3.0 * math.pi * r ** 3 / 8.0, n)


# ------------------------------------------------------------------ tangency / corner cases
def test_surface_is_inside_and_one_grid_step_is_outside():
    sc = one_sphere(0.5)
    on = g([[0.5, 0.0, 0.0], [0.0, -0.5, 0.0], [0.3, 0.4, 0.0]])
    off = g([[0.5 + Q, 0.0, 0.0], [0.0, 0.0, -0.5 - Q], [0.3, 0.4 + Q, 0.0]])
    assert O.label(I.POINT3, on, sc).tolist() == [1, 1, 1]
    assert O.label(I.POINT3, off, sc).tolist() == [0, 0, 0]


def test_ray_grazing_and_pointing_away():
    sc = one_sphere(0.5)
    rays = g([
        [-2.0, 0.5, 0.0, 1.0, 0.0, 0.0],        # grazes at distance exactly r -> 1
        [-2.0, 0.5 + Q, 0.0, 1.0, 0.0, 0.0],    # one grid step further -> 0
        [2.0, 0.0, 0.0, 1.0, 0.0, 0.0],         # points away from the ball -> 0
        [0.25, 0.0, 0.0, 1.0, 0.0, 0.0],        # origin inside the ball -> 1
        [0.5, 0.0, 0.0, 1.0, 0.0, 0.0],         # origin on the surface, pointing away -> 1
        [-2.0, 0.0, 0.0, 0.0, 0.0, 0.0],        # zero direction: the origin alone -> 0
        [-2.0, 0.3, 0.0, 3.0, 0.0, 0.0],        # non-unit direction -> 1
    ])
    assert O.label(I.RAY3, rays, sc).tolist() == [1, 0, 0, 1, 1, 0, 1]


def test_plane_touching():
    sc = one_sphere(0.5)
    planes = g([[0, 0, 1, 0.5], [0, 0, 1, 0.5 + Q], [0, 0, 1, -0.5], [0, 0, -1, 0.5],
                [0.6, 0.8, 0, 0.5], [0.6, 0.8, 0, 0.5 + Q], [0, 0, 0, 0.0], [0, 0, 0, 0.25]])
    assert O.label(I.PLANE3, planes, sc).tolist() == [1, 0, 1, 1, 1, 0, 1, 0]


def test_box_face_and_corner_contact():
    # sphere radius 5/16 at the origin; box corner at (3/16, 4/16, 0): distance exactly 5/16
    sc = one_sphere(5 / 16)
    e = 0.25
    boxes = g([
        [3 / 16 + e, 4 / 16 + e, e, e, e, e],        # touches at the corner -> 1
        [3 / 16 + e + Q, 4 / 16 + e, e, e, e, e],    # one grid step away -> 0
        [5 / 16 + e, 0.0, 0.0, e, e, e],             # face contact -> 1
        [0.0, 0.0, 0.0, 0.0, 0.0, 0.0],              # degenerate box = point at the centre -> 1
        [0.9, 0.9, 0.9, 0.01, 0.01, 0.01],           # far -> 0
    ])
    assert O.label(I.BOX3, boxes, sc).tolist() == [1, 0, 1, 1, 0]


def test_point4t_moving_contact():
    sc = one_sphere(0.25, vel=(0.5, 0.0, 0.0))
    q = g([[0.5, 0, 0, 1.0], [0.5, 0, 0, 0.0], [0.75, 0, 0, 1.0], [0.75 + Q, 0, 0, 1.0],
           [0.25, 0, 0, 0.0], [0.5, 0, 0, 0.5]])
    assert O.label(I.POINT4T, q, sc).tolist() == [1, 0, 1, 0, 1, 1]


def test_off_grid_input_is_rejected():
    sc = one_sphere(0.5)
    with pytest.raises(ValueError):
        O.label(I.POINT3, np.array([[1e-9, 0, 0]], dtype=np.float32), sc)
    with pytest.raises(ValueError):
        O.label(I.POINT3, np.array([[np.nan, 0, 0]], dtype=np.float32), sc)


# --------------------------------------------------- brute force in exact rationals
def _fr(v):
    return Fr(float(v))


def _brute(kind, q, sc):
    """Direct geometric definitions in exact rational arithmetic (different
    formulations from the oracle's: projection / clamping, not inequality algebra)."""
    out = []
    for row in q:
        row = [_fr(v) for v in row]
        hit = 0
        for s in range(sc.n_spheres):
            c = [_fr(v) for v in sc.centres[s]]
            r = _fr(sc.radii[s])
            if kind in (I.POINT2, I.POINT3):
                d2 = sum((a - b) ** 2 for a, b in zip(row, c))
            elif kind == I.POINT4T:
                v = [_fr(x) for x in sc.vel[s]]
                t = row[3]
                d2 = sum((row[i] - (c[i] + v[i] * t)) ** 2 for i in range(3))
            elif kind == I.RAY3:
                o, d = row[:3], row[3:]
                dd = sum(x * x for x in d)
                sstar = Fr(0) if dd == 0 else max(Fr(0), sum((c[i] - o[i]) * d[i] for i in range(3)) / dd)
                p = [o[i] + sstar * d[i] for i in range(3)]
                d2 = sum((p[i] - c[i]) ** 2 for i in range(3))
            elif kind == I.PLANE3:
                nrm, off = row[:3], row[3]
                nn = sum(x * x for x in nrm)
                dist = sum(nrm[i] * c[i] for i in range(3)) - off
                if nn == 0:
                    hit |= int(off == 0)
                    continue
                d2 = dist * dist / nn
            elif kind == I.BOX3:
                b, e = row[:3], row[3:]
                p = [min(max(c[i], b[i] - e[i]), b[i] + e[i]) for i in range(3)]
                d2 = sum((p[i] - c[i]) ** 2 for i in range(3))
            hit |= int(d2 <= r * r)
        out.append(hit)
    return out


@pytest.mark.parametrize("kind", [I.POINT2, I.POINT3, I.POINT4T, I.RAY3, I.PLANE3, I.BOX3])
def test_brute_force_rationals(kind):
    dim = 2 if kind == I.POINT2 else 3
    # radii large enough that roughly half the queries hit
    sc = I.make_scene(100 + kind, 4, dim, 0.2, 0.6, moving=(kind == I.POINT4T))
    q = I.sample_queries(kind, 200 + kind, 300)
    y = O.label(kind, q, sc)
    assert y.tolist() == _brute(kind, q, sc)
    assert 0 < y.sum() < len(y)


# ------------------------------------------------------- Monte Carlo (Alg. 1) agreement
@pytest.mark.parametrize("kind,dens", [(I.RAY3, (2, 5, 9)), (I.BOX3, (1, 3, 8)), (I.PLANE3, (1, 3, 8))])
def test_mc_implies_exact_and_converges(kind, dens):
    sc = I.make_scene(300 + kind, 3, 3, 0.1, 0.4)
    q = I.sample_queries(kind, 400 + kind, 400)
    y = O.label(kind, q, sc)
    misses = []
    for d in dens:
        ym = O.mc_label(kind, q, sc, d)
        assert not np.any((ym == 1) & (y == 0)), "a sample hit where the exact test says no"
        misses.append(int(np.sum((y == 1) & (ym == 0))))
    assert misses[0] >= misses[1] >= misses[2]
    assert misses[-1] <= max(2, y.sum() // 20)


# ----------------------------------------------------------------------- network, loss
def _torch_mlp_f64(widths, params, X):
    import torch
    p = torch.tensor(params.astype(np.float64), requires_grad=True)
    a = torch.tensor(X.astype(np.float64))
    off = 0
    L = len(widths) - 1
    for l in range(L):
        fi, fo = widths[l], widths[l + 1]
        W = p[off:off + fo * fi].view(fo, fi)
        off += fo * fi
        b = p[off:off + fo]
        off += fo
        a = a @ W.T + b
        if l < L - 1:
            a = torch.relu(a)
    return p, a[:, 0]


def test_param_count_matches_paper():
    # 3 -> 50 -> 50 -> 1 with biases has 2,801 parameters (Sec. 4.4, 3D point network)
    assert O.param_count([3, 50, 50, 1]) == 2801
    assert I.param_count([3, 50, 50, 1]) == 2801


def test_forward_special_cases():
    # one layer: z = w.x + b
    w = [2, 1]
    params = np.array([0.5, -2.0, 0.25], dtype=np.float32)
    X = np.array([[1.0, 1.0], [4.0, 0.5], [0.0, 0.0]], dtype=np.float32)
    assert O.forward(w, params, X).tolist() == [-1.25, 1.25, 0.25]
    # zero weights: z = b_L whatever the input
    w = [3, 8, 8, 1]
    p = np.zeros(I.param_count(w), dtype=np.float32)
    p[-1] = 0.75
    assert np.all(O.forward(w, p, I.sample_queries("point3", 1, 10)) == 0.75)
    # ReLU kills negative pre-activations: x -> relu(x) -> -relu(x) + 1
    w = [1, 1, 1]
    p = np.array([1.0, 0.0, -1.0, 1.0], dtype=np.float32)
    X = np.array([[-3.0], [2.0]], dtype=np.float32)
    assert O.forward(w, p, X).tolist() == [1.0, -1.0]


def test_forward_matches_autograd_framework():
    w = [6, 32, 32, 1]
    p = I.init_params(5, w)
    X = I.sample_queries("ray3", 6, 500)
    _, z = _torch_mlp_f64(w, p, X)
    np.testing.assert_allclose(O.forward(w, p, X), z.detach().numpy(), rtol=1e-12, atol=1e-12)


def test_loss_and_gradient_match_autograd():
    import torch
    w = [3, 16, 16, 1]
    p = I.init_params(7, w)
    X = I.sample_queries("point3", 8, 256)
    y = (np.random.default_rng(9).random(256) < 0.3).astype(np.uint8)
    alpha, beta = 37.5, 1.0
    loss, grad = O.loss_grad(w, p, X, y, alpha, beta)
    pt, z = _torch_mlp_f64(w, p, X)
    yt = torch.tensor(y.astype(np.float64))
    s = torch.sigmoid(z)
    L = -(alpha * yt * torch.log(s) + beta * (1 - yt) * torch.log(1 - s)).mean()
    L.backward()
    assert abs(loss - L.item()) <= 1e-12 * abs(L.item())
    np.testing.assert_allclose(grad, pt.grad.numpy(), rtol=1e-10, atol=1e-14)


def test_symmetric_weights_reduce_to_textbook_bce():
    w = [2, 8, 1]
    p = I.init_params(3, w)
    X = I.sample_queries("point2", 4, 100)
    y = (np.arange(100) % 3 == 0).astype(np.uint8)
    loss, _ = O.loss_grad(w, p, X, y, 1.0, 1.0)
    z = O.forward(w, p, X)
    s = 1 / (1 + np.exp(-z))
    bce = -np.mean(y * np.log(s) + (1 - y) * np.log(1 - s))
    assert abs(loss - bce) < 1e-12


def test_gradient_central_differences():
    w = [2, 6, 5, 1]
    p = I.init_params(21, w).astype(np.float64)
    X = I.sample_queries("point2", 22, 40)
    y = (np.arange(40) % 4 == 1).astype(np.uint8)
    alpha, beta = 5.0, 1.5

    # keep the pre-activations away from the ReLU kink so the loss is smooth
    def pre_acts(params):
        a = X.astype(np.float64)
        off, m = 0, np.inf
        for l in range(len(w) - 1):
            fi, fo = w[l], w[l + 1]
            W = params[off:off + fo * fi].reshape(fo, fi)
            off += fo * fi
            b = params[off:off + fo]
            off += fo
            zz = a @ W.T + b
            if l < len(w) - 2:
                m = min(m, np.min(np.abs(zz)))
                a = np.maximum(zz, 0)
        return m

    assert pre_acts(p) > 1e-3
    # the oracle reads FP32 parameters, so difference on a grid that FP32 represents
    h = 2.0 ** -14
    p32 = p.astype(np.float32)
    _, grad = O.loss_grad(w, p32, X, y, alpha, beta)
    rng = np.random.default_rng(0)
    idx = rng.choice(len(p32), size=25, replace=False)
    for i in idx:
        pp, pm = p32.copy(), p32.copy()
        pp[i] += np.float32(h)
        pm[i] -= np.float32(h)
        lp, _ = O.loss_grad(w, pp, X, y, alpha, beta)
        lm, _ = O.loss_grad(w, pm, X, y, alpha, beta)
        fd = (lp - lm) / (float(pp[i]) - float(pm[i]))
        assert abs(fd - grad[i]) <= 1e-6 + 1e-5 * abs(grad[i]), (i, fd, grad[i])


# ------------------------------------------------------------------------------ Adam
def test_adam_hand_worked_two_steps():
    # theta0 = 1, g1 = 0.5, g2 = -0.25, lr 1e-3, betas (0.9, 0.999), eps 1e-8
    # step 1: m = 0.05, v = 2.5e-4, m^ = 0.5, v^ = 0.25 -> update 1e-3 * 0.5 / (0.5 + 1e-8)
    # step 2: m = 0.02, v = 3.1225e-4, m^ = 0.02 / 0.19, v^ = 3.1225e-4 / 0.001999
    th = np.array([1.0])
    m = np.zeros(1)
    v = np.zeros(1)
    O.adam(th, m, v, np.array([0.5]), 1)
    th1 = 1.0 - 1e-3 * 0.5 / (0.5 + 1e-8)
    assert abs(th[0] - th1) < 1e-15
    O.adam(th, m, v, np.array([-0.25]), 2)
    assert abs(m[0] - 0.02) < 1e-15 and abs(v[0] - 3.1225e-4) < 1e-16
    upd = 1e-3 * (0.02 / 0.19) / (math.sqrt(3.1225e-4 / 0.001999) + 1e-8)
    assert abs(th[0] - (th1 - upd)) < 1e-15
    assert abs(upd - 2.66337e-4) < 1e-9


def test_adam_matches_torch_optimizer():
    import torch
    rng = np.random.default_rng(1)
    th0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) * 10.0 ** rng.integers(-4, 1) for _ in range(5)]
    th, m, v = th0.copy(), np.zeros(50), np.zeros(50)
    for t, gr in enumerate(grads, 1):
        O.adam(th, m, v, gr, t)
    pt = torch.tensor(th0, requires_grad=True)
    opt = torch.optim.Adam([pt], lr=1e-3)
    for gr in grads:
        opt.zero_grad()
        pt.grad = torch.tensor(gr)
        opt.step()
    np.testing.assert_allclose(th, pt.detach().numpy(), rtol=0, atol=1e-12)


# ----------------------------------------------------------------------- calibration
def test_calibration_gives_zero_fn_and_is_the_rounded_down_minimum():
    rng = np.random.default_rng(2)
    z = rng.standard_normal(10_000) * 3
    y = (rng.random(10_000) < 0.2).astype(np.uint8)
    eps = 1e-5
    tau, npos = O.calibrate(z, y, eps)
    assert npos == int(y.sum())
    mn = z[y == 1].min()
    # tau is the largest double not above (min - eps), evaluated exactly
    exact = Fr(float(mn)) - Fr(eps)
    assert Fr(tau) <= exact < Fr(float(np.nextafter(tau, np.inf)))
    c = O.count(z, y, tau)
    assert c["FN"] == 0
    assert c["TP"] == npos and c["FP"] + c["TN"] == 10_000 - npos
    # no positives: tau = +inf, every query decided outside
    tau2, n2 = O.calibrate(z, np.zeros_like(y), eps)
    assert n2 == 0 and tau2 == math.inf


def test_count_cost_table():
    z = np.array([-1.0, 0.0, 2.0, 3.0, -5.0])
    y = np.array([1, 0, 1, 0, 0], dtype=np.uint8)
    assert O.count(z, y, 0.0) == {"FN": 1, "FP": 2, "TP": 1, "TN": 1}


def test_forward_scale_definition():
    # one layer: scale = sum |w| |x| + |b|
    w = [2, 1]
    p = np.array([0.5, -2.0, 0.25], dtype=np.float32)
    X = np.array([[1.0, 1.0], [-4.0, 0.5]], dtype=np.float32)
    assert O.forward_scale(w, p, X).tolist() == [2.75, 3.25]
    # hidden layers: |W_L| . relu(...) + |b_L|, against the autograd forward
    import torch
    w = [3, 8, 8, 1]
    p = I.init_params(31, w)
    X = I.sample_queries("point3", 32, 50)
    pt, _ = _torch_mlp_f64(w, p, X)
    a = torch.tensor(X.astype(np.float64))
    off = 0
    for l in range(2):
        fi, fo = w[l], w[l + 1]
        W = pt[off:off + fo * fi].view(fo, fi)
        off += fo * fi
        a = torch.relu(a @ W.T + pt[off:off + fo])
        off += fo
    s = (a @ pt[off:off + 8].abs().detach() + pt[off + 8].abs()).detach().numpy()
    np.testing.assert_allclose(O.forward_scale(w, p, X), s, rtol=1e-12)


def test_benefit_break_even_worked_example():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "benefit_worked_example.json")))
    t_star, side = O.benefit_break_even(g["t_a"], g["t_b"], g["p_a"], g["p_b"])
    assert abs(t_star - g["t_star"]) <= 1e-12 and side == g["side"]
    # the inequality itself: A's total time is below B's just above t*, above it just below
    for t, wins in ((t_star * 1.001, True), (t_star * 0.999, False)):
        assert (g["t_a"] + g["p_a"] * t < g["t_b"] + g["p_b"] * t) == wins
    # a cascade with the network in front of the exact test against the box test alone
    # (p_b = 1, t_a = t_b + t_nn) pays off once t > t_nn / (1 - p_a)
    t_nn, p = 0.37, 0.82
    t_star, side = O.benefit_break_even(1.0 + t_nn, 1.0, p, 1.0)
    assert side == ">" and abs(t_star - t_nn / (1 - p)) <= 1e-12


# ----------------------------------------------------------------------------- inverted bounds
def test_swapped_weights_equal_the_complement_with_negated_logit():
    # Sec. 4.4: the inverted bound swaps the asymmetry weights.  Training on g with
    # (alpha, beta) swapped is training on 1 - g with the logit negated: the loss is the
    # same number and the gradient differs only in the sign of the head's entries.
    w = [3, 16, 16, 1]
    p = I.init_params(11, w)
    X = I.sample_queries("point3", 12, 300)
    y = (np.random.default_rng(13).random(300) < 0.4).astype(np.uint8)
    alpha, beta = 1.0, 42.0
    loss_s, g_s = O.loss_grad(w, p, X, y, beta, alpha)  # swapped weights on g
    H = w[-2]
    p_neg = p.copy()
    p_neg[-(H + 1):] *= -1  # head weights and bias negated
    loss_c, g_c = O.loss_grad(w, p_neg, X, 1 - y, alpha, beta)  # complement, usual weights
    assert np.array_equal(O.forward(w, p_neg, X), -O.forward(w, p, X))
    assert loss_s == loss_c
    # dL/dz uses sigma(z) on one side and sigma(-z) = 1 - sigma(z) on the other: equal up
    # to the rounding of that identity
    sc = np.max(np.abs(g_s))
    np.testing.assert_allclose(g_s[:-(H + 1)], g_c[:-(H + 1)], rtol=1e-12, atol=1e-14 * sc)
    np.testing.assert_allclose(g_s[-(H + 1):], -g_c[-(H + 1):], rtol=1e-12, atol=1e-14 * sc)
    # and it is not an identity of any two weightings: the unswapped loss differs
    assert abs(O.loss_grad(w, p, X, y, alpha, beta)[0] - loss_s) > 1e-3


def _codes_1d(w_o, b_o, tau_o, w_i, b_i, tau_i, xs):
    X = np.array([[x] for x in xs], dtype=np.float32)
    z_o = O.forward([1, 1], np.array([w_o, b_o], dtype=np.float32), X)
    z_i = O.forward([1, 1], np.array([w_i, b_i], dtype=np.float32), X)
    return O.three_way(z_o, tau_o, z_i, tau_i).tolist()


def test_three_way_hand_worked():
    # outer z = 2x - 1 (tau 0): certainly outside for x < 0.5
    # inner z = -4x + 3: certainly inside where z < tau_i
    xs = [0.0, 0.125, 0.25, 0.5, 1.0]
    # tau_i = 2.5: inside for x > 0.125; x = 0.25 is claimed by both (a conflict -> 2),
    # ties z = tau count as "not certain" for both networks
    assert _codes_1d(2.0, -1.0, 0.0, -4.0, 3.0, 2.5, xs) == [0, 0, 2, 1, 1]
    # tau_i = -2: inside only for x > 1.25; between 0.5 and 1.25 neither network is certain
    assert _codes_1d(2.0, -1.0, 0.0, -4.0, 3.0, -2.0, [0.0, 0.5, 0.75, 1.25, 1.5]) == [0, 2, 2, 2, 1]


def test_three_way_respects_labels_on_the_calibration_set():
    rng = np.random.default_rng(21)
    n = 20_000
    y = (rng.random(n) < 0.35).astype(np.uint8)
    # noisy logits of a bound and of a complement bound
    z_o = np.where(y == 1, 2.0, -2.0) + rng.standard_normal(n) * 1.5
    z_i = np.where(y == 1, -2.0, 2.0) + rng.standard_normal(n) * 1.5
    tau_o, _ = O.calibrate(z_o, y)
    tau_i, _ = O.calibrate(z_i, 1 - y)
    c = O.three_way(z_o, tau_o, z_i, tau_i)
    assert not np.any((c == 0) & (y == 1))  # certainly outside is never a hit
    assert not np.any((c == 1) & (y == 0))  # certainly inside is never a miss
    # on the calibration set no query is claimed by both networks
    assert not np.any((z_o < tau_o) & (z_i < tau_i))
    assert np.sum(c == 0) > 0 and np.sum(c == 1) > 0 and np.sum(c == 2) > 0


# ----------------------------------------------------------------------------- paper encoding
def test_paper_encoding_box_corners_and_plane_point():
    box = I.sample_queries("box3", 32, 500)
    enc = O.paper_encoding(I.BOX3, box)
    assert enc.shape == (500, 6)
    # the corners' midpoint is the centre and their half-difference the half-extents
    np.testing.assert_array_equal((enc[:, :3] + enc[:, 3:]) / 2, box[:, :3].astype(np.float64))
    np.testing.assert_array_equal((enc[:, 3:] - enc[:, :3]) / 2, box[:, 3:].astype(np.float64))
    pl = I.sample_queries("plane3", 33, 500)
    e = O.paper_encoding(I.PLANE3, pl)
    n, off = pl[:, :3].astype(np.float64), pl[:, 3].astype(np.float64)
    # p0 lies on the plane n . x = off and is its point nearest the origin (parallel to n)
    np.testing.assert_allclose(np.sum(n * e[:, :3], axis=1), off, rtol=0, atol=1e-12)
    np.testing.assert_allclose(np.cross(e[:, :3], n), 0.0, atol=1e-12)
    np.testing.assert_array_equal(e[:, 3:], n)
    # a hand case: the plane z = 0.5 with normal (0, 0, 2), offset 1
    h = O.paper_encoding(I.PLANE3, np.array([[0.0, 0.0, 2.0, 1.0]], dtype=np.float32))
    assert h.tolist() == [[0.0, 0.0, 0.5, 0.0, 0.0, 2.0]]
    # rays and points are unchanged
    r = I.sample_queries("ray3", 34, 10)
    assert np.array_equal(O.paper_encoding(I.RAY3, r), r.astype(np.float64))
