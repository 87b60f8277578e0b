"""Pins of the oracle's sinusoidal hidden activation (Sec. 3.4 "Architecture": sinusoidal
activations in the hidden layers): closed forms of one- and two-neuron networks, an
independent float64 autograd framework, central differences (sin is smooth everywhere,
so every parameter can be differenced), and the special cases that tie it to the ReLU
network (zero weights).  Runs on CPU only."""
import math

import numpy as np

from oracle import oracle as O
from paper_2310_06822_gb300 import inputs as I


def _torch_mlp_sine_f64(widths, params, X):
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
            a = torch.sin(a)
    return p, a[:, 0]


def test_one_neuron_closed_form():
    # z = w2 sin(w1 x + b1) + b2
    w1, b1, w2, b2 = 2.0, 0.5, 3.0, -1.0
    p = np.array([w1, b1, w2, b2], dtype=np.float32)
    X = np.array([[0.25], [-1.0], [0.0]], dtype=np.float32)
    z = O.forward([1, 1, 1], p, X, act="sine")
    want = [w2 * math.sin(w1 * x + b1) + b2 for x in (0.25, -1.0, 0.0)]
    assert np.allclose(z, want, rtol=0, atol=1e-15)
    # loss gradient of one sample by hand: dL/dz = alpha y (s - 1) + beta (1 - y) s,
    # dz/dw2 = sin(u), dz/db2 = 1, dz/dw1 = w2 cos(u) x, dz/db1 = w2 cos(u), u = w1 x + b1
    x, y, alpha, beta = 0.25, 1, 7.0, 1.0
    loss, g = O.loss_grad([1, 1, 1], p, np.array([[x]], np.float32), np.array([y], np.uint8), alpha, beta,
                          act="sine")
    u = w1 * x + b1
    zz = w2 * math.sin(u) + b2
    s = 1 / (1 + math.exp(-zz))
    dz = alpha * y * (s - 1)
    assert abs(loss - alpha * math.log1p(math.exp(-zz))) < 1e-14
    assert np.allclose(g, [dz * w2 * math.cos(u) * x, dz * w2 * math.cos(u), dz * math.sin(u), dz],
                       rtol=1e-13, atol=1e-16)


def test_two_hidden_layers_closed_form():
    # z = w3 sin(w2 sin(w1 x + b1) + b2) + b3, every term by hand
    p = np.array([1.5, -0.25, -2.0, 0.75, 0.5, 0.125], dtype=np.float32)
    X = np.array([[0.3], [-0.7]], dtype=np.float32)
    z = O.forward([1, 1, 1, 1], p, X, act="sine")
    want = [0.5 * math.sin(-2.0 * math.sin(1.5 * float(np.float32(x)) - 0.25) + 0.75) + 0.125 for x in (0.3, -0.7)]
    assert np.allclose(z, want, rtol=0, atol=1e-15)


def test_sine_forward_and_gradient_match_autograd():
    import torch
    w = [6, 24, 24, 1]
    p = I.init_params(31, w)
    X = I.sample_queries("ray3", 32, 300)
    y = (np.random.default_rng(33).random(300) < 0.4).astype(np.uint8)
    alpha, beta = 12.0, 1.0
    pt, z = _torch_mlp_sine_f64(w, p, X)
    np.testing.assert_allclose(O.forward(w, p, X, act="sine"), z.detach().numpy(), rtol=1e-12, atol=1e-12)
    yt = torch.tensor(y.astype(np.float64))
    s = torch.sigmoid(z)
    L = -(alpha * yt * torch.log(s) + beta * (1 - yt) * torch.log(1 - s)).mean()
    L.backward()
    loss, grad = O.loss_grad(w, p, X, y, alpha, beta, act="sine")
    assert abs(loss - L.item()) <= 1e-12 * abs(L.item())
    np.testing.assert_allclose(grad, pt.grad.numpy(), rtol=1e-10, atol=1e-14)


def test_sine_gradient_central_differences():
    w = [2, 6, 5, 1]
    p32 = I.init_params(41, w)
    X = I.sample_queries("point2", 42, 40)
    y = (np.arange(40) % 3 == 1).astype(np.uint8)
    alpha, beta = 4.0, 1.5
    _, grad = O.loss_grad(w, p32, X, y, alpha, beta, act="sine")
    # the oracle reads FP32 parameters: difference with steps FP32 represents exactly
    h = 2.0 ** -12
    for i in range(len(p32)):
        pp, pm = p32.copy(), p32.copy()
        pp[i] = np.float32(p32[i] + h)
        pm[i] = np.float32(p32[i] - h)
        hh = (float(pp[i]) - float(pm[i])) / 2
        lp, _ = O.loss_grad(w, pp, X, y, alpha, beta, act="sine")
        lm, _ = O.loss_grad(w, pm, X, y, alpha, beta, act="sine")
        fd = (lp - lm) / (2 * hh)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(grad[i])), (i, fd, grad[i])


def test_zero_first_layer_gives_constant_logit():
    # zero weights and biases in the first layer: sin(0) = 0, the second layer sees zeros,
    # so the logit is sum_n W2_n sin(b1_n) + b2 for every input
    w = [3, 8, 8, 1]
    p = I.init_params(51, w)
    p[: 8 * 3 + 8] = 0.0
    X = I.sample_queries("point3", 52, 20)
    zs = O.forward(w, p, X, act="sine")
    b1 = p[8 * 3 + 8 + 64: 8 * 3 + 8 + 72].astype(np.float64)
    W2 = p[8 * 3 + 8 + 72: 8 * 3 + 8 + 80].astype(np.float64)
    assert np.allclose(zs, np.dot(W2, np.sin(b1)) + float(p[-1]), rtol=0, atol=1e-14)
    # ReLU and sine differ on ordinary weights
    p2 = I.init_params(53, w)
    assert not np.allclose(O.forward(w, p2, X, act="sine"), O.forward(w, p2, X, act="relu"))
