"""Parity at the benchmark's full sizes, in the launch configurations bench.py times:
every decision of the fast forms against the certified FP32 single-object form (both
re-checked, so they must agree bit for bit), sampled logits and labels against the FP64
oracle, one by one.  Networks are at their initial scale times three (logits spanning
tens of units), so no training is needed to exercise the band and the re-check."""
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


def _sample_idx(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, k, replace=False))


def test_fp8_boxes_64m(nb):
    """64M boxes against the 256-sphere union, 6->256x4->1 in E4M3: decisions equal the
    FP32 form's on all of them; sampled labels, logits and decisions against the oracle."""
    import torch
    widths = [6, 256, 256, 256, 256, 1]
    sc = I.make_scene(1003, 256, 3, 0.02, 0.2)
    shape = nb.Shape(sc)
    n = 64 << 20
    q = nb.sample(I.BOX3, n, seed=3008)
    y = nb.label(shape, I.BOX3, q)
    p = (I.init_params(4008, widths) * 3.0).astype(np.float32)
    f8 = nb.Model(widths, infer_prec="fp8")
    f8.set_params(p)
    f32 = nb.Model(widths)
    f32.set_params(p)
    idx = _sample_idx(n, 20000, 1)
    qs = q[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    # labels of the sample against the oracle, bit for bit
    assert np.array_equal(nb.bits_to_numpy(y, n)[idx], O.label(I.BOX3, qs, sc).astype(bool))
    z64 = O.forward(widths, p, qs)
    _, z8 = f8.query(q, logits=True)
    _, z32 = f32.query(q, logits=True)
    # the FP32 form's logits are within 1e-5 of the scale of the oracle's on the sample
    S = O.forward_scale(widths, p, qs)
    assert np.max(np.abs(z32.cpu().numpy()[idx].astype(np.float64) - z64) / np.maximum(np.abs(z64), S)) <= 1e-5
    # the margin covers the E4M3 error on every query (twice its maximum, as the benchmark)
    err = float((z8 - z32).abs().max().item())
    del z8, z32
    tau = float(np.quantile(z64, 0.5))
    f8.tau = tau
    f32.tau = tau
    margin = 2.0 * err + 0.05
    b8, st = f8.query(q, margin=margin, stats=True)
    b32 = f32.query(q, margin=1e-2)
    assert torch.equal(b8, b32)
    assert st["n_unresolved"] == 0
    dec = nb.bits_to_numpy(b8, n)[idx]
    tie = np.abs(z64 - tau) <= 1e-12 * max(1.0, abs(tau))
    assert np.array_equal(dec[~tie], (z64 >= tau)[~tie])


def test_grouped_4d_256_objects_1m_points(nb):
    """256 objects x 1M points each through the grouped split-FP16 launch (autotuned
    split): decisions equal the grouped FP32 form's; sampled points of every 32nd object
    against the oracle."""
    import torch
    widths = [4, 64, 64, 64, 1]
    K, NE = 256, 1 << 20
    off = np.arange(K + 1, dtype=np.int64) * NE
    q = nb.sample(I.POINT4T, K * NE, seed=7001)
    P = np.stack([(I.init_params(6000 + o, widths) * 3.0).astype(np.float32) for o in range(K)])
    gs = nb.Group(widths, K, infer_prec="f16x3")
    gs.set_params(P)
    gf = nb.Group(widths, K)
    gf.set_params(P)
    best, _ = gs.autotune(off, q, op="query", candidates=(8192, 32768))
    plan = nb.Plan(off, chunk_rows=best)
    taus = np.zeros(K)
    checks = {}
    for o in range(0, K, 32):
        idx = o * NE + _sample_idx(NE, 2000, o)
        qs = q[torch.as_tensor(idx, device="cuda")].cpu().numpy()
        z64 = O.forward(widths, P[o], qs)
        taus[o] = float(np.quantile(z64, 0.5))
        checks[o] = (idx, z64)
    gs.tau = taus
    gf.tau = taus
    bs, st = gs.query(plan, q, margin=0.05, stats=True)
    bf = gf.query(plan, q, margin=1e-2)
    assert torch.equal(bs, bf)
    assert st["n_unresolved"] == 0
    dec = nb.bits_to_numpy(bs, K * NE)
    for o, (idx, z64) in checks.items():
        tie = np.abs(z64 - taus[o]) <= 1e-12 * max(1.0, abs(taus[o]))
        assert np.array_equal(dec[idx][~tie], (z64 >= taus[o])[~tie]), o


def test_cascade_64m_rays_equals_plain(nb):
    """64M world rays against 1,024 objects: the cascade (box/ball -> neural bound ->
    exact) with thresholds calibrated on these rays' own pairs finds exactly the hits of
    the box -> exact path, chunk by chunk; sampled rays against brute force."""
    import torch
    widths = [6, 128, 128, 128, 1]
    K = 1024
    ms = I.make_multi_scene(5000, K, 32)
    ws = nb.WorldScene(ms)
    g = nb.Group(widths, K, infer_prec="f16x3")
    g.set_params(np.stack([(I.init_params(5200 + k, widths) * 3.0).astype(np.float32) for k in range(K)]))
    NR, CH = 64 << 20, 16 << 20
    chunks = [torch.as_tensor(I.sample_world_rays(5300 + c, CH), device="cuda") for c in range(NR // CH)]
    taus = np.full(K, np.inf)
    for ch in chunks:
        off, off_d, pair_ray, pair_q, _ = nb.cascade_bin(ws, ch, canonical=True)
        rows = int(off[-1])
        lab = torch.zeros(nb.n_words(rows), dtype=torch.int32, device="cuda")
        nb.cascade_exact(ws, ch, pair_ray, off_d, rows, pair_hits=lab)
        taus = np.minimum(taus, g.calibrate(nb.Plan(off, chunk_rows=2048), pair_q, lab))
        del off_d, pair_ray, pair_q, lab
    g.tau = taus
    sc_all = I.Scene(ms.centres, ms.radii, None, ms.qexp)
    for c, ch in enumerate(chunks):
        off, off_d, pair_ray, pair_q, _ = nb.cascade_bin(ws, ch, canonical=True)
        neural = g.query(nb.Plan(off, chunk_rows=2048), pair_q, margin=0.05)
        hc = torch.zeros(nb.n_words(CH), dtype=torch.int32, device="cuda")
        nb.cascade_exact(ws, ch, pair_ray, off_d, int(off[-1]), pass_bits=neural, ray_hits=hc)
        del off_d, pair_ray, pair_q, neural
        off, off_d, pair_ray, _, _ = nb.cascade_bin(ws, ch, canonical=False)
        hp = torch.zeros_like(hc)
        nb.cascade_exact(ws, ch, pair_ray, off_d, int(off[-1]), ray_hits=hp)
        assert torch.equal(hc, hp), c
        idx = _sample_idx(CH, 2000, 50 + c)
        rs = ch[torch.as_tensor(idx, device="cuda")].cpu().numpy()
        assert np.array_equal(nb.bits_to_numpy(hp, CH)[idx], O.label(I.RAY3, rs, sc_all).astype(bool))
        del off_d, pair_ray
