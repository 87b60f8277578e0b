"""Split-FP16 tcgen05 forward (NB_F16X3) against the FP64 oracle: logits within 2e-2
absolute (in practice a few FP32 roundings of the scale), decisions bit-exact with the
margin band re-checked, ragged sizes across several tiles, both hidden widths."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_06822_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NETS = [("ray3", [6, 128, 128, 128, 128, 1]), ("point3", [3, 128, 128, 128, 128, 1]),
        ("ray3", [6, 128, 128, 128, 1]), ("point4t", [4, 64, 64, 64, 1]), ("plane3", [4, 64, 64, 1]),
        # the paper's own network sizes (25, 50, 75 wide), run zero-padded to 64 / 128
        ("point2", [2, 25, 25, 1]), ("point3", [3, 50, 50, 1]), ("ray3", [6, 50, 50, 1]),
        ("point4t", [4, 75, 75, 1])]


@pytest.fixture(scope="module")
def nb():
    from paper_2310_06822_gb300 import nb as _nb
    _nb.lib()
    return _nb


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


@pytest.mark.parametrize("kind,widths", NETS)
@pytest.mark.parametrize("n", [1, 127, 129, 300_007])
def test_split_logits_and_decisions(nb, kind, widths, n):
    p = I.init_params(50 + n % 7, widths)
    # scale the weights up so logits span tens of units, like trained networks
    p = (p * 3.0).astype(np.float32)
    m = nb.Model(widths, infer_prec="f16x3")
    m.set_params(p)
    q = I.sample_queries(kind, 60 + n, n)
    z64 = O.forward(widths, p, q)
    tau = float(np.quantile(z64, 0.4)) if n > 1 else 0.0
    m.tau = tau
    bits, z, st = m.query(_dev(q), margin=0.05, logits=True, stats=True)
    z = z.cpu().numpy().astype(np.float64)
    S = O.forward_scale(widths, p, q)
    assert np.max(np.abs(z - z64)) <= 2e-2
    assert np.max(np.abs(z - z64) / np.maximum(np.abs(z64), S)) <= 1e-4
    dec = nb.bits_to_numpy(bits, n)
    tie = np.abs(z64 - tau) <= 1e-12 * max(1.0, abs(tau))
    assert np.array_equal(dec[~tie], (z64 >= tau)[~tie])
    assert st["n_unresolved"] <= int(tie.sum())


def test_split_matches_fp32_form_at_full_size(nb):
    """16M rays in the launch configuration the benchmark times: decisions equal the FP32
    form's (both certified by the re-check), sampled logits against the oracle."""
    import torch
    widths = [6, 128, 128, 128, 128, 1]
    p = (I.init_params(77, widths) * 3.0).astype(np.float32)
    n = 16 << 20
    q = I.sample_queries("ray3", 78, n)
    qd = _dev(q)
    ms = nb.Model(widths, infer_prec="f16x3")
    ms.set_params(p)
    mf = nb.Model(widths)
    mf.set_params(p)
    idx = np.random.default_rng(1).choice(n, 20000, replace=False)
    z64 = O.forward(widths, p, q[idx])
    tau = float(np.quantile(z64, 0.6))
    ms.tau = tau
    mf.tau = tau
    bs, zs = ms.query(qd, margin=0.05, logits=True)
    bf = mf.query(qd, margin=0.05)
    assert torch.equal(bs, bf)
    assert np.max(np.abs(zs.cpu().numpy()[idx].astype(np.float64) - z64)) <= 2e-2


@pytest.mark.parametrize("widths,kind", [([3, 50, 50, 1], "point3"), ([6, 75, 75, 75, 1], "ray3")])
def test_padded_narrow_network_bf16_and_training(nb, widths, kind):
    """A 50- or 75-wide network on the BF16 forward (zero-padded to 64 / 128): decisions
    equal the oracle's once the band is re-checked, and parameter updates reach the padded
    copy; BF16 training needs the kernels' own widths, FP32 training takes any width."""
    p = (I.init_params(91, widths) * 3.0).astype(np.float32)
    m = nb.Model(widths, infer_prec="bf16")
    m.set_params(p)
    n = 50_001
    q = I.sample_queries(kind, 92, n)
    for step in range(2):
        z64 = O.forward(widths, m.get_params(), q)
        tau = float(np.quantile(z64, 0.5))
        m.tau = tau
        bits, z = m.query(_dev(q), margin=0.5, logits=True)
        assert np.max(np.abs(z.cpu().numpy() - z64)) <= 0.25
        tie = np.abs(z64 - tau) <= 1e-12 * max(1.0, abs(tau))
        assert np.array_equal(nb.bits_to_numpy(bits, n)[~tie], (z64 >= tau)[~tie])
        # one FP32 training step moves the weights; the padded copy follows
        y = _dev(I.pack_bits(z64 >= tau).view(np.int32))
        m.train_step(_dev(q[:4096]), y[:128], 2.0)
    with pytest.raises(nb.NBError):
        nb.Model(widths, train_prec="bf16")


@pytest.mark.parametrize("chunk_rows,pinned", [(0, True), (0, False), (4096, True), (100_000, False)])
def test_query_from_host_memory_equals_device_query(nb, chunk_rows, pinned):
    """nb_query_host reads pinned host queries in place over the coherent host link (chunk
    0) or streams them through two staging chunks (copy on one stream, decide on another):
    bits and statistics equal those of one device-side nb_query either way."""
    import torch
    widths = [6, 128, 128, 128, 128, 1]
    p = (I.init_params(95, widths) * 3.0).astype(np.float32)
    m = nb.Model(widths, infer_prec="f16x3")
    m.set_params(p)
    n = 300_007
    q = I.sample_queries("ray3", 96, n)
    m.tau = float(np.quantile(O.forward(widths, p, q[:5000]), 0.5))
    ref, st_ref = m.query(_dev(q), margin=0.05, stats=True)
    hq = torch.as_tensor(q)
    if pinned:
        hq = hq.pin_memory()
    bits, st = m.query_host(hq, margin=0.05, stats=True, chunk_rows=chunk_rows)
    assert np.array_equal(bits.numpy(), ref.cpu().numpy())
    assert st == st_ref
    # the empty call
    assert m.query_host(hq[:0]).numel() == 0
