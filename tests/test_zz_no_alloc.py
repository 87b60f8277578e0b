"""nb_train_step_noalloc, the training step that allocates nothing, against
nb_train_step through the C ABI.

Callers that cannot call cudaMalloc (device memory reserved up front by another
allocator, or training loops that must not take the device-wide synchronisation of
an allocation) use this variant; it keeps its gradient partials in a static device
array instead of a growable workspace.  Two calls in a row must give what the
regular entry point gives, within the tolerances of the other training tests
(gradient 1e-4 relative per tensor, loss 1e-5 relative), and leave the device's free
memory and PyTorch's reserved memory unchanged.  With a tensor-core inference precision
the step also refreshes the model's low-precision weight images from the updated FP32
weights, which the fast-path logits then reflect.  This file is collected last, so a
run that stops at its first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_06822_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _per_tensor(widths):
    out, off = [], 0
    for l in range(len(widths) - 1):
        nW = widths[l + 1] * widths[l]
        out.append((off, off + nW))
        out.append((off + nW, off + nW + widths[l + 1]))
        off += nW + widths[l + 1]
    return out


def _noalloc_step(nb, m, q, bits, alpha, beta, st):
    import torch
    lib = nb.lib()
    rc = lib.nb_train_step_noalloc(m._h, ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(bits.data_ptr()),
                                   q.shape[0], ctypes.c_float(alpha), ctypes.c_float(beta),
                                   ctypes.c_void_p(st.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.nb_last_error()


@pytest.mark.parametrize("kind,widths,n,infer", [("point2", [2, 32, 32, 32, 1], 1024, "f32"),
                                                 ("ray3", [6, 128, 128, 128, 128, 1], 65536, "f32"),
                                                 ("point2", [2, 32, 32, 32, 1], 1024, "f16x3"),
                                                 ("ray3", [6, 128, 128, 128, 128, 1], 65536, "f16x3")])
def test_noalloc_step_matches_regular_step(kind, widths, n, infer):
    import torch
    from paper_2310_06822_gb300 import nb
    kid = I.kind_id(kind)
    sc = I.make_scene(71, 16, 2 if kid == I.POINT2 else 3, 0.1, 0.4)
    p0 = I.init_params(72, widths)
    reg, na = nb.Model(widths, infer_prec=infer), nb.Model(widths, infer_prec=infer)
    reg.set_params(p0)
    na.set_params(p0)
    eq = torch.as_tensor(I.sample_queries(kind, 79, 4096), device="cuda")
    for step in range(2):
        q = I.sample_queries(kind, 73 + step, n)
        y = O.label(kid, q, sc)
        qd = torch.as_tensor(q, device="cuda")
        bd = torch.as_tensor(I.pack_bits(y).view(np.int32), device="cuda")
        st_r, st_n = nb.step_stats_tensor(), nb.step_stats_tensor()
        alpha = 1.0 + 49.0 * step
        reg.train_step(qd, bd, alpha, 1.0, stats=st_r)
        torch.cuda.synchronize()
        p_before = na.get_params()
        free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
        _noalloc_step(nb, na, qd, bd, alpha, 1.0, st_n)
        torch.cuda.synchronize()
        # nothing was allocated: torch's pool is unchanged, and so is the device's free
        # memory from the second call on (the first call on a device looks up the static
        # array's address, which under lazy module loading also loads the library module
        # that holds the array)
        assert torch.cuda.memory_reserved() == reserved0
        if step > 0:
            assert torch.cuda.mem_get_info()[0] == free0
        gr, gn = reg.get_grad().astype(np.float64), na.get_grad().astype(np.float64)
        for a, b in _per_tensor(widths):
            den = max(np.linalg.norm(gr[a:b]), 1e-30)
            assert np.linalg.norm(gn[a:b] - gr[a:b]) / den <= 1e-4
        sr, sn = nb.read_step_stats(st_r), nb.read_step_stats(st_n)
        assert abs(sn["loss"] - sr["loss"]) <= 1e-5 * abs(sr["loss"])
        assert sn["fn"] == sr["fn"] and sn["fp"] == sr["fp"]
        # Adam's first steps move each weight by about lr sign(g); compare the updated
        # weights wherever the gradient is not at rounding level
        pr, pn = reg.get_params(), na.get_params()
        sig = np.abs(gr) > 1e-3 * np.sqrt(np.mean(gr ** 2))
        assert np.max(np.abs(pn[sig] - pr[sig])) <= 2e-6
        assert np.mean(sig) > 0.5
        if infer != "f32":
            # the fast path's weight images were rebuilt from the updated weights: its
            # logits follow the oracle on the new parameters (split FP16 keeps them within
            # 1e-3 here), not the old ones, which differ by far more
            _, z = na.query(eq, logits=True)
            e_np = eq.cpu().numpy()
            z_new = O.forward(widths, pn, e_np)
            z_old = O.forward(widths, p_before, e_np)
            assert np.max(np.abs(z.cpu().numpy() - z_new)) <= 1e-3
            assert np.max(np.abs(z_new - z_old)) > 1e-2
        # the next call starts from the same state, so it checks the entry point again on
        # equal inputs (and that it clears what the previous call left in the array)
        na.set_state(reg.get_state())

