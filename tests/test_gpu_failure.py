"""Failure detection without a fault: a bounded device wait that nothing completes gives
up, the library reports NB_ETIMEOUT, and the context stays usable for the next query."""
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


def test_bounded_wait_gives_up_and_the_context_stays_usable(nb):
    import torch
    for polls in (1, 1000):
        assert nb.selftest_bounded_wait(polls) == 4  # NB_ETIMEOUT
    widths = [6, 128, 128, 1]
    p = (I.init_params(5, widths) * 3.0).astype(np.float32)
    m = nb.Model(widths, infer_prec="f16x3")
    m.set_params(p)
    q = I.sample_queries("ray3", 6, 10_000)
    z64 = O.forward(widths, p, q)
    m.tau = float(np.median(z64))
    bits = m.query(torch.as_tensor(q, device="cuda"), margin=0.05)
    m.check()  # no wait of the forward gave up
    tie = np.abs(z64 - m.tau) <= 1e-12 * max(1.0, abs(m.tau))
    assert np.array_equal(nb.bits_to_numpy(bits, len(q))[~tie], (z64 >= m.tau)[~tie])
