"""The stepwise asymmetry schedule (Suppl. "Weight schedule"): host logic of the library,
pinned by a hand-worked sequence of windows.  Runs on CPU only."""
import pytest


@pytest.fixture(scope="module")
def nb():
    from paper_2310_06822_gb300 import nb as _nb
    _nb.lib()
    return _nb


def test_hand_worked_windows(nb):
    s = nb.Stepwise(dim=3, period=3, stop_windows=2)
    assert (s.alpha, s.beta, s.period) == (1.0, 1.0, 3)
    # a window with false negatives: first adjustment, alpha 1 + 0.2, beta 1 / 100
    assert s.window(5) is False
    assert s.adjustments == 1 and s.alpha == pytest.approx(1.2) and s.beta == pytest.approx(0.01)
    # a clean window changes nothing
    assert s.window(0) is False
    assert s.alpha == pytest.approx(1.2) and s.beta == pytest.approx(0.01)
    # false negatives again: second adjustment, and the clean count restarts
    assert s.window(7) is False
    assert s.adjustments == 2 and s.alpha == pytest.approx(1.4) and s.beta == pytest.approx(0.005)
    assert s.window(0) is False
    # the second consecutive clean window ends training
    assert s.window(0) is True


@pytest.mark.parametrize("dim,rate", [(2, 20), (3, 100), (4, 200)])
def test_rates_per_dimension_and_growing_asymmetry(nb, dim, rate):
    s = nb.Stepwise(dim=dim)
    ratios = []
    for k in range(1, 6):
        assert s.window(1) is False  # never stops while false negatives remain
        assert s.beta == pytest.approx(1.0 / (rate * k))
        assert s.alpha == pytest.approx(1.0 + 0.2 * k)
        ratios.append(s.alpha / s.beta)
    assert all(b > a for a, b in zip(ratios, ratios[1:]))
    # stop_windows = 0: clean windows never end training
    assert not any(s.window(0) for _ in range(10))


def test_rejects_bad_arguments(nb):
    with pytest.raises(nb.NBError):
        nb.Stepwise(dim=3, period=0)
    with pytest.raises(nb.NBError):
        nb.Stepwise(dim=3, fn_step=-1.0)
    with pytest.raises(nb.NBError):
        nb.Stepwise(dim=3, stop_windows=-1)
