"""Host-side analysis of the mixing experiment (Sec. 4: max g(r) against
force evaluations, fitted by a + b exp(-x / tau)): the fits recover the
parameters of exact exponentials, and the speed-ups are ratios of the fitted
relaxation times."""
import numpy as np
import pytest

from paper_2005_08348_gb300 import mixing

pytest.importorskip("scipy")


def _curve(a, b, tau, n=40, x1=4e5):
    x = np.linspace(0.0, x1, n)
    return x, a + b * np.exp(-x / tau)


def test_exp_fit_recovers_exact_exponentials():
    for a, b, tau in ((1.05, 0.9, 6e4), (1.2, 2.5, 1.5e5), (0.98, 0.3, 2e4)):
        x, y = _curve(a, b, tau)
        f = mixing.exp_fit(x, y)
        assert f is not None
        assert f["a"] == pytest.approx(a, rel=1e-6) and f["b"] == pytest.approx(b, rel=1e-6)
        assert f["tau"] == pytest.approx(tau, rel=1e-6)
    assert mixing.exp_fit([0, 1, 2], [1, 2, 3]) is None          # too few points


def test_exp_fit_with_a_given_plateau():
    x, y = _curve(1.1, 1.4, 8e4)
    f = mixing.exp_fit_plateau(x, y, 1.1)
    assert f["tau"] == pytest.approx(8e4, rel=1e-6) and f["b"] == pytest.approx(1.4, rel=1e-6)


def test_speedups_are_ratios_of_relaxation_times():
    taus = dict(md=3e5, mcmd=6e4, mdas=1e5)
    res = {}
    for k, tau in taus.items():
        x, y = _curve(1.05, 1.0, tau, n=60, x1=2e6)
        res[k] = dict(force_evaluations=x, max_g=y, fit=mixing.exp_fit(x, y))
    s = mixing.speedups(res)
    assert s["free_fit"]["mcmd"] == pytest.approx(5.0, rel=1e-5)
    assert s["free_fit"]["mdas"] == pytest.approx(3.0, rel=1e-5)
    cp = s["common_plateau"]
    assert cp["plateau"] == pytest.approx(1.05, rel=1e-6)
    assert cp["speedup"]["mcmd"] == pytest.approx(5.0, rel=1e-5)
