"""Host logic of the single-molecule experiments (Sec. 4.1-4.2): the fits of
Eq. 5 and Eq. 7 recover known parameters from synthetic data."""
import math

import numpy as np
import pytest

from paper_1608_03722_gb300 import mechanics as M


def test_wlc_fit_recovers_length_and_persistence():
    pytest.importorskip("scipy")
    rng = np.random.default_rng(0)
    L, lp = 100.3, 47.0
    x = np.linspace(0.3, 0.93, 12)
    F = M.wlc_force(x, lp)
    Rz = x * L * (1.0 + rng.normal(0.0, 1e-3, size=x.size))
    Lf, lpf, eL, elp = M.fit_wlc(F, Rz, 102.0)
    assert abs(Lf - L) < 0.01 * L and abs(lpf - lp) < 0.05 * lp, (Lf, lpf)
    assert eL > 0 and elp > 0


def test_wlc_force_limits():
    """Eq. 5: zero force at zero extension, divergence as x -> 1, and the
    small-extension slope 3 kT / (2 l_p L) (Gaussian chain)."""
    assert M.wlc_force(np.array([0.0]), 50.0)[0] == 0.0
    assert M.wlc_force(np.array([0.999]), 50.0)[0] > 1e3
    x = 1e-4
    assert abs(M.wlc_force(np.array([x]), 50.0)[0] / x - 1.5 / 50.0) < 1e-3


def test_torsion_fit_recovers_C():
    C = 88.0
    slope = C / (M.A0 / M.THETA0)                 # dGamma/dsigma in kT
    sigma = np.linspace(-0.02, 0.02, 7)
    gamma = slope * sigma + 0.1
    Cf, eC = M.fit_torsion(gamma, sigma)
    assert abs(Cf - C) < 1e-9 * C and eC < 1e-6
    assert abs(M.A0 / M.THETA0 - 0.34 / (2 * math.pi / 10)) < 1e-15
