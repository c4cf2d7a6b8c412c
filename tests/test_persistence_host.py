"""Host logic of the persistence-length measurement (Sec. 3.1, 3.2): the
correlators and fits recover known decay lengths from synthetic chains."""
import math

import numpy as np

from paper_1608_03722_gb300 import persistence as P


def _chain(rng, n, lp, ltau):
    """Centreline with <t(n).t(n+1)> = exp(-1/lp) (random small rotations of the
    tangent) and twist increments theta0 + N(0, 2/ltau) (so <cos DOmega(m)> =
    exp(-m/ltau))."""
    t = np.array([0.0, 0.0, 1.0])
    c = 1.0 - math.exp(-1.0 / lp)                 # 1 - <cos theta> per step
    pts = [np.zeros(3)]
    for _ in range(n - 1):
        a = rng.normal(size=3)
        a -= a.dot(t) * t
        a /= np.linalg.norm(a)
        th = math.acos(1.0 - rng.exponential(c))  # cos(theta) = 1 - Exp(mean c): mean 1 - c
        t = math.cos(th) * t + math.sin(th) * a
        pts.append(pts[-1] + 0.34 * t)
    tw = (P.THETA0 + rng.normal(0.0, math.sqrt(2.0 / ltau), size=n - 2)) / (2.0 * math.pi)
    return np.array(pts), tw


def test_correlators_recover_known_lengths():
    rng = np.random.default_rng(0)
    acc = P.Correlators(groups=4, s_max=120, m_max=150)
    for k in range(800):     # l_tau exceeds the chain: it needs many independent chains
        cen, tw = _chain(rng, 300, 143.0, 512.0)
        acc.add(k % 4, cen, tw, trim=5)
    r = acc.result((1, 100), (1, 150))
    assert abs(r["l_p_bp"] - 143.0) < 0.06 * 143.0, r["l_p_bp"]
    assert abs(r["l_tau_bp"] - 512.0) < 0.08 * 512.0, r["l_tau_bp"]
    assert abs(r["twist_per_bp_deg"] - 36.0) < 0.1
    assert r["l_p_err_bp"] > 0 and r["l_tau_err_bp"] > 0


def test_fit_of_an_exact_exponential():
    k = np.arange(200)
    assert abs(P._fit_decay(np.exp(-k / 77.0), 1, 150) - 77.0) < 1e-9
