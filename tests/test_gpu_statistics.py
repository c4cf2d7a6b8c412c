"""Statistical agreement of the mixed-precision engine with the FP64 oracle.

Trajectories of the two diverge after a few hundred steps (chaos), so beyond
that the comparison is between ensembles: the oracle's statistics are stored
in tests/golden/oracle_tethered_stats.txt (written by
tests/golden/make_oracle_stats.py, which runs only the oracle), and the
engine runs the same protocol with other noise.  A tethered 300 bp molecule
is pulled with 5 kT/nm and twisted with 2 kT about z (Sec. 4.1-4.2) from a
relaxed straight start; per replica the extension R_z (Sec. 4.1), the excess
twist Tw - Tw_relaxed (Sec. 3.2) and the denatured fraction (Sec. 5) are
averaged over samples every 100 steps from step 10^4 to 6 x 10^4.  The
replica means of engine and oracle must agree within three combined
standard errors, at the paper's hydrogen-bond stiffness (K2 = 6) and at
K2 = 2, where a few percent of the base pairs are open at any time.
"""
import numpy as np
import pytest

from paper_1608_03722_gb300 import dsdna as D
from paper_1608_03722_gb300 import inputs as I
from tests.conftest import read_golden

pytestmark = pytest.mark.gpu

REPLICAS = 128


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    yield


@pytest.mark.parametrize("cond", ["k2_6", "k2_2"])
def test_tethered_ensemble_agrees_with_the_oracle(cond):
    g = read_golden("oracle_tethered_stats.txt")
    n_bp, steps, start, every = int(g["n_bp"]), int(g["steps"]), int(g["from"]), int(g["every"])
    f, tq, k2 = float(g["force"]), float(g["torque"]), float(g[cond + ".K2"])
    X, u = I.straight_helix(n_bp)
    Xs = np.concatenate([X] * REPLICAS)
    us = np.concatenate([u] * REPLICAS)
    p = D.dsdna_default_params(K2=k2, seed=777)
    ctx = D.Context(p, [n_bp] * REPLICAS, X=Xs, u=us, tether=[1] * REPLICAS)   # Maxwell-Boltzmann start
    ctx.set_external_force_torque(-1, [0.0, 0.0, f], [0.0, 0.0, tq])
    acc = np.zeros((REPLICAS, 3))
    ns, done = 0, 0
    while done < steps:
        ctx.step(every)
        done += every
        if done >= start:
            for m in range(REPLICAS):
                o = ctx.observables(m, D.OBS_EXT | D.OBS_DENAT | D.OBS_TW)
                acc[m] += (o["rz"], o["tw"] - o["tw_ideal"], o["denat"])
            ns += 1
    ctx.close()
    acc /= ns
    print()
    for j, name in enumerate(("rz", "dtw", "denat")):
        mg, sg = acc[:, j].mean(), acc[:, j].std(ddof=1) / np.sqrt(REPLICAS)
        mo, so = float(g[f"{cond}.{name}_mean"]), float(g[f"{cond}.{name}_se"])
        z = abs(mg - mo) / np.hypot(sg, so)
        print(f"{cond} {name}: engine {mg:.5g} +- {sg:.2g}, oracle {mo:.5g} +- {so:.2g}, {z:.2f} combined SE")
        assert z < 3.0, (cond, name, mg, sg, mo, so)
    if cond == "k2_2":
        assert float(g["k2_2.denat_mean"]) > 0.005      # the comparison sees open base pairs
