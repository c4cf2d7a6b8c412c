"""Host logic of the sweep driver: grouping by temperature, timestep per
temperature, and the retry that drops a molecule whose backbone broke."""
import numpy as np

from paper_1608_03722_gb300 import surrogate as S


def test_sweep_timestep_is_0005_brownian_times_at_the_run_temperature():
    assert S.sweep_dt(1.0) == 0.005
    assert abs(S.sweep_dt(1.4) - 0.005 / 1.4) < 1e-15
    assert S.sweep_dt(0.8) > S.sweep_dt(1.0) > S.sweep_dt(1.4)


def test_broken_molecule_is_rerun_at_half_the_timestep(monkeypatch):
    """A molecule that breaks leaves its group (rerun without it) and is then
    simulated alone at refine = 2; if it breaks again its labels are NaN."""
    pts = np.array([[1.0, 0.0, 500, 1.4], [2.0, 1.0, 600, 1.0], [3.0, -1.0, 700, 1.4], [4.0, 2.0, 800, 1.4],
                    [5.0, 0.5, 900, 1.0]])
    calls = []

    def fake(lengths, loads, kT, seed, steps, measure_from, every, refine=1):
        calls.append((kT, list(lengths), refine))
        bad = [k for k, l in enumerate(lengths) if l == 700 or (l == 900 and refine == 1)]
        if bad:
            return None, bad
        return np.array([[l, f, kT * refine] for l, (f, g) in zip(lengths, loads)], float), None

    monkeypatch.setattr(S, "_run_group", fake)
    out = S.simulate_sweep(pts, steps=10, measure_from=0, every=10)
    assert calls == [(1.0, [600, 900], 1), (1.0, [600], 1), (1.4, [500, 700, 800], 1), (1.4, [500, 800], 1),
                     (1.0, [900], 2), (1.4, [700], 2)]
    assert np.isnan(out[2]).all()
    assert np.array_equal(out[[0, 1, 3, 4]], [[500, 1.0, 1.4], [600, 2.0, 1.0], [800, 4.0, 1.4], [900, 5.0, 2.0]])


def test_metrics_skip_points_without_labels():
    T = np.array([[1.0, 2.0, 3.0], [np.nan, np.nan, np.nan], [2.0, 3.0, 5.0]])
    Y = np.array([[1.0, 2.0, 3.0], [9.0, 9.0, 9.0], [2.0, 3.0, 5.0]])
    m = S._metrics(Y, T)
    assert m["rmse"] == [0.0, 0.0, 0.0] and m["r2"] == [1.0, 1.0, 1.0]
