"""Host logic of the sweep driver: grouping by temperature, timestep per
temperature, and the retry that drops a molecule whose backbone broke."""
import numpy as np

from paper_1608_03722_gb300 import surrogate as S


def test_sweep_timestep_is_0005_brownian_times_at_the_run_temperature():
    assert S.sweep_dt(1.0) == 0.005
    assert abs(S.sweep_dt(1.4) - 0.005 / 1.4) < 1e-15
    assert S.sweep_dt(0.8) > S.sweep_dt(1.0) > S.sweep_dt(1.4)


def test_broken_molecule_gets_nan_and_its_group_reruns_without_it(monkeypatch):
    pts = np.array([[1.0, 0.0, 500, 1.4], [2.0, 1.0, 600, 1.0], [3.0, -1.0, 700, 1.4], [4.0, 2.0, 800, 1.4]])
    calls = []

    def fake(lengths, loads, kT, seed, steps, measure_from, every):
        calls.append((kT, list(lengths)))
        if kT == 1.4 and 700 in lengths:
            return None, [lengths.index(700)]
        return np.array([[l, f, kT] for l, (f, g) in zip(lengths, loads)], float), None

    monkeypatch.setattr(S, "_run_group", fake)
    out = S.simulate_sweep(pts, steps=10, measure_from=0, every=10)
    assert calls == [(1.0, [600]), (1.4, [500, 700, 800]), (1.4, [500, 800])]
    assert np.isnan(out[2]).all()
    assert np.array_equal(out[[0, 1, 3]], [[500, 1.0, 1.4], [600, 2.0, 1.0], [800, 4.0, 1.4]])


def test_metrics_skip_points_without_labels():
    T = np.array([[1.0, 2.0, 3.0], [np.nan, np.nan, np.nan], [2.0, 3.0, 5.0]])
    Y = np.array([[1.0, 2.0, 3.0], [9.0, 9.0, 9.0], [2.0, 3.0, 5.0]])
    m = S._metrics(Y, T)
    assert m["rmse"] == [0.0, 0.0, 0.0] and m["r2"] == [1.0, 1.0, 1.0]
