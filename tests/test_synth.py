"""The seeded workload generators: parameter grids and ranges of the sweep
(256 x 256 box), the uneven-replica distribution and the fixed-point grid."""
import numpy as np

from paper_1310_0998_gb300 import synth


def test_sweep_points_cover_the_grid():
    pts = synth.sweep_points()
    assert len(pts) == 6 * 3 * 3
    grid = {(p["phi"], p["gamma"], p["zeta"]) for p in pts}
    assert grid == {(f, g, z) for f in (0.1, 0.2, 0.3, 0.4, 0.5, 0.6) for g in (1.0, 4.5, 20.0)
                    for z in (0.01, 0.1, 1.0)}
    for p in pts:
        assert p["L"] == 256.0 and p["fp"] == 1.0
        # area fraction reading: N_d = 2 phi L^2 (r_h = r_c / 4, l = 1)
        assert p["n_dimers"] == round(2.0 * p["phi"] * 256.0 ** 2)
    assert max(p["n_dimers"] for p in pts) <= 3 * 256 * 256 // 2


def test_ensemble_points_ranges():
    pts = synth.ensemble_points(256, seed=0)
    for p in pts:
        assert 32.0 <= p["L"] <= 192.0 and p["L"] * 256.0 == int(p["L"] * 256.0)
        assert 0.05 <= p["phi"] <= 0.6 and 0.5 <= p["gamma"] <= 50.0
        assert 0.005 <= p["zeta"] <= 2.0 and 0.5 <= p["fp"] <= 2.0
    assert synth.ensemble_points(8, seed=3) == synth.ensemble_points(8, seed=3)


def test_on_grid_is_exact():
    L = 37.0
    x = synth.on_grid(np.random.default_rng(0).random((100, 2)) * L, L)
    X = x / L * 2.0 ** 32
    assert np.all(X == np.rint(X)) and np.all((x >= 0) & (x < L))
