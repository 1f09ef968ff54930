"""Three-dimensional variant on the GPU against the FP64 all-pairs oracle
(orc3_*, pinned to the 2D oracle by planar embedding).  Bounds as in 2D:
forces ||dF|| / ||F|| <= 1e-5 and max_i |dF_i| <= 1e-5 max(|F_i|, F_rms);
positions after 100 steps within 1e-4."""
import math

import numpy as np
import pytest

from paper_1310_0998_gb300 import synth

pytestmark = pytest.mark.gpu

BASE = dict(a=25.0, gamma=4.5, kBT=1.0, rc=1.0, kbond=100.0, r0=0.5, fp=1.0, zeta=0.1, dt=0.01)


def _kw(**kw):
    p = dict(BASE)
    p.update(kw)
    return dict(a=p["a"], gamma=p["gamma"], kBT=p["kBT"], rc=p["rc"], k_bond=p["kbond"], r0=p["r0"], f_p=p["fp"],
                zeta=p["zeta"], dt=p["dt"], seed=p.get("seed", 0), wexp=p.get("wexp", 0.0))


def _op(orc, L, **kw):
    p = dict(BASE)
    p.update(kw)
    return orc.params(L=L, **p)


def _check(f, fo):
    fn = np.linalg.norm(fo, axis=1)
    frms = math.sqrt(float(np.mean(fn ** 2)))
    err = np.linalg.norm(f.astype(np.float64) - fo, axis=1)
    assert np.linalg.norm(err) / np.linalg.norm(fo) <= 1e-5
    assert np.max(err / np.maximum(fn, frms)) <= 1e-5


@pytest.fixture(scope="module")
def Sim3():
    import torch
    assert torch.cuda.is_available()
    from paper_1310_0998_gb300 import Sim3
    return Sim3


@pytest.mark.parametrize("L,nd,seed,wexp", [(6.0, 324, 1, 0.0), (7.5, 630, 2, 0.0), (3.5, 64, 3, 0.0),
                                            (6.0, 324, 4, 0.5)])
def test_setup_force_parity(Sim3, orc, L, nd, seed, wexp):
    x, _ = synth.dimers3(nd, L, 0.5, seed=seed)
    v = synth.velocities3(2 * nd, 1.0, seed=seed + 10)
    with Sim3(L, 2 * nd, **_kw(seed=seed, wexp=wexp)) as s:
        s.set_positions(x, v, step=5)
        xg, vg, f, st = s.get_state()
    assert st == 5
    np.testing.assert_array_equal(xg, x)
    fo, npairs = orc.forces3(_op(orc, L, seed=seed, wexp=wexp), x, v.astype(np.float64), 5)
    assert npairs > 0
    _check(f, fo)


def test_trajectory_parity_100_steps(Sim3, orc):
    L, nd = 6.0, 324
    x, v = synth.dimers3(nd, L, 0.5, seed=5)
    with Sim3(L, 2 * nd, **_kw(seed=6)) as s:
        s.set_positions(x, v)
        s.step(100)
        xg, vg, _, st = s.get_state()
    assert st == 100
    o = orc.State3(_op(orc, L, seed=6), x, v)
    o.run(100)
    d = xg - o.x
    d -= L * np.rint(d / L)
    assert np.abs(d).max() <= 1e-4, np.abs(d).max()
    assert np.abs(vg - o.v).max() <= 2e-2


def test_thermo_and_momentum(Sim3):
    L, nd = 6.0, 324
    x, _ = synth.dimers3(nd, L, 0.5, seed=7)
    v = synth.velocities3(2 * nd, 1.0, seed=8)
    with Sim3(L, 2 * nd, **_kw(seed=9, zeta=0.0, fp=0.0)) as s:
        s.set_positions(x, v)
        P0 = v.astype(np.float64).sum(axis=0)
        s.step(500)
        _, vg, _, _ = s.get_state()
        th = s.thermo()
    vv = vg.astype(np.float64)
    ke = 0.5 * np.sum(vv * vv)
    assert abs(th[0] - ke) <= 1e-6 * ke
    np.testing.assert_allclose(th[1:4], vv.sum(axis=0), atol=1e-4 * np.abs(vv).sum())
    np.testing.assert_allclose(th[1:4], P0, atol=2e-3 * np.abs(vv).sum())   # momentum conserved (FP32 sums)
    assert th[4] == pytest.approx(2 * ke / (3 * 2 * nd - 3), rel=1e-6)


def test_equilibrium_temperature(Sim3):
    L, nd = 8.0, 768
    x, v = synth.dimers3(nd, L, 0.5, seed=10)
    T = []
    with Sim3(L, 2 * nd, **_kw(seed=11, zeta=0.0, fp=0.0)) as s:
        s.set_positions(x, v)
        s.step(2000)
        for _ in range(200):
            s.step(50)
            T.append(s.thermo()[4])
    assert abs(np.mean(T) - 1.0) < 0.02, np.mean(T)


def test_nonfinite_input_reported(Sim3):
    from paper_1310_0998_gb300._lib import DpdError
    L, nd = 6.0, 100
    x, v = synth.dimers3(nd, L, 0.5, seed=12)
    x[3, 1] = np.nan
    with Sim3(L, 2 * nd) as s:
        with pytest.raises(DpdError) as e:
            s.set_positions(x, v)
        assert e.value.status == -4
