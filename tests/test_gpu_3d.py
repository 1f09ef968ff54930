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
    # momentum conserved: the fixed-point pair sums cancel exactly, what is
    # left is the FP32 rounding of each bead's kick
    np.testing.assert_allclose(th[1:4], P0, atol=1e-5 * np.abs(vv).sum())
    assert th[4] == pytest.approx(2 * ke / (3 * 2 * nd - 3), rel=1e-6)


def test_reproducible_bit_for_bit(Sim3):
    """Fixed-point force sums: two runs from the same state give the same
    bits, although the in-cell order of the counting sort (atomic tickets),
    and so the order in which pairs are met, differs from run to run."""
    L, nd = 8.0, 768
    x, v = synth.dimers3(nd, L, 0.5, seed=12)
    out = []
    for _ in range(2):
        with Sim3(L, 2 * nd, **_kw(seed=13)) as s:
            s.set_positions(x, v)
            s.step(200)
            out.append(s.get_state())
    for a, b in zip(out[0][:3], out[1][:3]):
        np.testing.assert_array_equal(a, b)


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


# ------------------------------------------------------------ observables
def _state3(L, nd, seed):
    x, _ = synth.dimers3(nd, L, 0.5, seed=seed)
    v = synth.velocities3(2 * nd, 1.0, seed=seed + 10)
    return x, v


@pytest.mark.parametrize("L,nd,M,eps", [(6.0, 324, 8, 0.0), (7.5, 630, 16, 0.0), (10.0, 1500, 16, 2.0),
                                        (9.0, 1000, 5, 0.0)])
def test_field_spectrum_vorticity_parity(Sim3, L, nd, M, eps):
    """Window counts exact, field, E(k) and curl to rounding order against the
    FP64 oracle on the same canonical state (odd M: field and curl only)."""
    from oracle import observables as ob
    x, v = _state3(L, nd, 31)
    with Sim3(L, 2 * nd, **_kw()) as s:
        s.set_positions(x, v)
        s.step(3)
        xg, vg, _, _ = s.get_state()
        u, n = s.velocity_field(M, eps)
        E = s.energy_spectrum(M, eps) if M & (M - 1) == 0 else None
        om = s.vorticity(M, eps)
    c, vc = ob.agent_com(xg, vg, L)
    e = eps if eps > 0 else ob.filter_width3(L, nd)
    uo, no = ob.velocity_field3(c, vc, L, M, e)
    np.testing.assert_array_equal(n, no)
    np.testing.assert_allclose(u, uo, rtol=1e-10, atol=1e-12)
    if E is not None:
        Eo = ob.energy_spectrum3(uo)
        np.testing.assert_allclose(E, Eo, rtol=1e-9, atol=1e-15 * Eo.max())
    oo = ob.vorticity3(uo, L)
    np.testing.assert_allclose(om, oo, rtol=1e-9, atol=1e-10 * np.abs(oo).max())


@pytest.mark.parametrize("L,nd,dr,nbins", [
    (6.0, 324, 0.25, 12), (10.0, 1500, 0.5, 20), (8.0, 2000, 0.2, 40),      # r_max >= L/3: all agent pairs
    (10.0, 1500, 0.25, 12), (16.0, 4000, 0.3, 10),                          # cell grids of 3^3 and 5^3
    (12.0, 3000, 0.2, 19)])                                                  # 3^3, r_max not a cell multiple
def test_velocity_correlation_parity(Sim3, L, nd, dr, nbins):
    from oracle import observables as ob
    x, v = _state3(L, nd, 32)
    with Sim3(L, 2 * nd, **_kw()) as s:
        s.set_positions(x, v)
        s.step(3)
        xg, vg, _, _ = s.get_state()
        g, Li, num, cnt = s.velocity_correlation(dr, nbins)
    c, vc = ob.agent_com(xg, vg, L)
    go, Lo, numo, cnto = ob.velocity_correlation3(c, vc, L, dr, nbins)
    np.testing.assert_array_equal(cnt, cnto)
    np.testing.assert_allclose(num, numo, rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(g, go, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(Li, Lo, rtol=1e-8, atol=1e-10)


def test_observables_at_density_3(Sim3):
    """Cube of side 32 at density 3 (49,152 agents): E(k) on 32^3 against the
    oracle, and the pair counts of the first 16 shells of 0.25 (the cell-grid
    pass, 8^3 cells) against an exact CPU count (periodic k-d tree
    candidates, shells by the same FP64 expressions)."""
    spatial = pytest.importorskip("scipy.spatial")
    from oracle import observables as ob
    L, nd, M = 32.0, 3 * 32 ** 3 // 2, 32
    x, v = _state3(L, nd, 33)
    with Sim3(L, 2 * nd, **_kw()) as s:
        s.set_positions(x, v)
        s.step(5)
        xg, vg, _, _ = s.get_state()
        E = s.energy_spectrum(M)
        g, Li, num, cnt = s.velocity_correlation(0.25, 16)
    c, vc = ob.agent_com(xg, vg, L)
    uo, _ = ob.velocity_field3(c, vc, L, M, ob.filter_width3(L, nd))
    np.testing.assert_allclose(E, ob.energy_spectrum3(uo), rtol=1e-9)
    pairs = spatial.cKDTree(c, boxsize=L).query_pairs(4.0 + 1e-6, output_type="ndarray")
    d = c[pairs[:, 0]] - c[pairs[:, 1]]
    d -= L * np.rint(d / L)
    b = np.floor(np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]) / 0.25)
    keep = b < 16
    np.testing.assert_array_equal(cnt, np.bincount(b[keep].astype(np.int64), minlength=16)[:16])
    dots = (vc[pairs[keep, 0]] * vc[pairs[keep, 1]]).sum(-1)
    np.testing.assert_allclose(num, np.bincount(b[keep].astype(np.int64), weights=dots, minlength=16)[:16],
                               rtol=1e-9, atol=1e-9 * np.abs(dots).sum())
    assert np.isfinite(Li)
