"""GPU parity of the simulation hot path against the FP64 oracle.

Tolerances (written here, from the hot path's stated parity bounds):
  forces at identical input state: ||F_gpu - F_orc|| / ||F_orc|| <= 1e-5 and
    max_i |dF_i| <= 1e-5 * max(|F_i|, F_rms);
  positions after 100 steps (C1): max |minimg(x_gpu - x_orc)| <= 1e-4;
  cell counts and neighbour counts: bit-exact (pairs within 4e-6 r_c^2 of
    the cutoff, where FP32 and FP64 may decide differently, are excluded).
Inputs come from the seeded generator on the fixed-point grid X L / 2^32, so
the simulator holds exactly the positions the oracle reads.
"""
import math

import numpy as np
import pytest

from paper_1310_0998_gb300 import synth

pytestmark = pytest.mark.gpu

C1 = dict(a=25.0, gamma=4.5, kBT=1.0, rc=1.0, kbond=100.0, r0=0.5, fp=1.0, zeta=0.1, dt=0.01, mass=1.0)


@pytest.fixture(scope="module")
def Sim():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1310_0998_gb300 import Sim
    return Sim


def oparams(orc, L, seed=0, **kw):
    p = dict(C1)
    p.update(kw)
    return orc.params(L=L, seed=seed, **p)


def sim_kw(seed=0, **kw):
    p = dict(C1)
    p.update(kw)
    return dict(a=p["a"], gamma=p["gamma"], kBT=p["kBT"], rc=p["rc"], k_bond=p["kbond"], r0=p["r0"],
                f_p=p["fp"], zeta=p["zeta"], dt=p["dt"], mass=p["mass"], seed=seed,
                **{k: v for k, v in kw.items() if k in ("tile", "noise", "exclude_bonded", "variant", "wexp")})


def minimg(d, L):
    return d - L * np.rint(d / L)


def force_check(f_gpu, f_orc):
    fn = np.linalg.norm(f_orc, axis=1)
    frms = math.sqrt(float(np.mean(fn ** 2)))
    err = np.linalg.norm(f_gpu.astype(np.float64) - f_orc, axis=1)
    rel = float(np.linalg.norm(err) / np.linalg.norm(f_orc))
    worst = float(np.max(err / np.maximum(fn, frms)))
    assert rel <= 1e-5, (rel, worst)
    assert worst <= 1e-5, (rel, worst)
    return rel, worst


CASES = [
    # (L, n_dimers, tile, seed): C1, a ragged multi-tile box, single tiles
    (32.0, 512, 8, 0),
    (37.0, 600, 8, 1),
    (37.0, 600, 4, 2),
    (37.0, 600, 16, 3),
    (3.5, 6, 8, 4),
    (9.0, 100, 16, 5),
]


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("L,nd,tile,seed", CASES)
def test_setup_force_parity(Sim, orc, L, nd, tile, seed, variant):
    x, _ = synth.dimers(nd, L, 0.5, seed=seed)
    v = synth.velocities(2 * nd, 1.0, seed=seed + 10)
    with Sim(L, 2 * nd, **sim_kw(seed=seed + 100, tile=tile, variant=variant)) as s:
        s.set_positions(x, v, step=7)
        xg, vg, f, step = s.get_state()
        assert step == 7
        np.testing.assert_array_equal(xg, x)
        np.testing.assert_array_equal(vg, v)
        fo, _ = orc.forces(oparams(orc, L, seed=seed + 100), x.astype(np.float64), v.astype(np.float64), 7)
        force_check(f, fo)


def test_gaussian_noise_and_no_exclusion(Sim, orc):
    L, nd = 20.0, 300
    x, _ = synth.dimers(nd, L, 0.5, seed=3)
    v = synth.velocities(2 * nd, 1.0, seed=4)
    with Sim(L, 2 * nd, **sim_kw(seed=9, noise=1, exclude_bonded=0)) as s:
        s.set_positions(x, v, step=123456789012)
        _, _, f, _ = s.get_state()
    fo, _ = orc.forces(oparams(orc, L, seed=9, noise=1, exclude_bonded=0), x.astype(np.float64),
                       v.astype(np.float64), 123456789012)
    force_check(f, fo)


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("L,nd,tile,seed", CASES[:4])
def test_cell_and_pair_counts_bit_exact(Sim, orc, L, nd, tile, seed, variant):
    x, _ = synth.dimers(nd, L, 0.5, seed=seed)
    with Sim(L, 2 * nd, **sim_kw(tile=tile, variant=variant)) as s:
        s.set_positions(x)
        nc = s.info().n_cells_side
        assert nc == math.floor(L / 1.0)
        np.testing.assert_array_equal(s.cell_counts(), orc.cell_counts(x, L, nc))
        cnt, tot = s.pair_counts()
    co, amb, toto = orc.pair_counts(oparams(orc, L), x.astype(np.float64), tie=4e-6)
    clean = amb == 0
    np.testing.assert_array_equal(cnt[clean], co[clean])
    assert abs(int(tot) - toto) <= int(amb.sum())


def test_cell_table_after_many_steps_multiblock_scan(Sim, orc):
    """L = 512 at density 3: 262,144 cells, 64 scan blocks, so a block's
    look-back reaches past its 32 nearest predecessors.  After 20, 40 and 60
    steps the device cell table (from the scan) equals the cell counts of the
    positions read back (exact multiples of L / 2^32 for this L)."""
    L, nd = 512.0, 393216
    x, _ = synth.dimers(nd, L, 0.5, seed=21)
    with Sim(L, 2 * nd, **sim_kw(seed=21)) as s:
        s.set_positions(x)
        nc = s.info().n_cells_side
        for _ in range(3):
            s.step(20)
            xg, _, _, _ = s.get_state()
            np.testing.assert_array_equal(s.cell_counts(), orc.cell_counts(xg, L, nc))


@pytest.mark.parametrize("variant", [2, 3, 4, 5])
def test_trajectory_parity_c1_100_steps(Sim, orc, variant):
    """C1: 512 dimers, L = 32, seed 0: positions after 100 steps."""
    L, nd = 32.0, 512
    x, v = synth.dimers(nd, L, 0.5, seed=0)
    with Sim(L, 2 * nd, **sim_kw(seed=0, variant=variant)) as s:
        s.set_positions(x, v)
        s.step(100)
        xg, vg, f, step = s.get_state()
    assert step == 100
    st = orc.State(oparams(orc, L, seed=0), x, v)
    st.run(100)
    dx = minimg(xg - st.x, L)
    assert np.abs(dx).max() <= 1e-4, np.abs(dx).max()
    # velocities and forces at step 100 follow the same trajectory
    assert np.abs(vg - st.v).max() <= 2e-2
    rel = np.linalg.norm(f - st.f) / np.linalg.norm(st.f)
    assert rel <= 1e-3, rel


@pytest.mark.parametrize("variant", [2, 3, 4, 5])
@pytest.mark.parametrize("s", [0.5, 1.0, 3.0])
def test_weight_exponent_force_parity(Sim, orc, s, variant):
    """Changed exponent of w (w_D = w^s, w_R = w^(s/2)): set-up forces
    against the oracle on a ragged multi-tile box."""
    L, nd = 37.0, 600
    x, _ = synth.dimers(nd, L, 0.5, seed=31)
    v = synth.velocities(2 * nd, 1.0, seed=32)
    with Sim(L, 2 * nd, **sim_kw(seed=5, variant=variant, wexp=s)) as sm:
        sm.set_positions(x, v, step=7)
        _, _, f, _ = sm.get_state()
    fo, _ = orc.forces(oparams(orc, L, seed=5, wexp=s), x, v.astype(np.float64), 7)
    force_check(f, fo)


def test_weight_exponent_trajectory(Sim, orc):
    """s = 0.5, C1 geometry: positions after 100 steps within 1e-4."""
    L, nd = 32.0, 512
    x, v = synth.dimers(nd, L, 0.5, seed=0)
    with Sim(L, 2 * nd, **sim_kw(seed=0, wexp=0.5)) as sm:
        sm.set_positions(x, v)
        sm.step(100)
        xg, _, _, _ = sm.get_state()
    st = orc.State(oparams(orc, L, seed=0, wexp=0.5), x, v)
    st.run(100)
    assert np.abs(minimg(xg - st.x, L)).max() <= 1e-4


def test_thermo_fp64_reductions(Sim):
    L, nd = 32.0, 512
    x, _ = synth.dimers(nd, L, 0.5, seed=2)
    v = synth.velocities(2 * nd, 1.3, seed=3)
    with Sim(L, 2 * nd, **sim_kw(mass=1.7)) as s:
        s.set_positions(x, v)
        s.step(5)
        _, vg, _, _ = s.get_state()
        vv = vg.astype(np.float64)
        ke = 0.5 * 1.7 * np.sum(vv * vv)
        np.testing.assert_allclose(s.kinetic_energy(), ke, rtol=1e-6)
        np.testing.assert_allclose(s.momentum(), 1.7 * vv.sum(axis=0), atol=1e-4 * np.abs(vv).sum())
        np.testing.assert_allclose(s.temperature(), 2 * ke / (2 * 2 * nd - 2), rtol=1e-6)
        log = s.thermo_log(1, 5)
        np.testing.assert_allclose(log[-1, 0], ke, rtol=1e-6)
        # the scalar getters and the log read the same FP64 ring entry: equal
        # bit for bit (a status word staged over the entry would show here)
        assert s.kinetic_energy() == log[-1, 0]
        assert tuple(s.momentum()) == (log[-1, 1], log[-1, 2])
        assert s.temperature() == log[-1, 3]


def test_restart_from_full_state(Sim):
    """set_state with forces resumes a run: 20 + 30 steps equals 50 steps up
    to FP32 accumulation order."""
    L, nd = 24.0, 300
    x, v = synth.dimers(nd, L, 0.5, seed=6)
    with Sim(L, 2 * nd, **sim_kw(seed=3)) as a, Sim(L, 2 * nd, **sim_kw(seed=3)) as b:
        a.set_positions(x, v)
        a.step(50)
        xa, va, fa, sa = a.get_state()
        b.set_positions(x, v)
        b.step(20)
        xm, vm, fm, sm = b.get_state()
        b.set_state(xm, vm, fm, sm)
        xr, vr, fr, sr = b.get_state()
        b.step(30)
        xb, vb, fb, sb = b.get_state()
    # the state survives a round trip through the ABI bit for bit
    np.testing.assert_array_equal(xr, xm)
    np.testing.assert_array_equal(vr, vm)
    np.testing.assert_array_equal(fr, fm)
    assert sr == 20 and sa == sb == 50
    assert np.abs(minimg(xa - xb, L)).max() < 1e-5


@pytest.mark.parametrize("L", [24.0, 37.0, 333.25])
def test_upload_wraps_periodic_images_exactly(Sim, L):
    """Positions given as periodic images (x + m L, m = -3..2) upload to the
    same fixed-point state: the round trip returns the wrapped grid values
    bit for bit, including points on the box edge."""
    nd = 200
    x, v = synth.dimers(nd, L, 0.5, seed=11)
    u = L / 2.0 ** 32
    x[:4] = [[0.0, 0.0], [L - u, u], [0.0, L / 2], [L / 3, L - u]]   # box edges and corners
    x = synth.on_grid(x, L)
    f = np.zeros_like(v)
    rng = np.random.default_rng(3)
    shift = rng.integers(-3, 3, size=x.shape).astype(np.float64) * L
    with Sim(L, 2 * nd, **sim_kw(seed=1)) as s:
        s.set_state(x, v, f, 5)
        x0, v0, _, _ = s.get_state()
        s.set_state(x + shift, v, f, 5)
        x1, v1, _, _ = s.get_state()
    np.testing.assert_array_equal(x0, x)
    np.testing.assert_array_equal(x1, x0)
    np.testing.assert_array_equal(v1, v0)


def test_momentum_conserved_without_drag_and_propulsion(Sim):
    L, nd = 32.0, 512
    x, _ = synth.dimers(nd, L, 0.5, seed=7)
    v = synth.velocities(2 * nd, 1.0, seed=8)
    with Sim(L, 2 * nd, **sim_kw(zeta=0.0, fp=0.0)) as s:
        s.set_positions(x, v)
        p0 = s.momentum()
        s.step(1000)
        log = s.thermo_log(1, 1000)
    scale = np.abs(v.astype(np.float64)).sum()
    assert np.abs(log[:, 1:3] - p0).max() <= 1e-5 * scale


def test_single_dimer_drift(Sim):
    L, r0, fp, zeta, dt = 32.0, 0.5, 1.0, 0.1, 0.01
    th = 0.3
    c = np.array([10.0, 12.0])
    h = 0.5 * r0 * np.array([math.cos(th), math.sin(th)])
    x = synth.on_grid(np.array([c + h, c - h]), L)
    with Sim(L, 2, **sim_kw(zeta=zeta, fp=fp, dt=dt)) as s:
        s.set_positions(x)
        s.step(3000)
        _, vg, _, _ = s.get_state()
    u, fcur, hh = 0.0, fp, 0.5 * dt
    for _ in range(3000):
        uh = u + hh * fcur
        fcur = fp - zeta * uh
        u = uh + hh * fcur
    d = minimg(x[0] - x[1], L)
    n = d / np.linalg.norm(d)
    np.testing.assert_allclose(vg[0] @ n, u, rtol=1e-5)
    # both beads move together up to FP32 rounding over 3000 steps
    np.testing.assert_allclose(vg[1], vg[0], atol=1e-5 * max(1.0, abs(u)))


def test_init_random_initial_condition(Sim):
    L, nd, r0 = 40.0, 2000, 0.5
    with Sim(L, 2 * nd, **sim_kw()) as s:
        s.init_random(5)
        xg, vg, f, step = s.get_state()
    assert step == 0
    assert np.all(xg >= 0) and np.all(xg < L)
    assert np.all(vg == 0)
    d = minimg(xg[0::2] - xg[1::2], L)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), r0, atol=2e-6)
    com = np.mod(xg[1::2] + 0.5 * d, L)
    hist = np.histogram2d(com[:, 0], com[:, 1], bins=4, range=[[0, L], [0, L]])[0]
    assert hist.min() > nd / 16 * 0.7
    ang = np.arctan2(d[:, 1], d[:, 0])
    assert abs(np.mean(np.cos(ang))) < 0.1 and abs(np.mean(np.sin(ang))) < 0.1


def test_nonfinite_state_is_reported(Sim):
    from paper_1310_0998_gb300._lib import DpdError
    L, nd = 10.0, 20
    x, v = synth.dimers(nd, L, 0.5, seed=1)
    v[3, 0] = np.nan
    with Sim(L, 2 * nd, **sim_kw()) as s:
        with pytest.raises(DpdError) as e:
            s.set_positions(x, v)
        assert e.value.status == -4
        # a clean state clears the latch
        v[3, 0] = 0.0
        s.set_positions(x, v)
        s.step(3)
        s.sync()
        with pytest.raises(DpdError) as e:
            s.set_positions(np.where(np.arange(2 * nd)[:, None] == 5, np.inf, x), v)
        assert e.value.status == -4


@pytest.mark.parametrize("variant", [2, 3, 4, 5])
def test_overflow_path_and_capacity_growth(Sim, orc, variant):
    """All beads squeezed into a quarter of the box (density 12): tiles
    overflow shared memory and take the global-memory path, whose set-up
    forces must match the oracle; synchronising calls then grow the tile
    capacity until no tile overflows, and the shared-memory path gives the
    same forces."""
    L, nd = 48.0, 3456
    x, _ = synth.dimers(nd, L, 0.5, seed=21)
    x = synth.on_grid(x * 0.5, L)
    v = synth.velocities(2 * nd, 0.5, seed=22)
    fo, _ = orc.forces(oparams(orc, L, seed=4), x, v.astype(np.float64), 3, cells=True)
    with Sim(L, 2 * nd, **sim_kw(seed=4, variant=variant)) as s:
        s.set_positions(x, v, step=3)
        _, _, f1, _ = s.get_state()
        ovf = s.info().overflow_tiles
        assert ovf > 0
        force_check(f1, fo)
        grew = False
        for _ in range(12):
            s.step(1)
            s.sync()
            o = s.info().overflow_tiles
            if o == ovf:
                grew = True
                break
            ovf = o
        assert grew, "capacity did not grow to fit the dense tiles"
        s.set_positions(x, v, step=3)
        _, _, f2, _ = s.get_state()
        assert s.info().overflow_tiles == ovf
    force_check(f2, fo)


def test_full_size_forces_sampled(Sim, orc):
    """C3 geometry (L = 1024, 3,145,728 beads, density 3) in the benchmark's
    launch configuration: set-up forces of the whole system against the
    cell-list FP64 oracle (itself checked against the all-pairs oracle)."""
    L = 1024.0
    nd = 3 * 1024 * 1024 // 2
    x, _ = synth.dimers(nd, L, 0.5, seed=0)
    v = synth.velocities(2 * nd, 1.0, seed=1)
    with Sim(L, 2 * nd, **sim_kw(seed=0)) as s:
        s.set_positions(x, v, step=3)
        _, _, f, _ = s.get_state()
        assert s.info().overflow_tiles == 0
    fo, _ = orc.forces(oparams(orc, L, seed=0), x.astype(np.float64), v.astype(np.float64), 3, cells=True)
    force_check(f, fo)


def test_trajectory_bit_identical_across_kernel_shapes(Sim):
    """Every pair variant and tile size produces the same trajectory bits: the
    pair term is an exact function of the two beads (exact fixed-point
    separation, Philox keyed on the unordered pair), opposite from the two
    sides, and a bead's pair forces are summed in fixed point, so
    neither the staging order, the Newton-3 side nor the atomic cell order
    changes a bit.  A clustered quarter makes some tiles take the
    global-memory path in some shapes; that path gives the same bits too."""
    L, nd = 37.0, 700
    x, _ = synth.dimers(nd, L, 0.5, seed=21)
    # 150 dimers packed into a 5 x 5 patch (bead density 12), bonds at rest
    rng = np.random.default_rng(5)
    centre = 2.0 + rng.random((150, 2)) * 5.0
    ang = rng.random(150) * 2.0 * np.pi
    n = 0.25 * np.stack([np.cos(ang), np.sin(ang)], axis=1)
    x[0:300:2] = centre + n
    x[1:300:2] = centre - n
    x = synth.on_grid(x % L, L)
    v = synth.velocities(2 * nd, 1.0, seed=22)
    ref = None
    for tile, variant in [(8, 2), (8, 2), (4, 1), (16, 3), (8, 3), (4, 2), (16, 2), (8, 1), (8, 4), (4, 4), (16, 4), (8, 5), (4, 5), (16, 5)]:
        with Sim(L, 2 * nd, **sim_kw(seed=3, tile=tile, variant=variant)) as s:
            s.set_positions(x, v)
            s.step(60)
            got = s.get_state()[:3]
        if ref is None:
            ref = got
            continue
        for a, b, name in zip(ref, got, ("x", "v", "f")):
            np.testing.assert_array_equal(a, b, err_msg=f"{name} tile={tile} variant={variant}")


def test_page_locked_host_buffers(Sim):
    """Page-locked host buffers (the end-to-end benchmark's) give the same
    bits as pageable ones: set-up, steps, download and restart."""
    import torch
    L, nd = 37.0, 600
    x, _ = synth.dimers(nd, L, 0.5, seed=12)
    v = synth.velocities(2 * nd, 1.0, seed=13)

    def pinned(a):
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True).numpy()
        t[:] = a
        return t

    xp, vp = pinned(x), pinned(v)
    with Sim(L, 2 * nd, **sim_kw(seed=5)) as a, Sim(L, 2 * nd, **sim_kw(seed=5)) as b:
        a.set_positions(x, v)
        b.set_positions(xp, vp)
        a.step(20)
        b.step(20)
        ra = a.get_state()
        outs = [pinned(np.zeros_like(q)) for q in ra[:3]]
        rb = b.get_state(*outs)
        for p, q, name in zip(ra[:3], rb[:3], ("x", "v", "f")):
            np.testing.assert_array_equal(p, q, err_msg=name)
        b.set_state(outs[0], outs[1], outs[2], rb[3])
        a.step(10)
        b.step(10)
        for p, q, name in zip(a.get_state()[:3], b.get_state()[:3], ("x", "v", "f")):
            np.testing.assert_array_equal(p, q, err_msg=name)
