"""The batched persistent kernel advances every replica exactly as the
single-system path does, for replicas of uneven box size, bead count and
parameters; its grid barrier gives up after a bounded wait.

Pair forces are summed per bead in fixed point (order-independent) from
pair terms that are exact negations of each other whichever bead or tile
evaluates them, so a replica's trajectory is the same bits in the batch and
alone, whatever the cell order the atomic binning produced.  Only the FP64
thermo sums, whose block order differs, are compared with a tolerance."""
import numpy as np
import pytest

from paper_1310_0998_gb300 import synth

pytestmark = pytest.mark.gpu

BASE = dict(a=25.0, gamma=4.5, kBT=1.0, rc=1.0, k_bond=100.0, r0=0.5, f_p=1.0, zeta=0.1, dt=0.01)


def minimg(d, L):
    return d - L * np.rint(d / L)


def _points():
    # box sides on the 1/256 grid, uneven sizes, densities and frictions
    spec = [(24.0, 300, 4.5, 0.1, 1.0), (32.5, 900, 1.0, 0.5, 1.5), (17.25, 150, 20.0, 0.01, 0.5),
            (40.0, 2000, 0.7, 1.3, 2.0), (9.0, 40, 4.5, 0.0, 0.0), (64.0, 4000, 3.0, 0.05, 1.0)]
    pts = []
    for r, (L, nd, g, z, fp) in enumerate(spec):
        pts.append(dict(BASE, L=L, n_beads=2 * nd, gamma=g, zeta=z, f_p=fp, seed=100 + r, replica=r))
    return pts


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available()
    from paper_1310_0998_gb300 import Ensemble, Sim
    return Ensemble, Sim


@pytest.mark.parametrize("variant", [2, 3, 4, 5])
def test_batch_matches_single_system(mods, variant):
    Ensemble, Sim = mods
    pts = [dict(p, variant=variant) for p in _points()]
    states = []
    with Ensemble(pts) as ens:
        for r, pt in enumerate(pts):
            x, _ = synth.dimers(pt["n_beads"] // 2, pt["L"], 0.5, seed=r)
            v = synth.velocities(pt["n_beads"], 0.5, seed=r + 7)
            ens.replica(r).set_positions(x, v)
            states.append((x, v))
        ens.step(40)
        ens.sync()
        got = [ens.replica(r).get_state() for r in range(len(pts))]
        logs = [ens.replica(r).thermo_log(1, 40) for r in range(len(pts))]
        info = ens.info()
    assert info["replicas"] == len(pts) and info["grid"] > 0
    for r, pt in enumerate(pts):
        kw = {k: v for k, v in pt.items() if k not in ("L", "n_beads")}
        with Sim(pt["L"], pt["n_beads"], **kw) as s:
            s.set_positions(*states[r])
            s.step(40)
            xs, vs, fs, st = s.get_state()
            log = s.thermo_log(1, 40)
        xb, vb, fb, sb = got[r]
        assert sb == st == 40
        np.testing.assert_array_equal(xb, xs, err_msg=str(r))
        np.testing.assert_array_equal(vb, vs, err_msg=str(r))
        np.testing.assert_array_equal(fb, fs, err_msg=str(r))
        np.testing.assert_allclose(logs[r], log, rtol=1e-12, atol=1e-12 * np.abs(log).max())


def test_batch_with_weight_exponents(mods):
    """Replicas with different exponents of w in one persistent launch match
    the same replicas run alone."""
    Ensemble, Sim = mods
    pts = [dict(p, wexp=s) for p, s in zip(_points()[:4], (0.0, 0.5, 3.0, 1.0))]
    states = []
    with Ensemble(pts) as ens:
        for r, pt in enumerate(pts):
            x, _ = synth.dimers(pt["n_beads"] // 2, pt["L"], 0.5, seed=40 + r)
            v = synth.velocities(pt["n_beads"], 0.5, seed=50 + r)
            ens.replica(r).set_positions(x, v)
            states.append((x, v))
        ens.step(30)
        ens.sync()
        got = [ens.replica(r).get_state() for r in range(len(pts))]
    for r, pt in enumerate(pts):
        kw = {k: v for k, v in pt.items() if k not in ("L", "n_beads")}
        with Sim(pt["L"], pt["n_beads"], **kw) as s:
            s.set_positions(*states[r])
            s.step(30)
            xs, vs, fs, _ = s.get_state()
        np.testing.assert_array_equal(got[r][0], xs, err_msg=str(r))
        np.testing.assert_array_equal(got[r][1], vs, err_msg=str(r))
        np.testing.assert_array_equal(got[r][2], fs, err_msg=str(r))


def test_batch_against_oracle(mods, orc):
    """One replica of the batch against the FP64 oracle, 100 steps."""
    Ensemble, _ = mods
    pts = _points()[:3]
    L, nd = pts[1]["L"], pts[1]["n_beads"] // 2
    x, v = synth.dimers(nd, L, 0.5, seed=5)
    with Ensemble(pts) as ens:
        ens.init_random(9)
        ens.replica(1).set_positions(x, v)
        ens.step(100)
        xb, _, _, _ = ens.replica(1).get_state()
    p = pts[1]
    op = orc.params(L=L, a=p["a"], gamma=p["gamma"], kBT=p["kBT"], rc=p["rc"], kbond=p["k_bond"], r0=p["r0"],
                    fp=p["f_p"], zeta=p["zeta"], dt=p["dt"], seed=p["seed"], replica=p["replica"])
    st = orc.State(op, x, v)
    st.run(100)
    assert np.abs(minimg(xb - st.x, L)).max() <= 1e-4


def test_barrier_timeout_is_reported_and_batch_survives(mods):
    Ensemble, _ = mods
    pts = _points()[:2]
    with Ensemble(pts) as ens:
        ens.init_random(1)
        assert ens.barrier_selftest() == -5          # DPD_ERR_TIMEOUT
        ens.step(5)
        ens.sync()
        _, _, _, s = ens.replica(0).get_state()
        assert s == 5


def test_replica_views_are_borrowed(mods):
    Ensemble, _ = mods
    from paper_1310_0998_gb300 import _lib
    pts = _points()[:2]
    with Ensemble(pts) as ens:
        ens.init_random(3)
        view = ens.replica(0)
        _lib.lib().dpd_destroy(view._h)   # ignored for a replica
        ens.step(3)
        ens.sync()
        assert view.get_state()[3] == 3


def test_profile_runs_the_same_steps(mods):
    """The phase-logged launch advances the replicas exactly as an ordinary
    step call does, and reports positive phase times with the busy time of a
    block inside its phase."""
    Ensemble, _ = mods
    pts = _points()[:4]
    out = []
    for prof in (True, False):
        with Ensemble(pts) as ens:
            ens.init_random(21)
            if prof:
                ph = ens.profile(12)
            else:
                ens.step(12)
                ens.sync()
            out.append([ens.replica(r).get_state() for r in range(len(pts))])
    for a, b in zip(out[0], out[1]):
        assert a[3] == b[3] == 12
        for u, w in zip(a[:3], b[:3]):
            np.testing.assert_array_equal(u, w)
    for k in ("scan", "scatter", "force"):
        assert ph[k + "_ms"] > 0 and 0 < ph[k + "_busy_ms"] <= ph[k + "_ms"] * 1.05, ph


def test_full_size_c4_batch(mods, orc):
    """The 256-replica uneven batch (box side U(32, 192), area fraction
    U(0.05, 0.6), gamma log-U(0.5, 50), zeta log-U(0.005, 2), f_p U(0.5, 2);
    4.7 M beads) in the bench's launch configuration (16 x 16 cell blocks,
    pair queue): the set-up forces of four replicas spread over the sizes
    against the FP64 cell-list oracle (||dF|| / ||F|| and max_i |dF_i| /
    max(|F_i|, F_rms) within 1e-5), and after 20 batched steps every replica
    equals, bit for bit, the same replica restarted alone from its initial
    canonical state."""
    Ensemble, Sim = mods
    pts = []
    for r, e in enumerate(synth.ensemble_points(256, 0)):
        pts.append(dict(a=25.0, kBT=1.0, rc=1.0, k_bond=100.0, r0=0.5, dt=0.01, L=e["L"], n_beads=2 * e["n_dimers"],
                        gamma=e["gamma"], zeta=e["zeta"], f_p=e["fp"], seed=r, replica=r, tile=16, variant=2))
    with Ensemble(pts) as ens:
        ens.init_random(0)
        ens.sync()
        init = [ens.replica(r).get_state() for r in range(len(pts))]
        ens.step(20)
        ens.sync()
        got = [ens.replica(r).get_state()[:3] for r in range(len(pts))]
    for r in (0, 85, 170, 255):
        x, v, f, st = init[r]
        p = pts[r]
        op = orc.params(L=p["L"], a=p["a"], gamma=p["gamma"], kBT=p["kBT"], rc=p["rc"], kbond=p["k_bond"], r0=p["r0"],
                        fp=p["f_p"], zeta=p["zeta"], dt=p["dt"], seed=p["seed"], replica=p["replica"])
        fo, _ = orc.forces(op, x, v.astype(np.float64), st, cells=True)
        fn = np.linalg.norm(fo, axis=1)
        frms = float(np.sqrt(np.mean(fn ** 2)))
        err = np.linalg.norm(f.astype(np.float64) - fo, axis=1)
        assert np.linalg.norm(err) / np.linalg.norm(fo) <= 1e-5, r
        assert np.max(err / np.maximum(fn, frms)) <= 1e-5, r
    for r, p in enumerate(pts):
        kw = {k: v for k, v in p.items() if k not in ("L", "n_beads")}
        with Sim(p["L"], p["n_beads"], **kw) as s:
            x, v, f, st = init[r]
            s.set_state(x, v, f, st)
            s.step(20)
            alone = s.get_state()[:3]
        for a, b, name in zip(got[r], alone, ("x", "v", "f")):
            np.testing.assert_array_equal(a, b, err_msg=f"replica {r} {name}")
