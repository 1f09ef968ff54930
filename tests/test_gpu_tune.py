"""Kernel-shape autotuner on the GPU: every shape is timed, the fastest is
picked and used by contexts created afterwards, and the tuned context gives
the same trajectory bits as the built-in shape (and the FP64 oracle's
positions within the 1e-4 bound after 100 steps)."""
import numpy as np
import pytest

from paper_1310_0998_gb300 import synth

pytestmark = pytest.mark.gpu

PHYS = dict(a=25.0, gamma=4.5, kBT=1.0, rc=1.0, k_bond=100.0, r0=0.5, f_p=1.0, zeta=0.1, dt=0.01)


@pytest.fixture()
def mods():
    import torch
    assert torch.cuda.is_available()
    from paper_1310_0998_gb300 import Ensemble, Sim, tune
    tune.clear()
    yield Sim, Ensemble, tune
    tune.clear()


def _check_report(rep, n_shapes):
    shapes = rep["shapes"]
    assert len(shapes) == n_shapes
    ms = [s["ms_per_step"] for s in shapes]
    assert all(m > 0 for m in ms), ms
    best = min(range(n_shapes), key=lambda i: ms[i])
    assert (rep["best"]["tile"], rep["best"]["variant"]) == (shapes[best]["tile"], shapes[best]["variant"])
    assert rep["best"]["ms_per_step"] == ms[best]


def test_single_system_tuning(mods, orc):
    Sim, _, tune = mods
    L, nd = 32.0, 512
    x, v = synth.dimers(nd, L, 0.5, seed=0)
    rep = tune.autotune(L, 2 * nd, x, v, steps=5, seed=0, **PHYS)
    _check_report(rep, 15)
    best = (rep["best"]["tile"], rep["best"]["variant"])
    assert tune.lookup(L, 2 * nd) == best
    with Sim(L, 2 * nd, seed=0, **PHYS) as s:          # tile = variant = 0: the tuned shape
        info = s.info()
        assert (info.tile, info.variant) == best
        s.set_positions(x, v)
        s.step(100)
        xt, vt, ft, _ = s.get_state()
    with Sim(L, 2 * nd, seed=0, tile=8, variant=2, **PHYS) as s:
        s.set_positions(x, v)
        s.step(100)
        xd, vd, fd, _ = s.get_state()
    np.testing.assert_array_equal(xt, xd)
    np.testing.assert_array_equal(vt, vd)
    np.testing.assert_array_equal(ft, fd)
    op = orc.params(L=L, seed=0, a=PHYS["a"], gamma=PHYS["gamma"], kBT=PHYS["kBT"], rc=PHYS["rc"],
                    kbond=PHYS["k_bond"], r0=PHYS["r0"], fp=PHYS["f_p"], zeta=PHYS["zeta"], dt=PHYS["dt"])
    st = orc.State(op, x, v)
    st.run(100)
    d = xt - st.x
    d -= L * np.rint(d / L)
    assert np.abs(d).max() <= 1e-4


def test_batch_tuning(mods):
    Sim, Ensemble, tune = mods
    pts = [dict(PHYS, L=24.0, n_beads=600, seed=3, replica=0), dict(PHYS, L=32.5, n_beads=1800, seed=4, replica=1),
           dict(PHYS, L=17.25, n_beads=300, gamma=20.0, seed=5, replica=2)]
    rep = tune.batch_autotune(pts, steps=3)
    _check_report(rep, 12)
    best = (rep["best"]["tile"], rep["best"]["variant"])
    states = []
    for shape in (None, (8, 2)):
        q = [dict(p, tile=shape[0], variant=shape[1]) if shape else dict(p) for p in pts]
        with Ensemble(q) as ens:
            if shape is None:
                info = ens.replica(1).info()
                assert (info.tile, info.variant) == best
            ens.init_random(11)
            ens.step(20)
            ens.sync()
            states.append([ens.replica(r).get_state()[:3] for r in range(len(pts))])
    for a, b in zip(states[0], states[1]):
        for u, w in zip(a, b):
            np.testing.assert_array_equal(u, w)
