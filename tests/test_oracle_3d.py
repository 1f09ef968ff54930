"""Pins of the three-dimensional oracle (orc3_*): the vector force laws of
Sec. 2 in a periodic cube.  They are pinned to the (independently pinned)
two-dimensional oracle by planar embedding, and to rotation covariance,
momentum conservation and the equilibrium temperature."""
import math

import numpy as np
import pytest

from paper_1310_0998_gb300 import synth

BASE = dict(a=25.0, gamma=4.5, kBT=1.0, rc=1.0, kbond=100.0, r0=0.5, fp=1.0, zeta=0.1, dt=0.01)


def P(orc, **kw):
    b = dict(BASE)
    b.update(kw)
    return orc.params(**b)


def test_planar_embedding_reproduces_the_2d_oracle(orc):
    """All beads in one plane z = z0 with v_z = 0: forces and 100 steps of
    velocity-Verlet equal the two-dimensional oracle's (z stays z0)."""
    L = 9.0
    x2, _ = synth.dimers(120, L, 0.5, seed=3)
    v2 = synth.velocities(240, 0.8, seed=4).astype(np.float64)
    x3 = np.concatenate([x2, np.full((240, 1), 4.25)], axis=1)
    v3 = np.concatenate([v2, np.zeros((240, 1))], axis=1)
    p = P(orc, L=L, seed=5)
    f2, n2 = orc.forces(p, x2, v2, 7)
    f3, n3 = orc.forces3(p, x3, v3, 7)
    assert n2 == n3 > 0
    np.testing.assert_allclose(f3[:, :2], f2, rtol=0, atol=1e-11)
    assert np.all(f3[:, 2] == 0.0)
    s2 = orc.State(p, x2, v2, step=7)
    s3 = orc.State3(p, x3, v3, step=7)
    s2.run(100)
    s3.run(100)
    np.testing.assert_allclose(s3.x[:, :2], s2.x, rtol=0, atol=1e-9)
    assert np.all(s3.x[:, 2] == 4.25) and np.all(s3.v[:, 2] == 0.0)


def test_forces_rotate_with_the_configuration(orc):
    """A cluster far from the box walls, rotated rigidly (positions and
    velocities) about the box centre: the forces rotate with it (alpha is keyed
    by ids and step only)."""
    rng = np.random.default_rng(6)
    L = 40.0
    ctr = np.full(3, L / 2)
    x, _ = synth.dimers3(60, 3.0, 0.5, seed=7)
    x = x - 1.5 + ctr
    v = rng.standard_normal(x.shape)
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    R = q * np.sign(np.linalg.det(q))
    p = P(orc, L=L, seed=8)
    f0, n0 = orc.forces3(p, x, v, 3)
    f1, n1 = orc.forces3(p, (x - ctr) @ R.T + ctr, v @ R.T, 3)
    assert n0 == n1 > 50
    np.testing.assert_allclose(f1, f0 @ R.T, rtol=0, atol=1e-9 * np.abs(f0).max())


def test_momentum_conserved_without_drag_and_propulsion(orc):
    L = 5.0
    x, v = synth.dimers3(150, L, 0.5, seed=9)
    v = synth.velocities3(300, 1.0, seed=10).astype(np.float64)
    st = orc.State3(P(orc, L=L, zeta=0.0, fp=0.0, seed=11), x, v)
    P0 = st.v.sum(axis=0)
    log = st.run(300, thermo=True)
    scale = np.abs(st.v).sum()
    np.testing.assert_allclose(log[:, 1:4], np.tile(P0, (300, 1)), rtol=0, atol=1e-10 * scale)


def test_equilibrium_temperature(orc):
    """zeta = f_p = 0: T = 2 KE / (3N - 3) settles at kBT within 2%."""
    L = 5.0
    x, v = synth.dimers3(188, L, 0.5, seed=12)
    st = orc.State3(P(orc, L=L, zeta=0.0, fp=0.0, seed=13), x, v)
    st.run(1000)
    log = st.run(12000, thermo=True)
    n = x.shape[0]
    T = 2.0 * log[:, 0] / (3 * n - 3)
    assert abs(T.mean() - 1.0) < 0.02, T.mean()
