"""Pins of the FP64 observables (Sec. 5.3-5.4) against closed forms and
invariants; no GPU."""
import math

import numpy as np
import pytest

from oracle import observables as ob


def _lattice_agents(L, n_side, vfun):
    """Agents on a regular n_side x n_side lattice (head = tail = site), with
    COM velocity vfun(site)."""
    g = (np.arange(n_side) + 0.25) * (L / n_side)
    X, Y = np.meshgrid(g, g, indexing="xy")
    c = np.stack([X.ravel(), Y.ravel()], axis=1)
    vc = vfun(c)
    x = np.repeat(c, 2, axis=0)
    v = np.repeat(vc, 2, axis=0)
    return x, v


def test_agent_com_minimum_image():
    L = 10.0
    x = np.array([[9.9, 5.0], [0.3, 5.0], [2.0, 2.0], [2.0, 3.0]])
    v = np.array([[1.0, 0.0], [3.0, 2.0], [0.0, 0.0], [0.0, 1.0]])
    c, vc = ob.agent_com(x, v, L)
    np.testing.assert_allclose(c[0], [0.1, 5.0], atol=1e-12)   # straddles the boundary
    np.testing.assert_allclose(c[1], [2.0, 2.5])
    np.testing.assert_allclose(vc, [[2.0, 1.0], [0.0, 0.5]])


def test_uniform_field_has_no_energy_off_zero():
    L, M = 64.0, 32
    x, v = _lattice_agents(L, 64, lambda c: np.tile([1.0, -0.5], (c.shape[0], 1)))
    c, vc = ob.agent_com(x, v, L)
    eps = ob.filter_width(L, c.shape[0], 10.0)
    u, n = ob.velocity_field(c, vc, L, M, eps)
    assert (n > 0).all()
    np.testing.assert_allclose(u[..., 0], 1.0, atol=1e-14)
    np.testing.assert_allclose(u[..., 1], -0.5, atol=1e-14)
    E = ob.energy_spectrum(u)
    assert np.abs(E).max() < 1e-28
    uh = ob.fourier(u)
    np.testing.assert_allclose(uh[0, 0], [1.0, -0.5], atol=1e-14)


def test_filter_window_counts():
    """Window of side eps: a lattice with spacing h and eps = 3h holds exactly
    3 x 3 sites when centred between sites; empty windows give u = 0."""
    L, M = 32.0, 8
    ns = 32  # spacing 1; grid points at (i + 1/2) * 4
    x, v = _lattice_agents(L, ns, lambda c: np.ones_like(c))
    c, vc = ob.agent_com(x, v, L)
    u, n = ob.velocity_field(c, vc, L, M, 3.0)
    # sites at k + 0.25; window [4i + 2 - 1.5, 4i + 2 + 1.5] holds k = 1,2,3 (+0.25)
    assert np.all(n == 9)
    u2, n2 = ob.velocity_field(c[:1], vc[:1], L, M, 1.0)
    assert n2.sum() == 0 and np.all(u2 == 0)


def test_single_mode_lands_in_its_shell():
    L, M, m = 64.0, 64, 5
    amp = 0.7
    x, v = _lattice_agents(L, 128, lambda c: np.stack(
        [np.zeros(c.shape[0]), amp * np.cos(2 * math.pi * m * c[:, 0] / L)], axis=1))
    c, vc = ob.agent_com(x, v, L)
    eps = ob.filter_width(L, c.shape[0], 10.0)
    u, _ = ob.velocity_field(c, vc, L, M, eps)
    E = ob.energy_spectrum(u)
    assert E[m - 1] / E.sum() > 0.999
    # box filter of width eps attenuates a cosine by sinc; E = 2 * (1/2)(A s/2)^2
    # (kx = +/- m) up to the grid sampling of the lattice inside the window
    assert 0.2 * amp ** 2 < 4 * E[m - 1] <= amp ** 2 * 1.0001


def test_parseval_and_shell_accounting():
    rng = np.random.default_rng(3)
    M = 32
    u = rng.standard_normal((M, M, 2))
    uh = ob.fourier(u)
    total = 0.5 * np.sum(np.abs(uh) ** 2)
    np.testing.assert_allclose(total, np.sum(u ** 2) / (2 * M * M), rtol=1e-12)
    E = ob.energy_spectrum(u)
    sh = ob.shell_index(M)
    e2 = 0.5 * np.sum(np.abs(uh) ** 2, axis=-1)
    outside = e2[(sh == 0) | (sh > M // 2)].sum()
    np.testing.assert_allclose(E.sum() + outside, total, rtol=1e-12)
    # every shell from 1 to M/2 has modes
    assert all((sh == k).sum() > 0 for k in range(1, M // 2 + 1))


def test_low_k_slope_recovers_power_law():
    k = np.arange(1, 65, dtype=np.float64)
    for a in (0.8, -0.5, -4.0):
        E = 3.0 * k ** a
        assert abs(ob.low_k_slope(E) - a) < 1e-12


def test_vcf_limits():
    L = 40.0
    rng = np.random.default_rng(0)
    n = 3000
    c = rng.random((n, 2)) * L
    # all equal velocities: denominator vanishes
    g = ob.vcf_from_sums(*ob.vcf_sums(c, np.ones((n, 2)), L, 0.5, 20), np.ones((n, 2)))
    assert np.all(np.isnan(g))
    # independent velocities: g ~ 0 within a few sigma of the bin average
    vc = rng.standard_normal((n, 2))
    num, cnt = ob.vcf_sums(c, vc, L, 0.5, 40)
    g = ob.vcf_from_sums(num, cnt, vc)
    assert np.all(np.abs(g) < 6.0 / np.sqrt(cnt))
    # brute force on a handful of agents
    cs, vs = c[:40], vc[:40]
    num2, cnt2 = ob.vcf_sums(cs, vs, L, 1.0, 25)
    bnum = np.zeros(25); bcnt = np.zeros(25, np.int64)
    for i in range(40):
        for j in range(i + 1, 40):
            d = cs[i] - cs[j]
            d -= L * np.round(d / L)
            b = int(math.floor(math.hypot(*d) / 1.0))
            if b < 25:
                bnum[b] += vs[i] @ vs[j]
                bcnt[b] += 1
    np.testing.assert_allclose(num2, bnum, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(cnt2, bcnt)


def test_integral_length_grows_with_patch_size():
    """Velocity constant on square patches of side s (random per patch):
    the correlation extends over ~s, so L_gv grows with s."""
    L = 48.0
    rng = np.random.default_rng(1)
    n = 4000
    c = rng.random((n, 2)) * L
    Ls = []
    for s in (2.0, 4.0, 8.0):
        npatch = int(L / s)
        pv = rng.standard_normal((npatch, npatch, 2))
        idx = np.floor(c / s).astype(int)
        vc = pv[idx[:, 1], idx[:, 0]]
        g, Lg, num, cnt = ob.velocity_correlation(c, vc, L, 0.25, int(L / 2 / 0.25))
        assert g[0] > 0.8      # agents closer than 0.25 share a patch almost surely
        Ls.append(Lg)
    assert Ls[0] < Ls[1] < Ls[2]


def test_trapezoid_closed_form():
    # g(r) = 1 - r/R on bin centres: the trapezoid is exact for a linear g
    dr, R = 0.5, 10.0
    nb = int(R / dr)
    r = (np.arange(nb) + 0.5) * dr
    g = 1 - r / R
    cnt = np.ones(nb, np.int64)
    Lg = ob.integral_length(g, cnt, dr)
    rl = r[-1]
    np.testing.assert_allclose(Lg, rl - rl ** 2 / (2 * R), rtol=1e-12)


def _grid(M, L):
    g = (np.arange(M) + 0.5) * (L / M)
    X, Y = np.meshgrid(g, g, indexing="xy")   # [iy, ix]
    return X, Y


@pytest.mark.parametrize("m", [1, 3, 7])
def test_vorticity_of_a_shear_wave(m):
    """u = (sin(k y), 0), k = 2 pi m / L: the central difference of a sine is
    the exact discrete form, omega = -(sin(k h) / h) cos(k y)."""
    M, L = 64, 40.0
    h = L / M
    X, Y = _grid(M, L)
    k = 2 * math.pi * m / L
    u = np.zeros((M, M, 2))
    u[..., 0] = np.sin(k * Y)
    om = ob.vorticity(u, L)
    np.testing.assert_allclose(om, -(math.sin(k * h) / h) * np.cos(k * Y), atol=1e-12)


def test_vorticity_of_a_discrete_gradient_vanishes():
    """u = (D_x phi, D_y phi) with the same central differences: the discrete
    curl of a discrete gradient is zero (the difference operators commute)."""
    M, L = 48, 30.0
    h = L / M
    rng = np.random.default_rng(2)
    phi = rng.standard_normal((M, M))
    u = np.zeros((M, M, 2))
    u[..., 0] = (np.roll(phi, -1, axis=1) - np.roll(phi, 1, axis=1)) / (2 * h)
    u[..., 1] = (np.roll(phi, -1, axis=0) - np.roll(phi, 1, axis=0)) / (2 * h)
    assert np.abs(ob.vorticity(u, L)).max() < 1e-12


def test_vorticity_sign_and_zero_mean():
    """A counter-clockwise cell (u = (-sin(k y), sin(k x))) has omega > 0 at
    its centre; on a periodic grid the vorticity of any field sums to zero."""
    M, L = 32, 16.0
    X, Y = _grid(M, L)
    k = 2 * math.pi / L
    u = np.zeros((M, M, 2))
    u[..., 0] = -np.sin(k * (Y - L / 4))
    u[..., 1] = np.sin(k * (X - L / 4))
    om = ob.vorticity(u, L)
    iy = ix = int(round(L / 4 / (L / M) - 0.5))
    assert om[iy, ix] > 0
    rng = np.random.default_rng(3)
    w = ob.vorticity(rng.standard_normal((M, M, 2)), L)
    assert abs(w.sum()) < 1e-10 * np.abs(w).sum()
