"""Pins of the three-dimensional FP64 observables against closed forms, the
(pinned) two-dimensional observables on fields that do not depend on z, and
brute force; no GPU."""
import itertools
import math

import numpy as np
import pytest

from oracle import observables as ob


def _grid(M, L):
    x = (np.arange(M) + 0.5) * (L / M)
    return np.meshgrid(x, x, x, indexing="ij")   # Z, Y, X


@pytest.mark.parametrize("k", [(3, 0, 0), (0, 2, 1), (1, 1, 1), (2, -2, 3)])
def test_single_mode_lands_in_its_shell(k):
    """u = A cos(2 pi k.x / L) e: uhat(+-k) = A/2 e, so E = A^2/4 in the shell
    nint|k| and nothing elsewhere."""
    L, M, A = 8.0, 16, 0.7
    Z, Y, X = _grid(M, L)
    ph = 2 * np.pi * (k[0] * X + k[1] * Y + k[2] * Z) / L
    for comp in range(3):
        u = np.zeros((M, M, M, 3))
        u[..., comp] = A * np.cos(ph)
        E = ob.energy_spectrum3(u)
        sh = int(round(math.sqrt(sum(q * q for q in k))))
        assert abs(E[sh - 1] - A * A / 4) < 1e-13
        E[sh - 1] = 0.0
        assert np.abs(E).max() < 1e-25


def test_parseval_and_shell_accounting():
    """Sum of E over the shells plus the modes outside every shell (k = 0 and
    nint|k| > M/2) equals the mean of |u|^2 / 2."""
    rng = np.random.default_rng(3)
    M = 8
    u = rng.standard_normal((M, M, M, 3))
    E = ob.energy_spectrum3(u)
    uh = ob.fourier3(u)
    e2 = 0.5 * np.sum(np.abs(uh) ** 2, axis=-1)
    sh = ob.shell_index3(M)
    outside = e2[(sh == 0) | (sh > M // 2)].sum()
    assert abs(E.sum() + outside - 0.5 * np.mean(np.sum(u * u, axis=-1))) < 1e-12


def test_planar_field_matches_two_dimensional_spectrum():
    """u(x, y) independent of z with u_z = 0: only kz = 0 modes, equal to the
    2D coefficients, so E3 equals the 2D E(k)."""
    rng = np.random.default_rng(4)
    M = 16
    u2 = rng.standard_normal((M, M, 2))
    u3 = np.zeros((M, M, M, 3))
    u3[..., 0:2] = u2[None, :, :, :]
    np.testing.assert_allclose(ob.energy_spectrum3(u3), ob.energy_spectrum(u2), rtol=1e-12, atol=1e-15)


def test_velocity_field_brute_force():
    """Window means against loops over every agent and grid point."""
    rng = np.random.default_rng(5)
    L, M, eps, n = 6.0, 4, 2.3, 60
    c = rng.random((n, 3)) * L
    vc = rng.standard_normal((n, 3))
    u, cnt = ob.velocity_field3(c, vc, L, M, eps)
    xm = (np.arange(M) + 0.5) * (L / M)
    for iz, iy, ix in itertools.product(range(M), repeat=3):
        g = np.array([xm[ix], xm[iy], xm[iz]])
        d = g[None, :] - c
        d -= L * np.rint(d / L)
        inside = np.all(np.abs(d) <= eps / 2, axis=1)
        assert cnt[iz, iy, ix] == inside.sum()
        want = vc[inside].mean(axis=0) if inside.any() else np.zeros(3)
        np.testing.assert_allclose(u[iz, iy, ix], want, atol=1e-14)


def test_filter_width_holds_n_f_agents():
    L, n = 40.0, 8000
    eps = ob.filter_width3(L, n, 10.0)
    assert abs(n * (eps / L) ** 3 - 10.0) < 1e-10


@pytest.mark.parametrize("m", [1, 3])
def test_vorticity_of_a_shear_wave(m):
    """u = (sin(a y), 0, 0), a = 2 pi m / L: central differences give
    omega_z = -cos(a y) sin(a h) / h exactly and omega_x = omega_y = 0."""
    L, M = 10.0, 16
    h = L / M
    a = 2 * np.pi * m / L
    Z, Y, X = _grid(M, L)
    u = np.zeros((M, M, M, 3))
    u[..., 0] = np.sin(a * Y)
    om = ob.vorticity3(u, L)
    np.testing.assert_allclose(om[..., 2], -np.cos(a * Y) * np.sin(a * h) / h, atol=1e-13)
    assert np.abs(om[..., 0:2]).max() < 1e-13


def test_vorticity_of_planar_field_matches_two_dimensional():
    rng = np.random.default_rng(6)
    L, M = 12.0, 8
    u2 = rng.standard_normal((M, M, 2))
    u3 = np.zeros((M, M, M, 3))
    u3[..., 0:2] = u2[None]
    om = ob.vorticity3(u3, L)
    np.testing.assert_allclose(om[..., 2], np.broadcast_to(ob.vorticity(u2, L), (M, M, M)), atol=1e-13)
    assert np.abs(om[..., 0:2]).max() < 1e-13


def test_vorticity_of_a_gradient_vanishes():
    """The curl of a discrete gradient (central differences commute) is zero."""
    rng = np.random.default_rng(7)
    L, M = 9.0, 8
    phi = rng.standard_normal((M, M, M))
    h = L / M
    grad = lambda f, ax: (np.roll(f, -1, axis=ax) - np.roll(f, 1, axis=ax)) / (2 * h)
    u = np.stack([grad(phi, 2), grad(phi, 1), grad(phi, 0)], axis=-1)
    assert np.abs(ob.vorticity3(u, L)).max() < 1e-12


def test_vcf_brute_force_and_planar_embedding():
    rng = np.random.default_rng(8)
    L, n, dr, nb = 5.0, 70, 0.3, 9
    c = rng.random((n, 3)) * L
    vc = rng.standard_normal((n, 3))
    num, cnt = ob.vcf_sums3(c, vc, L, dr, nb)
    bn = np.zeros(nb)
    bc = np.zeros(nb, np.int64)
    for a in range(n):
        for b in range(a + 1, n):
            d = c[a] - c[b]
            d -= L * np.rint(d / L)
            r = math.sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])
            k = int(math.floor(r / dr))
            if k < nb:
                bn[k] += float(vc[a] @ vc[b])
                bc[k] += 1
    np.testing.assert_array_equal(cnt, bc)
    np.testing.assert_allclose(num, bn, rtol=1e-12, atol=1e-12)
    # all agents in one plane, v_z = 0: the 2D pair sums
    c2 = c.copy()
    c2[:, 2] = 1.0
    v2 = vc.copy()
    v2[:, 2] = 0.0
    n3, k3 = ob.vcf_sums3(c2, v2, L, dr, nb)
    n2, k2 = ob.vcf_sums(c2[:, :2], v2[:, :2], L, dr, nb)
    np.testing.assert_array_equal(k3, k2)
    np.testing.assert_allclose(n3, n2, rtol=1e-12, atol=1e-12)


def test_vcf_limits():
    """Bins reaching past the largest minimum-image distance (L sqrt(3) / 2)
    hold every pair once; independent random velocities give g near 0 at
    every separation; v_b = v_a for the two members of close pairs gives g = 1
    in the first bin."""
    rng = np.random.default_rng(9)
    L, n = 6.0, 400
    c = rng.random((n, 3)) * L
    vc = rng.standard_normal((n, 3))
    nb = int(math.ceil(L * math.sqrt(3.0) / 2 / 0.5)) + 1
    g, Li, num, cnt = ob.velocity_correlation3(c, vc, L, 0.5, nb)
    assert cnt.sum() == n * (n - 1) // 2
    assert np.nanmax(np.abs(g[:6])) < 0.15
    # isolated twin agents (same velocity, 0.01 apart), far from all others
    m = 40
    cc = np.zeros((2 * m, 3))
    grid = np.array(list(itertools.product(range(4), range(4), range(3))))[:m] * 1.5 + 0.2
    cc[0::2] = grid
    cc[1::2] = grid + 0.01
    vv = np.repeat(rng.standard_normal((m, 3)), 2, axis=0)
    vv -= vv.mean(axis=0)
    g, Li, num, cnt = ob.velocity_correlation3(cc, vv, L, 0.1, 3)
    assert cnt[0] == m and cnt[1] == 0 and cnt[2] == 0
    assert abs(g[0] - 1.0) < 1e-12
