"""FP64 observables of Sec. 5.3-5.4 (arXiv:1310.0998), numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper used here (each one a choice where the text is silent or
garbled):
  * Agents are filtered, not beads: the COM position of agent k is the tail
    position plus half the minimum-image head-tail vector, wrapped into
    [0, L); its velocity is v_COM = (v_head + v_tail)/2 (Sec. 5.3).
  * Filter psi of Sec. 5.4: a square window of side eps centred on the grid
    point, |dx| <= eps/2 and |dy| <= eps/2 in the minimum image; grid points
    x_M = (i + 1/2) L/M; u_M = mean velocity of the agents in the window,
    0 for an empty window; eps = L sqrt(N_f/N), Eq. (filterwidth).
  * Fourier coefficients, Eq. (fourierTrans01): uhat(k) = M^-2 sum_x u(x)
    exp(-2 pi i k.x/L), integer components in [-M/2, M/2).
  * Shell sum, Eq. (ESPf): E(k) = sum over modes with nint(|k|) = k of
    (|uhat_x|^2 + |uhat_y|^2)/2, k = 1..M/2.
  * Low-wavenumber slope: least squares of ln(E/E_1) on ln k over k = 1..10.
  * Velocity correlation, Eqs. (VCF), (spatial01): all agent pairs i < j with
    minimum-image COM separation in [b dr, (b+1) dr); the mean <v> and <|v|^2>
    are global averages over agents:
      g(b) = (<v_a.v_b>_b - |<v>|^2) / (<|v|^2> - |<v>|^2).
  * Integral length: trapezoid over the nodes r = 0 (g = 1) and the bin
    centres (b + 1/2) dr of the non-empty bins.
  * Vorticity omega = (curl u_M) . e_z (Sec. 5.3): second-order central
    differences on the periodic grid of u_M.
"""
from __future__ import annotations

import numpy as np


def _minimg(d, L):
    return d - L * np.rint(d / L)


def agent_com(x, v, L):
    """COM positions and velocities of the agents; x, v: [n_beads, 2]."""
    x = np.asarray(x, np.float64)
    v = np.asarray(v, np.float64)
    xh, xt = x[0::2], x[1::2]
    d = _minimg(xh - xt, L)
    c = xt + 0.5 * d
    c = c - L * np.floor(c / L)
    vc = 0.5 * (v[0::2] + v[1::2])
    return c, vc


def filter_width(L, n_agents, n_f=10.0):
    """eps = L sqrt(N_f / N), Eq. (filterwidth)."""
    return L * np.sqrt(n_f / n_agents)


def velocity_field(c, vc, L, M, eps, chunk=65536):
    """u_M on the M x M grid, layout [iy, ix, component]."""
    c = np.asarray(c, np.float64)
    vc = np.asarray(vc, np.float64)
    dx_grid = L / M
    xm = (np.arange(M) + 0.5) * dx_grid
    half = 0.5 * eps
    n = np.zeros((M, M))
    sx = np.zeros((M, M))
    sy = np.zeros((M, M))
    for a0 in range(0, c.shape[0], chunk):
        cc, vv = c[a0:a0 + chunk], vc[a0:a0 + chunk]
        # inclusion per axis, [agent, grid index]
        ixf = (np.abs(_minimg(xm[None, :] - cc[:, 0:1], L)) <= half).astype(np.float64)
        iyf = (np.abs(_minimg(xm[None, :] - cc[:, 1:2], L)) <= half).astype(np.float64)
        n += iyf.T @ ixf                                  # [iy, ix]
        sx += (iyf * vv[:, 0:1]).T @ ixf
        sy += (iyf * vv[:, 1:2]).T @ ixf
    u = np.zeros((M, M, 2), np.float64)
    nz = n > 0
    u[..., 0][nz] = sx[nz] / n[nz]
    u[..., 1][nz] = sy[nz] / n[nz]
    return u, n


def vorticity(u, L):
    """Scalar vorticity omega = (curl u_M) . e_z of a field u [iy, ix, comp]
    on the periodic M x M grid of spacing L / M (Sec. 5.3): second-order
    central differences, omega = d u_y / dx - d u_x / dy."""
    u = np.asarray(u, np.float64)
    h = L / u.shape[0]
    duy_dx = (np.roll(u[..., 1], -1, axis=1) - np.roll(u[..., 1], 1, axis=1)) / (2.0 * h)
    dux_dy = (np.roll(u[..., 0], -1, axis=0) - np.roll(u[..., 0], 1, axis=0)) / (2.0 * h)
    return duy_dx - dux_dy


def fourier(u):
    """uhat = M^-2 sum u exp(-2 pi i k.x/L) per component; [ky, kx, comp]."""
    M = u.shape[0]
    return np.stack([np.fft.fft2(u[..., 0]), np.fft.fft2(u[..., 1])], axis=-1) / (M * M)


def shell_index(M):
    k = np.fft.fftfreq(M, d=1.0 / M)                  # integers in [-M/2, M/2)
    kk = np.sqrt(k[:, None] ** 2 + k[None, :] ** 2)
    return np.rint(kk).astype(np.int64)


def energy_spectrum(u):
    """E(k), k = 1..M/2 (index 0 of the result is k = 1)."""
    M = u.shape[0]
    uh = fourier(u)
    e2 = 0.5 * (np.abs(uh[..., 0]) ** 2 + np.abs(uh[..., 1]) ** 2)
    sh = shell_index(M)
    E = np.zeros(M // 2, np.float64)
    for k in range(1, M // 2 + 1):
        E[k - 1] = e2[sh == k].sum()
    return E


def low_k_slope(E, kmax=10):
    """Least-squares slope of ln(E/E_1) against ln k over k = 1..kmax."""
    k = np.arange(1, kmax + 1, dtype=np.float64)
    y = np.log(E[:kmax] / E[0])
    A = np.stack([np.log(k), np.ones_like(k)], axis=1)
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    return float(coef[0])


def vcf_sums(c, vc, L, dr, nbins, chunk=2048):
    """Pair sums per separation bin: (sum v_a.v_b, pair count)."""
    c = np.asarray(c, np.float64)
    vc = np.asarray(vc, np.float64)
    n = c.shape[0]
    num = np.zeros(nbins, np.float64)
    cnt = np.zeros(nbins, np.int64)
    for a0 in range(0, n, chunk):
        a1 = min(n, a0 + chunk)
        dx = _minimg(c[a0:a1, None, 0] - c[None, :, 0], L)
        dy = _minimg(c[a0:a1, None, 1] - c[None, :, 1], L)
        r = np.sqrt(dx * dx + dy * dy)
        b = np.floor(r / dr)
        dot = vc[a0:a1, None, 0] * vc[None, :, 0] + vc[a0:a1, None, 1] * vc[None, :, 1]
        ia = np.arange(a0, a1)[:, None]
        jb = np.arange(n)[None, :]
        keep = (jb > ia) & (b < nbins)
        bi = b[keep].astype(np.int64)
        num += np.bincount(bi, weights=dot[keep], minlength=nbins)
        cnt += np.bincount(bi, minlength=nbins)
    return num, cnt


def vcf_from_sums(num, cnt, vc):
    vc = np.asarray(vc, np.float64)
    vm = vc.mean(axis=0)
    v2 = float(np.mean(np.sum(vc * vc, axis=1)))
    m2 = float(vm @ vm)
    den = v2 - m2
    g = np.full(num.shape, np.nan)
    nz = cnt > 0
    if den > 0:
        g[nz] = (num[nz] / cnt[nz] - m2) / den
    return g


def integral_length(g, cnt, dr):
    """L_gv by the trapezoid rule on (0, 1) and the non-empty bin centres."""
    nz = cnt > 0
    r = np.concatenate([[0.0], (np.nonzero(nz)[0] + 0.5) * dr])
    gg = np.concatenate([[1.0], g[nz]])
    return float(np.sum(0.5 * (gg[1:] + gg[:-1]) * np.diff(r)))


def velocity_correlation(c, vc, L, dr, nbins):
    num, cnt = vcf_sums(c, vc, L, dr, nbins)
    g = vcf_from_sums(num, cnt, vc)
    return g, integral_length(g, cnt, dr), num, cnt


# ---------------------------------------------------------------------------
# Three dimensions.  The paper defines the observables in two dimensions; the
# three-dimensional variant carries each over axis by axis (readings):
#   * cubic window of side eps, |dx|, |dy|, |dz| <= eps/2 (minimum image),
#     grid points (i + 1/2) L/M per axis, default eps = L (N_f/N)^(1/3) (the
#     window holds N_f agents on average, as the square window does in 2D);
#   * uhat = M^-3 sum u exp(-2 pi i k.x/L), E(k) = sum over nint|k| = k of
#     (|uhat_x|^2 + |uhat_y|^2 + |uhat_z|^2)/2, k = 1..M/2;
#   * vorticity: the curl of u_M by central differences;
#   * velocity correlation: all pairs, r = sqrt((dx^2 + dy^2) + dz^2).
# agent_com, vcf_from_sums and integral_length above work in any dimension.
# Layouts: grids [iz, iy, ix] (+ component last).

def filter_width3(L, n_agents, n_f=10.0):
    """eps = L (N_f / N)^(1/3)."""
    return L * (n_f / n_agents) ** (1.0 / 3.0)


def velocity_field3(c, vc, L, M, eps, chunk=8192):
    """u_M on the M^3 grid, layout [iz, iy, ix, component], and the counts."""
    c = np.asarray(c, np.float64)
    vc = np.asarray(vc, np.float64)
    xm = (np.arange(M) + 0.5) * (L / M)
    half = 0.5 * eps
    n = np.zeros((M, M, M))
    s = np.zeros((3, M, M, M))
    for a0 in range(0, c.shape[0], chunk):
        cc, vv = c[a0:a0 + chunk], vc[a0:a0 + chunk]
        inc = [(np.abs(_minimg(xm[None, :] - cc[:, d:d + 1], L)) <= half).astype(np.float64) for d in range(3)]
        n += np.einsum("az,ay,ax->zyx", inc[2], inc[1], inc[0])
        for d in range(3):
            s[d] += np.einsum("az,ay,ax->zyx", inc[2] * vv[:, d:d + 1], inc[1], inc[0])
    u = np.zeros((M, M, M, 3), np.float64)
    nz = n > 0
    for d in range(3):
        u[..., d][nz] = s[d][nz] / n[nz]
    return u, n


def fourier3(u):
    """uhat = M^-3 sum u exp(-2 pi i k.x/L) per component; [kz, ky, kx, comp]."""
    M = u.shape[0]
    return np.stack([np.fft.fftn(u[..., d]) for d in range(3)], axis=-1) / float(M) ** 3


def shell_index3(M):
    k = np.fft.fftfreq(M, d=1.0 / M)
    kk = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    return np.rint(kk).astype(np.int64)


def energy_spectrum3(u):
    """E(k), k = 1..M/2 (index 0 of the result is k = 1)."""
    M = u.shape[0]
    uh = fourier3(u)
    e2 = 0.5 * np.sum(np.abs(uh) ** 2, axis=-1)
    sh = shell_index3(M)
    return np.array([e2[sh == k].sum() for k in range(1, M // 2 + 1)], np.float64)


def vorticity3(u, L):
    """curl u of a field u [iz, iy, ix, comp] on the periodic M^3 grid of
    spacing L / M, second-order central differences; [iz, iy, ix, 3]."""
    u = np.asarray(u, np.float64)
    h = L / u.shape[0]

    def d(comp, axis):   # axis 0 = z, 1 = y, 2 = x of the grid
        return (np.roll(u[..., comp], -1, axis=axis) - np.roll(u[..., comp], 1, axis=axis)) / (2.0 * h)

    return np.stack([d(2, 1) - d(1, 0), d(0, 0) - d(2, 2), d(1, 2) - d(0, 1)], axis=-1)


def vcf_sums3(c, vc, L, dr, nbins, chunk=1024):
    """Pair sums per separation bin in 3D: (sum v_a.v_b, pair count)."""
    c = np.asarray(c, np.float64)
    vc = np.asarray(vc, np.float64)
    n = c.shape[0]
    num = np.zeros(nbins, np.float64)
    cnt = np.zeros(nbins, np.int64)
    for a0 in range(0, n, chunk):
        a1 = min(n, a0 + chunk)
        dx = _minimg(c[a0:a1, None, 0] - c[None, :, 0], L)
        dy = _minimg(c[a0:a1, None, 1] - c[None, :, 1], L)
        dz = _minimg(c[a0:a1, None, 2] - c[None, :, 2], L)
        r = np.sqrt(dx * dx + dy * dy + dz * dz)
        b = np.floor(r / dr)
        dot = (vc[a0:a1, None, 0] * vc[None, :, 0] + vc[a0:a1, None, 1] * vc[None, :, 1]
               + vc[a0:a1, None, 2] * vc[None, :, 2])
        keep = (np.arange(n)[None, :] > np.arange(a0, a1)[:, None]) & (b < nbins)
        bi = b[keep].astype(np.int64)
        num += np.bincount(bi, weights=dot[keep], minlength=nbins)
        cnt += np.bincount(bi, minlength=nbins)
    return num, cnt


def velocity_correlation3(c, vc, L, dr, nbins):
    num, cnt = vcf_sums3(c, vc, L, dr, nbins)
    g = vcf_from_sums(num, cnt, vc)
    return g, integral_length(g, cnt, dr), num, cnt
