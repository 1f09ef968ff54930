"""Seeded synthetic inputs for the DPD dimer simulator.

This module holds no arithmetic of the method: it only draws initial states
and parameter points, so that the CUDA path and the CPU oracle start from the
same bits.  numpy only.

Initial condition (Sec. 5 of arXiv:1310.0998): agents at uniformly random
centres and uniformly random orientations, every velocity zero.  Agent k is
beads 2k (head) and 2k+1 (tail), placed at centre +/- (r0/2)(cos t, sin t) and
wrapped into [0, L).  Positions are returned as float64 values on the grid
x = X L / 2^32 with integer X (the simulator's fixed-point state holds them
exactly, so both sides start from the same bits); velocities are float32.

Workloads (seed 0 unless stated), in reduced units (r_c = 1, m = 1):
  C1  L=32, 512 dimers, a=25, gamma=4.5, kBT=1, kappa=100, r0=0.5, f_p=1,
      zeta=0.1, dt=0.01.
  C2  L=256, area fraction phi -> N_d = 2 phi L^2, gamma in {1, 4.5, 20},
      zeta in {0.01, 0.1, 1}.
  C3  L=1024, bead density 3 -> N_b = 3 L^2 = 3,145,728 beads.
  C4  256 replicas: L ~ U(32, 192), phi ~ U(0.05, 0.6), gamma log-U(0.5, 50),
      zeta log-U(0.005, 2), f_p ~ U(0.5, 2).
Area fraction reading: phi = N l 2 r_h / L^2 with r_h = r_c/4 and
l = r0 + 2 r_h = 1 at r_c = 1, r0 = 0.5, so N_d = 2 phi L^2.
"""
from __future__ import annotations

import math

import numpy as np

BASE = dict(a=25.0, gamma=4.5, kBT=1.0, rc=1.0, kbond=100.0, r0=0.5, fp=1.0, zeta=0.1,
            dt=0.01, mass=1.0)

# the paper's own parameter set (Sec. 5.1), nondimensional: l = 1, a = l/(2 r_h) = 4,
# r_c = 0.5, Phi = 1.5, Pe = 20 (kBT = 1/Pe), kappa = 1e3, L = 100, dt = 3e-3;
# centre-to-centre rest length l - 2 r_h = 0.75.
PAPER = dict(a=1.5, gamma=8.0, kBT=0.05, rc=0.5, kbond=1000.0, r0=0.75, fp=1.0, zeta=0.5,
             dt=3.0e-3, mass=1.0)


def dimers_for_area_fraction(phi: float, L: float) -> int:
    return int(round(2.0 * phi * L * L))


def on_grid(x, L: float):
    """Round positions onto the fixed-point grid X L / 2^32, X in [0, 2^32).
    L must have at most 21 significant bits so that X L / 2^32 is exact."""
    L = float(L)
    u = L / 2.0 ** 32
    X = np.rint(np.mod(np.asarray(x, np.float64), L) / u).astype(np.int64) % (1 << 32)
    g = X.astype(np.float64) * u
    assert np.all(g / u == X), "L has too many significant bits for an exact grid"
    return g


def dimers(n_dimers: int, L: float, r0: float, seed: int = 0):
    """Random centres and orientations, zero velocities.
    Returns (x [2n,2] float64 on the grid in [0,L), v [2n,2] float32 zeros)."""
    rng = np.random.default_rng(seed)
    c = rng.random((n_dimers, 2)) * L
    t = rng.random(n_dimers) * (2.0 * math.pi)
    h = 0.5 * r0 * np.stack([np.cos(t), np.sin(t)], axis=1)
    x = np.empty((2 * n_dimers, 2), np.float64)
    x[0::2] = c + h
    x[1::2] = c - h
    return on_grid(x, L), np.zeros((2 * n_dimers, 2), np.float32)


def velocities(n_beads: int, scale: float, seed: int = 1):
    """Gaussian velocities (for force tests at non-zero relative velocity)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n_beads, 2)) * scale).astype(np.float32)


def dimers3(n_dimers: int, L: float, r0: float, seed: int = 0):
    """Three-dimensional variant: centres uniform in the periodic cube,
    orientations uniform on the unit sphere, zero velocities.
    Returns (x [2n,3] float64 on the grid in [0,L), v [2n,3] float32 zeros)."""
    rng = np.random.default_rng(seed)
    c = rng.random((n_dimers, 3)) * L
    u = rng.standard_normal((n_dimers, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    h = 0.5 * r0 * u
    x = np.empty((2 * n_dimers, 3), np.float64)
    x[0::2] = c + h
    x[1::2] = c - h
    return on_grid(x, L), np.zeros((2 * n_dimers, 3), np.float32)


def velocities3(n_beads: int, scale: float, seed: int = 1):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n_beads, 3)) * scale).astype(np.float32)


def uniform_beads(n_beads: int, L: float, seed: int = 0):
    """Beads uniformly in the box (any pairing), on the grid."""
    rng = np.random.default_rng(seed)
    return on_grid(rng.random((n_beads, 2)) * L, L)


def ensemble_points(R: int, seed: int = 0):
    """The uneven-replica distribution (C4): list of dicts with L, n_dimers,
    gamma, zeta, fp (other parameters from BASE)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(R):
        L = round(float(rng.uniform(32.0, 192.0)) * 256.0) / 256.0   # exact fixed-point grid
        phi = float(rng.uniform(0.05, 0.6))
        gamma = float(math.exp(rng.uniform(math.log(0.5), math.log(50.0))))
        zeta = float(math.exp(rng.uniform(math.log(0.005), math.log(2.0))))
        fp = float(rng.uniform(0.5, 2.0))
        out.append(dict(L=L, phi=phi, n_dimers=max(1, dimers_for_area_fraction(phi, L)),
                        gamma=gamma, zeta=zeta, fp=fp))
    return out


def sweep_points(L: float = 256.0, phis=(0.1, 0.2, 0.3, 0.4, 0.5, 0.6), gammas=(1.0, 4.5, 20.0),
                 zetas=(0.01, 0.1, 1.0)):
    """The parameter sweep of the 256 x 256 box (C2): every (area fraction,
    gamma, zeta) of the grid, f_p = 1; list of dicts with L, phi, n_dimers,
    gamma, zeta, fp (other parameters from BASE)."""
    return [dict(L=float(L), phi=float(p), n_dimers=dimers_for_area_fraction(p, L), gamma=float(g), zeta=float(z),
                 fp=1.0) for p in phis for g in gammas for z in zetas]


def surrogate_points(n: int, seed: int = 0):
    """Parameter rows (area fraction, gamma, zeta, f_p) [n][4] drawn from the
    ranges of the uneven-replica distribution (C4): phi U(0.05, 0.6), gamma
    log-U(0.5, 50), zeta log-U(0.005, 2), f_p U(0.5, 2)."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(0.05, 0.6, n), np.exp(rng.uniform(math.log(0.5), math.log(50.0), n)),
                     np.exp(rng.uniform(math.log(0.005), math.log(2.0), n)), rng.uniform(0.5, 2.0, n)], axis=1)
