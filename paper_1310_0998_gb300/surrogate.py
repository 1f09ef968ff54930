"""Learned surrogate of the simulator's ensemble statistics (wraps sur_*).

The statistics of a parameter point (area fraction phi, gamma, zeta, f_p)
come from this simulator alone: a periodic box of side `L` holding
N_d = 2 phi L^2 dimers (other parameters as in BASE) is started from the
paper's initial condition, run `burn` steps, then sampled `n_snap` times every
`every` steps.  At each snapshot the device computes E(k) on a 128^2 grid
(Sec. 5.4), the velocity correlation g(r) of the agents' COM velocities
(Sec. 5.3) and the FP64 temperature; the snapshot averages give 40 targets:

  0-31  ln of E averaged over shell pairs (2b+1, 2b+2), b = 0..31
  32    xi: first r where g(r) <= 1/e (linear interpolation), correlation length
  33    L_gv: integral length (trapezoid up to L/2)
  34    T
  35    low-wavenumber slope of ln(E/E_1) on ln k, k = 1..10
  36    high-wavenumber slope, k = 30..60
  37    k of the largest E(k)
  38    ln E_1
  39    mean |v_COM|

The network maps (phi, gamma, zeta, f_p) to these 40 numbers; its K members
disagree where the training data do not constrain them, and any query whose
member spread exceeds a threshold is answered by running the simulation.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import check

NOUT = 40
SUR_L = 48.0
BASE = dict(a=25.0, kBT=1.0, rc=1.0, k_bond=100.0, r0=0.5, dt=0.01)


def targets(E_snaps, g_snaps, T_snaps, vcom_snaps, dr):
    """The 40 statistics from per-snapshot E(k) [s, >= 64], g(r) [s, nb], T
    [s], mean |v_COM| [s] (sur_targets of the library)."""
    E = np.ascontiguousarray(E_snaps, np.float64)
    g = np.ascontiguousarray(g_snaps, np.float64)
    T = np.ascontiguousarray(T_snaps, np.float64).ravel()
    vc = np.ascontiguousarray(vcom_snaps, np.float64).ravel()
    out = np.zeros(NOUT, np.float64)
    check(_lib.lib().sur_targets(E.shape[0], E.shape[1], g.shape[1], float(dr), _lib.ptr(E), _lib.ptr(g),
                                 _lib.ptr(T), _lib.ptr(vc), _lib.ptr(out)), "sur_targets")
    return out


def point_params(phi, gamma, zeta, fp, L=SUR_L, seed=0, replica=0):
    nd = max(1, int(round(2.0 * phi * L * L)))
    return dict(BASE, L=float(L), n_beads=2 * nd, gamma=float(gamma), zeta=float(zeta), f_p=float(fp),
                seed=int(seed), replica=int(replica))


def _snapshot(sim, M, dr, nbins):
    E = sim.energy_spectrum(M)
    g, _, _, _ = sim.velocity_correlation(dr, nbins)
    return E, g, sim.temperature(), sim.agent_speed()


def simulate(X, L=SUR_L, burn=2000, n_snap=10, every=200, M=128, dr=0.25, seed=0, batched=True, chunk=256):
    """Statistics [n][40] of the parameter rows X [n][4] = (phi, gamma, zeta,
    f_p).  batched: the points as ensembles of up to `chunk` replicas
    (persistent kernel); else one simulation after another (the plain path).
    Point i starts from the random initial condition of seed + i."""
    from .ensemble import Ensemble
    from .sim import Sim
    X = np.asarray(X, np.float64)
    nbins = int(L / 2 / dr)
    pts = [point_params(*X[i], L=L, seed=seed + i, replica=i) for i in range(X.shape[0])]
    snaps = [[[], [], [], []] for _ in pts]
    if batched:
        # replicas in batches of at most `chunk` per persistent launch; replica
        # i keeps seed + i and replica key i whatever batch it lands in
        for c0 in range(0, len(pts), chunk):
            ens = Ensemble(pts[c0:c0 + chunk])
            try:
                for r in range(len(pts[c0:c0 + chunk])):
                    ens.replica(r).init_random(seed + c0 + r)
                ens.step(burn)
                for _ in range(n_snap):
                    ens.step(every)
                    ens.sync()
                    for r in range(len(pts[c0:c0 + chunk])):
                        for a, b in zip(snaps[c0 + r], _snapshot(ens.replica(r), M, dr, nbins)):
                            a.append(b)
            finally:
                ens.close()
    else:
        for i, pt in enumerate(pts):
            kw = {k: v for k, v in pt.items() if k not in ("L", "n_beads")}
            with Sim(pt["L"], pt["n_beads"], **kw) as s:
                s.init_random(seed + i)
                s.step(burn)
                for _ in range(n_snap):
                    s.step(every)
                    for a, b in zip(snaps[i], _snapshot(s, M, dr, nbins)):
                        a.append(b)
    return np.stack([targets(*snaps[i], dr) for i in range(len(pts))])


class Surrogate:
    """Deep ensemble of K MLPs trained on simulator statistics."""

    def __init__(self, members: int = 4, max_rows: int = 4096, seed: int = 0, stream=None):
        self._lib = _lib.lib()
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(int(stream)) if stream else None
        check(self._lib.sur_create(int(members), int(max_rows), int(seed), st, ctypes.byref(h)), "sur_create")
        self._h = h
        self.members = members

    def fit(self, X, Y, epochs=500, batch=64, lr=1e-3) -> float:
        X = np.ascontiguousarray(X, np.float32)
        Y = np.ascontiguousarray(Y, np.float32)
        loss = ctypes.c_float()
        check(self._lib.sur_train(self._h, _lib.ptr(X), _lib.ptr(Y), X.shape[0], int(epochs), int(batch),
                                  ctypes.c_float(lr), ctypes.byref(loss)), "sur_train")
        return loss.value

    def predict(self, X):
        X = np.ascontiguousarray(X, np.float32)
        Y = np.zeros((X.shape[0], NOUT), np.float32)
        S = np.zeros((X.shape[0], NOUT), np.float32)
        check(self._lib.sur_predict(self._h, _lib.ptr(X), X.shape[0], _lib.ptr(Y), _lib.ptr(S)), "sur_predict")
        return Y, S

    def set_backend(self, tcgen05: bool):
        """Matrix products (training and prediction) on tcgen05 or mma.sync."""
        check(self._lib.sur_set_backend(self._h, 1 if tcgen05 else 0), "sur_set_backend")

    def bench_forward(self, n: int, reps: int = 20) -> float:
        """Device ms per forward pass of all members over the last n predicted
        rows (no host copies)."""
        ms = ctypes.c_double()
        check(self._lib.sur_bench_forward(self._h, int(n), int(reps), ctypes.byref(ms)), "sur_bench_forward")
        return ms.value

    def gradients(self, member, X, Y):
        X = np.ascontiguousarray(X, np.float32)
        Y = np.ascontiguousarray(Y, np.float32)
        g = [np.zeros((256, 16), np.float32), np.zeros(256, np.float32), np.zeros((256, 256), np.float32),
             np.zeros(256, np.float32), np.zeros((48, 256), np.float32), np.zeros(48, np.float32)]
        loss = ctypes.c_float()
        check(self._lib.sur_gradients(self._h, int(member), _lib.ptr(X), _lib.ptr(Y), X.shape[0], ctypes.byref(loss),
                                      *[_lib.ptr(a) for a in g]), "sur_gradients")
        return loss.value, g

    def set_weights(self, member, params):
        arrs = [np.ascontiguousarray(a, np.float32) for a in params]
        self._keep = arrs
        check(self._lib.sur_set_weights(self._h, int(member), *[_lib.ptr(a) for a in arrs]), "sur_set_weights")

    def set_scaling(self, mu_x, sd_x, mu_y, sd_y):
        a = [np.ascontiguousarray(v, np.float32) for v in (mu_x, sd_x, mu_y, sd_y)]
        check(self._lib.sur_set_scaling(self._h, *[_lib.ptr(v) for v in a]), "sur_set_scaling")

    def query(self, X, threshold, simulate_kw=None):
        """Predictions; rows whose largest relative member spread (spread /
        (|mean| + 1)) exceeds `threshold` are answered by the library running
        the simulation protocol (sur_query; simulate_kw: L, burn, n_snap,
        every, M, dr, seed as in simulate).  Returns (Y, used_fallback [n] bool)."""
        kw = dict(L=SUR_L, burn=2000, n_snap=10, every=200, M=128, dr=0.25, seed=0)
        kw.update(simulate_kw or {})
        pr = _lib.SurProtocol(float(kw["L"]), float(kw["dr"]), int(kw["burn"]), int(kw["n_snap"]),
                              int(kw["every"]), int(kw["M"]), int(kw["seed"]))
        X = np.ascontiguousarray(X, np.float32)
        Y = np.zeros((X.shape[0], NOUT), np.float32)
        fb = np.zeros(X.shape[0], np.int32)
        check(self._lib.sur_query(self._h, _lib.ptr(X), X.shape[0], ctypes.c_float(threshold), ctypes.byref(pr),
                                  _lib.ptr(Y), None, _lib.ptr(fb)), "sur_query")
        return Y, fb.astype(bool)

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.sur_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
