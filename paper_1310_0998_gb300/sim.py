"""Python face of one simulated system (wraps dpd_* of include/dpd.h)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import DpdInfo, DpdParams, check, ptr, where

DEFAULTS = dict(a=25.0, gamma=4.5, kBT=1.0, rc=1.0, k_bond=100.0, r0=0.5, f_p=1.0, zeta=0.1,
                dt=0.01, mass=1.0, seed=0, replica=0, exclude_bonded=1, noise=0, tile=0, variant=0, wexp=0.0)


def make_params(L: float, n_beads: int, **kw) -> DpdParams:
    v = dict(DEFAULTS)
    alias = {"kbond": "k_bond", "fp": "f_p"}
    for k, x in kw.items():
        v[alias.get(k, k)] = x
    return DpdParams(float(L), int(n_beads), float(v["a"]), float(v["gamma"]), float(v["kBT"]),
                     float(v["rc"]), float(v["k_bond"]), float(v["r0"]), float(v["f_p"]), float(v["zeta"]),
                     float(v["dt"]), float(v["mass"]), int(v["seed"]), int(v["replica"]),
                     int(v["exclude_bonded"]), int(v["noise"]), int(v["tile"]), int(v["variant"]), 0,
                     float(v["wexp"]))


class Sim:
    """One periodic box of N beads (N/2 dimers) on the current CUDA device."""

    def __init__(self, L: float, n_beads: int, stream=None, _view=None, **params):
        self.L = self._lib = None
        self._lib = _lib.lib()
        self.params = make_params(L, n_beads, **params)
        self.L = float(L)
        self.n = int(n_beads)
        self._owned = _view is None
        if _view is not None:       # a replica of a batch: borrowed handle
            self._h = _view
            return
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(int(stream)) if stream else None
        check(self._lib.dpd_create(ctypes.byref(self.params), st, ctypes.byref(h)), "dpd_create")
        self._h = h

    # -------------------------------------------------------------- state
    def set_state(self, x, v, f=None, step: int = 0):
        """x: [N,2] float64 positions, v: [N,2] float32 velocities, f: [N,2]
        float32 forces of that state or None (set-up force); id order; numpy
        arrays (host) or CUDA tensors (device)."""
        if hasattr(x, "is_cuda"):
            import torch
            torch.cuda.current_stream().synchronize()
        else:
            x = np.ascontiguousarray(x, np.float64)
            v = np.ascontiguousarray(v, np.float32)
            if f is not None:
                f = np.ascontiguousarray(f, np.float32)
        assert tuple(x.shape) == (self.n, 2) and tuple(v.shape) == (self.n, 2)
        check(self._lib.dpd_set_state(self._h, ptr(x), ptr(v), ptr(f), int(step), where(x)), "dpd_set_state")

    def set_positions(self, x, v=None, step: int = 0):
        if v is None:
            v = np.zeros((self.n, 2), np.float32)
        self.set_state(x, v, None, step)

    def init_random(self, seed: int = 0):
        check(self._lib.dpd_init_random(self._h, int(seed)), "dpd_init_random")

    def step(self, n: int = 1):
        check(self._lib.dpd_step(self._h, int(n)), "dpd_step")

    def sync(self):
        check(self._lib.dpd_sync(self._h), "dpd_sync")

    def get_state(self, out_x=None, out_v=None, out_f=None):
        """Canonical (x [N,2] float64, v [N,2] float32, f [N,2] float32, step);
        host numpy unless CUDA tensors are passed as outputs."""
        x = out_x if out_x is not None else np.empty((self.n, 2), np.float64)
        v = out_v if out_v is not None else np.empty((self.n, 2), np.float32)
        f = out_f if out_f is not None else np.empty((self.n, 2), np.float32)
        s = ctypes.c_int64()
        check(self._lib.dpd_get_state(self._h, ptr(x), ptr(v), ptr(f), ctypes.byref(s), where(x)),
              "dpd_get_state")
        return x, v, f, s.value

    # -------------------------------------------------------- observables
    def kinetic_energy(self) -> float:
        x = ctypes.c_double()
        check(self._lib.dpd_kinetic_energy(self._h, ctypes.byref(x)), "dpd_kinetic_energy")
        return x.value

    def momentum(self):
        p = np.zeros(2, np.float64)
        check(self._lib.dpd_momentum(self._h, ptr(p)), "dpd_momentum")
        return p

    def temperature(self) -> float:
        x = ctypes.c_double()
        check(self._lib.dpd_temperature(self._h, ctypes.byref(x)), "dpd_temperature")
        return x.value

    def thermo_log(self, first: int, count: int):
        out = np.zeros((count, 4), np.float64)
        check(self._lib.dpd_thermo_log(self._h, int(first), int(count), ptr(out)), "dpd_thermo_log")
        return out

    def velocity_field(self, M: int = 128, eps: float = 0.0):
        u = np.zeros((M, M, 2), np.float64)
        n = np.zeros((M, M), np.float64)
        check(self._lib.dpd_velocity_field(self._h, int(M), float(eps), ptr(u), ptr(n)), "dpd_velocity_field")
        return u, n

    def energy_spectrum(self, M: int = 128, eps: float = 0.0):
        E = np.zeros(M // 2, np.float64)
        check(self._lib.dpd_energy_spectrum(self._h, int(M), float(eps), ptr(E)), "dpd_energy_spectrum")
        return E

    def vorticity(self, M: int = 128, eps: float = 0.0):
        om = np.zeros((M, M), np.float64)
        check(self._lib.dpd_vorticity(self._h, int(M), float(eps), ptr(om)), "dpd_vorticity")
        return om

    def velocity_correlation(self, dr: float, nbins: int):
        g = np.zeros(nbins, np.float64)
        num = np.zeros(nbins, np.float64)
        cnt = np.zeros(nbins, np.int64)
        Li = ctypes.c_double()
        check(self._lib.dpd_velocity_correlation(self._h, float(dr), int(nbins), ptr(g), ctypes.byref(Li),
                                                 ptr(num), ptr(cnt)), "dpd_velocity_correlation")
        return g, Li.value, num, cnt

    # -------------------------------------------------------------- debug
    def agent_speed(self) -> float:
        """Mean over agents of |v_COM| (Sec. 5.3), FP64 on the device."""
        out = ctypes.c_double()
        check(self._lib.dpd_agent_speed(self._h, ctypes.byref(out)), "dpd_agent_speed")
        return out.value

    def cell_counts(self):
        nc = self.info().n_cells_side
        out = np.zeros((nc, nc), np.uint32)
        check(self._lib.dpd_cell_counts(self._h, ptr(out)), "dpd_cell_counts")
        return out

    def pair_counts(self):
        cnt = np.zeros(self.n, np.uint32)
        tot = ctypes.c_uint64()
        check(self._lib.dpd_pair_counts(self._h, ptr(cnt), ctypes.byref(tot)), "dpd_pair_counts")
        return cnt, tot.value

    def profile_step(self):
        """One step with per-kernel CUDA-event times (scan, scatter, force) in ms."""
        ms = np.zeros(3, np.float64)
        check(self._lib.dpd_profile_step(self._h, ptr(ms)), "dpd_profile_step")
        return ms

    def error_info(self):
        """(site, v1, v2, v3) of the first failed device check (site 0: none)."""
        out = np.zeros(4, np.int64)
        check(self._lib.dpd_error_info(self._h, ptr(out)), "dpd_error_info")
        return tuple(int(v) for v in out)

    def info(self) -> DpdInfo:
        inf = DpdInfo()
        check(self._lib.dpd_get_info(self._h, ctypes.byref(inf)), "dpd_get_info")
        return inf

    def close(self):
        if getattr(self, "_h", None) is not None and self._lib is not None:
            if getattr(self, "_owned", True):
                self._lib.dpd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Sim3:
    """Three-dimensional variant: one periodic cube of N beads (wraps dpd3_*)."""

    def __init__(self, L: float, n_beads: int, stream=None, **params):
        self._lib = _lib.lib()
        self.L, self.n = float(L), int(n_beads)
        self._p = make_params(L, n_beads, **params)
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(int(stream)) if stream else None
        check(self._lib.dpd3_create(ctypes.byref(self._p), st, ctypes.byref(h)), "dpd3_create")
        self._h = h

    def set_positions(self, x, v=None, step: int = 0):
        x = np.ascontiguousarray(x, np.float64)
        v = np.zeros((self.n, 3), np.float32) if v is None else np.ascontiguousarray(v, np.float32)
        check(self._lib.dpd3_set_state(self._h, ptr(x), ptr(v), int(step)), "dpd3_set_state")

    def step(self, n: int = 1):
        check(self._lib.dpd3_step(self._h, int(n)), "dpd3_step")

    def sync(self):
        check(self._lib.dpd3_sync(self._h), "dpd3_sync")

    def get_state(self):
        x = np.zeros((self.n, 3), np.float64)
        v = np.zeros((self.n, 3), np.float32)
        f = np.zeros((self.n, 3), np.float32)
        st = ctypes.c_int64()
        check(self._lib.dpd3_get_state(self._h, ptr(x), ptr(v), ptr(f), ctypes.byref(st)), "dpd3_get_state")
        return x, v, f, st.value

    def thermo(self):
        """(KE, Px, Py, Pz, T) of the current step, FP64."""
        out = np.zeros(5, np.float64)
        check(self._lib.dpd3_thermo(self._h, ptr(out)), "dpd3_thermo")
        return out

    # ---------------------------------------------------- observables
    def velocity_field(self, M: int = 32, eps: float = 0.0):
        """u_M [iz, iy, ix, 3] and the window counts [iz, iy, ix]."""
        u = np.zeros((M, M, M, 3), np.float64)
        n = np.zeros((M, M, M), np.float64)
        check(self._lib.dpd3_velocity_field(self._h, int(M), float(eps), ptr(u), ptr(n)), "dpd3_velocity_field")
        return u, n

    def energy_spectrum(self, M: int = 32, eps: float = 0.0):
        E = np.zeros(M // 2, np.float64)
        check(self._lib.dpd3_energy_spectrum(self._h, int(M), float(eps), ptr(E)), "dpd3_energy_spectrum")
        return E

    def vorticity(self, M: int = 32, eps: float = 0.0):
        """curl u_M [iz, iy, ix, 3]."""
        om = np.zeros((M, M, M, 3), np.float64)
        check(self._lib.dpd3_vorticity(self._h, int(M), float(eps), ptr(om)), "dpd3_vorticity")
        return om

    def velocity_correlation(self, dr: float, nbins: int):
        g = np.zeros(nbins, np.float64)
        num = np.zeros(nbins, np.float64)
        cnt = np.zeros(nbins, np.int64)
        Li = ctypes.c_double()
        check(self._lib.dpd3_velocity_correlation(self._h, float(dr), int(nbins), ptr(g), ctypes.byref(Li),
                                                  ptr(num), ptr(cnt)), "dpd3_velocity_correlation")
        return g, Li.value, num, cnt

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.dpd3_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
