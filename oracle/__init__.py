"""FP64 CPU oracle for the self-propelled DPD dimer model (arXiv:1310.0998).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, ``__graft_entry__.smoke()`` (``build()`` compiles it) and the
CPU-baseline leg and reference arm of ``bench.py`` do.  It shares no code with
the CUDA library.

The particle dynamics (Sec. 2, Sec. 5) live in ``dpd_oracle.c`` (compiled with
``build()``); the observables of Sec. 5.3-5.4 live in ``observables.py`` (numpy,
FP64).  Arrays are in id order: bead i at row i, beads 2k and 2k+1 form agent k.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libdpd_oracle.so")
_lock = threading.Lock()
_lib = None


class OrcParams(ctypes.Structure):
    """Mirror of ``orc_params`` in dpd_oracle.c (the oracle's own definition)."""

    _fields_ = [
        ("L", ctypes.c_double),
        ("a", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("kBT", ctypes.c_double),
        ("rc", ctypes.c_double),
        ("kbond", ctypes.c_double),
        ("r0", ctypes.c_double),
        ("fp", ctypes.c_double),
        ("zeta", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("mass", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("replica", ctypes.c_uint32),
        ("exclude_bonded", ctypes.c_int32),
        ("noise", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("wexp", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile dpd_oracle.c into oracle/_build/libdpd_oracle.so (gcc, OpenMP,
    no floating-point contraction so x86 and Arm give the same bits)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER
            d, i64, u32, u64 = ctypes.c_double, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
            vp = ctypes.c_void_p
            L.orc_philox_batch.argtypes = [i64, vp, u32, u32, vp]
            L.orc_alpha.argtypes = [u32, u32, i64, u64, u32, ctypes.c_int]
            L.orc_alpha.restype = d
            L.orc_forces.argtypes = [P(OrcParams), i64, vp, vp, i64, vp]
            L.orc_forces.restype = i64
            L.orc_forces_cells.argtypes = [P(OrcParams), i64, vp, vp, i64, vp]
            L.orc_forces_cells.restype = i64
            L.orc_pair_forces_only.argtypes = [P(OrcParams), i64, vp, vp, i64, vp]
            L.orc_run.argtypes = [P(OrcParams), i64, vp, vp, vp, P(i64), i64, ctypes.c_int, vp]
            L.orc_cell_counts.argtypes = [i64, vp, d, ctypes.c_int32, vp]
            L.orc_pair_counts.argtypes = [P(OrcParams), i64, vp, d, vp, vp]
            L.orc_pair_counts.restype = i64
            L.orc_num_threads.restype = ctypes.c_int
            L.orc3_forces.argtypes = [P(OrcParams), i64, vp, vp, i64, vp]
            L.orc3_forces.restype = i64
            L.orc3_run.argtypes = [P(OrcParams), i64, vp, vp, vp, P(i64), i64, vp]
            _lib = L
    return _lib


def params(L, a, gamma, kBT, rc, kbond, r0, fp, zeta, dt, mass=1.0, seed=0, replica=0,
           exclude_bonded=1, noise=0, wexp=0.0) -> OrcParams:
    return OrcParams(float(L), float(a), float(gamma), float(kBT), float(rc), float(kbond),
                     float(r0), float(fp), float(zeta), float(dt), float(mass), int(seed),
                     int(replica), int(exclude_bonded), int(noise), 0, float(wexp))


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def philox(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32-10 of counters ctr [n,4] (uint32) under key (k0, k1)."""
    c, cp = _c(ctr, np.uint32)
    out = np.empty_like(c)
    lib().orc_philox_batch(c.shape[0], cp, int(key[0]), int(key[1]), out.ctypes.data_as(ctypes.c_void_p))
    return out


def alpha(i, j, step, seed, replica=0, noise=0) -> float:
    return lib().orc_alpha(int(i), int(j), int(step), int(seed), int(replica), int(noise))


def forces(p: OrcParams, x, v, step: int, cells: bool = False):
    """Total force (Sec. 2) on every bead; returns (f [n,2], interacting pairs)."""
    x, xp = _c(x, np.float64)
    v, vp = _c(v, np.float64)
    n = x.shape[0]
    f = np.zeros((n, 2), np.float64)
    fn = lib().orc_forces_cells if cells else lib().orc_forces
    npairs = fn(ctypes.byref(p), n, xp, vp, int(step), f.ctypes.data_as(ctypes.c_void_p))
    return f, int(npairs)


def pair_forces_only(p: OrcParams, x, v, step: int):
    x, xp = _c(x, np.float64)
    v, vp = _c(v, np.float64)
    f = np.zeros((x.shape[0], 2), np.float64)
    lib().orc_pair_forces_only(ctypes.byref(p), x.shape[0], xp, vp, int(step), f.ctypes.data_as(ctypes.c_void_p))
    return f


class State:
    """Canonical velocity-Verlet state (x_s, v_s, f_s) at step s, FP64."""

    def __init__(self, p: OrcParams, x, v, step: int = 0, f=None, cells: bool = False):
        self.p = p
        self.cells = cells
        self.x = np.array(x, np.float64, copy=True, order="C")
        self.v = np.array(v, np.float64, copy=True, order="C")
        self.step = int(step)
        if f is None:
            # set-up force: current velocities, random stream of this step
            f, _ = forces(p, self.x, self.v, self.step, cells)
        self.f = np.array(f, np.float64, copy=True, order="C")

    def run(self, nsteps: int, thermo: bool = False):
        """Advance nsteps velocity-Verlet steps; optional per-step
        (KE, Px, Py, sum Fx, sum Fy) log."""
        n = self.x.shape[0]
        st = ctypes.c_int64(self.step)
        log = np.zeros((max(nsteps, 1), 5), np.float64) if thermo else None
        lib().orc_run(ctypes.byref(self.p), n, self.x.ctypes.data_as(ctypes.c_void_p),
                      self.v.ctypes.data_as(ctypes.c_void_p), self.f.ctypes.data_as(ctypes.c_void_p),
                      ctypes.byref(st), int(nsteps), int(self.cells),
                      log.ctypes.data_as(ctypes.c_void_p) if thermo else None)
        self.step = st.value
        return log[:nsteps] if thermo else None


def forces3(p: OrcParams, x, v, step: int):
    """Three-dimensional variant: total force on every bead in the periodic
    cube of side p.L; returns (f [n,3], interacting pairs)."""
    x, xp = _c(x, np.float64)
    v, vp = _c(v, np.float64)
    f = np.zeros((x.shape[0], 3), np.float64)
    npairs = lib().orc3_forces(ctypes.byref(p), x.shape[0], xp, vp, int(step), f.ctypes.data_as(ctypes.c_void_p))
    return f, int(npairs)


class State3:
    """Velocity-Verlet state of the three-dimensional variant, FP64, all pairs."""

    def __init__(self, p: OrcParams, x, v, step: int = 0):
        self.p = p
        self.x = np.array(x, np.float64, copy=True, order="C")
        self.v = np.array(v, np.float64, copy=True, order="C")
        self.step = int(step)
        self.f, _ = forces3(p, self.x, self.v, self.step)

    def run(self, nsteps: int, thermo: bool = False):
        """Advance nsteps steps; optional per-step (KE, Px, Py, Pz, 0) log."""
        st = ctypes.c_int64(self.step)
        log = np.zeros((max(nsteps, 1), 5), np.float64) if thermo else None
        lib().orc3_run(ctypes.byref(self.p), self.x.shape[0], self.x.ctypes.data_as(ctypes.c_void_p),
                       self.v.ctypes.data_as(ctypes.c_void_p), self.f.ctypes.data_as(ctypes.c_void_p),
                       ctypes.byref(st), int(nsteps), log.ctypes.data_as(ctypes.c_void_p) if thermo else None)
        self.step = st.value
        return log[:nsteps] if thermo else None


def cell_counts(x, L: float, nc: int) -> np.ndarray:
    """Per-cell bead counts, cell floor(x nc / L), row-major [nc, nc]; x on
    the fixed-point grid X L / 2^32."""
    x, xp = _c(x, np.float64)
    out = np.zeros(nc * nc, np.uint32)
    lib().orc_cell_counts(x.shape[0], xp, float(L), int(nc), out.ctypes.data_as(ctypes.c_void_p))
    return out.reshape(nc, nc)


def pair_counts(p: OrcParams, x, tie: float = 4e-6):
    """Brute-force per-bead neighbour counts, ambiguous-tie counts, total."""
    x, xp = _c(x, np.float64)
    n = x.shape[0]
    cnt = np.zeros(n, np.uint32)
    amb = np.zeros(n, np.uint32)
    tot = lib().orc_pair_counts(ctypes.byref(p), n, xp, float(tie), cnt.ctypes.data_as(ctypes.c_void_p),
                                amb.ctypes.data_as(ctypes.c_void_p))
    return cnt, amb, int(tot)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def thermo(x, v, mass=1.0):
    """Kinetic energy, momentum and temperature; T = sum m|v|^2 / (2N - 2)
    (two translational degrees of freedom per bead, total momentum removed)."""
    v = np.asarray(v, np.float64)
    n = v.shape[0]
    ke = 0.5 * mass * float(np.sum(v * v))
    p = mass * v.sum(axis=0)
    T = 2.0 * ke / (2 * n - 2) if n > 1 else 0.0
    return ke, p, T


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print(_LIB)
