"""Python face of the kernel-shape autotuner (wraps dpd_autotune,
dpd_batch_autotune and the dpd_tune_* cache calls of include/dpd.h)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import DpdParams, DpdTuneReport, check, ptr, where
from .sim import make_params


def autotune(L: float, n_beads: int, x=None, v=None, steps: int = 10, stream=None, **params) -> dict:
    """Time every (tile, variant) on the state x, v (None: the random initial
    condition of `seed`); the fastest is cached for (n_beads, L, r_c) and used
    by contexts created afterwards with tile = variant = 0."""
    p = make_params(L, n_beads, **params)
    rep = DpdTuneReport()
    xv = vv = None
    w = _lib.DPD_HOST
    if x is not None:
        w = where(x)
        if w == _lib.DPD_HOST:
            x = np.ascontiguousarray(x, np.float64)
            v = np.ascontiguousarray(np.zeros_like(x, dtype=np.float32) if v is None else v, np.float32)
        xv, vv = ptr(x), ptr(v)
    st = ctypes.c_void_p(int(stream)) if stream else None
    check(_lib.lib().dpd_autotune(ctypes.byref(p), xv, vv, w, int(steps), st, ctypes.byref(rep)), "dpd_autotune")
    return rep.as_dict()


def batch_autotune(points, steps: int = 10, stream=None) -> dict:
    """Time every (tile, variant 2-5) for a batch of replicas (same points as
    Ensemble); the fastest is cached for that replica mix."""
    arr = (DpdParams * len(points))()
    for r, pt in enumerate(points):
        pt = dict(pt)
        L, n = float(pt.pop("L")), int(pt.pop("n_beads"))
        arr[r] = make_params(L, n, **pt)
    rep = DpdTuneReport()
    st = ctypes.c_void_p(int(stream)) if stream else None
    check(_lib.lib().dpd_batch_autotune(ctypes.cast(arr, ctypes.c_void_p), len(points), int(steps), st,
                                        ctypes.byref(rep)), "dpd_batch_autotune")
    return rep.as_dict()


def store(L: float, n_beads: int, tile: int, variant: int, **params):
    """Seed the shape cache for one system (host only)."""
    p = make_params(L, n_beads, **params)
    check(_lib.lib().dpd_tune_store(ctypes.byref(p), 1, int(tile), int(variant)), "dpd_tune_store")


def lookup(L: float, n_beads: int, **params):
    """Cached (tile, variant) for one system, or None (host only)."""
    p = make_params(L, n_beads, **params)
    t, v = ctypes.c_int(), ctypes.c_int()
    s = _lib.lib().dpd_tune_lookup(ctypes.byref(p), 1, ctypes.byref(t), ctypes.byref(v))
    if s == _lib.DPD_OK:
        return int(t.value), int(v.value)
    if s == -6:
        return None
    check(s, "dpd_tune_lookup")


def clear():
    _lib.lib().dpd_tune_clear()
