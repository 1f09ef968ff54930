"""Python face of a batched ensemble (wraps dpd_batch_* of include/dpd.h)."""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import DpdParams, check
from .sim import Sim, make_params


class Ensemble:
    """R replicas of uneven size and parameters, advanced together by one
    persistent kernel per call.  `points`: list of dicts with L, n_beads and
    any make_params keyword."""

    def __init__(self, points, stream=None):
        self._lib = _lib.lib()
        self.R = len(points)
        arr = (DpdParams * self.R)()
        self.points = []
        for r, pt in enumerate(points):
            pt = dict(pt)
            L, n = float(pt.pop("L")), int(pt.pop("n_beads"))
            arr[r] = make_params(L, n, **pt)
            self.points.append((L, n, dict(pt)))
        self._arr = arr
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(int(stream)) if stream else None
        check(self._lib.dpd_batch_create(ctypes.cast(arr, ctypes.c_void_p), self.R, st, ctypes.byref(h)),
              "dpd_batch_create")
        self._h = h
        self._views = [None] * self.R

    def replica(self, r: int) -> Sim:
        """Borrowed view of replica r: every Sim call except close() frees
        nothing."""
        if self._views[r] is None:
            v = ctypes.c_void_p()
            check(self._lib.dpd_batch_replica(self._h, int(r), ctypes.byref(v)), "dpd_batch_replica")
            L, n, kw = self.points[r]
            self._views[r] = Sim(L, n, _view=v, **kw)
        return self._views[r]

    def init_random(self, seed: int = 0):
        check(self._lib.dpd_batch_init_random(self._h, int(seed)), "dpd_batch_init_random")

    def step(self, n: int = 1):
        check(self._lib.dpd_batch_step(self._h, int(n)), "dpd_batch_step")

    def sync(self):
        check(self._lib.dpd_batch_sync(self._h), "dpd_batch_sync")

    def barrier_selftest(self) -> int:
        return int(self._lib.dpd_batch_barrier_selftest(self._h))

    def profile(self, nsteps: int = 16):
        """Run nsteps steps with the phase log on: per-step ms of the scan,
        scatter and force phases (barrier to barrier) and the mean ms a block
        worked in each."""
        import numpy as np
        out = np.zeros(6, np.float64)
        check(self._lib.dpd_batch_profile(self._h, int(nsteps), _lib.ptr(out)), "dpd_batch_profile")
        return {"scan_ms": out[0], "scatter_ms": out[1], "force_ms": out[2],
                "scan_busy_ms": out[3], "scatter_busy_ms": out[4], "force_busy_ms": out[5]}

    def info(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(self._lib.dpd_batch_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "dpd_batch_info")
        return dict(replicas=a.value, grid=b.value, work_tiles=c.value)

    def close(self):
        if getattr(self, "_h", None) is not None:
            for v in self._views:
                if v is not None:
                    v._h = None
            self._lib.dpd_batch_destroy(self._h)
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
