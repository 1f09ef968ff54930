"""ctypes binding of libdpd (include/dpd.h): argument marshalling only.

Every step of the simulation runs in the CUDA library; this module only
converts arguments.  If the library cannot be loaded the calls raise: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdpd.so")

DPD_OK = 0
DPD_HOST, DPD_DEVICE = 0, 1
STATUS = {0: "DPD_OK", -1: "DPD_ERR_INVALID_ARG", -2: "DPD_ERR_CUDA", -3: "DPD_ERR_OOM",
          -4: "DPD_ERR_NONFINITE", -5: "DPD_ERR_TIMEOUT", -6: "DPD_ERR_STATE", -7: "DPD_ERR_INTERNAL"}


class DpdError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


class DpdParams(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_double),
        ("n_beads", ctypes.c_int64),
        ("a", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("kBT", ctypes.c_double),
        ("rc", ctypes.c_double),
        ("k_bond", ctypes.c_double),
        ("r0", ctypes.c_double),
        ("f_p", ctypes.c_double),
        ("zeta", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("mass", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("replica", ctypes.c_uint32),
        ("exclude_bonded", ctypes.c_int32),
        ("noise", ctypes.c_int32),
        ("tile", ctypes.c_int32),
        ("variant", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("wexp", ctypes.c_double),
    ]


class DpdInfo(ctypes.Structure):
    _fields_ = [
        ("n_beads", ctypes.c_int64),
        ("n_cells_side", ctypes.c_int32),
        ("tile", ctypes.c_int32),
        ("n_tiles", ctypes.c_int32),
        ("variant", ctypes.c_int32),
        ("step", ctypes.c_int64),
        ("overflow_tiles", ctypes.c_int64),
        ("device_bytes", ctypes.c_int64),
    ]


class DpdTuneReport(ctypes.Structure):
    _fields_ = [
        ("n_shapes", ctypes.c_int32),
        ("best_tile", ctypes.c_int32),
        ("best_variant", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("best_ms_per_step", ctypes.c_double),
        ("tile", ctypes.c_int32 * 16),
        ("variant", ctypes.c_int32 * 16),
        ("ms_per_step", ctypes.c_double * 16),
    ]

    def as_dict(self):
        n = self.n_shapes
        return {"best": {"tile": self.best_tile, "variant": self.best_variant,
                         "ms_per_step": self.best_ms_per_step},
                "shapes": [{"tile": self.tile[i], "variant": self.variant[i],
                            "ms_per_step": self.ms_per_step[i]} for i in range(n)]}


class SurProtocol(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_double),
        ("dr", ctypes.c_double),
        ("burn", ctypes.c_int32),
        ("n_snap", ctypes.c_int32),
        ("every", ctypes.c_int32),
        ("M", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
    ]


_lock = threading.Lock()
_lib = None


def _declare(L):
    P, vp, c_int, i64, u64, d = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sig = {
        "dpd_status_string": ([c_int], ctypes.c_char_p),
        "dpd_create": ([P(DpdParams), vp, P(vp)], c_int),
        "dpd_destroy": ([vp], None),
        "dpd_set_params": ([vp, P(DpdParams)], c_int),
        "dpd_set_state": ([vp, vp, vp, vp, i64, c_int], c_int),
        "dpd_init_random": ([vp, u64], c_int),
        "dpd_step": ([vp, i64], c_int),
        "dpd_sync": ([vp], c_int),
        "dpd_get_state": ([vp, vp, vp, vp, P(i64), c_int], c_int),
        "dpd_kinetic_energy": ([vp, P(d)], c_int),
        "dpd_momentum": ([vp, vp], c_int),
        "dpd_temperature": ([vp, P(d)], c_int),
        "dpd_thermo_log": ([vp, i64, i64, vp], c_int),
        "dpd_velocity_field": ([vp, c_int, d, vp, vp], c_int),
        "dpd_energy_spectrum": ([vp, c_int, d, vp], c_int),
        "dpd_energy_spectrum_noalloc": ([vp, c_int, d, vp], c_int),
        "dpd_vorticity": ([vp, c_int, d, vp], c_int),
        "dpd_velocity_correlation": ([vp, d, c_int, vp, P(d), vp, vp], c_int),
        "dpd_agent_speed": ([vp, P(d)], c_int),
        "dpd_cell_counts": ([vp, vp], c_int),
        "dpd_pair_counts": ([vp, vp, P(u64)], c_int),
        "dpd_get_info": ([vp, P(DpdInfo)], c_int),
        "dpd_profile_step": ([vp, vp], c_int),
        "dpd_error_info": ([vp, vp], c_int),
        "dpd_batch_create": ([vp, c_int, vp, P(vp)], c_int),
        "dpd_batch_destroy": ([vp], None),
        "dpd_batch_replica": ([vp, c_int, P(vp)], c_int),
        "dpd_batch_init_random": ([vp, u64], c_int),
        "dpd_batch_step": ([vp, i64], c_int),
        "dpd_batch_sync": ([vp], c_int),
        "dpd_batch_barrier_selftest": ([vp], c_int),
        "dpd_batch_info": ([vp, P(c_int), P(c_int), P(c_int)], c_int),
        "dpd_batch_profile": ([vp, c_int, vp], c_int),
        "dpd_autotune": ([P(DpdParams), vp, vp, c_int, c_int, vp, P(DpdTuneReport)], c_int),
        "dpd_batch_autotune": ([vp, c_int, c_int, vp, P(DpdTuneReport)], c_int),
        "dpd_tune_store": ([P(DpdParams), c_int, c_int, c_int], c_int),
        "dpd_tune_lookup": ([P(DpdParams), c_int, P(c_int), P(c_int)], c_int),
        "dpd_tune_clear": ([], None),
        "dpd3_create": ([P(DpdParams), vp, P(vp)], c_int),
        "dpd3_destroy": ([vp], None),
        "dpd3_set_state": ([vp, vp, vp, i64], c_int),
        "dpd3_step": ([vp, i64], c_int),
        "dpd3_sync": ([vp], c_int),
        "dpd3_get_state": ([vp, vp, vp, vp, P(i64)], c_int),
        "dpd3_thermo": ([vp, vp], c_int),
        "dpd3_velocity_field": ([vp, c_int, d, vp, vp], c_int),
        "dpd3_energy_spectrum": ([vp, c_int, d, vp], c_int),
        "dpd3_vorticity": ([vp, c_int, d, vp], c_int),
        "dpd3_velocity_correlation": ([vp, d, c_int, vp, P(d), vp, vp], c_int),
        "sur_create": ([c_int, c_int, u64, vp, P(vp)], c_int),
        "sur_destroy": ([vp], None),
        "sur_set_weights": ([vp, c_int, vp, vp, vp, vp, vp, vp], c_int),
        "sur_set_scaling": ([vp, vp, vp, vp, vp], c_int),
        "sur_gradients": ([vp, c_int, vp, vp, c_int, P(ctypes.c_float), vp, vp, vp, vp, vp, vp], c_int),
        "sur_train": ([vp, vp, vp, c_int, c_int, c_int, ctypes.c_float, P(ctypes.c_float)], c_int),
        "sur_predict": ([vp, vp, c_int, vp, vp], c_int),
        "sur_set_backend": ([vp, c_int], c_int),
        "sur_bench_forward": ([vp, c_int, c_int, P(d)], c_int),
        "sur_targets": ([c_int, c_int, c_int, d, vp, vp, vp, vp, vp], c_int),
        "sur_query": ([vp, vp, c_int, ctypes.c_float, P(SurProtocol), vp, vp, vp], c_int),
    }
    for name, (args, res) in sig.items():
        if hasattr(L, name):
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
    return L


def lib(build_if_missing: bool = True):
    """Load libdpd.so (building it in-tree first if needed).  Raises if the
    library cannot be built or loaded."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                from . import build as _build
                _build.build()
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libdpd.so missing at {LIB_PATH}; run paper_1310_0998_gb300/build.py")
            _lib = _declare(ctypes.CDLL(LIB_PATH))
    return _lib


def check(status: int, what: str):
    if status != DPD_OK:
        raise DpdError(status, what)


def ptr(a) -> ctypes.c_void_p:
    """Address of a C-contiguous numpy array or a torch tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    assert isinstance(a, np.ndarray) and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def where(a) -> int:
    if hasattr(a, "is_cuda") and a.is_cuda:
        return DPD_DEVICE
    return DPD_HOST
