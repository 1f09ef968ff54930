"""The C-ABI library builds, loads and exports every declared entry point;
argument validation happens before any CUDA call (so it runs on the CPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b((?:dpd3?|ens|sur)_[A-Za-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    from paper_1310_0998_gb300 import _lib
    L = _lib.lib()
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_validation_without_gpu():
    from paper_1310_0998_gb300 import _lib, make_params
    L = _lib.lib()
    h = ctypes.c_void_p()
    bad = [
        make_params(2.9, 10),               # L < 3 r_c
        make_params(10.0, 9),               # odd bead count
        make_params(10.0, 0),
        make_params(10.0, 10, dt=0.0),
        make_params(10.0, 10, mass=-1.0),
        make_params(10.0, 10, gamma=-1.0),
        make_params(10.0, 10, tile=5),
        make_params(10.0, 10, noise=3),
        make_params(10.0, 10, rc=0.0),
    ]
    for p in bad:
        assert L.dpd_create(ctypes.byref(p), None, ctypes.byref(h)) == -1
    assert L.dpd_create(None, None, ctypes.byref(h)) == -1
    assert L.dpd_status_string(-5) == b"bounded device wait timed out"
    assert L.dpd_step(None, 1) == -1
    L.dpd_destroy(None)


def test_cell_side_rule():
    """n_c = floor(L / r_c): cells at least r_c wide."""
    import math
    for L, rc, nc in [(32.0, 1.0, 32), (1024.0, 1.0, 1024), (100.0, 0.5, 200), (3.0, 1.0, 3), (2.9, 1.0, 2)]:
        assert math.floor(L / rc) == nc
