"""Host-side logic of the kernel-shape autotuner: the cache of tuned shapes
and argument validation (no GPU: these calls never touch CUDA)."""
import ctypes

import pytest


@pytest.fixture()
def tune():
    from paper_1310_0998_gb300 import tune as t
    t.clear()
    yield t
    t.clear()


def test_store_lookup_and_key(tune):
    assert tune.lookup(32.0, 1024) is None
    tune.store(32.0, 1024, 16, 4)
    assert tune.lookup(32.0, 1024) == (16, 4)
    # the key is (n_beads, L, r_c): physics parameters do not change it
    assert tune.lookup(32.0, 1024, gamma=20.0, zeta=1.0) == (16, 4)
    assert tune.lookup(32.0, 1026) is None
    assert tune.lookup(33.0, 1024) is None
    assert tune.lookup(32.0, 1024, rc=0.5) is None
    tune.store(32.0, 1024, 8, 2)          # a later result replaces the entry
    assert tune.lookup(32.0, 1024) == (8, 2)
    tune.clear()
    assert tune.lookup(32.0, 1024) is None


def test_batch_keys_are_separate(tune):
    from paper_1310_0998_gb300 import _lib, make_params
    L = _lib.lib()
    arr = (_lib.DpdParams * 2)(make_params(24.0, 600), make_params(32.0, 900))
    t, v = ctypes.c_int(), ctypes.c_int()
    assert L.dpd_tune_lookup(arr, 2, ctypes.byref(t), ctypes.byref(v)) == -6
    assert L.dpd_tune_store(arr, 2, 4, 3) == 0
    assert L.dpd_tune_lookup(arr, 2, ctypes.byref(t), ctypes.byref(v)) == 0
    assert (t.value, v.value) == (4, 3)
    # the first replica alone is a different (single-system) key
    assert tune.lookup(24.0, 600) is None
    # a different mix misses
    arr2 = (_lib.DpdParams * 2)(make_params(24.0, 600), make_params(32.0, 902))
    assert L.dpd_tune_lookup(arr2, 2, ctypes.byref(t), ctypes.byref(v)) == -6


def test_invalid_arguments_rejected(tune):
    from paper_1310_0998_gb300 import _lib, make_params
    L = _lib.lib()
    p = make_params(32.0, 1024)
    for tile, var in [(5, 2), (8, 0), (8, 6), (0, 0)]:
        assert L.dpd_tune_store(ctypes.byref(p), 1, tile, var) == -1
    assert L.dpd_tune_store(None, 1, 8, 2) == -1
    assert L.dpd_tune_store(ctypes.byref(p), 0, 8, 2) == -1
    rep = _lib.DpdTuneReport()
    # validation happens before any CUDA call
    assert L.dpd_autotune(ctypes.byref(p), None, None, 0, 0, None, ctypes.byref(rep)) == -1
    assert L.dpd_autotune(ctypes.byref(make_params(2.0, 10)), None, None, 0, 5, None, ctypes.byref(rep)) == -1
    assert L.dpd_autotune(ctypes.byref(p), None, None, 0, 5, None, None) == -1
    assert L.dpd_batch_autotune(None, 1, 5, None, ctypes.byref(rep)) == -1
