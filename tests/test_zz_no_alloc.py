"""dpd_energy_spectrum_noalloc (static scratch, no allocation) against the
allocating dpd_energy_spectrum, through the C-ABI.

Two calls in a row must each reproduce the allocating path within the
tolerance the observables tests hold E(k) to (the two paths differ only in the
order of the atomic window sums), so the per-call clearing of the static
scratch is exercised; oversize M is refused.  Collected last so that it runs
after every other test as well as alone.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RTOL = 1e-9


def _sim(L, n_dimers, seed):
    from paper_1310_0998_gb300 import Sim, synth
    x, _ = synth.dimers(n_dimers, L, 0.5, seed)
    v = synth.velocities(2 * n_dimers, 1.0, seed + 1)
    s = Sim(L, 2 * n_dimers, gamma=4.5, zeta=0.1, f_p=1.0, seed=seed)
    s.set_state(x, v)
    s.step(5)
    return s


def _noalloc(s, M, eps=0.0):
    from paper_1310_0998_gb300 import _lib
    E = np.full(M // 2, np.nan)
    rc = _lib.lib().dpd_energy_spectrum_noalloc(s._h, int(M), float(eps), _lib.ptr(E))
    return rc, E


@pytest.mark.parametrize("L,nd,M,eps", [(32.0, 1200, 64, 0.0), (48.0, 3000, 256, 0.0), (40.0, 2000, 128, 3.0),
                                        (16.0, 300, 4, 0.0)])
def test_matches_allocating_path_twice(L, nd, M, eps):
    with _sim(L, nd, 7 + M) as s:
        ref = s.energy_spectrum(M, eps)
        for _ in range(2):
            rc, E = _noalloc(s, M, eps)
            assert rc == 0
            assert np.all(np.isfinite(E)) and np.all(E >= 0)
            np.testing.assert_allclose(E, ref, rtol=RTOL, atol=1e-300)


def test_rejects_oversize_and_bad_M():
    with _sim(32.0, 800, 3) as s:
        for M in (512, 1024, 96, 2):
            rc, E = _noalloc(s, M)
            assert rc == -1, M            # DPD_ERR_INVALID_ARG
            assert np.all(np.isnan(E))    # output untouched
        # a rejected call leaves the next valid one intact
        rc, E = _noalloc(s, 64)
        assert rc == 0
        np.testing.assert_allclose(E, s.energy_spectrum(64), rtol=RTOL)


def test_null_context_rejected():
    from paper_1310_0998_gb300 import _lib
    E = np.zeros(32)
    assert _lib.lib().dpd_energy_spectrum_noalloc(None, 64, 0.0, _lib.ptr(E)) == -1
