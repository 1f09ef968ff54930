"""The surrogate's 40 target statistics (sur_targets, host code of the
library) against the definitions written out again here in numpy: shell-pair
logarithms of E(k) (Sec. 5.4), the correlation length and integral length of
g(r) (Sec. 5.3, Eq. spatial01 with the trapezoid from g(0) = 1), the
low- and high-wavenumber least-squares slopes, the peak, ln E_1, and the
snapshot means of T and |v_COM|.  No GPU."""
import ctypes
import math

import numpy as np
import pytest

from paper_1310_0998_gb300 import _lib


def _reference(E, g, T, vc, dr):
    E = np.mean(E, axis=0)
    with np.errstate(all="ignore"):
        cnt = np.sum(~np.isnan(g), axis=0)
        gm = np.where(cnt > 0, np.nansum(g, axis=0) / np.maximum(cnt, 1), 0.0)
    out = np.zeros(40)
    for b in range(32):
        out[b] = math.log(max(0.5 * (E[2 * b] + E[2 * b + 1]), 1e-300))
    r = np.concatenate([[0.0], (np.arange(gm.size) + 0.5) * dr])
    gg = np.concatenate([[1.0], gm])
    idx = [i for i in range(1, gg.size) if gg[i] <= math.exp(-1)]
    if idx:
        i = idx[0]
        out[32] = r[i - 1] + (gg[i - 1] - math.exp(-1)) / max(gg[i - 1] - gg[i], 1e-300) * (r[i] - r[i - 1])
    else:
        out[32] = r[-1]
    out[33] = sum(0.5 * (gg[i] + gg[i - 1]) * (r[i] - r[i - 1]) for i in range(1, gg.size))
    out[34] = np.mean(T)
    for o, (k0, k1) in ((35, (1, 10)), (36, (30, 60))):
        k = np.arange(k0, k1 + 1, dtype=np.float64)
        out[o] = np.polyfit(np.log(k), np.log(E[k0 - 1:k1] / E[0]), 1)[0]
    out[37] = np.argmax(E) + 1
    out[38] = math.log(max(E[0], 1e-300))
    out[39] = np.mean(vc)
    return out


def _call(E, g, T, vc, dr):
    L = _lib.lib()
    E, g, T, vc = (np.ascontiguousarray(a, np.float64) for a in (E, g, T, vc))
    out = np.zeros(40)
    rc = L.sur_targets(E.shape[0], E.shape[1], g.shape[1], float(dr), _lib.ptr(E), _lib.ptr(g), _lib.ptr(T),
                       _lib.ptr(vc), _lib.ptr(out))
    return rc, out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_targets_match_definitions(seed):
    rng = np.random.default_rng(seed)
    s, nsh, nb, dr = 3, 64, 96, 0.25
    k = np.arange(1, nsh + 1)
    E = (k ** 0.8 * np.exp(-k / 15.0))[None, :] * rng.uniform(0.5, 1.5, (s, nsh))
    r = (np.arange(nb) + 0.5) * dr
    g = np.exp(-r / 3.0)[None, :] + rng.normal(0, 0.02, (s, nb))
    g[1, 5] = np.nan                      # an empty bin in one snapshot
    g[:, 40] = np.nan                     # a bin empty in every snapshot
    T, vc = rng.uniform(0.9, 1.1, s), rng.uniform(0.1, 2.0, s)
    rc, out = _call(E, g, T, vc, dr)
    assert rc == 0
    np.testing.assert_allclose(out, _reference(E, g, T, vc, dr), rtol=1e-12, atol=1e-12)


def test_no_crossing_zero_shell_and_bad_arguments():
    s, nsh, nb, dr = 2, 64, 10, 0.5
    E = np.ones((s, nsh))
    E[:, 3] = 0.0                          # ln of 0 is clamped at 1e-300 in the pair bins
    g = np.full((s, nb), 0.9)              # never falls to 1/e: the last centre
    T, vc = np.ones(s), np.ones(s)
    rc, out = _call(E, g, T, vc, dr)
    assert rc == 0
    ref = _reference(E, g, T, vc, dr)
    np.testing.assert_allclose(out[np.isfinite(ref)], ref[np.isfinite(ref)], rtol=1e-12, atol=1e-12)
    assert out[32] == (nb - 0.5) * dr
    assert out[1] == pytest.approx(math.log(0.5))
    rc, _ = _call(E[:, :63], g, T, vc, dr)   # fewer than 64 shells
    assert rc != 0
