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


def test_plain_c_consumer_compiles_links_and_runs(tmp_path):
    """include/dpd.h is a C header (no C++ in its declarations): a C99
    program includes it, links against libdpd.so and calls a host-only entry
    point (sur_targets, no device work) and the status strings."""
    import shutil
    import subprocess
    from paper_1310_0998_gb300 import _lib
    _lib.lib()   # builds the library if needed
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "consumer.c"
    src.write_text(r'''
#include <math.h>
#include <stdio.h>
#include "dpd.h"
int main(void) {
    double E[64], g[4], T[1] = {1.0}, vc[1] = {0.5}, out[40];
    for (int k = 0; k < 64; ++k) E[k] = 1.0 / (k + 1);
    for (int b = 0; b < 4; ++b) g[b] = 1.0 - 0.3 * b;
    int rc = sur_targets(1, 64, 4, 0.5, E, g, T, vc, out);
    if (rc != DPD_OK) return 1;
    if (fabs(out[34] - 1.0) > 1e-15 || fabs(out[39] - 0.5) > 1e-15) return 2;
    if (dpd_status_string(DPD_ERR_INVALID_ARG) == NULL) return 3;
    if (sur_targets(1, 63, 4, 0.5, E, g, T, vc, out) == DPD_OK) return 4;
    printf("ok\n");
    return 0;
}
''')
    exe = tmp_path / "consumer"
    libdir = os.path.dirname(_lib.LIB_PATH)
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-ldpd", "-lm", "-Wl,-rpath," + libdir], check=True, timeout=120)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert out.stdout.strip() == "ok"
