"""The recorded paper-preset run (Secs. 4-5.4): its summary under profiles/
holds the study's JSON output; the qualitative statements of Sec. 5.4 are
re-evaluated from the recorded spectra with the bands fixed in
paper_1310_0998_gb300.study, and must give the outcomes the summary
reports (held or not).  No GPU: this reads the record."""
import json
import math
import os
import re

import numpy as np
import pytest

from paper_1310_0998_gb300 import study

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RECORD = os.path.join(ROOT, "profiles", "paper_preset_study.md")


@pytest.fixture(scope="module")
def rec():
    text = open(RECORD).read()
    m = re.search(r"```json\n(.*?)\n```", text, re.S)
    assert m, "no JSON block in the record"
    return json.loads(m.group(1)), text


def test_record_is_the_paper_protocol(rec):
    r, _ = rec
    assert r["steps"] == 2_000_000 and r["burn"] == 1_800_000
    assert r["snapshots"] == 10 and r["every"] == 20_000
    pts = [(p["phi"], p["Gamma"], p["Gamma_s"]) for p in r["points"]]
    assert pts == [tuple(p) for p in study.POINTS]
    for p in r["points"]:
        assert p["agents"] == study.n_agents(p["phi"])


def test_slopes_and_peaks_follow_from_the_spectra(rec):
    """The recorded fit values are the study's own fits of the recorded
    normalised spectra (E / E_1 has the same log-slopes as E)."""
    r, _ = rec
    for p in r["points"]:
        e = np.asarray(p["E_over_E1"], np.float64)
        assert e.shape == (64,) and e[0] == 1.0 and np.all(e > 0)
        assert math.isclose(study.slope(e, 1, 10), p["alpha_low_k1_10"], rel_tol=1e-9, abs_tol=1e-12)
        assert math.isclose(study.slope(e, 20, 40), p["alpha_high_k20_40"], rel_tol=1e-9, abs_tol=1e-12)
        assert math.isclose(study.slope(e, 30, 60), p["alpha_high_k30_60"], rel_tol=1e-9, abs_tol=1e-12)
        assert int(np.argmax(e) + 1) == p["k_peak"]


def test_statement_outcomes_match_the_record(rec):
    """study.checks on the record equals the checks the run printed, and the
    summary's table states each outcome."""
    r, text = rec
    got = study.checks(r)
    assert got == r["checks"]
    for name, ok in got.items():
        line = next(l for l in text.splitlines() if l.startswith(f"| {name} "))
        assert ("| holds |" in line) == ok and ("| does not hold |" in line) == (not ok)


def test_temperatures_are_physical(rec):
    """Every point ran to a finite, positive temperature near or above k_BT
    (activity heats the fluid; Stokes friction cools it)."""
    r, _ = rec
    for p in r["points"]:
        assert math.isfinite(p["T"]) and 0.0 < p["T"] < 10.0
        assert math.isfinite(p["omega_rms"]) and p["omega_rms"] > 0.0
