"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test would fail under a plausible slip in the oracle (a dropped term, a
wrong sign or index, a wrong factor).  No GPU needed.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1310_0998_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def P(orc, **kw):
    base = dict(L=10.0, a=25.0, gamma=4.5, kBT=1.0, rc=1.0, kbond=100.0, r0=0.5, fp=1.0,
                zeta=0.1, dt=0.01, mass=1.0, seed=0, exclude_bonded=1, noise=0)
    base.update(kw)
    return orc.params(**base)


# --------------------------------------------------------------------------
# Philox4x32-10
# --------------------------------------------------------------------------

def test_philox_matches_triton_interpreter(orc, tmp_path):
    """Triton ships an independent Philox4x32-10 (tl.philox); its CPU
    interpreter evaluates it with numpy.  The oracle must agree bit for bit."""
    pytest.importorskip("triton")
    import subprocess
    import sys

    rng = np.random.default_rng(7)
    n = 256
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    helper = os.path.join(os.path.dirname(__file__), "triton_philox_ref.py")
    for k, seed in enumerate((0, 0x123456789ABCDEF, 2**64 - 1)):
        path = str(tmp_path / f"ctr{k}.npz")
        np.savez(path, ctr=ctr, seed=np.uint64(seed))
        env = dict(os.environ, TRITON_INTERPRET="1")
        subprocess.run([sys.executable, helper, path], check=True, env=env, timeout=600)
        tri = np.load(path + ".out.npy")
        ours = orc.philox(ctr, (seed & 0xFFFFFFFF, seed >> 32))
        np.testing.assert_array_equal(ours, tri)


def test_philox_uniformity_and_alpha_moments(orc):
    n = 1 << 20
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    ctr[:, 2] = 12345
    w = orc.philox(ctr, (0xDEADBEEF, 0x1234))
    u = ((w[:, 0] >> 8).astype(np.float64) + 0.5) / 2**24
    assert abs(u.mean() - 0.5) < 3e-4 * 4
    assert abs(u.var() - 1.0 / 12.0) < 2e-4
    hist = np.bincount((w[:, 1] >> 24).astype(np.int64), minlength=256)
    chi2 = float(((hist - n / 256) ** 2 / (n / 256)).sum())
    assert chi2 < 255 + 6 * math.sqrt(2 * 255)
    # the alpha mapping: zero mean, unit variance, symmetric in (i, j)
    a = np.array([orc.alpha(i, i + 1 + (i % 7), 3, 99) for i in range(20000)])
    assert abs(a.mean()) < 4 / math.sqrt(20000)
    assert abs(a.var() - 1.0) < 0.03
    assert np.abs(a).max() < math.sqrt(3.0)
    for i, j in [(0, 1), (5, 900), (123456, 7)]:
        assert orc.alpha(i, j, 17, 5) == orc.alpha(j, i, 17, 5)
        assert orc.alpha(i, j, 17, 5) != orc.alpha(i, j, 18, 5)
        assert orc.alpha(i, j, 17, 5) != orc.alpha(i, j, 17, 6)
    g = np.array([orc.alpha(i, 2 * i + 3, 1, 4, noise=1) for i in range(20000)])
    assert abs(g.mean()) < 4 / math.sqrt(20000)
    assert abs(g.var() - 1.0) < 0.04
    assert abs(float(np.mean(g ** 4)) - 3.0) < 0.25


# --------------------------------------------------------------------------
# Pair force, hand-derived (golden fixtures)
# --------------------------------------------------------------------------

def test_pair_force_golden_cases(orc):
    cases = json.load(open(os.path.join(GOLDEN, "pair_cases.json")))["cases"]
    for c in cases:
        p = P(orc, L=c["L"], a=c["a"], gamma=c["gamma"], kBT=c["kBT"], rc=c["rc"], exclude_bonded=0)
        f = orc.pair_forces_only(p, np.array(c["x"]), np.array(c["v"]), 1)
        np.testing.assert_allclose(f[0], c["f0"], atol=1e-12, err_msg=c["name"])
        np.testing.assert_allclose(f[1], -np.array(c["f0"]), atol=1e-12, err_msg=c["name"])


def test_random_force_scaling(orc):
    """f_R = sqrt(2 gamma kBT) w alpha dt^-1/2 e: pure random part with A = 0
    and zero velocities scales as sqrt(gamma kBT / dt); its direction is e."""
    x = np.array([[5.0, 5.0], [5.0, 5.6]])
    v = np.zeros((2, 2))
    base = orc.pair_forces_only(P(orc, a=0.0, gamma=2.0, kBT=1.0, dt=0.01, exclude_bonded=0), x, v, 9)
    assert abs(base[0, 0]) < 1e-14 and abs(base[0, 1]) > 0
    al = orc.alpha(0, 1, 9, 0)
    np.testing.assert_allclose(base[0, 1], -math.sqrt(2 * 2.0 * 1.0) * 0.4 * al / math.sqrt(0.01), rtol=1e-13)
    f2 = orc.pair_forces_only(P(orc, a=0.0, gamma=8.0, kBT=1.0, dt=0.04, exclude_bonded=0), x, v, 9)
    np.testing.assert_allclose(f2, base, rtol=1e-13)   # 4x gamma, 4x dt
    f3 = orc.pair_forces_only(P(orc, a=0.0, gamma=2.0, kBT=4.0, dt=0.01, exclude_bonded=0), x, v, 9)
    np.testing.assert_allclose(f3, 2 * base, rtol=1e-13)


def test_bonded_pair_switched_off_and_superposition(orc):
    """Sec. 2.2: no pair force inside a dimer; pair forces superpose."""
    x = np.array([[5.0, 5.0], [5.4, 5.0], [5.0, 5.7], [8.0, 8.0]])
    v = np.zeros((4, 2))
    p_on = P(orc, gamma=0.0, kBT=0.0, exclude_bonded=1)
    f = orc.pair_forces_only(p_on, x, v, 1)
    # bead 0 sees only bead 2 (bead 1 is its partner): r = 0.7, w = 0.3, e = -y
    np.testing.assert_allclose(f[0], [0.0, -25 * 0.3], atol=1e-12)
    # bead 1 sees bead 2: d = (0.4, -0.7), r = 0.806..., beyond? r < 1
    d = np.array([0.4, -0.7]); r = np.hypot(*d)
    np.testing.assert_allclose(f[1], 25 * (1 - r) * d / r, atol=1e-12)
    np.testing.assert_allclose(f[3], [0, 0], atol=1e-14)
    p_off = P(orc, gamma=0.0, kBT=0.0, exclude_bonded=0)
    f_off = orc.pair_forces_only(p_off, x, v, 1)
    np.testing.assert_allclose(f_off[0] - f[0], [-25 * 0.6, 0.0], atol=1e-12)


# --------------------------------------------------------------------------
# Dynamics: conservation laws and closed forms
# --------------------------------------------------------------------------

def _bead_momentum(v):
    return v.sum(axis=0)


def test_momentum_conserved_without_drag_and_propulsion(orc):
    x, _ = synth.dimers(128, 12.0, 0.5, seed=3)
    v = synth.velocities(256, 1.0, seed=4).astype(np.float64)
    p = P(orc, L=12.0, zeta=0.0, fp=0.0)
    st = orc.State(p, x, v, step=0)
    P0 = _bead_momentum(st.v).copy()
    scale = np.abs(st.v).sum()
    st.run(1000)
    assert np.abs(_bead_momentum(st.v) - P0).max() <= 1e-10 * scale


def test_discrete_momentum_balance(orc):
    """With drag and propulsion: pair and bond forces cancel, so the total
    force is sum_k 2 f_p n_k - zeta sum_i v_i(half step).  With the per-step
    log, v_half = v_{s+1} - (dt/2m) f_{s+1} gives
    sum F_{s+1} (1 - zeta dt / 2m) = 2 f_p sum_k n_k - zeta P_{s+1}."""
    L = 12.0
    x, v = synth.dimers(128, L, 0.5, seed=5)
    p = P(orc, L=L, zeta=0.7, fp=1.3, dt=0.01)
    st = orc.State(p, x, v)
    for _ in range(5):
        log = st.run(20, thermo=True)
        xh, xt = st.x[0::2], st.x[1::2]
        d = xh - xt
        d -= L * np.rint(d / L)
        n = d / np.linalg.norm(d, axis=1)[:, None]
        lhs = log[-1, 3:5] * (1 - 0.7 * 0.01 / 2)
        rhs = 2 * 1.3 * n.sum(axis=0) - 0.7 * log[-1, 1:3]
        np.testing.assert_allclose(lhs, rhs, atol=1e-9 * (1 + np.abs(rhs).max()))
        # integrator bookkeeping: P_{s+1} - P_s = dt/2 (F_s + F_{s+1})
        dP = log[1:, 1:3] - log[:-1, 1:3]
        np.testing.assert_allclose(dP, 0.005 * (log[1:, 3:5] + log[:-1, 3:5]), atol=1e-10)


def test_continuous_momentum_balance(orc):
    """dP/dt = sum F_p - zeta P, the balance of total momentum under propulsion
    and drag, to O(dt^2)."""
    L = 12.0
    x, v = synth.dimers(100, L, 0.5, seed=8)
    zeta, fp, dt = 0.5, 1.0, 0.005
    p = P(orc, L=L, zeta=zeta, fp=fp, dt=dt)
    st = orc.State(p, x, v)
    st.run(50)
    P0 = st.v.sum(axis=0).copy()
    xh, xt = st.x[0::2], st.x[1::2]
    d = xh - xt; d -= L * np.rint(d / L)
    Fp = 2 * fp * (d / np.linalg.norm(d, axis=1)[:, None]).sum(axis=0)
    st.run(1)
    dPdt = (st.v.sum(axis=0) - P0) / dt
    np.testing.assert_allclose(dPdt, Fp - zeta * P0, atol=0.02 * (1 + np.abs(Fp).max()))


def test_single_dimer_drift_speed(orc):
    """One dimer alone: both beads feel f_p n - zeta v, the bond stays at
    rest, and the speed obeys the velocity-Verlet recurrence with the drag on
    the half-step velocity; it tends to the terminal speed f_p/zeta."""
    L, r0, fp, zeta, dt = 32.0, 0.5, 1.0, 0.1, 0.01
    th = 0.3
    c = np.array([10.0, 12.0])
    h = 0.5 * r0 * np.array([math.cos(th), math.sin(th)])
    x = np.array([c + h, c - h])
    v = np.zeros((2, 2))
    p = P(orc, L=L, r0=r0, fp=fp, zeta=zeta, dt=dt)
    st = orc.State(p, x, v)
    # scalar recurrence along n (not the oracle's code: one particle, one force)
    u, fcur, hh = 0.0, fp, 0.5 * dt
    for _ in range(3000):
        uh = u + hh * fcur
        fcur = fp - zeta * uh
        u = uh + hh * fcur
    st.run(3000)
    n = np.array([math.cos(th), math.sin(th)])
    np.testing.assert_allclose(st.v[0] @ n, u, rtol=1e-12)
    np.testing.assert_allclose(st.v[1], st.v[0], atol=1e-12)
    st.run(20000)
    assert abs(st.v[0] @ n - fp / zeta) < 1e-3 * fp / zeta


def test_bond_oscillation_frequency(orc):
    """Two beads on a spring kappa: the separation oscillates about r0 with
    omega = sqrt(2 kappa / m) (reduced mass m/2), Eq. (stiffSpring)."""
    kb, r0, dt, delta = 100.0, 0.5, 0.001, 0.05
    x = np.array([[5.0 + 0.5 * (r0 + delta), 5.0], [5.0 - 0.5 * (r0 + delta), 5.0]])
    p = P(orc, L=10.0, kbond=kb, r0=r0, fp=0.0, zeta=0.0, gamma=0.0, kBT=0.0, dt=dt)
    st = orc.State(p, x, np.zeros((2, 2)))
    seps = []
    for _ in range(2000):
        st.run(1)
        seps.append(st.x[0, 0] - st.x[1, 0] - r0)
    seps = np.array(seps)
    t = (np.arange(len(seps)) + 1) * dt
    crossings = t[1:][np.sign(seps[1:]) != np.sign(seps[:-1])]
    period = 2 * np.mean(np.diff(crossings))
    omega = math.sqrt(2 * kb)
    assert abs(period - 2 * math.pi / omega) < 2e-3 * (2 * math.pi / omega)
    assert abs(np.abs(seps).max() - delta) < 2e-3


@pytest.mark.slow
def test_equilibrium_temperature(orc):
    """zeta = f_p = 0: the DPD thermostat holds T = kBT (fluctuation-
    dissipation sigma^2 = 2 gamma kBT, w_D = w_R^2; Sec. 2.1).  C1 geometry.
    The random start relaxes over ~5e3 steps and T then wanders slowly; over
    steps 5e3..4.5e4 one run's <T> scatters by 0.56% between seeds about
    1.005 (24 seeds), so the 2% bound is more than five of those."""
    L = 32.0
    x, v = synth.dimers(512, L, 0.5, seed=0)
    p = P(orc, L=L, zeta=0.0, fp=0.0, seed=11)
    st = orc.State(p, x, v, cells=True)
    st.run(5000)
    log = st.run(40000, thermo=True)
    n = x.shape[0]
    T = 2 * log[:, 0] / (2 * n - 2)
    assert abs(T.mean() - 1.0) < 0.02, T.mean()


def test_weight_exponent_reduces_to_printed_form(orc):
    """The changed-exponent path (pow) at s = 2 + 1e-12 gives the forces of the
    printed Eq. (DPDcdr) (w^2 and w, the s = 2 path) to rounding."""
    L = 9.0
    x, _ = synth.dimers(150, L, 0.5, seed=4)
    v = synth.velocities(300, 1.0, seed=5)
    f2, n2 = orc.forces(P(orc, L=L), x, v.astype(np.float64), 3)
    fs, ns = orc.forces(P(orc, L=L, wexp=2.0 + 1e-12), x, v.astype(np.float64), 3)
    assert n2 == ns
    np.testing.assert_allclose(fs, f2, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("s", [0.5, 1.0, 3.0])
def test_weight_exponent_power_laws(orc, s):
    """With the exponent s, the random part scales as w^(s/2) and the
    dissipative part as w^s with the separation (same pair, same step, so the
    same alpha): ratios at two separations along e."""
    v0 = np.zeros((2, 2))
    vr = np.array([[0.0, 0.0], [0.0, 0.7]])   # j (above i) recedes along +y
    r1, r2 = 0.35, 0.8
    w1, w2 = 1 - r1, 1 - r2
    out = {}
    for r in (r1, r2):
        x = np.array([[5.0, 5.0], [5.0, 5.0 + r]])
        fr = orc.pair_forces_only(P(orc, a=0.0, gamma=2.0, kBT=1.0, wexp=s, exclude_bonded=0), x, v0, 9)
        fd = orc.pair_forces_only(P(orc, a=0.0, gamma=2.0, kBT=0.0, wexp=s, exclude_bonded=0), x, vr, 9)
        out[r] = (fr[0, 1], fd[0, 1])
    np.testing.assert_allclose(out[r1][0] / out[r2][0], (w1 / w2) ** (s / 2), rtol=1e-12)
    np.testing.assert_allclose(out[r1][1] / out[r2][1], (w1 / w2) ** s, rtol=1e-12)
    # the dissipative force opposes the separation: it pulls i after j (+y)
    assert out[r1][1] > 0 and out[r2][1] > 0


def test_equilibrium_temperature_changed_weight_exponent(orc):
    """s = 0.5: w_D = w_R^2 keeps the fluctuation-dissipation balance, so the
    thermostat still holds T = kBT (zeta = f_p = 0).  Were the random weight
    w^s instead of w^(s/2), T would settle near 0.63 kBT."""
    L = 32.0
    x, v = synth.dimers(512, L, 0.5, seed=0)
    p = P(orc, L=L, zeta=0.0, fp=0.0, seed=12, dt=0.005, wexp=0.5)
    st = orc.State(p, x, v, cells=True)
    st.run(5000)
    log = st.run(40000, thermo=True)
    n = x.shape[0]
    T = 2 * log[:, 0] / (2 * n - 2)
    assert abs(T.mean() - 1.0) < 0.02, T.mean()


def test_cell_list_variant_matches_all_pairs(orc):
    L = 9.0
    x, _ = synth.dimers(150, L, 0.5, seed=2)
    v = synth.velocities(300, 1.0, seed=2)
    p = P(orc, L=L)
    f1, n1 = orc.forces(p, x.astype(np.float64), v.astype(np.float64), 4)
    f2, n2 = orc.forces(p, x.astype(np.float64), v.astype(np.float64), 4, cells=True)
    assert n1 == n2
    np.testing.assert_allclose(f2, f1, atol=1e-11)


def test_cell_rule_stencil_is_sufficient(orc):
    """With n_c = floor(L / r_c) cells per side and bead x in cell
    floor(x n_c / L) (exact on the fixed-point grid), every interacting pair
    sits in the same or an adjacent cell (periodically), so a 3 x 3 stencil
    finds all pairs; the counts cover every bead once."""
    for L, seed in [(3.0, 0), (7.0, 1), (32.0, 2), (1024.0, 3), (100.0, 4)]:
        rc = 0.5 if L == 100.0 else 1.0
        nc = int(math.floor(L / rc))
        rng = np.random.default_rng(seed)
        n = 400
        x = rng.random((n, 2)) * L
        # pairs straddling cell edges at just under r_c
        k = min(nc, 50)
        edges = np.arange(k) * (L / nc)
        x[:k, 0] = edges + 1e-9 * L
        x[k:2 * k, 0] = x[:k, 0] + rc * (1 - 1e-7)
        x[k:2 * k, 1] = x[:k, 1]
        x = synth.on_grid(x, L)
        cnt = orc.cell_counts(x, L, nc)
        assert cnt.sum() == n
        X = np.rint(x / L * 2.0 ** 32).astype(np.int64)
        cx = (X[:, 0] * nc) >> 32
        cy = (X[:, 1] * nc) >> 32
        assert np.all(cx * (L / nc) <= x[:, 0] + 1e-12) and np.all(x[:, 0] < (cx + 1) * (L / nc) + 1e-12)
        np.testing.assert_array_equal(cnt, np.histogram2d(cy, cx, bins=nc, range=[[0, nc], [0, nc]])[0])
        d = x[:, None, :] - x[None, :, :]
        d -= L * np.rint(d / L)
        r2 = (d ** 2).sum(-1)
        ii, jj = np.nonzero(np.triu(r2 < rc * rc, 1))
        ddx = np.abs(cx[ii] - cx[jj]); ddx = np.minimum(ddx, nc - ddx)
        ddy = np.abs(cy[ii] - cy[jj]); ddy = np.minimum(ddy, nc - ddy)
        assert ddx.max(initial=0) <= 1 and ddy.max(initial=0) <= 1


# --------------------------------------------------------------------------
# Neighbour counts (reference for the bit-exact count tests) and the thermo
# reductions, pinned on hand-built configurations
# --------------------------------------------------------------------------

def test_pair_counts_hand_built(orc):
    """Beads placed by hand in a box of side 10 (r_c = 1): pairs at r well
    inside r_c, just inside, just outside, inside the tie band around r_c,
    exactly at r = 0, across the periodic boundary, and a bonded pair with the
    exclusion switched on and off.  Expected counts are written down from the
    geometry (Sec. 2.1: the pair force acts for r < r_c only; Sec. 2.2: bonded
    beads have no other interaction)."""
    L = 10.0
    x = np.array([
        [1.0, 1.0],    # 0: bonded to 1 at r = 0.5
        [1.5, 1.0],    # 1
        [1.0, 1.9],    # 2: r(0,2) = 0.9, r(1,2) = sqrt(0.25 + 0.81) > 1
        [5.0, 5.0],    # 3: r(3,4) = 1 - 1e-3 (inside, outside the tie band)
        [5.0, 5.999],  # 4
        [7.0, 7.0],    # 5: r(5,6) = 1 + 1e-3 (outside)
        [8.001, 7.0],  # 6
        [3.0, 8.0],    # 7: r(7,8) = 1 - 1e-7: inside the tie band -> ambiguous
        [3.0, 8.9999999],  # 8
        [0.2, 5.0],    # 9: across x = 0: r(9,10) = 0.2 + 0.3 = 0.5
        [9.7, 5.0],    # 10
        [6.0, 2.0],    # 11: coincident with 12: r = 0 counts as no pair
        [6.0, 2.0],    # 12
        [8.5, 9.8],    # 13: across the corner: r(13,14) = sqrt(0.3^2+0.4^2) = 0.5
        [8.8, 0.2],    # 14
        [5.0, 5.9995],  # 15: near 3 and 4: r(3,15) = 0.9995 inside, r(4,15) = 5e-4 inside
    ])
    p = P(orc, L=L)
    cnt, amb, tot = orc.pair_counts(p, x, tie=1e-6)
    # pairs inside r_c: (0,2), (3,4), (9,10), (13,14), (3,15), (4,15); (0,1) excluded (bonded)
    exp_cnt = np.zeros(16, np.uint32)
    for i, j in [(0, 2), (3, 4), (9, 10), (13, 14), (3, 15), (4, 15)]:
        exp_cnt[i] += 1
        exp_cnt[j] += 1
    exp_amb = np.zeros(16, np.uint32)
    exp_amb[7] = exp_amb[8] = 1
    np.testing.assert_array_equal(cnt, exp_cnt)
    np.testing.assert_array_equal(amb, exp_amb)
    assert tot == 6
    # exclusion off: the bonded pair (0, 1) at r = 0.5 counts as well
    cnt2, amb2, tot2 = orc.pair_counts(P(orc, L=L, exclude_bonded=0), x, tie=1e-6)
    exp2 = exp_cnt.copy()
    exp2[0] += 1
    exp2[1] += 1
    np.testing.assert_array_equal(cnt2, exp2)
    np.testing.assert_array_equal(amb2, exp_amb)
    assert tot2 == 7
    # a tie band of 3e-3 r_c^2 swallows the pairs at r = 1 - 1e-3, 1 + 1e-3
    # and 1 - 5e-4 (|r^2 - 1| = 2e-3, 2e-3, 1e-3) besides the one at 1 - 1e-7
    cnt3, amb3, tot3 = orc.pair_counts(p, x, tie=3e-3)
    assert tot3 == 4
    np.testing.assert_array_equal(amb3[[3, 4, 5, 6, 7, 8, 15]], [2, 1, 1, 1, 1, 1, 1])
    assert cnt3[3] == 0 and cnt3[4] == 1 and cnt3[15] == 1   # only (4, 15) at 5e-4 remains


def test_pair_counts_brute_force_in_numpy(orc):
    """Random dimers: the oracle's counts equal an independent numpy count of
    the minimum-image pairs with r < r_c, bonded pairs excluded, ties removed."""
    L = 6.0
    x, _ = synth.dimers(60, L, 0.5, seed=11)
    x = x.astype(np.float64)
    cnt, amb, tot = orc.pair_counts(P(orc, L=L), x, tie=4e-6)
    d = x[:, None, :] - x[None, :, :]
    d -= L * np.rint(d / L)
    r2 = (d ** 2).sum(-1)
    n = x.shape[0]
    idx = np.arange(n)
    bonded = (idx[:, None] ^ 1) == idx[None, :]
    off = ~np.eye(n, dtype=bool) & ~bonded
    tie = off & (np.abs(r2 - 1.0) < 4e-6)
    inside = off & ~tie & (r2 < 1.0) & (r2 > 0.0)
    np.testing.assert_array_equal(cnt, inside.sum(1).astype(np.uint32))
    np.testing.assert_array_equal(amb, tie.sum(1).astype(np.uint32))
    assert tot == int(np.triu(inside, 1).sum())


def test_thermo_two_beads_by_hand(orc):
    """KE = 1/2 m sum |v|^2, P = m sum v and T = sum m |v|^2 / (2N - 2) for
    two beads with v = (3, 4) and (-1, 2), m = 2: KE = 2 (25 + 5) / 2 = 30,
    P = 2 (2, 6) = (4, 12), T = 2 * 30 / 2 = 30."""
    ke, p, T = orc.thermo(np.zeros((2, 2)), np.array([[3.0, 4.0], [-1.0, 2.0]]), mass=2.0)
    assert ke == 30.0
    np.testing.assert_array_equal(p, [4.0, 12.0])
    assert T == 30.0
    # four beads at rest but one: T divides by 2N - 2 = 6
    ke, p, T = orc.thermo(np.zeros((4, 2)), np.array([[0.0, 0.0], [0.0, 0.0], [0.0, 0.0], [1.0, 1.0]]))
    assert ke == 1.0 and T == 2.0 / 6.0
    np.testing.assert_array_equal(p, [1.0, 1.0])


def test_pair_counts_exactly_at_cutoff(orc):
    """With no tie band a pair at exactly r = r_c has w = 0 and is not a
    neighbour (r < r_c strictly); one a binary ulp closer is."""
    L = 8.0
    x = np.array([[2.0, 2.0], [2.0, 4.5], [3.0, 2.0], [6.0, 6.0], [6.0, 7.0 - 2.0 ** -40], [1.0, 6.0]])
    cnt, amb, tot = orc.pair_counts(P(orc, L=L, exclude_bonded=0), x, tie=0.0)
    assert tot == 1 and amb.sum() == 0
    np.testing.assert_array_equal(cnt, [0, 0, 0, 1, 1, 0])
