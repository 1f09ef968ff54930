"""Long-run statistics of the GPU path against the FP64 oracle (same seed,
same initial state; the trajectories decorrelate, the statistics must not).

Bounds: time-averaged temperature within 1%; time-averaged E(k) within 5% per
shell for k = 2..M/2 (k = 1 has too few modes), averaged over six seeds on
each side.  Measured with this protocol over six seeds, one run's E(k)
scatters by 2-3% (k = 2, 3) down to 0.5% (k >= 9) about the seed mean, so
the difference of two six-seed means has a spread of about 1.4% at k = 2, 3
and well under 1% beyond: the 5% bound is three and a half of those at the
noisiest shell (with three seeds per side it was two and a half, and one run
in several missed by 0.1% at k = 2).  A missing or mis-scaled force term
moves these statistics by far more.
"""
import numpy as np
import pytest

from oracle import observables as ob
from paper_1310_0998_gb300 import synth

pytestmark = pytest.mark.gpu

L, ND, M = 32.0, 512, 32
BASE = dict(a=25.0, gamma=4.5, kBT=1.0, rc=1.0, kbond=100.0, r0=0.5, dt=0.01)


def _oracle(orc, seed, steps, every, burn, zeta, fp, box=(L, ND, M)):
    Lb, nd, m = box
    x, v = synth.dimers(nd, Lb, 0.5, seed=seed)
    p = orc.params(L=Lb, fp=fp, zeta=zeta, seed=seed, **BASE)
    st = orc.State(p, x, v, cells=True)
    st.run(burn)
    eps = ob.filter_width(Lb, nd, 10.0)
    E, T = np.zeros(m // 2), []
    n = 0
    for _ in range((steps - burn) // every):
        log = st.run(every, thermo=True)
        T.append(2 * log[:, 0] / (2 * 2 * nd - 2))
        c, vc = ob.agent_com(st.x, st.v, Lb)
        E += ob.energy_spectrum(ob.velocity_field(c, vc, Lb, m, eps)[0])
        n += 1
    return E / n, float(np.mean(np.concatenate(T)))


def _gpu(seed, steps, every, burn, zeta, fp, box=(L, ND, M)):
    from paper_1310_0998_gb300 import Sim
    Lb, nd, m = box
    x, v = synth.dimers(nd, Lb, 0.5, seed=seed)
    kw = dict(a=BASE["a"], gamma=BASE["gamma"], kBT=BASE["kBT"], rc=BASE["rc"], k_bond=BASE["kbond"],
              r0=BASE["r0"], dt=BASE["dt"], f_p=fp, zeta=zeta, seed=seed)
    E, T = np.zeros(m // 2), []
    n = 0
    with Sim(Lb, 2 * nd, **kw) as s:
        s.set_positions(x, v)
        s.step(burn)
        for _ in range((steps - burn) // every):
            s.step(every)
            T.append(s.thermo_log(s.info().step - every + 1, every)[:, 3])
            E += s.energy_spectrum(m)
            n += 1
    return E / n, float(np.mean(np.concatenate(T)))


ACT_SEEDS = (1, 2, 3, 4, 5, 6)


def _oracle_active(seed):
    """Oracle statistics of the active C1 run (runs in a spawned worker)."""
    import oracle as orc
    return _oracle(orc, seed, 60000, 100, 2000, 0.1, 1.0)


def _threads(n):
    import os
    os.environ["OMP_NUM_THREADS"] = str(n)


def _spawn_map(fn, seeds):
    """Map over seeds in spawned workers that share the host cores (the
    oracle's OpenMP team per worker sized to its share)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    per = max(1, (os.cpu_count() or 1) // len(seeds))
    with cf.ProcessPoolExecutor(max_workers=len(seeds), mp_context=mp.get_context("spawn"), initializer=_threads,
                                initargs=(per,)) as ex:
        return list(ex.map(fn, seeds))


def test_active_run_statistics(orc):
    """C1 (f_p = 1, zeta = 0.1): <T> and <E(k)> over steps 2e3..6e4, six
    seeds on both sides (the oracle's in spawned workers).  With one run
    scattering by 2-3% at k = 2, 3, the difference of two six-seed means has
    a spread of about 1.4% there and less beyond, so the 5% bound is three
    and a half of those at the noisiest shell."""
    o = _spawn_map(_oracle_active, ACT_SEEDS)
    g = [_gpu(s, 60000, 100, 2000, 0.1, 1.0) for s in ACT_SEEDS]
    Eo, To = np.mean([e for e, _ in o], axis=0), float(np.mean([t for _, t in o]))
    Eg, Tg = np.mean([e for e, _ in g], axis=0), float(np.mean([t for _, t in g]))
    assert abs(Tg - To) <= 0.01 * To, (Tg, To)
    rel = np.abs(Eg - Eo) / Eo
    assert rel[1:].max() <= 0.05, rel


# The energy spectrum on the 128^2 grid of the parameter sweep's protocol, on
# a box the oracle runs in minutes: L = 64 at area fraction 0.4 (3,277
# agents), f_p = 1, zeta = 0.1, E(k) every 200 steps over steps 2e3..2e4.
BOX128 = (64.0, 3277, 128)
SEEDS128 = tuple(range(1, 13))


def _oracle_box128(seed):
    import oracle as orc
    return _oracle(orc, seed, 20000, 200, 2000, 0.1, 1.0, box=BOX128)


def test_active_run_spectrum_m128(orc):
    """<E(k)> on 128^2 and <T>, twelve seeds on each side.  Measured on the
    GPU over 24 seeds with this protocol, one run's E(k) scatters by 6% at
    k = 2, 3.4% at k = 3, 2-3% up to k = 10 and 0.7-1.6% beyond, so the
    difference of two twelve-seed means has a spread of 1.4% at k = 3 and
    under 1.2% from k = 4 on: the 5% bound on k = 3..64 is 3.6 of those at the
    noisiest shell (k = 1, 2 hold 4 and 12 modes and are left out).  One
    run's <T> scatters by 0.16%."""
    o = _spawn_map(_oracle_box128, SEEDS128)
    g = [_gpu(s, 20000, 200, 2000, 0.1, 1.0, box=BOX128) for s in SEEDS128]
    Eo, To = np.mean([e for e, _ in o], axis=0), float(np.mean([t for _, t in o]))
    Eg, Tg = np.mean([e for e, _ in g], axis=0), float(np.mean([t for _, t in g]))
    assert abs(Tg - To) <= 0.01 * To, (Tg, To)
    rel = np.abs(Eg - Eo) / Eo
    assert rel[2:].max() <= 0.05, rel


EQ_SEEDS, EQ_BURN, EQ_STEPS = (1, 2, 3, 4, 5, 6), 5000, 45000


def _oracle_T(seed):
    """Oracle <T> over steps EQ_BURN..EQ_STEPS at zeta = f_p = 0 (runs in a
    spawned worker)."""
    import oracle as orc
    x, v = synth.dimers(ND, L, 0.5, seed=seed)
    p = orc.params(L=L, fp=0.0, zeta=0.0, seed=seed, **BASE)
    st = orc.State(p, x, v, cells=True)
    st.run(EQ_BURN)
    log = st.run(EQ_STEPS - EQ_BURN, thermo=True)
    return float(np.mean(2 * log[:, 0] / (2 * 2 * ND - 2)))


def test_equilibrium_temperature(orc):
    """zeta = f_p = 0: the GPU thermostat holds the oracle's <T> (= kBT up to
    the time-step bias) within 1%.  At this state the temperature relaxes
    from the random start over ~5e3 steps and then wanders slowly (1e3-step
    block means scatter by ~3% and stay correlated over many blocks), so one
    run's <T> over steps 2e3..2e4 scatters by 1.6% between seeds.  With the
    start-up discarded (5e3 steps) and a 4e4-step window, 24 oracle seeds gave
    <T> = 1.0048 with a per-run scatter of 0.56%: the difference of two
    six-seed means then has a spread of 0.32%, and the 1% bound is three of
    those."""
    To = float(np.mean(_spawn_map(_oracle_T, EQ_SEEDS)))
    from paper_1310_0998_gb300 import Sim
    Tg = []
    for seed in EQ_SEEDS:
        x, v = synth.dimers(ND, L, 0.5, seed=seed)
        with Sim(L, 2 * ND, a=BASE["a"], gamma=BASE["gamma"], kBT=BASE["kBT"], rc=BASE["rc"],
                 k_bond=BASE["kbond"], r0=BASE["r0"], dt=BASE["dt"], f_p=0.0, zeta=0.0, seed=seed) as s:
            s.set_positions(x, v)
            s.step(EQ_BURN)
            s.step(EQ_STEPS - EQ_BURN)
            Tg.append(float(np.mean(s.thermo_log(EQ_BURN + 1, EQ_STEPS - EQ_BURN)[:, 3])))
    Tg = float(np.mean(Tg))
    assert abs(Tg - To) <= 0.01 * To, (Tg, To)
    assert abs(Tg - 1.0) <= 0.02
