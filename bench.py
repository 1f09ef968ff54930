"""Benchmark: particle-steps/s of the DPD dimer hot path on one GB300.

Workload (default, "c3"): periodic box L = 1024 (r_c = 1), bead density 3 ->
3,145,728 beads (1,572,864 dimers) at random centres/orientations (seed 0),
a = 25, gamma = 4.5, kBT = 1, kappa = 100, r0 = 0.5, f_p = 1, zeta = 0.1,
dt = 0.01.  One step = one velocity-Verlet step of the whole system (cell
scan, scatter, fused pair/bond/propulsion/drag force + integration + FP64
thermo reduction).

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the simulator's stream, with a 512 MiB write + read L2 flush between
timed steps (outside the events).  value = beads * K / sum(step times).
Under torchrun each rank runs an independent replica (no collective on the
data path; "replicas only"), value = all ranks' bead-steps / max time.

--impl reference times the FP64 CPU oracle (cell-list variant, OpenMP) on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PHYS = dict(a=25.0, gamma=4.5, kBT=1.0, rc=1.0, kbond=100.0, r0=0.5, fp=1.0, zeta=0.1, dt=0.01, mass=1.0)


def max_over_ranks(t_local: float, world: int, device="cpu") -> float:
    """The slowest rank's timed-region duration (every rank runs the same
    amount of work); a no-op on one rank."""
    if world <= 1:
        return float(t_local)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: int, steps: int, t_max: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest time
    (replicas only: each rank advances its own box of units_per_rank beads)."""
    return world * units_per_rank * steps / t_max
CONFIGS = {
    "c3": dict(L=1024.0, n_beads=3 * 1024 * 1024, name="c3: L=1024, density 3, 3,145,728 beads"),
    "c2": dict(L=256.0, n_beads=3 * 256 * 256, name="c2-size: L=256, density 3, 196,608 beads"),
    "c3q": dict(L=512.0, n_beads=3 * 512 * 512, name="c3-quarter: L=512, density 3, 786,432 beads"),
    "c1": dict(L=32.0, n_beads=1024, name="c1: L=32, 512 dimers"),
}
# algorithmic ALU operations of one step, counted on the benchmarked state:
# OPS_TEST per half-stencil distance test (candidate pair), OPS_PAIR per
# interacting pair (Philox4x32-10 ~80 + pair force ~30), OPS_BEAD per bead
# (bond, propulsion, drag, two half kicks, drift, binning)
OPS_TEST, OPS_PAIR, OPS_BEAD = 8.0, 110.0, 70.0
BYTES_PER_BEAD_STEP = 36.0     # algorithmic HBM bytes per bead-step (read 20, write 16)
LANES = 128                    # FP32/INT32 lanes per SM
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "force_traffic_c3.md")
ISSUE_PROFILE = os.path.join(ROOT, "profiles", "force_issue_c3q.md")
SCHEDULERS = 4                 # warp schedulers per SM
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1310_0998_gb300", "csrc", f)
                  for f in ("sim_kernels.cuh", "dpd_device.cuh", "sim.cu")]


def sm_count() -> int:
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def profile_record(path: str, key: str, tile: int, variant: int):
    """A value from a committed ncu summary (its `- key: value` lines), if it
    was taken on this exact kernel source and shape; else None."""
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if line.startswith("- ") and ": " in line:
            k, v = line[2:].split(": ", 1)
            kv[k.strip()] = v.strip().strip("`")
    try:
        if kv.get("source_sha256_16") != kernel_source_hash():
            return None
        if int(kv["tile"]) != tile or int(kv["variant"]) != variant:
            return None
        return float(kv[key])
    except (KeyError, ValueError):
        return None


def measured_traffic(tile: int, variant: int):
    """DRAM bytes per force-kernel launch at C3 (ncu, body step)."""
    return profile_record(TRAFFIC_PROFILE, "dram_bytes_per_launch", tile, variant)


def measured_warp_inst_per_bead(tile: int, variant: int):
    """Warp instructions the force kernel executes per bead (ncu, body step of
    a density-3 box; the count per bead does not depend on the box size)."""
    return profile_record(ISSUE_PROFILE, "warp_inst_per_bead", tile, variant)


def algorithmic_ops(counts: np.ndarray, pairs: int, n_beads: int):
    """Candidates of the forward half stencil (own cell after the bead, E, NE,
    N, NW) from the cell populations, the interacting pairs, and the step's
    algorithmic operation count."""
    n = counts.astype(np.float64)
    fwd = np.roll(n, -1, 1) + np.roll(np.roll(n, -1, 1), -1, 0) + np.roll(n, -1, 0) + np.roll(np.roll(n, 1, 1), -1, 0)
    cand = float((n * (n - 1.0) / 2.0).sum() + (n * fwd).sum())
    return cand, OPS_TEST * cand + OPS_PAIR * pairs + OPS_BEAD * n_beads


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
        return dict(hbm=float(p["hbm_gbs"]), sm_max_mhz=float(p.get("sm_max_mhz", 2070.0)), src="measured")
    return dict(hbm=6800.0, sm_max_mhz=2070.0, src="fallback")


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if bus_id:
            cmd.insert(1, f"--id={bus_id}")
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 8:
                continue
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except ValueError:
                continue
            for nm, val in zip(names, r[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(np.max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_rate(L, n_beads, budget_s=12.0, seed=0):
    """Time the FP64 cell-list oracle (OpenMP) on the host; returns
    (bead-steps/s, threads, description of the sample)."""
    import oracle
    from paper_1310_0998_gb300 import synth
    oracle.build()
    x, v = synth.dimers(n_beads // 2, L, PHYS["r0"], seed=seed)
    p = oracle.params(L=L, seed=seed, **PHYS)
    st = oracle.State(p, x, v, cells=True)
    t0 = time.perf_counter()
    st.run(1)
    t1 = time.perf_counter()
    per = max(t1 - t0, 1e-6)
    more = max(1, int(budget_s / per) - 1)
    st.run(more)
    t2 = time.perf_counter()
    steps = 1 + more
    rate = n_beads * steps / (t2 - t0)
    return rate, oracle.num_threads(), f"{steps} steps of the FP64 cell-list oracle on a {n_beads}-bead box (L={L:g}, density 3), {t2 - t0:.1f} s"


def ensemble_leg(R, steps, warmup, seed=0, variant=0, tile=0, seq_steps=500):
    """C4: R replicas drawn from the uneven distribution (box side U(32, 192),
    area fraction U(0.05, 0.6), gamma log-U(0.5, 50), zeta log-U(0.005, 2),
    f_p U(0.5, 2)).  The kernel shape is tuned for this replica mix (unless
    given), then `steps` steps of the batched persistent kernel are timed, and
    `seq_steps` steps of every replica run alone through the single-system
    path (scaled to `steps`: the per-step cost of a replica is steady)."""
    import torch
    from paper_1310_0998_gb300 import Ensemble, synth, tune
    pts = []
    for r, e in enumerate(synth.ensemble_points(R, seed)):
        pts.append(dict(a=PHYS["a"], kBT=PHYS["kBT"], rc=PHYS["rc"], k_bond=PHYS["kbond"], r0=PHYS["r0"],
                        dt=PHYS["dt"], L=e["L"], n_beads=2 * e["n_dimers"], gamma=e["gamma"], zeta=e["zeta"],
                        f_p=e["fp"], seed=seed + r, replica=r, variant=variant, tile=tile))
    beads = sum(p["n_beads"] for p in pts)
    tuning = None
    if variant == 0 and tile == 0:
        tuning = tune.batch_autotune(pts, steps=5)
    ens = Ensemble(pts)
    ens.init_random(seed)
    ens.step(warmup)
    ens.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ens.step(steps)
    ens.sync()
    t_batch = time.perf_counter() - t0
    views = [ens.replica(r) for r in range(R)]
    for v in views:
        v.step(1)
    for v in views:
        v.sync()
    t0 = time.perf_counter()
    for v in views:
        v.step(seq_steps)
    for v in views:
        v.sync()
    t_seq = (time.perf_counter() - t0) * steps / seq_steps
    phases = ens.profile(32)
    info = ens.info()
    shape = views[0].info()
    ens.close()
    out = {"replicas": R, "beads": beads, "steps": steps, "batched_s": t_batch,
           "batched_ms_per_step": 1e3 * t_batch / steps, "sequential_ms_per_step": 1e3 * t_seq / steps,
           "sequential_steps_timed": seq_steps, "speedup": t_seq / t_batch,
           "batched_particle_steps_per_s": beads * steps / t_batch, "grid": info["grid"],
           "work_tiles": info["work_tiles"], "tile": shape.tile, "variant": shape.variant,
           "phases_ms_per_step": phases,
           "timing": "wall clock around each synchronised leg; batched: the full step count in one persistent "
                     "launch per call; sequential: each replica alone, one after another, for "
                     f"{seq_steps} steps, scaled to {steps}"}
    if tuning is not None:
        out["tuning"] = tuning
    return out


def sweep_leg(steps=20000, snaps=5, every=2000, M=128, seq_steps=2000, seed=0, sur=None):
    """C2: the parameter sweep of the 256 x 256 box (area fraction 0.1-0.6 x
    gamma {1, 4.5, 20} x zeta {0.01, 0.1, 1}, 54 points, f_p = 1), each point
    `steps` steps from the paper's initial condition with the FP64 E(k) on
    M^2 averaged over `snaps` snapshots `every` steps apart at the end of the
    run.  Batched: all points in the persistent ensemble kernel (shape tuned
    for the mix).  Plain: every point alone through the single-system path,
    one after another (context creation, initial state, `seq_steps` steps
    scaled to `steps`, and all its snapshots, timed).  With a trained
    surrogate, the time it takes to answer the same 54 points (fallback rule
    included) is reported beside them."""
    import torch
    from paper_1310_0998_gb300 import Ensemble, Sim, synth, tune
    pts = []
    for r, e in enumerate(synth.sweep_points()):
        pts.append(dict(a=PHYS["a"], kBT=PHYS["kBT"], rc=PHYS["rc"], k_bond=PHYS["kbond"], r0=PHYS["r0"],
                        dt=PHYS["dt"], L=e["L"], n_beads=2 * e["n_dimers"], gamma=e["gamma"], zeta=e["zeta"],
                        f_p=e["fp"], seed=seed + r, replica=r))
    R = len(pts)
    beads = sum(p["n_beads"] for p in pts)
    every = max(1, min(every, steps // snaps))
    burn = max(0, steps - snaps * every)
    seq_steps = max(1, min(seq_steps, steps))
    tuning = tune.batch_autotune(pts, steps=5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ens = Ensemble(pts)
    ens.init_random(seed)
    ens.sync()
    t_setup = time.perf_counter() - t0
    E = np.zeros((R, M // 2))
    t0 = time.perf_counter()
    for k in range(snaps + 1):
        n = burn if k == 0 else every
        while n > 0:
            c = min(n, 10000)
            ens.step(c)
            ens.sync()
            n -= c
        if k > 0:
            for r in range(R):
                E[r] += ens.replica(r).energy_spectrum(M) / snaps
    t_run = time.perf_counter() - t0
    shape = ens.replica(0).info()
    ens.close()
    t_seq = 0.0
    for r, p in enumerate(pts):
        kw = dict(p)
        L, n = kw.pop("L"), kw.pop("n_beads")
        t0 = time.perf_counter()
        s = Sim(L, n, **kw)
        s.init_random(seed)
        s.sync()
        t1 = time.perf_counter()
        s.step(seq_steps)
        s.sync()
        t2 = time.perf_counter()
        for _ in range(snaps):
            s.energy_spectrum(M)
        t3 = time.perf_counter()
        s.close()
        t_seq += (t1 - t0) + (t2 - t1) * steps / seq_steps + (t3 - t2)
    out = {"points": R, "beads": beads, "steps": steps, "snapshots": snaps, "every": every, "M": M,
           "batched_setup_s": t_setup, "batched_run_s": t_run, "batched_s": t_setup + t_run,
           "batched_particle_steps_per_s": beads * steps / t_run,
           "plain_s": t_seq, "plain_steps_timed_per_point": seq_steps,
           "speedup": t_seq / (t_setup + t_run), "tile": shape.tile, "variant": shape.variant,
           "spectra_finite": bool(np.all(np.isfinite(E)) and np.all(E > 0)), "tuning": tuning,
           "timing": "wall clock; batched: set-up, then all steps in persistent launches of up to 1e4 steps and "
                     "the E(k) of every point at each snapshot; plain: per point set-up, seq_steps steps scaled "
                     "to the full count, and every snapshot's E(k)"}
    if sur is not None:
        Xq = np.array([[synth.sweep_points()[r]["phi"], p["gamma"], p["zeta"], p["f_p"]]
                       for r, p in enumerate(pts)], np.float32)
        model, thr, proto = sur
        t0 = time.perf_counter()
        _, fb = model.query(Xq, thr, dict(proto, seed=seed))
        t_q = time.perf_counter() - t0
        out.update({"surrogate_s": t_q, "surrogate_fallback_points": int(fb.sum()),
                    "surrogate_speedup_vs_plain": t_seq / t_q,
                    "surrogate_note": "the surrogate answers its own sampling protocol's statistics (L = 48 box) "
                                      "at the sweep's parameters; its accuracy is the surrogate leg's"})
    return out


def observables_leg(sim, nb, reps=5):
    """Observables on the device (Secs. 5.3-5.4): E(k) at M = 128 on the main
    box's state (agent centres of mass, windowed velocity field, the library's
    own FFT, shell sums); the velocity correlation g(r) for r < 16 (64 bins of
    0.25) on the same state (cell-grid pass over the agent pairs within
    r_max); and g(r) over all agent pairs (512 bins up to L/2) of a
    196,608-bead box of side 256 (98,304 agents)."""
    from paper_1310_0998_gb300 import Sim, synth
    sim.energy_spectrum(128)
    t0 = time.perf_counter()
    for _ in range(reps):
        sim.energy_spectrum(128)
    t_spec = (time.perf_counter() - t0) / reps
    sim.velocity_correlation(0.25, 64)
    t0 = time.perf_counter()
    for _ in range(reps):
        _, _, _, cnt_c = sim.velocity_correlation(0.25, 64)
    t_vcf_c = (time.perf_counter() - t0) / reps
    Lv, nbv = 256.0, 196608
    x, _ = synth.dimers(nbv // 2, Lv, PHYS["r0"], seed=1)
    vel = synth.velocities(nbv, 1.0, seed=2)
    with Sim(Lv, nbv, a=PHYS["a"], gamma=PHYS["gamma"], kBT=PHYS["kBT"], rc=PHYS["rc"], k_bond=PHYS["kbond"],
             r0=PHYS["r0"], f_p=PHYS["fp"], zeta=PHYS["zeta"], dt=PHYS["dt"]) as s:
        s.set_positions(x, vel)
        s.velocity_correlation(0.25, 512)
        t0 = time.perf_counter()
        s.velocity_correlation(0.25, 512)
        t_vcf = time.perf_counter() - t0
    na = nbv // 2
    return {"spectrum_M": 128, "spectrum_agents": nb // 2, "spectrum_ms": 1e3 * t_spec,
            "spectrum_state_gbs": 16.0 * nb / t_spec / 1e9,
            "vcf_rmax16_agents": nb // 2, "vcf_rmax16_bins": 64, "vcf_rmax16_ms": 1e3 * t_vcf_c,
            "vcf_rmax16_pairs": int(np.sum(cnt_c)), "vcf_rmax16_pairs_per_s": float(np.sum(cnt_c)) / t_vcf_c,
            "vcf_allpairs_agents": na, "vcf_allpairs_bins": 512, "vcf_allpairs_ms": 1e3 * t_vcf,
            "vcf_allpairs_agent_pairs_per_s": na * (na - 1) / 2 / t_vcf,
            "timing": "wall clock per synchronising call (device work and the copy of the result to the host)"}


OPS_PER_BEAD_STEP_3D = 1200.0   # 40.5 half-stencil tests x 10 + 6.3 pairs x 115 + 70 integration


def three_d_leg(steps=20, warmup=3, L=64.0, seed=0):
    """Three-dimensional variant: density-3 cube of side L (3 L^3 beads), the
    C3 parameters; wall clock around `steps` synchronised steps."""
    from paper_1310_0998_gb300 import Sim3, synth
    nb = int(3 * L ** 3) // 2 * 2
    x, v = synth.dimers3(nb // 2, L, PHYS["r0"], seed=seed)
    with Sim3(L, nb, seed=seed, a=PHYS["a"], gamma=PHYS["gamma"], kBT=PHYS["kBT"], rc=PHYS["rc"],
              k_bond=PHYS["kbond"], r0=PHYS["r0"], f_p=PHYS["fp"], zeta=PHYS["zeta"], dt=PHYS["dt"]) as s:
        s.set_positions(x, v)
        s.step(warmup)
        s.sync()
        t0 = time.perf_counter()
        s.step(steps)
        s.sync()
        dt = time.perf_counter() - t0
        s.energy_spectrum(64)
        t0 = time.perf_counter()
        for _ in range(3):
            s.energy_spectrum(64)
        spec_ms = (time.perf_counter() - t0) / 3 * 1e3
        s.velocity_correlation(0.25, 16)
        t0 = time.perf_counter()
        _, _, _, vcnt = s.velocity_correlation(0.25, 16)
        vcf_ms = (time.perf_counter() - t0) * 1e3
    rate = nb * steps / dt
    pk = peaks()
    alu_peak = sm_count() * LANES * pk["sm_max_mhz"] * 1e6
    return {"beads": nb, "L": L, "steps": steps, "particle_steps_per_s": rate, "ms_per_step": 1e3 * dt / steps,
            "roofline": {"bound": "alu", "achieved": OPS_PER_BEAD_STEP_3D * rate / 1e12, "peak": alu_peak / 1e12,
                         "unit": "Tops/s", "frac": OPS_PER_BEAD_STEP_3D * rate / alu_peak},
            "spectrum_M": 64, "spectrum_ms": spec_ms, "vcf_r4_ms": vcf_ms, "vcf_r4_pairs": int(vcnt.sum()),
            "timing": "wall clock around synchronised steps (scan, scatter, pair forces, integration per step); "
                      "spectrum: per synchronising call (COM, windowed field on 64^3, FFT, shells); velocity "
                      "correlation r < 4 (16 shells): per call (cell grid)"}


def surrogate_leg(n_train=2000, n_test=200, n_noise=50, seed=0, keep=False):
    """C5: the learned surrogate of the simulator's statistics.  Parameter
    points (area fraction, gamma, zeta, f_p) from the C4 ranges; the training
    statistics come from batched-ensemble runs (chunks of 256 replicas), the
    held-out ones from plain simulations one after another (L = 48, 1500
    steps burn-in, 6 snapshots 250 steps apart, E(k) on 128^2, g(r) to
    L/2 in shells of 0.25).  A 4-member ensemble is trained on tcgen05; then
    the held-out errors (per point: E(k) over the 32 shell-pair bins as
    |E_pred / E_sim - 1|, xi and L_gv as relative errors), the same errors of
    two model-free predictors (training mean, nearest training point), the
    run-to-run noise floor of the statistics (a second plain run of the first
    n_noise held-out points with other seeds), the fallback rate, the query
    speedup, and the device throughput of the tensor-core forward pass.
    keep: also return the trained model, its fallback threshold and protocol
    (the caller closes the model)."""
    import numpy as np
    from paper_1310_0998_gb300 import surrogate as S, synth
    proto = dict(L=48.0, burn=1500, n_snap=6, every=250)
    X = synth.surrogate_points(n_train + n_test, seed=seed + 17).astype(np.float32)
    Xtr, Xte = X[:n_train], X[n_train:]
    t0 = time.perf_counter()
    Ytr = S.simulate(Xtr, batched=True, seed=seed, **proto)
    t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    Yte = S.simulate(Xte, batched=False, seed=seed + 100000, **proto)
    t_plain = time.perf_counter() - t0
    Yno = S.simulate(Xte[:n_noise], batched=False, seed=seed + 200000, **proto)
    ok_tr = np.all(np.isfinite(Ytr), axis=1)
    ok_te = np.all(np.isfinite(Yte), axis=1)
    sur = S.Surrogate(members=4, max_rows=4096, seed=seed)
    trained = False
    try:
        t0 = time.perf_counter()
        loss = sur.fit(Xtr[ok_tr], Ytr[ok_tr], epochs=300, batch=64, lr=2e-3)
        t_fit = time.perf_counter() - t0
        P, Sd = sur.predict(Xte)
        Pt, St = sur.predict(Xtr[ok_tr])
        thr = 2.0 * float(np.max(St / (np.abs(Pt) + 1.0)))
        fb = float(np.mean(np.max(Sd / (np.abs(P) + 1.0), axis=1) > thr))
        rows = 4096
        Xb = np.resize(Xte, (rows, 4)).astype(np.float32)
        for _ in range(3):
            sur.predict(Xb)
        reps = 20
        t0 = time.perf_counter()
        for _ in range(reps):
            sur.predict(Xb)
        t_pred = (time.perf_counter() - t0) / reps
        trained = True
    finally:
        if not (keep and trained):
            sur.close()

    def errors(A, B):
        """median over points of the mean E(k) error, and of the xi / L_gv errors"""
        eE = np.mean(np.abs(np.exp(A[:, :32] - B[:, :32]) - 1.0), axis=1)
        exi = np.abs(A[:, 32] / B[:, 32] - 1.0)
        eL = np.abs(A[:, 33] / B[:, 33] - 1.0)
        return {"E_k_rel_err_median": float(np.median(eE)), "E_k_rel_err_mean": float(np.mean(eE)),
                "xi_rel_err_median": float(np.median(exi)), "L_gv_rel_err_median": float(np.median(eL)),
                "xi_rel_err_mean": float(np.mean(exi)), "L_gv_rel_err_mean": float(np.mean(eL))}

    z = lambda A: np.stack([A[:, 0], np.log(A[:, 1]), np.log(A[:, 2]), A[:, 3]], 1).astype(np.float64)
    ztr, zte = z(Xtr[ok_tr]), z(Xte)
    sz = ztr.std(0)
    nn = np.array([int(np.argmin((((zte[i] - ztr) / sz) ** 2).sum(-1))) for i in range(zte.shape[0])])
    m = ok_te
    out = {"train_points": int(ok_tr.sum()), "test_points": int(m.sum()), "members": 4, "targets": 40,
           "protocol": proto, "simulate_batched_s": t_batch, "simulate_plain_s": t_plain,
           "simulate_plain_s_per_point": t_plain / n_test, "simulate_batched_s_per_point": t_batch / n_train,
           "train_s": t_fit, "train_loss": loss, "train_backend": "tcgen05",
           "surrogate": errors(P[m], Yte[m]),
           "baseline_training_mean": errors(np.broadcast_to(Ytr[ok_tr].mean(0), Yte[m].shape), Yte[m]),
           "baseline_nearest_point": errors(Ytr[ok_tr][nn[m]], Yte[m]),
           "noise_floor_two_plain_runs": errors(Yno[np.all(np.isfinite(Yno), 1) & m[:n_noise]],
                                                Yte[:n_noise][np.all(np.isfinite(Yno), 1) & m[:n_noise]]),
           "targets_spec": {"E_k": 0.10, "xi": 0.05, "L_gv": 0.05},
           "fallback_rate": fb, "fallback_threshold": thr,
           "predict_rows_per_s": rows / t_pred, "predict_s_per_point": t_pred / rows,
           "speedup_vs_plain_simulation_per_point": (t_plain / n_test) / (t_pred / rows)}
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"] \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1900.0
    # device time of the forward products alone at a dense-map batch
    # (4 members x 262,144 rows), tcgen05 fused kernel against warp-level mma.sync
    big = 262144
    Xg = synth.surrogate_points(big, seed=seed + 23).astype(np.float32)
    sg = S.Surrogate(members=4, max_rows=big, seed=seed + 1)
    try:
        sg.predict(Xg)
        fwd = {}
        for tc in (True, False):
            sg.set_backend(tc)
            sg.bench_forward(big, 3)
            fwd["tcgen05" if tc else "mma_sync"] = sg.bench_forward(big, 20)
    finally:
        sg.close()
    fl_big = 2.0 * 4 * big * (16 * 256 + 256 * 256 + 256 * 48)
    tc_tflops = fl_big / fwd["tcgen05"] / 1e9
    out.update({"forward_rows": big, "forward_ms_tcgen05": fwd["tcgen05"], "forward_ms_mma_sync": fwd["mma_sync"],
                "roofline": {"bound": "tensor", "kernel": "k_mlp_fwd_tc", "achieved": tc_tflops, "peak": peak,
                             "unit": "TFLOP/s", "frac": tc_tflops / peak, "peak_src": "measured bf16 burst"},
                "note": "errors: medians over held-out points; E_k error is the mean over the 32 shell-pair bins "
                        "of |E_pred/E_sim - 1|; predict_rows_per_s: 4096-row C-ABI calls with host copies"})
    return (out, (sur, thr, proto)) if keep else out


def run_reference(args, cfg):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # bounded sample: a density-3 sub-box whose oracle step is well under a second
    Ls = 128.0 if cfg["n_beads"] > 200000 else cfg["L"]
    nb = int(round(cfg["n_beads"] * (Ls / cfg["L"]) ** 2)) // 2 * 2
    import oracle
    from paper_1310_0998_gb300 import synth
    oracle.build()
    x, v = synth.dimers(nb // 2, Ls, PHYS["r0"], seed=0)
    st = oracle.State(oracle.params(L=Ls, seed=0, **PHYS), x, v, cells=True)
    st.run(args.warmup)
    t0 = time.perf_counter()
    st.run(args.steps)
    dt = time.perf_counter() - t0
    value = nb * args.steps / dt
    line = {"impl": "reference", "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "bead_density": 3.0, "sample_beads": nb},
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{args.steps} steps of the FP64 cell-list oracle on a {nb}-bead sub-box (L={Ls:g}) of the same density and parameters"},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c3", choices=sorted(CONFIGS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate leg")
    ap.add_argument("--no-3d", action="store_true", help="skip the three-dimensional leg")
    ap.add_argument("--no-obs", action="store_true", help="skip the observables leg")
    ap.add_argument("--wexp", type=float, default=0.0,
                    help="exponent s of w in the dissipative/random forces (0 = 2, the printed form)")
    ap.add_argument("--variant", type=int, default=0,
                    help="pair kernel: 0 tuned, 1 thread-per-bead, 2 queue, 3 grid-order queue, 4 flat ranges, "
                         "5 queue over merged ranges")
    ap.add_argument("--tile", type=int, default=0, help="cell-block side: 0 tuned, 4, 8, 16")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched-ensemble leg")
    ap.add_argument("--ens-replicas", type=int, default=256)
    ap.add_argument("--ens-steps", type=int, default=10000)
    ap.add_argument("--ens-seq-steps", type=int, default=500)
    ap.add_argument("--no-sweep", action="store_true", help="skip the C2 parameter-sweep leg")
    ap.add_argument("--sweep-steps", type=int, default=20000)
    ap.add_argument("--sweep-seq-steps", type=int, default=2000)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    cfg = CONFIGS[args.config]
    if args.impl == "reference":
        run_reference(args, cfg)
        return

    import torch
    import torch.distributed as dist
    from paper_1310_0998_gb300 import Sim, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    L, nb = cfg["L"], cfg["n_beads"]
    stream = torch.cuda.Stream(device=dev)
    x, v = synth.dimers(nb // 2, L, PHYS["r0"], seed=rank)
    phys = dict(a=PHYS["a"], gamma=PHYS["gamma"], kBT=PHYS["kBT"], rc=PHYS["rc"], k_bond=PHYS["kbond"],
                r0=PHYS["r0"], f_p=PHYS["fp"], zeta=PHYS["zeta"], dt=PHYS["dt"], mass=PHYS["mass"], wexp=args.wexp)
    tuning = None
    if args.variant == 0 and args.tile == 0:
        # kernel shape: every (cell-block side, pair walk) timed on this
        # workload; the context below takes the fastest (all shapes give the
        # same trajectory bits)
        from paper_1310_0998_gb300 import tune
        tuning = tune.autotune(L, nb, x, v, steps=5, stream=stream.cuda_stream, seed=rank, **phys)
    sim = Sim(L, nb, stream=stream.cuda_stream, seed=rank, variant=args.variant, tile=args.tile, **phys)
    sim.set_positions(x, v)
    sim.step(args.warmup)
    sim.sync()
    counts = sim.cell_counts()
    _, npairs = sim.pair_counts()
    n_cand, ops_step = algorithmic_ops(counts, int(npairs), nb)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)     # 512 MiB
    sink = torch.zeros(1, dtype=torch.float32, device=dev)

    def l2_flush(k):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
            sink.add_(flush[:: 1 << 12].sum())

    bus = None
    try:
        pr = torch.cuda.get_device_properties(dev)
        bus = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
        n_sm = int(pr.multi_processor_count)
    except Exception:
        bus, n_sm = None, 152
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # the K timed steps are one library call (CUDA graphs of 8 steps and a
    # final step that also writes the canonical state), bracketed by events on
    # the simulator's stream; every step touches ~200 MB (> the 129 MB L2).
    # The clock sampler starts 0.6 s of untimed steps before the timed region
    # so that it sees the GPU under this load whatever K is.
    clocks = Clocks(bus)
    t_pre = time.perf_counter()
    while time.perf_counter() - t_pre < 0.6:
        sim.step(64)
        sim.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    sim.sync()
    t_dev = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, dev)
    if world > 1:
        dist.barrier()
    value = job_throughput(world, nb, args.steps, t_dev)

    # per-kernel device times (same kernels, launched one by one between events)
    prof = []
    for k in range(min(args.steps, 20)):
        prof.append(sim.profile_step())
        l2_flush(k)
        torch.cuda.synchronize()
    prof = np.array(prof)
    force_s = float(prof[:, 2].mean()) / 1e3

    # end to end through the C ABI with host (pinned) buffers: upload the full
    # state (x double, v, f float), one step, download it
    x_h = torch.empty((nb, 2), dtype=torch.float64, pin_memory=True).numpy()
    v_h = torch.empty((nb, 2), dtype=torch.float32, pin_memory=True).numpy()
    f_h = torch.empty((nb, 2), dtype=torch.float32, pin_memory=True).numpy()
    _, _, _, s_cur = sim.get_state(x_h, v_h, f_h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        sim.set_state(x_h, v_h, f_h, s_cur)
        sim.step(1)
        _, _, _, s_cur = sim.get_state(x_h, v_h, f_h)
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world, dev)
    e2e_val = job_throughput(world, nb, args.e2e_steps, e2e_s)
    info = sim.info()

    pk = peaks()
    alu_peak = n_sm * LANES * pk["sm_max_mhz"] * 1e6
    alu_ach = ops_step / force_s
    hbm_ach = BYTES_PER_BEAD_STEP * value / world / 1e9
    traffic = measured_traffic(info.tile, info.variant) if cfg["name"].startswith("c3:") and args.wexp in (0.0, 2.0) \
        else None
    wipb = measured_warp_inst_per_bead(info.tile, info.variant) if args.wexp in (0.0, 2.0) else None
    issue = None
    if wipb is not None:
        slots = n_sm * SCHEDULERS * force_s * pk["sm_max_mhz"] * 1e6
        issue = {"warp_inst_per_bead": wipb, "frac": wipb * nb / slots,
                 "note": "warp instructions per bead from the committed ncu summary (this kernel source) x beads / "
                         "(SMs x 4 schedulers x the force kernel's event time x max SM clock): the share of issue "
                         "slots the kernel fills, the bound that binds"}
    line = {
        "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": cfg["name"], "beads": nb, "L": L, "bead_density": nb / L / L,
                   "tile": info.tile, "variant": info.variant, "wexp": args.wexp if args.wexp > 0 else 2.0,
                   "l2": "inputs larger than L2: every step reads and writes ~200 MB of state (L2 129 MB)",
                   "pairs_per_bead": npairs / nb, "candidates_per_bead": n_cand / nb,
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "alu", "kernel": "force_integrate", "achieved": alu_ach / 1e12,
                     "peak": alu_peak / 1e12, "unit": "Tops/s", "frac": alu_ach / alu_peak, "traffic": traffic,
                     "traffic_unit": "DRAM bytes per launch (ncu, body step of a multi-step call; null unless "
                                     "profiles/force_traffic_c3.md was taken on this kernel source and shape)",
                     "traffic_per_bead": traffic / nb if traffic else None,
                     "ops_per_bead_step": ops_step / nb,
                     "ops_model": f"{OPS_TEST:g} x candidate tests + {OPS_PAIR:g} x pairs + {OPS_BEAD:g} x beads, "
                                  "counted on the benchmarked state",
                     "peak_src": f"{n_sm} SMs x {LANES} lanes x {pk['sm_max_mhz']:.0f} MHz (max SM clock, "
                                 f"{pk['src']} peaks file)",
                     "ms": force_s * 1e3, "issue": issue},
        "hbm": {"achieved_gbs": hbm_ach, "peak_gbs": pk["hbm"], "frac": hbm_ach / pk["hbm"],
                "bytes_per_bead_step": BYTES_PER_BEAD_STEP, "peak_src": pk["src"]},
        "kernels_ms": {"scan": float(prof[:, 0].mean()), "scatter": float(prof[:, 1].mean()),
                       "force_integrate": float(prof[:, 2].mean())},
        "e2e": {"value": e2e_val, "unit": "particle-steps/s", "h2d_bytes_per_step": 32 * nb,
                "d2h_bytes_per_step": 32 * nb, "steps": args.e2e_steps},
        "gpu_launches": 3 * args.steps,
        "overflow_tiles": int(info.overflow_tiles),
        "clocks": clk,
    }
    if tuning is not None:
        line["tuning"] = tuning
    if rank == 0 and not args.no_ensemble:
        line["ensemble"] = ensemble_leg(args.ens_replicas, args.ens_steps, args.warmup, variant=args.variant,
                                        tile=args.tile, seq_steps=min(args.ens_seq_steps, args.ens_steps))
    model = None
    if rank == 0 and not args.no_surrogate:
        line["surrogate"], model = surrogate_leg(keep=True)
    if rank == 0 and not args.no_sweep:
        line["sweep"] = sweep_leg(steps=args.sweep_steps, seq_steps=min(args.sweep_seq_steps, args.sweep_steps),
                                  sur=model)
    if model is not None:
        model[0].close()
    if rank == 0 and not args.no_obs:
        line["observables"] = observables_leg(sim, nb)
    if rank == 0 and not args.no_3d:
        line["three_d"] = three_d_leg()
    if rank == 0 and not args.no_cpu:
        Lc = 128.0 if nb > 200000 else L
        nbc = int(round(nb * (Lc / L) ** 2)) // 2 * 2
        rate, cores, sample = cpu_oracle_rate(Lc, nbc)
        line["cpu_baseline"] = {"value": rate, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
                                "sample": sample}
    sim.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
