#!/usr/bin/env python
"""Throughput of the GB300 PIC/MCC particle loop (one JSON line).

Main line: the batched path.  64 independent 13.56 MHz argon discharges
(seed-drawn gap 1.5-5 cm, 2-50 Pa, 100-500 V, N_G 200-800, 1e4-2e6
particles per species, steady-shape states; ~2e7 electrons and ~2.3e7 Ar+ in
all, 0.7 GB of FP32 particle state, far above the 126 MB L2) are stepped
together, one push launch per species and one finalize launch per time step
for all discharges, replayed as one CUDA graph per ion subcycle.  One bench
step = 400 time steps (20 ion subcycles).  The metric is particle-steps/s
(electron pushes every step + ion pushes on ion steps); the roofline is that
of the electron particle kernel against the measured HBM copy bandwidth.

Beside it, on the same GPU: "plain" (the reference discharge of the paper's
Table 2 alone, ~4e5 e- + 4e5 Ar+, one RF cycle per bench step),
"dual_frequency" (1.356 + 27.12 MHz, N_G = 800, ~2e6 per species, one full LF
cycle), "df_sweep_table3" (the 20 dual-frequency discharges of Table 3 as one
batch), "null_collision_ions" (the batch with the null-collision method for
Ar+) and "served" (a Poisson stream of requests through the continuous-
batching server).  With --gpus N under torchrun every rank runs its own batch
(independent discharges: no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (FP64, one thread) on a bounded
sample of the same batch.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s and % HBM roofline; batched/served vs plain at ≤2% profile error"
UNIT = "particle-steps/s"
HBM_PEAK_FALLBACK = 6800.0   # GB/s: the profiling recipe's fallback, used only without MEASURED_PEAKS.json
BYTES_PER_PUSH_FP32 = 24     # read x, vx, vy, vz (16 B) + write x, vx (8 B)
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the electron
# particle kernel on the 64-discharge batch, from one ncu capture
# (profiles/k_push_electron_batch64.md: 336.512 + 125.846 MB for 19 973 477
# electrons), valid for the kernel source whose hash is given (null
# otherwise); scaled to a launch of the bench by its electron count (traffic
# grows in proportion: the particle streams dominate it).
TRAFFIC = {"sha": "47f25bf9b1035364", "bytes": 336512256 + 125845504, "particles": 19973477}
BATCH_DISCHARGES = 64
BATCH_STEPS = 400             # time steps per bench step (20 ion subcycles)
N_STEADY = 500_000            # plain leg: particles per species of the steady-shape state
DF_N = 2_000_000              # dual-frequency particles per species
DF_SWEEP_N = 100_000  # particles per species in each Table 3 discharge
# served leg: the C5 stream shape (200 Poisson requests of 20-200 RF cycles,
# parameters as the batch) with the particle counts scaled by SERVED_SCALE so
# that the stream fits the bench's time budget (--served-scale 1 for full size)
SERVED_REQUESTS = 200
SERVED_CYCLES = (20, 200)
SERVED_SCALE = 0.15
SERVED_LOAD = 0.8  # arrival rate as a fraction of the main line's measured throughput
CPU_SAMPLE_DISCHARGES = 4     # oracle sample: the first discharges of the batch
CPU_SAMPLE_WORK = 4e8         # particle-steps of the oracle sample (~15 s on one core)
_T0 = time.time()


def _log(msg: str):
    """Progress on stderr (stdout carries only the JSON line)."""
    print(f"[bench {time.time() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the plain, dual-frequency and served legs")
    ap.add_argument("--reference-sample", type=int, default=20,
                    help="time steps of the oracle per bench step in --impl reference")
    ap.add_argument("--served-requests", type=int, default=SERVED_REQUESTS)
    ap.add_argument("--served-cycles", type=int, nargs=2, default=SERVED_CYCLES)
    ap.add_argument("--served-scale", type=float, default=SERVED_SCALE,
                    help="particle counts of the served requests relative to the batch's (1 = config size)")
    ap.add_argument("--served-max-wall", type=float, default=300.0)
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    except Exception:
        return HBM_PEAK_FALLBACK, "fallback"


def _kernel_sha():
    h = hashlib.sha256()
    for f in ("edupic_kernels.cuh", "edupic_launch.cuh", "kernels_f32.cu", "edupic_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2103_09642_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu_index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.f.read().splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
            except ValueError:
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_over_ranks(ms_total: float, work: float, ws: int, device: str):
    """Whole-job figures of a replica run: the slowest rank's time and the
    work of all ranks (one all-reduce each; nothing else crosses ranks)."""
    if ws <= 1:
        return float(ms_total), float(work)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms_total)], dtype=torch.float64, device=device)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def _shapes_desc(shapes) -> dict:
    """The particle kernel's launch shapes the autotuner chose, per species."""
    from paper_2103_09642_gb300 import edupic as ed

    return {name: dict(index=int(sh), **ed.describe_push_shape(ed.FP32, int(sh)))
            for name, sh in zip(("electrons", "ions"), shapes)}


def _batch(rank: int):
    from paper_2103_09642_gb300 import workloads as wl

    return wl.batch_mix(n_discharges=BATCH_DISCHARGES, seed0=1000 + BATCH_DISCHARGES * rank)


BATCH_WORKLOAD = ("64 independent 13.56 MHz Ar CCPs (seed 1000+k): gap U[1.5,5] cm, p logU[2,50] Pa, "
                  "V0 U[100,500] V, N_G U{200..800}, n logU[1e4,2e6] per species, steady-shape states; "
                  "N_T=4000, N_SUB=20, FP32 particles, FP64 field and diagnostics")


def _oracle_sample(mix, step_work: float):
    """The first CPU_SAMPLE_DISCHARGES discharges of the batch in the oracle;
    steps (a multiple of N_SUB) sized to about `step_work` particle-steps."""
    import oracle
    from paper_2103_09642_gb300 import workloads as wl

    se, si = wl.standin_cross_sections()
    sims = [oracle.Sim(d, se, si, wl.CS_DE_EV, e, i) for d, e, i in mix[:CPU_SAMPLE_DISCHARGES]]
    n = sum(e.n + i.n / 20.0 for _, e, i in mix[:CPU_SAMPLE_DISCHARGES])
    steps = int(max(20, min(2000, step_work / max(n, 1.0))) // 20 * 20)
    return sims, steps


def _run_oracle(sims, steps):
    t0 = time.perf_counter()
    c0 = [s.counters() for s in sims]
    for s in sims:
        s.step(steps, measure=True)
    dt = time.perf_counter() - t0
    ps = 0
    for s, a in zip(sims, c0):
        c = s.counters()
        ps += (c["push_e"] - a["push_e"]) + (c["push_i"] - a["push_i"])
    return ps, dt


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _oracle_one_discharge(args):
    """One discharge of the batch in the oracle for `steps` time steps
    (a worker of the all-core baseline; CPU only)."""
    k, steps = args
    import numpy as np

    import oracle
    from paper_2103_09642_gb300 import workloads as wl

    d, e, i = wl.draw_discharge(np.random.default_rng(1000 + k), 1000 + k)  # discharge k of the batch
    se, si = wl.standin_cross_sections()
    s = oracle.Sim(d, se, si, wl.CS_DE_EV, e, i)
    c0 = s.counters()
    t0 = time.perf_counter()
    s.step(steps, measure=True)
    dt = time.perf_counter() - t0
    c = s.counters()
    return (c["push_e"] - c0["push_e"]) + (c["push_i"] - c0["push_i"]), dt


def cpu_baseline_all_cores(mix, pool, cores: int) -> dict:
    """The oracle on every host core at once: discharge k of the batch in
    worker k (independent discharges, as the batch is), each for a number of
    time steps sized to about CPU_SAMPLE_WORK / 4 particle-steps."""
    jobs = []
    for k in range(cores):
        d, e, i = mix[k % len(mix)]
        n = e.n + i.n / 20.0
        jobs.append((k % len(mix), int(max(20, min(2000, CPU_SAMPLE_WORK / 4 / max(n, 1.0))) // 20 * 20)))
    t0 = time.perf_counter()
    res = pool.map(_oracle_one_discharge, jobs)
    wall = time.perf_counter() - t0
    ps = sum(r[0] for r in res)
    return {"value": ps / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"discharges 0-{cores - 1} of the 64-discharge batch, one per process on {cores} cores "
                      f"({', '.join(str(j[1]) for j in jobs[:4])}... time steps each), FP64 "
                      f"({ps} particle-steps in {wall:.1f} s of wall time)"}


def cpu_baseline(mix, pool=None, cores: int = 1) -> dict:
    """The oracle (FP64) on a bounded sample of the same batch: one host
    thread on discharges 0-3, and, with a worker pool, all host cores."""
    sims, steps = _oracle_sample(mix, CPU_SAMPLE_WORK)
    ps, dt = _run_oracle(sims, steps)
    one = {"value": ps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"discharges 0-{CPU_SAMPLE_DISCHARGES - 1} of the 64-discharge batch, {steps} time steps each, "
                     f"FP64, one host thread ({ps} particle-steps in {dt:.1f} s)"}
    if pool is None:
        one["cpu_model"] = _cpu_model()
        return one
    out = cpu_baseline_all_cores(mix, pool, cores)
    out["one_core"] = one
    out["cpu_model"] = _cpu_model()
    out["nproc"] = os.cpu_count()
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    mix = _batch(0)
    sample = max(1, args.reference_sample)  # time steps per bench step (default: one ion subcycle)
    sims, _ = _oracle_sample(mix, 0)
    del mix
    for _ in range(args.warmup):
        _run_oracle(sims, sample)
    ps_tot, dt_tot = 0, 0.0
    for _ in range(args.steps):
        ps, dt = _run_oracle(sims, sample)
        ps_tot += ps
        dt_tot += dt
    v = ps_tot / dt_tot
    desc = (f"discharges 0-{CPU_SAMPLE_DISCHARGES - 1} of the 64-discharge batch, {sample} time steps each per "
            f"bench step, FP64, one host thread")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt_tot / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": BATCH_WORKLOAD + " (bounded oracle sample)",
                                            "sample": desc},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _roofline(sim, nd, peak, peak_kind, measure=True, steps=400):
    """Electron-kernel roofline, timed live with CUDA events around every
    launch (edupic_profile_steps) on the simulation's own stream."""
    tot = lambda: sum(sim.counters(k)["push_e"] for k in range(nd))
    p0 = tot()
    ms_k, launches = sim.profile_steps(steps, measure=measure)
    per_launch = (tot() - p0) / max(launches[0], 1)
    dur_s = ms_k[0] / max(launches[0], 1) / 1000.0
    achieved = BYTES_PER_PUSH_FP32 * per_launch / dur_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "kernel": "k_push<float, electrons>", "bytes_per_particle_step": BYTES_PER_PUSH_FP32,
            "particles_per_launch": per_launch, "avg_launch_us": dur_s * 1e6, "peak_kind": peak_kind,
            "kernel_time_share": {k: float(v) / max(float(ms_k.sum()), 1e-12)
                                  for k, v in zip(("push_e", "push_i", "finalize"), ms_k)}}


def _timed(stream, flush, steps, run):
    """Device time (ms) of `steps` calls of run(), an L2-sized buffer written
    before each one outside the events."""
    import torch

    ms = 0.0
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run()
        b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
    return ms


def leg_plain(args, peak, peak_kind, flush) -> dict:
    """The reference discharge (Table 2: 250 V, 13.56 MHz, 25 mm, 10 Pa,
    350 K, N_G = 400) alone, steady-shape state of ~4e5 e- + 4e5 Ar+ (weight
    1.4e4), one RF cycle (4000 time steps) per bench step."""
    from paper_2103_09642_gb300 import edupic as ed
    from paper_2103_09642_gb300 import workloads as wl

    d, e, i = wl.reference_steady(seed=1, n=N_STEADY, capacity=2 * N_STEADY)
    se, si = wl.standin_cross_sections()
    sim = ed.simulation_for([d], ed.FP32, sigma=(se, si), de_ev=wl.CS_DE_EV, particles=[(e, i)])
    grid, _ = sim.autotune(subcycles=10, measure=True)
    graphs = sim.graphs()
    shapes = sim.push_shape()
    for _ in range(args.warmup):
        sim.run_cycles(1, measure=True)
    sim.synchronize()
    c0 = sim.counters(0)
    steps = max(3, min(args.steps, 10))
    ms = _timed(sim.stream, flush, steps, lambda: sim.run_cycles(1, measure=True))
    c1 = sim.counters(0)
    ps = (c1["push_e"] - c0["push_e"]) + (c1["push_i"] - c0["push_i"])
    n_e, n_i, _ = sim.counts(0)
    roof = _roofline(sim, 1, peak, peak_kind)
    sim.close()
    # end to end through the public API: particles from host arrays, one cycle, diagnostics back
    sim2 = ed.simulation_for([d], ed.FP32, sigma=(se, si), de_ev=wl.CS_DE_EV)
    for sp in (0, 1):
        sim2.set_push_shape(sp, shapes[sp])  # the launch the autotuner chose
    sim2.set_graphs(graphs)
    tot_ps, tot_t = 0, 0.0
    for r in range(3):
        t0 = time.perf_counter()
        sim2.load(0, ed.ELECTRONS, e)
        sim2.load(0, ed.IONS, i)
        ca = sim2.counters(0)
        sim2.run_cycles(1, measure=True)
        sim2.diagnostics(0)
        cb = sim2.counters(0)
        sim2.reset_diagnostics(0)
        if r > 0:  # the first repetition builds the graph
            tot_t += time.perf_counter() - t0
            tot_ps += (cb["push_e"] - ca["push_e"]) + (cb["push_i"] - ca["push_i"])
    sim2.close()
    # the same cycle with the xt diagnostics (N_XT = 200) accumulated
    simx = ed.simulation_for([d.replace(xt_bins=200)], ed.FP32, sigma=(se, si), de_ev=wl.CS_DE_EV,
                             particles=[(e, i)])
    simx.run_cycles(1, measure=True)
    simx.synchronize()
    cx0 = simx.counters(0)
    msx = _timed(simx.stream, flush, steps, lambda: simx.run_cycles(1, measure=True))
    cx1 = simx.counters(0)
    psx = (cx1["push_e"] - cx0["push_e"]) + (cx1["push_i"] - cx0["push_i"])
    simx.close()
    return {"workload": "reference argon discharge (Table 2 settings, N_G=400, N_T=4000, N_SUB=20) in a "
                        "steady-shape state, weight 1.4e4, one RF cycle per bench step",
            "with_xt_diagnostics": {"value": psx / (msx / 1000.0), "unit": UNIT, "xt_bins": 200,
                                    "ms_per_rf_cycle": msx / steps},
            "particles_e": int(n_e), "particles_i": int(n_i), "value": ps / (ms / 1000.0), "unit": UNIT,
            "ms_per_rf_cycle": ms / steps, "us_per_time_step": 1000.0 * ms / (steps * d.steps_per_cycle),
            "steps": steps, "push_grid": grid, "push_shape": _shapes_desc(shapes), "roofline": roof,
            "e2e": {"value": tot_ps / tot_t, "unit": UNIT, "h2d_bytes_per_step": 16 * (e.n + i.n),
                    "d2h_bytes_per_step": 8 * (3 * d.n_grid + d.eepf_bins + 2 * d.ifed_bins)}}


def leg_dual_frequency(args, peak, peak_kind, flush) -> dict:
    """Dual-frequency discharge (1.356 MHz 300 V + 27.12 MHz 100 V, 5 Pa,
    N_G = 800, 16 000 steps per HF cycle, ~2e6 particles per species),
    timed over one full LF cycle (320 000 time steps)."""
    from paper_2103_09642_gb300 import edupic as ed
    from paper_2103_09642_gb300 import workloads as wl

    d, e, i = wl.dual_frequency(seed=1, v_lf=300.0, n=DF_N, capacity=2 * DF_N)
    se, si = wl.standin_cross_sections()
    sim = ed.simulation_for([d], ed.FP32, sigma=(se, si), de_ev=wl.CS_DE_EV, particles=[(e, i)])
    n_e0, n_i0 = e.n, i.n
    del e, i
    grid, _ = sim.autotune(subcycles=10, measure=True)
    sim.step(max(args.warmup, 3) * 200, measure=True)
    sim.synchronize()
    c0 = sim.counters(0)
    ms = _timed(sim.stream, flush, 1, lambda: sim.run_cycles(1, measure=True))
    c1 = sim.counters(0)
    ps = (c1["push_e"] - c0["push_e"]) + (c1["push_i"] - c0["push_i"])
    n_e, n_i, _ = sim.counts(0)
    roof = _roofline(sim, 1, peak, peak_kind)
    sim.close()
    return {"workload": "dual-frequency Ar CCP: 1.356 MHz 300 V + 27.12 MHz 100 V, 25 mm, 5 Pa, 350 K, N_G=800, "
                        "16000 steps per HF cycle, steady-shape state, one LF cycle timed",
            "particles_e0": int(n_e0), "particles_i0": int(n_i0), "particles_e": int(n_e), "particles_i": int(n_i),
            "value": ps / (ms / 1000.0), "unit": UNIT, "time_steps": int(d.steps_per_cycle),
            "ms_per_lf_cycle": ms, "us_per_time_step": 1000.0 * ms / d.steps_per_cycle,
            "push_grid": grid, "roofline": roof}


def leg_null_collision(args, mix, flush) -> dict:
    """The 64-discharge batch with the null-collision method (Sec. 2.1.6) for
    Ar+ + Ar (the thermal partner is drawn for the picked ions only) and the
    direct test for e- + Ar, the same bench steps as the main line."""
    from paper_2103_09642_gb300 import edupic as ed
    from paper_2103_09642_gb300 import workloads as wl

    ds = [m[0].replace(null_collision=2) for m in mix]
    nd = len(ds)
    se, si = wl.standin_cross_sections()
    sim = ed.simulation_for(ds, ed.FP32, sigma=(se, si), de_ev=wl.CS_DE_EV, particles=[(m[1], m[2]) for m in mix])
    for _ in range(args.warmup):
        sim.step(BATCH_STEPS, measure=True)
    sim.synchronize()
    tot = lambda key: sum(sim.counters(k)[key] for k in range(nd))
    c0 = tot("push_e") + tot("push_i")
    steps = max(3, min(args.steps, 5))
    ms = _timed(sim.stream, flush, steps, lambda: sim.step(BATCH_STEPS, measure=True))
    ps = tot("push_e") + tot("push_i") - c0
    ms_k, launches = sim.profile_steps(BATCH_STEPS, measure=True)
    sim.close()
    return {"workload": "the 64-discharge batch, null-collision method for Ar+ (null_collision = 2), direct test "
                        "for e-", "value": ps / (ms / 1000.0), "unit": UNIT, "steps": steps,
            "us_per_time_step": 1000.0 * ms / (steps * BATCH_STEPS),
            "us_per_launch": {k: float(v) / max(int(n), 1) * 1000.0
                              for k, v, n in zip(("push_e", "push_i", "finalize"), ms_k, launches)}}


def leg_df_sweep(args, peak, peak_kind, flush) -> dict:
    """The 20 dual-frequency discharges of Table 3 (2 MHz + 10/20 MHz at 20 Pa,
    2 MHz + 30/40 MHz at 3 Pa, V_LF 0-400 V; the table's W, N_G and N_T),
    1e5 particles per species each, stepped as one batch."""
    from paper_2103_09642_gb300 import edupic as ed
    from paper_2103_09642_gb300 import workloads as wl

    mix = wl.df_sweep(n=DF_SWEEP_N)
    ds = [m[0] for m in mix]
    nd = len(ds)
    se, si = wl.standin_cross_sections()
    sim = ed.simulation_for(ds, ed.FP32, sigma=(se, si), de_ev=wl.CS_DE_EV, particles=[(m[1], m[2]) for m in mix])
    del mix
    for _ in range(args.warmup):
        sim.step(BATCH_STEPS, measure=True)
    sim.synchronize()
    tot = lambda: sum(sim.counters(k)["push_e"] + sim.counters(k)["push_i"] for k in range(nd))
    c0 = tot()
    steps = max(3, min(args.steps, 5))
    ms = _timed(sim.stream, flush, steps, lambda: sim.step(BATCH_STEPS, measure=True))
    ps = tot() - c0
    n_e = sum(sim.counts(k)[0] for k in range(nd))
    roof = _roofline(sim, nd, peak, peak_kind, steps=BATCH_STEPS)
    sim.close()
    return {"workload": "Table 3 dual-frequency sweep: 20 discharges (CASE 1 20 Pa, CASE 2 3 Pa; f_LF 2 MHz, "
                        "V_LF 0-400 V), 1e5 particles per species each, one batch",
            "discharges": nd, "particles_e": int(n_e), "value": ps / (ms / 1000.0), "unit": UNIT, "steps": steps,
            "time_steps_per_step": BATCH_STEPS, "us_per_time_step": 1000.0 * ms / (steps * BATCH_STEPS),
            "roofline": roof}


def leg_served(args, capacity_ps: float) -> dict:
    """The served configuration: a Poisson stream of requests through the
    request server (continuous batching), drawn like the 64-discharge batch
    (particle counts scaled by --served-scale), each asking for a number of RF
    cycles drawn from --served-cycles; arrivals at SERVED_LOAD x the main
    line's throughput divided by the mean request work."""
    import math

    import torch

    from paper_2103_09642_gb300 import edupic as ed
    from paper_2103_09642_gb300 import serving
    from paper_2103_09642_gb300 import workloads as wl

    lo, hi = args.served_cycles
    mean_n = (2e6 - 1e4) / math.log(2e6 / 1e4) * args.served_scale  # log-uniform mean per species
    mean_ps = mean_n * (1.0 + 1.0 / 20.0) * 4000 * 0.5 * (lo + hi)
    rate = SERVED_LOAD * capacity_ps / mean_ps
    specs = serving.poisson_stream(args.served_requests, rate_hz=rate, seed=7, cycles=(lo, hi),
                                   scale=args.served_scale)
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.5 * free) // 256 * 256
    se, si = wl.standin_cross_sections()
    srv = ed.Server(budget, max_slots=96, max_grid=800, max_eepf_bins=2000, precision=ed.FP32)
    srv.set_cross_sections(ed.ELECTRONS, se, wl.CS_DE_EV)
    srv.set_cross_sections(ed.IONS, si, wl.CS_DE_EV)
    rep = serving.run_stream(srv, specs, chunk_subcycles=5, max_wall_s=args.served_max_wall)
    srv.close()
    return {"workload": f"{args.served_requests} Poisson-arrival requests (rate {rate:.3g}/s = {SERVED_LOAD} x the "
                        f"main line's throughput / mean request work), parameters as the 64-discharge batch with "
                        f"particle counts x{args.served_scale:g}, {lo}-{hi} RF cycles each",
            "particle_scale": args.served_scale, "rate_hz": rate,
            "value": rep["particle_steps_per_s"], "unit": UNIT,
            "p50_time_to_result_s": rep["p50_time_to_result_s"], "p99_time_to_result_s": rep["p99_time_to_result_s"],
            "makespan_s": rep["makespan_s"], "requests": rep["requests"], "failed": rep["failed"],
            "hbm_budget_bytes": budget}


def run_ours(args):
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2103_09642_gb300 import edupic as ed
    from paper_2103_09642_gb300 import workloads as wl

    # the all-core oracle baseline's workers, started (spawn) before any GPU work
    pool, cores = None, 1
    if rank == 0 and ws == 1 and not args.no_cpu:
        import multiprocessing as mp

        cores = max(1, min(os.cpu_count() or 1, BATCH_DISCHARGES))
        pool = mp.get_context("spawn").Pool(cores)
    ed.load_library()
    peak, peak_kind = _peak_hbm()
    _log("generating the 64-discharge batch")
    mix = _batch(rank)
    ds = [m[0] for m in mix]
    nd = len(ds)
    se, si = wl.standin_cross_sections()
    sim = ed.simulation_for(ds, ed.FP32, sigma=(se, si), de_ev=wl.CS_DE_EV, particles=[(m[1], m[2]) for m in mix])
    stream = sim.stream
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    _log("batch created; autotuning the stepping mode")
    grid, _ = sim.autotune(subcycles=5, measure=True)  # launch shapes and graph replay, by timing (warm-up steps)
    graphs = sim.graphs()
    shapes = sim.push_shape()
    grids = sim.push_grid()
    _log("warm-up")

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        sim.step(BATCH_STEPS, measure=True)
    sim.synchronize()
    split = lambda: [sum(sim.counters(k)[key] for k in range(nd)) for key in ("push_e", "push_i")]
    tot = lambda: sum(split())
    s0 = split()
    c0 = sum(s0)
    ne0 = sum(sim.counts(k)[0] for k in range(nd))
    ni0 = sum(sim.counts(k)[1] for k in range(nd))
    _log("timed steps")
    clocks = Clocks(local)
    barrier()
    ms_total = _timed(stream, flush, args.steps, lambda: sim.step(BATCH_STEPS, measure=True))
    barrier()
    clk = clocks.stop()
    sim.synchronize()
    s1 = split()
    ps = sum(s1) - c0
    ms_max, ps_all = reduce_over_ranks(ms_total, ps, ws, "cuda")
    value = ps_all / (ms_max / 1000.0)
    # electron pushes (every step) and ion pushes (ion steps), this rank, per second of its device time
    pushes = {"electrons": (s1[0] - s0[0]) / (ms_total / 1000.0), "ions": (s1[1] - s0[1]) / (ms_total / 1000.0),
              "unit": "particle-steps/s", "scope": "rank 0" if ws > 1 else "all"}
    n_e = sum(sim.counts(k)[0] for k in range(nd))
    n_i = sum(sim.counts(k)[1] for k in range(nd))
    _log("roofline")
    roof = _roofline(sim, nd, peak, peak_kind)
    sha = _kernel_sha()
    roof["kernel_src"] = sha
    roof["traffic"] = (TRAFFIC["bytes"] / TRAFFIC["particles"] * roof["particles_per_launch"]
                       if TRAFFIC["sha"] == sha else None)
    sim.close()

    # end to end through the public API: every discharge's particles from host
    # FP64 arrays (converted and copied as FP32), one bench step, diagnostics back
    e2e = None
    if not args.no_e2e:
        _log("end to end")
        sim2 = ed.simulation_for(ds, ed.FP32, sigma=(se, si), de_ev=wl.CS_DE_EV)
        for sp in (0, 1):
            sim2.set_push_shape(sp, shapes[sp])  # the launch shapes and
        sim2.set_graphs(graphs)  # the stepping mode the autotuner chose
        h2d = 16 * sum(m[1].n + m[2].n for m in mix)
        d2h = sum(8 * (3 * d.n_grid + d.eepf_bins + 2 * d.ifed_bins) for d in ds)
        reps = max(2, min(args.steps, 3))
        tot_ps, tot_t = 0, 0.0
        for r in range(reps + 1):
            t0 = time.perf_counter()
            for k, (d, e, i) in enumerate(mix):
                sim2.load(k, ed.ELECTRONS, e)
                sim2.load(k, ed.IONS, i)
            ca = sum(sim2.counters(k)["push_e"] + sim2.counters(k)["push_i"] for k in range(nd))
            sim2.step(BATCH_STEPS, measure=True)
            for k in range(nd):
                sim2.diagnostics(k)
            cb = sum(sim2.counters(k)["push_e"] + sim2.counters(k)["push_i"] for k in range(nd))
            for k in range(nd):
                sim2.reset_diagnostics(k)
            if r > 0:  # the first repetition builds the graph
                tot_t += time.perf_counter() - t0
                tot_ps += cb - ca
        sim2.close()
        e2e = {"value": tot_ps / tot_t, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "steps": reps, "note": "64 discharges loaded from host FP64 arrays + 400 time steps + diagnostics "
                                      "of every discharge read back, per step"}

    extra = {}
    if rank == 0 and ws == 1 and not args.no_extra:
        _log("plain leg")
        extra["plain"] = leg_plain(args, peak, peak_kind, flush)
        _log("dual-frequency leg")
        extra["dual_frequency"] = leg_dual_frequency(args, peak, peak_kind, flush)
        _log("Table 3 sweep leg")
        extra["df_sweep_table3"] = leg_df_sweep(args, peak, peak_kind, flush)
        _log("null-collision leg")
        extra["null_collision_ions"] = leg_null_collision(args, mix, flush)
        _log("served leg")
        extra["served"] = leg_served(args, value)
    if rank == 0 and ws == 1 and not args.no_cpu:
        _log("cpu baseline")
    cpu = cpu_baseline(mix, pool, cores) if (rank == 0 and ws == 1 and not args.no_cpu) else None
    if pool is not None:
        pool.close()
        pool.join()
    _log("done")

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "discharges": nd, "time_steps_per_step": BATCH_STEPS,
                       "particles_e": int(n_e), "particles_i": int(n_i),
                       "l2": "256 MB buffer written between timed steps (outside the timed events); "
                             "particle state 0.7 GB > L2",
                       "parallelism": f"replicas x{ws}", "cross_sections": "stand-in set",
                       "push_grid": list(grids), "push_shape": _shapes_desc(shapes), "graph_replay": graphs,
                       # the steady-shape states still relax during the timed steps; `value` counts the
                       # pushes actually made, so it is exact for the population of the timed region
                       "population_timed": {"e_start": int(ne0), "e_end": int(n_e), "i_start": int(ni0),
                                            "i_end": int(n_i)}},
            "roofline": roof,
            "pushes": pushes,
            "gpu_launches": int(args.steps * (2 * BATCH_STEPS + BATCH_STEPS // ds[0].ion_subcycle)),
            "clocks": clk,
        }
        if e2e:
            line["e2e"] = e2e
        if cpu:
            line["cpu_baseline"] = cpu
        line.update(extra)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
