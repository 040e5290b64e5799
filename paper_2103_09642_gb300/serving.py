"""A Poisson-arrival stream of discharge requests through the request server.

  python -m paper_2103_09642_gb300.serving [--requests 200] [--rate R] [--budget-frac 0.5]
                                           [--cycles 20 200] [--scale 1.0] [--out result.json]

Each request is an independent 13.56 MHz argon discharge drawn like the
64-discharge batch (gap 1.5-5 cm, 2-50 Pa, 100-500 V, N_G 200-800, 1e4-2e6
particles per species, steady-shape initial state) asking for a number of RF
cycles drawn uniformly from --cycles.  Requests arrive at exponentially
distributed intervals (rate --rate per second), are admitted by the server
while slots and HBM budget allow, run batched with everything else that is
resident, and are retired with their diagnostics.  The report gives p50/p99
time-to-result (arrival to result available on the host) and the aggregate
particle-steps/s over the stream.
"""
from __future__ import annotations

import argparse
import json
import math
import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import workloads as wl


@dataclass
class RequestSpec:
    arrival_s: float
    n_cycles: int
    discharge: wl.Discharge
    electrons: wl.Particles
    ions: wl.Particles
    record: dict = field(default_factory=dict)


def poisson_stream(n_requests: int, rate_hz: float, seed: int = 7, cycles=(20, 200), scale: float = 1.0,
                   steps_per_cycle: int = 4000, seed0: int = 5000) -> List[RequestSpec]:
    """Requests with exponential inter-arrival times (mean 1/rate_hz) and
    C4-style discharges; request k uses seed seed0 + k."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n_requests):
        t += rng.exponential(1.0 / rate_hz) if rate_hz > 0 else 0.0
        nc = int(rng.integers(cycles[0], cycles[1] + 1))
        d, e, i = wl.draw_discharge(np.random.default_rng(seed0 + k), seed0 + k, scale=scale,
                                    steps_per_cycle=steps_per_cycle)
        out.append(RequestSpec(t, nc, d, e, i))
    return out


def percentile(v, q: float) -> Optional[float]:
    """Nearest-rank percentile (q in [0, 100]) of a non-empty list, else None."""
    if not len(v):
        return None
    s = sorted(v)
    k = max(0, min(len(s) - 1, int(math.ceil(q / 100.0 * len(s))) - 1))
    return float(s[k])


def run_stream(server, specs: List[RequestSpec], chunk_subcycles: int = 5, clock=time.perf_counter,
               sleep=time.sleep, keep_results: bool = False, max_wall_s: Optional[float] = None) -> dict:
    """Feed `specs` to `server` at their arrival times (relative to the start
    of this call), keep calling server.advance(chunk_subcycles) while work is
    resident or queued, and collect each request's timing and counters.
    Raises TimeoutError after `max_wall_s` seconds (if given)."""
    order = sorted(range(len(specs)), key=lambda k: specs[k].arrival_s)
    t0 = clock()
    srv0 = server.stats()["now"]
    nxt = 0
    live = {}
    log = []
    done = 0
    while done < len(specs):
        now = clock() - t0
        if max_wall_s is not None and now > max_wall_s:
            raise TimeoutError(f"request stream not finished after {max_wall_s} s "
                               f"({done} of {len(specs)} done, {len(live)} live)")
        while nxt < len(order) and specs[order[nxt]].arrival_s <= now:
            s = specs[order[nxt]]
            tk = server.submit(s.discharge, s.electrons, s.ions, s.n_cycles)
            s.record = {"ticket": tk, "arrival_s": s.arrival_s, "submit_s": clock() - t0, "n_cycles": s.n_cycles,
                        "n_e0": int(s.electrons.n), "n_i0": int(s.ions.n), "n_grid": s.discharge.n_grid,
                        "bytes": server.request_bytes(s.discharge)}
            live[tk] = s
            nxt += 1
        running, queued = server.advance(chunk_subcycles)
        for tk in list(live):
            inf = server.info(tk)
            if inf["state"] < 2:
                continue
            s = live.pop(tk)
            r = s.record
            r["admit_s"] = inf["t_admit"] - srv0 if inf["t_admit"] >= 0 else None
            r["done_s"] = inf["t_done"] - srv0
            r["time_to_result_s"] = r["done_s"] - s.arrival_s
            r["state"] = "done" if inf["state"] == 2 else "failed"
            r["status"] = inf["status"]
            r["steps"] = inf["steps_done"]
            if inf["state"] == 2:
                res = server.result(tk)
                c = res["counters"]
                r["particle_steps"] = c["push_e"] + c["push_i"]
                if keep_results:
                    r["result"] = res
            else:
                r["particle_steps"] = 0
            server.release(tk)
            log.append(r)
            done += 1
        if running == 0 and queued == 0 and nxt < len(order):
            wait = specs[order[nxt]].arrival_s - (clock() - t0)
            if wait > 0:
                sleep(min(wait, 0.05))
    makespan = max((r["done_s"] for r in log), default=0.0)
    ttr = [r["time_to_result_s"] for r in log if r["state"] == "done"]
    ps = sum(r["particle_steps"] for r in log)
    return {"requests": len(log), "failed": sum(1 for r in log if r["state"] != "done"),
            "p50_time_to_result_s": percentile(ttr, 50), "p99_time_to_result_s": percentile(ttr, 99),
            "makespan_s": makespan, "particle_steps": ps,
            "particle_steps_per_s": ps / makespan if makespan > 0 else None, "log": log}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=None, help="arrivals per second (default: 0.8 x capacity)")
    ap.add_argument("--capacity-ps", type=float, default=8.5e10,
                    help="batched particle-steps/s used to set the default rate")
    ap.add_argument("--cycles", type=int, nargs=2, default=(20, 200))
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--budget-frac", type=float, default=0.5, help="fraction of free HBM given to the server")
    ap.add_argument("--slots", type=int, default=96)
    ap.add_argument("--chunk", type=int, default=5, help="ion subcycles per scheduling round")
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()

    import torch

    from . import edupic as ed

    torch.cuda.set_device(0)
    # mean work of one request: particles of both species (ions every N_SUB steps) x steps
    mean_n = (2e6 - 1e4) / math.log(2e6 / 1e4) * a.scale
    mean_ps = mean_n * (1.0 + 1.0 / 20.0) * 4000 * 0.5 * (a.cycles[0] + a.cycles[1])
    rate = a.rate if a.rate else 0.8 * a.capacity_ps / mean_ps
    specs = poisson_stream(a.requests, rate, a.seed, tuple(a.cycles), a.scale)
    free, _ = torch.cuda.mem_get_info()
    budget = int(a.budget_frac * free) // 256 * 256
    se, si = wl.standin_cross_sections()
    srv = ed.Server(budget, max_slots=a.slots, max_grid=800, max_eepf_bins=2000, precision=ed.FP32)
    srv.set_cross_sections(ed.ELECTRONS, se, wl.CS_DE_EV)
    srv.set_cross_sections(ed.IONS, si, wl.CS_DE_EV)
    rep = run_stream(srv, specs, chunk_subcycles=a.chunk)
    rep.update({"rate_hz": rate, "budget_bytes": budget, "slots": a.slots, "chunk_subcycles": a.chunk,
                "cycles": list(a.cycles), "scale": a.scale})
    srv.close()
    line = {k: v for k, v in rep.items() if k != "log"}
    print(json.dumps(line))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rep, f)


if __name__ == "__main__":
    main()
