"""A short, fixed run of the particle loop for profiler captures.

  python -m paper_2103_09642_gb300.profile_case --n 5000000 --steps 3 [--fp64] [--discharges K]
  python -m paper_2103_09642_gb300.profile_case --mix 64 --steps 3 [--shape S]

Runs the reference discharge in a steady-shape state with n particles per
species (split over K independent discharges), or with --mix K the batch of
K seed-drawn discharges (seeds 1000 + k), `warmup` + `steps` time steps
launched one by one, then prints the counters.  Sizes above ~3e6 per
species put the FP32 particle state (16 B per particle) above the 126 MB L2.
"""
from __future__ import annotations

import argparse
import json


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=5_000_000)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--discharges", type=int, default=1)
    ap.add_argument("--measure", action="store_true")
    ap.add_argument("--mix", type=int, default=0, help="the batch of this many seed-drawn discharges")
    ap.add_argument("--shape", type=int, default=-1, help="launch shape of the particle kernel (both species)")
    a = ap.parse_args()

    import torch

    from . import edupic as ed
    from . import workloads as wl

    torch.cuda.set_device(0)
    ds, parts = [], []
    if a.mix:
        for d, e, i in wl.batch_mix(n_discharges=a.mix, seed0=1000):
            ds.append(d)
            parts.append((e, i))
    else:
        per = a.n // a.discharges
        for k in range(a.discharges):
            d, e, i = wl.reference_steady(seed=1 + k, n=per, capacity=2 * per)
            ds.append(d)
            parts.append((e, i))
    se, si = wl.standin_cross_sections()
    sim = ed.simulation_for(ds, ed.FP64 if a.fp64 else ed.FP32, sigma=(se, si), de_ev=wl.CS_DE_EV,
                            particles=parts)
    sim.set_graphs(False)
    if a.shape >= 0:
        sim.set_push_shape(ed.ELECTRONS, a.shape)
        sim.set_push_shape(ed.IONS, a.shape)
    sim.step(a.warmup, measure=a.measure)
    sim.synchronize()
    sim.step(a.steps, measure=a.measure)
    sim.synchronize()
    print(json.dumps({"discharges": len(ds), "n_e": sum(sim.counts(k)[0] for k in range(len(ds))),
                      "n_i": sum(sim.counts(k)[1] for k in range(len(ds))), "counters_0": sim.counters(0)}))
    sim.close()


if __name__ == "__main__":
    main()
