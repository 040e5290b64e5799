"""Oracle runs executed in worker processes by the GPU tests (CPU only: this
module imports neither torch nor the CUDA package, so a spawned worker
starts without touching the GPU)."""
import numpy as np

from paper_2103_09642_gb300 import workloads as wl


def run_statistics(seed: int, n: int, warm: int, measured: int) -> dict:
    """The reference discharge in a steady-shape state (n per species),
    `warm` unmeasured and `measured` measured RF cycles in the oracle;
    returns the diagnostics and the counter increments of the measured part."""
    import oracle

    se, si = wl.standin_cross_sections()
    d, e, i = wl.reference_steady(seed=seed, n=n)
    ref = oracle.Sim(d, se, si, wl.CS_DE_EV, e, i)
    ref.step(warm * d.steps_per_cycle, measure=False)
    c0 = ref.counters()
    ref.step(measured * d.steps_per_cycle, measure=True)
    c1 = ref.counters()
    dg = ref.diagnostics()
    return {"n_e": np.asarray(dg["n_e"]), "n_i": np.asarray(dg["n_i"]),
            "eepf_counts": np.asarray(dg["eepf_counts"]), "ifed_pow_counts": np.asarray(dg["ifed_pow_counts"]),
            "ifed_gnd_counts": np.asarray(dg["ifed_gnd_counts"]),
            "counters0": c0, "counters1": c1}


def run_dual_frequency(seed: int, n: int, steps: int) -> dict:
    """The dual-frequency discharge (1.356 + 27.12 MHz) in a steady-shape
    state of n per species, `steps` measured steps in the oracle."""
    import oracle

    se, si = wl.standin_cross_sections()
    d, e, i = wl.dual_frequency(seed=seed, v_lf=300.0, n=n)
    ref = oracle.Sim(d, se, si, wl.CS_DE_EV, e, i)
    c0 = ref.counters()
    ref.step(steps, measure=True)
    c1 = ref.counters()
    dg = ref.diagnostics()
    return {"n_e": np.asarray(dg["n_e"]), "n_i": np.asarray(dg["n_i"]),
            "eepf_counts": np.asarray(dg["eepf_counts"]), "ifed_pow_counts": np.asarray(dg["ifed_pow_counts"]),
            "ifed_gnd_counts": np.asarray(dg["ifed_gnd_counts"]),
            "counters0": c0, "counters1": c1}
