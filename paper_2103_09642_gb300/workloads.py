"""Seeded synthetic inputs shaped like the paper's discharges.

This module only *generates inputs*: discharge parameter sets, a stand-in
cross-section set, and initial particle states.  It holds none of the PIC/MCC
method's arithmetic and is the one module that both the CUDA path and the CPU
oracle are fed from.

Workloads (the paper's Table 2 reference discharge and Sec. 4.2 dual-frequency
discharges give their shape):

* ``reference_start``: Table 2 discharge (250 V, 13.56 MHz, W = 7e4, L = 25 mm,
  10 Pa, 350 K, N_G = 400, N_T = 4000) seeded with 1000 e- + 1000 Ar+ uniform in
  x with Maxwellian velocities (e- at 1 eV, Ar+ at the gas temperature).
* ``reference_steady``: the same discharge at a weight lowered to 1.4e4, so a
  steady-shape state holds ~5e5 particles per species (the paper's ~1e5 at
  W = 7e4 is the same density).
* ``dual_frequency``: 1.356 MHz (0-300 V) + 27.12 MHz (100 V), 5 Pa, N_G = 800,
  16000 steps per 27.12 MHz period, ~2e6 particles per species.
* ``batch_mix``: independent discharges with seed-drawn gap, pressure, voltage,
  N_G and particle count.

Cross sections: the Phelps analytic fits the paper tabulates (Sec. 3.2) are not
available here, so ``standin_cross_sections`` returns a smooth, self-written
set with argon's thresholds (11.5 eV lumped excitation, 15.8 eV ionisation)
and magnitudes of the right order.  It is labelled a stand-in wherever used.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Tuple

import numpy as np

# Physical constants for input generation only (CODATA 2018).
_QE = 1.602176634e-19
_ME = 9.1093837015e-31
_KB = 1.380649e-23
_M_AR = 39.948 * 1.66053906660e-27

CS_DE_EV = 1.0e-3          # DE_CS, Sec. 3.2
CS_ENTRIES = 1_000_000     # CS_RANGES: DE_CS * CS_RANGES = 1000 eV


@dataclasses.dataclass
class Discharge:
    """Parameters of one discharge (Table 1 / Table 2 names in comments)."""
    gap_m: float = 0.025                 # L
    pressure_pa: float = 10.0            # PRESSURE
    gas_temp_k: float = 350.0            # TEMPERATURE
    area_m2: float = 1.0e-4              # electrode area A
    weight: float = 7.0e4                # WEIGHT
    n_grid: int = 400                    # N_G
    steps_per_cycle: int = 4000          # N_T
    ion_subcycle: int = 20               # N_SUB
    cycle_freq_hz: float = 13.56e6       # FREQUENCY (period = one RF cycle)
    harmonics: Tuple[Tuple[float, float], ...] = ((13.56e6, 250.0),)  # (f, V)
    seed: int = 1
    eepf_bins: int = 2000                # N_EEPF
    eepf_de_ev: float = 0.05             # DE_EEPF
    ifed_bins: int = 200                 # N_IFED
    ifed_de_ev: float = 1.0              # DE_IFED
    capacity: int = 1 << 16              # MAX_N_P analogue, per species
    e_exc_ev: float = 11.5
    e_ion_ev: float = 15.8
    # surface processes (Sec. 5), (powered, grounded): ion-induced secondary
    # electron yield gamma, elastic electron reflection probability eta_e;
    # temperature of the emitted electrons (eV).  Off by default, as in the
    # paper's code.
    see_gamma: Tuple[float, float] = (0.0, 0.0)
    refl_eta: Tuple[float, float] = (0.0, 0.0)
    see_te_ev: float = 1.0
    # null-collision method (Sec. 2.1.6) instead of the direct test, per
    # species: 1 electrons, 2 ions, 3 both, 0 off
    null_collision: int = 0
    # spatio-temporal diagnostics (Sec. 3.5): time bins per RF cycle, 0 = off
    xt_bins: int = 0
    # periodic cell sort of the particle arrays (GPU locality, not in the
    # paper): every sort_every ion subcycles, 0 = off
    sort_every: int = 0

    def replace(self, **kw) -> "Discharge":
        return dataclasses.replace(self, **kw)


@dataclasses.dataclass
class Particles:
    """SoA particle state of one species (float64 on the host)."""
    x: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @staticmethod
    def empty() -> "Particles":
        z = np.zeros(0, dtype=np.float64)
        return Particles(z, z.copy(), z.copy(), z.copy())


# --------------------------------------------------------------------------
# Stand-in cross sections (NOT the Phelps fits; see module docstring).
# --------------------------------------------------------------------------
def _standin_electron(e: np.ndarray, e_exc: float, e_ion: float) -> np.ndarray:
    el = 1e-20 * (5.0 * np.exp(-e / 0.15) + 0.15
                  + 18.0 * e * e / (e * e + 100.0) / (1.0 + e / 60.0))
    de = np.maximum(e - e_exc, 0.0)
    exc = 1e-20 * 1.2 * de / (de + 8.0) * np.sqrt(30.0 / (e + 10.0))
    ion = np.zeros_like(e)
    m = e > e_ion
    ion[m] = 1.9e-17 * np.log(e[m] / e_ion) / (e[m] * e_ion)
    return np.stack([el, exc, ion])


def _standin_ion(e: np.ndarray) -> np.ndarray:
    iso = 1e-20 * (40.0 / np.sqrt(1.0 + e / 0.05) + 2.0)
    back = 1e-20 * 30.0 / (1.0 + 0.15 * np.log1p(e / 0.05))
    return np.stack([iso, back])


def standin_cross_sections(n_entries: int = CS_ENTRIES, de_ev: float = CS_DE_EV,
                           e_exc_ev: float = 11.5, e_ion_ev: float = 15.8):
    """Tabulated stand-in cross sections at energies k*de_ev, k = 0..n-1.

    Returns (sigma_e [3, n] for elastic / excitation / ionisation by LAB energy,
    sigma_i [2, n] for isotropic / backward Ar+ + Ar by COM energy), in m^2.
    """
    e = np.arange(n_entries, dtype=np.float64) * de_ev
    return (np.ascontiguousarray(_standin_electron(e, e_exc_ev, e_ion_ev)),
            np.ascontiguousarray(_standin_ion(e)))


def constant_cross_sections(n_entries: int, de_ev: float, sigma_e=(1e-19, 0.0, 0.0),
                            sigma_i=(1e-19, 0.0)):
    """Energy-independent tables (for swarm tests with known collision rates)."""
    se = np.stack([np.full(n_entries, s, dtype=np.float64) for s in sigma_e])
    si = np.stack([np.full(n_entries, s, dtype=np.float64) for s in sigma_i])
    return np.ascontiguousarray(se), np.ascontiguousarray(si)


# --------------------------------------------------------------------------
# Initial particle states.
# --------------------------------------------------------------------------
def maxwellian(n: int, gap_m: float, kt_joule: float, mass: float, rng: np.random.Generator,
               x: np.ndarray | None = None) -> Particles:
    """Uniform positions in (0, L) (unless given) and Maxwellian velocities."""
    if x is None:
        x = rng.uniform(0.0, gap_m, n)
    s = math.sqrt(kt_joule / mass)
    v = rng.normal(0.0, s, (3, n))
    return Particles(np.ascontiguousarray(x, dtype=np.float64), v[0].copy(), v[1].copy(), v[2].copy())


def _sample_profile(n: int, gap_m: float, floor: float, rng, left: Tuple[float, float],
                    right: Tuple[float, float]) -> np.ndarray:
    """Positions drawn from a flat-bulk profile that, towards each electrode,
    falls linearly to `floor` (relative) between the distances (start, end)
    (fractions of the gap) given for that side, and is `floor` closer in."""
    out = np.empty(0)
    while out.size < n:
        x = rng.uniform(0.0, 1.0, 2 * (n - out.size) + 16)
        near_left = x < 0.5
        d = np.where(near_left, x, 1.0 - x)
        start = np.where(near_left, left[0], right[0])
        end = np.where(near_left, left[1], right[1])
        p = floor + (1.0 - floor) * np.clip((d - start) / (end - start), 0.0, 1.0)
        keep = rng.uniform(0.0, 1.0, x.size) < p
        out = np.concatenate([out, x[keep]])
    return np.clip(out[:n] * gap_m, 1e-12 * gap_m, gap_m * (1.0 - 1e-12))


def sheath_fraction(d: Discharge, n_particles: int) -> float:
    """Sheath width (fraction of the gap) of a synthetic state: the width
    over which the bulk ion space charge holds the peak drive voltage,
    s = sqrt(2 eps0 V / (e n)), clamped to [0.08, 0.3]."""
    v = sum(abs(a) for _, a in d.harmonics) or 1.0
    n0 = d.weight * n_particles / (d.area_m2 * d.gap_m) if d.weight > 0 else 0.0
    if n0 <= 0:
        return 0.15
    s = math.sqrt(2 * 8.8541878128e-12 * v / (_QE * n0))
    return float(min(0.3, max(0.08, s / d.gap_m)))


def matched_electrons(n_i: int, sheath_frac: float) -> int:
    """Electron count whose bulk density equals the ion bulk density for the
    profiles of steady_shape (the sheaths hold ions but few electrons)."""
    s = sheath_frac
    return int(round(n_i * (1.0 - 1.26 * s) / (1.0 - 0.45 * s)))


def steady_shape(n_e: int, n_i: int, d: Discharge, rng: np.random.Generator,
                 te_ev: float = 2.5, sheath_frac: float | None = None,
                 ion_drift_ms: float = 8.0e3) -> Tuple[Particles, Particles]:
    """A synthetic state shaped like a converged CCP: flat bulk, electrons
    depleted in the sheaths, ions partly depleted and drifting towards the
    nearer electrode inside the sheaths (speed rising linearly to
    `ion_drift_ms` at the wall)."""
    L = d.gap_m
    if sheath_frac is None:
        sheath_frac = sheath_fraction(d, n_i)
    s = sheath_frac
    # the state matches the drive at t = 0 (V = sum of the amplitudes on the
    # powered electrode at x = 0): ions hold a symmetric, time-averaged
    # profile; the electrons fill the collapsed sheath at x = 0 and leave the
    # full sheath at x = L empty
    xi = _sample_profile(n_i, L, 0.55, rng, (0.0, s), (0.0, s))
    xe = _sample_profile(n_e, L, 0.0, rng, (0.02 * s, 0.3 * s), (s, 1.2 * s))
    e = maxwellian(n_e, L, te_ev * _QE, _ME, rng, x=xe)
    i = maxwellian(n_i, L, _KB * d.gas_temp_k, _M_AR, rng, x=xi)
    dist = np.minimum(xi, L - xi) / L
    depth = np.clip(1.0 - dist / sheath_frac, 0.0, 1.0)
    i.vx += np.where(xi < 0.5 * L, -1.0, 1.0) * ion_drift_ms * depth
    return e, i


# --------------------------------------------------------------------------
# Named workloads.
# --------------------------------------------------------------------------
def reference_discharge(**kw) -> Discharge:
    """Table 2 parameters."""
    return Discharge(**kw)


def reference_start(seed: int = 1, n0: int = 1000, capacity: int = 1 << 16):
    """Table 2 discharge seeded with n0 e- (1 eV) + n0 Ar+ (gas temperature)."""
    d = reference_discharge(seed=seed, capacity=capacity)
    rng = np.random.default_rng(seed)
    e = maxwellian(n0, d.gap_m, 1.0 * _QE, _ME, rng)
    i = maxwellian(n0, d.gap_m, _KB * d.gas_temp_k, _M_AR, rng)
    return d, e, i


def reference_steady(seed: int = 1, n: int = 500_000, capacity: int | None = None):
    """Table 2 discharge at W = 1.4e4 in a ~5e5-per-species steady-shape state."""
    cap = capacity if capacity is not None else int(n * 1.25) + 4096
    d = reference_discharge(seed=seed, weight=7.0e4 * 1.0e5 / n, capacity=cap)
    rng = np.random.default_rng(10_000 + seed)
    e, i = steady_shape(matched_electrons(n, sheath_fraction(d, n)), n, d, rng)
    return d, e, i


def dual_frequency(seed: int = 1, v_lf: float = 300.0, n: int = 2_000_000,
                   capacity: int | None = None):
    """Dual-frequency discharge: 1.356 MHz (v_lf) + 27.12 MHz (100 V), 5 Pa."""
    cap = capacity if capacity is not None else int(n * 1.25) + 4096
    density = 2.8e15
    w = density * 1e-4 * 0.025 / n
    d = Discharge(gap_m=0.025, pressure_pa=5.0, gas_temp_k=350.0, weight=w, n_grid=800,
                  steps_per_cycle=16000 * 20, ion_subcycle=20, cycle_freq_hz=1.356e6,
                  harmonics=((1.356e6, v_lf), (27.12e6, 100.0)), seed=seed, capacity=cap)
    rng = np.random.default_rng(20_000 + seed)
    e, i = steady_shape(matched_electrons(n, sheath_fraction(d, n)), n, d, rng)
    return d, e, i


def draw_discharge(rng: np.random.Generator, seed: int, n_min: float = 1e4, n_max: float = 2e6,
                   scale: float = 1.0, steps_per_cycle: int = 4000) -> Tuple[Discharge, Particles, Particles]:
    """One 13.56 MHz discharge with gap 1.5-5 cm, pressure 2-50 Pa
    (log-uniform), voltage 100-500 V, N_G 200-800 and particle count
    n_min-n_max per species (log-uniform), in a steady-shape state.  `scale`
    multiplies the particle count (small test versions)."""
    gap = rng.uniform(0.015, 0.05)
    p = math.exp(rng.uniform(math.log(2.0), math.log(50.0)))
    v0 = rng.uniform(100.0, 500.0)
    ng = int(rng.integers(200, 801))
    n = max(16, int(scale * math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
    density = 2.8e15 * (p / 10.0) ** 0.5
    w = density * 1e-4 * gap / n
    d = Discharge(gap_m=gap, pressure_pa=p, weight=w, n_grid=ng, steps_per_cycle=steps_per_cycle,
                  harmonics=((13.56e6, v0),), seed=seed, capacity=int(n * 2.0) + 4096)
    e, i = steady_shape(matched_electrons(n, sheath_fraction(d, n)), n, d, rng, te_ev=rng.uniform(2.0, 3.0))
    return d, e, i


def batch_mix(n_discharges: int = 64, seed0: int = 1000, n_min: float = 1e4, n_max: float = 2e6,
              scale: float = 1.0) -> List[Tuple[Discharge, Particles, Particles]]:
    """Independent discharges drawn by draw_discharge with seeds seed0 + k."""
    return [draw_discharge(np.random.default_rng(seed0 + k), seed0 + k, n_min, n_max, scale)
            for k in range(n_discharges)]


# The dual-frequency parameter sets of Table 3: L = 25 mm, T_g = 350 K,
# f_LF = 2 MHz, V_LF = 0..400 V; per (pressure, f_HF / V_HF) row the weight W,
# N_G and N_T (time steps per LF cycle) of each V_LF column.
DF_SWEEP_VLF = (0.0, 100.0, 200.0, 300.0, 400.0)
DF_SWEEP_ROWS = (
    # (case, p [Pa], f_HF [Hz], V_HF [V], W per V_LF, N_G per V_LF, N_T per V_LF)
    (1, 20.0, 10e6, 500.0, (1.1e5, 1.0e5, 8.2e4, 6.1e4, 4.2e4), (600, 600, 600, 600, 600),
     (31100, 31200, 31400, 31700, 33200)),
    (1, 20.0, 20e6, 250.0, (1.7e5, 1.2e5, 9.2e4, 7.8e4, 6.8e4), (600, 500, 500, 500, 500),
     (30700, 25800, 26100, 26200, 26400)),
    (2, 3.0, 30e6, 250.0, (1.6e5, 1.5e5, 1.5e5, 5.5e4, 1.9e4), (500, 500, 500, 500, 400),
     (30800, 30900, 31300, 31900, 27200)),
    (2, 3.0, 40e6, 150.0, (1.5e5, 1.3e5, 1.1e5, 8.8e4, 2.8e4), (500, 500, 500, 500, 400),
     (30700, 30900, 31100, 31300, 26300)),
)


def df_sweep(n: int = 100_000, seed0: int = 3000) -> List[Tuple[Discharge, Particles, Particles]]:
    """The 20 dual-frequency discharges of Table 3 (CASE 1: 20 Pa with 10 MHz /
    500 V or 20 MHz / 250 V; CASE 2: 3 Pa with 30 MHz / 250 V or 40 MHz /
    150 V; each with a 2 MHz component of 0-400 V), with the table's W, N_G
    and N_T, each in a steady-shape state of `n` particles per species
    (density n W / (A L)).  Seeds seed0 + k in table order."""
    out = []
    k = 0
    for _, p, f_hf, v_hf, ws, ngs, nts in DF_SWEEP_ROWS:
        for j, v_lf in enumerate(DF_SWEEP_VLF):
            d = Discharge(gap_m=0.025, pressure_pa=p, gas_temp_k=350.0, weight=ws[j], n_grid=ngs[j],
                          steps_per_cycle=nts[j], ion_subcycle=20, cycle_freq_hz=2e6,
                          harmonics=((f_hf, v_hf), (2e6, v_lf)), seed=seed0 + k, capacity=2 * n + 4096)
            rng = np.random.default_rng(seed0 + k)
            e, i = steady_shape(matched_electrons(n, sheath_fraction(d, n)), n, d, rng)
            out.append((d, e, i))
            k += 1
    return out
