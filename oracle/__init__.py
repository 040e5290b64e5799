"""CPU oracle of the eduPIC PIC/MCC particle loop (arXiv 2103.09642).

TEST INFRASTRUCTURE ONLY: only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
never calls it, and it shares no code with the CUDA path.

The arithmetic lives in ``edupic_oracle.c`` (plain single-threaded FP64 C,
compiled with ``gcc -O2 -ffp-contract=off``); this module compiles it on
demand and exposes it through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "edupic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libedupic_oracle.so")
_lock = threading.Lock()
_lib = None

MAX_HARM = 4
N_COUNTERS = 19
XT_NAMES = ("pot", "efield", "ne", "ni", "je", "ji", "powere", "poweri", "meanee", "meanei", "ioniz")
COUNTER_NAMES = ("abs_e_pow", "abs_e_gnd", "abs_i_pow", "abs_i_gnd", "coll_e_ela", "coll_e_exc",
                 "coll_e_ion", "coll_i_iso", "coll_i_back", "subthreshold", "created", "dropped",
                 "push_e", "push_i", "reflected", "emitted_pow", "emitted_gnd",
                 "null_tested", "null_over")


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [
        ("gap_m", ctypes.c_double), ("pressure_pa", ctypes.c_double), ("gas_temp_k", ctypes.c_double),
        ("area_m2", ctypes.c_double), ("weight", ctypes.c_double),
        ("n_grid", ctypes.c_int), ("steps_per_cycle", ctypes.c_int), ("ion_subcycle", ctypes.c_int),
        ("cycle_freq_hz", ctypes.c_double), ("n_harm", ctypes.c_int),
        ("harm_freq_hz", ctypes.c_double * MAX_HARM), ("harm_volt_v", ctypes.c_double * MAX_HARM),
        ("seed", ctypes.c_uint64), ("eepf_bins", ctypes.c_int), ("eepf_de_ev", ctypes.c_double),
        ("ifed_bins", ctypes.c_int), ("ifed_de_ev", ctypes.c_double), ("capacity", ctypes.c_int64),
        ("e_exc_ev", ctypes.c_double), ("e_ion_ev", ctypes.c_double),
        ("see_gamma", ctypes.c_double * 2), ("refl_eta", ctypes.c_double * 2), ("see_te_ev", ctypes.c_double),
        ("null_collision", ctypes.c_int), ("xt_bins", ctypes.c_int), ("sort_every", ctypes.c_int),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_Q = ctypes.POINTER(ctypes.c_int64)
_U32 = ctypes.POINTER(ctypes.c_uint32)


def lib():
    """Load (building first if needed) the oracle library."""
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_philox4x32_10.argtypes = [_U32, _U32, _U32]
            L.orc_u53.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            L.orc_u53.restype = ctypes.c_double
            L.orc_u24.argtypes = [ctypes.c_uint32]
            L.orc_u24.restype = ctypes.c_float
            L.orc_deposit_paper.argtypes = [_D, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D]
            L.orc_deposit_fixed.argtypes = [_D, ctypes.c_int64, ctypes.c_int, ctypes.c_double, _Q]
            L.orc_deposit_fixed_f32.argtypes = [_F, ctypes.c_int64, ctypes.c_int, ctypes.c_float, _Q]
            L.orc_density_from_fixed.argtypes = [_Q, ctypes.c_int, ctypes.c_double, _D]
            L.orc_poisson.argtypes = [_D, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, _D]
            L.orc_create.argtypes = [ctypes.POINTER(_Params)]
            L.orc_create.restype = ctypes.c_void_p
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_set_cross_sections.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_double, _D]
            L.orc_load_particles.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, _D, _D, _D, _D]
            L.orc_count.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_count.restype = ctypes.c_int64
            L.orc_get_particles.argtypes = [ctypes.c_void_p, ctypes.c_int, _D, _D, _D, _D]
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
            L.orc_prepare_fields.argtypes = [ctypes.c_void_p]
            L.orc_get_step.argtypes = [ctypes.c_void_p]
            L.orc_get_step.restype = ctypes.c_int64
            L.orc_set_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
            L.orc_get_fields.argtypes = [ctypes.c_void_p, _D, _D, _D, _D, _Q, _Q]
            L.orc_get_counters.argtypes = [ctypes.c_void_p, _Q]
            L.orc_get_diagnostics.argtypes = [ctypes.c_void_p, _D, _D, _D, _Q, _Q, _Q]
            L.orc_get_diagnostics.restype = ctypes.c_int64
            L.orc_get_power.argtypes = [ctypes.c_void_p, _D]
            L.orc_get_power.restype = ctypes.c_int64
            L.orc_eepf_normalise.argtypes = [_Q, ctypes.c_int, ctypes.c_double, _D, _D]
            L.orc_ifed_normalise.argtypes = [_Q, ctypes.c_int, ctypes.c_double, _D, _D]
            L.orc_get_derived.argtypes = [ctypes.c_void_p, _D]
            L.orc_set_bias.argtypes = [ctypes.c_void_p, ctypes.c_double]
            L.orc_seed.argtypes = [ctypes.c_void_p, ctypes.c_int64]
            L.orc_seed.restype = ctypes.c_int
            L.orc_get_xt.argtypes = [ctypes.c_void_p, ctypes.c_int, _D]
            L.orc_get_xt.restype = ctypes.c_int
            L.orc_set_bias.restype = None
            L.orc_unit_collide_electron.argtypes = [ctypes.c_void_p, ctypes.c_int, _D, ctypes.c_double,
                                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]
            L.orc_unit_collide_ion.argtypes = [ctypes.c_void_p, ctypes.c_int, _D, _D, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double]
            L.orc_select_process.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double]
            L.orc_test_uniform_f32.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
            L.orc_test_uniform_f32.restype = ctypes.c_float
            L.orc_select_process_f32.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_float]
            L.orc_draw_u24.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int]
            L.orc_draw_u24.restype = ctypes.c_float
            _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- unit calls
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return out


def u53(a: int, b: int) -> float:
    return lib().orc_u53(a, b)


def u24(a: int) -> float:
    return lib().orc_u24(a)


def draw_u24(seed: int, slot: int, step: int, species: int, block: int, word: int) -> float:
    """FP32 per-particle uniform (24 bits) of Philox block `block`, word 0 or 1."""
    return lib().orc_draw_u24(seed, slot, step, species, block, word)


def test_uniform_f32(seed: int, slot: int, step: int, species: int) -> float:
    """Collision-test uniform of the FP32 particle mode."""
    return lib().orc_test_uniform_f32(seed, slot, step, species)


def deposit_paper(x, n_grid: int, inv_dx: float, factor_w: float) -> np.ndarray:
    x = _f64(x)
    out = np.zeros(n_grid)
    lib().orc_deposit_paper(_p(x, ctypes.c_double), x.size, n_grid, inv_dx, factor_w, _p(out, ctypes.c_double))
    return out


def deposit_fixed(x, n_grid: int, inv_dx: float) -> np.ndarray:
    x = _f64(x)
    q = np.zeros(n_grid, dtype=np.int64)
    lib().orc_deposit_fixed(_p(x, ctypes.c_double), x.size, n_grid, inv_dx, _p(q, ctypes.c_int64))
    return q


def deposit_fixed_f32(x, n_grid: int, inv_dx_f32: float) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    q = np.zeros(n_grid, dtype=np.int64)
    lib().orc_deposit_fixed_f32(_p(x, ctypes.c_float), x.size, n_grid, ctypes.c_float(inv_dx_f32),
                                _p(q, ctypes.c_int64))
    return q


def density_from_fixed(q, factor_w: float) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.int64)
    out = np.zeros(q.size)
    lib().orc_density_from_fixed(_p(q, ctypes.c_int64), q.size, factor_w, _p(out, ctypes.c_double))
    return out


def poisson(rho, dx: float, v_left: float):
    rho = _f64(rho)
    phi = np.zeros(rho.size)
    ef = np.zeros(rho.size)
    lib().orc_poisson(_p(rho, ctypes.c_double), rho.size, dx, v_left, _p(phi, ctypes.c_double),
                      _p(ef, ctypes.c_double))
    return phi, ef


def eepf_normalise(h, de: float):
    h = np.ascontiguousarray(h, dtype=np.int64)
    e = np.zeros(h.size)
    f = np.zeros(h.size)
    lib().orc_eepf_normalise(_p(h, ctypes.c_int64), h.size, de, _p(e, ctypes.c_double), _p(f, ctypes.c_double))
    return e, f


def ifed_normalise(h, de: float):
    h = np.ascontiguousarray(h, dtype=np.int64)
    e = np.zeros(h.size)
    f = np.zeros(h.size)
    lib().orc_ifed_normalise(_p(h, ctypes.c_int64), h.size, de, _p(e, ctypes.c_double), _p(f, ctypes.c_double))
    return e, f


# ---------------------------------------------------------------- simulation
def _params(d) -> _Params:
    p = _Params()
    p.gap_m = d.gap_m
    p.pressure_pa = d.pressure_pa
    p.gas_temp_k = d.gas_temp_k
    p.area_m2 = d.area_m2
    p.weight = d.weight
    p.n_grid = d.n_grid
    p.steps_per_cycle = d.steps_per_cycle
    p.ion_subcycle = d.ion_subcycle
    p.cycle_freq_hz = d.cycle_freq_hz
    p.n_harm = len(d.harmonics)
    for k, (f, v) in enumerate(d.harmonics):
        p.harm_freq_hz[k] = f
        p.harm_volt_v[k] = v
    p.seed = d.seed
    p.eepf_bins = d.eepf_bins
    p.eepf_de_ev = d.eepf_de_ev
    p.ifed_bins = d.ifed_bins
    p.ifed_de_ev = d.ifed_de_ev
    p.capacity = d.capacity
    p.e_exc_ev = d.e_exc_ev
    p.e_ion_ev = d.e_ion_ev
    for k in range(2):
        p.see_gamma[k] = d.see_gamma[k]
        p.refl_eta[k] = d.refl_eta[k]
    p.see_te_ev = d.see_te_ev
    p.null_collision = int(d.null_collision)
    p.xt_bins = int(d.xt_bins)
    p.sort_every = int(d.sort_every)
    return p


class Sim:
    """One discharge stepped by the oracle."""

    def __init__(self, d, sigma_e, sigma_i, de_ev: float, electrons=None, ions=None):
        self.d = d
        self._pp = _params(d)
        self._h = lib().orc_create(ctypes.byref(self._pp))
        if not self._h:
            raise ValueError("oracle: invalid parameters")
        self.set_cross_sections(0, sigma_e, de_ev)
        self.set_cross_sections(1, sigma_i, de_ev)
        if electrons is not None:
            self.load(0, electrons)
        if ions is not None:
            self.load(1, ions)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_cross_sections(self, species: int, sigma, de_ev: float):
        s = _f64(sigma)
        if lib().orc_set_cross_sections(self._h, species, s.shape[0], s.shape[1], de_ev, _p(s, ctypes.c_double)):
            raise ValueError("oracle: bad cross-section table")

    def load(self, species: int, parts):
        a = [_f64(getattr(parts, k)) for k in ("x", "vx", "vy", "vz")]
        if lib().orc_load_particles(self._h, species, a[0].size, *[_p(v, ctypes.c_double) for v in a]):
            raise ValueError("oracle: bad particle load")

    def seed(self, n: int) -> None:
        """init(N_INIT) of Algorithm 1: n e- and n Ar+ at rest, uniform in the gap."""
        if lib().orc_seed(self._h, ctypes.c_int64(int(n))):
            raise ValueError("oracle: bad seed count")

    def step(self, n: int, measure: bool = False):
        rc = lib().orc_step(self._h, n, 1 if measure else 0)
        if rc == -1:
            raise RuntimeError("oracle: cross sections missing")
        return rc

    def count(self, species: int) -> int:
        return lib().orc_count(self._h, species)

    def particles(self, species: int):
        n = self.count(species)
        a = [np.zeros(n) for _ in range(4)]
        lib().orc_get_particles(self._h, species, *[_p(v, ctypes.c_double) for v in a])
        return a

    @property
    def step_index(self) -> int:
        return lib().orc_get_step(self._h)

    @step_index.setter
    def step_index(self, s: int):
        lib().orc_set_step(self._h, s)

    def prepare_fields(self):
        """Densities and field of the current step, without advancing it."""
        lib().orc_prepare_fields(self._h)
        return self.fields()

    def fields(self):
        ng = self.d.n_grid
        out = [np.zeros(ng) for _ in range(4)] + [np.zeros(ng, dtype=np.int64) for _ in range(2)]
        lib().orc_get_fields(self._h, *[_p(v, ctypes.c_double) for v in out[:4]],
                             *[_p(v, ctypes.c_int64) for v in out[4:]])
        return dict(zip(("n_e", "n_i", "phi", "efield", "q_e", "q_i"), out))

    def counters(self) -> dict:
        c = np.zeros(N_COUNTERS, dtype=np.int64)
        lib().orc_get_counters(self._h, _p(c, ctypes.c_int64))
        return {k: int(c[i]) for i, k in enumerate(COUNTER_NAMES)}

    def diagnostics(self) -> dict:
        d = self.d
        ng = d.n_grid
        ne, ni, phi = np.zeros(ng), np.zeros(ng), np.zeros(ng)
        eepf = np.zeros(d.eepf_bins, dtype=np.int64)
        ip = np.zeros(d.ifed_bins, dtype=np.int64)
        ig = np.zeros(d.ifed_bins, dtype=np.int64)
        m = lib().orc_get_diagnostics(self._h, *[_p(v, ctypes.c_double) for v in (ne, ni, phi)],
                                      *[_p(v, ctypes.c_int64) for v in (eepf, ip, ig)])
        return dict(measured_steps=int(m), n_e=ne, n_i=ni, phi=phi, eepf_counts=eepf,
                    ifed_pow_counts=ip, ifed_gnd_counts=ig)

    def power(self) -> dict:
        """Power absorption densities of e- and Ar+ (W/m^3), space and time
        averaged over the measured steps."""
        out = np.zeros(2)
        m = lib().orc_get_power(self._h, _p(out, ctypes.c_double))
        return dict(measured_steps=int(m), electrons=float(out[0]), ions=float(out[1]))

    def xt(self, quantity: int) -> np.ndarray:
        """xt map [n_grid, xt_bins] of quantity (XT_NAMES order)."""
        out = np.zeros((self.d.n_grid, self.d.xt_bins))
        if lib().orc_get_xt(self._h, int(quantity), _p(out, ctypes.c_double)) != 0:
            raise ValueError("no xt diagnostics")
        return out

    def set_bias(self, v_bias: float) -> None:
        lib().orc_set_bias(self._h, ctypes.c_double(v_bias))

    def derived(self) -> dict:
        out = np.zeros(16)
        lib().orc_get_derived(self._h, _p(out, ctypes.c_double))
        names = ("dx", "inv_dx", "dt_e", "dt_i", "factor_w", "factor_e", "factor_i", "n_gas", "ar_mass",
                 "mu_e", "mu_arar", "sigma_th_ar", "nu_star_e", "nu_star_i", "p_star_e", "p_star_i")
        return dict(zip(names, out.tolist()))

    # unit collisions with explicit random numbers
    def collide_electron(self, k: int, v, u_proc, u_chi, u_eta, u_opal):
        vv = _f64(v).copy()
        vej = np.zeros(3)
        proc = lib().orc_unit_collide_electron(self._h, k, _p(vv, ctypes.c_double), u_proc, u_chi, u_eta, u_opal,
                                               _p(vej, ctypes.c_double))
        return proc, vv, vej

    def collide_ion(self, k: int, v, va, u_proc, u_chi, u_eta):
        vv = _f64(v).copy()
        a = _f64(va).copy()
        proc = lib().orc_unit_collide_ion(self._h, k, _p(vv, ctypes.c_double), _p(a, ctypes.c_double), u_proc,
                                          u_chi, u_eta)
        return proc, vv

    def select_process(self, species: int, k: int, u: float, f32: bool = False) -> int:
        if f32:
            return lib().orc_select_process_f32(self._h, species, k, ctypes.c_float(u))
        return lib().orc_select_process(self._h, species, k, u)
