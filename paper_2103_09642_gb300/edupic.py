"""Thin Python binding of the C ABI in ``include/edupic.h``.

Argument marshalling only: device memory (one arena per simulation) and the
stream come from PyTorch; every step of the particle loop runs in the CUDA
library ``_build/libedupic_gb300.so``.  There is no CPU fallback: if the
library is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, List, Optional, Sequence

import numpy as np

from .workloads import Discharge, Particles

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libedupic_gb300.so")

FP64, FP32 = 0, 1
ELECTRONS, IONS = 0, 1
MAX_HARMONICS = 4
N_COUNTERS = 19
XT_NAMES = ("pot", "efield", "ne", "ni", "je", "ji", "powere", "poweri", "meanee", "meanei", "ioniz")
STEP_EVENTS = 65536
BOUND_BUCKETS = 2048
COUNTER_NAMES = ("abs_e_pow", "abs_e_gnd", "abs_i_pow", "abs_i_gnd", "coll_e_ela", "coll_e_exc",
                 "coll_e_ion", "coll_i_iso", "coll_i_back", "subthreshold", "created", "dropped",
                 "push_e", "push_i", "reflected", "emitted_pow", "emitted_gnd",
                 "null_tested", "null_over")
STATUS = {0: "ok", -1: "EINVAL", -2: "ENOMEM", -3: "ECAPACITY", -4: "ECUDA", -5: "ESTATE", -6: "ENAN",
          -7: "EIO", -8: "ETIMEOUT", -9: "ETOOBIG", -10: "ESTABILITY"}
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3
REQ_STATES = {REQ_QUEUED: "queued", REQ_RUNNING: "running", REQ_DONE: "done", REQ_FAILED: "failed"}


class EdupicError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)} ({status})")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("gap_m", ctypes.c_double), ("pressure_pa", ctypes.c_double), ("gas_temp_k", ctypes.c_double),
        ("area_m2", ctypes.c_double), ("weight", ctypes.c_double),
        ("n_grid", ctypes.c_int32), ("steps_per_cycle", ctypes.c_int32), ("ion_subcycle", ctypes.c_int32),
        ("n_harmonics", ctypes.c_int32), ("cycle_freq_hz", ctypes.c_double),
        ("harm_freq_hz", ctypes.c_double * MAX_HARMONICS), ("harm_volt_v", ctypes.c_double * MAX_HARMONICS),
        ("seed", ctypes.c_uint64), ("eepf_bins", ctypes.c_int32), ("ifed_bins", ctypes.c_int32),
        ("eepf_de_ev", ctypes.c_double), ("ifed_de_ev", ctypes.c_double),
        ("capacity_e", ctypes.c_int64), ("capacity_i", ctypes.c_int64),
        ("e_exc_ev", ctypes.c_double), ("e_ion_ev", ctypes.c_double),
        ("cs_entries", ctypes.c_int32), ("sort_every", ctypes.c_int32),
        ("see_gamma", ctypes.c_double * 2), ("refl_eta", ctypes.c_double * 2), ("see_te_ev", ctypes.c_double),
        ("null_collision", ctypes.c_int32), ("xt_bins", ctypes.c_int32),
    ]


def to_params(d: Discharge, cs_entries: int) -> Params:
    p = Params()
    p.gap_m, p.pressure_pa, p.gas_temp_k, p.area_m2, p.weight = (d.gap_m, d.pressure_pa, d.gas_temp_k,
                                                                  d.area_m2, d.weight)
    p.n_grid, p.steps_per_cycle, p.ion_subcycle = d.n_grid, d.steps_per_cycle, d.ion_subcycle
    p.n_harmonics = len(d.harmonics)
    p.cycle_freq_hz = d.cycle_freq_hz
    for k, (f, v) in enumerate(d.harmonics):
        p.harm_freq_hz[k] = f
        p.harm_volt_v[k] = v
    p.seed = d.seed
    p.eepf_bins, p.ifed_bins, p.eepf_de_ev, p.ifed_de_ev = d.eepf_bins, d.ifed_bins, d.eepf_de_ev, d.ifed_de_ev
    p.capacity_e = p.capacity_i = d.capacity
    p.e_exc_ev, p.e_ion_ev = d.e_exc_ev, d.e_ion_ev
    p.cs_entries = cs_entries
    for k in range(2):
        p.see_gamma[k], p.refl_eta[k] = d.see_gamma[k], d.refl_eta[k]
    p.see_te_ev = d.see_te_ev
    p.null_collision = int(d.null_collision)
    p.xt_bins = int(d.xt_bins)
    p.sort_every = int(d.sort_every)
    return p


class Accuracy(ctypes.Structure):
    _fields_ = [("debye_ratio", ctypes.c_double), ("wpe_dt", ctypes.c_double), ("pcoll_max_e", ctypes.c_double),
                ("pcoll_max_i", ctypes.c_double), ("cfl_max_ev_e", ctypes.c_double), ("cfl_max_ev_i", ctypes.c_double),
                ("te_ev", ctypes.c_double), ("ne_max", ctypes.c_double), ("failed", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("max_grid", ctypes.c_int32), ("max_eepf_bins", ctypes.c_int32),
                ("ion_subcycle", ctypes.c_int32), ("cs_entries", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("slot", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("steps_target", ctypes.c_int64), ("steps_done", ctypes.c_int64),
                ("n_e", ctypes.c_int64), ("n_i", ctypes.c_int64), ("bytes", ctypes.c_int64),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("now", ctypes.c_double), ("steps_run", ctypes.c_int64), ("heap_bytes", ctypes.c_int64),
                ("heap_used", ctypes.c_int64), ("running", ctypes.c_int32), ("queued", ctypes.c_int32)]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_Q = ctypes.POINTER(ctypes.c_int64)
_VP = ctypes.c_void_p


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA extension not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER(Params)
    sig = {
        "edupic_arena_bytes": ([ctypes.c_int, P, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
        "edupic_create": ([ctypes.c_int, P, ctypes.c_int, _VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)]),
        "edupic_destroy": ([_VP]),
        "edupic_set_cross_sections": ([_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D]),
        "edupic_load_particles": ([_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _D, _D, _D, _D]),
        "edupic_step": ([_VP, ctypes.c_int64, ctypes.c_int]),
        "edupic_run_cycles": ([_VP, ctypes.c_int, ctypes.c_int]),
        "edupic_synchronize": ([_VP]),
        "edupic_selftest_wait_expiry": ([_VP, ctypes.c_int, ctypes.c_int64]),
        "edupic_set_graphs": ([_VP, ctypes.c_int]),
        "edupic_profile_steps": ([_VP, ctypes.c_int64, ctypes.c_int, _D, _Q]),
        "edupic_set_push_grid": ([_VP, ctypes.c_int, ctypes.c_int]),
        "edupic_get_push_grid": ([_VP, ctypes.POINTER(ctypes.c_int)]),
        "edupic_set_push_shape": ([_VP, ctypes.c_int, ctypes.c_int]),
        "edupic_get_push_shape": ([_VP, ctypes.POINTER(ctypes.c_int)]),
        "edupic_electron_bound_table": ([ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D,
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "edupic_describe_push_shape": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "edupic_autotune": ([_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _D]),
        "edupic_check_accuracy": ([_VP, ctypes.c_int, ctypes.POINTER(Accuracy)]),
        "edupic_get_power": ([_VP, ctypes.c_int, _D]),
        "edupic_set_bias": ([_VP, ctypes.c_int, ctypes.c_double]),
        "edupic_seed": ([_VP, ctypes.c_int, ctypes.c_int64]),
        "edupic_get_graphs": ([_VP, ctypes.POINTER(ctypes.c_int)]),
        "edupic_get_xt": ([_VP, ctypes.c_int, ctypes.c_int, _D]),
        "edupic_get_bias": ([_VP, ctypes.c_int, _D]),
        "edupic_self_bias_step": ([_VP, ctypes.c_int64, ctypes.c_int, _D, _D]),
        "edupic_get_counts": ([_VP, ctypes.c_int, _Q, _Q, _Q]),
        "edupic_get_particles": ([_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _D, _D, _D, _D, _Q]),
        "edupic_get_fields": ([_VP, ctypes.c_int, _D, _D, _D, _D, _Q, _Q]),
        "edupic_get_diagnostics": ([_VP, ctypes.c_int, _D, _D, _D, _Q, _Q, _Q, _Q]),
        "edupic_get_eepf": ([_VP, ctypes.c_int, _D, _D]),
        "edupic_get_ifed": ([_VP, ctypes.c_int, _D, _D, _D]),
        "edupic_get_counters": ([_VP, ctypes.c_int, _Q]),
        "edupic_reset_diagnostics": ([_VP, ctypes.c_int]),
        "edupic_save_state": ([_VP, ctypes.c_int, ctypes.c_char_p]),
        "edupic_load_state": ([_VP, ctypes.c_int, ctypes.c_char_p]),
    }
    SC = ctypes.POINTER(ServerConfig)
    D4 = _D * 4
    sig.update({
        "edupic_server_arena_bytes": ([SC, ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
        "edupic_server_create": ([SC, ctypes.c_int, _VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)]),
        "edupic_server_destroy": ([_VP]),
        "edupic_server_set_cross_sections": ([_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D]),
        "edupic_server_request_bytes": ([_VP, P, ctypes.POINTER(ctypes.c_size_t)]),
        "edupic_server_submit": ([_VP, P, ctypes.c_int, ctypes.c_int64, D4, ctypes.c_int64, D4,
                                  ctypes.POINTER(ctypes.c_uint64)]),
        "edupic_server_advance": ([_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "edupic_server_info": ([_VP, ctypes.c_uint64, ctypes.POINTER(RequestInfo)]),
        "edupic_server_result": ([_VP, ctypes.c_uint64, _D, _D, _D, _Q, _Q, _Q, _Q, _Q]),
        "edupic_server_release": ([_VP, ctypes.c_uint64]),
        "edupic_server_stats": ([_VP, ctypes.POINTER(ServerStats)]),
    })
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.edupic_strerror.argtypes = [ctypes.c_int]
    L.edupic_strerror.restype = ctypes.c_char_p
    _lib = L
    return L


def _ck(rc: int, what: str):
    if rc != 0:
        raise EdupicError(rc, what)


def _ptr(a: np.ndarray, ct=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class Simulation:
    """n discharges stepped together on one CUDA stream.

    ``precision`` is FP64 or FP32 (particles, push and collisions; the field
    solve and diagnostics stay FP64).  Device memory is a single torch uint8
    tensor (the arena); ``stream`` is a ``torch.cuda.Stream`` (default: a new
    stream on the current device).
    """

    def __init__(self, discharges: Sequence[Discharge], precision: int = FP64, stream=None,
                 cs_entries: int = 1_000_000, device: Optional[str] = None):
        import torch

        self._torch = torch
        self.L = load_library()
        self.discharges = list(discharges)
        self.nd = len(self.discharges)
        self.precision = precision
        arr = (Params * self.nd)(*[to_params(d, cs_entries) for d in self.discharges])
        self._params = arr
        nbytes = ctypes.c_size_t(0)
        _ck(self.L.edupic_arena_bytes(self.nd, arr, precision, ctypes.byref(nbytes)), "arena_bytes")
        self.arena_bytes = int(nbytes.value)
        dev = torch.device(device) if device else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self.arena = torch.empty(self.arena_bytes, dtype=torch.uint8, device=dev)
        h = _VP()
        with torch.cuda.device(dev):
            _ck(self.L.edupic_create(self.nd, arr, precision, ctypes.c_void_p(self.arena.data_ptr()),
                                     self.arena_bytes, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
                "create")
        self._h = h

    # ------------------------------------------------------------- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            self.L.edupic_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------- set-up
    def set_cross_sections(self, species: int, sigma: np.ndarray, de_ev: float):
        s = np.ascontiguousarray(sigma, dtype=np.float64)
        _ck(self.L.edupic_set_cross_sections(self._h, species, s.shape[0], s.shape[1], de_ev, _ptr(s)),
            "set_cross_sections")

    def load(self, d: int, species: int, parts: Particles):
        a = [np.ascontiguousarray(getattr(parts, k), dtype=np.float64) for k in ("x", "vx", "vy", "vz")]
        _ck(self.L.edupic_load_particles(self._h, d, species, a[0].size, *[_ptr(v) for v in a]), "load_particles")

    # ------------------------------------------------------------- stepping
    def step(self, n: int, measure: bool = False):
        _ck(self.L.edupic_step(self._h, int(n), 1 if measure else 0), "step")

    def run_cycles(self, n: int, measure: bool = False):
        _ck(self.L.edupic_run_cycles(self._h, int(n), 1 if measure else 0), "run_cycles")

    def synchronize(self):
        _ck(self.L.edupic_synchronize(self._h), "synchronize")

    def selftest_wait_expiry(self, d: int, limit_ns: int) -> int:
        """Status of a bounded wait on a barrier nothing arms (EDUPIC_ETIMEOUT)."""
        return int(self.L.edupic_selftest_wait_expiry(self._h, d, int(limit_ns)))

    def profile_steps(self, n: int, measure: bool = False):
        """Per-kernel device time (ms) and launch counts over n steps:
        (electron push, ion push, finalize)."""
        ms = np.zeros(3)
        cnt = np.zeros(3, dtype=np.int64)
        _ck(self.L.edupic_profile_steps(self._h, int(n), 1 if measure else 0, _ptr(ms), _ptr(cnt, ctypes.c_int64)),
            "profile_steps")
        return ms, cnt

    def set_graphs(self, enable: bool):
        _ck(self.L.edupic_set_graphs(self._h, 1 if enable else 0), "set_graphs")

    def graphs(self) -> bool:
        v = ctypes.c_int(0)
        _ck(self.L.edupic_get_graphs(self._h, ctypes.byref(v)), "get_graphs")
        return bool(v.value)

    def set_push_grid(self, species: int, blocks: int):
        _ck(self.L.edupic_set_push_grid(self._h, species, int(blocks)), "set_push_grid")

    def push_grid(self):
        g = (ctypes.c_int * 2)()
        _ck(self.L.edupic_get_push_grid(self._h, g), "get_push_grid")
        return g[0], g[1]

    def set_push_shape(self, species: int, shape: int):
        _ck(self.L.edupic_set_push_shape(self._h, species, int(shape)), "set_push_shape")

    def push_shape(self):
        g = (ctypes.c_int * 2)()
        _ck(self.L.edupic_get_push_shape(self._h, g), "get_push_shape")
        return g[0], g[1]

    def describe_push_shape(self, shape: int) -> dict:
        return describe_push_shape(self.precision, shape)

    def autotune(self, subcycles: int = 5, measure: bool = False):
        """Pick graph replay or kernel-by-kernel stepping by timing (advances
        the simulation); returns (grid in use, trial ms per step)."""
        g = (ctypes.c_int * 2)()
        ms = ctypes.c_double(0)
        _ck(self.L.edupic_autotune(self._h, int(subcycles), 1 if measure else 0, g, ctypes.byref(ms)), "autotune")
        return g[0], ms.value

    # ------------------------------------------------------------- read-back
    def counts(self, d: int = 0):
        ne, ni, st = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _ck(self.L.edupic_get_counts(self._h, d, ctypes.byref(ne), ctypes.byref(ni), ctypes.byref(st)), "counts")
        return ne.value, ni.value, st.value

    def particles(self, d: int, species: int) -> List[np.ndarray]:
        n = self.counts(d)[species]
        a = [np.zeros(n) for _ in range(4)]
        out = ctypes.c_int64()
        _ck(self.L.edupic_get_particles(self._h, d, species, n, *[_ptr(v) for v in a], ctypes.byref(out)),
            "get_particles")
        return a

    def fields(self, d: int = 0) -> dict:
        ng = self.discharges[d].n_grid
        f = [np.zeros(ng) for _ in range(4)]
        q = [np.zeros(ng, dtype=np.int64) for _ in range(2)]
        _ck(self.L.edupic_get_fields(self._h, d, *[_ptr(v) for v in f], *[_ptr(v, ctypes.c_int64) for v in q]),
            "get_fields")
        return dict(zip(("n_e", "n_i", "phi", "efield", "q_e", "q_i"), f + q))

    def diagnostics(self, d: int = 0) -> dict:
        dd = self.discharges[d]
        ng = dd.n_grid
        avg = [np.zeros(ng) for _ in range(3)]
        e = np.zeros(dd.eepf_bins, dtype=np.int64)
        ip = np.zeros(dd.ifed_bins, dtype=np.int64)
        ig = np.zeros(dd.ifed_bins, dtype=np.int64)
        m = ctypes.c_int64()
        _ck(self.L.edupic_get_diagnostics(self._h, d, *[_ptr(v) for v in avg],
                                          *[_ptr(v, ctypes.c_int64) for v in (e, ip, ig)], ctypes.byref(m)),
            "get_diagnostics")
        return dict(measured_steps=m.value, n_e=avg[0], n_i=avg[1], phi=avg[2], eepf_counts=e,
                    ifed_pow_counts=ip, ifed_gnd_counts=ig)

    def eepf(self, d: int = 0):
        n = self.discharges[d].eepf_bins
        e, f = np.zeros(n), np.zeros(n)
        _ck(self.L.edupic_get_eepf(self._h, d, _ptr(e), _ptr(f)), "get_eepf")
        return e, f

    def ifed(self, d: int = 0):
        n = self.discharges[d].ifed_bins
        e, fp, fg = np.zeros(n), np.zeros(n), np.zeros(n)
        _ck(self.L.edupic_get_ifed(self._h, d, _ptr(e), _ptr(fp), _ptr(fg)), "get_ifed")
        return e, fp, fg

    def counters(self, d: int = 0) -> dict:
        c = np.zeros(N_COUNTERS, dtype=np.int64)
        _ck(self.L.edupic_get_counters(self._h, d, _ptr(c, ctypes.c_int64)), "get_counters")
        return {k: int(c[i]) for i, k in enumerate(COUNTER_NAMES)}

    def power(self, d: int = 0) -> dict:
        """Power absorption densities of e- and Ar+ (W/m^3), space and time
        averaged over the measured steps (Sec. 3.5)."""
        out = np.zeros(2)
        _ck(self.L.edupic_get_power(self._h, d, _ptr(out)), "get_power")
        return {"electrons": float(out[0]), "ions": float(out[1])}

    def xt(self, d: int, quantity) -> np.ndarray:
        """Spatio-temporal map [n_grid, xt_bins] (Sec. 3.5) of a quantity
        named in XT_NAMES (or its index)."""
        q = XT_NAMES.index(quantity) if isinstance(quantity, str) else int(quantity)
        dd = self.discharges[d]
        out = np.zeros((dd.n_grid, dd.xt_bins))
        _ck(self.L.edupic_get_xt(self._h, d, q, _ptr(out)), "get_xt")
        return out

    def seed(self, d: int, n_init: int) -> None:
        """init(N_INIT) of Algorithm 1: n_init e- and n_init Ar+ at rest,
        uniform in the gap (replaces discharge d's particles)."""
        _ck(self.L.edupic_seed(self._h, d, int(n_init)), "seed")

    def set_bias(self, d: int, v_bias: float) -> None:
        """DC self-bias voltage added at the powered electrode (Sec. 5)."""
        _ck(self.L.edupic_set_bias(self._h, d, float(v_bias)), "set_bias")

    def bias(self, d: int = 0) -> float:
        out = np.zeros(1)
        _ck(self.L.edupic_get_bias(self._h, d, _ptr(out)), "get_bias")
        return float(out[0])

    def self_bias_step(self, n_steps: int, gain_v, measure: bool = False) -> np.ndarray:
        """One self-bias iteration (Sec. 5) over n_steps time steps; gain_v
        (volts) per discharge or one value for all.  Returns the biases."""
        g = np.ascontiguousarray(np.broadcast_to(np.asarray(gain_v, dtype=np.float64), (len(self.discharges),)))
        out = np.zeros(len(self.discharges))
        _ck(self.L.edupic_self_bias_step(self._h, int(n_steps), 1 if measure else 0, _ptr(g), _ptr(out)),
            "self_bias_step")
        return out

    def check_accuracy(self, d: int = 0) -> dict:
        """Accuracy and stability conditions of Sec. 2.2 from the measured
        diagnostics; 'ok' is False when condition 1, 2 or 3 fails."""
        a = Accuracy()
        rc = self.L.edupic_check_accuracy(self._h, d, ctypes.byref(a))
        if rc not in (0, -10):
            _ck(rc, "check_accuracy")
        out = {k: getattr(a, k) for k, _ in Accuracy._fields_ if k != "reserved"}
        out["ok"] = rc == 0
        return out

    def reset_diagnostics(self, d: int = 0):
        _ck(self.L.edupic_reset_diagnostics(self._h, d), "reset_diagnostics")

    def save_state(self, d: int, path: str):
        _ck(self.L.edupic_save_state(self._h, d, path.encode()), "save_state")

    def load_state(self, d: int, path: str):
        _ck(self.L.edupic_load_state(self._h, d, path.encode()), "load_state")


PUSH_SHAPES = 4


def describe_push_shape(precision: int, shape: int) -> dict:
    """Threads per block, ring stages and targeted blocks per SM of a launch shape."""
    L = load_library()
    t, s, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _ck(L.edupic_describe_push_shape(precision, shape, ctypes.byref(t), ctypes.byref(s), ctypes.byref(m)),
        "describe_push_shape")
    return dict(threads=t.value, stages=s.value, min_blocks=m.value)


def electron_bound_table(precision: int, sigma_sum, de_ev: float):
    """The electrons' collision bound per v^2 bucket (edupic_electron_bound_table):
    (table of BOUND_BUCKETS values, first bucket, number of buckets)."""
    L = load_library()
    sig = np.ascontiguousarray(sigma_sum, dtype=np.float64)
    out = np.zeros(BOUND_BUCKETS)
    base, nb = ctypes.c_int(), ctypes.c_int()
    _ck(L.edupic_electron_bound_table(precision, int(sig.size), float(de_ev), _ptr(sig), _ptr(out),
                                      ctypes.byref(base), ctypes.byref(nb)), "electron_bound_table")
    return out, base.value, nb.value


def simulation_for(discharges: Iterable, precision: int = FP64, sigma=None, de_ev: float = 1e-3,
                   particles=None, **kw) -> Simulation:
    """Create a simulation, set cross sections and load (e, i) particle pairs."""
    ds = list(discharges)
    n_entries = sigma[0].shape[1] if sigma is not None else 1
    sim = Simulation(ds, precision=precision, cs_entries=max(n_entries, 1), **kw)
    if sigma is not None:
        sim.set_cross_sections(ELECTRONS, sigma[0], de_ev)
        sim.set_cross_sections(IONS, sigma[1], de_ev)
    if particles is not None:
        for d, (e, i) in enumerate(particles):
            sim.load(d, ELECTRONS, e)
            sim.load(d, IONS, i)
    return sim


def server_arena_bytes(heap_bytes: int, max_slots: int = 64, max_grid: int = 800, max_eepf_bins: int = 2000,
                       ion_subcycle: int = 20, cs_entries: int = 1_000_000, precision: int = FP32) -> int:
    """Arena bytes of a server with `heap_bytes` of request memory."""
    L = load_library()
    cfg = ServerConfig(max_slots, max_grid, max_eepf_bins, ion_subcycle, cs_entries, 0)
    b = ctypes.c_size_t(0)
    _ck(L.edupic_server_arena_bytes(ctypes.byref(cfg), precision, int(heap_bytes), ctypes.byref(b)), "server_arena")
    return int(b.value)


class Server:
    """Continuous-batching request server (edupic_server_* of the C ABI).

    ``budget_bytes`` of device memory (one torch uint8 tensor) hold the
    shared region and the request heap; requests are admitted while a slot
    and heap memory are free.  ``advance(k)`` retires finished requests,
    admits queued ones and enqueues k ion subcycles for all running ones.
    """

    def __init__(self, budget_bytes: int, max_slots: int = 64, max_grid: int = 800, max_eepf_bins: int = 2000,
                 ion_subcycle: int = 20, cs_entries: int = 1_000_000, precision: int = FP32, stream=None,
                 device: Optional[str] = None):
        import torch

        self._torch = torch
        self.L = load_library()
        self.precision = precision
        self.cs_entries = cs_entries
        cfg = ServerConfig(max_slots, max_grid, max_eepf_bins, ion_subcycle, cs_entries, 0)
        self._cfg = cfg
        need = ctypes.c_size_t(0)
        _ck(self.L.edupic_server_arena_bytes(ctypes.byref(cfg), precision, 0, ctypes.byref(need)), "server_arena")
        if budget_bytes < need.value:
            raise EdupicError(-2, f"server budget below the shared region ({need.value} B)")
        dev = torch.device(device) if device else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self.arena = torch.empty(int(budget_bytes), dtype=torch.uint8, device=dev)
        h = _VP()
        with torch.cuda.device(dev):
            _ck(self.L.edupic_server_create(ctypes.byref(cfg), precision, ctypes.c_void_p(self.arena.data_ptr()),
                                            int(budget_bytes), ctypes.c_void_p(self.stream.cuda_stream),
                                            ctypes.byref(h)), "server_create")
        self._h = h
        self._req = {}

    def close(self):
        if getattr(self, "_h", None):
            self.L.edupic_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_cross_sections(self, species: int, sigma: np.ndarray, de_ev: float):
        s = np.ascontiguousarray(sigma, dtype=np.float64)
        _ck(self.L.edupic_server_set_cross_sections(self._h, species, s.shape[0], s.shape[1], de_ev, _ptr(s)),
            "server_set_cross_sections")

    def request_bytes(self, d: Discharge) -> int:
        p = to_params(d, self.cs_entries)
        b = ctypes.c_size_t(0)
        _ck(self.L.edupic_server_request_bytes(self._h, ctypes.byref(p), ctypes.byref(b)), "request_bytes")
        return int(b.value)

    def submit(self, d: Discharge, e: Particles, i: Particles, n_cycles: int) -> int:
        p = to_params(d, self.cs_entries)
        arrs = []
        ptrs = []
        for parts in (e, i):
            a = [np.ascontiguousarray(getattr(parts, k), dtype=np.float64) for k in ("x", "vx", "vy", "vz")]
            arrs.append(a)
            ptrs.append((_D * 4)(*[_ptr(v) for v in a]))
        t = ctypes.c_uint64(0)
        _ck(self.L.edupic_server_submit(self._h, ctypes.byref(p), int(n_cycles), arrs[0][0].size, ptrs[0],
                                        arrs[1][0].size, ptrs[1], ctypes.byref(t)), "server_submit")
        self._req[int(t.value)] = d
        return int(t.value)

    def advance(self, n_subcycles: int = 1):
        r, q = ctypes.c_int(0), ctypes.c_int(0)
        _ck(self.L.edupic_server_advance(self._h, int(n_subcycles), ctypes.byref(r), ctypes.byref(q)),
            "server_advance")
        return r.value, q.value

    def info(self, ticket: int) -> dict:
        x = RequestInfo()
        _ck(self.L.edupic_server_info(self._h, ticket, ctypes.byref(x)), "server_info")
        return {k: getattr(x, k) for k, _ in RequestInfo._fields_ if k != "reserved"}

    def result(self, ticket: int) -> dict:
        d = self._req[ticket]
        ng = d.n_grid
        avg = [np.zeros(ng) for _ in range(3)]
        e = np.zeros(d.eepf_bins, dtype=np.int64)
        ip = np.zeros(d.ifed_bins, dtype=np.int64)
        ig = np.zeros(d.ifed_bins, dtype=np.int64)
        c = np.zeros(N_COUNTERS, dtype=np.int64)
        m = ctypes.c_int64()
        _ck(self.L.edupic_server_result(self._h, ticket, *[_ptr(v) for v in avg],
                                        *[_ptr(v, ctypes.c_int64) for v in (e, ip, ig, c)], ctypes.byref(m)),
            "server_result")
        return dict(measured_steps=m.value, n_e=avg[0], n_i=avg[1], phi=avg[2], eepf_counts=e,
                    ifed_pow_counts=ip, ifed_gnd_counts=ig,
                    counters={k: int(c[j]) for j, k in enumerate(COUNTER_NAMES)})

    def release(self, ticket: int):
        _ck(self.L.edupic_server_release(self._h, ticket), "server_release")
        self._req.pop(ticket, None)

    def stats(self) -> dict:
        x = ServerStats()
        _ck(self.L.edupic_server_stats(self._h, ctypes.byref(x)), "server_stats")
        return {k: getattr(x, k) for k, _ in ServerStats._fields_}
