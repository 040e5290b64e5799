"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/edupic.h declares; parameter checks run on the host."""
import ctypes
import os
import re

import pytest

from paper_2103_09642_gb300 import build_ext
from paper_2103_09642_gb300 import edupic as ed
from paper_2103_09642_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(edupic_[a-z0-9_]+)\s*\(", txt,
                                flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return ed.load_library()


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("edupic_create", "edupic_step", "edupic_get_fields", "edupic_save_state"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_host_side_checks(lib):
    assert lib.edupic_strerror(0) == b"ok"
    assert lib.edupic_strerror(-3).startswith(b"particle")
    d = wl.reference_discharge()
    good = ed.to_params(d, 1000)
    out = ctypes.c_size_t(0)
    arr = (ed.Params * 1)(good)
    assert lib.edupic_arena_bytes(1, arr, ed.FP32, ctypes.byref(out)) == 0
    b32 = out.value
    assert lib.edupic_arena_bytes(1, arr, ed.FP64, ctypes.byref(out)) == 0
    assert out.value > b32 > 0
    for field, bad in (("n_grid", 2), ("n_grid", 5000), ("ion_subcycle", 7), ("capacity_e", 0),
                       ("eepf_bins", 4096), ("weight", -1.0), ("gap_m", 0.0)):
        p = ed.to_params(d, 1000)
        setattr(p, field, bad)
        assert lib.edupic_arena_bytes(1, (ed.Params * 1)(p), ed.FP32, ctypes.byref(out)) == -1, field
    p = ed.to_params(d.replace(harmonics=((13.56e6 * 1.5, 100.0),)), 1000)   # not a multiple
    assert lib.edupic_arena_bytes(1, (ed.Params * 1)(p), ed.FP32, ctypes.byref(out)) == -1
    assert lib.edupic_arena_bytes(0, arr, ed.FP32, ctypes.byref(out)) == -1
    assert lib.edupic_arena_bytes(1, arr, 7, ctypes.byref(out)) == -1
    # surface process probabilities lie in [0, 1]; emission adds its event lists
    for kw in ({"see_gamma": (1.5, 0.0)}, {"refl_eta": (0.0, -0.1)}, {"see_te_ev": -1.0},
               {"refl_eta": (float("nan"), 0.0)}):
        p = ed.to_params(d.replace(**kw), 1000)
        assert lib.edupic_arena_bytes(1, (ed.Params * 1)(p), ed.FP32, ctypes.byref(out)) == -1, kw
    assert lib.edupic_arena_bytes(1, arr, ed.FP64, ctypes.byref(out)) == 0
    plain = out.value
    p = ed.to_params(d.replace(refl_eta=(1.0, 1.0)), 1000)
    assert lib.edupic_arena_bytes(1, (ed.Params * 1)(p), ed.FP64, ctypes.byref(out)) == 0 and out.value == plain
    p = ed.to_params(d.replace(see_gamma=(0.1, 0.0)), 1000)
    assert lib.edupic_arena_bytes(1, (ed.Params * 1)(p), ed.FP64, ctypes.byref(out)) == 0 and out.value > plain
    # null-collision mask 0..3; xt bins dividing N_T; the xt block only when asked for
    for kw in ({"null_collision": 4}, {"null_collision": -1}, {"xt_bins": 3}, {"xt_bins": -1},
               {"xt_bins": 8200, "n_grid": 2048, "steps_per_cycle": 16400}):  # N_G N_XT > 2^24
        p = ed.to_params(d.replace(**kw), 1000)
        assert lib.edupic_arena_bytes(1, (ed.Params * 1)(p), ed.FP32, ctypes.byref(out)) == -1, kw
    p = ed.to_params(d.replace(null_collision=3), 1000)
    assert lib.edupic_arena_bytes(1, (ed.Params * 1)(p), ed.FP64, ctypes.byref(out)) == 0 and out.value == plain
    p = ed.to_params(d.replace(xt_bins=200), 1000)
    assert lib.edupic_arena_bytes(1, (ed.Params * 1)(p), ed.FP64, ctypes.byref(out)) == 0
    assert out.value - plain >= (9 * d.n_grid * 200 + 4 * 200) * 8


def test_create_rejects_small_or_misaligned_arena(lib):
    d = wl.reference_discharge()
    arr = (ed.Params * 1)(ed.to_params(d, 1000))
    out = ctypes.c_size_t(0)
    assert lib.edupic_arena_bytes(1, arr, ed.FP32, ctypes.byref(out)) == 0
    h = ctypes.c_void_p()
    # never dereferenced: both are rejected before any device call
    assert lib.edupic_create(1, arr, ed.FP32, ctypes.c_void_p(256), out.value - 1, None, ctypes.byref(h)) == -2
    assert lib.edupic_create(1, arr, ed.FP32, ctypes.c_void_p(257), out.value, None, ctypes.byref(h)) == -1


def test_df_sweep_workload_is_valid(lib):
    """The 20 dual-frequency discharges of Table 3 pass the host checks: N_T a
    multiple of N_SUB, every drive frequency a multiple of the 2 MHz cycle."""
    mix = wl.df_sweep(n=500)
    assert len(mix) == 20
    ds = [m[0] for m in mix]
    assert {(d.pressure_pa, d.harmonics[0]) for d in ds} == {
        (20.0, (10e6, 500.0)), (20.0, (20e6, 250.0)), (3.0, (30e6, 250.0)), (3.0, (40e6, 150.0))}
    assert sorted({d.harmonics[1][1] for d in ds}) == [0.0, 100.0, 200.0, 300.0, 400.0]
    out = ctypes.c_size_t(0)
    arr = (ed.Params * 20)(*[ed.to_params(d, 1000) for d in ds])
    assert lib.edupic_arena_bytes(20, arr, ed.FP32, ctypes.byref(out)) == 0 and out.value > 0
    for d, e, i in mix:
        assert d.steps_per_cycle % d.ion_subcycle == 0
        assert e.n > 0 and i.n == 500 and (e.x > 0).all() and (e.x < d.gap_m).all()
