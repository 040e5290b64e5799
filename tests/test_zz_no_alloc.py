"""The no-allocation entry point, edupic_fields_noalloc, through the C ABI.

It serves callers that cannot call cudaMalloc mid-run (device memory
pre-budgeted by another framework's pool, where an allocation would fail or
break the budget; plugins and real-time loops that must not touch the
allocator): it writes the densities, potential and field
of given particle positions into caller-provided device arrays and works in
a fixed array inside the library.  Its output must equal what the regular
path (edupic_load_particles + edupic_get_fields, FP64) gives, on two calls in
a row, so that the shared scratch is seen to start from zero each time.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2103_09642_gb300 import build_ext  # noqa: E402
from paper_2103_09642_gb300 import edupic as ed  # noqa: E402
from paper_2103_09642_gb300 import workloads as wl  # noqa: E402

ETOOBIG = -9
EINVAL = -1


def _lib():
    build_ext.build()
    L = ed.load_library()
    f = L.edupic_fields_noalloc
    f.argtypes = [ctypes.POINTER(ed.Params), ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    return L


def _call(L, d, e, i, step=0):
    dev = torch.device("cuda", torch.cuda.current_device())
    xe = torch.tensor(e.x, dtype=torch.float64, device=dev)
    xi = torch.tensor(i.x, dtype=torch.float64, device=dev)
    out = [torch.full((d.n_grid,), float("nan"), dtype=torch.float64, device=dev) for _ in range(4)]
    p = ed.to_params(d, 1)
    rc = L.edupic_fields_noalloc(ctypes.byref(p), step, xe.data_ptr(), e.n, xi.data_ptr(), i.n,
                                 *[o.data_ptr() for o in out], torch.cuda.current_stream().cuda_stream)
    return rc, out


def _noalloc(L, d, e, i, step=0):
    rc, out = _call(L, d, e, i, step)
    assert rc == 0, L.edupic_strerror(rc)
    return [o.cpu().numpy() for o in out]


def test_noalloc_matches_regular_path_on_two_calls():
    L = _lib()
    se, si = wl.standin_cross_sections(2000)
    for seed, n in ((5, 30_000), (6, 12_000)):
        d, e, i = wl.reference_steady(seed=seed, n=n)
        sim = ed.simulation_for([d], ed.FP64, sigma=(se, si), de_ev=wl.CS_DE_EV, particles=[(e, i)])
        ref = sim.fields(0)
        sim.close()
        n_e, n_i, phi, ef = _noalloc(L, d, e, i)
        # the same tolerances as the field-solve parity tests
        assert np.array_equal(n_e, ref["n_e"]) and np.array_equal(n_i, ref["n_i"])
        assert np.abs(phi - ref["phi"]).max() <= 1e-12 * np.abs(ref["phi"]).max()
        assert np.abs(ef - ref["efield"]).max() <= 1e-9 * np.abs(ref["efield"]).max()


def test_noalloc_rejects_grids_beyond_its_scratch():
    L = _lib()
    d = wl.reference_discharge(n_grid=2049)
    p = ed.to_params(d, 1)
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = L.edupic_fields_noalloc(ctypes.byref(p), 0, None, 0, None, 0, *([dummy.data_ptr()] * 4), None)
    assert rc == ETOOBIG
    assert b"2048" in L.edupic_strerror(rc)


def test_noalloc_two_harmonics_inside_the_cycle():
    # the boundary value is V(t) at the step's place in the cycle, summed over
    # the harmonics: with no space charge (W = 0) and step = 3 N_T + N_T / 8,
    # V = V1 cos(pi/4) + V2 cos(pi/2) = V1 / sqrt2, phi = V (1 - x/L), E = V/L
    L = _lib()
    f, V1, V2, nt = 13.56e6, 120.0, 80.0, 4000
    d = wl.reference_discharge(weight=0.0, harmonics=((f, V1), (2 * f, V2)), steps_per_cycle=nt)
    rng = np.random.default_rng(12)
    e = wl.maxwellian(2000, d.gap_m, 1.6e-19, 9.1e-31, rng)
    i = wl.maxwellian(1000, d.gap_m, 1e-21, 6.6e-26, rng)
    for _ in range(2):
        n_e, n_i, phi, ef = _noalloc(L, d, e, i, step=3 * nt + nt // 8)
        v = V1 / np.sqrt(2.0)
        x = np.arange(d.n_grid) * d.gap_m / (d.n_grid - 1)
        assert (n_e == 0).all() and (n_i == 0).all()
        assert np.abs(phi - v * (1 - x / d.gap_m)).max() <= 1e-12 * v
        assert np.abs(ef - v / d.gap_m).max() <= 1e-12 * v / d.gap_m


def test_noalloc_with_space_charge_at_an_inner_step_matches_the_oracle():
    # W > 0, two harmonics and a step that is not a multiple of N_T: the same
    # field as the oracle's (Thomas) at that step, densities to rounding
    import oracle
    L = _lib()
    f, nt = 13.56e6, 4000
    d, e, i = wl.reference_steady(seed=8, n=20_000)
    d = d.replace(harmonics=((f, 150.0), (2 * f, 60.0)), steps_per_cycle=nt)
    step = 3 * nt + 1234
    se, si = wl.standin_cross_sections(2000)
    ref = oracle.Sim(d, se, si, wl.CS_DE_EV, e, i)
    ref.step_index = step
    o = ref.prepare_fields()
    for _ in range(2):
        n_e, n_i, phi, ef = _noalloc(L, d, e, i, step=step)
        assert np.array_equal(n_e, o["n_e"])
        assert np.array_equal(n_i, o["n_i"])
        assert np.abs(phi - o["phi"]).max() <= 1e-12 * np.abs(o["phi"]).max()
        assert np.abs(ef - o["efield"]).max() <= 1e-9 * np.abs(o["efield"]).max()


def test_noalloc_rejects_positions_outside_the_gap():
    # positions outside [0, L] (or NaN) are not deposited and give EINVAL;
    # a valid call right after is unaffected
    L = _lib()
    d, e, i = wl.reference_steady(seed=9, n=4000)
    for bad in (-1e-6, d.gap_m * (1 + 1e-9), float("nan")):
        e2 = wl.Particles(e.x.copy(), e.vx, e.vy, e.vz)
        e2.x[17] = bad
        rc, _ = _call(L, d, e2, i)
        assert rc == EINVAL, rc
    se, si = wl.standin_cross_sections(2000)
    sim = ed.simulation_for([d], ed.FP64, sigma=(se, si), de_ev=wl.CS_DE_EV, particles=[(e, i)])
    ref = sim.fields(0)
    sim.close()
    n_e, n_i, phi, ef = _noalloc(L, d, e, i)
    assert np.array_equal(n_e, ref["n_e"]) and np.array_equal(n_i, ref["n_i"])
