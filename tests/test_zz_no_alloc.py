"""The no-allocation entry point, edupic_fields_noalloc, through the C ABI.

It serves callers that cannot call cudaMalloc mid-run (device memory
pre-budgeted by another framework's pool, plugins and real-time loops, work
issued during stream capture): it writes the densities, potential and field
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


def _lib():
    build_ext.build()
    L = ed.load_library()
    f = L.edupic_fields_noalloc
    f.argtypes = [ctypes.POINTER(ed.Params), ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    return L


def _noalloc(L, d, e, i):
    dev = torch.device("cuda", torch.cuda.current_device())
    xe = torch.tensor(e.x, dtype=torch.float64, device=dev)
    xi = torch.tensor(i.x, dtype=torch.float64, device=dev)
    out = [torch.full((d.n_grid,), float("nan"), dtype=torch.float64, device=dev) for _ in range(4)]
    p = ed.to_params(d, 1)
    rc = L.edupic_fields_noalloc(ctypes.byref(p), 0, xe.data_ptr(), e.n, xi.data_ptr(), i.n,
                                 *[o.data_ptr() for o in out], torch.cuda.current_stream().cuda_stream)
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
