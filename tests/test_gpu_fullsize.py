"""Parity on the paths the particle kernel takes only at large sizes.

* The block-local deposition counters are flushed to the discharge's int64
  accumulator every 64 000 particles a block processes.  With the persistent
  grid of two blocks per SM, a launch needs about 2*10^7 particles of one
  species before every block passes that point, so these tests step that
  many electrons and ions once (66 000 per block of the grid; ion subcycle
  1, so both densities are re-deposited in that step) and require the fused
  deposition to equal the fixed-point definition (Algorithm 2) of the
  stored positions exactly.
  In FP64 the whole step is also compared with the oracle.
* Event lists above 8192 entries per step are sorted in global memory
  instead of shared memory before the canonical hole fill (Algorithm 5):
  a narrow gap with hot particles absorbs more than that in one step.
"""
import numpy as np
import pytest

import oracle
from paper_2103_09642_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2103_09642_gb300 import build_ext  # noqa: E402
from paper_2103_09642_gb300 import edupic as ed  # noqa: E402

build_ext.build()

QE, ME, KB = 1.602176634e-19, 9.1093837015e-31, 1.380649e-23
MAR = 39.948 * 1.66053906660e-27
SE, SI = wl.standin_cross_sections(300_000)
DE = wl.CS_DE_EV


def _deposit_of_positions(x, d, inv_dx, precision):
    if precision == ed.FP64:
        return oracle.deposit_fixed(x, d.n_grid, inv_dx)
    return oracle.deposit_fixed_f32(x.astype(np.float32), d.n_grid, np.float32(inv_dx))


@pytest.mark.parametrize("precision", [ed.FP64, ed.FP32])
def test_one_step_at_full_size_fused_deposition_is_exact(precision):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 2 * sms * 66_000  # every block of the two-per-SM grid takes more than the 64 000-particle flush interval
    # no space charge and no drive (E = 0): the step is push, absorption,
    # collisions (stand-in cross sections) and the fused deposition
    d = wl.reference_discharge(weight=0.0, harmonics=((13.56e6, 0.0),), ion_subcycle=1,
                               capacity=n + n // 16, seed=11)
    rng = np.random.default_rng(2024)
    e = wl.maxwellian(n, d.gap_m, 3.0 * QE, ME, rng)
    i = wl.maxwellian(n, d.gap_m, 0.05 * QE, MAR, rng)
    sim = ed.simulation_for([d], precision, sigma=(SE, SI), de_ev=DE, particles=[(e, i)])
    grid = sim.push_grid()
    assert max(grid) * 65_000 < n, grid  # each block passes the flush point
    sim.step(1)
    f = sim.fields(0)
    ne, ni, step = sim.counts(0)
    assert step == 1 and ne >= n - n // 50 and ni >= n - n // 50
    inv_dx = oracle.Sim(d, SE, SI, DE).derived()["inv_dx"]
    g_e = sim.particles(0, 0)
    g_i = sim.particles(0, 1)
    # every block flushed mid-loop; the sums are still the exact definition
    assert np.array_equal(f["q_e"], _deposit_of_positions(g_e[0], d, inv_dx, precision))
    assert np.array_equal(f["q_i"], _deposit_of_positions(g_i[0], d, inv_dx, precision))
    assert int(f["q_e"].sum()) == ne * 2 ** 32 and int(f["q_i"].sum()) == ni * 2 ** 32
    c = sim.counters(0)
    assert c["push_e"] == n and c["push_i"] == n
    assert c["coll_e_ela"] > 0 and c["abs_e_pow"] + c["abs_e_gnd"] > 0
    assert ne == n - c["abs_e_pow"] - c["abs_e_gnd"] + c["created"]
    if precision == ed.FP64:
        ref = oracle.Sim(d, SE, SI, DE, e, i)
        ref.step(1)
        assert sim.counters(0) == ref.counters()
        # the oracle deposits at the start of a step (Algorithm 2): the
        # densities of its next step, which the GPU has already formed
        o = ref.prepare_fields()
        assert np.array_equal(f["q_e"], o["q_e"]) and np.array_equal(f["q_i"], o["q_i"])
        for sp, g in ((0, g_e), (1, g_i)):
            r = ref.particles(sp)
            assert g[0].size == r[0].size
            # E = 0: positions are x + v dt in both, bit for bit
            assert np.array_equal(g[0], r[0]), sp
            for k in (1, 2, 3):
                vs = max(float(np.sqrt(np.mean(r[k] ** 2))), 1.0)
                assert np.abs(g[k] - r[k]).max() <= 1e-12 * vs, (sp, k)
    sim.close()


def test_more_than_8192_absorptions_in_a_step_fp64():
    # a 1 mm gap with hot particles: >8192 electrons and >8192 ions leave in
    # the first step, so both hole lists take the global-memory sort; the
    # compaction order must still be the canonical one of the oracle
    d = wl.reference_discharge(gap_m=1e-3, n_grid=101, weight=0.0, harmonics=((13.56e6, 0.0),),
                               capacity=1 << 22, seed=12)
    rng = np.random.default_rng(2025)
    e = wl.maxwellian(400_000, d.gap_m, 30.0 * QE, ME, rng)
    i = wl.maxwellian(2_000_000, d.gap_m, 200.0 * QE, MAR, rng)
    sim = ed.simulation_for([d], ed.FP64, sigma=(SE, SI), de_ev=DE, particles=[(e, i)])
    ref = oracle.Sim(d, SE, SI, DE, e, i)
    for k in range(3):
        sim.step(1)
        ref.step(1)
        c = ref.counters()
        if k == 0:
            assert c["abs_e_pow"] + c["abs_e_gnd"] > 8192
            assert c["abs_i_pow"] + c["abs_i_gnd"] > 8192
        assert sim.counters(0) == c, f"step {k}"
        for sp in (0, 1):
            g = sim.particles(0, sp)
            r = ref.particles(sp)
            assert g[0].size == r[0].size, (k, sp)
            assert np.abs(g[0] - r[0]).max() <= 1e-12 * d.gap_m, (k, sp)
            for comp in (1, 2, 3):
                vs = max(float(np.sqrt(np.mean(r[comp] ** 2))), 1.0)
                assert np.abs(g[comp] - r[comp]).max() <= 1e-12 * vs, (k, sp, comp)
    sim.close()
