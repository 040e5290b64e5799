"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a published
known-answer vector, the paper's worked example, a closed-form solution, a
conservation law, a textbook average or brute force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2103_09642_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
QE, ME, EPS0, KB = 1.602176634e-19, 9.1093837015e-31, 8.8541878128e-12, 1.380649e-23
MAR = 39.948 * 1.66053906660e-27


def _quiet(**kw):
    """A discharge with no drive and no space charge (W = 0): E = 0 exactly."""
    base = dict(weight=0.0, harmonics=((0.0, 0.0),), n_grid=101, capacity=1 << 17)
    base.update(kw)
    return wl.Discharge(**base)


def _tables(n=200_000, de=1e-3, **kw):
    return wl.constant_cross_sections(n, de, **kw)


# ------------------------------------------------------------------ RNG
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(o) for o in out] == v[6:10]


def test_uniform_ranges():
    assert oracle.u53(0, 0) == 0.0
    assert oracle.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert oracle.u53(0x80000000, 0) == 0.5
    assert oracle.u24(0) == 0.0
    assert oracle.u24(0xFFFFFFFF) == np.float32(1.0 - 2.0 ** -24)
    assert oracle.u24(0x80000000) == 0.5


# ------------------------------------------------------------------ derived quantities (Table 1/2)
def test_reference_discharge_derived():
    d = wl.reference_discharge()
    se, si = _tables(1000)
    s = oracle.Sim(d, se, si, 1e-3)
    dv = s.derived()
    assert dv["dx"] == pytest.approx(0.025 / 399, rel=1e-15)
    assert dv["dt_e"] == pytest.approx(1.0 / (13.56e6 * 4000), rel=1e-15)
    assert dv["dt_i"] == pytest.approx(20.0 / (13.56e6 * 4000), rel=1e-15)
    assert dv["n_gas"] == pytest.approx(10.0 / (KB * 350.0), rel=1e-15)
    # printed magnitudes: dx = 6.266e-5 m, dt_e = 1.8437e-11 s, n = 2.069e21 m^-3
    assert abs(dv["dx"] - 6.266e-5) < 1e-8
    assert abs(dv["dt_e"] - 1.8437e-11) < 1e-15
    assert abs(dv["n_gas"] - 2.069e21) < 1e18


# ------------------------------------------------------------------ deposition (Sec. 2.1.1, Alg. 2)
def test_weight_density_worked_example():
    g = {}
    for l in open(os.path.join(GOLDEN, "weight_density_example.txt")):
        if l.strip() and l[0] != "#":
            k, v = l.split()
            g[k] = float(v)
    n, L, A, W = int(g["n_particles"]), g["gap_m"], g["area_m2"], g["weight"]
    ng = 251
    dx = L / (ng - 1)
    x = (np.arange(n) + 0.5) * (L / n)
    dens = oracle.deposit_paper(x, ng, 1.0 / dx, W / (A * dx))
    vol = np.full(ng, A * dx)
    vol[0] = vol[-1] = A * dx / 2
    mean = (dens * vol).sum() / (A * L)
    assert mean == pytest.approx(g["mean_density_m3"], rel=1e-12)


def test_deposit_single_particle_brute_force():
    ng, L = 11, 1.0
    dx = L / (ng - 1)
    for x in (0.0, 0.05, 0.37, 0.5, 0.999, 1.0):
        dens = oracle.deposit_paper([x], ng, 1.0 / dx, 1.0)
        p = min(int(x / dx), ng - 2)
        w1 = (p + 1) - x / dx
        expect = np.zeros(ng)
        expect[p] += w1
        expect[p + 1] += 1 - w1
        expect[0] *= 2
        expect[-1] *= 2
        assert np.allclose(dens, expect, atol=1e-15), x


def test_deposit_total_weight_and_fixed_point():
    rng = np.random.default_rng(3)
    ng, L, W, A = 400, 0.025, 7e4, 1e-4
    dx = L / (ng - 1)
    x = rng.uniform(0, L, 20_000)
    x[:3] = [0.0, L, L * 0.5]
    fw = W / (A * dx)
    dens = oracle.deposit_paper(x, ng, 1.0 / dx, fw)
    vol = np.full(ng, A * dx)
    vol[0] = vol[-1] = A * dx / 2
    assert (dens * vol).sum() == pytest.approx(W * x.size, rel=1e-12)
    q = oracle.deposit_fixed(x, ng, 1.0 / dx)
    assert int(q.sum()) == x.size * 2 ** 32          # exact: each particle is 2^32 units
    assert (q >= 0).all()
    dens_q = oracle.density_from_fixed(q, fw)
    # fixed-point rounding is at most 1/2 unit of 2^-32 per particle and point
    cnt = np.bincount(np.minimum((x / dx).astype(int), ng - 2), minlength=ng)
    per_point = cnt + np.concatenate([[0], cnt[:-1]])
    bound = fw * (per_point + 1) * 2.0 ** -33 * 2 + 1e-6
    assert (np.abs(dens_q - dens) <= bound).all()


def test_deposit_fixed_f32_matches_f64_on_exact_positions():
    ng, L = 64, 1.0
    dx = L / (ng - 1)
    x = (np.arange(1, 500) / 512.0).astype(np.float32)  # exactly representable
    q32 = oracle.deposit_fixed_f32(x, ng, np.float32(1.0 / dx))
    assert int(q32.sum()) == x.size * 2 ** 32
    q64 = oracle.deposit_fixed(x.astype(np.float64), ng, 1.0 / dx)
    # the same cell for every particle, splits within FP32 rounding
    assert np.abs(q32 - q64).max() < 2 ** 32 * 1e-5 * 8


# ------------------------------------------------------------------ Poisson (Sec. 2.1.2, Alg. 3)
@pytest.mark.parametrize("ng", [3, 7, 400, 801])
def test_poisson_uniform_charge_parabola(ng):
    L, V, rho0 = 0.025, 250.0, 3e-4
    dx = L / (ng - 1)
    x = np.arange(ng) * dx
    phi, ef = oracle.poisson(np.full(ng, rho0), dx, V)
    exact = V * (1 - x / L) + rho0 * x * (L - x) / (2 * EPS0)
    scale = np.abs(exact).max()
    assert np.abs(phi - exact).max() <= 1e-12 * scale
    e_exact = V / L - rho0 * (L - 2 * x) / (2 * EPS0)   # E = -dphi/dx, exact also at the electrodes
    assert np.abs(ef - e_exact).max() <= 1e-10 * np.abs(e_exact).max()


def test_poisson_satisfies_discrete_equation():
    rng = np.random.default_rng(5)
    ng, L, V = 400, 0.025, -117.0
    dx = L / (ng - 1)
    rho = rng.normal(0, 1e-4, ng)
    phi, ef = oracle.poisson(rho, dx, V)
    assert phi[0] == V and phi[-1] == 0.0
    lhs = (-phi[:-2] + 2 * phi[1:-1] - phi[2:]) / dx ** 2
    assert np.abs(lhs - rho[1:-1] / EPS0).max() <= 1e-9 * np.abs(rho / EPS0).max()
    assert np.allclose(ef[1:-1], (phi[:-2] - phi[2:]) / (2 * dx), rtol=0, atol=1e-12 * np.abs(ef).max())
    assert ef[0] == pytest.approx((phi[0] - phi[1]) / dx - rho[0] * dx / (2 * EPS0), rel=1e-14)


# ------------------------------------------------------------------ leapfrog (Sec. 2.1.4, Alg. 4)
def test_leapfrog_uniform_field_closed_form():
    V = 0.02  # E = 0.8 V/m: electrons move ~2 mm in 1e4 steps
    d = _quiet(harmonics=((0.0, V),), gap_m=0.025)
    se, si = _tables(1000, sigma_e=(0, 0, 0), sigma_i=(0, 0))
    rng = np.random.default_rng(7)
    n = 64
    x0 = rng.uniform(0.010, 0.015, n)
    v0 = rng.uniform(-2e3, 2e3, n)
    e = wl.Particles(x0.copy(), v0.copy(), np.zeros(n), np.zeros(n))
    i = wl.Particles(x0.copy(), (v0 / 50).copy(), np.zeros(n), np.zeros(n))
    s = oracle.Sim(d, se, si, 1e-3, e, i)
    dv = s.derived()
    nsteps = 10_000
    s.step(nsteps)
    E = V / d.gap_m
    a_e = -QE * E / ME
    dt = dv["dt_e"]
    x, vx, _, _ = s.particles(0)
    k = nsteps
    xe = x0 + k * v0 * dt + a_e * dt * dt * k * (k + 1) / 2
    ve = v0 + k * a_e * dt
    assert s.count(0) == n
    assert np.abs(x - xe).max() <= 1e-12 * np.abs(xe).max()
    assert np.abs(vx - ve).max() <= 1e-12 * np.abs(ve).max()
    # ions: pushed every N_SUB-th step with dt_i
    a_i = QE * E / MAR
    dti = dv["dt_i"]
    ki = nsteps // d.ion_subcycle
    xi, vxi, _, _ = s.particles(1)
    xie = x0 + ki * (v0 / 50) * dti + a_i * dti * dti * ki * (ki + 1) / 2
    assert np.abs(xi - xie).max() <= 1e-12 * np.abs(xie).max()
    vie = (v0 / 50) + ki * a_i * dti
    assert np.abs(vxi - vie).max() <= 1e-12 * np.abs(vie).max()


# ------------------------------------------------------------------ boundaries (Sec. 2.1.5, Alg. 5)
def test_absorption_and_canonical_compaction():
    d = _quiet(gap_m=1.0, n_grid=11)
    se, si = _tables(1000, sigma_e=(0, 0, 0), sigma_i=(0, 0))
    s = oracle.Sim(d, se, si, 1e-3)
    dt = s.derived()["dt_e"]
    n = 10
    x = np.full(n, 0.5)
    vx = np.zeros(n)
    # slots 1 and 8 leave through x < 0 and x > L; slot 9 (tail) also leaves
    x[1], vx[1] = 1e-9, -1e3 / dt * 1e-6
    x[8], vx[8] = 1 - 1e-9, 1e3 / dt * 1e-6
    x[9], vx[9] = 1 - 1e-9, 1e3 / dt * 1e-6
    x += np.arange(n) * 1e-3 * (vx == 0)
    s.load(0, wl.Particles(x, vx, np.arange(n, dtype=float), np.zeros(n)))
    s.load(1, wl.Particles.empty())
    s.step(1)
    c = s.counters()
    assert c["abs_e_pow"] == 1 and c["abs_e_gnd"] == 2
    xs, _, vy, _ = s.particles(0)
    # N' = 7: hole 1 is filled by the first tail survivor (slot 7)
    assert list(vy) == [0, 7, 2, 3, 4, 5, 6]


# ------------------------------------------------------------------ collisions (Sec. 2.1.6, Alg. 6)
def _unit_sim(se=None, si=None, n=200_000, de=1e-3):
    d = wl.reference_discharge()
    if se is None:
        se, si = wl.standin_cross_sections(n, de)
    return oracle.Sim(d, se, si, de)


def _com_parts(v1, v2, m1, m2):
    w = (m1 * v1 + m2 * v2) / (m1 + m2)
    return w, v1 - v2


def test_process_selection_partition():
    se, si = wl.standin_cross_sections(100_000, 1e-3)
    s = _unit_sim(se, si)
    k = 50_000  # 50 eV: all three processes open
    u = (np.arange(100_000) + 0.5) / 100_000
    picks = np.array([s.select_process(0, k, float(x)) for x in u])
    frac = np.bincount(picks, minlength=3) / u.size
    assert np.allclose(frac, se[:, k] / se[:, k].sum(), atol=2e-5)
    picks_i = np.array([s.select_process(1, 3000, float(x)) for x in u])
    assert np.allclose(np.bincount(picks_i, minlength=2) / u.size, si[:, 3000] / si[:, 3000].sum(), atol=2e-5)


def test_elastic_electron_conservation_and_angle():
    se, si = _tables(100_000, sigma_e=(1e-19, 0, 0))
    s = _unit_sim(se, si)
    rng = np.random.default_rng(11)
    mu = ME * MAR / (ME + MAR)
    loss = []
    for _ in range(4000):
        v = rng.normal(0, 6e5, 3)
        uc, ue = rng.random(), rng.random()
        proc, v1, _ = s.collide_electron(100, v, 0.3, uc, ue, 0.5)
        assert proc == 0
        v2p = (ME * v - ME * v1) / MAR                   # atom recoil from momentum conservation
        ke0 = 0.5 * ME * v @ v
        ke1 = 0.5 * ME * v1 @ v1 + 0.5 * MAR * v2p @ v2p
        assert ke1 == pytest.approx(ke0, rel=1e-10)
        w, g = _com_parts(v, np.zeros(3), ME, MAR)
        gp = (v1 - w) * (ME + MAR) / MAR
        assert np.linalg.norm(gp) == pytest.approx(np.linalg.norm(g), rel=1e-12)
        cos_chi = gp @ g / (np.linalg.norm(gp) * np.linalg.norm(g))
        assert cos_chi == pytest.approx(1 - 2 * uc, abs=1e-10)
        loss.append((ke0 - 0.5 * ME * v1 @ v1) / ke0)
    # textbook: mean fractional energy loss for isotropic scattering on a
    # target at rest is 2 m M / (m + M)^2
    expect = 2 * ME * MAR / (ME + MAR) ** 2
    assert np.mean(loss) == pytest.approx(expect, rel=0.06)
    assert mu > 0


def test_isotropy_of_deflection():
    se, si = _tables(100_000, sigma_e=(1e-19, 0, 0))
    s = _unit_sim(se, si)
    rng = np.random.default_rng(12)
    v = np.array([3e5, -2e5, 4e5])
    dirs = []
    for _ in range(3000):
        _, v1, _ = s.collide_electron(100, v, 0.1, rng.random(), rng.random(), 0.5)
        w = ME * v / (ME + MAR)
        dirs.append((v1 - w) / np.linalg.norm(v1 - w))
    dirs = np.array(dirs)
    # isotropic unit vectors: each Cartesian component is uniform on [-1, 1]
    from scipy import stats
    for c in range(3):
        assert stats.kstest(dirs[:, c], "uniform", args=(-1, 2)).pvalue > 1e-3


def test_excitation_energy_loss():
    se, si = _tables(100_000, sigma_e=(0, 1e-19, 0))
    s = _unit_sim(se, si)
    rng = np.random.default_rng(13)
    mu = ME * MAR / (ME + MAR)
    for _ in range(500):
        v = rng.normal(0, 1.6e6, 3)
        eps_c = 0.5 * mu * (v @ v) / QE
        proc, v1, _ = s.collide_electron(100, v, 0.5, rng.random(), rng.random(), 0.5)
        w, g = _com_parts(v, np.zeros(3), ME, MAR)
        gp = (v1 - w) * (ME + MAR) / MAR
        if eps_c > 11.5:
            assert proc == 1
            assert 0.5 * mu * (gp @ gp) / QE == pytest.approx(eps_c - 11.5, rel=1e-9, abs=1e-9)
        else:  # below threshold: executed as elastic
            assert proc == 0
            assert np.linalg.norm(gp) == pytest.approx(np.linalg.norm(g), rel=1e-12)


def test_ionization_energy_sharing():
    se, si = _tables(100_000, sigma_e=(0, 0, 1e-19))
    s = _unit_sim(se, si)
    rng = np.random.default_rng(14)
    mu = ME * MAR / (ME + MAR)
    eps0 = 60.0
    vmag = math.sqrt(2 * eps0 * QE / mu)
    ee = []
    for _ in range(3000):
        d = rng.normal(size=3)
        v = vmag * d / np.linalg.norm(d)
        uo = rng.random()
        proc, v1, vej = s.collide_electron(100, v, 0.5, 0.3, rng.random(), uo)
        assert proc == 2
        w, g = _com_parts(v, np.zeros(3), ME, MAR)
        gp = (v1 - w) * (ME + MAR) / MAR
        e_s = 0.5 * mu * (gp @ gp) / QE
        e_e = 0.5 * ME * (vej @ vej) / QE
        avail = 0.5 * mu * (v @ v) / QE - 15.8
        assert e_s + e_e == pytest.approx(avail, rel=1e-10)
        # angles: cos(chi) = sqrt(eps / (eps - eps_ion)) for both electrons
        gh = g / np.linalg.norm(g)
        assert gp @ gh / np.linalg.norm(gp) == pytest.approx(math.sqrt(e_s / avail), abs=1e-9)
        assert vej @ gh / np.linalg.norm(vej) == pytest.approx(math.sqrt(e_e / avail), abs=1e-9)
        # azimuths differ by pi: the perpendicular parts are antiparallel
        ps = gp - (gp @ gh) * gh
        pe = vej - (vej @ gh) * gh
        if np.linalg.norm(ps) > 1e-6 * np.linalg.norm(gp) and np.linalg.norm(pe) > 1e-6 * np.linalg.norm(vej):
            assert ps @ pe / (np.linalg.norm(ps) * np.linalg.norm(pe)) == pytest.approx(-1.0, abs=1e-9)
        ee.append(e_e)
    # Opal distribution: F(e) = atan(e / w) / atan(avail / (2 w)) on [0, avail / 2]
    from scipy import stats
    avail = 0.5 * mu * vmag ** 2 / QE - 15.8
    cdf = lambda e: np.arctan(np.asarray(e) / 10.0) / math.atan(avail / 20.0)
    assert max(ee) <= avail / 2 + 1e-9
    assert stats.kstest(ee, cdf).pvalue > 1e-3


def test_ion_backward_gives_partner_velocity_and_isotropic_conserves():
    se, si = _tables(100_000, sigma_i=(0.0, 1e-19))
    s = _unit_sim(se, si)
    rng = np.random.default_rng(15)
    for _ in range(200):
        v = rng.normal(0, 3e3, 3)
        va = rng.normal(0, 300, 3)
        proc, v1 = s.collide_ion(10, v, va, 0.5, rng.random(), rng.random())
        assert proc == 1
        assert np.abs(v1 - va).max() <= 1e-12 * np.abs(v).max()
    se, si = _tables(100_000, sigma_i=(1e-19, 0.0))
    s = _unit_sim(se, si)
    for _ in range(200):
        v = rng.normal(0, 3e3, 3)
        va = rng.normal(0, 300, 3)
        proc, v1 = s.collide_ion(10, v, va, 0.5, rng.random(), rng.random())
        assert proc == 0
        v2p = v + va - v1                                  # equal masses: momentum
        assert v1 @ v1 + v2p @ v2p == pytest.approx(v @ v + va @ va, rel=1e-10)


def test_electron_collision_rate_constant_nu():
    # constant sigma, field off, mono-energetic: P = 1 - exp(-n sigma v dt) per step
    n, steps = 40_000, 4
    d = _quiet(gap_m=0.025, n_grid=51, capacity=1 << 17)
    sig = 2e-18
    se, si = _tables(100_000, sigma_e=(sig, 0, 0), sigma_i=(0, 0))
    s = oracle.Sim(d, se, si, 1e-3)
    rng = np.random.default_rng(16)
    eps = 1.0
    v = math.sqrt(2 * eps * QE / ME)
    dirs = rng.normal(size=(3, n))
    dirs /= np.linalg.norm(dirs, axis=0)
    e = wl.Particles(rng.uniform(0.010, 0.015, n), v * dirs[0], v * dirs[1], v * dirs[2])
    s.load(0, e)
    s.load(1, wl.Particles.empty())
    s.step(steps)
    hits = s.counters()["coll_e_ela"]
    dv = s.derived()
    p = 1 - math.exp(-dv["n_gas"] * sig * v * dv["dt_e"])
    mean, sd = n * steps * p, math.sqrt(n * steps * p * (1 - p))
    assert abs(hits - mean) < 4.5 * sd


def test_electron_collision_rate_sigma_inverse_velocity():
    # sigma ~ 1/v gives a velocity-independent collision frequency
    nent, de = 100_000, 1e-3
    energies = np.arange(nent) * de
    energies[0] = de / 2
    c = 1e-18 * math.sqrt(2 * 1.0 * QE / ME)
    sig = c / np.sqrt(2 * energies * QE / ME)
    se = np.stack([sig, 0 * sig, 0 * sig])
    si = np.zeros((2, nent))
    d = _quiet(gap_m=0.025, n_grid=51, capacity=1 << 17)
    rates = []
    for eps in (0.5, 4.0, 20.0):
        s = oracle.Sim(d, se, si, de)
        rng = np.random.default_rng(int(eps * 10))
        n = 30_000
        v = math.sqrt(2 * eps * QE / ME)
        dirs = rng.normal(size=(3, n))
        dirs /= np.linalg.norm(dirs, axis=0)
        s.load(0, wl.Particles(rng.uniform(0.012, 0.013, n), v * dirs[0], v * dirs[1], v * dirs[2]))
        s.load(1, wl.Particles.empty())
        s.step(2)
        rates.append(s.counters()["coll_e_ela"] / (2 * n))
    assert max(rates) - min(rates) < 5 * math.sqrt(rates[0] / 60_000)


def test_ion_thermalisation():
    # Ar+ in Ar at E = 0 relaxes to <M v^2 / 2> = 3/2 k T_g
    d = _quiet(gap_m=0.05, n_grid=51, ion_subcycle=1, steps_per_cycle=40)
    se, si = _tables(100_000, sigma_e=(0, 0, 0), sigma_i=(4e-17, 4e-17))
    s = oracle.Sim(d, se, si, 1e-3)
    n = 6000
    rng = np.random.default_rng(17)
    s.load(0, wl.Particles.empty())
    s.load(1, wl.Particles(rng.uniform(0.02, 0.03, n), np.full(n, 2000.0), np.zeros(n), np.zeros(n)))
    s.step(400)
    _, vx, vy, vz = s.particles(1)
    mean_e = 0.5 * MAR * np.mean(vx ** 2 + vy ** 2 + vz ** 2)
    assert s.counters()["coll_i_iso"] > 20 * n
    assert mean_e == pytest.approx(1.5 * KB * d.gas_temp_k, rel=0.05)


# ------------------------------------------------------------------ bookkeeping and diagnostics
def test_particle_bookkeeping_reference_start():
    d, e, i = wl.reference_start(seed=2, n0=1500)
    se, si = wl.standin_cross_sections(300_000)
    s = oracle.Sim(d, se, si, wl.CS_DE_EV, e, i)
    ne0, ni0 = s.count(0), s.count(1)
    s.step(400)
    c = s.counters()
    assert s.count(0) == ne0 - c["abs_e_pow"] - c["abs_e_gnd"] + c["created"]
    assert s.count(1) == ni0 - c["abs_i_pow"] - c["abs_i_gnd"] + c["created"]
    assert c["coll_e_ela"] > 0 and c["abs_e_pow"] + c["abs_e_gnd"] > 0


def test_eepf_normalisation_and_maxwellian_slope():
    d = _quiet(gap_m=0.025, n_grid=51, capacity=1 << 18, eepf_bins=400, eepf_de_ev=0.05)
    se, si = _tables(100_000, sigma_e=(0, 0, 0), sigma_i=(0, 0))
    s = oracle.Sim(d, se, si, 1e-3)
    rng = np.random.default_rng(18)
    kt = 2.0
    n = 200_000
    e = wl.maxwellian(n, d.gap_m, kt * QE, ME, rng, x=rng.uniform(0.46 * d.gap_m, 0.54 * d.gap_m, n))
    s.load(0, e)
    s.load(1, wl.Particles.empty())
    s.step(1, measure=True)
    h = s.diagnostics()["eepf_counts"]
    assert h.sum() == n - (0.5 * ME * (e.vx ** 2 + e.vy ** 2 + e.vz ** 2) / QE >= 20.0).sum()
    en, f = oracle.eepf_normalise(h, d.eepf_de_ev)
    assert (f * np.sqrt(en) * d.eepf_de_ev).sum() == pytest.approx(1.0, rel=1e-12)
    m = (en > 0.5) & (en < 8.0)
    slope = np.polyfit(en[m], np.log(f[m]), 1, w=np.sqrt(h[m]))[0]
    assert slope == pytest.approx(-1.0 / kt, rel=0.04)


def test_ifed_normalisation_and_energy():
    d = _quiet(gap_m=0.025, n_grid=51, ion_subcycle=1, ifed_bins=200, ifed_de_ev=1.0)
    se, si = _tables(1000, sigma_e=(0, 0, 0), sigma_i=(0, 0))
    s = oracle.Sim(d, se, si, 1e-3)
    dt = s.derived()["dt_i"]
    n = 300
    e_ev = np.linspace(0.2, 150.0, n)
    v = np.sqrt(2 * e_ev * QE / MAR)
    x = np.full(n, 1e-12)
    s.load(0, wl.Particles.empty())
    s.load(1, wl.Particles(x, -v, np.zeros(n), np.zeros(n)))
    s.step(1, measure=True)
    hp = s.diagnostics()["ifed_pow_counts"]
    assert s.counters()["abs_i_pow"] == n
    assert (hp == np.bincount(np.floor(e_ev).astype(int), minlength=200)).all()
    en, F = oracle.ifed_normalise(hp, 1.0)
    assert (F * 1.0).sum() == pytest.approx(1.0, rel=1e-12)
    assert dt > 0


def test_power_absorption_is_the_work_of_the_field():
    """Sec. 3.5 power absorption = space-time average of j E.  In a leapfrog
    step m (v_new - v_old) = q E dt, so q E dt v_c with v_c = (v_old +
    v_new) / 2 is exactly the change of (m/2) v_x^2: without collisions and
    absorption, the summed work of the field over the measured steps equals
    the change of the x kinetic energy, species by species (the ions only on
    their N_SUB-th steps)."""
    rng = np.random.default_rng(21)
    d = wl.reference_discharge(seed=21, capacity=1 << 14)
    n = 3000
    e = wl.maxwellian(n, d.gap_m, 2.0 * QE, ME, rng, x=rng.uniform(0.35 * d.gap_m, 0.65 * d.gap_m, n))
    i = wl.maxwellian(n, d.gap_m, 1.380649e-23 * 350.0, MAR, rng, x=rng.uniform(0.35 * d.gap_m, 0.65 * d.gap_m, n))
    se, si = wl.constant_cross_sections(1000, wl.CS_DE_EV, (0.0, 0.0, 0.0), (0.0, 0.0))
    ref = oracle.Sim(d, se, si, wl.CS_DE_EV, e, i)
    v0 = [ref.particles(sp)[1].copy() for sp in (0, 1)]
    steps = 2 * d.ion_subcycle
    ref.step(steps, measure=True)
    c = ref.counters()
    assert c["abs_e_pow"] + c["abs_e_gnd"] + c["abs_i_pow"] + c["abs_i_gnd"] == 0
    v1 = [ref.particles(sp)[1] for sp in (0, 1)]
    p = ref.power()
    dt_e = ref.derived()["dt_e"]
    to_work = d.area_m2 * d.gap_m * p["measured_steps"] * dt_e / d.weight
    for sp, m, key in ((0, ME, "electrons"), (1, MAR, "ions")):
        dke = 0.5 * m * (v1[sp] ** 2 - v0[sp] ** 2)
        work = p[key] * to_work
        scale = 0.5 * m * float(np.abs(v1[sp] ** 2 - v0[sp] ** 2).sum())
        assert abs(work - dke.sum()) <= 1e-9 * scale, (key, work, dke.sum())
        assert abs(work) > 1e-3 * scale  # the field did work


# ------------------------------------------------------------------ surface processes (Sec. 5)
def _walls(seed, n, species_mass, speed, rng, d, dt):
    """n particles within one step of the electrodes, half at each, moving
    outwards fast enough to cross within dt."""
    side = rng.integers(0, 2, n)
    gap = rng.uniform(0.1, 0.9, n) * speed * dt
    x = np.where(side == 0, gap, d.gap_m - gap)
    vx = np.where(side == 0, -speed, speed) * rng.uniform(1.0, 1.5, n)
    vy = rng.normal(0, speed / 3, n)
    vz = rng.normal(0, speed / 3, n)
    return wl.Particles(x, vx, vy, vz), side


def test_reflection_mirrors_every_electron_when_eta_is_one():
    d = _quiet(n_grid=101, gap_m=0.02, refl_eta=(1.0, 1.0))
    rng = np.random.default_rng(41)
    dt = 1.0 / (d.cycle_freq_hz * d.steps_per_cycle)
    e, side = _walls(41, 4000, ME, 1e6, rng, d, dt)
    i = wl.Particles.empty()
    ref = oracle.Sim(d, *_tables(200_000, wl.CS_DE_EV, sigma_e=(0, 0, 0), sigma_i=(0, 0)), wl.CS_DE_EV, e, i)
    ref.step(1)
    c = ref.counters()
    assert c["reflected"] == e.n and c["abs_e_pow"] + c["abs_e_gnd"] == 0
    x1, vx1, vy1, vz1 = ref.particles(0)
    xn = e.x + e.vx * dt  # the push in a zero field
    mirror = np.where(side == 0, -xn, 2 * d.gap_m - xn)
    assert np.array_equal(x1, mirror) and np.array_equal(vx1, -e.vx)
    assert np.array_equal(vy1, e.vy) and np.array_equal(vz1, e.vz)


def test_reflection_and_emission_probabilities():
    d = _quiet(n_grid=101, gap_m=0.02, refl_eta=(0.3, 0.0), see_gamma=(0.25, 0.6), see_te_ev=2.0)
    rng = np.random.default_rng(42)
    dt = 1.0 / (d.cycle_freq_hz * d.steps_per_cycle)
    n = 40_000
    e, e_side = _walls(42, n, ME, 1e6, rng, d, dt)
    i, i_side = _walls(43, n, MAR, 3e4, rng, d, d.ion_subcycle * dt)
    ref = oracle.Sim(d, *_tables(200_000, wl.CS_DE_EV, sigma_e=(0, 0, 0), sigma_i=(0, 0)), wl.CS_DE_EV, e, i)
    ref.step(1)  # step 0 is an ion step
    c = ref.counters()
    n_pow, n_gnd = int((e_side == 0).sum()), int((e_side == 1).sum())
    # electrons: reflected with probability 0.3 at the powered electrode, never at the grounded one
    assert c["abs_e_gnd"] == n_gnd
    assert c["reflected"] + c["abs_e_pow"] == n_pow
    assert abs(c["reflected"] - 0.3 * n_pow) <= 5 * math.sqrt(0.3 * 0.7 * n_pow)
    # ions: every one absorbed; each emits an electron with probability gamma of its electrode
    i_pow, i_gnd = int((i_side == 0).sum()), int((i_side == 1).sum())
    assert c["abs_i_pow"] == i_pow and c["abs_i_gnd"] == i_gnd
    for key, g, n_side in (("emitted_pow", 0.25, i_pow), ("emitted_gnd", 0.6, i_gnd)):
        assert abs(c[key] - g * n_side) <= 5 * math.sqrt(g * (1 - g) * n_side), key
    # the emitted electrons were appended last, at the electrodes, pointing into the gap
    x1, vx1, vy1, vz1 = ref.particles(0)
    k = c["emitted_pow"] + c["emitted_gnd"]
    xe, vxe = x1[-k:], vx1[-k:]
    assert np.all((xe == 0.0) | (xe == d.gap_m))
    assert np.all(vxe[xe == 0.0] > 0) and np.all(vxe[xe == d.gap_m] < 0)
    # half-Maxwellian at 2 eV: mean kinetic energy 3/2 kT
    ke = 0.5 * ME * (vxe ** 2 + vy1[-k:] ** 2 + vz1[-k:] ** 2) / QE
    assert abs(ke.mean() - 3.0) <= 5 * math.sqrt(1.5 * 2.0 ** 2 / k) + 0.02


# ------------------------------------------------------------------ null-collision method (Sec. 2.1.6)
def _mono_electrons(rng, n, eps_ev, lo=0.010, hi=0.015):
    v = math.sqrt(2 * eps_ev * QE / ME)
    dirs = rng.normal(size=(3, n))
    dirs /= np.linalg.norm(dirs, axis=0)
    return wl.Particles(rng.uniform(lo, hi, n), v * dirs[0], v * dirs[1], v * dirs[2]), v


def test_null_collision_bound_closed_form():
    # constant sigma: nu* = n sigma v at the top of the last table bin
    nent, de, sig = 1000, 1e-2, 3e-19
    d = _quiet(null_collision=3)
    s = oracle.Sim(d, *_tables(nent, de, sigma_e=(sig, 0, 0), sigma_i=(0, sig)), de)
    dv = s.derived()
    v_top = math.sqrt(2 * (nent - 0.5) * de * QE / ME)
    g_top = math.sqrt(2 * (nent - 0.5) * de * QE / (MAR / 2))
    assert dv["nu_star_e"] == pytest.approx(dv["n_gas"] * sig * v_top, rel=1e-14)
    assert dv["nu_star_i"] == pytest.approx(dv["n_gas"] * sig * g_top, rel=1e-14)
    assert dv["p_star_e"] == pytest.approx(-math.expm1(-dv["nu_star_e"] * dv["dt_e"]), rel=1e-12)
    assert dv["p_star_i"] == pytest.approx(-math.expm1(-dv["nu_star_i"] * dv["dt_i"]), rel=1e-12)


def test_null_collision_electron_rates():
    # mono-energetic electrons, constant sigma, E = 0: a share P* is picked,
    # and a picked one collides with probability v / v_top (nu / nu*)
    nent, de, sig, eps = 2000, 1e-2, 2.2e-18, 5.0
    d = _quiet(gap_m=0.025, n_grid=51, capacity=1 << 17, null_collision=1)
    se, si = _tables(nent, de, sigma_e=(sig, 0, 0), sigma_i=(0, 0))
    s = oracle.Sim(d, se, si, de)
    n, steps = 60_000, 2
    e, v = _mono_electrons(np.random.default_rng(31), n, eps)
    s.load(0, e)
    s.load(1, wl.Particles.empty())
    s.step(steps)
    c, dv = s.counters(), s.derived()
    p_star = dv["p_star_e"]
    assert 0.05 < p_star < 0.5
    trials = n * steps
    assert abs(c["null_tested"] - trials * p_star) <= 5 * math.sqrt(trials * p_star * (1 - p_star))
    p_real = p_star * v / math.sqrt(2 * (nent - 0.5) * de * QE / ME)
    assert abs(c["coll_e_ela"] - trials * p_real) <= 5 * math.sqrt(trials * p_real * (1 - p_real))
    assert c["null_over"] == 0
    # to first order in nu dt the same rate as the direct test (Algorithm 6)
    p_direct = -math.expm1(-dv["n_gas"] * sig * v * dv["dt_e"])
    assert abs(p_real - p_direct) <= 0.5 * p_star * p_direct


def test_null_collision_past_the_table_always_collides():
    # energies beyond the table exceed nu*: every picked electron collides and is counted
    nent, de, sig = 500, 1e-2, 4e-17
    d = _quiet(gap_m=0.025, n_grid=51, capacity=1 << 17, null_collision=1)
    s = oracle.Sim(d, *_tables(nent, de, sigma_e=(sig, 0, 0), sigma_i=(0, 0)), de)
    e, _ = _mono_electrons(np.random.default_rng(32), 20_000, 40.0)
    s.load(0, e)
    s.load(1, wl.Particles.empty())
    s.step(1)
    c = s.counters()
    assert c["null_tested"] > 1000
    assert c["null_over"] == c["null_tested"] == c["coll_e_ela"]


def test_null_collision_ion_rate_thermal_partner():
    # Ar+ at rest, constant sigma: g is the partner speed, a Maxwell speed of
    # mean 2 sqrt(2 k T / (pi M)); real collisions P* <g> / g_top
    nent, de, sig = 1000, 1e-3, 1e-15
    d = _quiet(gap_m=0.025, n_grid=51, ion_subcycle=1, steps_per_cycle=40, capacity=1 << 18,
               null_collision=2)
    s = oracle.Sim(d, *_tables(nent, de, sigma_e=(0, 0, 0), sigma_i=(sig, sig)), de)
    n = 200_000
    x = np.random.default_rng(33).uniform(0.01, 0.015, n)
    s.load(0, wl.Particles.empty())
    s.load(1, wl.Particles(x, np.zeros(n), np.zeros(n), np.zeros(n)))
    s.step(1)  # step 0 is an ion step
    c, dv = s.counters(), s.derived()
    p_star = dv["p_star_i"]
    assert abs(c["null_tested"] - n * p_star) <= 5 * math.sqrt(n * p_star * (1 - p_star))
    g_mean = 2 * math.sqrt(2 * KB * d.gas_temp_k / (math.pi * MAR))
    p_real = p_star * g_mean / math.sqrt(2 * (nent - 0.5) * de * QE / (MAR / 2))
    hits = c["coll_i_iso"] + c["coll_i_back"]
    assert abs(hits - n * p_real) <= 5 * math.sqrt(n * p_real)
    # backward and isotropic in the ratio of their cross sections (equal here)
    assert abs(c["coll_i_iso"] - c["coll_i_back"]) <= 5 * math.sqrt(hits)


# ------------------------------------------------------------------ DC self-bias (Sec. 5)
def test_self_bias_adds_to_the_powered_electrode():
    # no space charge (W = 0): phi = (V + V_bias)(1 - x/L) and E = (V + V_bias)/L
    V, vb = 0.02, -0.35
    d = _quiet(harmonics=((0.0, V),), gap_m=0.025, n_grid=101)
    se, si = _tables(1000, sigma_e=(0, 0, 0), sigma_i=(0, 0))
    rng = np.random.default_rng(9)
    e = wl.Particles(rng.uniform(0.01, 0.015, 8), np.zeros(8), np.zeros(8), np.zeros(8))
    s = oracle.Sim(d, se, si, 1e-3, e, wl.Particles.empty())
    s.set_bias(vb)
    s.step(1)
    f = s.fields()
    x = np.arange(d.n_grid) * d.gap_m / (d.n_grid - 1)
    assert np.abs(f["phi"] - (V + vb) * (1 - x / d.gap_m)).max() <= 1e-12 * abs(V + vb)
    assert np.abs(f["efield"] - (V + vb) / d.gap_m).max() <= 1e-12
    # the electrons accelerate towards the more positive electrode (x = L here)
    assert (s.particles(0)[1] > 0).all()


# ------------------------------------------------------------------ xt diagnostics (Sec. 3.5)
XT = {name: k for k, name in enumerate(oracle.XT_NAMES)}


def test_xt_uniform_drift_closed_form():
    # e- all moving with v0 along x, a weight so small that the field is ~0:
    # j_e = -e v0 n_e and the mean energy (1/2) m v0^2 at every point and bin
    v0, n = 1.0e5, 4000
    d = _quiet(weight=1e-9, n_grid=51, steps_per_cycle=400, ion_subcycle=20, xt_bins=20)
    se, si = _tables(1000, sigma_e=(0, 0, 0), sigma_i=(0, 0))
    rng = np.random.default_rng(21)
    e = wl.Particles(rng.uniform(0.005, 0.02, n), np.full(n, v0), np.zeros(n), np.zeros(n))
    s = oracle.Sim(d, se, si, 1e-3, e, wl.Particles.empty())
    s.step(60, measure=True)  # bins 0, 1, 2 of 20 steps
    ne, je, mee = s.xt(XT["ne"]), s.xt(XT["je"]), s.xt(XT["meanee"])
    assert (ne[:, 3:] == 0).all() and (ne[:, :3] > 0).any()
    assert np.abs(je + QE * v0 * ne).max() <= 1e-9 * QE * v0 * ne.max()
    hit = s.xt(XT["ne"]) > 0
    assert np.abs(mee[hit] - 0.5 * ME * v0 ** 2 / QE).max() <= 1e-9 * 0.5 * ME * v0 ** 2 / QE
    assert (mee[~hit] == 0).all() and (s.xt(XT["ji"]) == 0).all()
    # the field map is the drive's (none) plus the tiny space charge
    assert np.abs(s.xt(XT["efield"])).max() < 1e-3
    assert np.array_equal(s.xt(XT["powere"]), je * s.xt(XT["efield"]))


def test_xt_bins_average_to_the_time_averages():
    # over whole bins, the step-weighted mean of the n_e, n_i, phi maps is the
    # time average of the measured steps
    d, e, i = wl.reference_steady(seed=3, n=3000)
    d = d.replace(xt_bins=400)  # 10 steps per bin
    se, si = wl.standin_cross_sections(20_000)
    s = oracle.Sim(d, se, si, wl.CS_DE_EV, e, i)
    s.step(50, measure=True)
    diag = s.diagnostics()
    for key, name in (("n_e", "ne"), ("n_i", "ni"), ("phi", "pot")):
        m = s.xt(XT[name])[:, :5].mean(axis=1)  # 5 full bins of 10 steps
        assert np.abs(m - diag[key]).max() <= 1e-12 * np.abs(diag[key]).max(), key


def test_xt_ionisation_rate_integrates_to_the_events():
    # sum over space and time of the rate map: W x (ionisations of the measured steps)
    d, e, i = wl.reference_steady(seed=4, n=8000)
    d = d.replace(xt_bins=200, harmonics=((13.56e6, 400.0),))  # N_BIN = 20
    se, si = wl.standin_cross_sections(300_000)
    s = oracle.Sim(d, se, si, wl.CS_DE_EV, e, i)
    s.step(200, measure=True)
    events = s.counters()["coll_e_ion"]
    assert events > 10
    dv = s.derived()
    rate = s.xt(XT["ioniz"])
    vol = np.full(d.n_grid, d.area_m2 * dv["dx"])
    vol[[0, -1]] *= 0.5
    steps = np.zeros(d.xt_bins)
    steps[:10] = 20
    total = (rate * vol[:, None] * steps[None, :] * dv["dt_e"]).sum()
    assert total == pytest.approx(d.weight * events, rel=1e-12)


# ------------------------------------------------------------------ init(N_INIT) of Algorithm 1
def test_seed_uniform_at_rest():
    # n electrons and n ions, uniform on (0, L) (KS test) and at rest; the
    # deposited charge is n 2^32 per species; the two species are independent
    from scipy import stats

    d = wl.reference_discharge(capacity=50_000)
    se, si = _tables(1000)
    s = oracle.Sim(d, se, si, 1e-3)
    s.seed(20_000)
    assert s.count(0) == s.count(1) == 20_000
    for sp in (0, 1):
        x, vx, vy, vz = s.particles(sp)
        assert (x >= 0).all() and (x < d.gap_m).all()
        assert stats.kstest(x / d.gap_m, "uniform").pvalue > 1e-3
        assert not vx.any() and not vy.any() and not vz.any()
    f = s.fields()
    assert int(f["q_e"].sum()) == int(f["q_i"].sum()) == 20_000 * 2 ** 32
    assert not np.array_equal(s.particles(0)[0], s.particles(1)[0])


def test_xt_ion_drift_closed_form():
    # Ar+ all moving with v0 along x, bins of N_SUB steps (one ion step each):
    # j_i = e v0 n_i and the mean ion energy (1/2) M v0^2, normalised per ion
    # step (a division by all steps of the bin would be N_SUB times smaller)
    v0, n = 1.0e3, 4000
    d = _quiet(weight=1e-9, n_grid=51, steps_per_cycle=400, ion_subcycle=20, xt_bins=20)
    se, si = _tables(1000, sigma_e=(0, 0, 0), sigma_i=(0, 0))
    rng = np.random.default_rng(22)
    i = wl.Particles(rng.uniform(0.005, 0.02, n), np.full(n, v0), np.zeros(n), np.zeros(n))
    s = oracle.Sim(d, se, si, 1e-3, wl.Particles.empty(), i)
    s.step(60, measure=True)  # bins 0, 1, 2, one ion step each
    ni, ji, mei = s.xt(XT["ni"]), s.xt(XT["ji"]), s.xt(XT["meanei"])
    assert (ni[:, :3] > 0).any() and (ni[:, 3:] == 0).all()
    assert np.abs(ji - QE * v0 * ni).max() <= 1e-9 * QE * v0 * ni.max()
    hit = ni > 0
    e_ion = 0.5 * MAR * v0 ** 2 / QE
    assert np.abs(mei[hit] - e_ion).max() <= 1e-9 * e_ion
    assert (s.xt(XT["je"]) == 0).all() and (s.xt(XT["ne"]) == 0).all()


# ------------------------------------------------------------------ drive V(t) (Sec. 2, Sec. 4.2)
def _phi0_and_field(d, steps):
    """Boundary potential phi_0 and field of the solve made at each global
    step, with no space charge (W = 0): phi_0 = V(t) and E = V(t) / L."""
    se, si = _tables(1000, sigma_e=(0, 0, 0), sigma_i=(0, 0))
    s = oracle.Sim(d, se, si, 1e-3, wl.Particles.empty(), wl.Particles.empty())
    out = []
    for st in steps:
        s.step_index = st
        f = s.prepare_fields()
        out.append((f["phi"][0], f["efield"].copy()))
    return out


def _check_drive(d, expected, v_scale):
    got = _phi0_and_field(d, list(expected))
    for (st, v), (phi0, ef) in zip(expected.items(), got):
        assert abs(phi0 - v) <= 1e-10 * v_scale, (st, phi0, v)
        assert np.abs(ef - v / d.gap_m).max() <= 1e-10 * v_scale / d.gap_m, st


def test_drive_single_frequency_special_phases():
    # V(t) = V0 cos(2 pi f t) at the cycle's quarter points, an eighth, and
    # after cycle wraps (the phase is that of the step inside the cycle)
    V0, nt = 250.0, 4000
    d = _quiet(harmonics=((13.56e6, V0),), cycle_freq_hz=13.56e6, steps_per_cycle=nt)
    r = 1.0 / math.sqrt(2.0)
    _check_drive(d, {0: V0, nt // 8: V0 * r, nt // 4: 0.0, nt // 2: -V0, 3 * nt // 4: 0.0,
                     nt + nt // 8: V0 * r, 3 * nt + nt // 2: -V0, 7 * nt: V0}, V0)
    # the step itself solves with the same boundary value (one step after a wrap)
    se, si = _tables(1000, sigma_e=(0, 0, 0), sigma_i=(0, 0))
    s = oracle.Sim(d, se, si, 1e-3, wl.Particles.empty(), wl.Particles.empty())
    s.step_index = 2 * nt + nt // 2
    s.step(1)
    assert abs(s.fields()["phi"][0] + V0) <= 1e-10 * V0


def test_drive_two_harmonics_special_phases():
    # V(t) = V1 cos(2 pi f t) + V2 cos(4 pi f t), cycle = the lower frequency:
    # t = 0 -> V1 + V2, T/8 -> V1/sqrt2, T/4 -> -V2, T/2 -> V2 - V1
    f, V1, V2, nt = 13.56e6, 120.0, 80.0, 4000
    d = _quiet(harmonics=((f, V1), (2 * f, V2)), cycle_freq_hz=f, steps_per_cycle=nt)
    _check_drive(d, {0: V1 + V2, nt // 8: V1 / math.sqrt(2.0), nt // 4: -V2, nt // 2: V2 - V1,
                     5 * nt + nt // 4: -V2}, V1 + V2)


def test_drive_dual_frequency_lf_cycle():
    # the dual-frequency drive of Sec. 4.2 (1.356 MHz + 27.12 MHz, the cycle is
    # the low-frequency period, 20 HF periods): T/4 -> V_HF, T/8 -> V_LF/sqrt2 - V_HF
    V_lf, V_hf, nt = 300.0, 100.0, 320_000
    d = _quiet(harmonics=((1.356e6, V_lf), (27.12e6, V_hf)), cycle_freq_hz=1.356e6, steps_per_cycle=nt)
    _check_drive(d, {0: V_lf + V_hf, nt // 4: V_hf, nt // 8: V_lf / math.sqrt(2.0) - V_hf,
                     nt // 2: V_hf - V_lf, nt + nt // 40: -V_hf + V_lf * math.cos(math.pi / 20)}, V_lf + V_hf)


# ------------------------------------------------------------------ Ar+ direct collision test (Sec. 2.1.6, Alg. 6)
def test_ion_collision_rate_direct_thermal_partner():
    # Ar+ at rest in a field-free gap, constant sigma, direct test on an ion
    # step (dt_i = N_SUB dt_e): the relative speed is the partner's Maxwell
    # speed, so the collision probability is the Maxwell average of
    # 1 - exp(-n sigma g dt_i), evaluated here by quadrature
    from scipy import integrate
    sig = 2.0e-15
    d = _quiet(gap_m=0.025, n_grid=51, ion_subcycle=20, steps_per_cycle=4000, capacity=1 << 18)
    se, si = _tables(1000, 1e-3, sigma_e=(0, 0, 0), sigma_i=(0.6 * sig, 0.4 * sig))
    s = oracle.Sim(d, se, si, 1e-3)
    n = 200_000
    x = np.random.default_rng(41).uniform(0.01, 0.015, n)
    s.load(0, wl.Particles.empty())
    s.load(1, wl.Particles(x, np.zeros(n), np.zeros(n), np.zeros(n)))
    s.step(1)  # step 0 is an ion step
    c, dv = s.counters(), s.derived()
    assert dv["dt_i"] == pytest.approx(20 * dv["dt_e"], rel=1e-15)
    a = MAR / (2 * KB * d.gas_temp_k)
    lam = dv["n_gas"] * sig * dv["dt_i"]

    def maxwell(g):
        return 4 * math.pi * (a / math.pi) ** 1.5 * g * g * math.exp(-a * g * g)

    gmax = 12 / math.sqrt(a)
    norm = integrate.quad(maxwell, 0, gmax, epsabs=0, epsrel=1e-12)[0]
    p = integrate.quad(lambda g: maxwell(g) * -math.expm1(-lam * g), 0, gmax, epsabs=0, epsrel=1e-12)[0]
    assert norm == pytest.approx(1.0, rel=1e-10)
    assert 0.3 < p < 0.6  # far from the linear regime: 1 - exp matters
    hits = c["coll_i_iso"] + c["coll_i_back"]
    assert abs(hits - n * p) <= 4.5 * math.sqrt(n * p * (1 - p))
    # isotropic against backward in the ratio of their cross sections
    assert abs(c["coll_i_iso"] - 0.6 * hits) <= 4.5 * math.sqrt(hits * 0.24)
    # the ions still sit where they were (E = 0) and no electron is involved
    assert s.count(1) == n and c["coll_e_ela"] + c["coll_e_exc"] + c["coll_e_ion"] == 0


# ------------------------------------------------------------------ ionisation products (Sec. 2.1.6, reading 17)
def test_ionisation_ions_come_from_the_gas_maxwellian():
    # every electron ionises (ionisation only, P_coll = 1): the new Ar+ sits at
    # its parent's position with a velocity of the gas Maxwellian at T_g,
    # so <M v^2 / 2> = 3/2 k T_g and each component has variance k T_g / M
    d = _quiet(gap_m=0.025, n_grid=51, capacity=1 << 17)
    se, si = _tables(200_000, 1e-3, sigma_e=(0, 0, 1e-16), sigma_i=(0, 0))
    s = oracle.Sim(d, se, si, 1e-3)
    n = 40_000
    e, _ = _mono_electrons(np.random.default_rng(42), n, 100.0)
    s.load(0, e)
    s.load(1, wl.Particles.empty())
    s.step(1)
    c = s.counters()
    assert c["coll_e_ion"] == n and c["created"] == n
    assert s.count(0) == 2 * n and s.count(1) == n
    xe = s.particles(0)[0]
    xi, vx, vy, vz = s.particles(1)
    assert np.array_equal(xi, xe[:n])  # parents keep their slots; products follow in parent order
    kt_m = KB * d.gas_temp_k / MAR
    mean_e = 0.5 * MAR * np.mean(vx ** 2 + vy ** 2 + vz ** 2)
    assert abs(mean_e / (1.5 * KB * d.gas_temp_k) - 1) <= 4.5 * math.sqrt(2.0 / 3.0 / n)
    for comp in (vx, vy, vz):
        assert abs(np.mean(comp)) <= 4.5 * math.sqrt(kt_m / n)
        assert abs(np.mean(comp ** 2) / kt_m - 1) <= 4.5 * math.sqrt(2.0 / n)


# ------------------------------------------------------------------ table index (Algorithm 6)
def test_table_index_is_the_nearest_entry_electrons():
    # sigma non-zero only in entry k + 1: energies (k + 0.7) de round to it and
    # always collide, energies (k + 0.3) de round to entry k and never do;
    # flooring the index would swap the two outcomes
    k, de, nent = 5000, 1e-3, 20_000
    sig = np.zeros(nent)
    sig[k + 1] = 1e-15
    se = np.stack([sig, np.zeros(nent), np.zeros(nent)])
    si = np.zeros((2, nent))
    d = _quiet(gap_m=0.025, n_grid=51, capacity=1 << 15)
    for frac, expect_all in ((0.7, True), (0.3, False)):
        s = oracle.Sim(d, se, si, de)
        e, _ = _mono_electrons(np.random.default_rng(43), 5000, (k + frac) * de)
        s.load(0, e)
        s.load(1, wl.Particles.empty())
        s.step(1)
        assert s.counters()["coll_e_ela"] == (5000 if expect_all else 0), frac


def test_table_index_is_the_nearest_entry_ions_by_com_energy():
    # the ion table is indexed by the centre-of-mass energy mu g^2 / 2 (mu =
    # M / 2); a near-zero gas temperature makes g the ion's own speed
    k, de, nent = 5, 1e-3, 200
    sig = np.zeros(nent)
    sig[k + 1] = 1e-14
    se = np.zeros((3, nent))
    si = np.stack([sig, np.zeros(nent)])
    d = _quiet(gap_m=0.025, n_grid=51, capacity=1 << 15, gas_temp_k=1e-5, pressure_pa=1e-5)
    n = 5000
    rng = np.random.default_rng(44)
    for frac, expect_all in ((0.7, True), (0.3, False)):
        s = oracle.Sim(d, se, si, de)
        g = math.sqrt(2 * (k + frac) * de * QE / (MAR / 2))
        dirs = rng.normal(size=(3, n))
        dirs /= np.linalg.norm(dirs, axis=0)
        s.load(0, wl.Particles.empty())
        s.load(1, wl.Particles(rng.uniform(0.01, 0.015, n), g * dirs[0], g * dirs[1], g * dirs[2]))
        s.step(1)
        c = s.counters()
        assert c["coll_i_iso"] == (n if expect_all else 0), frac


# ------------------------------------------------------------------ periodic cell sort (slot order)
def _cells(x, d):
    # the cell of the deposition (Algorithm 2): floor(x / dx) formed as
    # x * (1 / dx), the last cell taking x = L
    inv_dx = 1.0 / (d.gap_m / (d.n_grid - 1))
    return np.minimum(np.floor(x * inv_dx).astype(np.int64), d.n_grid - 2)


def _sort_pair(sort_every, steps):
    d, e, i = wl.reference_start(seed=31, n0=3000)
    se, si = wl.standin_cross_sections(300_000)
    a = oracle.Sim(d.replace(sort_every=sort_every), se, si, wl.CS_DE_EV, e, i)
    b = oracle.Sim(d, se, si, wl.CS_DE_EV, e, i)
    a.step(steps)
    b.step(steps)
    return d, a, b


def test_cell_sort_is_a_stable_counting_sort_by_cell():
    # after the 20th step (one ion subcycle) the arrays are the unsorted run's
    # arrays in numpy's stable order of their deposition cells
    d, a, b = _sort_pair(1, 20)
    for sp in (0, 1):
        pa, pb = a.particles(sp), b.particles(sp)
        order = np.argsort(_cells(pb[0], d), kind="stable")
        for k in range(4):
            assert np.array_equal(pa[k], pb[k][order]), (sp, k)
        assert (np.diff(_cells(pa[0], d)) >= 0).all()
    # the densities do not depend on the order
    assert np.array_equal(a.prepare_fields()["q_e"], b.prepare_fields()["q_e"])
    assert np.array_equal(a.prepare_fields()["q_i"], b.prepare_fields()["q_i"])


def test_cell_sort_happens_only_every_sort_every_subcycles():
    # sort_every = 2: nothing before step 40, sorted right after it
    d, a, b = _sort_pair(2, 39)
    for sp in (0, 1):
        assert all(np.array_equal(u, v) for u, v in zip(a.particles(sp), b.particles(sp)))
    a.step(1)
    b.step(1)
    pa, pb = a.particles(0), b.particles(0)
    order = np.argsort(_cells(pb[0], d), kind="stable")
    assert np.array_equal(pa[0], pb[0][order]) and not np.array_equal(pa[0], pb[0])
    # after that, the sorted run draws other random numbers per particle
    # (slots moved) but keeps the same particle count bookkeeping
    a.step(20)
    c = a.counters()
    assert a.count(0) == 3000 - c["abs_e_pow"] - c["abs_e_gnd"] + c["created"]
