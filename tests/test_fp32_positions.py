"""What FP32 particle positions cost the ions (CPU, numpy only).

In FP32 mode a position is stored as float32 and advanced once per ion step
by x <- fma(v, dt_i, x) (Sec. 2.1.4, Algorithm 4).  On [2^-6, 2^-5) m, which
holds 0.63 L .. L of the reference gap (L = 2.5 cm), the spacing of float32
values is s = 2^-29 m ~ 1.9e-9 m, while a thermal Ar+ at 350 K moves
sigma_v dt_i ~ 1e-7 m per ion step (N_SUB = 20, dt_e = 1/(13.56 MHz * 4000)).
x sits on that grid, so each step adds the displacement v dt_i rounded to a
whole number of spacings: in a field-free stretch an ion moves with a
quantised velocity.  The study evolves thermal ions there for 1000 ion steps
in float64 (the reference), in float32 as the kernels do, and as a uint32
fraction of L (the alternative, spacing L / 2^32 ~ 5.8e-12 m), and states:

* per ion the displacement error after k steps is at most k s / 2, i.e. a
  relative velocity error of at most s / (2 |v_x| dt_i): ~1 % for a thermal
  ion, more for slower ones;
* the error is unbiased over ions (its mean is Monte Carlo noise of the
  uniformly distributed rounding);
* the mean squared displacement, which ion transport follows, carries the
  rounding's variance s^2 / 12 per step: ~3e-5 relative;
* ions with |v_x| dt_i < s / 2 (|v_x| < 2.5 m/s, 0.75 % of a 350 K
  Maxwellian) do not move at all; their share of the mean squared
  displacement is ~2e-7;
* the uint32 fraction of L is 320 times finer, bounds the error by
  k L / 2^33, and leaves no ion standing.

In the discharge the field changes v_x every ion step, so the rounding of
successive steps decorrelates; ions near the electrodes are accelerated by
the sheath well above thermal speeds.  The FP32 runs are compared with the
FP64 oracle through the statistical tier (densities, EEPF, ion flux, IFED).
"""
import numpy as np

KB, MAR = 1.380649e-23, 39.948 * 1.66053906660e-27
L = 0.025
DT_I = 20.0 / (13.56e6 * 4000)
S32 = 2.0 ** -29   # float32 spacing on [2^-6, 2^-5) m
SU = L / 2.0 ** 32  # uint32 fraction of L


def _evolve(x0, v, steps):
    x64 = x0.copy()
    x32 = x0.astype(np.float32)
    v32, dt32 = v.astype(np.float32), np.float32(DT_I)
    u = np.round(x0 / SU).astype(np.int64)
    du = np.round(v * DT_I / SU).astype(np.int64)
    for _ in range(steps):
        x64 = x64 + v * DT_I
        # fused multiply-add of float32 operands, rounded once to float32
        x32 = (x32.astype(np.float64) + v32.astype(np.float64) * np.float64(dt32)).astype(np.float32)
        u = u + du
    return x64, x32.astype(np.float64), u * SU


def test_fp32_position_rounding_of_thermal_ions():
    rng = np.random.default_rng(2103)
    n, steps = 200_000, 1000
    x0 = rng.uniform(0.65 * L, 0.98 * L, n)
    v = rng.normal(0.0, np.sqrt(KB * 350.0 / MAR), n)
    x64, x32, xu = _evolve(x0, v, steps)
    assert (x32 >= 2.0 ** -6).all() and (x32 < 2.0 ** -5).all()  # one binade: spacing S32 throughout
    d64 = x64 - x0
    d32 = x32 - x0.astype(np.float32).astype(np.float64)  # from the rounded start the kernel holds
    du = xu - np.round(x0 / SU) * SU
    err32, erru = d32 - d64, du - d64
    step_len = np.sqrt(KB * 350.0 / MAR) * DT_I
    assert 50 * S32 < step_len < 60 * S32
    # per ion: at most half a spacing per step, a quantised velocity
    assert np.all(np.abs(err32) <= steps * S32 / 2 * (1 + 1e-6))
    moving = np.abs(v) * DT_I > S32 / 2
    rel_v = np.abs(err32[moving]) / np.abs(d64[moving])
    assert np.all(rel_v <= S32 / (2 * np.abs(v[moving]) * DT_I) * (1 + 1e-6))
    assert 0.005 < np.median(rel_v) < 0.02  # ~1 % for thermal ions
    # unbiased over ions: the mean is the noise of uniform roundings
    assert abs(err32.mean()) < 5 * steps * (S32 / np.sqrt(12)) / np.sqrt(n)
    # mean squared displacement: + s^2 / 12 per step squared, relative
    msd64, msd32, msdu = (d64 ** 2).mean(), (d32 ** 2).mean(), (du ** 2).mean()
    expected = S32 ** 2 / 12 / (step_len ** 2)
    assert 0.3 * expected < msd32 / msd64 - 1 < 3 * expected
    assert expected < 1e-4
    # ions below half a spacing per step stand still
    stalled = ~moving
    assert 0.004 < stalled.mean() < 0.012
    assert np.all(d32[np.abs(v) * DT_I < 0.49 * S32] == 0.0)
    assert (d64[stalled] ** 2).sum() / (d64 ** 2).sum() < 1e-6
    # the uint32 fraction of L: 320 times finer, error at most k L / 2^33, no ion standing
    assert S32 / SU > 300
    assert np.all(np.abs(erru) <= steps * SU / 2 * (1 + 1e-6))
    assert np.all(du[np.abs(v) * DT_I >= SU] != 0.0)
    assert abs(msdu / msd64 - 1) < 1e-6
