"""The electrons' collision bound (host logic, no GPU): for every v^2 the
particle kernel can meet, the table entry of its bucket is at least
sigma_tot(nearest entry) * v, the quantity P_coll = 1 - exp(-n sigma v dt) is
bounded by after the kernel multiplies by n dt (Algorithm 6's test only
skips particles whose uniform lies above it).  The bucket and the entry index
are formed here as the header states and the kernel computes them: the
exponent and top five mantissa bits of v^2 in the particle precision, and the
nearest table entry (FP32: v^2 s + 0.5 in one rounding, s = (m/2e)/DE in
FP32)."""
import numpy as np
import pytest

from paper_2103_09642_gb300 import build_ext
from paper_2103_09642_gb300 import edupic as ed
from paper_2103_09642_gb300 import workloads as wl

ME, QE = 9.1093837015e-31, 1.602176634e-19
DE = wl.CS_DE_EV


@pytest.fixture(scope="module")
def sigma_sum():
    build_ext.build()
    se, _ = wl.standin_cross_sections(200_000)
    return se.sum(axis=0)  # elastic + excitation + ionisation per entry, in this order


def _case(precision):
    if precision == ed.FP64:
        return np.float64, np.uint64, 47
    return np.float32, np.uint32, 18


def _bucket(w2, ftype, itype, shift, base, nb):
    b = (np.asarray(w2, dtype=ftype).view(itype) >> itype(shift)).astype(np.int64)
    return np.clip(b, base, base + nb - 1) - base


def _entry(w2, precision, n):
    w = np.asarray(w2, dtype=np.float64)
    if precision == ed.FP32:
        s = np.float64(np.float32(0.5 * ME / QE / DE))
        r = (w * s + 0.5).astype(np.float32).astype(np.float64)  # fmaf: the product is exact in FP64
    else:
        r = 0.5 * ME * w / QE / DE + 0.5
    return np.minimum(np.floor(np.minimum(r, 4e18)), n - 1).astype(np.int64)


@pytest.mark.parametrize("precision", [ed.FP32, ed.FP64])
def test_bound_covers_every_speed(sigma_sum, precision):
    ftype, itype, shift = _case(precision)
    table, base, nb = ed.electron_bound_table(precision, sigma_sum, DE)
    assert 2 <= nb <= ed.BOUND_BUCKETS
    assert np.isinf(table[nb - 1]) and np.isinf(table[nb:]).all() and np.isfinite(table[: nb - 1]).all()
    sig = sigma_sum.astype(ftype).astype(np.float64)  # the table the kernel holds
    rng = np.random.default_rng(3)
    # random speeds over the whole table and beyond, and every bucket boundary with its neighbours
    w_rand = np.exp(rng.uniform(np.log(1e4), np.log(4e16), 400_000)).astype(ftype)
    edges = (np.arange(base + 1, base + nb, dtype=np.int64).astype(itype) << itype(shift)).view(ftype)
    near, up, dn = [edges], edges, edges
    for _ in range(3):
        up, dn = np.nextafter(up, ftype(np.inf)), np.nextafter(dn, ftype(0))
        near += [up, dn]
    w2 = np.concatenate([w_rand] + near)
    w2 = w2[np.isfinite(w2) & (w2 >= 0)]
    j = _bucket(w2, ftype, itype, shift, base, nb)
    k = _entry(w2, precision, sig.size)
    need = sig[k] * np.sqrt(w2.astype(np.float64))
    have = table[j]
    bad = ~(have >= need)
    assert not bad.any(), (w2[bad][:5], have[bad][:5], need[bad][:5])
    # and it is tight where sigma varies little over a bucket (not a trivial bound)
    fin = np.isfinite(have) & (need > 0)
    ratio = have[fin] / need[fin]
    assert np.median(ratio) < 1.05, np.median(ratio)


def test_bound_table_rejects_bad_arguments(sigma_sum):
    with pytest.raises(ed.EdupicError):
        ed.electron_bound_table(ed.FP32, -sigma_sum, DE)
    with pytest.raises(ed.EdupicError):
        ed.electron_bound_table(ed.FP64, sigma_sum, 0.0)
