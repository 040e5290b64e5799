"""Failure detection, in forms that fault, trap or hang no GPU.

* A bounded device wait runs out: one block waits, with the particle
  kernel's own bounded wait, on a barrier that nothing arrives on.  The wait
  gives up after its limit, the error is recorded in the discharge's error
  bits, the API reports EDUPIC_ETIMEOUT, and the context stays usable.
* A corrupted or truncated checkpoint is refused with the documented status
  and leaves the simulation exactly as it was.
* A request cancelled while it runs returns its slot and heap memory, and
  the requests beside it finish with the results they have alone.
"""
import os

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

SE, SI = wl.standin_cross_sections(300_000)
DE = wl.CS_DE_EV
EINVAL, ECAPACITY, ESTATE, EIO, ETIMEOUT = -1, -3, -5, -7, -8


# --------------------------------------------------------------- bounded waits
def test_bounded_wait_expires_and_reports_timeout():
    d, e, i = wl.reference_start(seed=4, n0=500, capacity=1 << 14)
    sim = ed.simulation_for([d], ed.FP64, sigma=(SE, SI), de_ev=DE, particles=[(e, i)])
    assert sim.selftest_wait_expiry(0, 1_000_000) == ETIMEOUT  # a 1 ms limit
    with pytest.raises(ed.EdupicError) as ex:
        sim.synchronize()
    assert ex.value.status == ETIMEOUT
    # out-of-range limits are refused without launching anything
    assert sim.selftest_wait_expiry(0, 10) == EINVAL
    assert sim.selftest_wait_expiry(0, 2_000_000_000) == EINVAL
    sim.close()
    # the context is still usable: a fresh simulation steps like the oracle
    sim = ed.simulation_for([d], ed.FP64, sigma=(SE, SI), de_ev=DE, particles=[(e, i)])
    ref = oracle.Sim(d, SE, SI, DE, e, i)
    sim.step(25)
    ref.step(25)
    sim.synchronize()
    assert sim.counters(0) == ref.counters()
    g, r = sim.particles(0, 0), ref.particles(0)
    assert np.abs(g[0] - r[0]).max() <= 1e-12 * d.gap_m
    sim.close()


# --------------------------------------------------------------- checkpoints
HDR = 8 + 8 + 24  # magic, (version, n_grid) int32, (step, n_e, n_i) int64


def _snapshot(sim):
    return sim.counts(0), [sim.particles(0, sp) for sp in (0, 1)], sim.fields(0)


def _same_snapshot(a, b):
    assert a[0] == b[0]
    for sp in (0, 1):
        for k in range(4):
            assert np.array_equal(a[1][sp][k], b[1][sp][k])
    for k in ("q_e", "q_i", "phi", "efield"):
        assert np.array_equal(a[2][k], b[2][k]), k


def test_corrupt_checkpoints_are_refused_and_change_nothing(tmp_path):
    d, e, i = wl.reference_start(seed=6, n0=2000, capacity=1 << 14)
    sim = ed.simulation_for([d], ed.FP64, sigma=(SE, SI), de_ev=DE, particles=[(e, i)])
    sim.step(40)
    good = str(tmp_path / "good.bin")
    sim.save_state(0, good)
    raw = open(good, "rb").read()
    ne = int(np.frombuffer(raw[24:32], dtype=np.int64)[0])
    ni = int(np.frombuffer(raw[32:40], dtype=np.int64)[0])
    assert len(raw) == HDR + 32 * (ne + ni)

    def patched(offset, value_bytes):
        b = bytearray(raw)
        b[offset:offset + len(value_bytes)] = value_bytes
        return bytes(b)

    nan = np.array([np.nan]).tobytes()
    cases = {
        "truncated in the ion data": (raw[:-100], EIO),
        "truncated in the header": (raw[:20], EIO),
        "bad magic": (patched(0, b"XDUPICCK"), EIO),
        "other version": (patched(8, np.int32(2).tobytes()), EIO),
        "other N_G": (patched(12, np.int32(d.n_grid + 1).tobytes()), EIO),
        "negative count": (patched(24, np.int64(-5).tobytes()), EIO),
        "longer than its counts": (raw + b"\0" * 8, EIO),
        "count above capacity": (patched(32, np.int64(1 << 20).tobytes()), ECAPACITY),
        "step of another ion phase": (patched(16, np.int64(40 + 3).tobytes()), ESTATE),
        "electron position outside the gap": (patched(HDR + 8 * 17, np.float64(2 * d.gap_m).tobytes()), EINVAL),
        "NaN ion velocity": (patched(HDR + 32 * ne + 8 * ni + 8 * 5, nan), EINVAL),
    }
    before = _snapshot(sim)
    for name, (blob, status) in cases.items():
        path = str(tmp_path / "bad.bin")
        with open(path, "wb") as f:
            f.write(blob)
        with pytest.raises(ed.EdupicError) as ex:
            sim.load_state(0, path)
        assert ex.value.status == status, name
        _same_snapshot(before, _snapshot(sim))
    with pytest.raises(ed.EdupicError) as ex:
        sim.load_state(0, str(tmp_path / "missing.bin"))
    assert ex.value.status == EIO
    # after all refusals the run continues exactly as one that never saw them
    twin = ed.simulation_for([d], ed.FP64, sigma=(SE, SI), de_ev=DE, particles=[(e, i)])
    twin.step(40)
    sim.step(60)
    twin.step(60)
    _same_snapshot(_snapshot(twin), _snapshot(sim))
    assert sim.counters(0) == twin.counters(0)
    # and the good file restores
    sim.load_state(0, good)
    assert sim.counts(0) == (ne, ni, 40)
    os.remove(good)
    sim.close()
    twin.close()


# --------------------------------------------------------------- cancellation
NT = 4000


def _requests(k0, n):
    out = []
    for k in range(n):
        rng = np.random.default_rng(700 + k0 + k)
        d, e, i = wl.draw_discharge(rng, 700 + k0 + k, n_min=2e4, n_max=5e4, steps_per_cycle=NT)
        out.append((d, e, i, 1))
    return out


def _server(slots):
    srv = ed.Server(1 << 30, max_slots=slots, max_grid=800, max_eepf_bins=2000, ion_subcycle=20,
                    cs_entries=SE.shape[1], precision=ed.FP32)
    srv.set_cross_sections(ed.ELECTRONS, SE, DE)
    srv.set_cross_sections(ed.IONS, SI, DE)
    return srv


def _finish(srv, tickets):
    res = {}
    for _ in range(10_000):
        srv.advance(1)
        for j, t in tickets.items():
            if j not in res and srv.info(t)["state"] >= ed.REQ_DONE:
                assert srv.info(t)["state"] == ed.REQ_DONE
                res[j] = srv.result(t)
        if len(res) == len(tickets):
            return res
    raise AssertionError("requests did not finish")


def test_cancelled_request_frees_its_slot_and_leaves_the_others_unchanged():
    a, b, c, q = _requests(0, 4)
    srv = _server(slots=2)
    ta = srv.submit(*a[:3], a[3])
    tb = srv.submit(*b[:3], b[3])
    tc = srv.submit(*c[:3], c[3])  # waits: both slots are busy
    tq = srv.submit(*q[:3], q[3])
    srv.advance(3)
    srv.advance(3)
    assert srv.info(tb)["state"] == ed.REQ_RUNNING and srv.info(tc)["state"] == ed.REQ_QUEUED
    used = srv.stats()["heap_used"]
    srv.release(tq)  # a queued request leaves the queue
    srv.release(tb)  # a running request is cancelled mid-run
    st = srv.stats()
    assert st["running"] == 1 and st["queued"] == 1
    assert st["heap_used"] == used - srv.request_bytes(b[0])
    with pytest.raises(ed.EdupicError):
        srv.info(tb)
    res = _finish(srv, {"a": ta, "c": tc})  # c takes the freed slot
    assert srv.stats()["heap_used"] == 0
    srv.close()
    for key, r in (("a", a), ("c", c)):
        alone_srv = _server(slots=1)
        alone = _finish(alone_srv, {key: alone_srv.submit(*r[:3], r[3])})[key]
        alone_srv.close()
        for k in ("n_e", "n_i", "phi", "eepf_counts", "ifed_pow_counts", "ifed_gnd_counts"):
            assert np.array_equal(res[key][k], alone[k]), (key, k)
        assert res[key]["counters"] == alone["counters"]
