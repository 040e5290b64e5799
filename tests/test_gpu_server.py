"""The request server (continuous batching) through the C ABI.

A request's results must not depend on what runs beside it: every request
is compared bit for bit between a mixed run (requests admitted while others
are running, queued when slots are full) and a run alone, and with a plain
simulation object stepped for the same number of steps.
"""
import dataclasses

import numpy as np
import pytest

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
NT = 4000  # time steps per RF cycle (the paper's N_T)


def _requests(k0=0, n=4):
    out = []
    for k in range(n):
        rng = np.random.default_rng(900 + k0 + k)
        d, e, i = wl.draw_discharge(rng, 900 + k0 + k, n_min=2e4, n_max=6e4, steps_per_cycle=NT)
        out.append((d, e, i, 1 + k % 2))
    return out


def _server(precision, slots, budget=1 << 30):
    srv = ed.Server(budget, max_slots=slots, max_grid=800, max_eepf_bins=2000, ion_subcycle=20,
                    cs_entries=SE.shape[1], precision=precision)
    srv.set_cross_sections(ed.ELECTRONS, SE, DE)
    srv.set_cross_sections(ed.IONS, SI, DE)
    return srv


def _serve(srv, reqs, arrivals, allow_fail=()):
    """Submit request j at scheduling round arrivals[j]; advance one ion
    subcycle per round until every request has finished."""
    tickets = {}
    results = {}
    rnd = 0
    while len(results) < len(reqs):
        for j, a in enumerate(arrivals):
            if a == rnd:
                d, e, i, nc = reqs[j]
                tickets[j] = srv.submit(d, e, i, nc)
        srv.advance(1)
        for j, t in tickets.items():
            if j in results:
                continue
            inf = srv.info(t)
            if inf["state"] >= ed.REQ_DONE:
                if inf["state"] == ed.REQ_FAILED and j in allow_fail:
                    results[j] = (None, inf)
                    continue
                assert inf["state"] == ed.REQ_DONE, f"request {j} failed: {inf['status']}"
                results[j] = (srv.result(t), inf)
        rnd += 1
        assert rnd < 10_000
    return results


def _same(a, b):
    for k in ("n_e", "n_i", "phi", "eepf_counts", "ifed_pow_counts", "ifed_gnd_counts"):
        assert np.array_equal(a[k], b[k]), k
    assert a["counters"] == b["counters"]
    assert a["measured_steps"] == b["measured_steps"]


@pytest.mark.parametrize("precision", [ed.FP64, ed.FP32])
def test_results_same_alone_and_in_the_mix(precision):
    reqs = _requests()
    # two slots: requests 2 and 3 arrive while 0 and 1 run and wait for a slot
    mixed = _serve(_server(precision, slots=2), reqs, arrivals=[0, 0, 3, 5])
    for j, r in enumerate(reqs):
        alone = _serve(_server(precision, slots=1), [r], arrivals=[0])
        _same(mixed[j][0], alone[0][0])
        assert mixed[j][0]["measured_steps"] == r[3] * NT
        assert mixed[j][1]["steps_done"] == r[3] * NT
    # continuous batching: the late requests were admitted while others ran
    t_done01 = max(mixed[0][1]["t_done"], mixed[1][1]["t_done"])
    assert min(mixed[2][1]["t_admit"], mixed[3][1]["t_admit"]) < t_done01


def test_server_equals_plain_simulation():
    d, e, i, nc = _requests(k0=20, n=1)[0]
    res = _serve(_server(ed.FP64, slots=3), [(d, e, i, nc)], arrivals=[0])[0][0]
    sim = ed.simulation_for([d], ed.FP64, sigma=(SE, SI), de_ev=DE, particles=[(e, i)])
    sim.step(nc * NT, measure=True)
    diag = sim.diagnostics(0)
    for k in ("n_e", "n_i", "phi", "eepf_counts", "ifed_pow_counts", "ifed_gnd_counts"):
        assert np.array_equal(res[k], diag[k]), k
    assert res["counters"] == sim.counters(0)


def test_admission_waits_for_memory():
    reqs = _requests(k0=40, n=2)
    probe = _server(ed.FP32, slots=4)
    need = [probe.request_bytes(r[0]) for r in reqs]
    probe.close()
    # heap room for the larger request and half the smaller one: one at a time
    heap = max(need) + min(need) // 2
    budget = ed.server_arena_bytes(heap, max_slots=4, max_grid=800, max_eepf_bins=2000, ion_subcycle=20,
                                   cs_entries=SE.shape[1], precision=ed.FP32)
    srv = _server(ed.FP32, slots=4, budget=budget)
    res = _serve(srv, reqs, arrivals=[0, 0])
    first, second = sorted(res.values(), key=lambda r: r[1]["t_admit"])
    assert second[1]["t_admit"] >= first[1]["t_done"]
    # a request that can never fit the heap is refused at submission
    d, e, i, _ = reqs[0]
    with pytest.raises(ed.EdupicError):
        srv.submit(dataclasses.replace(d, capacity=20_000_000), e, i, 1)


def test_failing_request_leaves_the_others_unchanged():
    good = _requests(k0=60, n=1)[0]
    # a few hundred superparticles over hundreds of cells: the charge noise
    # drives an ionisation avalanche that overflows the particle capacity
    rng = np.random.default_rng(901)
    d, e, i = wl.draw_discharge(rng, 901, scale=0.004, steps_per_cycle=NT)
    bad = (d, e, i, 2)
    mixed = _serve(_server(ed.FP32, slots=2), [good, bad], arrivals=[0, 0], allow_fail=(1,))
    assert mixed[1][1]["state"] == ed.REQ_FAILED and mixed[1][1]["status"] == -3  # EDUPIC_ECAPACITY
    alone = _serve(_server(ed.FP32, slots=1), [good], arrivals=[0])
    _same(mixed[0][0], alone[0][0])
