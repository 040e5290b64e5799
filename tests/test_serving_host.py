"""Host logic of the request stream driver (no GPU): arrival order, retiring,
time-to-result bookkeeping and percentiles, against a fake server whose
requests each take a fixed number of scheduling rounds."""
import numpy as np

from paper_2103_09642_gb300 import serving
from paper_2103_09642_gb300 import workloads as wl


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeServer:
    """Requests run for n_cycles rounds; `slots` at a time; FIFO admission.
    Every advance() call moves the clock by `round_s`."""

    def __init__(self, clock, slots=2, round_s=0.1):
        self.clock, self.slots, self.round_s = clock, slots, round_s
        self.reqs, self.queue, self.running, self.next = {}, [], [], 1
        self.submitted = []

    def stats(self):
        return {"now": self.clock()}

    def request_bytes(self, d):
        return 1024

    def submit(self, d, e, i, n_cycles):
        t = self.next
        self.next += 1
        self.reqs[t] = {"left": n_cycles, "state": 0, "t_admit": -1.0, "t_done": -1.0, "n": e.n + i.n,
                        "steps": n_cycles}
        self.queue.append(t)
        self.submitted.append((t, self.clock()))
        return t

    def advance(self, k):
        for t in list(self.running):
            r = self.reqs[t]
            if r["left"] <= 0:
                r["state"], r["t_done"] = 2, self.clock()
                self.running.remove(t)
        while self.queue and len(self.running) < self.slots:
            t = self.queue.pop(0)
            self.reqs[t]["state"], self.reqs[t]["t_admit"] = 1, self.clock()
            self.running.append(t)
        for t in self.running:
            self.reqs[t]["left"] -= 1
        if self.running:
            self.clock.t += self.round_s
        return len(self.running), len(self.queue)

    def info(self, t):
        r = self.reqs[t]
        return {"state": r["state"], "status": 0, "t_admit": r["t_admit"], "t_done": r["t_done"],
                "steps_done": r["steps"]}

    def result(self, t):
        return {"counters": {"push_e": self.reqs[t]["n"], "push_i": 0}}

    def release(self, t):
        pass


def _specs(arrivals, cycles):
    out = []
    for k, (a, c) in enumerate(zip(arrivals, cycles)):
        d, e, i = wl.draw_discharge(np.random.default_rng(k), k, scale=0.001, steps_per_cycle=400)
        out.append(serving.RequestSpec(a, c, d, e, i))
    return out


def test_percentile_nearest_rank():
    v = list(range(1, 101))
    assert serving.percentile(v, 50) == 50
    assert serving.percentile(v, 99) == 99
    assert serving.percentile(v, 100) == 100
    assert serving.percentile([7.0], 99) == 7.0
    assert serving.percentile([], 50) is None


def test_stream_respects_arrivals_and_fifo():
    clk = FakeClock()
    srv = FakeServer(clk, slots=1, round_s=0.1)
    specs = _specs([0.0, 0.05, 1.0], [3, 2, 1])
    rep = serving.run_stream(srv, specs, clock=clk, sleep=clk.sleep)
    assert rep["requests"] == 3 and rep["failed"] == 0
    # submitted no earlier than their arrival, in arrival order
    subs = [s for _, s in srv.submitted]
    assert all(s >= a for s, a in zip(subs, [0.0, 0.05, 1.0])) and subs == sorted(subs)
    log = {r["ticket"]: r for r in rep["log"]}
    # one slot: request 2 is admitted only after request 1 is done
    assert log[2]["admit_s"] >= log[1]["done_s"]
    for r in rep["log"]:
        assert abs(r["time_to_result_s"] - (r["done_s"] - r["arrival_s"])) < 1e-12
        assert r["time_to_result_s"] > 0
    ttr = sorted(r["time_to_result_s"] for r in rep["log"])
    assert rep["p50_time_to_result_s"] == ttr[1] and rep["p99_time_to_result_s"] == ttr[2]
    assert rep["particle_steps"] == sum(s.electrons.n + s.ions.n for s in specs)


def test_poisson_stream_rate_and_ranges():
    specs = serving.poisson_stream(400, rate_hz=2.0, seed=3, cycles=(20, 200), scale=0.0005)
    gaps = np.diff([0.0] + [s.arrival_s for s in specs])
    assert abs(gaps.mean() - 0.5) < 0.1  # mean inter-arrival 1/rate
    assert all(20 <= s.n_cycles <= 200 for s in specs)
    assert all(0.015 <= s.discharge.gap_m <= 0.05 and 200 <= s.discharge.n_grid <= 800 for s in specs)


def test_stream_gives_up_after_its_wall_bound():
    clk = FakeClock()
    srv = FakeServer(clk, slots=0, round_s=0.0)  # nothing is ever admitted
    specs = _specs([0.0], [1])

    def advance(k):
        clk.t += 0.5
        return 0, len(srv.queue)

    srv.advance = advance
    import pytest

    with pytest.raises(TimeoutError):
        serving.run_stream(srv, specs, clock=clk, sleep=clk.sleep, max_wall_s=5.0)
