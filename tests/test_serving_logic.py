"""Scheduling logic of the continuous-batching server, on the CPU with a
fake engine and a fake clock (no GPU work)."""
import pytest

from paper_1004_0480_gb300 import workloads as W
from paper_1004_0480_gb300.serving import (Request, Server, percentile, serve_plain,
                                           summarize)


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 0.0)


class FakeEngine:
    """Steps cost cells * steps / rate seconds; families run concurrently
    (a tick costs the slowest family's work)."""

    def __init__(self, clock, rate=1e6):
        self.clock, self.rate = clock, rate
        self.members = {}
        self.pending = {}
        self.used = 0
        self.peak = 0
        self.budget_seen = []
        self.admit_order = []
        self.steps_done = {}
        self.nlaunch = 0

    def bytes_for(self, req):
        return req.cells * req.cfg["nspecies"] * 8

    def open(self, req):
        self.members.setdefault(req.family, []).append(req)
        self.used += self.bytes_for(req)
        self.peak = max(self.peak, self.used)
        self.admit_order.append(req.id)
        self.steps_done[req.id] = 0
        return req

    def step(self, fam, n):
        work = sum(r.cells for r in self.members[fam]) * n
        self.pending[fam] = self.pending.get(fam, 0.0) + work / self.rate
        for r in self.members[fam]:
            self.steps_done[r.id] += n
        self.nlaunch += n

    def sync(self, fam=None):
        if self.pending:
            self.clock.t += max(self.pending.values())
            self.pending.clear()

    def result(self, handle):
        return None

    def close(self, fam, handle):
        self.members[fam].remove(handle)
        self.used -= self.bytes_for(handle)

    def launches(self):
        return self.nlaunch

    def run_alone(self, req, collect):
        self.clock.t += req.cells * req.steps / self.rate
        self.steps_done[req.id] = req.steps
        return None, req.steps


def mk(i, arrival, n, steps, kind="brusselator"):
    f = {"brusselator": W.brusselator, "diffusion": W.diffusion_blob,
         "ch_front": W.ch_front}[kind]
    return Request(i, arrival, f(n, steps=steps))


def test_every_request_completes_with_its_step_count():
    clk = FakeClock()
    eng = FakeEngine(clk)
    reqs = [mk(i, 0.01 * i, 8 + i, 30 + 17 * i, ["brusselator", "diffusion", "ch_front"][i % 3])
            for i in range(12)]
    res, st = Server(eng, budget_bytes=1e12, quantum=25, clock=clk, sleep=clk.sleep).run(reqs)
    assert sorted(r.id for r in res) == list(range(12))
    assert all(eng.steps_done[r.id] == r.steps for r in reqs)
    assert all(r.finished >= r.admitted >= r.arrival for r in res)
    assert st.p50 <= st.p99
    assert st.n == 12 and st.glups > 0


def test_budget_is_never_exceeded_and_admission_is_fifo():
    clk = FakeClock()
    eng = FakeEngine(clk)
    reqs = [mk(i, 0.0, 16, 100) for i in range(6)]
    one = eng.bytes_for(reqs[0])
    budget = 2.5 * one                     # room for two at a time
    res, st = Server(eng, budget_bytes=budget, quantum=40, clock=clk, sleep=clk.sleep).run(reqs)
    assert eng.peak <= budget
    assert st.max_active == 2
    assert eng.admit_order == list(range(6))
    assert len(res) == 6


def test_late_arrivals_wait_for_the_clock_and_a_request_too_big_is_refused():
    clk = FakeClock()
    eng = FakeEngine(clk)
    reqs = [mk(0, 5.0, 8, 10)]
    res, _ = Server(eng, budget_bytes=1e12, quantum=10, clock=clk, sleep=clk.sleep).run(reqs)
    assert res[0].admitted >= 5.0
    with pytest.raises(ValueError):
        Server(FakeEngine(clk), budget_bytes=10, clock=clk, sleep=clk.sleep).run([mk(1, 0.0, 8, 5)])


def test_batching_beats_serial_plain_on_the_fake_engine():
    # with families running concurrently, batching finishes the same work sooner
    reqs = [mk(i, 0.0, 12, 200, ["brusselator", "diffusion", "ch_front"][i % 3]) for i in range(9)]
    c1 = FakeClock()
    _, batched = Server(FakeEngine(c1), budget_bytes=1e12, quantum=50, clock=c1,
                        sleep=c1.sleep).run(reqs)
    c2 = FakeClock()
    _, plain = serve_plain(FakeEngine(c2), reqs, clock=c2, sleep=c2.sleep)
    assert batched.makespan < plain.makespan
    assert batched.p99 <= plain.p99


def test_percentiles():
    assert percentile([3, 1, 2], 50) == 2
    assert percentile(list(range(101)), 99) == pytest.approx(99.0)
    st = summarize([], 1.0, 0, 0)
    assert st.n == 0
