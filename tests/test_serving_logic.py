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
    """Steps cost cells * steps / rate seconds; families run concurrently and
    independently: a family's chunk completes at its own time on the fake
    clock."""

    def __init__(self, clock, rate=1e6):
        self.clock, self.rate = clock, rate
        self.members = {}        # family -> running requests
        self.step_log = []       # (family, n, ids of the running requests)
        self.done_at = {}        # family -> fake time its last chunk completes
        self.used = 0
        self.peak = 0
        self.budget_seen = []
        self.admit_order = []
        self.steps_done = {}
        self.nlaunch = 0

    def bytes_for(self, req):
        return req.cells * req.cfg["nspecies"] * 8

    def open(self, req):
        self.used += self.bytes_for(req)
        self.peak = max(self.peak, self.used)
        self.admit_order.append(req.id)
        self.steps_done[req.id] = 0
        return req

    def start(self, fam, handle):
        self.members.setdefault(fam, []).append(handle)

    def step(self, fam, n, high=False):
        assert not self.busy(fam), "a family is stepped only when idle"
        self.step_log.append((fam, n, sorted(r.id for r in self.members[fam])))
        work = sum(r.cells for r in self.members[fam]) * n
        self.done_at[fam] = self.clock.t + work / self.rate
        for r in self.members[fam]:
            self.steps_done[r.id] += n
        self.nlaunch += n

    def busy(self, fam):
        return self.clock.t < self.done_at.get(fam, float("-inf"))

    def wait_any(self, fams, timeout):
        nxt = min(self.done_at[f] for f in fams)
        self.clock.t = max(self.clock.t, min(nxt, self.clock.t + max(timeout, 0.0)))

    def sync(self, fam=None):
        if self.done_at:
            self.clock.t = max(self.clock.t, max(self.done_at.values()))

    def result(self, handle):
        return None

    def close(self, fam, handle):
        if handle in self.members.get(fam, []):
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


def test_running_set_is_the_oldest_requests_up_to_run_cells():
    clk = FakeClock()
    eng = FakeEngine(clk)
    # 10^3 cells each; request 0 needs 10 steps, the others 30
    reqs = [mk(i, 0.0, 10, 10 if i == 0 else 30) for i in range(4)]
    res, st = Server(eng, budget_bytes=1e12, quantum=10, run_cells=2500, clock=clk,
                     sleep=clk.sleep).run(reqs)
    # first tick: 0, 1, 2 (2000 cells < 2500 before 2 joins, 3000 after)
    assert eng.step_log[0] == ("brusselator", 10, [0, 1, 2])
    # request 0 retired after that tick; 3 joins the running set
    assert eng.step_log[1] == ("brusselator", 10, [1, 2, 3])
    assert st.max_active == 4 and st.max_running == 3
    assert all(eng.steps_done[r.id] == r.steps for r in reqs)


def test_a_request_that_fills_the_gpu_runs_alone_in_arrival_order():
    clk = FakeClock()
    eng = FakeEngine(clk)
    reqs = [mk(i, 0.001 * i, 10, 20 + i, ["brusselator", "ch_front"][i % 2]) for i in range(5)]
    res, st = Server(eng, budget_bytes=1e12, quantum=8, run_cells=1000, clock=clk,
                     sleep=clk.sleep).run(reqs)
    assert st.max_running == 1
    assert [r.id for r in sorted(res, key=lambda r: r.finished)] == list(range(5))
    assert all(len(ids) == 1 for _, _, ids in eng.step_log)


def test_unbounded_running_set_advances_every_admitted_request():
    clk = FakeClock()
    eng = FakeEngine(clk)
    reqs = [mk(i, 0.0, 10, 50) for i in range(6)]
    _, st = Server(eng, budget_bytes=1e12, quantum=25, run_cells=float("inf"), clock=clk,
                   sleep=clk.sleep).run(reqs)
    assert st.max_running == 6
    assert eng.step_log[0] == ("brusselator", 25, list(range(6)))


def test_percentiles():
    assert percentile([3, 1, 2], 50) == 2
    assert percentile(list(range(101)), 99) == pytest.approx(99.0)
    st = summarize([], 1.0, 0, 0)
    assert st.n == 0


def test_families_run_independently():
    # a large diffusion request runs long chunks; small Brusselator requests
    # arriving meanwhile finish long before it, without waiting for its
    # chunks to end
    clk = FakeClock()
    eng = FakeEngine(clk)
    big = mk(0, 0.0, 60, 400, "diffusion")          # 216 000 cells x 400 steps
    small = [mk(i, 0.01 * i, 8, 20) for i in range(1, 5)]
    res, st = Server(eng, budget_bytes=1e12, quantum=200, clock=clk, sleep=clk.sleep,
                     poll_s=0.005).run([big] + small)
    lat = {r.id: r.latency for r in res}
    chunk = 216000 * 200 / eng.rate                   # one chunk of the big request
    assert all(lat[i] < 0.2 * chunk for i in range(1, 5))
    assert lat[0] >= 2 * chunk
    assert all(eng.steps_done[r.id] == r.steps for r in [big] + small)


def test_a_finished_request_never_takes_more_steps():
    # members of one family with different step counts: each stops exactly
    # at its count although the family keeps running
    clk = FakeClock()
    eng = FakeEngine(clk)
    reqs = [mk(i, 0.0, 10, 7 + 11 * i) for i in range(5)]
    Server(eng, budget_bytes=1e12, quantum=9, clock=clk, sleep=clk.sleep).run(reqs)
    assert all(eng.steps_done[r.id] == r.steps for r in reqs)

