"""Continuous-batching server for reaction-diffusion requests.

Requests (a problem, an arrival time, a step count) arrive over time.  The
server admits them in arrival order as soon as their device memory fits a
budget and keeps their state resident.  The oldest admitted requests, up to
``run_cells`` cells in all (at least one request), are running: those of one
kinetics family advance together with one batched launch sequence per tick
(``rd_batch_step``), each family on its own stream so the families' kernels
overlap on the device.  A request is retired the moment its step count is
reached; its memory is freed, the next admitted requests start running and
the next arrivals can be admitted.  Reports per-request latency (finish -
arrival), p50/p99 and aggregate GLUPS.

Each tick the family of the oldest running request gets a high-priority
stream, so that request's kernels are scheduled first where families
compete for SMs.

The running set is a first-come-first-served prefix sized to fill the GPU:
small requests share it (batching is what gets them past the launch-bound
regime of one small grid), while a request that fills the GPU by itself
runs nearly alone instead of being slowed by everything admitted after it,
as it would be if every admitted request advanced at once.

``serve_plain`` is the baseline: one request at a time in arrival order,
each stepped alone by the plain stepper (the fused kernel at one step per
launch, no graph).

The scheduling logic talks to an engine object, so it can run on the CPU
with a fake engine and a fake clock (see the tests); ``CudaEngine`` is the
real one, on the C ABI.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import workloads as W


@dataclass
class Request:
    id: int
    arrival: float          # seconds after the start of the run
    cfg: dict               # problem (workloads format); cfg["steps"] steps

    @property
    def steps(self):
        return int(self.cfg["steps"])

    @property
    def family(self):
        return self.cfg["model"]

    @property
    def cells(self):
        return W.cell_count(self.cfg)


@dataclass
class Result:
    id: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    cells: int
    fields: np.ndarray | None = None

    @property
    def latency(self):
        return self.finished - self.arrival


@dataclass
class Stats:
    n: int
    makespan: float
    glups: float
    p50: float
    p99: float
    mean: float
    max_bytes: int
    max_active: int
    launches: int = 0
    max_running: int = 0
    extra: dict = field(default_factory=dict)


def percentile(xs, q):
    """q-th percentile (0..100) with linear interpolation."""
    if not xs:
        return float("nan")
    xs = sorted(xs)
    k = (len(xs) - 1) * q / 100.0
    lo = math.floor(k)
    hi = min(lo + 1, len(xs) - 1)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def summarize(results, makespan, max_bytes, max_active, launches=0, max_running=0):
    lat = [r.latency for r in results]
    work = sum(r.cells * r.steps for r in results)
    return Stats(n=len(results), makespan=makespan,
                 glups=work / makespan / 1e9 if makespan > 0 else float("nan"),
                 p50=percentile(lat, 50), p99=percentile(lat, 99),
                 mean=float(np.mean(lat)) if lat else float("nan"),
                 max_bytes=max_bytes, max_active=max_active, launches=launches,
                 max_running=max_running)


# --------------------------------------------------------------- engines
class CudaEngine:
    """Requests as contexts of the CUDA library; one batch per family."""

    def __init__(self, storage="f32", batch_tuning=None):
        import torch

        from .sim import Batch, Sim, query_sizes
        self._torch = torch
        self._Sim = Sim
        self._Batch = Batch
        self._query = query_sizes
        self.storage = storage
        self.batch_tuning = batch_tuning or {}
        self.batches = {}
        self.streams = {}
        self.on_high = {}
        self.events = {}
        self.running = set()

    def bytes_for(self, req):
        st, sc = self._query(req.cfg, self.storage)
        return st + sc

    def _new_sim(self, req):
        # torch-owned memory: retiring a request returns it to torch's cache
        # instead of a device-synchronising cudaFree
        sim = self._Sim(req.cfg, self.storage, torch_memory=True)
        f = W.initial_fields_torch(req.cfg, "cuda")
        sim.set_fields(f)
        del f
        return sim

    def open(self, req):
        """Admit: allocate the request's state and set its initial fields."""
        return self._new_sim(req)

    def start(self, family, handle):
        """The request joins its family's batch and advances from now on."""
        if family not in self.batches:
            # a normal and a high-priority stream per family (see prioritize)
            lo, hi = self._torch.cuda.Stream.priority_range()
            pair = (self._torch.cuda.Stream(priority=lo), self._torch.cuda.Stream(priority=hi))
            b = self._Batch(family, self.storage, stream=pair[0])
            tun = self.batch_tuning.get(family)
            if tun:
                b.set_tuning(**tun)
            self.batches[family] = b
            self.streams[family] = pair
            self.on_high[family] = False
        self.batches[family].add(handle)
        self.running.add(id(handle))

    def _stream_for(self, family, high):
        """Put ``family``'s batch on its high- or normal-priority stream.  Only
        called while the family is idle, so the switch waits for nothing."""
        if self.on_high[family] != high:
            self.batches[family].set_stream(self.streams[family][1 if high else 0])
            self.on_high[family] = high

    def step(self, family, n, high=False):
        """Enqueue n steps of the family's batch and record an event after
        them; returns at once.  ``high``: on the family's high-priority
        stream (the family holding the oldest running request), so where
        families compete for SMs its kernels are scheduled first."""
        self._stream_for(family, high)
        self.batches[family].step(n)
        ev = self._torch.cuda.Event()
        ev.record(self.streams[family][1 if high else 0])
        self.events[family] = ev

    def step_each(self, family, counts, high=False):
        """As ``step``, each running request of the family advancing its own
        count (``counts``: (handle, steps) pairs; one batched launch sequence
        of the largest count, members whose count is used up left alone)."""
        self._stream_for(family, high)
        self.batches[family].step_each(dict(counts))
        ev = self._torch.cuda.Event()
        ev.record(self.streams[family][1 if high else 0])
        self.events[family] = ev

    def busy(self, family):
        """True while the family's last enqueued steps have not completed
        (cudaEventQuery: no synchronisation)."""
        ev = self.events.get(family)
        return ev is not None and not ev.query()

    def wait_any(self, families, timeout_s):
        """Return when one of ``families`` is idle or after timeout_s."""
        deadline = time.perf_counter() + max(timeout_s, 0.0)
        while True:
            if any(not self.busy(f) for f in families):
                return
            if time.perf_counter() >= deadline:
                return
            time.sleep(5e-5)

    def sync(self, family=None):
        fams = [family] if family else list(self.batches)
        for f in fams:
            self.batches[f].sync()

    def result(self, handle):
        return handle.get_fields()

    def close(self, family, handle):
        if id(handle) in self.running:
            self.batches[family].remove(handle)
            self.running.discard(id(handle))
        handle.close()

    def launches(self):
        return sum(b.launches for b in self.batches.values())

    def shutdown(self):
        for b in self.batches.values():
            b.close()
        self.batches.clear()

    # plain stepper: one request alone, one launch per step, no graph
    def run_alone(self, req, collect):
        sim = self._new_sim(req)
        sim.set_tuning(tsteps=1, graph=0)
        sim.step(req.steps)
        sim.sync()
        out = sim.get_fields() if collect else None
        launches = sim.launches
        sim.close()
        return out, launches


# ---------------------------------------------------------------- server
class Server:
    """Continuous batching under a device-memory budget.

    Each kinetics family's running requests form one batch on its own
    stream, and the families run asynchronously: whenever a family's last
    chunk has completed (its event, polled without synchronising the
    device), the server retires that family's finished requests, lets the
    next admitted requests join it, and enqueues its next chunk, while the
    other families keep running.  Arrivals are admitted between polls.

    ``quantum``    steps per chunk of a family batch (a chunk never steps a
                   request past its count: the batch advances by the smallest
                   remaining count if that is smaller, so the request that
                   finishes retires as soon as the chunk completes)
    ``budget``     bytes of device memory the admitted requests may hold
    ``run_cells``  cells the running requests may hold together: requests
                   start in admission order while the running ones hold
                   fewer (so the oldest always runs); ``inf`` runs every
                   admitted request at once
    ``clock``      seconds (monotonic); ``sleep`` waits for the next arrival
    """

    def __init__(self, engine, budget_bytes=120e9, quantum=200, run_cells=48e6,
                 clock=time.perf_counter, sleep=time.sleep, progress=None, poll_s=0.02):
        self.progress = progress     # called as progress(t, admitted, running, done)
        self.engine = engine
        self.budget = float(budget_bytes)
        self.quantum = int(quantum)
        self.run_cells = float(run_cells)
        self.clock = clock
        self.sleep = sleep
        self.poll_s = float(poll_s)  # longest wait before new arrivals are looked at

    def run(self, requests, collect_fields=False):
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.id)))
        for r in pending:
            if self.engine.bytes_for(r) > self.budget:
                raise ValueError(f"request {r.id} alone exceeds the memory budget")
        admitted = []            # slots in admission order
        results = []
        used = 0
        max_used = 0
        max_active = 0
        max_running = 0
        t0 = self.clock()
        while pending or admitted:
            now = self.clock() - t0
            # ---- admit arrivals, first come first served, while memory allows
            while pending and pending[0].arrival <= now:
                req = pending[0]
                need = self.engine.bytes_for(req)
                if used + need > self.budget:
                    break
                pending.popleft()
                handle = self.engine.open(req)
                used += need
                max_used = max(max_used, used)
                admitted.append(dict(req=req, handle=handle, left=req.steps, bytes=need,
                                     admitted=self.clock() - t0, running=False))
            max_active = max(max_active, len(admitted))
            # ---- which families are idle: one snapshot per pass, so a family
            # that completes during the pass is not relaunched before its
            # finished requests have left the batch
            idle = {}
            for s in admitted:
                f = s["req"].family
                if f not in idle:
                    idle[f] = not self.engine.busy(f)
            # ---- retire the finished requests of idle families
            done_at = self.clock() - t0
            for s in [s for s in admitted if s["running"] and s["left"] == 0
                      and idle[s["req"].family]]:
                req = s["req"]
                fields = self.engine.result(s["handle"]) if collect_fields else None
                results.append(Result(req.id, req.arrival, s["admitted"], done_at, req.steps,
                                      req.cells, fields))
                self.engine.close(req.family, s["handle"])
                used -= s["bytes"]
                admitted.remove(s)
            if not admitted:
                if pending:
                    wait = pending[0].arrival - (self.clock() - t0)
                    if wait > 0:
                        self.sleep(wait)
                continue
            # ---- the running set: the oldest admitted requests up to
            # run_cells; a request joins its family when the family is idle
            cells = 0
            for s in admitted:
                if cells >= self.run_cells:
                    break
                if not s["running"]:
                    if not idle[s["req"].family]:
                        cells += s["req"].cells
                        continue
                    self.engine.start(s["req"].family, s["handle"])
                    s["running"] = True
                cells += s["req"].cells
            running = [s for s in admitted if s["running"]]
            max_running = max(max_running, len(running))
            # ---- every idle family with unfinished running requests gets its
            # next chunk; the family of the oldest running request goes on its
            # high-priority stream
            by_family = collections.OrderedDict()
            for s in running:
                if s["left"] > 0:
                    by_family.setdefault(s["req"].family, []).append(s)
            oldest = running[0]["req"].family if running else None
            for fam, slots in by_family.items():
                if not idle[fam]:
                    continue
                # the chunk ends when its first member finishes, so that
                # member retires at once (per-member counts, step_each,
                # would let the others run on, but the finished member
                # then waits for the chunk's end: a longer tail, measured)
                n = min(self.quantum, min(s["left"] for s in slots))
                self.engine.step(fam, n, high=(fam == oldest))
                for s in slots:
                    s["left"] -= n
            if self.progress:
                self.progress(self.clock() - t0, len(admitted), len(running), len(results))
            # ---- wait for a family to go idle (or the next arrival)
            fams = {s["req"].family for s in running}
            busy = [f for f in fams if self.engine.busy(f)]
            if busy and len(busy) == len(fams):
                timeout = self.poll_s
                ahead = pending[0].arrival - (self.clock() - t0) if pending else 0.0
                if ahead > 0:            # wake up for an arrival still to come
                    timeout = min(timeout, ahead)
                self.engine.wait_any(busy, timeout)
        self.engine.sync()
        makespan = self.clock() - t0
        launches = self.engine.launches()
        return results, summarize(results, makespan, max_used, max_active, launches, max_running)


def serve_plain(engine, requests, collect_fields=False, clock=time.perf_counter,
                sleep=time.sleep, progress=None):
    """Baseline: requests one at a time in arrival order, each alone."""
    order = sorted(requests, key=lambda r: (r.arrival, r.id))
    results = []
    launches = 0
    t0 = clock()
    for req in order:
        now = clock() - t0
        if req.arrival > now:
            sleep(req.arrival - now)
        admitted = clock() - t0
        fields, nl = engine.run_alone(req, collect_fields)
        launches += nl
        results.append(Result(req.id, req.arrival, admitted, clock() - t0, req.steps, req.cells,
                               fields))
        if progress:
            progress(clock() - t0, 1, 1, len(results))
    makespan = clock() - t0
    return results, summarize(results, makespan, 0, 1, launches)


def requests_from_workload(specs):
    """Request objects from ``workloads.serving_requests`` entries."""
    return [Request(s["id"], s["arrival"], s["cfg"]) for s in specs]


def with_rate(requests, rate_per_s, seed=4):
    """The same requests with Poisson arrivals of the given rate."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=len(requests))
    t = np.cumsum(gaps) - gaps[0]
    return [Request(r.id, float(t[i]), r.cfg) for i, r in enumerate(requests)]
