"""FP64 oracle runs of the benchmark workloads at their full sizes, computed
in worker processes while the rest of the GPU suite runs.

The oracle is single-threaded (about 10-20 M cell-steps/s on one core), so
200 steps of a 256^3 or 512 x 512 x 64 problem take a few minutes.  Each leg
runs in its own process of a ``spawn`` pool (never forked from a process
that has touched the GPU); the pool is started when the session begins, so
the legs overlap the other tests, and each test waits only for its own leg.
A worker regenerates its inputs from the seeded workload (nothing large is
pickled), runs the oracle unchanged and writes the result to a ``.npy`` file
that the test maps back.

Legs (name -> problem, initial fields, steps):
  brusselator_256        256^3 periodic Brusselator, FP32 initial fields,
                         200 steps
  brusselator_256_bf16   the same from the BF16-rounded initial fields
                         (isolates the per-step storage loss of the BF16
                         variant)
  air_512                512 x 512 x 64 air problem, 200 steps
  ch_batch_<i>           instance i of the 32-instance front batch, 200 steps
                         (the largest and the three smallest instances)
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os
import tempfile

import numpy as np

STEPS = 200


def to_bf16(f):
    """FP32 values rounded to the nearest BF16 (ties to even), as FP32."""
    u = np.ascontiguousarray(f, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32)


def batch_members():
    """Indices of the batch instances compared: the three smallest, the largest."""
    from paper_1004_0480_gb300 import workloads as W
    sizes = W.batch_sizes_ch()
    order = np.argsort(sizes, kind="stable")
    return [int(i) for i in order[:3]] + [int(order[-1])]


def leg_inputs(name):
    """(problem, initial fields) of a leg, from the seeded workloads."""
    from paper_1004_0480_gb300 import workloads as W
    if name == "brusselator_256":
        cfg = W.cfg_brusselator_256()
        return cfg, W.initial_fields(cfg)
    if name == "brusselator_256_bf16":
        cfg = W.cfg_brusselator_256()
        return cfg, to_bf16(W.initial_fields(cfg))
    if name == "air_512":
        cfg = W.cfg_air_512()
        return cfg, W.initial_fields(cfg)
    if name.startswith("ch_batch_"):
        cfg = W.cfg_ch_front_batch()[int(name[len("ch_batch_"):])]
        return cfg, W.initial_fields(cfg)
    raise KeyError(name)


def leg_names():
    return (["brusselator_256", "brusselator_256_bf16", "air_512"]
            + [f"ch_batch_{i}" for i in batch_members()])


def _run_leg(name, out_dir):
    """Worker: the oracle on one leg; returns the path of its result."""
    import oracle
    cfg, f = leg_inputs(name)
    ref = oracle.run(cfg, f, STEPS)
    path = os.path.join(out_dir, name + ".npy")
    np.save(path, ref)
    return path


class Legs:
    """The running legs of one session."""

    def __init__(self):
        import oracle
        oracle.build()          # once, before the workers load it
        self.dir = tempfile.mkdtemp(prefix="rd_fullsize_")
        names = leg_names()
        self.pool = cf.ProcessPoolExecutor(max_workers=min(len(names), os.cpu_count() or 1),
                                           mp_context=mp.get_context("spawn"))
        self.futures = {n: self.pool.submit(_run_leg, n, self.dir) for n in names}

    def result(self, name, timeout=1500):
        """The oracle's fields after STEPS steps (float64, read-only map)."""
        return np.load(self.futures[name].result(timeout=timeout), mmap_mode="r")

    def close(self):
        for f in self.futures.values():
            f.cancel()
        # the workers are this session's own processes: end the ones still
        # running a leg instead of waiting minutes for them
        procs = list(getattr(self.pool, "_processes", {}).values())
        for p in procs:
            if p.is_alive():
                p.terminate()
        self.pool.shutdown(wait=True, cancel_futures=True)
        for name in os.listdir(self.dir):
            os.unlink(os.path.join(self.dir, name))
        os.rmdir(self.dir)


_LEGS = None


def start():
    """Start the legs once per session (idempotent)."""
    global _LEGS
    if _LEGS is None:
        _LEGS = Legs()
    return _LEGS


def stop():
    global _LEGS
    if _LEGS is not None:
        _LEGS.close()
        _LEGS = None
