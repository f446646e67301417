"""GB300 (sm_103a) reaction-diffusion stepper.

The hot path -- the forward-Euler method-of-lines step of the paper's
Section 2 with the 7-point Laplacian, reactions, upwind advection and
held boundary layers -- runs in the CUDA library built from ``csrc/`` and
exposed through the C ABI of ``include/rd.h``.  This package holds the
build script, the ctypes binding (``Sim``, ``Batch``), the serving loop and
the seeded workload generators.

Importing the package does not load the CUDA library; creating a ``Sim``
does, and fails loudly when it has not been built.
"""
from .workloads import initial_fields  # noqa: F401


def __getattr__(name):
    if name in ("Sim", "Batch", "make_config", "query_sizes"):
        from . import sim
        return getattr(sim, name)
    raise AttributeError(name)
