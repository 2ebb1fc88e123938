"""GB300-native batched 4-center electron-repulsion integrals (ab|cd) by the matrix form
of the McMurchie-Davidson recurrences (Asadchev & Valeev, arXiv:2307.03452).

The compute path is the CUDA library ``liblx_eri.so`` (C ABI in ``include/lx_eri.h``);
``lx`` is its Python binding and ``inputs`` draws seeded synthetic workloads.
"""
from . import inputs, lx  # noqa: F401

__all__ = ["inputs", "lx"]
