"""DADE-IVF on GB300: data-aware distance comparisons inside an IVF scan.

The compute path is the C-ABI library ``libdade.so`` (hand-written CUDA for
sm_103a, declared in include/dade.h).  ``paper_2411_17229_gb300.dade`` is its
thin ctypes binding; ``synth`` draws seeded synthetic workloads.  Importing
this package loads nothing; the library is loaded on first use and a missing
build raises instead of falling back to any CPU code.
"""
