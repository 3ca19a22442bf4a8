"""Failure paths that need no GPU: allocation failures injected on the host.

The library's allocation hook (dade_set_alloc_hook) refuses device
allocations on request; a build must then return DADE_ENOMEM with the hook
named in the message, having asked for exactly the bytes its first staging
buffer needs, and leave no index behind.  No CUDA call runs before that first
allocation, so this holds on a host without a GPU.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2411_17229_gb300 import dade

HOOK = C.CFUNCTYPE(C.c_int, C.c_size_t, C.c_void_p)


@pytest.fixture(scope="module")
def lib():
    from paper_2411_17229_gb300 import build
    build.build()
    return dade.lib()


def test_refused_allocation_is_enomem(lib):
    asked = []

    @HOOK
    def refuse(nbytes, user):
        asked.append(int(nbytes))
        return 1

    n, d = 500, 24
    base = np.random.default_rng(0).standard_normal((n, d)).astype(np.float32)
    o = dade.BuildOpts()
    lib.dade_build_opts_default(C.byref(o))
    o.n_clusters = 4
    o.eps_pairs = 100
    out = C.c_void_p(123)
    lib.dade_set_alloc_hook(C.cast(refuse, C.c_void_p), None)
    try:
        rc = lib.dade_build_index(base.ctypes.data, n, d, C.byref(o), C.byref(out), None)
    finally:
        lib.dade_set_alloc_hook(None, None)
    assert rc == dade.ENOMEM
    assert b"allocation hook" in lib.dade_last_error()
    assert asked and asked[0] == n * d * 4          # the staging copy of the host base comes first
    assert out.value is None                        # no index is returned


def test_hook_sees_no_call_once_removed(lib):
    asked = []

    @HOOK
    def count(nbytes, user):
        asked.append(int(nbytes))
        return 0

    lib.dade_set_alloc_hook(C.cast(count, C.c_void_p), None)
    lib.dade_set_alloc_hook(None, None)
    o = dade.BuildOpts()
    lib.dade_build_opts_default(C.byref(o))
    o.n_clusters = 0                                # rejected before any allocation
    out = C.c_void_p()
    base = np.zeros((4, 4), np.float32)
    assert lib.dade_build_index(base.ctypes.data, 4, 4, C.byref(o), C.byref(out), None) == dade.EINVAL
    assert asked == []
