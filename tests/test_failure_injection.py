"""Failure detection without a GPU fault, on the host (no GPU needed).

An allocation failure is injected into the library (leafi_debug_fail_allocations)
and must come back as LEAFI_ENOMEM with nothing written to the outputs; the
next call, with the injection spent, succeeds.
"""
import ctypes

import numpy as np

import fixtures as fx
import paper_2502_01836_b300 as lf


def test_injected_host_allocation_failure_is_enomem():
    X = fx.random_walk(2000, 32, seed=3)
    L = lf.lib()
    p = lf.BuildParams(leaf_capacity=200, device=-1)
    h = ctypes.c_void_p(12345)                      # a value the call must overwrite with NULL
    lf.leafi_debug_fail_allocations(0)
    st = L.leafi_build(X.ctypes.data, X.shape[0], X.shape[1], ctypes.byref(p), ctypes.byref(h))
    assert st == 2 and h.value is None
    assert b"alloc" in L.leafi_last_error()
    # the injection fired once and disarmed itself
    idx = lf.leafi_build(X, p)
    try:
        assert lf.leafi_get_info(idx).n_leaves > 1
    finally:
        lf.leafi_free(idx)


def test_injection_countdown_and_disarm():
    X = fx.random_walk(500, 16, seed=4)
    p = lf.BuildParams(leaf_capacity=100, device=-1)
    lf.leafi_debug_fail_allocations(1)              # the second gated allocation fails
    a = lf.leafi_build(X, p)
    lf.leafi_free(a)
    try:
        lf.leafi_build(X, p)
        raise AssertionError("the armed allocation did not fail")
    except lf.LeafiError as e:
        assert e.status == 2
    lf.leafi_debug_fail_allocations(5)
    lf.leafi_debug_fail_allocations(-1)             # disarmed before it fires
    for _ in range(8):
        lf.leafi_free(lf.leafi_build(X, p))
    assert lf.lib().leafi_debug_fail_allocations(-2) == 1
