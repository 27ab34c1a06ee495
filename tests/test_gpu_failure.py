"""Failure detection on the GPU without a fault, trap or hang.

Timeout: the tensor-core scan's bounded wait for a query's result-list lock is
given no attempts (leafi_debug_set_lock_tries(0)); the work item gives up,
sets the error word and the kernel leaves through its normal exits, so the
call returns LEAFI_ETIMEOUT and the context stays usable: with the default
budget restored the next search equals brute force.

Allocation: an injected device-allocation failure on a fresh index's first
search returns LEAFI_ENOMEM before anything is written to the outputs.
"""
import numpy as np
import pytest

import fixtures as fx
import oracle as O
import paper_2502_01836_b300 as lf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def data():
    X = fx.random_walk(30000, 128, seed=61)
    Q = fx.test_queries(X, 100, seed=62)
    return X, Q, O.knn(X, Q, 10)


def test_lock_timeout_returns_etimeout_and_index_recovers(data):
    X, Q, (bf, bf_d2) = data
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=1500, wave=8, device=0))
    try:
        assert lf.leafi_get_info(idx).tensor_scan == 1
        ids = np.zeros((100, 10), np.int64)
        d = np.zeros((100, 10), np.float32)
        lf.leafi_exact_search(idx, Q, 10, ids, d)
        assert np.array_equal(ids, bf)
        lf.leafi_debug_set_lock_tries(idx, 0)
        with pytest.raises(lf.LeafiError) as e:
            lf.leafi_exact_search(idx, Q, 10, np.zeros((100, 10), np.int64),
                                  np.zeros((100, 10), np.float32))
        assert e.value.status == 4 and "timed out" in str(e.value)
        lf.leafi_debug_set_lock_tries(idx, -1)
        ids2 = np.zeros((100, 10), np.int64)
        d2 = np.zeros((100, 10), np.float32)
        lf.leafi_exact_search(idx, Q, 10, ids2, d2)
        assert np.array_equal(ids2, bf) and np.array_equal(d2, np.sqrt(bf_d2))
    finally:
        lf.leafi_free(idx)


def test_injected_device_allocation_failure_is_enomem(data):
    X, Q, (bf, bf_d2) = data
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=1500, wave=8, device=0))
    try:
        ids = np.full((100, 10), -7, np.int64)
        d = np.full((100, 10), -7.0, np.float32)
        lf.leafi_debug_fail_allocations(0)
        with pytest.raises(lf.LeafiError) as e:
            lf.leafi_exact_search(idx, Q, 10, ids, d)
        assert e.value.status == 2
        assert (ids == -7).all() and (d == -7.0).all()
        lf.leafi_exact_search(idx, Q, 10, ids, d)
        assert np.array_equal(ids, bf) and np.array_equal(d, np.sqrt(bf_d2))
    finally:
        lf.leafi_debug_fail_allocations(-1)
        lf.leafi_free(idx)
