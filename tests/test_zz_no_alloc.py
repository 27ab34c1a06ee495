"""The allocation-free bounds entry point against the regular one.

leafi_leaf_lower_bounds_noalloc serves callers that cannot call cudaMalloc
(their GPU memory is held by another allocator, or their loop cannot take
cudaMalloc's device-wide synchronisation): its scratch is a static device
array instead of memory allocated per call.  Its output must equal leafi_leaf_lower_bounds'
(both evaluate the same float64 operations, so the comparison is exact), on
two calls in a row that reuse the same scratch.  This file is collected last.
"""
import numpy as np
import pytest

import fixtures as fx
import paper_2502_01836_b300 as lf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [lf.DSTREE, lf.ISAX])
def test_noalloc_bounds_equal_regular_bounds_twice(kind):
    torch = pytest.importorskip("torch")
    X = fx.random_walk(20000, 256, seed=91)
    idx = lf.leafi_build(X, lf.BuildParams(index_type=kind, leaf_capacity=700, device=0))
    try:
        L = lf.leafi_get_info(idx).n_leaves
        for call in range(2):
            Q = fx.test_queries(X, 150 + 17 * call, seed=92 + call)
            ref = np.zeros((Q.shape[0], L), np.float64)
            lf.leafi_leaf_lower_bounds(idx, Q, ref)
            out = torch.full((Q.shape[0], L), float("nan"), dtype=torch.float64, device="cuda")
            lf.leafi_leaf_lower_bounds_noalloc(idx, torch.from_numpy(Q).cuda(), out)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), ref), "call %d" % call
    finally:
        lf.leafi_free(idx)


def test_noalloc_rejects_oversize_and_host_arrays():
    torch = pytest.importorskip("torch")
    X = fx.random_walk(5000, 256, seed=93)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=500, device=0))
    try:
        L = lf.leafi_get_info(idx).n_leaves
        big = torch.zeros((20000, 256), dtype=torch.float32, device="cuda")
        out = torch.zeros((20000, L), dtype=torch.float64, device="cuda")
        with pytest.raises(lf.LeafiError) as e:
            lf.leafi_leaf_lower_bounds_noalloc(idx, big, out)
        assert e.value.status == 1 and "scratch" in str(e.value)
        # host arrays: refused by the wrapper, and by the C entry point itself
        with pytest.raises(TypeError):
            lf.leafi_leaf_lower_bounds_noalloc(idx, X[:4].copy(), np.zeros((4, L)))
        q, o = X[:4].copy(), np.zeros((4, L))
        st = lf.lib().leafi_leaf_lower_bounds_noalloc(idx, q.ctypes.data, 4, o.ctypes.data)
        assert st == 1 and "device" in lf.lib().leafi_last_error().decode()
    finally:
        lf.leafi_free(idx)


def test_noalloc_rejects_wrong_shapes_before_launch():
    torch = pytest.importorskip("torch")
    X = fx.random_walk(3000, 64, seed=94)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=400, device=0))
    try:
        L = lf.leafi_get_info(idx).n_leaves
        n0 = lf.leafi_launch_count()
        q = torch.zeros((8, 64), dtype=torch.float32, device="cuda")
        with pytest.raises(ValueError):
            lf.leafi_leaf_lower_bounds_noalloc(idx, torch.zeros((8, 63), device="cuda"),
                                               torch.zeros((8, L), dtype=torch.float64,
                                                           device="cuda"))
        with pytest.raises(ValueError):
            lf.leafi_leaf_lower_bounds_noalloc(idx, q, torch.zeros((8, L - 1),
                                                                   dtype=torch.float64,
                                                                   device="cuda"))
        with pytest.raises(ValueError):
            lf.leafi_leaf_lower_bounds_noalloc(idx, q, torch.zeros((7, L), dtype=torch.float64,
                                                                   device="cuda"))
        assert lf.leafi_launch_count() == n0, "a rejected call launched a kernel"
    finally:
        lf.leafi_free(idx)


def test_noalloc_rejects_memory_of_another_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.device_count() < 2:
        pytest.skip("needs a second visible GPU")
    X = fx.random_walk(3000, 64, seed=95)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=400, device=0))
    try:
        L = lf.leafi_get_info(idx).n_leaves
        q = torch.zeros((4, 64), dtype=torch.float32, device="cuda:1")
        out = torch.zeros((4, L), dtype=torch.float64, device="cuda:1")
        n0 = lf.leafi_launch_count()
        with pytest.raises(lf.LeafiError) as e:
            lib = lf.lib()
            st = lib.leafi_leaf_lower_bounds_noalloc(idx, q.data_ptr(), 4, out.data_ptr())
            lf._check(st)
        assert e.value.status == 1
        assert lf.leafi_launch_count() == n0
    finally:
        lf.leafi_free(idx)
