"""Trees built on the GPU (level by level) vs the sequential host build and
the oracle's tree: identical leaves, identical node ranges (the leaf lower
bounds of the same queries agree bit for bit) and identical search results.
DSTree and iSAX.

Cases: random walks with several leaf capacities and root segmentations (odd
lengths, segments of one point), embedding-like data, data whose first
members are identical (the sequential build retries the split with one more
member until a candidate separates them), and data that no split separates
(the leaf stays over capacity).
"""
import numpy as np
import pytest

import fixtures as fx
import oracle as O
import paper_2502_01836_b300 as lf

pytestmark = pytest.mark.gpu


def _build(X, cap, init, host):
    return lf.leafi_build(X, lf.BuildParams(leaf_capacity=cap, dstree_init_segments=init, wave=8,
                                            device=0, host_build=host))


def _same_tree(X, cap, init, Q):
    dev = _build(X, cap, init, 0)
    host = _build(X, cap, init, 1)
    try:
        t = O.Tree(X, "dstree", leaf_cap=cap, init_segments=init)
        assert np.array_equal(lf.leafi_leaf_of(dev), t.leaf_of())
        assert np.array_equal(lf.leafi_leaf_of(dev), lf.leafi_leaf_of(host))
        assert lf.leafi_get_info(dev).n_nodes == lf.leafi_get_info(host).n_nodes
        L = lf.leafi_get_info(dev).n_leaves
        lb_d = np.zeros((len(Q), L), np.float64)
        lb_h = np.zeros((len(Q), L), np.float64)
        lf.leafi_leaf_lower_bounds(dev, Q, lb_d)
        lf.leafi_leaf_lower_bounds(host, Q, lb_h)
        assert np.array_equal(lb_d, lb_h)
        rd = np.zeros(len(Q), np.int32)
        rh = np.zeros(len(Q), np.int32)
        lf.leafi_route(dev, Q, rd)
        lf.leafi_route(host, Q, rh)
        assert np.array_equal(rd, rh)
        k = 5
        ids = np.zeros((len(Q), k), np.int64)
        d = np.zeros((len(Q), k), np.float32)
        lf.leafi_exact_search(dev, Q, k, ids, d)
        bf_ids, bf_d2 = O.knn(X, Q, k)
        assert np.array_equal(ids, bf_ids) and np.array_equal(d, np.sqrt(bf_d2))
    finally:
        lf.leafi_free(dev)
        lf.leafi_free(host)


@pytest.mark.parametrize("n,m,cap,init", [(30000, 256, 500, 4), (20000, 97, 300, 7),
                                          (12000, 16, 40, 16), (5000, 64, 10000, 4)])
def test_device_build_random_walks(n, m, cap, init):
    X = fx.random_walk(n, m, seed=401 + m)
    _same_tree(X, cap, init, fx.test_queries(X, 40, seed=402))


def test_device_build_embedding_like():
    X = fx.embedding_like(40000, 96, seed=403)
    _same_tree(X, 1000, 4, fx.test_queries(X, 40, seed=404))


def test_device_build_retries_on_identical_members():
    """The first 60 series are identical: no candidate separates the first
    cap + 1 members, the split is decided on the first 61 (the first distinct
    series) - as sequential insertion decides it."""
    X = fx.random_walk(3000, 32, seed=405)
    X[1:60] = X[0]
    _same_tree(X, 20, 4, fx.test_queries(X, 20, seed=406))


def test_device_build_unsplittable_leaf():
    """Identical series cannot be separated: the leaf keeps all of them."""
    X = np.repeat(fx.random_walk(1, 24, seed=407), 50, axis=0)
    X = np.concatenate([X, fx.random_walk(400, 24, seed=408)])
    _same_tree(X, 10, 3, fx.test_queries(X, 10, seed=409))
    sizes_dev = None
    idx = _build(X, 10, 3, 0)
    try:
        sizes_dev = lf.leafi_leaf_sizes(idx)
    finally:
        lf.leafi_free(idx)
    assert sizes_dev.max() >= 50


def test_device_build_from_device_pointer():
    torch = pytest.importorskip("torch")
    X = fx.random_walk(8000, 64, seed=410)
    Xd = torch.from_numpy(X).cuda()
    a = lf.leafi_build(Xd, lf.BuildParams(leaf_capacity=200, wave=4, device=0))
    b = lf.leafi_build(X, lf.BuildParams(leaf_capacity=200, wave=4, device=0, host_build=1))
    try:
        assert np.array_equal(lf.leafi_leaf_of(a), lf.leafi_leaf_of(b))
    finally:
        lf.leafi_free(a)
        lf.leafi_free(b)


def _same_isax(X, cap, w, bits, Q):
    kw = dict(index_type=lf.ISAX, leaf_capacity=cap, isax_segments=w, isax_card_bits=bits, wave=8,
              device=0)
    dev = lf.leafi_build(X, lf.BuildParams(host_build=0, **kw))
    host = lf.leafi_build(X, lf.BuildParams(host_build=1, **kw))
    try:
        t = O.Tree(X, "isax", leaf_cap=cap, isax_w=w, isax_bits=bits)
        assert np.array_equal(lf.leafi_leaf_of(dev), t.leaf_of())
        assert np.array_equal(lf.leafi_leaf_of(dev), lf.leafi_leaf_of(host))
        assert lf.leafi_get_info(dev).n_nodes == lf.leafi_get_info(host).n_nodes
        L = lf.leafi_get_info(dev).n_leaves
        lb_d = np.zeros((len(Q), L), np.float64)
        lb_h = np.zeros((len(Q), L), np.float64)
        lf.leafi_leaf_lower_bounds(dev, Q, lb_d)
        lf.leafi_leaf_lower_bounds(host, Q, lb_h)
        assert np.array_equal(lb_d, lb_h)
        k = 3
        ids = np.zeros((len(Q), k), np.int64)
        d = np.zeros((len(Q), k), np.float32)
        lf.leafi_exact_search(dev, Q, k, ids, d)
        bf_ids, bf_d2 = O.knn(X, Q, k)
        assert np.array_equal(ids, bf_ids) and np.array_equal(d, np.sqrt(bf_d2))
    finally:
        lf.leafi_free(dev)
        lf.leafi_free(host)


@pytest.mark.parametrize("n,m,cap,w,bits", [(60000, 256, 500, 16, 8), (20000, 64, 50, 8, 4),
                                            (5000, 96, 20, 4, 2)])
def test_device_build_isax(n, m, cap, w, bits):
    """Includes saturated segments (2-bit cardinality: leaves that cannot split
    further stay over capacity) and one-sided refinements."""
    X = fx.random_walk(n, m, seed=420 + w)
    _same_isax(X, cap, w, bits, fx.test_queries(X, 30, seed=421))
