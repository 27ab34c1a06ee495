"""Parity at the full configuration sizes (GPU path vs oracle, C-ABI calls).

Correctness configuration: 100,000 random walks x 256, DSTree capacity 2,000,
one filter per leaf trained on 2,000 queries (1,500 global + 500 local per
leaf, Alg. 1), 100 test queries, recall target 0.99, and exact mode.

Batched configuration: 1,000,000 random walks x 256, capacity 10,000, filters
on the 100 largest leaves, 10,000 test queries searched in one call (launches
of 256 queries, several in flight) - the launch configuration bench.py times.
Mixed-k configuration (reduced from 25M series): iSAX, 16 PAA segments,
cardinality 256, uneven leaves; k drawn from {1, 10, 100}, recall targets from
{0.9, 0.95, 0.99}; training targets (the build phase) bit-exact.

Precision configuration (reduced from 10M series): embedding-like vectors
(1,000 Gaussian clusters, m = 96), k = 10, exact mode on the tensor-core path
(float16 products, float32 re-check band) and on the CUDA-core path; both equal
the canonical float32 brute force, and the error against float64 distances
stays within the float32 bound.

Outputs the oracle cannot produce for all queries at this size are checked on
a seeded sample (exact k-NN by brute force; LeaFi search with the GPU's trained
weights and auto-tuner tables), the rest through properties that hold at any
size (recall against exact mode at least the target).
"""
import numpy as np
import pytest

import fixtures as fx
import oracle as O
import paper_2502_01836_b300 as lf
from paper_2502_01836_b300.workflow import enhance

pytestmark = pytest.mark.gpu

M = 256
W_WAVE = 64


def _search(idx, Q, k, target):
    ids = np.zeros((len(Q), k), np.int64)
    d = np.zeros((len(Q), k), np.float32)
    st = lf.SearchStats()
    lf.leafi_search(idx, Q, k, target, ids, d, st)
    return ids, d, st


def _gpu_model(idx, F, nc):
    """The trained weights and fitted tables, read back through the ABI."""
    W = (np.zeros((F, M, M), np.float32), np.zeros((F, M), np.float32),
         np.zeros((F, M), np.float32), np.zeros(F, np.float32))
    lf.leafi_get_filters(idx, *W)
    alpha = np.zeros((F, nc))
    qp = np.zeros((1, nc))
    lf.leafi_get_autotuners(idx, alpha, qp)
    return W, alpha, qp[0]


def _pred_scale(W, Q):
    W1, b1, w2, b2 = (a.astype(np.float64) for a in W)
    z = np.einsum("fhm,qm->qfh", W1, Q.astype(np.float64)) + b1[None]
    return np.abs(b2)[None] + np.einsum("qfh,fh->qf", np.maximum(z, 0), np.abs(w2))


def _leafi_vs_oracle(idx, t, enh, Q, ids_gpu):
    F = len(enh.filter_leaf)
    nc = lf.leafi_get_info(idx).n_calib
    W, alpha, qp = _gpu_model(idx, F, nc)
    j = O.offset_position(qp, 0.99)
    wave = lf.leafi_get_info(idx).wave      # the schedule the autotuner chose
    o_ids, o_d2, _, margin = O.leafi_search(t, W, enh.filter_leaf, alpha, Q, 1, j, wave)
    tol = 2e-5 * _pred_scale(W, Q).max()
    same = (ids_gpu == o_ids).all(1)
    # a query may differ only where a filter decision sits within the prediction tolerance
    assert (same | (margin <= tol)).all()
    assert same.mean() >= 0.95


def test_correctness_config_100k():
    X = fx.random_walk(100_000, M)
    Q = fx.test_queries(X, 100)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=2000, wave=W_WAVE, device=0))
    try:
        t = O.Tree(X, "dstree", leaf_cap=2000, init_segments=4)
        assert np.array_equal(lf.leafi_leaf_of(idx), t.leaf_of())
        # exact mode: brute force, bit for bit, k = 1 and 10
        for k in (1, 10):
            ids, d, _ = _search(idx, Q, k, 1.0)
            bf_ids, bf_d2 = O.knn(X, Q, k)
            assert np.array_equal(ids, bf_ids) and np.array_equal(d, np.sqrt(bf_d2))
        # LeaFi mode: one filter per leaf
        L = lf.leafi_get_info(idx).n_leaves
        enh = enhance(idx, L)
        ids, d, st = _search(idx, Q, 1, 0.99)
        ex_ids, _ = O.knn(X, Q, 1)
        assert (ids[:, 0] == ex_ids[:, 0]).mean() >= 0.99
        assert st.series_scanned < len(Q) * len(X)
        _leafi_vs_oracle(idx, t, enh, Q, ids)
    finally:
        lf.leafi_free(idx)


def test_batched_config_1m_sampled():
    X = fx.random_walk(1_000_000, M)
    Q = fx.test_queries(X, 10_000)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=10_000, wave=W_WAVE, device=0))
    try:
        # exact mode over all 10,000 queries in one call; brute force on a sample
        ex_ids, ex_d, st = _search(idx, Q, 1, 1.0)
        assert st.batches == 40 and st.graph_batches == 39
        rng = np.random.default_rng(2502)
        sample = np.sort(rng.choice(len(Q), 200, replace=False))
        bf_ids, bf_d2 = O.knn(X, Q[sample], 1)
        assert np.array_equal(ex_ids[sample], bf_ids)
        assert np.array_equal(ex_d[sample], np.sqrt(bf_d2))
        # k = 10 on a 256-query slice (one full batch, the captured graph)
        ids10, d10, _ = _search(idx, np.ascontiguousarray(Q[:256]), 10, 1.0)
        bf10, bf10_d2 = O.knn(X, Q[:32], 10)
        assert np.array_equal(ids10[:32], bf10) and np.array_equal(d10[:32], np.sqrt(bf10_d2))
        # LeaFi mode, filters on the 100 largest leaves
        enh = enhance(idx, 100)
        ids, _, st = _search(idx, Q, 1, 0.99)
        assert (ids[:, 0] == ex_ids[:, 0]).mean() >= 0.99
        assert st.filter_pruned <= st.filter_evals <= len(Q) * 100
        t = O.Tree(X, "dstree", leaf_cap=10_000, init_segments=4)
        assert np.array_equal(lf.leafi_leaf_of(idx), t.leaf_of())
        few = sample[:40]
        _leafi_vs_oracle(idx, t, enh, np.ascontiguousarray(Q[few]), ids[few])
    finally:
        lf.leafi_free(idx)


def test_mixed_k_isax_config_reduced():
    X = fx.random_walk(200_000, M, seed=fx.SEED_DATA + 7)
    idx = lf.leafi_build(X, lf.BuildParams(index_type=lf.ISAX, leaf_capacity=2000, wave=16,
                                           device=0))
    try:
        t = O.Tree(X, "isax", leaf_cap=2000, isax_w=16, isax_bits=8)
        assert np.array_equal(lf.leafi_leaf_of(idx), t.leaf_of())
        sizes = lf.leafi_leaf_sizes(idx)
        assert sizes.max() >= 3 * max(1.0, float(np.median(sizes)))   # uneven leaves
        F = 24
        enh = enhance(idx, F, kclasses=(1, 10, 100), keep_queries=True, max_epochs=60, patience=5)
        # the build phase: node-wise nearest-neighbour targets, bit for bit
        Ql = np.ascontiguousarray(enh.Ql[:, :40])
        Qg = np.ascontiguousarray(enh.Qg[:300])
        Tg = np.zeros((300, F), np.float32)
        Tl = np.zeros((F, 40), np.float32)
        lf.leafi_train_targets(idx, Qg, Ql, Tg, Tl)
        oTg, oTl = O.train_targets(t, enh.filter_leaf, Qg, Ql)
        assert np.array_equal(Tg, oTg) and np.array_equal(Tl, oTl)
        # mixed requests: k in {1, 10, 100}, targets in {0.9, 0.95, 0.99}, some exact
        Q = fx.test_queries(X, 400, seed=fx.SEED_TEST + 7)
        rng = np.random.default_rng(25)
        kq = rng.choice([1, 10, 100], len(Q)).astype(np.int32)
        tg = rng.choice([0.9, 0.95, 0.99, 1.0], len(Q)).astype(np.float64)
        ids = np.zeros((len(Q), 100), np.int64)
        d = np.zeros((len(Q), 100), np.float32)
        lf.leafi_search_mixed(idx, Q, kq, tg, 100, ids, d)
        nc = lf.leafi_get_info(idx).n_calib
        W = (np.zeros((F, M, M), np.float32), np.zeros((F, M), np.float32),
             np.zeros((F, M), np.float32), np.zeros(F, np.float32))
        lf.leafi_get_filters(idx, *W)
        alpha = np.zeros((F, nc))
        qp = np.zeros((3, nc))
        lf.leafi_get_autotuners(idx, alpha, qp)
        cls = {1: 0, 10: 1, 100: 2}
        jpos = np.array([-1 if tg[i] >= 1 else O.offset_position(qp[cls[kq[i]]], tg[i], kk=kq[i])
                         for i in range(len(Q))], np.int32)
        o_ids, o_d2, _, margin = O.leafi_search(t, W, enh.filter_leaf, alpha, Q, kq, jpos,
                                                lf.leafi_get_info(idx).wave, kmax=100)
        tol = 2e-5 * _pred_scale(W, Q).max()
        same = (ids == o_ids).all(1)
        assert (same | (margin <= tol)).all()
        assert same[jpos < 0].all()
        assert same.mean() >= 0.95
        # padding beyond each query's k
        for i in range(len(Q)):
            assert (ids[i, kq[i]:] == -1).all()
    finally:
        lf.leafi_free(idx)


@pytest.mark.parametrize("path", [0, 1, 2])
def test_precision_config_reduced(path):
    m, n, k = 96, 300_000, 10
    X = fx.embedding_like(n, m)
    Q = fx.test_queries(X, 300, seed=fx.SEED_TEST + 3)   # two batches: two lanes
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=10_000, wave=W_WAVE, device=0,
                                           scan_path=path))
    try:
        info = lf.leafi_get_info(idx)
        assert bool(info.tensor_scan) == (path != 1)
        ids = np.zeros((len(Q), k), np.int64)
        d = np.zeros((len(Q), k), np.float32)
        st = lf.SearchStats()
        lf.leafi_exact_search(idx, Q, k, ids, d, st)
        bf_ids, bf_d2 = O.knn(X, Q, k)
        assert np.array_equal(ids, bf_ids) and np.array_equal(d, np.sqrt(bf_d2))
        # against float64 distances of the same series: the float32 canonical sum's bound
        X64, Q64 = X.astype(np.float64), Q.astype(np.float64)
        d64 = np.sqrt(np.einsum("qkm,qkm->qk", X64[ids] - Q64[:, None], X64[ids] - Q64[:, None]))
        rel = np.abs(d.astype(np.float64) - d64) / np.maximum(d64, 1e-30)
        assert rel.max() <= m * 2.0 ** -24
        # recall@10 against the float64 ranking (near-ties may swap the last place)
        sub = np.arange(0, len(Q), 10)
        truth = np.stack([np.argsort(((X64 - Q64[i]) ** 2).sum(-1), kind="stable")[:k]
                          for i in sub])
        rec = np.mean([len(set(ids[i]) & set(truth[j])) / k for j, i in enumerate(sub)])
        assert rec >= 0.99
        if path == 0:
            # the band admits few re-checks per query
            assert st.rechecks < 0.01 * st.series_scanned
    finally:
        lf.leafi_free(idx)
