"""CNN filters (Sec. 5.2 model-type study) on the GPU against the oracle.

Bars: the forward within the float32 error bound of its accumulations (stated
in `_bound`); one SGD epoch as close to the float64 oracle's as the MLP's;
the library's initial parameters bit-exact (both sides draw the same Philox
numbers and scale them in float64); Alg. 4 and Alg. 2 on the GPU's own
predictions bit-exact with the oracle's (same predictions, so every filter
decision is the same on both sides), scanned leaves and series included.
"""
import numpy as np
import pytest

import fixtures as fx
import oracle as O
import paper_2502_01836_b300 as lf

pytestmark = pytest.mark.gpu


def _bound(theta, C, Q):
    """Float32 error bound of the CNN forward: every output is a chain of
    accumulations (conv1: 3 terms, conv2: 3C + 1, pooling: m, head: C + 1), each
    adding at most (terms) * 2^-24 of the sum of the absolute values of its
    terms; the forward on |theta| and |q| bounds those sums (with non-negative
    inputs the ReLUs pass everything).  Twice the first-order bound."""
    m = Q.shape[1]
    mag = O.cnn_forward(np.abs(theta), C, np.abs(Q))
    return 2.0 * (4 * C + m + 16) * 2.0 ** -24 * mag


@pytest.mark.parametrize("m,C,nq", [(48, 48, 37), (96, 96, 19), (37, 20, 50)])
def test_cnn_forward_within_bound(m, C, nq):
    X = fx.random_walk(4000, m, seed=301)
    Q = fx.test_queries(X, nq, seed=302)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=400, wave=2, device=0))
    try:
        F = 5
        fl = np.arange(F, dtype=np.int32)
        theta = O.cnn_init(F, C, seed=303)
        lf.leafi_set_cnn_filters(idx, fl, C, theta)
        info = lf.leafi_get_info(idx)
        assert info.filter_model == lf.FILTER_CNN and info.filter_width == C
        P = np.zeros((nq, F), np.float32)
        lf.leafi_filter_predict(idx, Q, P)
        ref = O.cnn_forward(theta, C, Q)
        err = np.abs(P - ref)
        assert (err <= _bound(theta, C, Q)).all(), err.max()
        assert np.array_equal(lf.leafi_get_cnn_filters(idx), theta)
        with pytest.raises(lf.LeafiError):
            W = (np.zeros((F, C, m), np.float32), np.zeros((F, C), np.float32),
                 np.zeros((F, C), np.float32), np.zeros(F, np.float32))
            lf.leafi_get_filters(idx, *W)
    finally:
        lf.leafi_free(idx)


def test_cnn_initial_parameters_bit_exact():
    X = fx.random_walk(1000, 32, seed=311)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=200, device=0))
    try:
        for F, C, seed in ((3, 32, 5), (2, 7, 9)):
            assert np.array_equal(lf.leafi_initial_cnn_weights(idx, F, C, seed),
                                  O.cnn_init(F, C, seed))
    finally:
        lf.leafi_free(idx)


def test_cnn_too_wide_is_refused():
    X = fx.random_walk(1000, 256, seed=312)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=200, device=0))
    try:
        theta = np.zeros((1, lf.leafi_cnn_params(256)), np.float32)
        with pytest.raises(lf.LeafiError):
            lf.leafi_set_cnn_filters(idx, np.zeros(1, np.int32), 256, theta)
    finally:
        lf.leafi_free(idx)


@pytest.mark.parametrize("ltrain,lval", [(24, 6), (0, 0)])
def test_cnn_one_epoch_of_sgd_matches_oracle(ltrain, lval):
    m = C = 32
    X = fx.random_walk(6000, m, seed=321)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=500, wave=2, device=0))
    t = O.Tree(X, "dstree", leaf_cap=500, init_segments=4)
    try:
        F = 3
        sizes = t.leaf_sizes()
        fl = np.array(sorted(range(t.L), key=lambda l: (-sizes[l], l))[:F], np.int32)
        theta = O.cnn_init(F, C, seed=322)
        lf.leafi_set_cnn_filters(idx, fl, C, theta)
        members = fx.leaf_members_from(t.leaf_of(), fl)
        Qg, Ql = fx.training_queries(X, members, 100, ltrain + lval, seed=323)
        kw = dict(n_gtrain=80, n_gval=20, n_ltrain=ltrain, n_lval=lval, batch=16, max_epochs=1,
                  patience=5, lr0=1e-3, lr_min=1e-5)
        perms = fx.epoch_permutations(1, 80 + ltrain, seed=324)
        lf.leafi_train_filters_on(idx, lf.SgdParams(**kw), Qg, Ql, perms)
        got = lf.leafi_get_cnn_filters(idx)
        Tg, Tl = O.train_targets(t, fl, Qg, Ql)
        ref, _, _ = O.cnn_train(O.TrainParams(**kw), C, Qg, Tg, Ql, Tl, perms, theta)
        moved = np.abs(ref.astype(np.float64) - theta)
        assert moved.max() > 0
        assert np.abs(got.astype(np.float64) - ref).max() <= 1e-3 * moved.max() + 1e-6
    finally:
        lf.leafi_free(idx)


@pytest.fixture(scope="module")
def cnn_index():
    """Alg. 1 with CNN filters, run by the library (a short training)."""
    m = 64
    X = fx.random_walk(20000, m, seed=331)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=1000, wave=4, device=0))
    t = O.Tree(X, "dstree", leaf_cap=1000, init_segments=4)
    p = lf.TrainParams(n_filters=6, n_train=800, max_epochs=6, patience=3, kclasses=(1, 10),
                       tune_search=0, model=lf.FILTER_CNN, seed=332)
    _, _, rep = lf.leafi_train_filters(idx, p)
    yield X, idx, t, p, rep
    lf.leafi_free(idx)


def test_cnn_autotuner_bit_exact_on_gpu_predictions(cnn_index):
    X, idx, t, p, rep = cnn_index
    info = lf.leafi_get_info(idx)
    fl = lf.leafi_get_filter_leaves(idx)
    Qg, _, _, _ = lf.leafi_training_queries(idx, p, fl)
    Qc = Qg[rep["n_gtrain"]:]
    assert Qc.shape[0] == rep["n_gval"] == info.n_calib
    Pc = np.zeros((Qc.shape[0], len(fl)), np.float32)
    lf.leafi_filter_predict(idx, Qc, Pc)
    alpha = np.zeros((len(fl), Qc.shape[0]))
    qp = np.zeros((2, Qc.shape[0]))
    lf.leafi_get_autotuners(idx, alpha, qp)
    for i, k in enumerate((1, 10)):
        a_ref, q_ref = O.fit_autotuner_pred(t, Pc.astype(np.float64), fl, Qc, k, info.wave)
        assert np.array_equal(alpha, a_ref)
        assert np.array_equal(qp[i], q_ref), k


@pytest.mark.parametrize("k,target", [(1, 0.9), (10, 0.95)])
def test_cnn_leafi_search_bit_exact_on_gpu_predictions(cnn_index, k, target):
    X, idx, t, p, _ = cnn_index
    info = lf.leafi_get_info(idx)
    fl = lf.leafi_get_filter_leaves(idx)
    nc = info.n_calib
    alpha = np.zeros((len(fl), nc))
    qp = np.zeros((2, nc))
    lf.leafi_get_autotuners(idx, alpha, qp)
    Q = fx.test_queries(X, 150, seed=333)
    P = np.zeros((Q.shape[0], len(fl)), np.float32)
    lf.leafi_filter_predict(idx, Q, P)
    # the point estimate keeps the filters in play for this comparison
    lf.leafi_set_calibration_confidence(idx, 0.0)
    try:
        ids = np.zeros((Q.shape[0], k), np.int64)
        d = np.zeros((Q.shape[0], k), np.float32)
        st = lf.SearchStats()
        lf.leafi_search(idx, Q, k, target, ids, d, st)
    finally:
        lf.leafi_set_calibration_confidence(idx, 0.95)
    j = O.offset_position(qp[0 if k == 1 else 1], target, kk=k, confidence=0.0)
    assert j >= 0
    o_ids, o_d2, o_st, _ = O.leafi_search_pred(t, P.astype(np.float64), fl, alpha, Q, k, j,
                                               info.wave)
    assert np.array_equal(ids, o_ids)
    assert np.array_equal(d, np.sqrt(o_d2))
    assert st.leaves_scanned == o_st[:, 0].sum()
    assert st.series_scanned == o_st[:, 1].sum()
    assert st.filter_pruned == o_st[:, 3].sum() and st.lb_pruned == o_st[:, 2].sum()
    assert st.filter_evals == Q.shape[0] * len(fl)


def test_cnn_end_to_end_recall_meets_target(cnn_index):
    X, idx, t, p, _ = cnn_index
    Q = fx.test_queries(X, 300, seed=334)
    bf, _ = O.knn(X, Q, 1)
    for target in (0.9, 0.99):
        ids = np.zeros((Q.shape[0], 1), np.int64)
        d = np.zeros((Q.shape[0], 1), np.float32)
        lf.leafi_search(idx, Q, 1, target, ids, d)
        assert (ids[:, 0] == bf[:, 0]).mean() >= target, target
