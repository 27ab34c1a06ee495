"""Alg. 1 inside the library (leafi_train_filters) against the oracle.

The library draws its training queries, initial weights and SGD shuffles from
its own Philox4x32-10; the oracle has an independent implementation of the
same definition.  Picks, weights and shuffles must be bit-identical; queries
go through float64 logarithms and sines whose last bit may differ between the
device and the host maths library, so they are compared within one float32
rounding (and counted: virtually every value is identical).  The end-to-end
test runs build -> Alg. 1 -> search through the C ABI with inputs made by
numpy alone, no test fixtures.
"""
import numpy as np
import pytest

import oracle as O
import paper_2502_01836_b300 as lf

pytestmark = pytest.mark.gpu


def _walks(n, m, seed):
    """Random walks (cumulative sums of N(0,1) steps), z-normalised by the library."""
    rng = np.random.default_rng(seed)
    X = np.cumsum(rng.standard_normal((n, m)), axis=1).astype(np.float32)
    return lf.leafi_znormalize(X)


@pytest.fixture(scope="module")
def small():
    X = _walks(20000, 128, 5)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=1200, wave=4, device=0))
    t = O.Tree(X, "dstree", leaf_cap=1200, init_segments=4)
    yield X, idx, t
    lf.leafi_free(idx)


def test_znormalize_matches_float64(small):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = (rng.standard_normal((300, 96)) * 3 + 5).astype(np.float32)
    x[7] = 2.5                                     # constant row -> zeros
    ref = x.astype(np.float64)
    ref -= ref.mean(1, keepdims=True)
    sd = np.sqrt((ref * ref).mean(1, keepdims=True))
    ref = np.where(sd < 1e-8, 0.0, ref / np.where(sd < 1e-8, 1.0, sd))
    got = lf.leafi_znormalize(x)
    assert np.abs(got - ref).max() <= 2 * np.finfo(np.float32).eps * np.abs(ref).max()
    assert (got[7] == 0).all()
    # device arrays, in place
    d = torch.from_numpy(x).cuda()
    lf.leafi_znormalize(d, d)
    assert np.array_equal(d.cpu().numpy(), got)


def test_training_queries_equal_oracle_draws(small):
    X, idx, t = small
    p = lf.TrainParams(n_train=800, global_local_ratio=3.0, seed=77)
    sizes = t.leaf_sizes()
    fl = np.array([int(np.argmax(sizes)), int(np.argmin(sizes)), 3], np.int32)
    Qg, Ql, gp, lp = lf.leafi_training_queries(idx, p, fl)
    oQg, oQl, ogp, olp = O.training_queries(t, fl, 600, 200, 0.1, 0.4, 77)
    assert np.array_equal(gp, ogp) and np.array_equal(lp, olp)
    for a, b in ((Qg, oQg), (Ql, oQl)):
        assert np.abs(a - b).max() <= 4 * np.finfo(np.float32).eps
        assert np.mean(a == b) >= 0.999
    # their targets equal the oracle's targets on the oracle's own queries
    lf.leafi_set_filters(idx, fl, *lf.leafi_initial_weights(idx, 3, 128, 77))
    Tg = np.zeros((600, 3), np.float32)
    Tl = np.zeros((3, 200), np.float32)
    lf.leafi_train_targets(idx, Qg, Ql, Tg, Tl)
    oTg, oTl = O.train_targets(t, fl, oQg, oQl)
    assert np.allclose(Tg, oTg, rtol=1e-5, atol=1e-6) and np.allclose(Tl, oTl, rtol=1e-5, atol=1e-6)


def test_initial_weights_and_shuffles_equal_oracle(small):
    X, idx, t = small
    W = lf.leafi_initial_weights(idx, 5, 48, 2502)
    oW = O.filter_init(5, 48, 128, 2502)
    for a, b in zip(W, oW):
        assert np.array_equal(a, b)
    assert np.array_equal(lf.leafi_epoch_permutations(7, 333, 11), O.epoch_perms(7, 333, 11))


def test_alg1_end_to_end_through_the_abi():
    """build -> leafi_train_filters -> leafi_search with no test fixtures: the
    filters prune, exact mode equals brute force, and recall on held-out queries
    meets each target."""
    X = _walks(40000, 128, 7)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=1500, wave=4, device=0))
    try:
        L = lf.leafi_get_info(idx).n_leaves
        p = lf.TrainParams(n_filters=min(16, L), max_epochs=120, patience=8, kclasses=(1, 10),
                           seed=123)
        ep, bv, rep = lf.leafi_train_filters(idx, p)
        info = lf.leafi_get_info(idx)
        assert rep["n_filters"] == info.n_filters == min(16, L) and info.n_calib == 300
        assert (rep["n_gtrain"], rep["n_gval"], rep["n_ltrain"], rep["n_lval"]) == (1200, 300, 400, 100)
        assert (ep >= 1).all() and np.isfinite(bv).all()
        assert np.array_equal(lf.leafi_get_filter_leaves(idx), lf.leafi_select_leaves(idx, min(16, L)))
        # held-out queries: other series + noise, z-normalised by the library
        rng = np.random.default_rng(8)
        src = rng.choice(len(X), 400, replace=False)
        Q = X[src] + (rng.uniform(0.1, 0.4, (400, 1)) * rng.standard_normal((400, 128)))
        Q = lf.leafi_znormalize(Q.astype(np.float32))
        bf, bf_d2 = O.knn(X, Q, 10)
        ids = np.zeros((400, 10), np.int64)
        d = np.zeros((400, 10), np.float32)
        st = lf.SearchStats()
        lf.leafi_exact_search(idx, Q, 10, ids, d, st)
        assert np.array_equal(ids, bf) and np.array_equal(d, np.sqrt(bf_d2))
        exact_series = st.series_scanned
        for k in (1, 10):
            for target in (0.9, 0.99):
                ids = np.zeros((400, k), np.int64)
                d = np.zeros((400, k), np.float32)
                st = lf.SearchStats()
                lf.leafi_search(idx, Q, k, target, ids, d, st)
                rec = O.recall_at_k(ids, bf, k).mean()
                assert rec >= target, (k, target, rec)
                assert st.series_scanned <= exact_series
        # the same seed gives the same filters
        W1 = np.zeros((info.n_filters, 128, 128), np.float32)
        rest = (np.zeros((info.n_filters, 128), np.float32), np.zeros((info.n_filters, 128), np.float32),
                np.zeros(info.n_filters, np.float32))
        lf.leafi_get_filters(idx, W1, *rest)
        lf.leafi_train_filters(idx, p)
        W1b = np.zeros_like(W1)
        lf.leafi_get_filters(idx, W1b, *(np.zeros_like(r) for r in rest))
        assert np.array_equal(W1, W1b)
    finally:
        lf.leafi_free(idx)


def test_alg1_with_alg3_selection(small):
    """n_filters = -1 selects the leaves by Alg. 3 with the device's measured
    costs and the memory budget, as leafi_select_leaves_auto does."""
    X, idx, t = small
    p = lf.TrainParams(n_filters=-1, a=2.0, mem_cap=1_000_000, max_epochs=5, seed=9)
    _, _, rep = lf.leafi_train_filters(idx, p)
    fl = lf.leafi_get_filter_leaves(idx)
    auto, arep = lf.leafi_select_leaves_auto(idx, a=2.0, mem_cap=1_000_000)
    assert rep["n_filters"] == len(fl) == len(auto) >= 1
    assert np.array_equal(fl, auto)
    assert len(fl) * arep["filter_bytes"] <= 1_000_000
    sizes = t.leaf_sizes()
    assert (sizes[fl] >= rep["select_threshold"]).all()


def test_alg1_rejects_bad_parameters(small):
    X, idx, t = small
    for bad in (dict(n_train=1), dict(val_frac=0.0), dict(noise_lo=0.5, noise_hi=0.1),
                dict(n_filters=0), dict(kclasses=(10, 1)), dict(lr_min=1.0)):
        with pytest.raises(lf.LeafiError) as e:
            lf.leafi_train_filters(idx, lf.TrainParams(**bad))
        assert e.value.status == 1, bad
