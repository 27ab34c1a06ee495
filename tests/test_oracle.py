"""Pins of the oracle against facts fixed outside it (no GPU).

Each test checks one oracle function against something other than itself:
hand-worked golden cases (tests/golden/, cited), closed forms, textbook
library values, exhaustive enumeration on tiny inputs, or invariants that the
mathematics guarantees.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.stats

import fixtures as fx
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- distances

def test_sqdist_within_float32_bound_of_exact():
    """Canonical float32 d^2 is within gamma_{m+1} of the exact value (Higham)."""
    rng = np.random.default_rng(1)
    m = 256
    u = 2.0 ** -24
    gamma = (m + 1) * u / (1 - (m + 1) * u)
    for _ in range(200):
        q = rng.standard_normal(m).astype(np.float32)
        x = rng.standard_normal(m).astype(np.float32)
        exact = float(np.sum((q.astype(np.float64) - x.astype(np.float64)) ** 2))
        assert abs(float(O.sqdist(q, x)) - exact) <= gamma * exact


def test_sqdist_integer_data_exact():
    q = np.array([3, -1, 2, 0, 5], np.float32)
    x = np.array([1, 1, -2, 0, 5], np.float32)
    assert O.sqdist(q, x) == np.float32(4 + 4 + 16)


def test_knn_matches_exhaustive_enumeration_with_ties():
    """Integer-valued data makes every distance exact and ties frequent: the
    oracle must return the k smallest (d^2, id) pairs of the definition."""
    rng = np.random.default_rng(7)
    for m in (4, 8, 16):
        X = rng.integers(-2, 3, size=(64, m)).astype(np.float32)
        Q = rng.integers(-2, 3, size=(20, m)).astype(np.float32)
        for k in (1, 3, 10, 64):
            ids, d2 = O.knn(X, Q, k)
            for i in range(Q.shape[0]):
                d = ((X.astype(np.int64) - Q[i].astype(np.int64)) ** 2).sum(1)
                order = sorted(range(X.shape[0]), key=lambda s: (d[s], s))[:k]
                assert ids[i].tolist() == order
                assert d2[i].tolist() == [float(d[s]) for s in order]


def test_knn_pads_when_k_exceeds_n():
    X = np.eye(3, dtype=np.float32)
    ids, d2 = O.knn(X, X[:1], 5)
    assert ids[0].tolist() == [0, 1, 2, -1, -1]
    assert np.isinf(d2[0, 3:]).all()


# ---------------------------------------------------------------- statistics

def test_segment_stats_closed_form():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(96).astype(np.float32)
    for s, e in [(0, 96), (0, 1), (10, 37), (95, 96)]:
        mu, sd = O.segment_stats(x, s, e)
        seg = x[s:e].astype(np.float64)
        assert mu == pytest.approx(seg.mean(), abs=1e-13)
        assert sd == pytest.approx(seg.std(), abs=1e-7)


# ---------------------------------------------------------------- DSTree

def test_dstree_lb_hand_example():
    g = _golden("dstree_lb_hand.json")
    X = np.array(g["series"], np.float32)
    t = O.Tree(X, "dstree", leaf_cap=g["leaf_cap"], init_segments=g["init_segments"])
    assert t.L == 1
    lb = t.lb2(np.array([g["query"]], np.float32))
    assert lb[0, 0] == g["lb2"]
    _, d2 = O.knn(X, np.array([g["query"]], np.float32), 2)
    assert d2[0].tolist() == g["d2"]


def test_dstree_split_hand_example():
    g = _golden("dstree_split_hand.json")
    X = np.array(g["series"], np.float32)
    t = O.Tree(X, "dstree", leaf_cap=g["leaf_cap"], init_segments=g["init_segments"])
    assert t.L == g["n_leaves"]
    assert t.n_nodes == g["n_nodes"]
    assert t.leaf_of().tolist() == g["leaf_of"]
    # routing sends every series to its own leaf
    assert t.route(X).tolist() == g["leaf_of"]


def test_dstree_split_score_hand_example():
    """The QoS score decides among candidates of every kind: a horizontal split
    on sigma wins by 41/6 against 6, and each plausible misreading of the score
    (sigma range, unweighted children, no interval lengths) picks another
    partition (tests/golden/dstree_split_score_hand.json)."""
    g = _golden("dstree_split_score_hand.json")
    X = np.array(g["series"], np.float32)
    t = O.Tree(X, "dstree", leaf_cap=g["leaf_cap"], init_segments=g["init_segments"])
    assert t.L == g["n_leaves"] and t.n_nodes == g["n_nodes"]
    assert t.leaf_of().tolist() == g["leaf_of"]
    assert t.route(X).tolist() == g["leaf_of"]
    # the children's synopses are over the winner's segmentation
    assert t.lb2(X).tolist() == g["lb2_of_series"]


@pytest.fixture(scope="module")
def rw():
    X = fx.random_walk(6000, 64, seed=11)
    Q = fx.test_queries(X, 40, seed=12)
    return X, Q


def test_dstree_structure_and_lb_invariant(rw):
    X, Q = rw
    t = O.Tree(X, "dstree", leaf_cap=300, init_segments=4)
    sizes = t.leaf_sizes()
    assert sizes.sum() == X.shape[0] and sizes.max() <= 300 and sizes.min() >= 1
    lo = t.leaf_of()
    for leaf in range(t.L):
        mem = t.leaf_members(leaf)
        assert (lo[mem] == leaf).all() and (np.diff(mem) > 0).all()
    # every series routes to the leaf that holds it
    assert (t.route(X[::7]) == lo[::7]).all()
    lb = t.lb2(Q)
    leaves = np.tile(np.arange(t.L, dtype=np.int32), (Q.shape[0], 1))
    d2, _ = t.leaf_topk(Q, leaves, 1)
    # LB^2 <= leaf min d^2 (exact arithmetic); the deflated test never prunes a true minimum
    assert (lb * (1 - 1e-4) <= d2[:, :, 0]).all()
    assert (lb <= d2[:, :, 0] * (1 + 1e-5)).all()
    # a series' own leaf has LB 0 to itself (its statistics lie inside the ranges)
    own = t.lb2(X[:50])
    assert (own[np.arange(50), lo[:50]] == 0.0).all()


U32 = 2.0 ** -24  # unit roundoff of float32


def _stats64(X, cuts):
    """Segment means and sigmas of float32 rows from float64 running sums."""
    X = X.astype(np.float64)
    P1 = np.concatenate([np.zeros((len(X), 1)), np.cumsum(X, axis=1)], axis=1)
    P2 = np.concatenate([np.zeros((len(X), 1)), np.cumsum(X * X, axis=1)], axis=1)
    mu, sd = [], []
    for s, e in zip(cuts[:-1], cuts[1:]):
        u = (P1[:, e] - P1[:, s]) / (e - s)
        v = (P2[:, e] - P2[:, s]) / (e - s) - u * u
        mu.append(u)
        sd.append(np.sqrt(np.maximum(v, 0.0)))
    return np.stack(mu, 1), np.stack(sd, 1)


def _gap_and_slack(v, lo, hi):
    """float64 gap of v to [lo, hi] and how far the float32 enclosures of v,
    lo and hi can pull the float32 gap below it (one float32 ulp each)."""
    g = np.where(v < lo, lo - v, np.where(v > hi, v - hi, 0.0))
    mag = np.maximum(np.abs(v), np.maximum(np.where(np.isfinite(lo), np.abs(lo), 0.0),
                                           np.where(np.isfinite(hi), np.abs(hi), 0.0)))
    return g, 2.0 ** -22 * mag + 1e-44


def _within_enclosure_error(lb32, terms, n_terms):
    """The float32 bound lies between the float64 bound computed on the
    narrowed gaps and the float64 bound itself, each widened by the relative
    rounding of n_terms float32 products and sums."""
    lo_terms, hi_terms = terms
    grow = (1 + U32) ** (n_terms + 5)
    assert (lb32 <= hi_terms.sum(1) * grow).all(), np.max(lb32 / np.maximum(hi_terms.sum(1), 1e-300))
    assert (lb32 >= lo_terms.sum(1) / grow).all()


def test_dstree_float32_bound_within_enclosure_error():
    """The DSTree bound is evaluated in float32 on outward-rounded synopses and
    query statistics: against the float64 bound of the same one-leaf tree it
    is never larger beyond product/sum rounding, and never smaller than the
    gaps narrowed by one ulp of each end.  The queries sit just outside the
    ranges (gaps of 1e-5 in the mean, 1e-5 relative in sigma), where rounding
    the query statistic or a range end the wrong way would exceed the upper
    side by orders of magnitude; random queries and the series themselves
    (bound 0) are included."""
    m = 64
    X = fx.random_walk(500, m, seed=41)
    t = O.Tree(X, "dstree", leaf_cap=1000, init_segments=4)
    assert t.L == 1
    cuts = [0, 16, 32, 48, 64]
    mu, sd = _stats64(X, cuts)
    mlo, mhi, slo, shi = mu.min(0), mu.max(0), sd.min(0), sd.max(0)
    near = []
    for r in range(4):
        s, e = cuts[r], cuts[r + 1]
        hi_row = X[np.argmax(mu[:, r])].copy()
        hi_row[s:e] += np.float32(1e-5)
        lo_row = X[np.argmin(mu[:, r])].copy()
        lo_row[s:e] -= np.float32(1e-5)
        wide = X[np.argmax(sd[:, r])].copy()
        c = wide[s:e].astype(np.float64).mean()
        wide[s:e] = (c + (wide[s:e] - c) * (1 + 1e-5)).astype(np.float32)
        near += [hi_row, lo_row, wide]
    Q = np.concatenate([np.array(near, np.float32), fx.test_queries(X, 40, seed=42), X[:20]])
    qmu, qsd = _stats64(Q, cuts)
    gm, em = _gap_and_slack(qmu, mlo, mhi)
    gs, es = _gap_and_slack(qsd, slo, shi)
    ln = np.diff(cuts).astype(np.float64)
    hi_terms = ln * (gm * gm + gs * gs)
    lo_terms = ln * (np.maximum(gm - em, 0) ** 2 + np.maximum(gs - es, 0) ** 2)
    lb32 = t.lb2(Q)[:, 0]
    assert (gm[:12] > 0).any() and (hi_terms[:12].sum(1) < 1e-6).any()
    _within_enclosure_error(lb32, (lo_terms, hi_terms), 4)
    assert (lb32[-20:] == 0.0).all()
    assert (lb32 == lb32.astype(np.float32)).all()  # a float32 value


def test_isax_float32_bound_within_enclosure_error():
    """iSAX MINDIST in float32 against the float64 one, on a tree whose leaf
    words end at the breakpoint 0.6745 (not a float32): two series with PAA
    (0.3, 0.3) and (1.0, 0.3) share a root child of capacity 1, which splits
    segment 0 at that breakpoint.  Queries put PAA_0 1e-4 on either side of it,
    where rounding the breakpoint inward would raise the bound far above the
    float64 one."""
    beta = O.isax_breakpoints(2)[2]  # 0.67449...
    X = np.array([[0.3, 0.3, 0.3, 0.3], [1.0, 1.0, 0.3, 0.3]], np.float32)
    t = O.Tree(X, "isax", leaf_cap=1, isax_w=2, isax_bits=2)
    assert t.L == 2
    la, lb_ = t.leaf_of()
    # leaf of series 0: segment 0 in [0, beta), segment 1 in [0, inf);
    # leaf of series 1: segment 0 in [beta, inf), segment 1 in [0, inf)
    ranges = {la: ((0.0, beta), (0.0, np.inf)), lb_: ((beta, np.inf), (0.0, np.inf))}
    vals = [beta + 1e-4, beta - 1e-4, beta + 3e-7, beta - 3e-7, 2.0, -0.5, 0.1]
    Q = np.array([[v, v, w, w] for v in vals for w in (0.25, -0.01)], np.float32)
    paa = Q.astype(np.float64).reshape(len(Q), 2, 2).mean(2)
    lb32 = t.lb2(Q)
    for leaf, rg in ranges.items():
        lo = np.array([r[0] for r in rg])
        hi = np.array([r[1] for r in rg])
        g, e = _gap_and_slack(paa, lo, hi)
        hi_terms = 2.0 * g * g
        lo_terms = 2.0 * np.maximum(g - e, 0) ** 2
        _within_enclosure_error(lb32[:, leaf], (lo_terms, hi_terms), 2)
    # 1e-4 from the breakpoint with segment 1 inside its range: one leaf's
    # bound is 0, the other's positive and about 2e-8
    near = lb32[[0, 2]]
    assert (near.min(1) == 0).all() and (near.max(1) > 1e-8).all() and (near.max(1) < 3e-8).all()


# ---------------------------------------------------------------- iSAX

def test_isax_breakpoints_are_normal_quantiles():
    for bits in (1, 2, 3, 8):
        beta = O.isax_breakpoints(bits)
        C = 1 << bits
        ref = scipy.stats.norm.ppf(np.arange(1, C) / C)
        assert np.allclose(beta, ref, rtol=0, atol=1e-12)
    assert O.isax_breakpoints(8)[127] == 0.0
    b2 = O.isax_breakpoints(2)
    assert b2[1] == 0.0 and abs(b2[2] - 0.6744897501960817) < 1e-12


def test_isax_mindist_hand_example():
    g = _golden("isax_mindist_hand.json")
    X = np.array(g["series"], np.float32)
    t = O.Tree(X, "isax", leaf_cap=g["leaf_cap"], isax_w=g["w"], isax_bits=g["bits"])
    assert t.L == 1
    q = np.array([g["query"]], np.float32)
    assert t.lb2(q)[0, 0] == g["lb2"]
    assert O.knn(X, q, 1)[1][0, 0] == g["d2"]


def test_isax_structure_and_lb_invariant(rw):
    X, Q = rw
    t = O.Tree(X, "isax", leaf_cap=200, isax_w=16, isax_bits=8)
    sizes = t.leaf_sizes()
    assert sizes.sum() == X.shape[0] and sizes.min() >= 1
    lo = t.leaf_of()
    assert (t.route(X[::5]) == lo[::5]).all()
    lb = t.lb2(Q)
    leaves = np.tile(np.arange(t.L, dtype=np.int32), (Q.shape[0], 1))
    d2, _ = t.leaf_topk(Q, leaves, 1)
    assert (lb * (1 - 1e-4) <= d2[:, :, 0]).all()


# ---------------------------------------------------------------- MLP filter

def test_mlp_forward_hand_weights():
    """W1 = I, b1 = 0, w2 = 1, b2 = 0.5  =>  y = 0.5 + sum_i relu(q_i)."""
    m = 8
    W1 = np.eye(m, dtype=np.float32)[None]
    b1 = np.zeros((1, m), np.float32)
    w2 = np.ones((1, m), np.float32)
    b2 = np.array([0.5], np.float32)
    Q = np.array([[1, -2, 3, -4, 0.25, 0, -1, 2]], np.float32)
    y = O.mlp_forward(W1, b1, w2, b2, Q)
    assert y[0, 0] == 0.5 + 1 + 3 + 0.25 + 2
    # one-hot hidden unit with a negative bias is cut by the ReLU
    b1n = np.full((1, m), -10.0, np.float32)
    assert O.mlp_forward(W1, b1n, w2, b2, Q)[0, 0] == 0.5


def _loss(W1, b1, w2, b2, X, T):
    Z = X @ W1.T + b1
    Y = np.maximum(Z, 0) @ w2 + b2
    return np.mean((Y - T) ** 2)


def test_sgd_step_matches_finite_difference_gradient():
    """One full-batch SGD step moves every weight by -lr * dLoss/dw."""
    rng = np.random.default_rng(5)
    m = h = 6
    ng, nl = 10, 5
    Qg = rng.standard_normal((ng, m)).astype(np.float32)
    Ql = rng.standard_normal((1, nl, m)).astype(np.float32)
    Tg = rng.uniform(1, 3, (ng, 1)).astype(np.float32)
    Tl = rng.uniform(1, 3, (1, nl)).astype(np.float32)
    W1 = rng.uniform(-.5, .5, (1, h, m)).astype(np.float32)
    b1 = rng.uniform(-.5, .5, (1, h)).astype(np.float32)
    w2 = rng.uniform(-.5, .5, (1, h)).astype(np.float32)
    b2 = np.array([0.1], np.float32)
    p = O.TrainParams(n_gtrain=8, n_gval=2, n_ltrain=4, n_lval=1, batch=12, max_epochs=1,
                      patience=10, lr0=1e-3, lr_min=1e-5)
    perms = np.arange(12, dtype=np.int32)[None]
    (W1n, b1n, w2n, b2n), ep, _ = O.train(p, Qg, Tg, Ql, Tl, perms, W1, b1, w2, b2)
    X = np.concatenate([Qg[:8], Ql[0, :4]]).astype(np.float64)
    T = np.concatenate([Tg[:8, 0], Tl[0, :4]]).astype(np.float64)
    P0 = [a.astype(np.float64)[0] for a in (W1, b1, w2)] + [np.float64(b2[0])]

    def L(params):
        return _loss(params[0], params[1], params[2], params[3], X, T)

    eps = 1e-6
    newp = [W1n[0], b1n[0], w2n[0], b2n[0]]
    for pi in range(4):
        base = np.array(P0[pi], dtype=np.float64)
        flat = base.reshape(-1)
        for idx in range(flat.size):
            plus = [np.array(a, copy=True) for a in P0]
            minus = [np.array(a, copy=True) for a in P0]
            plus[pi].reshape(-1)[idx] += eps
            minus[pi].reshape(-1)[idx] -= eps
            g = (L(plus) - L(minus)) / (2 * eps)
            moved = float(np.asarray(newp[pi], np.float64).reshape(-1)[idx]) - flat[idx]
            assert moved == pytest.approx(-1e-3 * g, abs=2e-7)


def test_training_reduces_validation_loss_and_plateau_stops():
    rng = np.random.default_rng(9)
    m = h = 16
    Qg = rng.standard_normal((50, m)).astype(np.float32)
    Ql = rng.standard_normal((2, 20, m)).astype(np.float32)
    wtrue = rng.standard_normal(m)
    Tg = np.abs(Qg @ wtrue)[:, None].repeat(2, 1).astype(np.float32)
    Tl = np.abs(Ql @ wtrue).astype(np.float32)
    W = fx.filter_init(2, m, h, seed=3)
    p = O.TrainParams(n_gtrain=40, n_gval=10, n_ltrain=16, n_lval=4, batch=8, max_epochs=400,
                      patience=3, lr0=0.01, lr_min=1e-5)
    perms = fx.epoch_permutations(400, 56, seed=4)
    Wt, ep, bv = O.train(p, Qg, Tg, Ql, Tl, perms, *W)
    Xv = np.concatenate([Qg[40:], Ql[0, 16:]])
    Tv = np.concatenate([Tg[40:, 0], Tl[0, 16:]])
    before = _loss(*(a[0].astype(np.float64) for a in W[:3]), np.float64(W[3][0]), Xv, Tv)
    after = _loss(*(a[0].astype(np.float64) for a in Wt[:3]), np.float64(Wt[3][0]), Xv, Tv)
    assert after < 0.8 * before
    assert after == pytest.approx(bv[0], rel=1e-4)
    # lr goes 1e-2 -> 1e-3 -> 1e-4 -> 1e-5 and stops at the next plateau
    assert (ep < 400).all()


@pytest.mark.parametrize("case", ["constant", "constant_capped", "halving", "one_step"])
def test_sgd_plateau_schedule_hand_counted(case):
    """Epoch counts of the plateau schedule, the strict-improvement rule and the
    kept best-validation weights on cases counted by hand
    (tests/golden/sgd_plateau_hand.json)."""
    c = _golden("sgd_plateau_hand.json")["cases"][case]
    m = h = 2
    Qg = np.array([[1, 2], [-1, 0.5], [0.25, -2], [3, 1]], np.float32)
    Ql = np.array([[[2, 2], [-3, 1], [0, 1], [1, -1]]], np.float32)
    Tg = np.array([[c["train_target"]]] * 2 + [[c["val_target"]]] * 2, np.float32)
    Tl = np.array([[c["train_target"]] * 2 + [c["val_target"]] * 2], np.float32)
    W1 = np.zeros((1, h, m), np.float32)
    b1 = np.full((1, h), -1.0, np.float32)
    w2 = np.array([[0.5, -0.25]], np.float32)
    b2 = np.array([c["b2"]], np.float32)
    p = O.TrainParams(n_gtrain=2, n_gval=2, n_ltrain=2, n_lval=2, batch=4,
                      max_epochs=c["max_epochs"], patience=c["patience"], lr0=c["lr0"],
                      lr_min=c["lr_min"])
    perms = np.tile(np.array([2, 0, 3, 1], np.int32), (c["max_epochs"], 1))
    (W1n, b1n, w2n, b2n), ep, bv = O.train(p, Qg, Tg, Ql, Tl, perms, W1, b1, w2, b2)
    assert int(ep[0]) == c["epochs"]
    assert float(bv[0]) == c["best_val"]
    assert float(b2n[0]) == np.float32(c["b2_kept"])
    # dead hidden units: nothing else moves
    assert np.array_equal(W1n, W1) and np.array_equal(b1n, b1) and np.array_equal(w2n, w2)


# ---------------------------------------------------------------- Alg. 1 random draws

def test_philox_known_answers():
    """The oracle's Philox4x32-10 reproduces the generator's published
    known-answer vectors (tests/golden/philox4x32_kat.json)."""
    for v in _golden("philox4x32_kat.json")["vectors"]:
        out = O.philox4x32_10([int(w, 16) for w in v["ctr"]], [int(w, 16) for w in v["key"]])
        assert [int(w) for w in out] == [int(w, 16) for w in v["out"]]


@pytest.fixture(scope="module")
def gen_tree():
    X = fx.random_walk(4000, 64, seed=31)
    return X, O.Tree(X, "dstree", leaf_cap=300, init_segments=4)


def test_training_queries_picks(gen_tree):
    """Global picks are distinct dataset ids; local picks are members of their
    leaf, distinct when the leaf is large enough, drawn with replacement
    otherwise (Alg. 1's query generation)."""
    X, t = gen_tree
    sizes = t.leaf_sizes()
    small = int(np.argmin(sizes))
    big = int(np.argmax(sizes))
    nl = int(sizes[small]) + 5
    assert sizes[big] >= nl
    Qg, Ql, gp, lp = O.training_queries(t, [big, small], 700, nl, 0.1, 0.4, seed=5)
    assert len(set(gp.tolist())) == 700 and gp.min() >= 0 and gp.max() < X.shape[0]
    lo = t.leaf_of()
    assert (lo[lp[0]] == big).all() and len(set(lp[0].tolist())) == nl
    assert (lo[lp[1]] == small).all()          # more picks than members: repeats
    # deterministic, and another seed draws other series
    assert np.array_equal(O.training_queries(t, [big, small], 700, nl, 0.1, 0.4, seed=5)[2], gp)
    assert not np.array_equal(O.training_queries(t, [big, small], 700, nl, 0.1, 0.4, seed=6)[2],
                              gp)


def test_training_queries_noise_and_normalisation(gen_tree):
    """Every query is z-normalised (mean 0, population sigma 1) and its
    correlation with its source series is 1 / sqrt(1 + sigma^2) for unit-variance
    series plus N(0, sigma^2) noise (checked on the mean over many queries)."""
    X, t = gen_tree
    for sig in (0.1, 0.4):
        Qg, _, gp, _ = O.training_queries(t, [0], 3000, 1, sig, sig, seed=9)
        q = Qg.astype(np.float64)
        assert np.abs(q.mean(1)).max() < 1e-6
        assert np.abs(q.std(1) - 1.0).max() < 1e-6
        x = X[gp].astype(np.float64)
        corr = (q * x).mean(1)                      # both rows z-normalised
        expect = 1.0 / np.sqrt(1.0 + sig * sig)
        assert abs(corr.mean() - expect) < 0.002, (sig, corr.mean(), expect)


def test_floyd_picks_are_uniform():
    """Each of 10 ids is drawn with probability 3/10 over many seeds."""
    X = fx.random_walk(10, 8, seed=3)
    t = O.Tree(X, "dstree", leaf_cap=20, init_segments=2)
    counts = np.zeros(10)
    for seed in range(2000):
        gp = O.training_queries(t, [0], 3, 1, 0.1, 0.1, seed=seed)[2]
        assert len(set(gp.tolist())) == 3
        counts[gp] += 1
    assert np.abs(counts - 600).max() < 5 * np.sqrt(2000 * 0.3 * 0.7)


def test_filter_init_and_epoch_perms():
    W1, b1, w2, b2 = O.filter_init(3, 16, 64, seed=4)
    a1, a2 = 1 / np.sqrt(64), 1 / np.sqrt(16)
    assert np.abs(W1).max() <= a1 and np.abs(b1).max() <= a1
    assert np.abs(w2).max() <= a2 and np.abs(b2).max() <= a2
    assert abs(W1.mean()) < 0.05 * a1 and abs(W1.var() / (a1 * a1 / 3) - 1) < 0.05
    assert np.array_equal(O.filter_init(3, 16, 64, seed=4)[0], W1)
    P = O.epoch_perms(5, 100, seed=4)
    assert all(sorted(p.tolist()) == list(range(100)) for p in P)
    assert len({tuple(p.tolist()) for p in P}) == 5


# ---------------------------------------------------------------- Steffen

def test_steffen_properties():
    x = np.array([0.0, 1.0, 2.5, 3.0, 5.0])
    y = np.array([0.0, 0.5, 0.6, 2.0, 2.1])
    for xi, yi in zip(x, y):
        assert O.steffen_eval(x, y, xi) == pytest.approx(yi, abs=1e-15)
    xs = np.linspace(-1, 6, 701)
    ys = np.array([O.steffen_eval(x, y, v) for v in xs])
    assert (np.diff(ys) >= -1e-15).all()          # monotone on monotone data
    assert ys.min() >= y.min() - 1e-15 and ys.max() <= y.max() + 1e-15  # no overshoot
    lin = 3.0 * x - 1.0
    for v in np.linspace(0, 5, 51):
        assert O.steffen_eval(x, lin, v) == pytest.approx(3.0 * v - 1.0, abs=1e-12)


# ---------------------------------------------------------------- search

def _alg2_sequential(lb_row, route, lists, df_row, k, searched=None):
    """Literal Alg. 2 loop: route leaf first, then ascending (LB, id).
    `searched` (a set, optional) receives the leaves the loop searches."""
    L = lb_row.shape[0]
    order = [route] + sorted((l for l in range(L) if l != route), key=lambda l: (lb_row[l], l))
    res = []
    bsf = np.float32(np.inf)
    for leaf in order:
        if lb_row[leaf] * (1 - 1e-4) > float(bsf):
            continue
        if df_row is not None and not np.isnan(df_row[leaf]) and \
                df_row[leaf] > float(np.sqrt(np.float32(bsf))):
            continue
        if searched is not None:
            searched.add(leaf)
        d2, ids = lists[leaf]
        res = sorted(res + [(float(a), int(b)) for a, b in zip(d2, ids) if b >= 0])[:k]
        bsf = np.float32(res[k - 1][0]) if len(res) == k else np.float32(np.inf)
    return [b for _, b in res]


@pytest.fixture(scope="module")
def small_index():
    X = fx.random_walk(3000, 32, seed=21)
    t = O.Tree(X, "dstree", leaf_cap=150, init_segments=4)
    Q = fx.test_queries(X, 30, seed=22)
    return X, t, Q


def test_exact_search_equals_brute_force_for_any_wave(small_index):
    X, t, Q = small_index
    for k in (1, 5, 40):
        bf_ids, bf_d2 = O.knn(X, Q, k)
        for wave in (1, 3, 1000):
            ids, d2, st, _ = O.leafi_search(t, None, None, None, Q, k, -1, wave)
            assert np.array_equal(ids, bf_ids) and np.array_equal(d2, bf_d2)
            assert (st[:, 0] <= t.L).all()


def test_searched_leaves_of_wave_one_are_the_sequential_algorithms(small_index):
    """The per-query searched-leaf flags of the oracle's search (Alg. 2) at
    W = 1 are exactly the leaves a literal transcription of the loop searches,
    with filters and without; they agree with the search's own counters."""
    X, t, Q = small_index
    rng = np.random.default_rng(8)
    F = min(6, t.L)
    W = fx.filter_init(F, 32, 32, seed=9)
    fl = np.arange(F, dtype=np.int32)
    alpha = np.sort(rng.uniform(0, 3, (F, 7)), axis=1)[:, ::-1].copy()
    P = O.mlp_forward(*W, Q)
    lb = t.lb2(Q)
    route = t.route(Q)
    sizes = t.leaf_sizes()
    leaves = np.tile(np.arange(t.L, dtype=np.int32), (Q.shape[0], 1))
    for k in (1, 4):
        d2l, idl = t.leaf_topk(Q, leaves, k)
        for j in (-1, 0, 3, 6):
            _, _, st, _, sc = O.leafi_search_pred(t, P, fl, alpha, Q, k, j, 1, return_scanned=True)
            assert sc.dtype == np.uint8 and set(np.unique(sc).tolist()) <= {0, 1}
            assert np.array_equal(sc.sum(axis=1), st[:, 0])
            assert np.array_equal(sc.astype(np.int64) @ sizes, st[:, 1])
            pruned_some = False
            for i in range(Q.shape[0]):
                df = None
                if j >= 0:
                    df = np.full(t.L, np.nan)
                    df[fl] = P[i] - alpha[:, j]
                lists = [(d2l[i, l], idl[i, l]) for l in range(t.L)]
                searched = set()
                _alg2_sequential(lb[i], route[i], lists, df, k, searched)
                assert set(np.flatnonzero(sc[i]).tolist()) == searched, (k, j, i)
                pruned_some |= len(searched) < t.L
            assert pruned_some


def test_wave_one_is_the_sequential_algorithm(small_index):
    X, t, Q = small_index
    rng = np.random.default_rng(4)
    F = min(6, t.L)
    W = fx.filter_init(F, 32, 32, seed=5)
    fl = np.arange(F, dtype=np.int32)
    alpha = np.sort(rng.uniform(0, 3, (F, 7)), axis=1)[:, ::-1].copy()
    P = O.mlp_forward(*W, Q)
    lb = t.lb2(Q)
    route = t.route(Q)
    leaves = np.tile(np.arange(t.L, dtype=np.int32), (Q.shape[0], 1))
    for k in (1, 4):
        d2l, idl = t.leaf_topk(Q, leaves, k)
        for j in (0, 3, 6):
            ids, _, _, _ = O.leafi_search(t, W, fl, alpha, Q, k, j, 1)
            for i in range(Q.shape[0]):
                df = np.full(t.L, np.nan)
                df[fl] = P[i] - alpha[:, j]
                lists = [(d2l[i, l], idl[i, l]) for l in range(t.L)]
                ref = _alg2_sequential(lb[i], route[i], lists, df, k)
                assert ids[i, :len(ref)].tolist() == ref


def test_autotuner_hand_example():
    """Alg. 4 on a case worked by hand: the alpha table element by element and
    the quality at every sorted position, for k = 1 and 2 and two wave widths
    (tests/golden/alg4_autotuner_hand.json)."""
    g = _golden("alg4_autotuner_hand.json")
    X = np.array(g["series"], np.float32)
    t = O.Tree(X, "dstree", leaf_cap=g["leaf_cap"], init_segments=g["init_segments"])
    assert t.leaf_of().tolist() == g["leaf_of"]
    Qc = np.array(g["calibration"], np.float32)
    assert t.route(Qc).tolist() == g["route"]
    W = tuple(np.array(g[k], np.float32) for k in ("W1", "b1", "w2", "b2"))
    assert O.mlp_forward(*W, Qc).tolist() == g["predictions"]
    fl = np.array(g["filter_leaf"], np.int32)
    for k, qp_hand in g["qprime"].items():
        for wave in g["waves"]:
            alpha, qp = O.fit_autotuner(t, W, fl, Qc, int(k), wave)
            assert alpha.tolist() == g["alpha_sorted"]
            assert qp.tolist() == qp_hand, (k, wave)


def _informative_filters(t, Qc, seed):
    """Random filters whose output bias sits near each leaf's typical d^L, so
    that the offsets decide what is pruned."""
    F = t.L
    W1, b1, w2, b2 = fx.filter_init(F, t.m, t.m, seed=100 + seed)
    leaves = np.tile(np.arange(t.L, dtype=np.int32), (Qc.shape[0], 1))
    d2, _ = t.leaf_topk(Qc, leaves, 1)
    med = np.median(np.sqrt(d2[:, :, 0]), 0)
    b2 = (med + np.random.default_rng(seed).normal(0, 1.0, F)).astype(np.float32)
    return (W1, b1, w2 * 3, b2)


@pytest.mark.parametrize("seed,k,wave", [(21, 3, 1), (24, 3, 2), (3, 1, 2)])
def test_autotuner_table_matches_search_recall(seed, k, wave):
    """Alg. 4's simulated quality at each position, monotonised by the running
    minimum, equals the running minimum of the recall that the search itself
    reaches with those offsets, measured against brute force.  The first two
    cases have a non-monotone measured recall, so they exercise the running
    minimum."""
    X = fx.random_walk(3000, 32, seed=21)
    t = O.Tree(X, "dstree", leaf_cap=150, init_segments=4)
    Qc = fx.test_queries(X, 60, seed=22)[:24]
    W = _informative_filters(t, Qc, seed)
    fl = np.arange(t.L, dtype=np.int32)
    alpha, qp = O.fit_autotuner(t, W, fl, Qc, k, wave)
    assert (np.diff(alpha, axis=1) <= 0).all()          # descending per filter
    assert (np.diff(qp) <= 0).all() and qp[0] == 1.0
    bf, _ = O.knn(X, Qc, k)
    rec = np.array([O.recall_at_k(O.leafi_search(t, W, fl, alpha, Qc, k, j, wave)[0], bf,
                                  k).mean() for j in range(Qc.shape[0])])
    assert rec.min() < 0.9                                # the offsets matter here
    assert np.allclose(qp, np.minimum.accumulate(rec), rtol=0, atol=1e-12)
    if seed in (21, 24):
        assert (np.diff(rec) > 0).any()


def test_required_quality_is_the_binomial_tail_bound():
    """The quality that certifies target t with probability 0.95 from N
    calibration neighbours: (N - M*) / N where M* is the most misses whose
    binomial tail P(Bin(N, 1 - t) <= M*) stays at or below 0.05 (scipy's
    binomial distribution as the independent reference)."""
    for N, t in ((300, 0.99), (300, 0.95), (300, 0.9), (3000, 0.99), (80, 0.9), (30000, 0.95),
                 (1000, 0.5)):
        r = O.required_quality(N, t, 0.95)
        cdf = scipy.stats.binom.cdf(np.arange(N + 1), N, 1 - t)
        ok = np.nonzero(cdf <= 0.05)[0]
        if len(ok) == 0:
            assert r == 2.0
        else:
            assert r == (N - ok.max()) / N, (N, t, r)
    # hand values: 300 calibration queries at 0.99 allow no miss (0.99^300 = 0.049 <= 0.05,
    # one miss has tail 0.197); 80 queries cannot certify 0.99 (0.99^80 = 0.45)
    assert O.required_quality(300, 0.99, 0.95) == 1.0
    assert O.required_quality(80, 0.99, 0.95) == 2.0
    assert O.required_quality(300, 0.99, 0.0) == 0.99        # point estimate
    assert O.required_quality(300, 1.0, 0.95) == 2.0


def test_offset_position_step_rule():
    """STEP: the largest sorted position whose (non-increasing) quality reaches
    the required one; none -> -1 (exact search)."""
    qp = np.array([1.0, 1.0, 0.99, 0.97, 0.97, 0.9])
    assert O.offset_position(qp, 0.99, confidence=0.0) == 2
    assert O.offset_position(qp, 0.95, confidence=0.0) == 4
    assert O.offset_position(qp, 1.0, confidence=0.0) == -1
    assert O.offset_position(np.array([0.9, 0.8]), 0.95, confidence=0.0) == -1
    # 300 calibration queries at 0.95 with confidence 0.95 allow 8 misses (0.97333)
    qp = np.linspace(1.0, 0.9, 300)
    r = O.required_quality(300, 0.95)
    assert r == 292 / 300
    assert O.offset_position(qp, 0.95) == int(np.nonzero(qp >= r)[0].max())
    # k = 10: ten neighbours per query, 3000 trials
    assert O.offset_position(qp, 0.99, kk=10) == int(np.nonzero(qp >= O.required_quality(3000, 0.99))[0].max())


def test_huge_offsets_give_the_exact_answer(small_index):
    X, t, Q = small_index
    F = t.L
    W = fx.filter_init(F, 32, 32, seed=8)
    alpha = np.full((F, 1), 1e30)
    ids, d2, _, _ = O.leafi_search(t, W, np.arange(F, dtype=np.int32), alpha, Q, 3, 0, 4)
    bf_ids, bf_d2 = O.knn(X, Q, 3)
    assert np.array_equal(ids, bf_ids)


def test_train_targets_are_leaf_minima(small_index):
    X, t, Q = small_index
    fl = np.array([0, t.L - 1], np.int32)
    Ql = np.stack([Q[:5], Q[5:10]])
    Tg, Tl = O.train_targets(t, fl, Q, Ql)
    for f, leaf in enumerate(fl):
        mem = t.leaf_members(int(leaf))
        for i in range(Q.shape[0]):
            d = min(O.sqdist(Q[i], X[s]) for s in mem)
            assert Tg[i, f] == np.sqrt(np.float32(d))
        for i in range(5):
            d = min(O.sqdist(Ql[f, i], X[s]) for s in mem)
            assert Tl[f, i] == np.sqrt(np.float32(d))


def test_select_leaves_alg3_pins():
    """Alg. 3 on a hand example: leaves by size (ties: lower id), the size
    threshold, and the memory budget read as w^M + w <= c^M."""
    sizes = [5, 9, 9, 2, 7]
    # th = 6: the leaves of size 9, 9 and 7 qualify; a budget of two filters takes the two largest
    assert list(O.select_leaves_alg3(sizes, 6, 1, 2)) == [1, 2]
    assert list(O.select_leaves_alg3(sizes, 6, 1, 1e9)) == [1, 2, 4]
    # th = 0 and room for all: every leaf, largest first, equal sizes by id
    assert list(O.select_leaves_alg3(sizes, 0, 1, 1e9)) == [1, 2, 4, 0, 3]
    # 1.5 + 1.5 <= 3 admits two filters; a third would overshoot the budget
    assert list(O.select_leaves_alg3(sizes, 0, 1.5, 3.0)) == [1, 2]
    assert list(O.select_leaves_alg3(sizes, 10, 1, 1e9)) == []
    # th = 0 and a budget of F filters: the F largest (the configurations' rule)
    rng = np.random.default_rng(5)
    sz = rng.integers(1, 50, 200)
    order = sorted(range(200), key=lambda i: (-sz[i], i))
    assert list(O.select_leaves_alg3(sz, 0, 3.0, 3.0 * 17)) == order[:17]


# ---------------------------------------------------------------- CNN filters (Sec. 5.2)

def _cnn_theta(C, m, w1, b1, w2, b2, wo, bo):
    """Pack per-layer arrays into the flat layout w1, b1, w2, b2, wo, bo."""
    th = np.concatenate([np.asarray(w1, np.float32).ravel(), np.asarray(b1, np.float32).ravel(),
                         np.asarray(w2, np.float32).ravel(), np.asarray(b2, np.float32).ravel(),
                         np.asarray(wo, np.float32).ravel(), np.float32([bo])])
    assert th.size == O.cnn_params(C) == 3 * C * C + 6 * C + 1
    return th[None]


@pytest.mark.parametrize("tap", [0, 2])
def test_cnn_forward_hand_weights(tap):
    """Two channels: the first layer passes relu(x) and relu(-x); the second
    sums them (|x|) on channel 0 and shifts relu(x) by one position on channel
    1 (tap 0 meets position i - 1, tap 2 position i + 1; zero padding drops the
    series' last / first value).  With wo = (1, 2), bo = 0.5 and mean pooling:
        y = 0.5 + mean|x| + 2 (sum of relu(x) over the kept positions) / m."""
    C, m = 2, 5
    w1 = [[0, 1, 0], [0, -1, 0]]
    b1 = [0, 0]
    w2 = np.zeros((2, 2, 3), np.float32)
    w2[0, 0, 1] = w2[0, 1, 1] = 1.0
    w2[1, 0, tap] = 1.0
    th = _cnn_theta(C, m, w1, b1, w2, [0, 0], [1, 2], 0.5)
    x = np.array([[1.5, -2.0, 3.0, -0.5, 0.25]], np.float32)
    x64 = x.astype(np.float64)
    kept = x64[0, :-1] if tap == 0 else x64[0, 1:]
    want = 0.5 + np.abs(x64).sum() / m + 2 * np.maximum(kept, 0).sum() / m
    assert O.cnn_forward(th, C, x)[0, 0] == pytest.approx(want, abs=1e-15)
    # biases: b1 = -1 cuts both channels (|x| > 1 survives on channel 0 only
    # through relu(x - 1) + relu(-x - 1)); b2 = -10 silences channel 1
    th2 = _cnn_theta(C, m, w1, [-1, -1], w2, [0, -10], [1, 2], 0.5)
    want2 = 0.5 + (np.maximum(x64 - 1, 0) + np.maximum(-x64 - 1, 0)).sum() / m
    assert O.cnn_forward(th2, C, x)[0, 0] == pytest.approx(want2, abs=1e-15)


def test_cnn_sgd_step_matches_finite_difference_gradient():
    """One full-batch SGD step moves every CNN parameter by -lr dLoss/dtheta,
    the loss (the minibatch MSE) evaluated through the oracle forward that the
    hand-weight test pins.  Parameters sit on a 2^-12 grid so theta +- 2^-12 is
    exact in float32; along one parameter the prediction is piecewise linear
    (ReLU kinks) and the loss piecewise quadratic, so the central difference is
    exact up to rounding when no kink lies within the step (a coarser step,
    2^-8, does meet kinks on these data and is off by up to 30%)."""
    rng = np.random.default_rng(11)
    C, m, n = 3, 7, 6
    P = O.cnn_params(C)
    th = (np.round(rng.uniform(-0.6, 0.6, (1, P)) * 4096) / 4096).astype(np.float32)
    Qg = rng.standard_normal((n + 1, m)).astype(np.float32)
    Tg = rng.uniform(0.5, 2.0, (n + 1, 1)).astype(np.float32)
    Ql = np.zeros((1, 1, m), np.float32)
    Tl = np.zeros((1, 1), np.float32)
    lr = 0.0625
    p = O.TrainParams(n_gtrain=n, n_gval=1, n_ltrain=0, n_lval=0, batch=n, max_epochs=1,
                      patience=10, lr0=lr, lr_min=1e-5)
    perms = np.arange(n, dtype=np.int32)[None]
    th1, ep, _ = O.cnn_train(p, C, Qg, Tg, Ql, Tl, perms, th)
    assert int(ep[0]) == 1

    def loss(t):
        y = O.cnn_forward(t, C, Qg[:n])[:, 0]
        return np.mean((y - Tg[:n, 0].astype(np.float64)) ** 2)

    eps = 2.0 ** -12
    moved = th1[0].astype(np.float64) - th[0].astype(np.float64)
    for e in range(P):
        tp, tm = th.copy(), th.copy()
        tp[0, e] += np.float32(eps)
        tm[0, e] -= np.float32(eps)
        g = (loss(tp) - loss(tm)) / (2 * eps)
        assert moved[e] == pytest.approx(-lr * g, abs=2e-7, rel=1e-5), e


@pytest.mark.parametrize("case", ["constant", "constant_capped", "halving", "one_step"])
def test_cnn_sgd_plateau_schedule_hand_counted(case):
    """The CNN trainer keeps the MLP trainer's protocol: with both convolutions
    dead (b1 = b2 = -1, w1 = w2 = 0) the prediction is bo and only bo moves, so
    the hand-counted epochs, best loss and kept bias of the MLP cases hold
    (tests/golden/sgd_plateau_hand.json)."""
    c = _golden("sgd_plateau_hand.json")["cases"][case]
    C, m = 2, 2
    Qg = np.array([[1, 2], [-1, 0.5], [0.25, -2], [3, 1]], np.float32)
    Ql = np.array([[[2, 2], [-3, 1], [0, 1], [1, -1]]], np.float32)
    Tg = np.array([[c["train_target"]]] * 2 + [[c["val_target"]]] * 2, np.float32)
    Tl = np.array([[c["train_target"]] * 2 + [c["val_target"]] * 2], np.float32)
    th = _cnn_theta(C, m, np.zeros((2, 3)), [-1, -1], np.zeros((2, 2, 3)), [-1, -1],
                    [0.5, -0.25], c["b2"])
    p = O.TrainParams(n_gtrain=2, n_gval=2, n_ltrain=2, n_lval=2, batch=4,
                      max_epochs=c["max_epochs"], patience=c["patience"], lr0=c["lr0"],
                      lr_min=c["lr_min"])
    perms = np.tile(np.array([2, 0, 3, 1], np.int32), (c["max_epochs"], 1))
    th1, ep, bv = O.cnn_train(p, C, Qg, Tg, Ql, Tl, perms, th)
    assert int(ep[0]) == c["epochs"]
    assert float(bv[0]) == c["best_val"]
    assert float(th1[0, -1]) == np.float32(c["b2_kept"])
    assert np.array_equal(th1[0, :-1], th[0, :-1])


def test_cnn_init_bounds_and_determinism():
    C = 24
    th = O.cnn_init(3, C, seed=6)
    a1, a2, ao = 1 / np.sqrt(3), 1 / np.sqrt(3 * C), 1 / np.sqrt(C)
    w1b1, w2b2, wobo = th[:, :4 * C], th[:, 4 * C:4 * C + 3 * C * C + C], th[:, -(C + 1):]
    assert np.abs(w1b1).max() <= a1 and np.abs(w2b2).max() <= a2 and np.abs(wobo).max() <= ao
    assert np.abs(w1b1).max() > 0.9 * a1 and np.abs(w2b2).max() > 0.99 * a2
    assert abs(w2b2.var() / (a2 * a2 / 3) - 1) < 0.05
    assert np.array_equal(O.cnn_init(3, C, seed=6), th)
    assert not np.array_equal(O.cnn_init(3, C, seed=7), th)


def test_prediction_entry_points_equal_the_mlp_ones(small_index):
    """Alg. 4 and Alg. 2 on given predictions are the MLP entry points with the
    MLP's predictions (the CNN parity checks run through the former)."""
    X, t, _ = small_index
    Q = fx.test_queries(X, 80, seed=23)
    fl = np.arange(min(4, t.L), dtype=np.int32)
    W = O.filter_init(len(fl), 16, t.m, seed=2)
    a1, q1 = O.fit_autotuner(t, W, fl, Q[:40], 1, 4)
    a2, q2 = O.fit_autotuner_pred(t, O.mlp_forward(*W, Q[:40]), fl, Q[:40], 1, 4)
    assert np.array_equal(a1, a2) and np.array_equal(q1, q2)
    jp = np.full(len(Q) - 40, 10, np.int32)
    r1 = O.leafi_search(t, W, fl, a1, Q[40:], 1, jp, 4)
    r2 = O.leafi_search_pred(t, O.mlp_forward(*W, Q[40:]), fl, a1, Q[40:], 1, jp, 4)
    for u, v in zip(r1, r2):
        assert np.array_equal(u, v)
