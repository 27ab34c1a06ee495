"""ctypes wrapper of the LeaFi oracle (TEST INFRASTRUCTURE ONLY).

Each function mirrors one step of the paper; the arithmetic lives in
`leafi_oracle.c` and is cited there.  Arrays are numpy, C-contiguous.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

__all__ = [
    "build", "lib", "sqdist", "knn", "segment_stats", "Tree", "isax_breakpoints",
    "mlp_forward", "train_targets", "TrainParams", "train", "fit_autotuner",
    "offset_position", "required_quality", "philox4x32_10", "training_queries",
    "filter_init", "epoch_perms", "steffen_eval", "leafi_search", "recall_at_k", "select_leaves_alg3",
    "cnn_params", "cnn_forward", "cnn_init", "cnn_train", "fit_autotuner_pred", "leafi_search_pred",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "leafi_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99 + OpenMP, no fast-math)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "leafi_oracle.h"))):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu99", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _TrainParams(C.Structure):
    _fields_ = [("n_gtrain", C.c_int32), ("n_gval", C.c_int32), ("n_ltrain", C.c_int32),
                ("n_lval", C.c_int32), ("batch", C.c_int32), ("max_epochs", C.c_int32),
                ("patience", C.c_int32), ("lr0", C.c_double), ("lr_min", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        vp = C.c_void_p
        L.or_sqdist.argtypes = [f32p, f32p, C.c_int]
        L.or_sqdist.restype = C.c_float
        L.or_knn.argtypes = [f32p, C.c_int64, C.c_int, f32p, C.c_int64, C.c_int, i64p, f32p]
        L.or_segment_stats.argtypes = [f32p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double)]
        L.or_dstree_build.argtypes = [f32p, C.c_int64, C.c_int, C.c_int, C.c_int]
        L.or_dstree_build.restype = vp
        L.or_isax_build.argtypes = [f32p, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int]
        L.or_isax_build.restype = vp
        L.or_tree_free.argtypes = [vp]
        L.or_tree_n_leaves.argtypes = [vp]
        L.or_tree_n_leaves.restype = C.c_int32
        L.or_tree_n_nodes.argtypes = [vp]
        L.or_tree_n_nodes.restype = C.c_int32
        L.or_tree_leaf_of.argtypes = [vp, i32p]
        L.or_tree_leaf_sizes.argtypes = [vp, i64p]
        L.or_tree_leaf_members.argtypes = [vp, C.c_int32, i64p, C.c_int64]
        L.or_tree_leaf_members.restype = C.c_int64
        L.or_isax_breakpoints.argtypes = [C.c_int, f64p]
        L.or_leaf_lb2.argtypes = [vp, f32p, C.c_int64, f64p]
        L.or_route.argtypes = [vp, f32p, C.c_int64, i32p]
        L.or_leaf_topk.argtypes = [vp, f32p, C.c_int64, i32p, C.c_int, C.c_int, f32p, i64p]
        L.or_mlp_forward.argtypes = [f32p, f32p, f32p, f32p, C.c_int, C.c_int, C.c_int, f32p,
                                     C.c_int64, f64p]
        L.or_train_targets.argtypes = [vp, i32p, C.c_int, f32p, C.c_int64, f32p, C.c_int64, f32p,
                                       f32p]
        L.or_train.argtypes = [C.POINTER(_TrainParams), C.c_int, C.c_int, C.c_int, f32p, f32p,
                               f32p, f32p, i32p, f32p, f32p, f32p, f32p, i32p, f64p]
        L.or_fit_autotuner.argtypes = [vp, f32p, f32p, f32p, f32p, i32p, C.c_int, C.c_int, f32p,
                                       C.c_int64, C.c_int, C.c_int, f64p, f64p]
        L.or_select_leaves_alg3.argtypes = [C.POINTER(C.c_int64), C.c_int32, C.c_double,
                                            C.c_double, C.c_double, C.POINTER(C.c_int32)]
        L.or_select_leaves_alg3.restype = C.c_int32
        L.or_offset_position.argtypes = [f64p, C.c_int64, C.c_int64, C.c_double, C.c_double]
        L.or_offset_position.restype = C.c_int32
        u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
        L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.or_training_queries.argtypes = [vp, i32p, C.c_int, C.c_int64, C.c_int64, C.c_double,
                                          C.c_double, C.c_uint64, f32p, f32p, i64p, i64p]
        L.or_filter_init.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, f32p, f32p, f32p, f32p]
        L.or_epoch_perms.argtypes = [C.c_int, C.c_int, C.c_uint64, i32p]
        L.or_required_quality.argtypes = [C.c_int64, C.c_double, C.c_double]
        L.or_required_quality.restype = C.c_double
        L.or_steffen_eval.argtypes = [f64p, f64p, C.c_int, C.c_double]
        L.or_steffen_eval.restype = C.c_double
        L.or_leafi_search.argtypes = [vp, f32p, f32p, f32p, f32p, i32p, C.c_int, C.c_int, f64p,
                                      C.c_int64, f32p, C.c_int64, i32p, i32p, C.c_int, C.c_int,
                                      i64p, f32p, i64p, f64p]
        L.or_leafi_search_pred.argtypes = [vp, f64p, i32p, C.c_int, f64p, C.c_int64, f32p,
                                           C.c_int64, i32p, i32p, C.c_int, C.c_int, i64p, f32p,
                                           i64p, f64p, vp]
        L.or_fit_autotuner_pred.argtypes = [vp, f64p, i32p, C.c_int, f32p, C.c_int64, C.c_int,
                                            C.c_int, f64p, f64p]
        L.or_cnn_params.argtypes = [C.c_int]
        L.or_cnn_params.restype = C.c_int64
        L.or_cnn_forward.argtypes = [f32p, C.c_int, C.c_int, C.c_int, f32p, C.c_int64, f64p]
        L.or_cnn_init.argtypes = [C.c_int, C.c_int, C.c_uint64, f32p]
        L.or_cnn_train.argtypes = [C.POINTER(_TrainParams), C.c_int, C.c_int, C.c_int, f32p,
                                   f32p, f32p, f32p, i32p, f32p, i32p, f64p]
        _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def sqdist(q, x) -> np.float32:
    q, x = _f32(q), _f32(x)
    return np.float32(lib().or_sqdist(q, x, q.shape[0]))


def knn(X, Q, k):
    X, Q = _f32(X), _f32(Q)
    nq = Q.shape[0]
    ids = np.empty((nq, k), np.int64)
    d2 = np.empty((nq, k), np.float32)
    lib().or_knn(X, X.shape[0], X.shape[1], Q, nq, k, ids, d2)
    return ids, d2


def segment_stats(x, s, e):
    x = _f32(x)
    mu, sd = C.c_double(), C.c_double()
    lib().or_segment_stats(x, x.shape[0], s, e, C.byref(mu), C.byref(sd))
    return mu.value, sd.value


def isax_breakpoints(bits):
    out = np.empty((1 << bits) - 1, np.float64)
    lib().or_isax_breakpoints(bits, out)
    return out


class Tree:
    """A DSTree or iSAX index over X (X is kept alive by the object)."""

    def __init__(self, X, kind="dstree", leaf_cap=2000, init_segments=4, isax_w=16,
                 isax_bits=8):
        self.X = _f32(X)
        n, m = self.X.shape
        self.kind = kind
        if kind == "dstree":
            self._h = lib().or_dstree_build(self.X, n, m, leaf_cap, init_segments)
        elif kind == "isax":
            self._h = lib().or_isax_build(self.X, n, m, leaf_cap, isax_w, isax_bits)
        else:
            raise ValueError(kind)
        if not self._h:
            raise ValueError("oracle tree build rejected its parameters")
        self.n, self.m = n, m
        self.L = lib().or_tree_n_leaves(self._h)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_tree_free(self._h)
            self._h = None

    @property
    def n_nodes(self):
        return lib().or_tree_n_nodes(self._h)

    def leaf_of(self):
        out = np.empty(self.n, np.int32)
        lib().or_tree_leaf_of(self._h, out)
        return out

    def leaf_sizes(self):
        out = np.empty(self.L, np.int64)
        lib().or_tree_leaf_sizes(self._h, out)
        return out

    def leaf_members(self, leaf):
        sz = int(self.leaf_sizes()[leaf])
        out = np.empty(max(sz, 1), np.int64)
        lib().or_tree_leaf_members(self._h, leaf, out, sz)
        return out[:sz]

    def lb2(self, Q):
        Q = _f32(Q)
        out = np.empty((Q.shape[0], self.L), np.float64)
        lib().or_leaf_lb2(self._h, Q, Q.shape[0], out)
        return out

    def route(self, Q):
        Q = _f32(Q)
        out = np.empty(Q.shape[0], np.int32)
        lib().or_route(self._h, Q, Q.shape[0], out)
        return out

    def leaf_topk(self, Q, leaves, k):
        """leaves: int32 [nq, nl] (-1 = none) -> (d2 [nq,nl,k], ids [nq,nl,k])."""
        Q = _f32(Q)
        leaves = np.ascontiguousarray(leaves, np.int32)
        nq, nl = leaves.shape
        d2 = np.empty((nq, nl, k), np.float32)
        ids = np.empty((nq, nl, k), np.int64)
        lib().or_leaf_topk(self._h, Q, nq, leaves, nl, k, d2, ids)
        return d2, ids


def philox4x32_10(ctr, key):
    """Philox4x32-10 of a 4-word counter under a 2-word key (uint32 words)."""
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(c, k, out)
    return out


def training_queries(tree: Tree, filter_leaf, n_global, n_local, noise_lo, noise_hi, seed):
    """Alg. 1 GenerateGlobalQueries / GenerateLocalQueries -> (Qg [ng, m], Ql [F, nl, m], gpick [ng], lpick [F, nl])."""
    fl = np.ascontiguousarray(filter_leaf, np.int32)
    F = fl.shape[0]
    Qg = np.zeros((n_global, tree.m), np.float32)
    Ql = np.zeros((F, n_local, tree.m), np.float32)
    gp = np.zeros(max(n_global, 1), np.int64)
    lp = np.zeros((max(F * n_local, 1),), np.int64)
    lib().or_training_queries(tree._h, fl, F, n_global, n_local, float(noise_lo),
                              float(noise_hi), int(seed), Qg, Ql, gp, lp)
    return Qg, Ql, gp[:n_global], lp[:F * n_local].reshape(F, n_local)


def filter_init(F, h, m, seed):
    """Initial weights (W1 [F,h,m], b1 [F,h], w2 [F,h], b2 [F])."""
    W1 = np.zeros((F, h, m), np.float32)
    b1 = np.zeros((F, h), np.float32)
    w2 = np.zeros((F, h), np.float32)
    b2 = np.zeros(F, np.float32)
    lib().or_filter_init(F, h, m, int(seed), W1, b1, w2, b2)
    return W1, b1, w2, b2


def epoch_perms(epochs, n, seed):
    out = np.zeros((epochs, n), np.int32)
    lib().or_epoch_perms(epochs, n, int(seed), out)
    return out


def mlp_forward(W1, b1, w2, b2, Q):
    W1, b1, w2, b2, Q = map(_f32, (W1, b1, w2, b2, Q))
    F, h, m = W1.shape
    out = np.empty((Q.shape[0], F), np.float64)
    lib().or_mlp_forward(W1, b1, w2, b2, F, h, m, Q, Q.shape[0], out)
    return out


def train_targets(tree: Tree, filter_leaf, Qg, Ql):
    """Qg [ng, m]; Ql [F, nl, m] -> (Tg [ng, F], Tl [F, nl]) Euclidean float32."""
    fl = np.ascontiguousarray(filter_leaf, np.int32)
    F = fl.shape[0]
    Qg = _f32(Qg)
    Ql = _f32(Ql).reshape(F, -1, tree.m)
    nl = Ql.shape[1]
    Tg = np.empty((Qg.shape[0], F), np.float32)
    Tl = np.empty((F, nl), np.float32)
    lib().or_train_targets(tree._h, fl, F, Qg, Qg.shape[0], Ql, nl, Tg, Tl)
    return Tg, Tl


class TrainParams:
    def __init__(self, n_gtrain=1200, n_gval=300, n_ltrain=400, n_lval=100, batch=64,
                 max_epochs=1000, patience=10, lr0=0.01, lr_min=1e-5):
        self.__dict__.update(locals())
        del self.__dict__["self"]

    def c(self):
        return _TrainParams(self.n_gtrain, self.n_gval, self.n_ltrain, self.n_lval, self.batch,
                            self.max_epochs, self.patience, self.lr0, self.lr_min)


def train(p: TrainParams, Qg, Tg, Ql, Tl, perms, W1, b1, w2, b2):
    """Returns trained (W1, b1, w2, b2), epochs run and best validation loss per filter."""
    W1, b1, w2, b2 = (np.array(a, dtype=np.float32, copy=True) for a in (W1, b1, w2, b2))
    F, h, m = W1.shape
    ep = np.zeros(F, np.int32)
    bv = np.zeros(F, np.float64)
    cp = p.c()
    lib().or_train(C.byref(cp), F, h, m, _f32(Qg), _f32(Tg), _f32(Ql), _f32(Tl),
                   np.ascontiguousarray(perms, np.int32), W1, b1, w2, b2, ep, bv)
    return (W1, b1, w2, b2), ep, bv


def fit_autotuner(tree: Tree, weights, filter_leaf, Qc, k, wave):
    W1, b1, w2, b2 = map(_f32, weights)
    F, h, m = W1.shape
    Qc = _f32(Qc)
    nc = Qc.shape[0]
    alpha = np.empty((F, nc), np.float64)
    qp = np.empty(nc, np.float64)
    lib().or_fit_autotuner(tree._h, W1, b1, w2, b2, np.ascontiguousarray(filter_leaf, np.int32),
                           F, h, Qc, nc, k, wave, alpha, qp)
    return alpha, qp


def select_leaves_alg3(sizes, th, w, cap):
    """Alg. 3: ids of the selected leaves (largest first)."""
    sz = np.ascontiguousarray(sizes, np.int64)
    out = np.zeros(max(1, sz.shape[0]), np.int32)
    n = lib().or_select_leaves_alg3(sz.ctypes.data_as(C.POINTER(C.c_int64)), sz.shape[0],
                                    float(th), float(w), float(cap),
                                    out.ctypes.data_as(C.POINTER(C.c_int32)))
    return out[:n]


CONFIDENCE = 0.95   # the library's default calibration confidence


def required_quality(n_trials, target, confidence=CONFIDENCE):
    """Calibration quality that certifies `target` with probability `confidence`
    from n_trials = k * nc calibration neighbours."""
    return float(lib().or_required_quality(int(n_trials), float(target), float(confidence)))


def offset_position(qprime, target, kk=1, confidence=CONFIDENCE):
    """STEP position for `target` on a k-class table qprime [nc] (kk = min(k, n))."""
    qp = np.ascontiguousarray(qprime, np.float64)
    return int(lib().or_offset_position(qp, qp.shape[0], int(kk), float(target),
                                        float(confidence)))


def steffen_eval(x, y, xs):
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    return float(lib().or_steffen_eval(x, y, x.shape[0], float(xs)))


def leafi_search(tree: Tree, weights, filter_leaf, alpha_sorted, Q, k, jpos, wave, kmax=None):
    """Wave-semantics LeaFi search.  k, jpos: int arrays per query (jpos -1 = exact).

    Returns ids [nq, kmax], d2 [nq, kmax], stats [nq, 4], min_margin [nq]."""
    Q = _f32(Q)
    nq = Q.shape[0]
    k = np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.int32), (nq,)))
    jpos = np.ascontiguousarray(np.broadcast_to(np.asarray(jpos, np.int32), (nq,)))
    kmax = int(k.max()) if kmax is None else kmax
    if weights is None:
        W1 = np.zeros((1, 1, tree.m), np.float32)
        b1 = np.zeros((1, 1), np.float32)
        w2 = np.zeros((1, 1), np.float32)
        b2 = np.zeros(1, np.float32)
        F = 0
        fl = np.zeros(1, np.int32)
        alpha = np.zeros((1, 1), np.float64)
    else:
        W1, b1, w2, b2 = map(_f32, weights)
        F = W1.shape[0]
        fl = np.ascontiguousarray(filter_leaf, np.int32)
        alpha = np.ascontiguousarray(alpha_sorted, np.float64)
    h = W1.shape[1]
    nc = alpha.shape[1]
    ids = np.empty((nq, kmax), np.int64)
    d2 = np.empty((nq, kmax), np.float32)
    st = np.empty((nq, 4), np.int64)
    mm = np.empty(nq, np.float64)
    lib().or_leafi_search(tree._h, W1, b1, w2, b2, fl, F, h, alpha, nc, Q, nq, k, jpos, kmax,
                          wave, ids, d2, st, mm)
    return ids, d2, st, mm


def recall_at_k(ids, true_ids, k):
    """recall@k per query: |result top-k  ∩  true top-k| / k."""
    ids = np.asarray(ids)[:, :k]
    true_ids = np.asarray(true_ids)[:, :k]
    return np.array([len(set(a.tolist()) & set(b.tolist())) / float(k)
                     for a, b in zip(ids, true_ids)])


# ---------------------------------------------------------------- CNN filters

def cnn_params(C_):
    """Parameters of one CNN filter of C channels: 3C^2 + 6C + 1."""
    return int(lib().or_cnn_params(int(C_)))


def cnn_forward(theta, C_, Q):
    """theta [F, P] flat CNN parameters -> predictions [nq, F] (float64)."""
    theta = _f32(theta)
    Q = _f32(Q)
    F = theta.shape[0]
    assert theta.shape[1] == cnn_params(C_)
    out = np.empty((Q.shape[0], F), np.float64)
    lib().or_cnn_forward(theta, F, int(C_), Q.shape[1], Q, Q.shape[0], out)
    return out


def cnn_init(F, C_, seed):
    theta = np.zeros((F, cnn_params(C_)), np.float32)
    lib().or_cnn_init(F, int(C_), int(seed), theta)
    return theta


def cnn_train(p: TrainParams, C_, Qg, Tg, Ql, Tl, perms, theta):
    """Returns the trained theta [F, P], epochs run and best validation loss per filter."""
    theta = np.array(theta, dtype=np.float32, copy=True)
    F = theta.shape[0]
    Qg = _f32(Qg)
    m = Qg.shape[1]
    ep = np.zeros(F, np.int32)
    bv = np.zeros(F, np.float64)
    cp = p.c()
    lib().or_cnn_train(C.byref(cp), F, int(C_), m, Qg, _f32(Tg), _f32(Ql), _f32(Tl),
                       np.ascontiguousarray(perms, np.int32), theta, ep, bv)
    return theta, ep, bv


def fit_autotuner_pred(tree: Tree, Pc, filter_leaf, Qc, k, wave):
    """Alg. 4 on the calibration queries' predictions Pc [nc, F]."""
    Pc = np.ascontiguousarray(Pc, np.float64)
    Qc = _f32(Qc)
    nc, F = Pc.shape
    alpha = np.empty((F, nc), np.float64)
    qp = np.empty(nc, np.float64)
    lib().or_fit_autotuner_pred(tree._h, Pc, np.ascontiguousarray(filter_leaf, np.int32), F, Qc,
                                nc, k, wave, alpha, qp)
    return alpha, qp


def leafi_search_pred(tree: Tree, P, filter_leaf, alpha_sorted, Q, k, jpos, wave, kmax=None,
                      return_scanned=False):
    """leafi_search on given predictions P [nq, F] (any filter model).

    With return_scanned, a fifth result: uint8 [nq, n_leaves], 1 where Alg. 2
    searched the leaf for the query."""
    Q = _f32(Q)
    nq = Q.shape[0]
    P = np.ascontiguousarray(P, np.float64)
    k = np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.int32), (nq,)))
    jpos = np.ascontiguousarray(np.broadcast_to(np.asarray(jpos, np.int32), (nq,)))
    kmax = int(k.max()) if kmax is None else kmax
    alpha = np.ascontiguousarray(alpha_sorted, np.float64)
    F = P.shape[1]
    ids = np.empty((nq, kmax), np.int64)
    d2 = np.empty((nq, kmax), np.float32)
    st = np.empty((nq, 4), np.int64)
    mm = np.empty(nq, np.float64)
    sc = np.zeros((nq, tree.L), np.uint8) if return_scanned else None
    lib().or_leafi_search_pred(tree._h, P, np.ascontiguousarray(filter_leaf, np.int32), F, alpha,
                               alpha.shape[1], Q, nq, k, jpos, kmax, wave, ids, d2, st, mm,
                               sc.ctypes.data if return_scanned else None)
    if return_scanned:
        return ids, d2, st, mm, sc
    return ids, d2, st, mm
