"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/leafi.h declares, rejects bad arguments, and its host-side tree build
agrees with the oracle's independent one."""
import ctypes
import os
import re

import numpy as np
import pytest

import fixtures as fx
import oracle as O
import paper_2502_01836_b300 as lf
from paper_2502_01836_b300 import build as lfbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    lfbuild.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "leafi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(leafi_[a-z_]+)\s*\(", src)))


def test_header_symbols_exported():
    names = _declared()
    assert len(names) >= 20
    so = ctypes.CDLL(lf.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n
    assert sorted(lf.EXPORTED_SYMBOLS) == names


def test_bad_arguments_rejected_without_device():
    X = np.zeros((4, 8), np.float32)
    h = ctypes.c_void_p()
    L = lf.lib()
    p = lf.BuildParams(device=-1)
    assert L.leafi_build(X.ctypes.data, 0, 8, ctypes.byref(p), ctypes.byref(h)) == 1
    assert L.leafi_build(X.ctypes.data, 4, 0, ctypes.byref(p), ctypes.byref(h)) == 1
    assert L.leafi_build(None, 4, 8, ctypes.byref(p), ctypes.byref(h)) == 1
    bad = lf.BuildParams(wave=0, device=-1)
    assert L.leafi_build(X.ctypes.data, 4, 8, ctypes.byref(bad), ctypes.byref(h)) == 1
    bad = lf.BuildParams(wave=65537, device=-1)
    assert L.leafi_build(X.ctypes.data, 4, 8, ctypes.byref(bad), ctypes.byref(h)) == 1
    ok = lf.BuildParams(wave=65536, device=-1)
    assert L.leafi_build(X.ctypes.data, 4, 8, ctypes.byref(ok), ctypes.byref(h)) == 0
    L.leafi_free(h)
    bad = lf.BuildParams(index_type=7, device=-1)
    assert L.leafi_build(X.ctypes.data, 4, 8, ctypes.byref(bad), ctypes.byref(h)) == 1
    bad = lf.BuildParams(index_type=lf.ISAX, isax_segments=3, device=-1)
    assert L.leafi_build(X.ctypes.data, 4, 8, ctypes.byref(bad), ctypes.byref(h)) == 1
    assert b"isax_segments" in L.leafi_last_error()
    assert L.leafi_search(None, None, 0, 1, 1.0, None, None, None) == 1


def test_host_only_index_refuses_device_work():
    X = fx.random_walk(500, 16, seed=3)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=100, device=-1))
    try:
        with pytest.raises(lf.LeafiError) as e:
            lf.leafi_exact_search(idx, X[:2], 1, np.zeros((2, 1), np.int64),
                                  np.zeros((2, 1), np.float32))
        assert e.value.status == 1
    finally:
        lf.leafi_free(idx)


@pytest.mark.parametrize("m,cap,seg", [(64, 300, 4), (96, 500, 4), (30, 200, 3)])
def test_host_dstree_equals_oracle_tree(m, cap, seg):
    X = fx.random_walk(8000, m, seed=40 + m)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=cap, dstree_init_segments=seg,
                                           device=-1))
    try:
        info = lf.leafi_get_info(idx)
        t = O.Tree(X, "dstree", leaf_cap=cap, init_segments=seg)
        assert info.n_leaves == t.L and info.n_nodes == t.n_nodes
        assert np.array_equal(lf.leafi_leaf_of(idx), t.leaf_of())
        assert np.array_equal(lf.leafi_leaf_sizes(idx), t.leaf_sizes())
    finally:
        lf.leafi_free(idx)


def test_host_isax_equals_oracle_tree():
    X = fx.random_walk(8000, 64, seed=77)
    idx = lf.leafi_build(X, lf.BuildParams(index_type=lf.ISAX, leaf_capacity=150,
                                           isax_segments=16, isax_card_bits=8, device=-1))
    try:
        t = O.Tree(X, "isax", leaf_cap=150, isax_w=16, isax_bits=8)
        info = lf.leafi_get_info(idx)
        assert info.n_leaves == t.L
        assert np.array_equal(lf.leafi_leaf_of(idx), t.leaf_of())
    finally:
        lf.leafi_free(idx)


def test_select_leaves_is_largest_first():
    X = fx.random_walk(5000, 32, seed=5)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=200, device=-1))
    try:
        sizes = lf.leafi_leaf_sizes(idx)
        sel = lf.leafi_select_leaves(idx, 10)
        ref = sorted(range(len(sizes)), key=lambda l: (-sizes[l], l))[:10]
        assert sel.tolist() == ref
    finally:
        lf.leafi_free(idx)


def test_epoch_permutations_equal_the_oracle():
    """The SGD shuffles are drawn on the host by the library's Philox4x32-10:
    bit-identical to the oracle's independent implementation."""
    for epochs, n, seed in ((3, 1, 1), (5, 1600, 2502018361), (2, 97, 2 ** 63 + 5)):
        got = lf.leafi_epoch_permutations(epochs, n, seed)
        assert np.array_equal(got, O.epoch_perms(epochs, n, seed))
