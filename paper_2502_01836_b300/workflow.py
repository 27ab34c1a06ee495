"""Alg. 1 (LeaFi-enhanced index building) as a sequence of C-ABI calls.

The random draws (training-query picks and noise, initial weights, SGD
shuffles) come from the seeded generators in `fixtures`; every computation
runs in libleafi.so.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import fixtures as fx

from . import (BuildParams, TrainParams, leafi_build, leafi_fit_autotuners, leafi_leaf_of,
               leafi_select_leaves, leafi_set_filters, leafi_train_filters)


@dataclass
class Enhanced:
    index: object
    filter_leaf: np.ndarray
    init_weights: tuple
    Qg: np.ndarray
    Ql: np.ndarray
    perms: np.ndarray
    params: TrainParams
    kclasses: tuple
    epochs_run: np.ndarray
    best_val: np.ndarray


def enhance(index, X: np.ndarray, n_filters: int, params: TrainParams | None = None,
            kclasses=(1,), seed: int = fx.SEED_TRAIN, weight_seed: int = fx.SEED_WEIGHTS,
            hidden: int | None = None) -> Enhanced:
    """SelectLeafNode -> Generate{Global,Local}Queries -> TrainFilters -> FitAutoTuners."""
    params = params or TrainParams()
    m = X.shape[1]
    h = hidden or m  # hidden width = series length (Sec. 5.1)
    fl = leafi_select_leaves(index, n_filters)
    W = fx.filter_init(n_filters, m, h, seed=weight_seed)
    leafi_set_filters(index, fl, *W)
    members = fx.leaf_members_from(leafi_leaf_of(index), fl)
    Qg, Ql = fx.training_queries(X, members, params.n_gtrain + params.n_gval,
                                 params.n_ltrain + params.n_lval, seed=seed)
    perms = fx.epoch_permutations(params.max_epochs, params.n_gtrain + params.n_ltrain,
                                  seed=weight_seed)
    ep = np.zeros(n_filters, np.int32)
    bv = np.zeros(n_filters, np.float64)
    leafi_train_filters(index, params, Qg, Ql, perms, ep, bv)
    # the calibration set is the validation part of the global training queries (Sec. 4.4)
    leafi_fit_autotuners(index, np.ascontiguousarray(Qg[params.n_gtrain:]), kclasses)
    return Enhanced(index, fl, W, Qg, Ql, perms, params, tuple(kclasses), ep, bv)
