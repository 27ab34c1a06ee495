"""Alg. 1 (LeaFi-enhanced index building) through the C ABI.

One call, leafi_train_filters, runs the whole of Alg. 1 in libleafi.so: leaf
selection, the training queries and their targets, SGD of every filter and the
auto-tuners.  This module only packages its outputs.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import (TrainParams, leafi_get_filter_leaves, leafi_train_filters,
               leafi_training_queries)


@dataclass
class Enhanced:
    index: object
    filter_leaf: np.ndarray
    params: TrainParams
    kclasses: tuple
    epochs_run: np.ndarray
    best_val: np.ndarray
    report: dict
    Qg: np.ndarray | None = None   # the generated training queries, when asked for
    Ql: np.ndarray | None = None


def enhance(index, n_filters: int, params: TrainParams | None = None, kclasses=(1,),
            keep_queries: bool = False, **overrides) -> Enhanced:
    """SelectLeafNodes -> Generate{Global,Local}Queries -> TrainFilters -> FitAutoTuners."""
    kw = dict(n_filters=n_filters, kclasses=tuple(kclasses))
    if params is not None:
        kw.update({f: getattr(params, f) for f, _ in TrainParams._fields_
                   if f not in ("n_filters", "n_kclasses", "kclasses")})
    kw.update(overrides)
    p = TrainParams(**kw)
    ep, bv, rep = leafi_train_filters(index, p)
    fl = leafi_get_filter_leaves(index)
    Qg = Ql = None
    if keep_queries:
        Qg, Ql, _, _ = leafi_training_queries(index, p, fl)
    return Enhanced(index, fl, p, tuple(kclasses), ep, bv, rep, Qg, Ql)
