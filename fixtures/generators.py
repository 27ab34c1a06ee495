"""Seeded, counter-based workload generators (no search arithmetic lives here).

Every stream is a numpy Philox4x32-10 generator keyed by (seed, stream tag)
whose counter starts at the block number, so the values of a series depend
only on (seed, series id) and never on how the work is chunked.

Workloads follow the paper's experimental setup (Sec. 5.1):
  * RandWalk: cumulative sums of N(0,1) steps;
  * query sets: uniformly sampled dataset series plus Gaussian noise, the
    literature's standard generator, with noise levels 10%-40%;
  * the "embedding-like" stand-in for the Deep descriptors (length 96):
    a Gaussian mixture of clusters, z-normalised.
All series handed to the index are z-normalised in float64 (population sigma;
sigma < 1e-8 gives the all-zero series) and then stored as float32.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

__all__ = [
    "SEED_DATA", "SEED_TRAIN", "SEED_TEST", "SEED_WEIGHTS",
    "znorm_rows", "random_walk", "embedding_like", "pick_without_replacement",
    "noisy_queries", "test_queries", "filter_init", "epoch_permutations",
    "uniform_sigmas", "training_queries", "leaf_members_from",
]

SEED_DATA = 2502018360
SEED_TRAIN = SEED_DATA + 1
SEED_TEST = SEED_DATA + 2
SEED_WEIGHTS = SEED_DATA + 3

_BLOCK = 4096  # series per counter block

_TAG_WALK = 1
_TAG_EMB_CENTRES = 2
_TAG_EMB_POINTS = 3
_TAG_PICK = 4
_TAG_NOISE = 5
_TAG_SIGMA = 6
_TAG_W = 7
_TAG_PERM = 8


def _rng(seed: int, tag: int, block: int = 0) -> np.random.Generator:
    key = np.array([seed & 0xFFFFFFFFFFFFFFFF, tag], dtype=np.uint64)
    ctr = np.array([0, block, 0, 0], dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key, counter=ctr))


def znorm_rows(a: np.ndarray, out: np.ndarray | None = None) -> np.ndarray:
    """z-normalise each row in float64 (population sigma), return float32.

    `a` (float64) may be overwritten.  Rows with sigma < 1e-8 become zeros.
    """
    a = np.asarray(a, dtype=np.float64)
    if out is None:
        out = np.empty(a.shape, dtype=np.float32)
    mu = a.mean(axis=1, keepdims=True)
    a -= mu
    sd = np.sqrt(np.einsum("ij,ij->i", a, a) / a.shape[1])[:, None]
    ok = sd >= 1e-8
    np.divide(a, np.where(ok, sd, 1.0), out=a)
    a *= ok
    out[...] = a
    return out


def _random_walk_into(out: np.ndarray, m: int, seed: int, start: int, lo: int, hi_end: int):
    buf = np.empty((_BLOCK, m), dtype=np.float64)
    i = lo
    while i < hi_end:
        b = i // _BLOCK
        b0 = b * _BLOCK
        hi = min(hi_end, b0 + _BLOCK)
        g = _rng(seed, _TAG_WALK, b)
        blk = buf[:hi - b0]
        g.standard_normal(out=blk)
        np.cumsum(blk, axis=1, out=blk)
        znorm_rows(blk[i - b0:], out=out[i - start:hi - start])
        i = hi


def random_walk(n: int, m: int, seed: int = SEED_DATA, start: int = 0) -> np.ndarray:
    """Series start..start+n-1 of the RandWalk collection (n x m float32).

    Every block of 4096 series has its own counter-based stream, so the
    result does not depend on how the blocks are shared among threads."""
    out = np.empty((n, m), dtype=np.float32)
    end = start + n
    workers = min(16, os.cpu_count() or 1) if n >= (1 << 20) else 1
    if workers == 1:
        _random_walk_into(out, m, seed, start, start, end)
        return out
    # block-aligned ranges, one per task
    step = max(_BLOCK, ((n // (4 * workers)) // _BLOCK) * _BLOCK)
    edges = [start] + [b for b in range((start // step + 1) * step, end, step)] + [end]
    with ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(lambda r: _random_walk_into(out, m, seed, start, r[0], r[1]),
                    zip(edges[:-1], edges[1:])))
    return out


def embedding_like(n: int, m: int = 96, clusters: int = 1000, cluster_std: float = 0.3,
                   seed: int = SEED_DATA, start: int = 0) -> np.ndarray:
    """Gaussian-mixture vectors: centre ~ N(0, I), point = centre + N(0, std^2 I), z-normalised."""
    centres = _rng(seed, _TAG_EMB_CENTRES).standard_normal((clusters, m))
    out = np.empty((n, m), dtype=np.float32)
    i = start
    end = start + n
    while i < end:
        b = i // _BLOCK
        b0 = b * _BLOCK
        hi = min(end, b0 + _BLOCK)
        g = _rng(seed, _TAG_EMB_POINTS, b)
        cid = g.integers(0, clusters, size=hi - b0)
        pts = centres[cid] + cluster_std * g.standard_normal((hi - b0, m))
        out[i - start:hi - start] = znorm_rows(pts[i - b0:])
        i = hi
    return out


def pick_without_replacement(n: int, count: int, seed: int, stream: int = 0) -> np.ndarray:
    """`count` distinct indices in [0, n), uniformly at random."""
    g = _rng(seed, _TAG_PICK, stream)
    if count > n:
        raise ValueError("count > n")
    return g.choice(n, size=count, replace=False).astype(np.int64)


def uniform_sigmas(count: int, lo: float, hi: float, seed: int, stream: int = 0) -> np.ndarray:
    g = _rng(seed, _TAG_SIGMA, stream)
    return lo + (hi - lo) * g.random(count)


def noisy_queries(base: np.ndarray, sigmas: np.ndarray, seed: int, stream: int = 0) -> np.ndarray:
    """base + N(0, sigma_i^2) per point (float64), then re-z-normalised to float32."""
    base = np.asarray(base, dtype=np.float64)
    g = _rng(seed, _TAG_NOISE, stream)
    noise = g.standard_normal(base.shape)
    return znorm_rows(base + np.asarray(sigmas, dtype=np.float64)[:, None] * noise)


def test_queries(data: np.ndarray, count: int, seed: int = SEED_TEST,
                 levels=(0.1, 0.2, 0.3, 0.4)) -> np.ndarray:
    """The paper's query sets: uniform random dataset series + 10/20/30/40% noise.

    Noise levels cycle over `levels` so every level gets count/len(levels) queries.
    """
    idx = pick_without_replacement(data.shape[0], count, seed, stream=1)
    sig = np.asarray([levels[i % len(levels)] for i in range(count)], dtype=np.float64)
    return noisy_queries(data[idx], sig, seed, stream=1)


def filter_init(F: int, m: int, h: int, seed: int = SEED_WEIGHTS):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) initial weights for F MLP filters.

    Returns (W1 [F,h,m], b1 [F,h], w2 [F,h], b2 [F]) as float32.
    """
    g = _rng(seed, _TAG_W)
    a1 = 1.0 / np.sqrt(m)
    a2 = 1.0 / np.sqrt(h)
    W1 = g.uniform(-a1, a1, (F, h, m)).astype(np.float32)
    b1 = g.uniform(-a1, a1, (F, h)).astype(np.float32)
    w2 = g.uniform(-a2, a2, (F, h)).astype(np.float32)
    b2 = g.uniform(-a2, a2, (F,)).astype(np.float32)
    return W1, b1, w2, b2


def epoch_permutations(epochs: int, n: int, seed: int = SEED_WEIGHTS) -> np.ndarray:
    """One shuffle of range(n) per SGD epoch (int32 [epochs, n])."""
    g = _rng(seed, _TAG_PERM)
    out = np.empty((epochs, n), dtype=np.int32)
    for e in range(epochs):
        out[e] = g.permutation(n)
    return out


def training_queries(data: np.ndarray, leaf_members, n_global: int, n_local: int,
                     seed: int = SEED_TRAIN, sigma_lo: float = 0.1, sigma_hi: float = 0.4):
    """Training queries of Alg. 1 (GenerateGlobalQueries / GenerateLocalQueries).

    Global: `n_global` distinct dataset series; local: `n_local` series of each
    filtered leaf (members listed in `leaf_members[f]`, drawn without
    replacement when the leaf is large enough, else with replacement).  Every
    query gets Gaussian noise with sigma ~ U[sigma_lo, sigma_hi] and is
    re-z-normalised.  Returns (Qg [n_global, m], Ql [F, n_local, m]).
    """
    n, m = data.shape
    gi = pick_without_replacement(n, n_global, seed, stream=10)
    Qg = noisy_queries(data[gi], uniform_sigmas(n_global, sigma_lo, sigma_hi, seed, 10), seed, 10)
    F = len(leaf_members)
    Ql = np.empty((F, n_local, m), np.float32)
    for f, mem in enumerate(leaf_members):
        mem = np.asarray(mem, np.int64)
        s = 1000 + f
        if mem.shape[0] >= n_local:
            pick = mem[pick_without_replacement(mem.shape[0], n_local, seed, stream=s)]
        else:
            pick = mem[_rng(seed, _TAG_PICK, s).integers(0, mem.shape[0], n_local)]
        Ql[f] = noisy_queries(data[pick], uniform_sigmas(n_local, sigma_lo, sigma_hi, seed, s),
                              seed, s)
    return Qg, Ql


def leaf_members_from(leaf_of: np.ndarray, leaves) -> list:
    """Series ids (ascending) of each listed leaf, from a leaf-of-series array."""
    order = np.argsort(leaf_of, kind="stable")
    sorted_leaf = leaf_of[order]
    out = []
    for l in leaves:
        lo = np.searchsorted(sorted_leaf, l, "left")
        hi = np.searchsorted(sorted_leaf, l, "right")
        out.append(order[lo:hi])
    return out
