"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws data and initial factors only.  It holds none of the
sampler's arithmetic, so both the CUDA library's tests and the FP64 oracle can
take their inputs from it.  Everything is numpy with an explicit seed; the same
call returns the same arrays on every machine.

Workloads (the data sets of the paper are not available; these stand in for
their published shapes):

* ``dense_poisson``  -- Poisson NMF as in the synthetic and audio experiments
  of Sec. 4.1: W*, H* ~ Gamma(1, 1), V ~ Poisson(W* H*); every entry observed.
* ``sparse_ratings`` -- ratings-like sparse V as in the MovieLens experiment
  of Sec. 4.2: unique (i, j) pairs whose row and column degrees follow Zipf
  laws over randomly permuted ids, values clip(round(W* H* + N(0, 0.5^2)), 1, 5)
  with W*, H* iid |N(0, s^2)|, s^2 = 3 pi / (2 K*), so E[W* H*] is about 3.
* ``dense_gamma``    -- spectrogram-like V = |W* H*| * Gamma(2, rate 2).
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def dense_poisson(I: int, J: int, K_true: int, seed: int):
    """Dense Poisson-NMF data. Returns (V float32 I x J, W*, H*)."""
    g = _rng(seed)
    Wt = g.gamma(1.0, 1.0, size=(I, K_true))
    Ht = g.gamma(1.0, 1.0, size=(K_true, J))
    V = g.poisson(Wt @ Ht).astype(np.float32)
    return V, Wt, Ht


def dense_gamma(I: int, J: int, K_true: int, seed: int):
    """Dense positive data V = |W* H*| * Gamma(shape 2, rate 2)."""
    g = _rng(seed)
    Wt = np.abs(g.normal(0.0, 1.0, size=(I, K_true)))
    Ht = np.abs(g.normal(0.0, 1.0, size=(K_true, J)))
    V = (np.abs(Wt @ Ht) * g.gamma(2.0, 0.5, size=(I, J))).astype(np.float32)
    return V, Wt, Ht


def dense_to_coo(V: np.ndarray):
    """All entries of a dense matrix as (i, j, v) in row-major order."""
    I, J = V.shape
    ii, jj = np.meshgrid(np.arange(I, dtype=np.int32), np.arange(J, dtype=np.int32),
                         indexing="ij")
    return ii.ravel(), jj.ravel(), np.ascontiguousarray(V, dtype=np.float32).ravel()


def _zipf_weights(n: int, a: float, g: np.random.Generator) -> np.ndarray:
    """Zipf(a) weights over ranks 1..n, assigned to a random permutation of ids."""
    w = np.arange(1, n + 1, dtype=np.float64) ** (-a)
    w /= w.sum()
    out = np.empty(n)
    out[g.permutation(n)] = w
    return out


def sparse_pattern(I: int, J: int, nnz: int, zipf_row: float, zipf_col: float | None,
                   g: np.random.Generator):
    """nnz unique (i, j) pairs with Zipf row (and optionally column) degrees.

    Pairs are drawn independently from the two marginals and duplicates are
    dropped, until nnz distinct pairs exist; the first nnz distinct pairs in
    draw order are kept.  Rows or columns whose expected degree exceeds the
    other dimension saturate, as real rating matrices do.
    """
    if nnz > I * J:
        raise ValueError("nnz larger than I*J")
    pr = _zipf_weights(I, zipf_row, g)
    pc = _zipf_weights(J, zipf_col, g) if zipf_col else None
    keys = np.empty(0, dtype=np.int64)
    first = np.empty(0, dtype=np.int64)
    drawn = 0
    while True:
        need = nnz - len(keys)
        if need <= 0:
            break
        m = max(int(need * 1.25), 1024)
        ii = g.choice(I, size=m, p=pr)
        jj = g.choice(J, size=m, p=pc) if pc is not None else g.integers(0, J, size=m)
        k = ii.astype(np.int64) * J + jj
        allk = np.concatenate([keys, k])
        allpos = np.concatenate([first, drawn + np.arange(m, dtype=np.int64)])
        u, idx = np.unique(allk, return_index=True)
        keys, first = u, allpos[idx]
        drawn += m
    order = np.argsort(first, kind="stable")[:nnz]
    k = keys[order]
    return (k // J).astype(np.int32), (k % J).astype(np.int32)


def sparse_ratings(I: int, J: int, nnz: int, K_true: int, seed: int,
                   zipf_row: float = 1.1, zipf_col: float | None = 1.1,
                   noise_sd: float = 0.5):
    """Ratings-like sparse data. Returns (i int32, j int32, v float32)."""
    g = _rng(seed)
    i, j = sparse_pattern(I, J, nnz, zipf_row, zipf_col, g)
    s = math.sqrt(3.0 * math.pi / (2.0 * K_true))
    Wt = np.abs(g.normal(0.0, s, size=(I, K_true)))
    Ht = np.abs(g.normal(0.0, s, size=(K_true, J)))
    mean = np.einsum("nk,kn->n", Wt[i], Ht[:, j])
    v = np.clip(np.round(mean + g.normal(0.0, noise_sd, size=nnz)), 1, 5)
    return i, j, v.astype(np.float32)


def init_factors(I: int, J: int, K: int, seed: int, scale: float = 1.0,
                 nonneg: bool = True):
    """Initial W (I x K) and H (K x J), float32.

    Non-negative models start from Uniform(0.5, 1.5) * scale; Gaussian models
    from N(0, scale^2).
    """
    g = _rng(seed + 7919)
    if nonneg:
        W = g.uniform(0.5, 1.5, size=(I, K)) * scale
        H = g.uniform(0.5, 1.5, size=(K, J)) * scale
    else:
        W = g.normal(0.0, scale, size=(I, K))
        H = g.normal(0.0, scale, size=(K, J))
    return W.astype(np.float32), H.astype(np.float32)
