"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws data and initial factors only.  It holds none of the
sampler's arithmetic, so both the CUDA library's tests and the FP64 oracle can
take their inputs from it.  Everything draws from an explicitly seeded
generator: numpy (the default; the same call returns the same arrays on every
machine) or, for the full-size sparse workloads, torch on a CUDA device (same
recipe, a different random stream; repeatable on one device type).

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


def dense_poisson_device(I: int, J: int, K_true: int, seed: int, device):
    """dense_poisson drawn with torch on a CUDA device (for sizes whose host
    arrays would be too slow to draw): W*, H* ~ Gamma(1, 1) (= Exponential(1)),
    V ~ Poisson(W* H*).  Returns V (float32 I x J tensor on `device`)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    Wt = torch.empty((I, K_true), dtype=torch.float32, device=device).exponential_(1.0, generator=g)
    Ht = torch.empty((K_true, J), dtype=torch.float32, device=device).exponential_(1.0, generator=g)
    M = Wt @ Ht
    del Wt, Ht
    V = torch.poisson(M, generator=g)
    del M
    return V


def dense_gamma_device(I: int, J: int, K_true: int, seed: int, device):
    """dense_gamma drawn with torch on a CUDA device: V = |W* H*| * Gamma(2,
    rate 2) with W*, H* ~ |N(0, 1)|.  Returns V (float32 I x J tensor)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    Wt = torch.randn((I, K_true), generator=g, device=device).abs_()
    Ht = torch.randn((K_true, J), generator=g, device=device).abs_()
    M = Wt @ Ht
    del Wt, Ht
    shape = torch.full_like(M, 2.0)
    noise = torch._standard_gamma(shape, generator=g) / 2.0
    return (M * noise).contiguous()


def compound_poisson_gamma_params(mu, p: float, phi: float):
    """(lam, alpha, scale) of the compound Poisson-gamma law with mean mu,
    dispersion phi and power p in (1, 2) -- the observation model of the
    paper's Sec. 4 for 0 < beta < 1 (p = 2 - beta): v is the sum of N ~
    Poisson(lam) independent Gamma(alpha, scale) draws, with lam =
    mu^(2-p) / (phi (2-p)), alpha = (2-p)/(p-1), scale = phi (p-1) mu^(p-1),
    so that E v = mu, Var v = phi mu^p and P(v = 0) = exp(-lam)."""
    lam = mu ** (2.0 - p) / (phi * (2.0 - p))
    alpha = (2.0 - p) / (p - 1.0)
    scale = phi * (p - 1.0) * mu ** (p - 1.0)
    return lam, alpha, scale


def compound_poisson_gamma(mu, p: float, phi: float, g: np.random.Generator):
    """Draws of the compound Poisson-gamma law (one per element of mu): N ~
    Poisson(lam), and given N > 0 the sum of N Gamma(alpha, scale) draws,
    which is one Gamma(N alpha, scale) draw; 0 when N = 0."""
    mu = np.asarray(mu, dtype=np.float64)
    lam, alpha, scale = compound_poisson_gamma_params(mu, p, phi)
    n = g.poisson(lam)
    pos = n > 0
    v = g.gamma(np.where(pos, n * alpha, 1.0), scale)
    return np.where(pos, v, 0.0)


def dense_compound_poisson(I: int, J: int, K_true: int, seed: int, p: float = 1.5,
                           phi: float = 1.0):
    """Dense non-negative data with exact zeros: W*, H* ~ Gamma(1, 1) and
    v_ij ~ compound Poisson-gamma(mean (W* H*)_ij, phi, p), p in (1, 2).
    Returns (V float32 I x J, W*, H*)."""
    g = _rng(seed)
    Wt = g.gamma(1.0, 1.0, size=(I, K_true))
    Ht = g.gamma(1.0, 1.0, size=(K_true, J))
    V = compound_poisson_gamma(Wt @ Ht, p, phi, g).astype(np.float32)
    return V, Wt, Ht


def dense_compound_poisson_device(I: int, J: int, K_true: int, seed: int, device,
                                  p: float = 1.5, phi: float = 1.0, return_mean: bool = False):
    """dense_compound_poisson drawn with torch on a CUDA device (the same
    law; a different stream of random numbers).  Returns V (float32 I x J),
    or (V, the means W* H*) with return_mean."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    Wt = torch.empty((I, K_true), dtype=torch.float32, device=device).exponential_(1.0, generator=g)
    Ht = torch.empty((K_true, J), dtype=torch.float32, device=device).exponential_(1.0, generator=g)
    M = Wt @ Ht
    del Wt, Ht
    lam, alpha, scale = compound_poisson_gamma_params(M, p, phi)
    n = torch.poisson(lam, generator=g)
    del lam
    pos = n > 0
    conc = torch.where(pos, n * alpha, torch.ones_like(n))
    V = torch._standard_gamma(conc, generator=g) * scale
    V = torch.where(pos, V, torch.zeros_like(V)).contiguous()
    return (V, M) if return_mean else V


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
    dropped, in rounds, until at least nnz distinct pairs exist; a seeded
    random subset of nnz of them is kept, in row-major order.  Rows or columns
    whose expected degree exceeds the other dimension saturate, as in real
    rating matrices.
    """
    if nnz > I * J:
        raise ValueError("nnz larger than I*J")
    cr = np.cumsum(_zipf_weights(I, zipf_row, g))
    cc = np.cumsum(_zipf_weights(J, zipf_col, g)) if zipf_col else None
    keys = np.empty(0, dtype=np.int64)
    draw = int(nnz * 1.2) + 1024
    while len(keys) < nnz:
        ii = np.minimum(np.searchsorted(cr, g.random(draw) * cr[-1], side="right"), I - 1)
        if cc is not None:
            jj = np.minimum(np.searchsorted(cc, g.random(draw) * cc[-1], side="right"), J - 1)
        else:
            jj = g.integers(0, J, size=draw)
        before = len(keys)
        keys = np.unique(np.concatenate([keys, ii.astype(np.int64) * J + jj]))
        gained = len(keys) - before
        need = nnz - len(keys)
        if need > 0:   # next round sized from this round's yield of new pairs
            draw = int(need * draw / max(gained, 1) * 1.2) + 1024
    if len(keys) > nnz:
        keys = np.sort(g.choice(keys, size=nnz, replace=False))
    return (keys // J).astype(np.int32), (keys % J).astype(np.int32)


def _sparse_ratings_torch(I, J, nnz, K_true, seed, zipf_row, zipf_col, noise_sd, device):
    """The recipe of sparse_pattern + sparse_ratings with torch tensors on `device`."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = torch.float64

    def cdf(n, a):
        w = torch.arange(1, n + 1, dtype=f64, device=device) ** (-a)
        out = torch.empty_like(w)
        out[torch.randperm(n, generator=g, device=device)] = w / w.sum()
        return torch.cumsum(out, 0)

    cr = cdf(I, zipf_row)
    cc = cdf(J, zipf_col) if zipf_col else None
    keys = torch.empty(0, dtype=torch.int64, device=device)
    draw = int(nnz * 1.2) + 1024
    while keys.numel() < nnz:
        u = torch.rand(draw, generator=g, device=device, dtype=f64) * cr[-1]
        ii = torch.searchsorted(cr, u, right=True).clamp_(max=I - 1)
        if cc is not None:
            u = torch.rand(draw, generator=g, device=device, dtype=f64) * cc[-1]
            jj = torch.searchsorted(cc, u, right=True).clamp_(max=J - 1)
        else:
            jj = torch.randint(0, J, (draw,), generator=g, device=device)
        before = keys.numel()
        keys = torch.unique(torch.cat([keys, ii * J + jj]))
        gained = keys.numel() - before
        need = nnz - keys.numel()
        if need > 0:
            draw = int(need * draw / max(gained, 1) * 1.2) + 1024
    if keys.numel() > nnz:
        sel = torch.randperm(keys.numel(), generator=g, device=device)[:nnz]
        keys = torch.sort(keys[sel]).values
    i = (keys // J).to(torch.int32)
    j = (keys % J).to(torch.int32)
    s = math.sqrt(3.0 * math.pi / (2.0 * K_true))
    Wt = torch.randn(I, K_true, generator=g, device=device, dtype=f64).abs_() * s
    Ht = torch.randn(J, K_true, generator=g, device=device, dtype=f64).abs_() * s
    v = torch.empty(nnz, dtype=torch.float32, device=device)
    chunk = 1 << 22
    for a in range(0, nnz, chunk):
        b = min(nnz, a + chunk)
        mean = (Wt[i[a:b].long()] * Ht[j[a:b].long()]).sum(1)
        noise = torch.randn(b - a, generator=g, device=device, dtype=f64) * noise_sd
        v[a:b] = torch.clamp(torch.round(mean + noise), 1, 5).float()
    return i, j, v


def sparse_ratings(I: int, J: int, nnz: int, K_true: int, seed: int,
                   zipf_row: float = 1.1, zipf_col: float | None = 1.1,
                   noise_sd: float = 0.5, device=None):
    """Ratings-like sparse data. Returns (i int32, j int32, v float32).

    With `device` (a CUDA device) the arrays are torch tensors drawn there;
    otherwise numpy arrays drawn on the host.
    """
    if device is not None:
        return _sparse_ratings_torch(I, J, nnz, K_true, seed, zipf_row, zipf_col, noise_sd,
                                     device)
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
