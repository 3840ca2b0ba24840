"""The sparse path with BF16-gathered factors (gather_bf16 = 1) against the
FP64 oracle.

The gradient kernel gathers the other factor's rows from BF16 copies (kept
by the update kernel) while the own row, the products and every sum stay
FP32, so one part-step cannot match the oracle to FP32 precision.  What is
checked:

* one part-step: the drift S * grad log p(V | .) + grad log p(.) the GPU
  applied (recovered with the oracle's own Philox normals) is within a
  first-order bound of the BF16 rounding around the oracle's FP64 drift,
  element by element.  For an entry (i, j) of the part, the W side computes
  mu from x = w_i (FP32) and y = bf16(h_j): |dmu| <= u sum_k |w_ik h_kj|
  (u = 2^-8) plus the FP32 dot; e moves by |de/dmu| times that; G_W[i] =
  sum_j e_ij bf16(h_j) adds u |e_ij| |h_j|.  The H side is the mirror image
  with bf16(w_i).  A wrong row, a dropped term or a wrong power gives errors
  of the drift's own size, far outside the bound;
* full chains: posterior-mean reconstruction RMSE within 1 % of the FP64
  oracle chain (the shrunk sparse ratings workload of the chain tests);
* graph replay == direct launches bit for bit; enabling the option after
  the factors are set is refused until they are set again.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import U_BF16, U_FP32, Pair, recovered_drift, sparse_case
from paper_1506_01418_gb300 import datagen
from paper_1506_01418_gb300 import psgld as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

CASES = {
    # name: (I, J, K, B, p, phi, prior_kind, nnz, eps)
    "gauss_K50": (300, 200, 50, 3, 0.0, 1.0, 1, 20000, 1e-3),
    "gamma_K13": (120, 90, 13, 5, 2.0, 0.7, 0, 3000, 1e-3),
    "poisson_K100": (400, 300, 100, 4, 1.0, 1.0, 0, 30000, 1e-4),
    "poisson_K4_zipf": (500, 150, 4, 2, 1.0, 1.0, 0, 8000, 1e-3),
}


def _make(name, seed=7, **opts):
    I, J, K, B, p, phi, kind, nnz, eps = CASES[name]
    i, j, v = sparse_case(I, J, nnz, 5, seed=I + J)
    if p >= 1:
        v = v.astype(np.float32) + np.float32(0.25)   # positive data for mu^-p
    nonneg = kind == 0
    W0, H0 = datagen.init_factors(I, J, K, seed=3, scale=0.4 if nonneg else 0.3, nonneg=nonneg)
    pr = Pair(I, J, K, B, p, phi, i, j, v, W0, H0, prior_kind=kind, lam=(0.8, 1.2),
              sig=(0.9, 1.1), seed=seed, eps=eps, gather_bf16=1, **opts)
    return pr, (i, j, v)


def _pieces(n, B):
    return np.array([oracle.piece_start(r, n, B) for r in range(B + 1)])


def _sparse_bound(i, j, v, W, H, t, B, p, phi, S, mu_min=1e-10):
    """First-order bound on |drift_gpu - drift| of part t with BF16 gathers
    (see the module docstring); W I x K, H K x J in FP64."""
    I, K = W.shape
    J = H.shape[1]
    s = (t - 1) % B
    rp = np.searchsorted(_pieces(I, B), i, side="right") - 1
    cp = np.searchsorted(_pieces(J, B), j, side="right") - 1
    m = cp == (rp + s) % B
    ie, je, ve = i[m], j[m], v[m].astype(np.float64)
    w, h = W[ie], H[:, je].T
    A = (np.abs(w) * np.abs(h)).sum(1)
    mu = (w * h).sum(1)
    dmu = U_BF16 * A * 1.01 + 4 * K * U_FP32 * A
    if p > 0:
        mc = np.maximum(mu, mu_min)
        lo = np.maximum(mu - dmu, mu_min)
        e = (ve - mu) * mc ** -p / phi
        fprime = lo ** -p * (1 + p * (np.abs(ve - mu) + dmu) / lo) / phi
    else:
        e = (ve - mu) / phi
        fprime = np.full_like(mu, 1.0 / phi)
    de = fprime * dmu + 64 * U_FP32 * np.abs(e)
    coef = de + U_BF16 * np.abs(e)
    bW = np.zeros_like(W)
    bHt = np.zeros((J, K))
    np.add.at(bW, ie, coef[:, None] * np.abs(h))
    np.add.at(bHt, je, coef[:, None] * np.abs(w))
    # FP32 sums over a row's entries
    nI = np.bincount(ie, minlength=I).astype(np.float64)
    nJ = np.bincount(je, minlength=J).astype(np.float64)
    aW = np.zeros_like(W)
    aHt = np.zeros((J, K))
    np.add.at(aW, ie, np.abs(e)[:, None] * np.abs(h))
    np.add.at(aHt, je, np.abs(e)[:, None] * np.abs(w))
    bW += (nI * U_FP32)[:, None] * aW * (1 + U_BF16)
    bHt += (nJ * U_FP32)[:, None] * aHt * (1 + U_BF16)
    return S * bW, S * bHt.T


@pytest.mark.parametrize("name", sorted(CASES))
def test_bf16_gather_part_step_drift_within_bound(name):
    pr, (i, j, v) = _make(name)
    I, J, K, B, p, phi, kind, nnz, eps = CASES[name]
    mirror = kind == 0
    for t in range(1, B + 2):
        W0, H0 = pr.orc.get_factors()
        D_W, D_H = pr.orc.drift(t)
        S = pr.orc.scale(t)
        bW, bH = _sparse_bound(i, j, v, W0, H0, t, B, p, phi, S)
        pr.gpu.part_step(t)
        Wg, Hg = pr.gpu_factors()
        zW = oracle.noise_matrix(7, t, 0, I, K)
        zH = oracle.noise_matrix(7, t, 1, J, K).T
        for xg, x0, z, D, bnd, what in ((Wg, W0, zW, D_W, bW, "W"), (Hg, H0, zH, D_H, bH, "H")):
            Dg, mask, rec = recovered_drift(xg.astype(np.float64), x0, z, D, eps, mirror)
            err = np.abs(Dg - D)
            lim = bnd + rec
            bad = mask & (err > lim)
            assert not bad.any(), (name, t, what, int(bad.sum()), float(err[bad].max()),
                                   float(lim[bad].min()))
            assert mask.mean() > 0.8
            # rows with entries in the part: the drift there is far larger
            # than the bound, so the check has teeth
            active = mask & (bnd > 0)
            assert active.sum() > 0
            assert np.sqrt(np.mean(D[active] ** 2)) > 4 * np.sqrt(np.mean(bnd[active] ** 2)), (name, what)
        if mirror:
            assert Wg.min() >= 0 and Hg.min() >= 0
        pr.sync_oracle_to_gpu()
    pr.gpu.close()


def test_bf16_gather_graph_replay_equals_direct_launches():
    a, _ = _make("gauss_K50", use_graphs=1, burn_in_sweeps=1)
    b, _ = _make("gauss_K50", use_graphs=0, burn_in_sweeps=1)
    for n in (1, 2):
        a.gpu.sweep(n)
        b.gpu.sweep(n)
    Wa, Ha = a.gpu_factors()
    Wb, Hb = b.gpu_factors()
    assert np.array_equal(Wa, Wb) and np.array_equal(Ha, Hb)
    ma, mb = a.gpu.posterior_mean(), b.gpu.posterior_mean()
    for x, y in zip(ma[:4], mb[:4]):
        assert np.array_equal(x, y)


def test_bf16_gather_chain_rmse_within_one_percent_of_oracle():
    """The shrunk sparse ratings workload: 7000 x 1000, 100k entries with
    Zipf(1.1) degrees, K = 50, B = 32, Gaussian priors sigma = 1, eps = 2e-5,
    100 sweeps, posterior means over the last 50; the FP32 gather chain from
    the same inputs beside it."""
    I, J, nnz, K, B, sweeps = 7000, 1000, 100_000, 50, 32, 100
    i, j, v = datagen.sparse_ratings(I, J, nnz, 20, seed=5, zipf_row=1.1, zipf_col=1.1)
    W0, H0 = datagen.init_factors(I, J, K, seed=5, scale=0.3, nonneg=False)
    pr = Pair(I, J, K, B, 0.0, 1.0, i, j, v, W0, H0, prior_kind=1, sig=(1.0, 1.0), seed=13,
              eps=2e-5, burn_in_sweeps=sweeps // 2, gather_bf16=1)
    f32 = P.PSGLD(I, J, K, B, 0.0, 1.0, prior_kind=1, seed=13, eps=2e-5,
                  burn_in_sweeps=sweeps // 2)
    f32.set_data_coo(torch.as_tensor(i, device="cuda"), torch.as_tensor(j, device="cuda"),
                     torch.as_tensor(v, device="cuda"))
    f32.set_factors(torch.from_numpy(W0).cuda(), torch.from_numpy(H0.T.copy()).cuda())
    pr.gpu.sweep(sweeps)
    f32.sweep(sweeps)
    pr.orc.sweep(sweeps)
    r16, r32, r_or = pr.gpu.rmse(True), f32.rmse(True), pr.orc.rmse(True)
    assert abs(r16 - r_or) <= 0.01 * r_or, (r16, r32, r_or)
    assert abs(r32 - r_or) <= 0.01 * r_or, (r16, r32, r_or)
    f32.close()


def test_bf16_gather_enabled_after_factors_is_refused():
    I, J, K, B = 60, 50, 8, 2
    i, j, v = sparse_case(I, J, 600, 3, seed=1)
    W0, H0 = datagen.init_factors(I, J, K, seed=1, scale=0.3, nonneg=False)
    ch = P.PSGLD(I, J, K, B, 0.0, 1.0, prior_kind=1)
    ch.set_data_coo(torch.as_tensor(i, device="cuda"), torch.as_tensor(j, device="cuda"),
                    torch.as_tensor(v, device="cuda"))
    ch.set_factors(torch.from_numpy(W0).cuda(), torch.from_numpy(H0.T.copy()).cuda())
    ch.set_options(gather_bf16=1)
    with pytest.raises(P.PsgldError) as ex:
        ch.sweep(1)
    assert ex.value.status == P.PSGLD_ERR_STATE
    ch.set_factors(torch.from_numpy(W0).cuda(), torch.from_numpy(H0.T.copy()).cuda())
    ch.sweep(1)
    ch.close()
