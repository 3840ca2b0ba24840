"""The dense tensor-core path (dense_path = 1) against the FP64 oracle.

The block chain mu = W_b H_b -> E -> (E H_b^T, E^T W_b) runs with BF16
operands and FP32 accumulation, so one part-step cannot match the oracle to
FP32 precision.  What is checked:

* one part-step: the drift S * grad log p(V | .) + grad log p(.) that the GPU
  applied (recovered from its output with the oracle's own Philox normals) is
  within a first-order error bound of BF16 rounding around the oracle's FP64
  drift, element by element.  The bound follows the arithmetic: every operand
  of GEMM1 is rounded to BF16 (relative error <= u = 2^-8), which moves mu by
  at most 2u sum_k |w_ik h_kj|; that moves e by at most |de/dmu| times as much;
  e itself is rounded to BF16 (u |e|) and so is the other factor (u), and the
  FP32 sums add n 2^-24 of the absolute sum.  A transposed operand, a wrong
  block, a dropped term or a wrong Tweedie power gives errors of the size of
  the drift itself, far outside the bound;
* full chains: posterior-mean reconstruction RMSE within 1% of the FP64
  oracle chain (the configured dense Poisson NMF workload, 256 x 256, K = 8,
  B = 4);
* mu below mu_min (zero and tiny rows of W, zero columns of H): the drift
  within the same bound (the clamp enters its de/dmu), every output finite;
* graph replay == direct launches bit for bit; log-likelihood and RMSE over
  the dense data match the oracle in FP64; refused inputs;
* the single-pass kernel with GEMM1 on E4M3 (FP8) copies of the factors,
  one scale per 128-row / 128-column tile: the same drift test against the
  first-order bound with E4M3 rounding (u = 2^-4, plus half the subnormal
  spacing times the tile scale) for GEMM1's operands, where the bound can
  be as large as the drift, so the error must also stay below a quarter of
  the drift in RMS; the chain's posterior RMSE within 1 % of the oracle's.

Every case runs on both kernels: the single-pass one (mu once per entry, G_H
summed over a block's 128-row tiles by the update) and the two-sided one, in
both of its modes -- every item forming its own mu and E (dense_share_e=0),
or the rows items storing E and the columns items taking G_H = E^T W from it
(dense_share_e=1) -- also with V kept in BF16, where the bound adds the
rounding of v.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import Pair, dense_drift_bound, recovered_drift
from paper_1506_01418_gb300 import datagen
from paper_1506_01418_gb300 import psgld as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


DENSE = {
    # name: (I, J, K, B, p, phi, prior_kind, data, eps)
    "poisson_256_K8_B4": (256, 256, 8, 4, 1.0, 1.0, 0, "poisson", 1e-3),
    "poisson_ragged_K8": (67, 45, 8, 4, 1.0, 1.0, 0, "poisson", 1e-3),
    "gauss_K50_two_mtiles_three_ntiles": (300, 700, 50, 2, 0.0, 1.0, 1, "gamma", 1e-3),
    "gamma_K13": (120, 90, 13, 5, 2.0, 0.7, 0, "gamma", 1e-3),
    "cp_K100": (140, 170, 100, 2, 1.5, 1.0, 0, "gamma", 1e-3),
    "invgauss_K128": (90, 260, 128, 2, 3.0, 1.0, 0, "gamma", 1e-3),
    "poisson_K1_B7": (50, 61, 1, 7, 1.0, 1.0, 0, "poisson", 1e-3),
    "poisson_uneven_mtiles_K32": (257, 300, 32, 2, 1.0, 1.0, 0, "poisson", 1e-3),
    "poisson_K64_B1": (200, 150, 64, 1, 1.0, 1.0, 0, "poisson", 1e-3),
    "gaussnmf_K256_three_tiles": (400, 330, 256, 1, 0.0, 1.0, 0, "gamma", 1e-5),
    "poisson_K200_B3": (260, 390, 200, 3, 1.0, 1.0, 0, "poisson", 2e-4),
}

KERNELS = {
    "single_pass": dict(dense_path=3),
    "single_pass_fp8": dict(dense_path=3, dense_fp8=1),
    "auto": dict(dense_path=1),
    "two_sided": dict(dense_path=2, dense_share_e=0),
    "two_sided_bf16v": dict(dense_path=2, dense_v_bf16=1, dense_share_e=0),
    "two_sided_share": dict(dense_path=2, dense_share_e=1),
    "two_sided_bf16v_share": dict(dense_path=2, dense_v_bf16=1, dense_share_e=1),
}


def _cases():
    out = []
    for name in sorted(DENSE):
        for kern in KERNELS:
            if kern.startswith("single_pass") and DENSE[name][2] > 128:
                continue
            out.append((name, kern))
    return out


def _data(I, J, kind, p, seed):
    if kind == "poisson":
        V, _, _ = datagen.dense_poisson(I, J, 3, seed)
    else:
        V, _, _ = datagen.dense_gamma(I, J, 3, seed)
    if p >= 2:
        V = V + np.float32(0.5)
    return V


def _make(name, seed=7, kernel="auto", **opts):
    I, J, K, B, p, phi, kind, data, eps = DENSE[name]
    opts = {**KERNELS[kernel], **opts}
    V = _data(I, J, data, p, seed=I)
    i, j, v = datagen.dense_to_coo(V)
    nonneg = kind == 0
    W0, H0 = datagen.init_factors(I, J, K, seed=3, scale=0.4 if nonneg else 0.3, nonneg=nonneg)
    pr = Pair(I, J, K, B, p, phi, i, j, v, W0, H0, prior_kind=kind, lam=(0.8, 1.2),
              sig=(0.9, 1.1), seed=seed, eps=eps, V=V, **opts)
    return pr, V


@pytest.mark.parametrize("name,kernel", _cases())
def test_dense_part_step_drift_within_bf16_bound(name, kernel):
    pr, V = _make(name, kernel=kernel)
    I, J, K, B, p, phi, kind, data, eps = DENSE[name]
    v_bf16 = bool(KERNELS[kernel].get("dense_v_bf16", 0))
    fp8 = bool(KERNELS[kernel].get("dense_fp8", 0))
    mirror = kind == 0
    for t in range(1, B + 2):
        W0, H0 = pr.orc.get_factors()
        D_W, D_H = pr.orc.drift(t)
        S = pr.orc.scale(t)
        bW, bH = dense_drift_bound(V, W0, H0, t, B, p, phi, S, v_bf16=v_bf16, fp8=fp8)
        pr.gpu.part_step(t)
        Wg, Hg = pr.gpu_factors()
        zW = oracle.noise_matrix(7, t, 0, I, K)
        zH = oracle.noise_matrix(7, t, 1, J, K).T
        for xg, x0, z, D, bnd, what in ((Wg, W0, zW, D_W, bW, "W"), (Hg, H0, zH, D_H, bH, "H")):
            Dg, mask, rec = recovered_drift(xg.astype(np.float64), x0, z, D, eps, mirror)
            err = np.abs(Dg - D)
            lim = bnd + rec
            bad = mask & (err > lim)
            assert not bad.any(), (name, kernel, t, what, int(bad.sum()), float(err[bad].max()),
                                   float(lim[bad].min()))
            assert mask.mean() > 0.9
            rms_D = np.sqrt(np.mean(D[mask] ** 2))
            if fp8:
                # the worst-case E4M3 bound can reach the size of the drift
                # itself, so the error must also be well below the drift in
                # the mean: a wrong scale, byte order or operand gives errors
                # of the drift's own size
                assert np.sqrt(np.mean(err[mask] ** 2)) < 0.25 * rms_D, (name, what)
            else:
                # the drift itself is far larger than the bound: the check has teeth
                assert rms_D > 4 * np.sqrt(np.mean(bnd[mask] ** 2)), (name, what)
        if mirror:
            assert Wg.min() >= 0 and Hg.min() >= 0
        pr.sync_oracle_to_gpu()


@pytest.mark.parametrize("p", [1.0, 1.5, 2.0, 3.0])
@pytest.mark.parametrize("kernel", ["single_pass", "two_sided", "two_sided_bf16v", "two_sided_share"])
def test_dense_mu_below_mu_min_drift_within_bound(kernel, p):
    """mu below mu_min = 1e-2 on the tensor cores: every 5th row of W and
    every 7th column of H zero (mu = 0 exactly: BF16 keeps zeros, so e =
    v mu_min^(-p) / phi up to the rounding of e), every 5th row from the
    second tiny (0 < mu < mu_min).  The recovered drift stays within the
    BF16 bound (which takes max(mu - dmu, mu_min) in de/dmu), every output
    is finite, and on the zero rows and columns -- where the clamped factor
    is the whole signal -- the drift is far larger than the bound."""
    I, J, K, B, phi, eps, mu_min, seed = 140, 170, 24, 2, 0.8, 1e-4, 1e-2, 7
    V = _data(I, J, "gamma", p, seed=I)
    i, j, v = datagen.dense_to_coo(V)
    W0, H0 = datagen.init_factors(I, J, K, seed=3, scale=0.4, nonneg=True)
    W0[::5] = 0.0
    W0[1::5] = 1e-5
    H0[:, ::7] = 0.0
    pr = Pair(I, J, K, B, p, phi, i, j, v, W0, H0, prior_kind=0, lam=(0.8, 1.2), seed=seed,
              eps=eps, V=V, mu_min=mu_min, **KERNELS[kernel])
    v_bf16 = bool(KERNELS[kernel].get("dense_v_bf16", 0))
    for t in range(1, B + 1):
        pr.set_factors(W0, H0)
        Wc, Hc = pr.orc.get_factors()
        D_W, D_H = pr.orc.drift(t)
        S = pr.orc.scale(t)
        bW, bH = dense_drift_bound(V, Wc, Hc, t, B, p, phi, S, mu_min=mu_min, v_bf16=v_bf16)
        pr.gpu.part_step(t)
        Wg, Hg = pr.gpu_factors()
        assert np.all(np.isfinite(Wg)) and np.all(np.isfinite(Hg))
        zW = oracle.noise_matrix(seed, t, 0, I, K)
        zH = oracle.noise_matrix(seed, t, 1, J, K).T
        for xg, x0, z, D, bnd, zero, what in ((Wg, Wc, zW, D_W, bW, np.s_[::5, :], "W"),
                                               (Hg, Hc, zH, D_H, bH, np.s_[:, ::7], "H")):
            Dg, mask, rec = recovered_drift(xg.astype(np.float64), x0, z, D, eps, True)
            err = np.abs(Dg - D)
            bad = mask & (err > bnd + rec)
            assert not bad.any(), (kernel, p, t, what, int(bad.sum()))
            zm = mask[zero]
            assert zm.mean() > 0.5
            assert np.sqrt(np.mean(D[zero][zm] ** 2)) > 4 * np.sqrt(np.mean(bnd[zero][zm] ** 2))


@pytest.mark.parametrize("kernel", ["single_pass", "two_sided", "two_sided_share"])
def test_dense_graph_replay_equals_direct_launches(kernel):
    a, _ = _make("gauss_K50_two_mtiles_three_ntiles", kernel=kernel, use_graphs=1, burn_in_sweeps=1)
    b, _ = _make("gauss_K50_two_mtiles_three_ntiles", kernel=kernel, use_graphs=0, burn_in_sweeps=1)
    for n in (1, 2):
        a.gpu.sweep(n)
        b.gpu.sweep(n)
    Wa, Ha = a.gpu_factors()
    Wb, Hb = b.gpu_factors()
    assert np.array_equal(Wa, Wb) and np.array_equal(Ha, Hb)
    ma, mb = a.gpu.posterior_mean(), b.gpu.posterior_mean()
    for x, y in zip(ma[:4], mb[:4]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("kernel", ["single_pass", "two_sided_bf16v", "single_pass_fp8", "two_sided_bf16v_share"])
def test_dense_is_deterministic(kernel):
    a, _ = _make("poisson_uneven_mtiles_K32", kernel=kernel)
    b, _ = _make("poisson_uneven_mtiles_K32", kernel=kernel)
    a.gpu.sweep(2)
    b.gpu.sweep(2)
    Wa, Ha = a.gpu_factors()
    Wb, Hb = b.gpu_factors()
    assert np.array_equal(Wa, Wb) and np.array_equal(Ha, Hb)


@pytest.mark.parametrize("kernel", ["single_pass", "two_sided_bf16v"])
def test_dense_size_proportional_parts_drift_within_bound(kernel):
    """part_mode = 1 (condition C2) on the tensor-core path: every iteration
    uses the part the oracle draws, and the drift stays within the BF16
    bound of that part."""
    name = "gamma_K13"
    pr, V = _make(name, kernel=kernel, part_mode=1)
    pr.orc.set_part_mode(1)
    I, J, K, B, p, phi, kind, data, eps = DENSE[name]
    v_bf16 = bool(KERNELS[kernel].get("dense_v_bf16", 0))
    seen = set()
    for t in range(1, 3 * B + 1):
        s = pr.orc.part_index(t)
        seen.add(s)
        W0, H0 = pr.orc.get_factors()
        D_W, D_H = pr.orc.drift(t)
        S = pr.orc.scale(t)
        bW, bH = dense_drift_bound(V, W0, H0, t, B, p, phi, S, v_bf16=v_bf16, part=s)
        pr.gpu.part_step(t)
        Wg, Hg = pr.gpu_factors()
        zW = oracle.noise_matrix(7, t, 0, I, K)
        zH = oracle.noise_matrix(7, t, 1, J, K).T
        for xg, x0, z, D, bnd, what in ((Wg, W0, zW, D_W, bW, "W"), (Hg, H0, zH, D_H, bH, "H")):
            Dg, mask, rec = recovered_drift(xg.astype(np.float64), x0, z, D, eps, True)
            bad = mask & (np.abs(Dg - D) > bnd + rec)
            assert not bad.any(), (kernel, t, s, what, int(bad.sum()))
        pr.sync_oracle_to_gpu()
    assert len(seen) > 1


@pytest.mark.parametrize("kernel", ["two_sided", "two_sided_share"])
@pytest.mark.parametrize("name,sms", [("poisson_K200_B3", 7), ("poisson_K200_B3", 1),
                                      ("gaussnmf_K256_three_tiles", 2), ("gaussnmf_K256_three_tiles", 1),
                                      ("gauss_K50_two_mtiles_three_ntiles", 1)])
def test_two_sided_kernel_on_fewer_sms_gives_the_same_chain(name, sms, kernel):
    """max_sms only shrinks the persistent grid: every item still runs once,
    so the chain is the same bit for bit.  On one or two CTAs each CTA runs
    several rows items before its first columns item, whose stages then
    take over the rows items' shared memory."""
    a, _ = _make(name, kernel=kernel)
    b, _ = _make(name, kernel=kernel, max_sms=sms)
    a.gpu.sweep(2)
    b.gpu.sweep(2)
    Wa, Ha = a.gpu_factors()
    Wb, Hb = b.gpu_factors()
    assert np.array_equal(Wa, Wb) and np.array_equal(Ha, Hb)


@pytest.mark.parametrize("name", ["poisson_K200_B3", "gaussnmf_K256_three_tiles", "poisson_uneven_mtiles_K32"])
def test_two_sided_columns_item_width_does_not_change_the_chain(name):
    """wide_col_blocks only regroups the columns items (256 rows in two
    accumulators or 128 rows in one); every G_H row is the same sequence of
    MMAs, so the chain is the same bit for bit."""
    B = DENSE[name][3]
    out = []
    for w in (0, B, -1):
        pr, _ = _make(name, kernel="two_sided_share", wide_col_blocks=w)
        pr.gpu.sweep(2)
        out.append(pr.gpu_factors())
    for Wx, Hx in out[1:]:
        assert np.array_equal(Wx, out[0][0]) and np.array_equal(Hx, out[0][1])


@pytest.mark.parametrize("name", ["poisson_ragged_K8", "gauss_K50_two_mtiles_three_ntiles",
                                  "cp_K100", "gamma_K13", "poisson_K200_B3"])
def test_dense_log_lik_and_rmse_match_oracle(name):
    pr, _ = _make(name, burn_in_sweeps=0)
    pr.gpu.sweep(1)
    pr.sync_oracle_to_gpu()
    assert pr.gpu.log_lik() == pytest.approx(pr.orc.log_lik(), rel=1e-9, abs=1e-9)
    assert pr.gpu.rmse() == pytest.approx(pr.orc.rmse(False), rel=1e-9)


@pytest.mark.parametrize("kernel", ["auto", "two_sided_bf16v", "single_pass_fp8"])
def test_dense_chain_posterior_rmse_within_one_percent_of_oracle(kernel):
    """The configured dense Poisson NMF workload (Sec. 4.1 shape): 256 x 256,
    K = 8, B = 4, W*, H* ~ Gamma(1, 1), V ~ Poisson(W* H*), exponential priors
    rate 1, eps = 1e-4; 1000 sweeps, posterior means over the last 500."""
    I = J = 256
    K, B, sweeps = 8, 4, 1000
    V, _, _ = datagen.dense_poisson(I, J, K, seed=0)
    i, j, v = datagen.dense_to_coo(V)
    W0, H0 = datagen.init_factors(I, J, K, seed=0, scale=1.0, nonneg=True)
    pr = Pair(I, J, K, B, 1.0, 1.0, i, j, v, W0, H0, prior_kind=0, seed=11, eps=1e-4, V=V,
              burn_in_sweeps=sweeps // 2, **KERNELS[kernel])
    pr.gpu.sweep(sweeps)
    pr.orc.sweep(sweeps)
    r_gpu, r_or = pr.gpu.rmse(True), pr.orc.rmse(True)
    assert abs(r_gpu - r_or) <= 0.01 * r_or, (r_gpu, r_or)


@pytest.mark.parametrize("kernel", ["auto", "two_sided_bf16v", "fp32_gather"])
def test_compound_poisson_chain_within_one_percent_of_oracle(kernel):
    """Tweedie p = 1.5 on data drawn from its own law, the compound
    Poisson-gamma (the paper's Sec. 4 compound-Poisson experiment; exact
    zeros included): 256 x 256, K = 8, B = 4, W*, H* ~ Gamma(1, 1), phi = 1,
    exponential priors rate 1, eps = 1e-4; 1000 sweeps, posterior-mean RMSE
    within 1 % of the FP64 oracle chain's."""
    I = J = 256
    K, B, sweeps = 8, 4, 1000
    V, _, _ = datagen.dense_compound_poisson(I, J, K, seed=1, p=1.5, phi=1.0)
    assert (V == 0).mean() > 0.01
    i, j, v = datagen.dense_to_coo(V)
    W0, H0 = datagen.init_factors(I, J, K, seed=0, scale=1.0, nonneg=True)
    opts = dict(dense_path=0) if kernel == "fp32_gather" else KERNELS[kernel]
    pr = Pair(I, J, K, B, 1.5, 1.0, i, j, v, W0, H0, prior_kind=0, seed=11, eps=1e-4, V=V,
              burn_in_sweeps=sweeps // 2, **opts)
    pr.gpu.sweep(sweeps)
    pr.orc.sweep(sweeps)
    r_gpu, r_or = pr.gpu.rmse(True), pr.orc.rmse(True)
    assert abs(r_gpu - r_or) <= 0.01 * r_or, (r_gpu, r_or)


def test_compound_poisson_device_generator_law():
    """The device generator the serving jobs use for p = 1.5: over 2048 x 2048
    draws, standardised residuals (v - mu) / sqrt(phi mu^p) have mean 0 and
    variance 1, and the zero mass is the mean of exp(-lam)."""
    p, phi = 1.5, 1.3
    V, M = datagen.dense_compound_poisson_device(2048, 2048, 8, 3, torch.device("cuda"), p=p,
                                                 phi=phi, return_mean=True)
    V, M = V.double(), M.double()
    n = V.numel()
    z = (V - M) / torch.sqrt(phi * M ** p)
    assert abs(float(z.mean())) < 4 / np.sqrt(n)
    assert abs(float((z ** 2).mean()) - 1.0) < 0.01
    lam = M ** (2 - p) / (phi * (2 - p))
    p0 = float(torch.exp(-lam).mean())
    assert abs(float((V == 0).double().mean()) - p0) < 4 * np.sqrt(0.25 / n)
    assert float(V.min()) >= 0


def test_dense_refusals():
    I, J = 40, 30
    V = np.ones((I, J), np.float32)
    for K, opts in ((257, dict(dense_path=1)), (129, dict(dense_path=3)),
                    (8, dict(dense_path=3, dense_v_bf16=1)), (8, dict(dense_path=2, dense_fp8=1)),
                    (200, dict(dense_path=1, dense_fp8=1))):
        c = P.PSGLD(I, J, K, 2, 1.0, 1.0, **opts)
        with pytest.raises(P.PsgldError) as ex:
            c.set_data_dense(torch.from_numpy(V).cuda())
        assert ex.value.status == P.PSGLD_ERR_ARG
        c.close()
    with pytest.raises(P.PsgldError) as ex:
        P.PSGLD(I, J, 8, 2, 1.0, 1.0, dense_path=4)
    assert ex.value.status == P.PSGLD_ERR_ARG
    c = P.PSGLD(I, J, 8, 2, 1.0, 1.0, dense_path=1)
    bad = V.copy()
    bad[3, 4] = -1.0                          # negative entry, non-negative model
    with pytest.raises(P.PsgldError) as ex:
        c.set_data_dense(torch.from_numpy(bad).cuda())
    assert ex.value.status == P.PSGLD_ERR_ARG
    c.set_data_dense(torch.from_numpy(V).cuda())
    with pytest.raises(P.PsgldError) as ex:
        P.psgld_part_layout(c.ctx, 0, I)
    assert ex.value.status == P.PSGLD_ERR_STATE
    c.close()
