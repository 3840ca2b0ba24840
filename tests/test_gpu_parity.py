"""CUDA path vs the FP64 oracle, through the C ABI.

* schedule, piece bounds and per-part layouts: bit-exact;
* one FP32 part-step from identical factors, identical Philox stream:
  every element within 1e-5 of the magnitudes the step sums, and the
  increment (new - old factors) within 1e-5 of its own largest element plus
  the FP32 rounding of the stored result (see gpu_helpers.step_errors), for
  every part of a sweep, across team shapes (K = 1 .. 512), Tweedie powers,
  both priors, ragged piece sizes, rows split over many work units, empty
  parts, frozen factors, mu below mu_min (zero and tiny rows and columns)
  and the decaying step size eps_t = (a/t)^b;
* factors beyond L2 (the large sparse workload's two-stream order) within
  the same step tolerance;
* graph replay == direct launches, bit for bit;
* log-likelihood, RMSE and posterior moments against the oracle.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import STEP_RTOL, Pair, dense_case, rel_err, sparse_case, step_errors
from paper_1506_01418_gb300 import datagen
from paper_1506_01418_gb300 import psgld as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


# ---------------------------------------------------------------------------
# schedule and layouts
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("I,J,B,nnz", [(7, 5, 2, 20), (67, 45, 4, 900), (300, 200, 3, 20000),
                                       (9, 9, 9, 50), (513, 1000, 8, 30000), (10, 10, 1, 60)])
def test_schedule_and_layout_bit_exact(I, J, B, nnz):
    i, j, v = sparse_case(I, J, nnz, 4, seed=I + B)
    W0, H0 = datagen.init_factors(I, J, 4, seed=1)
    pr = Pair(I, J, 4, B, 1.0, 1.0, i, j, v, W0, H0)
    rs, cs = P.psgld_piece_bounds(pr.gpu.ctx, B)
    assert list(rs) == [oracle.piece_start(r, I, B) for r in range(B + 1)]
    assert list(cs) == [oracle.piece_start(r, J, B) for r in range(B + 1)]
    for t in (1, 2, B, B + 1, 5 * B + 3, (1 << 33) + 1):
        cp = P.psgld_part_schedule(pr.gpu.ctx, t, B)
        assert list(cp) == [oracle.part_col_piece(t, B, r) for r in range(B)]
    for s in range(B):
        ptr, cols = P.psgld_part_layout(pr.gpu.ctx, s, I)
        t = s + 1
        assert ptr[-1] == pr.orc.part_size(t)
        rows = np.repeat(np.arange(I), np.diff(ptr))
        for r in range(B):
            c = oracle.part_col_piece(t, B, r)
            bi, bj = pr.orc.block_entries(r, c)
            sel = (rows >= rs[r]) & (rows < rs[r + 1])
            assert np.array_equal(rows[sel], bi)
            assert np.array_equal(cols[sel], bj)


# ---------------------------------------------------------------------------
# one part-step vs the oracle
# ---------------------------------------------------------------------------

CASES = {
    # name: (I, J, K, B, p, phi, prior_kind, data, eps)
    "poisson_dense_K8_ragged": (67, 45, 8, 4, 1.0, 1.0, 0, ("dense", "poisson"), 1e-3),
    "gauss_sparse_K50_split": (300, 200, 50, 3, 0.0, 1.0, 1, ("sparse", 20000), 1e-3),
    "gamma_K13": (120, 90, 13, 5, 2.0, 0.7, 0, ("sparse", 3000), 1e-3),
    "cp_K100": (40, 70, 100, 2, 1.5, 1.0, 0, ("dense", "gamma"), 1e-4),
    "gauss_K160": (150, 130, 160, 3, 0.0, 2.0, 1, ("sparse", 8000), 1e-4),
    "invgauss_K300": (50, 60, 300, 2, 3.0, 1.0, 0, ("dense", "gamma"), 1e-5),
    "poisson_K512_B1": (33, 29, 512, 1, 1.0, 1.0, 0, ("dense", "poisson"), 1e-5),
    "poisson_K1_B7": (50, 61, 1, 7, 1.0, 1.0, 0, ("dense", "poisson"), 1e-3),
    "gauss_K32_BminIJ": (9, 12, 32, 9, 0.0, 1.0, 1, ("sparse", 80), 1e-3),
    "poisson_K64": (100, 80, 64, 4, 1.0, 1.0, 0, ("sparse", 4000), 1e-4),
    "empty_data": (20, 30, 6, 3, 1.0, 1.0, 0, ("sparse", 0), 1e-2),
    # rows whose entries in a part span many work units of the gradient
    # kernel (their partial sums added in unit order by the update kernel),
    # with K = 24 (one float4 group per lane) and K = 200 (several)
    "heavy_rows_B1_K24": (40, 1500, 24, 1, 1.0, 1.0, 0, ("dense", "poisson"), 1e-4),
    "heavy_rows_K200_B2": (30, 1100, 200, 2, 0.0, 1.0, 1, ("dense", "gamma"), 1e-4),
}


def _make(name, use_graphs=1, seed=7, **opts):
    I, J, K, B, p, phi, kind, data, eps = CASES[name]
    eps = opts.pop("eps", eps)
    if data[0] == "dense":
        i, j, v = dense_case(I, J, 3, seed=I, kind=data[1])
        if p >= 2:
            v = v + 0.5
    else:
        if data[1] == 0:
            i = np.zeros(0, np.int32); j = np.zeros(0, np.int32); v = np.zeros(0, np.float32)
        else:
            i, j, v = sparse_case(I, J, data[1], 5, seed=I + J)
    nonneg = kind == 0
    W0, H0 = datagen.init_factors(I, J, K, seed=3, scale=0.4 if nonneg else 0.3, nonneg=nonneg)
    return Pair(I, J, K, B, p, phi, i, j, v, W0, H0, prior_kind=kind, lam=(0.8, 1.2),
                sig=(0.9, 1.1), seed=seed, eps=eps, use_graphs=use_graphs, **opts)


@pytest.mark.parametrize("name", sorted(CASES))
def test_one_part_step_matches_oracle(name):
    pr = _make(name)
    B = pr.B
    for t in range(1, B + 2):
        Wg, Hg = pr.step_and_check(t)
        if CASES[name][6] == 0:
            assert Wg.min() >= 0 and Hg.min() >= 0
        pr.sync_oracle_to_gpu()


def test_large_iteration_index_uses_high_counter_bits():
    pr = _make("poisson_dense_K8_ragged")
    for t in ((1 << 32) + 3, (1 << 40) + 1):
        pr.step_and_check(t)
        pr.sync_oracle_to_gpu()


def _clamp_factors(W, H):
    """Every 7th row of W and every 11th column of H zero (mu = 0 on their
    entries), every 7th row from the third tiny (0 < mu < 1e-2)."""
    W = W.copy()
    H = H.copy()
    W[::7] = 0.0
    W[3::7] = 1e-5
    H[:, ::11] = 0.0
    return W, H


@pytest.mark.parametrize("p", [1.0, 1.5, 2.0, 3.0])
@pytest.mark.parametrize("data", ["sparse", "dense"])
def test_mu_below_mu_min_matches_oracle(p, data):
    """The clamp max(mu, mu_min) of the Tweedie factor (mu_min = 1e-2): zero
    rows of W and columns of H give mu = 0 on every entry they touch, tiny
    rows 0 < mu < mu_min.  Each part-step starts from such factors again."""
    I, J, K, B = (150, 130, 13, 3) if data == "sparse" else (67, 45, 100, 2)
    if data == "sparse":
        i, j, v = sparse_case(I, J, 6000, 5, seed=I + J)
    else:
        i, j, v = dense_case(I, J, 3, seed=I, kind="gamma")
    if p >= 2:
        v = v + np.float32(0.5)
    W0, H0 = datagen.init_factors(I, J, K, seed=3, scale=0.4, nonneg=True)
    W0, H0 = _clamp_factors(W0, H0)
    pr = Pair(I, J, K, B, p, 0.8, i, j, v, W0, H0, prior_kind=0, lam=(0.8, 1.2), seed=9,
              eps=1e-4, mu_min=1e-2)
    mu = W0.astype(np.float64) @ H0.astype(np.float64)
    assert (mu[i, j] == 0).sum() > 0 and ((mu[i, j] > 0) & (mu[i, j] < 1e-2)).sum() > 0
    for t in range(1, B + 2):
        Wg, Hg = pr.step_and_check(t, W0, H0)
        assert Wg.min() >= 0 and Hg.min() >= 0


@pytest.mark.parametrize("a,b", [(0.01, 0.51), (2e-5, 0.75)])
@pytest.mark.parametrize("name", ["gauss_sparse_K50_split", "poisson_dense_K8_ragged"])
def test_decaying_step_size_matches_oracle(name, a, b):
    """eps_mode = POLY: eps_t = (a/t)^b computed on the device from t (Sec. 2
    Eq. eps; Sec. 4.1 uses a = 0.01, b = 0.51), part-steps at t = 1, 2, B + 1
    and beyond 2^32 from the same factors, then a graph-replayed chain of
    four sweeps on both sides independently."""
    pr = _make(name, eps_mode=P.PSGLD_EPS_POLY, eps_a=a, eps_b=b)
    W0, H0 = pr.orc.get_factors()
    B = pr.B
    for t in (1, 2, B + 1, (1 << 32) + 3):
        pr.step_and_check(t, W0.astype(np.float32), H0.astype(np.float32))
    if a > 1e-3:
        return            # eps_1 ~ 0.1: a chain of this size is not stable
    pr.set_factors(W0.astype(np.float32), H0.astype(np.float32))
    pr.gpu.part_step(1)   # bring both to t = B at a sweep boundary
    pr.orc.part_step(1)
    for t in range(2, B + 1):
        pr.gpu.part_step(t)
        pr.orc.part_step(t)
    pr.sync_oracle_to_gpu()
    pr.gpu.sweep(4)
    pr.orc.sweep(4)
    Wg, Hg = pr.gpu_factors()
    Wo, Ho = pr.orc.get_factors()
    assert rel_err(Wg, Wo) < 1e-4 and rel_err(Hg, Ho) < 1e-4


def test_noise_stream_matches_oracle():
    """No data, flat Gaussian prior: the step is w + sqrt(2 eps) z exactly, so
    the normals themselves are compared (Philox words agree bit for bit, or z
    would differ completely)."""
    I, J, K, eps = 64, 48, 7, 0.5
    i = np.zeros(0, np.int32); j = np.zeros(0, np.int32); v = np.zeros(0, np.float32)
    W0 = np.zeros((I, K), np.float32); H0 = np.zeros((K, J), np.float32)
    pr = Pair(I, J, K, 2, 0.0, 1.0, i, j, v, W0, H0, prior_kind=1, sig=(1e18, 1e18),
              seed=0xDEADBEEF12345, eps=eps)
    t = 12345
    pr.gpu.part_step(t)
    Wg, Hg = pr.gpu_factors()
    zw = Wg / np.float32(np.sqrt(2 * eps))
    zh = Hg.T / np.float32(np.sqrt(2 * eps))
    np.testing.assert_allclose(zw, oracle.noise_matrix(0xDEADBEEF12345, t, 0, I, K),
                               rtol=2e-6, atol=2e-6)
    np.testing.assert_allclose(zh, oracle.noise_matrix(0xDEADBEEF12345, t, 1, J, K),
                               rtol=2e-6, atol=2e-6)


@pytest.mark.parametrize("frozen", ["W", "H"])
def test_frozen_factor_matches_oracle(frozen):
    """freeze_W / freeze_H: the frozen factor stays bit for bit, the other
    one steps as the oracle's does."""
    opts = {"freeze_W": 1} if frozen == "W" else {"freeze_H": 1}
    pr = _make("gauss_sparse_K50_split", **opts)
    W0, H0 = pr.gpu_factors()
    for t in range(1, 4):
        pr.step_and_check(t)
        pr.sync_oracle_to_gpu()
    W1, H1 = pr.gpu_factors()
    assert np.array_equal(W1, W0) == (frozen == "W")
    assert np.array_equal(H1, H0) == (frozen == "H")


def test_frozen_factor_is_unchanged():
    pr = _make("gauss_sparse_K50_split", freeze_H=1)
    Wb, Hb = pr.gpu_factors()
    pr.gpu.sweep(2)
    Wa, Ha = pr.gpu_factors()
    assert np.array_equal(Ha, Hb)
    assert not np.array_equal(Wa, Wb)


# ---------------------------------------------------------------------------
# sweeps: graphs vs launches, posterior sums, diagnostics
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["gauss_sparse_K50_split", "poisson_K1_B7", "gamma_K13",
                                  "heavy_rows_B1_K24"])
def test_graph_replay_equals_direct_launches(name):
    a = _make(name, use_graphs=1, burn_in_sweeps=1)
    b = _make(name, use_graphs=0, burn_in_sweeps=1)
    for n in (1, 2, 1):
        a.gpu.sweep(n)
        b.gpu.sweep(n)
    Wa, Ha = a.gpu_factors()
    Wb, Hb = b.gpu_factors()
    assert np.array_equal(Wa, Wb) and np.array_equal(Ha, Hb)
    ma = a.gpu.posterior_mean()
    mb = b.gpu.posterior_mean()
    assert ma[4] == mb[4] == 3
    for x, y in zip(ma[:4], mb[:4]):
        assert np.array_equal(x, y)
    assert a.gpu.iterations_done == 4 * a.B


def test_factors_beyond_l2_take_the_two_stream_order_and_match_oracle():
    """Factors above 64 MB (W: 180000 x 100 FP32, 72 MB) take the large
    sparse workload's order: W's gradient alone on the resident grid, then
    H's gradient on a second stream beside W's update.  Two part-steps
    match the oracle within the step tolerance, and a captured-graph sweep
    equals direct launches bit for bit."""
    I, J, K, B = 180000, 2000, 100, 8
    i, j, v = sparse_case(I, J, 1_500_000, 8, seed=17, zipf=1.2)
    W0, H0 = datagen.init_factors(I, J, K, seed=5, scale=0.25, nonneg=False)
    pr = Pair(I, J, K, B, 0.0, 1.0, i, j, v, W0, H0, prior_kind=1, sig=(0.9, 1.1), seed=13,
              eps=1e-4)
    for t in (1, 2):
        pr.step_and_check(t)
        pr.sync_oracle_to_gpu()
    pr.gpu.close()
    chains = []
    for graphs in (1, 0):
        c = P.PSGLD(I, J, K, B, 0.0, 1.0, prior_kind=1, seed=13, eps=1e-4, use_graphs=graphs)
        c.set_data_coo(torch.as_tensor(i, dtype=torch.int32, device="cuda"),
                       torch.as_tensor(j, dtype=torch.int32, device="cuda"),
                       torch.as_tensor(v, dtype=torch.float32, device="cuda"))
        c.set_factors(torch.as_tensor(np.ascontiguousarray(W0, dtype=np.float32), device="cuda"),
                      torch.as_tensor(np.ascontiguousarray(H0.T, dtype=np.float32), device="cuda"))
        c.sweep(1)
        c.sweep(1)
        chains.append(c)
    (Wa, Ha), (Wb, Hb) = (c.get_factors() for c in chains)
    assert torch.equal(Wa, Wb) and torch.equal(Ha, Hb)
    for c in chains:
        c.close()


def test_sweep_matches_oracle_chain():
    """A few sweeps run independently on both sides stay within the
    accumulated FP32 error; the posterior sums follow."""
    pr = _make("poisson_dense_K8_ragged", burn_in_sweeps=1)
    pr.gpu.sweep(4)
    pr.orc.sweep(4)
    Wg, Hg = pr.gpu_factors()
    Wo, Ho = pr.orc.get_factors()
    assert rel_err(Wg, Wo) < 1e-4 and rel_err(Hg, Ho) < 1e-4
    Wm, Wv, Hm, Hv, n = pr.gpu.posterior_mean()
    oWm, oWv, oHm, oHv, on = pr.orc.posterior()
    assert n == on == 3
    assert rel_err(Wm, oWm) < 1e-4 and rel_err(Hm, oHm.T) < 1e-4
    np.testing.assert_allclose(Wv, oWv, rtol=1e-2, atol=1e-6 * np.abs(oWm).max() ** 2)


@pytest.mark.parametrize("name", ["poisson_dense_K8_ragged", "gauss_sparse_K50_split",
                                  "gamma_K13", "cp_K100", "invgauss_K300"])
def test_log_lik_and_rmse_match_oracle(name):
    pr = _make(name, burn_in_sweeps=0)
    pr.gpu.sweep(1)
    pr.sync_oracle_to_gpu()
    ll_g, ll_o = pr.gpu.log_lik(), pr.orc.log_lik()
    assert ll_g == pytest.approx(ll_o, rel=1e-9, abs=1e-9)
    assert pr.gpu.rmse() == pytest.approx(pr.orc.rmse(False), rel=1e-9)


def test_rmse_of_posterior_mean_matches_definition():
    pr = _make("gauss_sparse_K50_split", burn_in_sweeps=0)
    pr.gpu.sweep(3)
    Wm, _, Hm, _, n = pr.gpu.posterior_mean()
    i, j, v = sparse_case(300, 200, 20000, 5, seed=500)
    want = np.sqrt(np.mean((v - np.einsum("nk,nk->n", Wm[i], Hm[j])) ** 2))
    assert pr.gpu.rmse(True) == pytest.approx(want, rel=1e-9)


@pytest.mark.parametrize("graphs", [0, 1])
def test_profile_counts_every_part_step(graphs):
    pr = _make("gauss_sparse_K50_split", use_graphs=graphs, profile=1)
    for _ in range(2):
        pr.gpu.sweep(1)
        ms, n = pr.gpu.profile_read()
        assert n == pr.B and ms > 0.0
    ms, n = pr.gpu.profile_read()
    assert n == 0 and ms == 0.0
    pr.gpu.part_step(pr.B + pr.B + 1)
    ms, n = pr.gpu.profile_read()
    assert n == 1 and ms > 0.0


# ---------------------------------------------------------------------------
# errors are reported, not hidden
# ---------------------------------------------------------------------------

def test_invalid_inputs_are_rejected():
    c = P.PSGLD(10, 10, 4, 2, 1.0, 1.0)
    dev = "cuda"
    t = lambda a, d: torch.as_tensor(a, dtype=d, device=dev)  # noqa: E731
    with pytest.raises(P.PsgldError) as e:
        c.part_step(1)
    assert e.value.status == P.PSGLD_ERR_STATE
    with pytest.raises(P.PsgldError) as e:   # duplicate pair
        c.set_data_coo(t([0, 1, 0], torch.int32), t([0, 1, 0], torch.int32),
                       t([1.0, 2.0, 3.0], torch.float32))
    assert e.value.status == P.PSGLD_ERR_ARG
    with pytest.raises(P.PsgldError):         # out of range
        c.set_data_coo(t([0, 10], torch.int32), t([0, 1], torch.int32),
                       t([1.0, 2.0], torch.float32))
    with pytest.raises(P.PsgldError):         # negative value in a non-negative model
        c.set_data_coo(t([0, 1], torch.int32), t([0, 1], torch.int32),
                       t([1.0, -2.0], torch.float32))
    c.set_data_coo(t([0, 1], torch.int32), t([0, 1], torch.int32), t([1.0, 2.0], torch.float32))
    with pytest.raises(P.PsgldError):         # negative factor in a non-negative model
        c.set_factors(-torch.ones(10, 4, device=dev), torch.ones(10, 4, device=dev))
    c.set_factors(torch.ones(10, 4, device=dev), torch.ones(10, 4, device=dev))
    c.part_step(1)
    with pytest.raises(P.PsgldError) as e:    # not at a sweep boundary
        c.sweep(1)
    assert e.value.status == P.PSGLD_ERR_STATE
    c.part_step(2)
    c.sweep(1)
    assert c.iterations_done == 4


def test_size_proportional_parts_match_oracle():
    """part_mode = 1 (condition C2): the part drawn at every iteration is the
    oracle's, bit for bit, and part-steps and a sweep follow it."""
    pr = _make("gamma_K13", part_mode=1)
    pr.orc.set_part_mode(1)
    B = pr.B
    for t in list(range(1, 301)) + [(1 << 32) + 5]:
        cp = P.psgld_part_schedule(pr.gpu.ctx, t, B)
        s = pr.orc.part_index(t)
        assert list(cp) == [(r + s) % B for r in range(B)], t
    seen = set()
    for t in range(1, 3 * B + 1):
        seen.add(pr.orc.part_index(t))
        pr.step_and_check(t, part=pr.orc.part_index(t))
        pr.sync_oracle_to_gpu()
    assert len(seen) > 1
    pr.gpu.sweep(2)
    pr.orc.sweep(2)
    Wg, Hg = pr.gpu_factors()
    Wo, Ho = pr.orc.get_factors()
    assert rel_err(Wg, Wo) < 1e-4 and rel_err(Hg, Ho) < 1e-4
