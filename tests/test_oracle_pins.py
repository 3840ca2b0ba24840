"""Pins of the FP64 oracle against facts fixed outside it.

Each test ties one oracle function to something other than the oracle itself:
published known-answer vectors, closed forms, textbook densities from scipy,
finite differences, brute-force enumeration, or an independent dense numpy
computation of the same equation.  A dropped term, a wrong sign, a wrong index
or a transposed operand anywhere in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1506_01418_gb300 import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Random numbers
# ---------------------------------------------------------------------------

def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors (SC'11)."""
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = oracle.philox4x32_10(r[0:4], r[4:6])
        assert list(out) == r[6:10]


def test_noise_is_standard_normal():
    """Box-Muller output: mean 0, variance 1, Kolmogorov-Smirnov vs N(0, 1)."""
    z = oracle.noise_matrix(seed=1234, t=7, mat=0, nrows=20000, K=10).ravel()
    assert abs(z.mean()) < 4.0 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 4.0 * math.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # fourth moment of a standard normal is 3
    assert abs(np.mean(z ** 4) - 3.0) < 0.1


def test_noise_inverts_to_philox_uniforms():
    """Inverting Box-Muller recovers the uniforms: radius^2 = -2 log u0 and
    angle = 2 pi u1.  Each recovered u must sit at (x >> 9) + 1/2 on the 2^-23
    grid, x being the (known-answer-pinned) Philox word of that counter."""
    seed, t = 0x1234ABCD5678, 9
    for row in (0, 3, 77):
        for q in range(3):
            z = [oracle.noise(seed, t, 1, row, 4 * q + n) for n in range(4)]
            x = oracle.philox4x32_10(
                [q, row, t & 0xFFFFFFFF, ((t >> 32) << 1) | 1],
                [seed & 0xFFFFFFFF, seed >> 32])
            for a, b, (xa, xb) in ((z[0], z[1], x[0:2]), (z[2], z[3], x[2:4])):
                u_rad = math.exp(-(a * a + b * b) / 2.0)
                u_ang = (math.atan2(b, a) / (2.0 * math.pi)) % 1.0
                assert u_rad * 2 ** 23 - 0.5 == pytest.approx(int(xa) >> 9, abs=1e-3)
                assert u_ang * 2 ** 23 - 0.5 == pytest.approx(int(xb) >> 9, abs=1e-3)


def test_noise_streams_are_independent():
    """Different t, matrix, seed or row give uncorrelated normals."""
    a = oracle.noise_matrix(5, 1, 0, 4000, 8).ravel()
    for other in (oracle.noise_matrix(5, 2, 0, 4000, 8),       # next iteration
                  oracle.noise_matrix(5, 1, 1, 4000, 8),       # other matrix
                  oracle.noise_matrix(6, 1, 0, 4000, 8),       # other seed
                  oracle.noise_matrix(5, 1 + (1 << 32), 0, 4000, 8)):  # high bits of t
        c = np.corrcoef(a, other.ravel())[0, 1]
        assert abs(c) < 5.0 / math.sqrt(a.size)
    # repeatable
    assert np.array_equal(a, oracle.noise_matrix(5, 1, 0, 4000, 8).ravel())
    # element k of row r is the single-element query
    m = oracle.noise_matrix(3, 11, 1, 5, 7)
    for r in range(5):
        for k in range(7):
            assert m[r, k] == oracle.noise(3, 11, 1, r, k)


# ---------------------------------------------------------------------------
# Partition and schedule: brute force on tiny inputs
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("B", list(range(1, 9)))
def test_partition_and_parts_brute_force(B):
    for n in range(B, 3 * B + 3):
        starts = [oracle.piece_start(r, n, B) for r in range(B + 1)]
        assert starts[0] == 0 and starts[-1] == n
        pieces = [set(range(starts[r], starts[r + 1])) for r in range(B)]
        # P_B([n]): B non-empty disjoint subsets whose union is [n]
        assert all(len(p) > 0 for p in pieces)
        assert set().union(*pieces) == set(range(n))
        assert sum(len(p) for p in pieces) == n
        for x in range(n):
            assert x in pieces[oracle.piece_of(x, n, B)]
        if n % B == 0:   # equal pieces, as in the experiments
            assert all(len(p) == n // B for p in pieces)
    for t0 in (1, 2 * B + 1, 7 * B + 1):
        seen = set()
        for t in range(t0, t0 + B):
            rows = list(range(B))
            cols = [oracle.part_col_piece(t, B, r) for r in rows]
            # Definition 2: the blocks of a part share no row and no column piece
            assert sorted(cols) == list(range(B))
            seen |= {(r, c) for r, c in zip(rows, cols)}
        # B consecutive parts cover every block exactly once (B*B distinct)
        assert len(seen) == B * B


def _tiny_model(I, J, K, B, nnz, seed, p=1.0, prior=oracle.PRIOR_EXPONENTIAL):
    g = np.random.default_rng(seed)
    cells = g.choice(I * J, size=nnz, replace=False)
    i = (cells // J).astype(np.int32)
    j = (cells % J).astype(np.int32)
    v = g.poisson(3.0, size=nnz).astype(np.float64) + (1.0 if p >= 2 else 0.0)
    m = oracle.Oracle(I, J, K, B, p, 1.0, prior_kind=prior)
    m.set_data(i, j, v)
    return m, i, j, v


@pytest.mark.parametrize("I,J,B", [(7, 5, 2), (9, 11, 3), (13, 13, 4), (6, 17, 5)])
def test_block_layout_brute_force(I, J, B):
    m, i, j, v = _tiny_model(I, J, 2, B, nnz=min(I * J, 40), seed=I + J + B)
    total = 0
    for r in range(B):
        for c in range(B):
            bi, bj = m.block_entries(r, c)
            rs = range(oracle.piece_start(r, I, B), oracle.piece_start(r + 1, I, B))
            cs = range(oracle.piece_start(c, J, B), oracle.piece_start(c + 1, J, B))
            want = sorted((a, b) for a, b in zip(i, j) if a in rs and b in cs)
            assert list(zip(bi.tolist(), bj.tolist())) == want
            total += len(bi)
    assert total == len(i)
    for t in range(1, 2 * B + 1):
        want = sum(len(m.block_entries(r, oracle.part_col_piece(t, B, r))[0]) for r in range(B))
        assert m.part_size(t) == want


def test_duplicate_entries_rejected():
    m = oracle.Oracle(4, 4, 2, 2, 1.0, 1.0)
    with pytest.raises(ValueError):
        m.set_data([0, 1, 0], [0, 1, 0], [1.0, 2.0, 3.0])
    with pytest.raises(ValueError):
        m.set_data([0, 4], [0, 1], [1.0, 2.0])


# ---------------------------------------------------------------------------
# Tweedie likelihood: closed forms and textbook densities
# ---------------------------------------------------------------------------

def test_beta_divergence_special_cases():
    g = np.random.default_rng(0)
    for _ in range(50):
        v, mu = g.uniform(0.1, 5.0, size=2)
        assert oracle.beta_div(v, mu, 0.0) == pytest.approx(0.5 * (v - mu) ** 2, rel=1e-13)
        assert oracle.beta_div(v, mu, 1.0) == pytest.approx(v * math.log(v / mu) - v + mu,
                                                           rel=1e-12, abs=1e-14)
        assert oracle.beta_div(v, mu, 2.0) == pytest.approx(v / mu - math.log(v / mu) - 1.0,
                                                           rel=1e-12, abs=1e-14)
        # the general formula tends to the named divergences at beta = 0, 1
        for p in (1.0, 2.0):
            for d in (1e-6, -1e-6):
                assert oracle.beta_div(v, mu, p + d) == pytest.approx(
                    oracle.beta_div(v, mu, p), rel=1e-4, abs=1e-8)
        assert oracle.beta_div(v, v, 1.5) == pytest.approx(0.0, abs=1e-12)
        assert oracle.beta_div(v, mu, 1.5) >= 0.0
    assert oracle.beta_div(0.0, 2.0, 1.0) == pytest.approx(2.0)   # 0 log 0 = 0


def _loglik_dense(V, W, H, p, phi, mu_min=1e-10):
    I, J = V.shape
    m = oracle.Oracle(I, J, W.shape[1], 1, p, phi, prior_kind=oracle.PRIOR_GAUSSIAN)
    m.set_options(mu_min=mu_min)
    ii, jj, vv = datagen.dense_to_coo(V)
    m.set_data(ii, jj, V.ravel().astype(np.float64))
    m.set_factors(W, H)
    return m.log_lik()


def _compound_poisson_gamma_logpdf(y, mu, p, phi):
    """Tweedie density for 1 < p < 2 as its definition: N ~ Poisson(lam),
    y = sum of N Gamma(alpha, scale gam) draws, lam = mu^(2-p) / (phi (2-p)),
    alpha = (2-p)/(p-1), gam = phi (p-1) mu^(p-1) (Jorgensen's compound
    Poisson-gamma); P(y = 0) = exp(-lam), otherwise the Poisson mixture of
    gamma densities, summed in log space over n = 1..300."""
    lam = mu ** (2 - p) / (phi * (2 - p))
    alpha = (2 - p) / (p - 1)
    gam = phi * (p - 1) * mu ** (p - 1)
    out = np.empty_like(y, dtype=np.float64)
    n = np.arange(1, 301, dtype=np.float64)
    for idx in np.ndindex(y.shape):
        if y[idx] == 0:
            out[idx] = -lam[idx]
            continue
        terms = (stats.poisson.logpmf(n, lam[idx]) +
                 stats.gamma.logpdf(y[idx], a=n * alpha, scale=gam[idx]))
        out[idx] = np.logaddexp.reduce(terms)
    return out


@pytest.mark.parametrize("p,phi", [(0.0, 0.7), (1.0, 1.0), (1.5, 0.6), (1.5, 1.3), (2.0, 0.5),
                                   (3.0, 0.8)])
def test_log_lik_matches_textbook_density(p, phi):
    """-(1/phi) sum d_beta differs from the exact log density by a mu-free
    constant (p = 1.5: the compound Poisson-gamma, zeros included)."""
    g = np.random.default_rng(int(p * 10))
    I, J, K = 3, 4, 2
    V = g.poisson(4.0, size=(I, J)).astype(np.float64) + 1.0
    if 1.0 < p < 2.0:
        V = np.round(g.gamma(1.5, 2.0, size=(I, J)) * 64) / 64   # exact in FP32
        V[0, 0] = V[2, 3] = 0.0             # the point mass at zero
    diffs = []
    for trial in range(2):
        W = g.uniform(0.5, 2.0, size=(I, K))
        H = g.uniform(0.5, 2.0, size=(K, J))
        mu = W @ H
        if p == 0.0:
            exact = stats.norm.logpdf(V, loc=mu, scale=math.sqrt(phi)).sum()
        elif p == 1.0:
            exact = stats.poisson.logpmf(V, mu).sum()
        elif 1.0 < p < 2.0:
            exact = _compound_poisson_gamma_logpdf(V, mu, p, phi).sum()
        elif p == 2.0:
            exact = stats.gamma.logpdf(V, a=1.0 / phi, scale=mu * phi).sum()
        else:
            lam = 1.0 / phi
            exact = stats.invgauss.logpdf(V, mu / lam, scale=lam).sum()
        diffs.append(_loglik_dense(V.astype(np.float32), W, H, p, phi) - exact)
    assert diffs[0] == pytest.approx(diffs[1], rel=1e-9, abs=1e-9)


# ---------------------------------------------------------------------------
# Gradient: finite differences of the log posterior
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("p", [0.0, 1.0, 1.5, 2.0, 3.0])
@pytest.mark.parametrize("prior", [oracle.PRIOR_EXPONENTIAL, oracle.PRIOR_GAUSSIAN])
def test_drift_is_gradient_of_log_posterior(p, prior):
    """B = 1: the drift of Eq. psgld_w / psgld_h is grad log p(W, H | V)."""
    g = np.random.default_rng(17)
    I, J, K = 4, 5, 3
    m = oracle.Oracle(I, J, K, 1, p, 0.8, prior_kind=prior, lambda_w=0.7,
                      lambda_h=1.3, sigma_w=0.9, sigma_h=1.4)
    V = g.gamma(2.0, 1.5, size=(I, J))
    ii, jj, _ = datagen.dense_to_coo(V.astype(np.float32))
    m.set_data(ii, jj, V.ravel())
    W = g.uniform(0.3, 1.5, size=(I, K))
    H = g.uniform(0.3, 1.5, size=(K, J))
    m.set_factors(W, H)
    dW, dH = m.drift(1)
    h = 1e-6
    for (M, D, which) in ((W, dW, 0), (H, dH, 1)):
        fd = np.zeros_like(M)
        for idx in np.ndindex(M.shape):
            Mp, Mm = M.copy(), M.copy()
            Mp[idx] += h
            Mm[idx] -= h
            m.set_factors(*((Mp, H) if which == 0 else (W, Mp)))
            lp = m.log_post()
            m.set_factors(*((Mm, H) if which == 0 else (W, Mm)))
            lm = m.log_post()
            fd[idx] = (lp - lm) / (2 * h)
        m.set_factors(W, H)
        np.testing.assert_allclose(D, fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())


@pytest.mark.parametrize("B,t", [(2, 1), (2, 2), (3, 2), (4, 7)])
def test_drift_on_a_part_is_scaled_part_gradient(B, t):
    """B > 1: drift = (N/|Pi_t|) grad sum_{Pi_t} log p(v|.) + grad log prior."""
    g = np.random.default_rng(B * 10 + t)
    I, J, K = 7, 9, 2
    m, i, j, v = _tiny_model(I, J, K, B, nnz=40, seed=t, p=1.0)
    W = g.uniform(0.3, 1.5, size=(I, K))
    H = g.uniform(0.3, 1.5, size=(K, J))
    m.set_factors(W, H)
    dW, dH = m.drift(t)
    S = m.scale(t)
    assert S == pytest.approx(len(i) / m.part_size(t))
    h = 1e-6
    for (M, D, which) in ((W, dW, 0), (H, dH, 1)):
        fd = np.zeros_like(M)
        for idx in np.ndindex(M.shape):
            vals = []
            for sgn in (1, -1):
                Mx = M.copy()
                Mx[idx] += sgn * h
                m.set_factors(*((Mx, H) if which == 0 else (W, Mx)))
                vals.append(S * m.log_lik_part(t) + (m.log_post() - m.log_lik()))
            fd[idx] = (vals[0] - vals[1]) / (2 * h)
        m.set_factors(W, H)
        np.testing.assert_allclose(D, fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())


# ---------------------------------------------------------------------------
# One iteration: independent dense numpy computation of the update equations
# ---------------------------------------------------------------------------

def _numpy_step(V, mask, W, H, p, phi, eps, S, prior, lam_w, lam_h, sig_w, sig_h,
                Zw, Zh, mu_min=1e-10):
    """Eq. psgld_w / psgld_h written densely: gradients masked to the part."""
    mu = W @ H
    fac = np.ones_like(mu) if p == 0 else np.maximum(mu, mu_min) ** (-p)
    E = mask * (V - mu) * fac / phi
    if prior == oracle.PRIOR_EXPONENTIAL:
        gw, gh = -lam_w * np.ones_like(W), -lam_h * np.ones_like(H)
    else:
        gw, gh = -W / sig_w ** 2, -H / sig_h ** 2
    Wn = W + eps * (S * (E @ H.T) + gw) + math.sqrt(2 * eps) * Zw
    Hn = H + eps * (S * (W.T @ E) + gh) + math.sqrt(2 * eps) * Zh
    if prior == oracle.PRIOR_EXPONENTIAL:
        Wn, Hn = np.abs(Wn), np.abs(Hn)
    return Wn, Hn


@pytest.mark.parametrize("p", [0.0, 1.0, 1.5, 2.0])
@pytest.mark.parametrize("prior", [oracle.PRIOR_EXPONENTIAL, oracle.PRIOR_GAUSSIAN])
def test_B1_part_step_is_langevin_step(p, prior):
    """With one block the part is all of V and PSGLD is a full-batch LD step."""
    I, J, K, seed, t, eps = 6, 5, 3, 99, 4, 0.05
    V, _, _ = datagen.dense_poisson(I, J, 2, seed=3)
    V = V.astype(np.float64) + 1.0
    W, H = datagen.init_factors(I, J, K, seed=1)
    W, H = W.astype(np.float64), H.astype(np.float64)
    m = oracle.Oracle(I, J, K, 1, p, 0.9, prior_kind=prior, lambda_w=0.5,
                      lambda_h=0.8, sigma_w=1.2, sigma_h=0.7)
    m.set_options(seed=seed, eps=eps)
    ii, jj, _ = datagen.dense_to_coo(V.astype(np.float32))
    m.set_data(ii, jj, V.ravel())
    m.set_factors(W, H)
    m.part_step(t)
    Wo, Ho = m.get_factors()
    Zw = oracle.noise_matrix(seed, t, 0, I, K)
    Zh = oracle.noise_matrix(seed, t, 1, J, K).T
    Wn, Hn = _numpy_step(V, np.ones_like(V), W, H, p, 0.9, eps, 1.0, prior, 0.5, 0.8,
                         1.2, 0.7, Zw, Zh)
    np.testing.assert_allclose(Wo, Wn, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(Ho, Hn, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("B,t", [(2, 1), (3, 5), (4, 3)])
def test_part_step_matches_masked_dense_update(B, t):
    """B > 1 on sparse data: only the part's entries drive the gradient."""
    I, J, K, seed, eps, p = 11, 10, 3, 5, 0.02, 1.0
    m, i, j, v = _tiny_model(I, J, K, B, nnz=60, seed=B + t, p=p)
    m.set_options(seed=seed, eps=eps)
    W, H = datagen.init_factors(I, J, K, seed=2)
    W, H = W.astype(np.float64), H.astype(np.float64)
    m.set_factors(W, H)
    m.part_step(t)
    Wo, Ho = m.get_factors()
    # part mask from the definitions, written independently of the oracle
    s = (t - 1) % B
    rp = np.array([max(r for r in range(B) if (r * I) // B <= x) for x in range(I)])
    cp = np.array([max(c for c in range(B) if (c * J) // B <= y) for y in range(J)])
    V = np.zeros((I, J))
    obs = np.zeros((I, J))
    V[i, j] = v
    obs[i, j] = 1.0
    part = (cp[None, :] == (rp[:, None] + s) % B).astype(float)
    mask = obs * part
    S = len(i) / mask.sum()
    Zw = oracle.noise_matrix(seed, t, 0, I, K)
    Zh = oracle.noise_matrix(seed, t, 1, J, K).T
    Wn, Hn = _numpy_step(V, mask, W, H, p, 1.0, eps, S, oracle.PRIOR_EXPONENTIAL, 1.0,
                         1.0, 1.0, 1.0, Zw, Zh)
    np.testing.assert_allclose(Wo, Wn, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(Ho, Hn, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------------------
# mu below mu_min: the clamp of the Tweedie factor (reading of Sec. 4 for
# mu -> 0, where (v - mu) mu^(-p) has no finite value)
# ---------------------------------------------------------------------------

def _clamp_model(p, phi, mu_min, prior=oracle.PRIOR_EXPONENTIAL):
    """Dense 5 x 6 data, K = 3, one block.  Row 1 of W is zero (mu = 0 on
    the whole row) and row 3 is tiny (0 < mu < mu_min); the other rows have
    mu well above mu_min.  For 1 < p < 2 two entries are zero (the point
    mass of the compound Poisson law)."""
    g = np.random.default_rng(int(10 * p) + 7)
    I, J, K = 5, 6, 3
    V = np.round(g.gamma(2.0, 1.5, size=(I, J)) * 64) / 64 + (0.25 if p >= 2 else 0.0)
    if 1.0 < p < 2.0:
        V[1, 2] = V[3, 0] = 0.0
    W = g.uniform(0.5, 1.5, size=(I, K))
    W[1] = 0.0
    W[3] = 1e-3
    H = g.uniform(0.5, 1.5, size=(K, J))
    m = oracle.Oracle(I, J, K, 1, p, phi, prior_kind=prior, lambda_w=0.7, lambda_h=1.3,
                      sigma_w=0.9, sigma_h=1.4)
    m.set_options(mu_min=mu_min)
    ii, jj, _ = datagen.dense_to_coo(V.astype(np.float32))
    m.set_data(ii, jj, V.ravel())
    m.set_factors(W, H)
    return m, V, W, H


@pytest.mark.parametrize("p", [1.0, 1.5, 2.0, 3.0])
def test_mu_min_clamp_closed_form_on_zero_and_tiny_rows(p):
    """With mu_min = 1e-2: a zero row of W has mu = 0 on every entry, so its
    drift is, in closed form, mu_min^(-p) / phi * (sum_j v_ij h_j) - lambda_w
    (the clamp enters the power only; the residual keeps the raw mu = 0),
    and it adds nothing to H's drift (its w is zero).  A tiny row (0 < mu <
    mu_min) has drift mu_min^(-p) / phi * sum_j (v_ij - mu_ij) h_j -
    lambda_w.  Rows with mu > mu_min keep the unclamped Tweedie gradient,
    checked against the textbook derivative of each density (Poisson
    v/mu - 1, gamma (v - mu)/(phi mu^2), ...) written out per p."""
    phi, mu_min, lam_w, lam_h = 0.8, 1e-2, 0.7, 1.3
    m, V, W, H = _clamp_model(p, phi, mu_min)
    dW, dH = m.drift(1)
    mu = W @ H
    assert mu[1].max() == 0.0 and 0.0 < mu[3].min() and mu[3].max() < mu_min
    assert np.delete(mu, [1, 3], axis=0).min() > 10 * mu_min
    # zero row: closed form, no max() anywhere
    np.testing.assert_allclose(dW[1], mu_min ** (-p) / phi * (V[1] @ H.T) - lam_w, rtol=1e-12)
    # tiny row: the power clamped, the residual raw
    np.testing.assert_allclose(dW[3], mu_min ** (-p) / phi * ((V[3] - mu[3]) @ H.T) - lam_w,
                               rtol=1e-12)
    # the other rows, and H (row 1 adds e * 0 to it; row 3's clamped e enters
    # H's drift times its tiny w)
    with np.errstate(divide="ignore", invalid="ignore"):    # rows 1, 3 are replaced below
        if p == 1.0:
            E = (V / mu - 1.0) / phi             # d/dmu of the Poisson log-pmf, over phi
        elif p == 2.0:
            E = (V - mu) / (phi * mu ** 2)       # gamma with mean mu, shape 1/phi
        else:
            E = (V - mu) * mu ** (-p) / phi      # Tweedie mean-derivative for p = 1.5, 3
    E[1] = V[1] * mu_min ** (-p) / phi
    E[3] = (V[3] - mu[3]) * mu_min ** (-p) / phi
    rows = [0, 2, 4]
    np.testing.assert_allclose(dW[rows], (E @ H.T)[rows] - lam_w, rtol=1e-12)
    np.testing.assert_allclose(dH, W.T @ E - lam_h, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("p", [1.0, 2.0])
def test_mu_min_clamp_is_inactive_above_mu_min(p):
    """Factors whose mu all exceed 1e-2: the drift and the log-likelihood
    with mu_min = 1e-2 equal those with the default 1e-10, bit for bit."""
    m1, V, W, H = _clamp_model(p, 0.8, 1e-2)
    W = W.copy()
    W[1] = W[3] = 0.4
    m1.set_factors(W, H)
    m2 = oracle.Oracle(5, 6, 3, 1, p, 0.8, prior_kind=oracle.PRIOR_EXPONENTIAL, lambda_w=0.7,
                       lambda_h=1.3)
    m2.set_options(mu_min=1e-10)
    ii, jj, _ = datagen.dense_to_coo(V.astype(np.float32))
    m2.set_data(ii, jj, V.ravel())
    m2.set_factors(W, H)
    assert (W @ H).min() > 1e-2
    a, b = m1.drift(1), m2.drift(1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert m1.log_lik() == m2.log_lik()


@pytest.mark.parametrize("p,phi", [(1.0, 1.0), (1.5, 0.7), (2.0, 0.5), (3.0, 0.8)])
def test_mu_min_clamp_in_log_lik_is_the_density_at_mu_min(p, phi):
    """log_lik clamps mu itself: an entry with mu < mu_min is scored as the
    density at mu_min.  So log_lik - sum log f(v; max(mu, mu_min)) is the
    same mu-free constant for factors with and without clamped entries
    (f: scipy's Poisson, gamma and inverse-Gaussian densities, and the
    compound Poisson-gamma for p = 1.5)."""
    mu_min = 1e-2
    m, V, W, H = _clamp_model(p, phi, mu_min)

    def density(mu):
        if p == 1.0:
            return stats.poisson.logpmf(np.round(V), mu).sum()
        if p == 2.0:
            return stats.gamma.logpdf(V, a=1.0 / phi, scale=mu * phi).sum()
        if p == 3.0:
            lam = 1.0 / phi
            return stats.invgauss.logpdf(V, mu / lam, scale=lam).sum()
        return _compound_poisson_gamma_logpdf(V, mu, p, phi).sum()

    if p == 1.0:
        V = np.round(V)      # counts for the Poisson pmf
        ii, jj, _ = datagen.dense_to_coo(V.astype(np.float32))
        m.set_data(ii, jj, V.ravel())
    # three factor sets: rows 1 (zero) and 3 (tiny) clamped; row 1 only;
    # nothing clamped
    Wb = W.copy()
    Wb[3] = 0.6
    Wc = Wb.copy()
    Wc[1] = 0.6
    diffs = []
    for Wt in (W, Wb, Wc):
        m.set_factors(Wt, H)
        diffs.append(m.log_lik() - density(np.maximum(Wt @ H, mu_min)))
    assert np.all(np.isfinite(diffs))
    assert diffs[0] == pytest.approx(diffs[2], rel=1e-9, abs=1e-9)
    assert diffs[1] == pytest.approx(diffs[2], rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("p", [1.0, 1.5, 2.0, 3.0])
def test_mu_min_clamp_in_langevin_step_matches_numpy(p):
    """The whole B = 1 step with a zero and a tiny row against the dense
    numpy step (which clamps with np.maximum on its own)."""
    phi, mu_min, eps, seed, t = 0.8, 1e-2, 1e-4, 5, 3
    m, V, W, H = _clamp_model(p, phi, mu_min)
    m.set_options(seed=seed, eps=eps, mu_min=mu_min)
    m.set_factors(W, H)
    m.part_step(t)
    Wo, Ho = m.get_factors()
    Zw = oracle.noise_matrix(seed, t, 0, 5, 3)
    Zh = oracle.noise_matrix(seed, t, 1, 6, 3).T
    Wn, Hn = _numpy_step(V, np.ones_like(V), W, H, p, phi, eps, 1.0, oracle.PRIOR_EXPONENTIAL,
                         0.7, 1.3, 0.9, 1.4, Zw, Zh, mu_min=mu_min)
    np.testing.assert_allclose(Wo, Wn, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(Ho, Hn, rtol=1e-12, atol=1e-14)


def test_mirroring_keeps_factors_non_negative():
    """Algorithm 1's mirroring: with a large step many raw updates go negative."""
    I, J, K = 8, 8, 4
    m, *_ = _tiny_model(I, J, K, 2, nnz=30, seed=3, p=1.0)
    m.set_options(seed=1, eps=0.5)
    W, H = datagen.init_factors(I, J, K, seed=3, scale=0.1)
    m.set_factors(W, H)
    for t in range(1, 41):
        m.part_step(t)
        Wo, Ho = m.get_factors()
        assert Wo.min() >= 0.0 and Ho.min() >= 0.0
    # the Gaussian-prior model is not mirrored and does go negative
    g, *_ = _tiny_model(I, J, K, 2, nnz=30, seed=3, p=0.0, prior=oracle.PRIOR_GAUSSIAN)
    g.set_options(seed=1, eps=0.5)
    g.set_factors(W, H)
    g.part_step(1)
    assert min(x.min() for x in g.get_factors()) < 0.0


def test_step_size_schedule():
    m = oracle.Oracle(4, 4, 2, 2, 1.0, 1.0)
    m.set_options(eps_mode=oracle.EPS_POLY, eps_a=0.01, eps_b=0.51)
    assert m.eps(1) == pytest.approx(0.01 ** 0.51, rel=1e-14)
    assert m.eps(100) == pytest.approx(1e-4 ** 0.51, rel=1e-14)
    # Eq. eps: b in (0.5, 1] makes sum eps diverge and sum eps^2 converge
    m.set_options(eps_mode=oracle.EPS_FIXED, eps=3e-3)
    assert m.eps(12345) == 3e-3


def test_freeze_and_sweep_boundary():
    I, J, K = 6, 6, 2
    m, *_ = _tiny_model(I, J, K, 3, nnz=20, seed=1, p=1.0)
    W, H = datagen.init_factors(I, J, K, seed=3)
    m.set_factors(W, H)
    m.set_options(seed=2, eps=0.01, freeze_H=True)
    m.sweep(2)
    Wo, Ho = m.get_factors()
    assert np.array_equal(Ho, H.astype(np.float64))
    assert not np.array_equal(Wo, W.astype(np.float64))
    assert m.iterations_done == 6
    m.part_step(7)
    with pytest.raises(RuntimeError):
        m.sweep(1)


# ---------------------------------------------------------------------------
# Posterior sums, RMSE
# ---------------------------------------------------------------------------

def test_posterior_moments_match_recorded_samples():
    I, J, K, B = 5, 6, 2, 3
    m, i, j, v = _tiny_model(I, J, K, B, nnz=25, seed=4, p=1.0)
    W, H = datagen.init_factors(I, J, K, seed=4)
    m.set_factors(W, H)
    m.set_options(seed=8, eps=0.01, burn_in=3)
    samples = []
    for s in range(12):
        m.sweep(1)
        if s >= 3:
            samples.append(m.get_factors())
    Wm, Wv, Hm, Hv, n = m.posterior()
    assert n == 9
    Ws = np.stack([a for a, _ in samples])
    Hs = np.stack([b for _, b in samples])
    np.testing.assert_allclose(Wm, Ws.mean(0), rtol=1e-12)
    np.testing.assert_allclose(Hm, Hs.mean(0), rtol=1e-12)
    np.testing.assert_allclose(Wv, Ws.var(0), rtol=1e-6, atol=1e-14)
    np.testing.assert_allclose(Hv, Hs.var(0), rtol=1e-6, atol=1e-14)
    # RMSE on observed entries, current factors and posterior means
    Wc, Hc = m.get_factors()
    r = np.sqrt(np.mean((v - (Wc @ Hc)[i, j]) ** 2))
    assert m.rmse(False) == pytest.approx(r, rel=1e-12)
    r = np.sqrt(np.mean((v - (Wm @ Hm)[i, j]) ** 2))
    assert m.rmse(True) == pytest.approx(r, rel=1e-12)


# ---------------------------------------------------------------------------
# Stationary distribution: closed-form Gaussian posterior (Theorem 1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prior", [oracle.PRIOR_EXPONENTIAL, oracle.PRIOR_GAUSSIAN])
def test_empty_part_moves_by_prior_and_noise_only(prior):
    """Entries only in block (0, 0) of a B = 3 grid: parts 1 and 2 hold no
    entry, so S = N / |Pi| is read as 0 there and the drift is the prior
    gradient alone (-lam, or -x / sigma^2); part 0's drift has the
    likelihood term scaled by N / |Pi_0| = 1."""
    I, J, K, B = 6, 9, 3, 3
    g = np.random.default_rng(3)
    ii, jj = np.meshgrid(np.arange(2), np.arange(3), indexing="ij")
    ii, jj = ii.ravel().astype(np.int32), jj.ravel().astype(np.int32)
    vv = g.uniform(0.5, 2.0, size=ii.size)
    m = oracle.Oracle(I, J, K, B, 1.0, 1.0, prior_kind=prior, lambda_w=0.8, lambda_h=1.2,
                      sigma_w=0.9, sigma_h=1.1)
    m.set_data(ii, jj, vv)
    W = g.uniform(0.2, 1.0, size=(I, K))
    H = g.uniform(0.2, 1.0, size=(K, J))
    m.set_factors(W, H)
    if prior == oracle.PRIOR_EXPONENTIAL:
        pW, pH = np.full_like(W, -0.8), np.full_like(H, -1.2)
    else:
        pW, pH = -W / 0.9 ** 2, -H / 1.1 ** 2
    assert [m.part_size(t) for t in (1, 2, 3)] == [ii.size, 0, 0]
    for t in (2, 3):
        assert m.scale(t) == 0.0
        dW, dH = m.drift(t)
        np.testing.assert_allclose(dW, pW, rtol=0, atol=1e-15)
        np.testing.assert_allclose(dH, pH, rtol=0, atol=1e-15)
    # part 0: the Poisson likelihood gradient of block (0, 0), S = 1
    assert m.scale(1) == 1.0
    dW, dH = m.drift(1)
    mu = W @ H
    E = np.zeros((I, J))
    E[ii, jj] = (vv - mu[ii, jj]) / mu[ii, jj]
    np.testing.assert_allclose(dW, E @ H.T + pW, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(dH, W.T @ E + pH, rtol=1e-12, atol=1e-12)


def test_mirrored_chain_samples_the_truncated_posterior():
    """p = 0, exponential prior (rate lam) with mirroring, K = 1, H fixed at
    h: each w_i >= 0 has the posterior proportional to
    exp(-(v_i - w h)^2 / (2 phi) - lam w) on [0, inf), a normal with mean
    (v_i h - lam phi) / h^2 and variance phi / h^2 truncated to w >= 0
    (scipy's truncnorm).  The mirrored Langevin chain (Sec. 3.2) must match
    its first two moments within 3 standard errors (batch means).  The rows
    are chosen so that truncation matters: most untruncated means are
    negative, so dropping the mirror, the prior or its sign fails."""
    I, J, K, B = 6, 1, 1, 1
    phi, lam, h = 1.0, 0.7, 1.0
    V = np.array([[0.2], [0.6], [1.0], [-0.3], [1.5], [0.0]])
    m = oracle.Oracle(I, J, K, B, 0.0, phi, prior_kind=oracle.PRIOR_EXPONENTIAL, lambda_w=lam,
                      lambda_h=1.0)
    ii, jj, _ = datagen.dense_to_coo(V.astype(np.float32))
    m.set_data(ii, jj, V.ravel())
    m.set_factors(np.full((I, K), 0.5), np.full((K, J), h))
    m.set_options(seed=5, eps=5e-3, freeze_H=True, burn_in=2000)
    m.sweep(2000)
    n_batches, per_batch = 40, 10000
    prev_m = np.zeros((I, K)); prev_s = np.zeros((I, K)); prev_n = 0
    bm, bs = [], []
    for b in range(n_batches):
        m.sweep(per_batch)
        Wm, Wv, _, _, n = m.posterior()
        tot, tot2 = Wm * n, (Wv + Wm ** 2) * n
        bm.append((tot - prev_m) / (n - prev_n))
        bs.append((tot2 - prev_s) / (n - prev_n))
        prev_m, prev_s, prev_n = tot, tot2, n
    bm, bs = np.array(bm)[:, :, 0], np.array(bs)[:, :, 0]
    se_mean = bm.std(0, ddof=1) / math.sqrt(n_batches)
    se_second = bs.std(0, ddof=1) / math.sqrt(n_batches)
    loc = (V[:, 0] * h - lam * phi) / h ** 2
    scale = math.sqrt(phi) / h
    for i in range(I):
        tn = stats.truncnorm((0.0 - loc[i]) / scale, np.inf, loc=loc[i], scale=scale)
        want_mean, want_second = tn.mean(), tn.var() + tn.mean() ** 2
        assert abs(bm[:, i].mean() - want_mean) < 3 * se_mean[i], (i, bm[:, i].mean(), want_mean)
        assert abs(bs[:, i].mean() - want_second) < 3 * se_second[i], \
            (i, bs[:, i].mean(), want_second)
        assert abs(want_mean - loc[i]) > 10 * se_mean[i] or loc[i] > 0   # truncation matters


def test_chain_samples_closed_form_gaussian_posterior():
    """p = 0, Gaussian prior, H held fixed: each row w_i of W has the posterior
    N(Sigma_i H_i v_i / phi, Sigma_i), Sigma_i = (H_i H_i^T / phi + I / sigma^2)^-1.
    PSGLD's sample mean and variance must agree within 3 standard errors
    (batch means), with a step small enough that the O(eps) bias is below it."""
    I, J, K, B = 4, 8, 2, 2
    phi, sig = 1.5, 0.8
    g = np.random.default_rng(11)
    H = g.normal(0.0, 0.6, size=(K, J))
    V = g.normal(1.0, 1.0, size=(I, J))
    m = oracle.Oracle(I, J, K, B, 0.0, phi, prior_kind=oracle.PRIOR_GAUSSIAN,
                      sigma_w=sig, sigma_h=1.0)
    ii, jj, _ = datagen.dense_to_coo(V.astype(np.float32))
    m.set_data(ii, jj, V.ravel())
    m.set_factors(np.zeros((I, K)), H)
    eps = 2e-3
    m.set_options(seed=21, eps=eps, freeze_H=True, burn_in=500)
    n_batches, per_batch = 40, 2000
    m.sweep(500)
    prev_m = np.zeros((I, K)); prev_s = np.zeros((I, K)); prev_n = 0
    bm, bs = [], []
    for b in range(n_batches):
        m.sweep(per_batch)
        Wm, Wv, _, _, n = m.posterior()
        tot = Wm * n
        tot2 = (Wv + Wm ** 2) * n
        bm.append((tot - prev_m) / (n - prev_n))
        bs.append((tot2 - prev_s) / (n - prev_n))
        prev_m, prev_s, prev_n = tot, tot2, n
    bm, bs = np.array(bm), np.array(bs)
    mean = bm.mean(0)
    second = bs.mean(0)
    se_mean = bm.std(0, ddof=1) / math.sqrt(n_batches)
    se_second = bs.std(0, ddof=1) / math.sqrt(n_batches)
    for i in range(I):
        prec = H @ H.T / phi + np.eye(K) / sig ** 2
        Sig = np.linalg.inv(prec)
        mu = Sig @ (H @ V[i] / phi)
        want_second = np.diag(Sig) + mu ** 2
        assert np.all(np.abs(mean[i] - mu) < 3 * se_mean[i] + 1e-12), (mean[i], mu, se_mean[i])
        assert np.all(np.abs(second[i] - want_second) < 3 * se_second[i]), \
            (second[i], want_second, se_second[i])


def test_results_do_not_depend_on_thread_count():
    """The blocks of a part write disjoint rows, so OpenMP over blocks gives
    bit-identical chains for any number of threads (the CPU baseline times
    both)."""
    I, J, K, B = 90, 70, 6, 5
    i, j, v = datagen.sparse_ratings(I, J, 2500, 3, seed=11)
    W0, H0 = datagen.init_factors(I, J, K, seed=11, scale=0.3, nonneg=False)
    out = []
    before = oracle.set_threads(0)
    for threads in (1, 4):
        oracle.set_threads(threads)
        m = oracle.Oracle(I, J, K, B, 0.0, 1.0, prior_kind=oracle.PRIOR_GAUSSIAN)
        m.set_options(seed=5, eps=1e-3)
        m.set_data(i, j, v.astype(np.float64))
        m.set_factors(W0.astype(np.float64), H0.astype(np.float64))
        m.sweep(3)
        out.append(m.get_factors())
    oracle.set_threads(before)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def _uneven_parts_model(seed=3):
    """B = 4 with very unequal part sizes: a dense diagonal band adds entries
    to the blocks of part 0 only."""
    I, J, K, B = 80, 80, 3, 4
    i, j, v = datagen.sparse_ratings(I, J, 800, 3, seed=seed)
    pairs = set(zip(i.tolist(), j.tolist()))
    extra = [(a, b) for a in range(I) for b in range(J)
             if oracle.piece_of(a, I, B) == oracle.piece_of(b, J, B) and (a, b) not in pairs][:1200]
    i = np.concatenate([i, np.array([a for a, _ in extra], np.int32)])
    j = np.concatenate([j, np.array([b for _, b in extra], np.int32)])
    v = np.concatenate([v, np.full(len(extra), 3.0, np.float32)])
    m = oracle.Oracle(I, J, K, B, 0.0, 1.0, prior_kind=oracle.PRIOR_GAUSSIAN)
    m.set_options(seed=seed, eps=1e-3)
    m.set_data(i, j, v.astype(np.float64))
    return m, B


def test_size_proportional_parts_follow_part_sizes():
    """Condition C2 (Sec. 3.1): part s is drawn with probability |Pi_s| / N,
    independently at every iteration.  Pinned by a chi-square test of the
    draw frequencies against the part sizes counted by brute force, with
    parts of very different sizes; the cyclic mode keeps (t-1) mod B."""
    m, B = _uneven_parts_model()
    sizes = np.array([m.part_size(s + 1) for s in range(B)], dtype=np.float64)   # cyclic: t = s+1
    assert [m.part_index(t) for t in range(1, 9)] == [(t - 1) % B for t in range(1, 9)]
    m.set_part_mode(1)
    T = 40000
    draws = np.array([m.part_index(t) for t in range(1, T + 1)])
    counts = np.bincount(draws, minlength=B)
    expected = T * sizes / sizes.sum()
    assert sizes.max() > 2 * sizes.min()           # the parts really differ
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert stats.chi2.sf(chi2, B - 1) > 1e-4, (counts, expected)
    # deterministic in (seed, t); a different seed gives a different stream
    assert [m.part_index(t) for t in (5, 77, 1 << 33)] == [m.part_index(t) for t in (5, 77, 1 << 33)]
    m2, _ = _uneven_parts_model()
    m2.set_options(seed=4, eps=1e-3)
    m2.set_part_mode(1)
    assert [m2.part_index(t) for t in range(1, 200)] != draws[:199].tolist()


def test_size_proportional_parts_make_the_scaled_gradient_unbiased():
    """Under C2 the expected scaled part gradient is the full-data gradient:
    sum_s (|Pi_s| / N) * (N / |Pi_s|) grad_s = sum_s grad_s.  Checked with the
    oracle's drifts of each part (prior removed) against a B = 1 drift on the
    same data."""
    m, B = _uneven_parts_model()
    I, J, K = 80, 80, 3
    W0, H0 = datagen.init_factors(I, J, K, seed=9, scale=0.3, nonneg=False)
    m.set_factors(W0.astype(np.float64), H0.astype(np.float64))
    N = sum(m.part_size(s + 1) for s in range(B))
    prior_W = -W0.astype(np.float64)               # Gaussian prior sigma = 1
    prior_H = -H0.astype(np.float64)
    EW = np.zeros((I, K)); EH = np.zeros((K, J))
    for s in range(B):
        dW, dH = m.drift(s + 1)                    # cyclic mode: part s at t = s + 1
        p_s = m.part_size(s + 1) / N
        EW += p_s * (dW - prior_W)
        EH += p_s * (dH - prior_H)
    full = oracle.Oracle(I, J, K, 1, 0.0, 1.0, prior_kind=oracle.PRIOR_GAUSSIAN)
    full.set_options(seed=3, eps=1e-3)
    mm, _ = _uneven_parts_model()
    # the same entries: read them back block by block from the B = 4 model
    ii, jj = [], []
    for r in range(B):
        for c in range(B):
            bi, bj = mm.block_entries(r, c)
            ii.append(bi); jj.append(bj)
    ii = np.concatenate(ii); jj = np.concatenate(jj)
    i0, j0, v0 = datagen.sparse_ratings(I, J, 800, 3, seed=3)
    lut = {(a, b): x for a, b, x in zip(i0.tolist(), j0.tolist(), v0.tolist())}
    vv = np.array([lut.get((a, b), 3.0) for a, b in zip(ii.tolist(), jj.tolist())])
    full.set_data(ii.astype(np.int32), jj.astype(np.int32), vv)
    full.set_factors(W0.astype(np.float64), H0.astype(np.float64))
    fW, fH = full.drift(1)
    np.testing.assert_allclose(EW, fW - prior_W, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(EH, fH - prior_H, rtol=1e-10, atol=1e-10)
