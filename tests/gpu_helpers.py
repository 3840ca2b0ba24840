"""Shared set-up of the GPU parity tests: one CUDA chain and one oracle chain
started from the same seeded inputs."""
import numpy as np

import oracle
from paper_1506_01418_gb300 import datagen
from paper_1506_01418_gb300 import psgld as P

# One FP32 part-step against the FP64 oracle, from identical factors and with
# the identical Philox stream (step_errors): element by element, |gpu -
# oracle| <= 1e-5 x max(|oracle|, |x0|, sqrt(2 eps) |z|, eps D_abs), the
# largest magnitude among the terms the GPU adds in FP32 to form x0 + eps
# (S sum_j e_j h_j + prior) + sqrt(2 eps) z, with D_abs = S sum_j |e_j| |h_j|
# + |prior gradient| the absolute sum of the drift's terms: every rounding
# error of the step (the FP32 sums of the drift included) is a few ulps of
# one of those magnitudes, times the number of terms summed.  No floor taken
# from the matrix as a whole.
STEP_RTOL = 1e-5

U_BF16 = 2.0 ** -8
U_FP32 = 2.0 ** -24
U_E4M3 = 2.0 ** -4          # 3 mantissa bits
ETA_E4M3 = 2.0 ** -10       # half the subnormal spacing, in units of the tile scale


def recovered_drift(x_new, x0, z, D_or, eps, mirror):
    """The drift a GPU step applied: x_new = m(x0 + eps drift + sqrt(2 eps) z),
    m = |.| or identity.  Returns (drift, mask of elements judged, recovery
    error): elements the oracle's step leaves near zero are not judged when
    the mirror applies (their sign is undetermined)."""
    sd = np.sqrt(2 * eps)
    y_or = x0 + eps * D_or + sd * z
    mask = np.abs(y_or) > 0.02 if mirror else np.ones_like(y_or, dtype=bool)
    sgn = np.sign(y_or) if mirror else 1.0
    D = (sgn * x_new - x0 - sd * z) / eps
    rec = (6 * U_FP32 * (np.abs(x0) + np.abs(y_or) + eps * np.abs(D_or))
           + sd * 3e-6 * (1 + np.abs(z))) / eps + 4 * U_FP32 * np.abs(D_or)
    return D, mask, rec


def step_errors(x_gpu, x_or, x0, z, sd, eps_dabs=None):
    """Errors of one part-step of one factor (arrays of one layout), from the
    same FP32 x0 and the same Philox normals z on both sides.

    elem: max |gpu - or| / max(|or|, |x0|, sd |z|, eps_dabs) (see STEP_RTOL;
        eps_dabs = eps D_abs, or None when the drift is small beside x0);
    inc: max |dx_gpu - dx_or| / max |dx_or|, dx = new - x0: the error of the
        increment (eps drift + noise, mirrored) on the increment's own scale;
    inc_bound: the bound inc is held to -- 1e-5 for the arithmetic of the
        increment (FP32 sums of the drift, the FP32 Box-Muller of the
        normals; on the scale of eps D_abs where that exceeds the largest
        increment, i.e. where the drift's terms cancel) plus the rounding of
        the stored FP32 result, 2^-24 of the largest |x| twice (the step's
        FMA chain and the final store), on the increment's scale."""
    x_gpu = np.asarray(x_gpu, dtype=np.float64)
    x_or = np.asarray(x_or, dtype=np.float64)
    x0 = np.asarray(x0, dtype=np.float64)
    if x_or.size == 0:
        return 0.0, 0.0, STEP_RTOL
    scale = np.maximum(np.maximum(np.abs(x_or), np.abs(x0)), sd * np.abs(z)) + 1e-300
    if eps_dabs is not None:
        scale = np.maximum(scale, eps_dabs)
    err = np.abs(x_gpu - x_or)
    elem = float(np.max(err / scale))
    dmax = float(np.max(np.abs(x_or - x0))) + 1e-300
    inc = float(np.max(err)) / dmax
    terms = 1.0 if eps_dabs is None else max(1.0, float(np.max(eps_dabs)) / dmax)
    inc_bound = STEP_RTOL * terms + 2 * U_FP32 * float(np.max(np.abs(x_or))) / dmax
    return elem, inc, inc_bound


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if b.size == 0:
        return 0.0
    floor = 1e-2 * np.sqrt(np.mean(b * b)) + 1e-30
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


class Pair:
    """A GPU chain (through the C ABI) and an oracle chain on the same inputs."""

    def __init__(self, I, J, K, B, p, phi, i, j, v, W0, H0, prior_kind=0, lam=(1.0, 1.0),
                 sig=(1.0, 1.0), seed=1, eps=1e-4, use_graphs=1, V=None, **opts):
        import torch
        self.torch = torch
        self.I, self.J, self.K, self.B = I, J, K, B
        self.seed = seed
        self.p, self.phi, self.prior_kind = p, phi, prior_kind
        self.lam, self.sig = lam, sig
        self.mu_min = opts.get("mu_min", 1e-10)
        self.i = np.asarray(i, dtype=np.int64)
        self.j = np.asarray(j, dtype=np.int64)
        self.v = np.asarray(v, dtype=np.float64)
        self.gpu = P.PSGLD(I, J, K, B, p, phi, prior_kind=prior_kind, lambda_w=lam[0],
                           lambda_h=lam[1], sigma_w=sig[0], sigma_h=sig[1], seed=seed,
                           eps=eps, use_graphs=use_graphs, **opts)
        dev = "cuda"
        if V is not None:    # dense I x J array; (i, j, v) lists the same entries
            self.gpu.set_data_dense(torch.as_tensor(np.ascontiguousarray(V, dtype=np.float32),
                                                    device=dev))
        else:
            self.gpu.set_data_coo(torch.as_tensor(i, dtype=torch.int32, device=dev),
                                  torch.as_tensor(j, dtype=torch.int32, device=dev),
                                  torch.as_tensor(v, dtype=torch.float32, device=dev))
        self.orc = oracle.Oracle(I, J, K, B, p, phi, prior_kind=prior_kind, lambda_w=lam[0],
                                 lambda_h=lam[1], sigma_w=sig[0], sigma_h=sig[1])
        oopts = {k: v for k, v in opts.items() if k in ("eps_mode", "eps_a", "eps_b",
                                                         "scale_mode", "mu_min", "freeze_W",
                                                         "freeze_H")}
        if "burn_in_sweeps" in opts:
            oopts["burn_in"] = opts["burn_in_sweeps"]
        self.orc.set_options(seed=seed, eps=eps, **oopts)
        self.orc.set_data(np.asarray(i), np.asarray(j), np.asarray(v, dtype=np.float64))
        self.set_factors(W0, H0)

    def set_factors(self, W, H):
        """W: I x K, H: K x J (float32 values; the oracle gets them exactly)."""
        torch = self.torch
        W = np.ascontiguousarray(W, dtype=np.float32)
        H = np.ascontiguousarray(H, dtype=np.float32)
        self.gpu.set_factors(torch.from_numpy(W).cuda(), torch.from_numpy(H.T.copy()).cuda())
        self.orc.set_factors(W.astype(np.float64), H.astype(np.float64))

    def gpu_factors(self):
        W, Ht = self.gpu.get_factors()
        self.torch.cuda.synchronize()
        return W.cpu().numpy(), Ht.cpu().numpy().T

    def step_both(self, t):
        self.gpu.part_step(t)
        self.orc.part_step(t)
        Wg, Hg = self.gpu_factors()
        Wo, Ho = self.orc.get_factors()
        return (Wg, Hg), (Wo, Ho)

    def abs_drift(self, t, W, H):
        """D_abs of iteration t at factors W (I x K), H (K x J): S sum_j |e_ij|
        |h_j| over the part's entries plus |prior gradient|, for W and H,
        written here from the definitions (pieces floor(r n / B), part s =
        the oracle's part index at t)."""
        B, p = self.B, self.p
        rs = np.array([(r * self.I) // B for r in range(B + 1)])
        cs = np.array([(r * self.J) // B for r in range(B + 1)])
        rp = np.searchsorted(rs, self.i, side="right") - 1
        cp = np.searchsorted(cs, self.j, side="right") - 1
        m = ((cp - rp) % B) == self.orc.part_index(t)
        i, j, v = self.i[m], self.j[m], self.v[m]
        Ht = H.T
        mu = np.einsum("nk,nk->n", W[i], Ht[j])
        fac = 1.0 if p == 0 else np.maximum(mu, self.mu_min) ** (-p)
        ea = np.abs(v - mu) * fac / self.phi
        GW = np.zeros_like(W)
        GH = np.zeros_like(Ht)
        np.add.at(GW, i, ea[:, None] * np.abs(Ht[j]))
        np.add.at(GH, j, ea[:, None] * np.abs(W[i]))
        S = self.orc.scale(t)
        if self.prior_kind == 0:
            pw, ph = self.lam[0], self.lam[1]
        else:
            pw, ph = np.abs(W) / self.sig[0] ** 2, np.abs(H) / self.sig[1] ** 2
        return S * GW + pw, (S * GH).T + ph

    def step_and_check(self, t, W0=None, H0=None, part=None):
        """One part-step on both sides from the current (or the given)
        factors; asserts step_errors for W and H and returns the GPU's new
        factors.  part: the part drawn at t (size-proportional mode), only
        for the message."""
        if W0 is not None:
            self.set_factors(W0, H0)
        W0, H0 = self.orc.get_factors()
        eps = self.orc.eps(t)
        sd = float(np.sqrt(2.0 * eps))
        aW, aH = self.abs_drift(t, W0, H0)
        (Wg, Hg), (Wo, Ho) = self.step_both(t)
        zW = oracle.noise_matrix(self.seed, t, 0, self.I, self.K)
        zH = oracle.noise_matrix(self.seed, t, 1, self.J, self.K).T
        for xg, xo, x0, z, ad, what in ((Wg, Wo, W0, zW, aW, "W"), (Hg, Ho, H0, zH, aH, "H")):
            elem, inc, inc_b = step_errors(xg, xo, x0, z, sd, eps * ad)
            assert np.all(np.isfinite(xg)), (t, what, "non-finite")
            assert elem <= STEP_RTOL, (t, part, what, "element", elem)
            assert inc <= inc_b, (t, part, what, "increment", inc, inc_b)
        return Wg, Hg

    def sync_oracle_to_gpu(self):
        Wg, Hg = self.gpu_factors()
        self.orc.set_factors(Wg.astype(np.float64), Hg.astype(np.float64))


def sparse_case(I, J, nnz, K_true, seed, zipf=1.1):
    return datagen.sparse_ratings(I, J, nnz, K_true, seed, zipf_row=zipf, zipf_col=zipf)


def dense_case(I, J, K_true, seed, kind="poisson"):
    if kind == "poisson":
        V, _, _ = datagen.dense_poisson(I, J, K_true, seed)
    else:
        V, _, _ = datagen.dense_gamma(I, J, K_true, seed)
    return datagen.dense_to_coo(V)


def tile_scales(X, axis):
    """Largest |x| / 448 of each 128-wide tile of X along `axis` (rows of a
    W block: axis 0; columns of an H block: axis 1), broadcast back."""
    n = X.shape[axis]
    out = np.zeros(n)
    for a in range(0, n, 128):
        sl = X[a:a + 128] if axis == 0 else X[:, a:a + 128]
        m = np.abs(sl).max() if sl.size else 0.0
        out[a:a + 128] = m / 448.0 if m > 0 else 1.0
    return out


def dense_drift_bound(V, W, H, t, B, p, phi, S, mu_min=1e-10, v_bf16=False, fp8=False, part=None):
    """First-order BF16 bound on |drift_gpu - drift| for part t (see module
    docstring); W I x K, H K x J, FP64.  With v_bf16 the data are rounded to
    BF16 too: e moves by at most |de/dv| u |v| = max(mu, mu_min)^-p u |v| / phi.
    With fp8, GEMM1's operands are E4M3 with one scale s per 128-row W tile
    and per 128-column H tile: |q(x) - x| <= u8 |x| + eta s (u8 = 2^-4, eta
    = 2^-10 from the subnormals), so mu moves by at most (2 u8 + u8^2) A +
    (1 + u8)(eta s_H sum_k |w| + eta s_W sum_k |h|) + K eta^2 s_W s_H, plus
    the FP32 rounding of the scales."""
    I, J = V.shape
    s = (t - 1) % B if part is None else part       # part: the drawn part (size-proportional)
    bW = np.zeros_like(W)
    bH = np.zeros_like(H)
    for r in range(B):
        c = (r + s) % B
        r0, r1 = oracle.piece_start(r, I, B), oracle.piece_start(r + 1, I, B)
        c0, c1 = oracle.piece_start(c, J, B), oracle.piece_start(c + 1, J, B)
        w, h, v = W[r0:r1], H[:, c0:c1], V[r0:r1, c0:c1].astype(np.float64)
        mu = w @ h
        A = np.abs(w) @ np.abs(h)
        if fp8:
            eW = ETA_E4M3 * tile_scales(w, 0)[:, None]
            eH = ETA_E4M3 * tile_scales(h, 1)[None, :]
            Kw = w.shape[1]
            dmu = ((2 * U_E4M3 + U_E4M3 ** 2) * A * 1.01
                   + (1 + U_E4M3) * (eH * np.abs(w).sum(1)[:, None] + eW * np.abs(h).sum(0)[None, :])
                   + Kw * eW * eH + (4 * Kw + 16) * U_FP32 * A * (1 + 2 * U_E4M3))
        else:
            dmu = 2 * U_BF16 * A * 1.01 + 4 * w.shape[1] * U_FP32 * A
        if p > 0:
            mc = np.maximum(mu, mu_min)
            lo = np.maximum(mu - dmu, mu_min)
            e = (v - mu) * mc ** -p / phi
            fprime = lo ** -p * (1 + p * (np.abs(v - mu) + dmu) / lo) / phi
        else:
            e = (v - mu) / phi
            fprime = np.full_like(mu, 1.0 / phi)
        de = fprime * dmu + 64 * U_FP32 * np.abs(e)
        if v_bf16:
            de = de + (np.maximum(mu - dmu, mu_min) ** -p if p > 0 else 1.0) * U_BF16 * np.abs(v) / phi
        ebf = de + U_BF16 * (np.abs(e) + de)            # error of the BF16 e
        nc, nr = c1 - c0, r1 - r0
        bW[r0:r1] = (ebf @ np.abs(h).T) * (1 + U_BF16) + (U_BF16 + nc * U_FP32) * (np.abs(e) @ np.abs(h).T)
        bH[:, c0:c1] = (np.abs(w).T @ ebf) * (1 + U_BF16) + (U_BF16 + nr * U_FP32) * (np.abs(w).T @ np.abs(e))
    return S * bW, S * bH
