"""Shared set-up of the GPU parity tests: one CUDA chain and one oracle chain
started from the same seeded inputs."""
import numpy as np

import oracle
from paper_1506_01418_gb300 import datagen
from paper_1506_01418_gb300 import psgld as P

# One FP32 part-step against the FP64 oracle, from identical factors and with
# the identical Philox stream: max |gpu - oracle| / max(|oracle|, floor), with
# the floor 1e-2 x the RMS of the oracle's matrix, so that elements the mirror
# or the noise moved through zero are judged on the matrix's own scale.
STEP_RTOL = 1e-5

U_BF16 = 2.0 ** -8
U_FP32 = 2.0 ** -24


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
