"""Full chains of the FP32 gather path against full FP64 oracle chains.

Two independent chains (CUDA FP32 and oracle FP64) run from the same seeded
data, initial factors and Philox key for the whole run; their posterior-mean
reconstruction RMSE (sqrt of the mean over observed entries of
(v - W_mean H_mean)^2, Sec. 4.1's Monte Carlo averages after burn-in) must
agree within 1%.

* the dense Poisson NMF workload through the entry layout: 256 x 256, K = 8,
  B = 4, V ~ Poisson(W* H*), W*, H* ~ Gamma(1, 1), exponential priors rate 1,
  eps = 1e-4, 1000 sweeps;
* the sparse Gaussian ratings workload, shrunk so that the oracle finishes in
  seconds: 7000 x 1000, 100k entries with Zipf(1.1) degrees, values
  clip(round(W* H* + N(0, 0.5^2)), 1, 5), K = 50, B = 32, Gaussian priors
  sigma = 1, eps = 2e-5, 100 sweeps.
"""
import numpy as np
import pytest

from gpu_helpers import Pair
from paper_1506_01418_gb300 import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _chain_rmse(pr, sweeps):
    pr.gpu.sweep(sweeps)
    pr.orc.sweep(sweeps)
    return pr.gpu.rmse(True), pr.orc.rmse(True)


def test_dense_poisson_chain_via_entry_layout():
    I = J = 256
    K, B, sweeps = 8, 4, 1000
    V, _, _ = datagen.dense_poisson(I, J, K, seed=0)
    i, j, v = datagen.dense_to_coo(V)
    W0, H0 = datagen.init_factors(I, J, K, seed=0, scale=1.0, nonneg=True)
    pr = Pair(I, J, K, B, 1.0, 1.0, i, j, v, W0, H0, prior_kind=0, seed=11, eps=1e-4,
              burn_in_sweeps=sweeps // 2)
    r_gpu, r_or = _chain_rmse(pr, sweeps)
    assert abs(r_gpu - r_or) <= 0.01 * r_or, (r_gpu, r_or)
    Wg, Hg = pr.gpu_factors()
    assert Wg.min() >= 0 and Hg.min() >= 0


def test_sparse_gaussian_ratings_chain_shrunk():
    I, J, nnz, K, B, sweeps = 7000, 1000, 100_000, 50, 32, 100
    i, j, v = datagen.sparse_ratings(I, J, nnz, 20, seed=5, zipf_row=1.1, zipf_col=1.1)
    W0, H0 = datagen.init_factors(I, J, K, seed=5, scale=0.3, nonneg=False)
    pr = Pair(I, J, K, B, 0.0, 1.0, i, j, v, W0, H0, prior_kind=1, sig=(1.0, 1.0), seed=13,
              eps=2e-5, burn_in_sweeps=sweeps // 2)
    r_gpu, r_or = _chain_rmse(pr, sweeps)
    assert abs(r_gpu - r_or) <= 0.01 * r_or, (r_gpu, r_or)
