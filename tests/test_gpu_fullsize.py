"""Parity at the full sizes of the benchmarked sparse workloads.

The same inputs bench.py draws (its workload definitions and generator),
the same launch configuration (CUDA graphs for the sweep), against the FP64
oracle fed the identical entries and initial factors:

* sparse Gaussian ratings, 70000 x 10000, 10M entries, K = 50, B = 32 (the
  benchmark workload): the first two part-steps element by element
  (<= 1e-5, oracle resynchronised to the GPU factors after each), then one
  whole graph-replayed sweep run independently on both sides (<= 1e-4: 32
  part-steps of FP32 rounding), and the log-likelihood in FP64;
* large sparse Gaussian ratings, 480000 x 18000, 100M entries, K = 100,
  B = 64: the first two part-steps element by element.
"""
import numpy as np
import pytest

import bench
import oracle
from gpu_helpers import STEP_RTOL, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _pair(name, seed=1000):
    wl = bench.WORKLOADS[name]
    dev = torch.device("cuda", 0)
    i, j, v, W0, H0 = bench.make_inputs(wl, seed, dev)
    chain = bench.new_chain(wl, seed, use_graphs=1)
    chain.set_data_coo(i, j, v)
    chain.set_factors(torch.from_numpy(W0).to(dev), torch.from_numpy(H0.T.copy()).to(dev))
    hi, hj, hv = (x.cpu().numpy() for x in (i, j, v))
    del i, j, v
    torch.cuda.empty_cache()
    orc = bench.oracle_setup(wl, hi, hj, hv.astype(np.float64), W0.astype(np.float64),
                             H0.astype(np.float64), seed)
    return wl, chain, orc


def _gpu_factors(chain):
    W, Ht = chain.get_factors()
    torch.cuda.synchronize()
    return W.cpu().numpy().astype(np.float64), Ht.cpu().numpy().T.astype(np.float64)


def _two_part_steps(chain, orc):
    for t in (1, 2):
        chain.part_step(t)
        orc.part_step(t)
        Wg, Hg = _gpu_factors(chain)
        Wo, Ho = orc.get_factors()
        ew, eh = rel_err(Wg, Wo), rel_err(Hg, Ho)
        assert ew <= STEP_RTOL and eh <= STEP_RTOL, (t, ew, eh)
        orc.set_factors(Wg, Hg)


def test_benchmark_workload_full_size():
    wl, chain, orc = _pair("sparse_gauss_70000x10000_nnz10M_K50_B32")
    _two_part_steps(chain, orc)
    # continue to the end of the first sweep with direct part-steps, then one
    # graph-replayed sweep on both sides independently
    for t in range(3, wl["B"] + 1):
        chain.part_step(t)
        orc.part_step(t)
        Wg, Hg = _gpu_factors(chain)
        orc.set_factors(Wg, Hg)
    chain.sweep(1)
    orc.sweep(1)
    Wg, Hg = _gpu_factors(chain)
    Wo, Ho = orc.get_factors()
    assert rel_err(Wg, Wo) < 1e-4 and rel_err(Hg, Ho) < 1e-4
    orc.set_factors(Wg, Hg)
    assert chain.log_lik() == pytest.approx(orc.log_lik(), rel=1e-9)
    chain.close()


def test_large_sparse_workload_full_size():
    wl, chain, orc = _pair("sparse_gauss_480000x18000_nnz100M_K100_B64")
    _two_part_steps(chain, orc)
    chain.close()
