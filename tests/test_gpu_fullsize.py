"""Parity at the full sizes of the benchmarked workloads.

The same inputs bench.py draws (its workload definitions and generator),
the same launch configuration (CUDA graphs for the sweep), against the FP64
oracle fed the identical entries and initial factors:

* sparse Gaussian ratings, 70000 x 10000, 10M entries, K = 50, B = 32 (the
  benchmark workload): the first two part-steps element by element
  (<= 1e-5, oracle resynchronised to the GPU factors after each), then one
  whole graph-replayed sweep run independently on both sides (<= 1e-4: 32
  part-steps of FP32 rounding), and the log-likelihood in FP64;
* large sparse Gaussian ratings, 480000 x 18000, 100M entries, K = 100,
  B = 64: the first two part-steps element by element;
* the dense tensor-core workload (32768 x 32768, K = 256, B = 16, BF16 V,
  the two-sided kernel): one part-step, and the drift the GPU applied to the
  2048 rows of W and the 2048 columns of H of block (0, 0) against the
  oracle on the same factors with that block's entries as its data (with
  the scale S = B = 16 the oracle's drift on those rows is the workload's),
  element by element within the BF16 bound (the sampled outputs are the
  whole block);
* the batched workload (256 chains): one batched sweep of all chains, then
  three of them swept alone from the same inputs end bit for bit in the
  same state.
"""
import numpy as np
import pytest

import bench
import oracle
from gpu_helpers import STEP_RTOL, dense_drift_bound, recovered_drift, rel_err, step_errors
from paper_1506_01418_gb300 import psgld as P

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


def _two_part_steps(chain, orc, seed=1000):
    I, K = orc.I, orc.K
    for t in (1, 2):
        W0, H0 = orc.get_factors()
        chain.part_step(t)
        orc.part_step(t)
        Wg, Hg = _gpu_factors(chain)
        Wo, Ho = orc.get_factors()
        sd = float(np.sqrt(2.0 * orc.eps(t)))
        zW = oracle.noise_matrix(seed, t, 0, I, K)
        zH = oracle.noise_matrix(seed, t, 1, orc.J, K).T
        for xg, xo, x0, z, what in ((Wg, Wo, W0, zW, "W"), (Hg, Ho, H0, zH, "H")):
            elem, inc, inc_b = step_errors(xg, xo, x0, z, sd)
            assert elem <= STEP_RTOL and inc <= inc_b, (t, what, elem, inc, inc_b)
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


def test_dense_standing_chain_full_size_block_drift():
    name = "dense_poisson_32768x32768_K256_B16_bf16"
    wl = bench.WORKLOADS[name]
    seed = 1000
    dev = torch.device("cuda", 0)
    _, _, V, W0, H0 = bench.make_inputs(wl, seed, dev)
    I, J, K, B = wl["I"], wl["J"], wl["K"], wl["B"]
    chain = bench.new_chain(wl, seed, use_graphs=1)
    chain.set_data_dense(V)
    chain.set_factors(torch.from_numpy(W0).to(dev), torch.from_numpy(H0.T.copy()).to(dev))
    r1, c1 = oracle.piece_start(1, I, B), oracle.piece_start(1, J, B)   # block (0, 0) of part 1
    Vb = V[:r1, :c1].cpu().numpy().astype(np.float64)
    del V
    torch.cuda.empty_cache()
    chain.part_step(1)
    W, Ht = chain.get_factors()
    torch.cuda.synchronize()
    Wg = W[:r1].cpu().numpy().astype(np.float64)
    Hg = Ht[:c1].cpu().numpy().T.astype(np.float64)
    chain.close()
    del W, Ht
    torch.cuda.empty_cache()
    # the oracle: the full factors, block (0, 0)'s entries as the data, S = B
    orc = oracle.Oracle(I, J, K, B, wl["p"], wl["phi"], prior_kind=oracle.PRIOR_EXPONENTIAL,
                        lambda_w=wl["lam"], lambda_h=wl["lam"])
    orc.set_options(seed=seed, eps=wl["eps"], scale_mode=oracle.SCALE_B)
    ii, jj = np.meshgrid(np.arange(r1, dtype=np.int32), np.arange(c1, dtype=np.int32), indexing="ij")
    orc.set_data(ii.ravel(), jj.ravel(), Vb.ravel())
    orc.set_factors(W0.astype(np.float64), H0.astype(np.float64))
    D_W, D_H = orc.drift(1)
    S = float(B)
    w0, h0 = W0[:r1].astype(np.float64), H0[:, :c1].astype(np.float64)
    bW, bH = dense_drift_bound(Vb, w0, h0, 1, 1, wl["p"], wl["phi"], S, v_bf16=True)
    zW = oracle.noise_matrix(seed, 1, 0, I, K)[:r1]
    zH = oracle.noise_matrix(seed, 1, 1, J, K)[:c1].T
    eps = wl["eps"]
    for xg, x0, z, D, bnd, what in ((Wg, w0, zW, D_W[:r1], bW, "W"), (Hg, h0, zH, D_H[:, :c1], bH, "H")):
        Dg, mask, rec = recovered_drift(xg, x0, z, D, eps, True)
        err = np.abs(Dg - D)
        bad = mask & (err > bnd + rec)
        assert not bad.any(), (what, int(bad.sum()), float(err[bad].max()))
        assert mask.mean() > 0.9
        assert np.sqrt(np.mean(D[mask] ** 2)) > 4 * np.sqrt(np.mean(bnd[mask] ** 2)), what


def test_batched_workload_full_size_chains_equal_alone():
    wl = bench.WORKLOADS["batched_dense_nmf_256chains_513xJ200-5000_K32_B8_bf16"]
    dev = torch.device("cuda", 0)
    specs = bench.batched_specs(wl, 1000)

    def build(sp):
        made = bench.batched_make(wl, sp, dev)
        for ch, V, W0, Ht0 in made:
            ch.set_data_dense(V)
            ch.set_factors(W0, Ht0)
        return [m[0] for m in made]

    chains = build(specs)
    P.psgld_batch_sweep(chains, 1)
    for k in (0, 101, 255):
        alone = build([specs[k]])[0]
        alone.sweep(1)
        Wa, Ha = alone.get_factors()
        Wb, Hb = chains[k].get_factors()
        torch.cuda.synchronize()
        assert torch.equal(Wa, Wb) and torch.equal(Ha, Hb), k
        alone.close()
    for ch in chains:
        ch.close()
