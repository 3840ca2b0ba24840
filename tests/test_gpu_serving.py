"""Serving loop on the GPU: a job's result is the same alone and in a mix.

Jobs of different sizes, Tweedie powers and ranks run concurrently on their
own streams, with memory from PyTorch's caching allocator.  Each job's chain
is fixed by its seed (Philox noise keyed by (seed, t), deterministic kernels,
no floating-point atomics), so its posterior means must be identical bit for
bit whether it runs alone, in a mix, under a memory budget that forces the
jobs to wait for each other, or directly through the library without the
server.  After every run the budget accounting returns to zero.  The same
holds with continuous batching (BatchedGpuExecutor), where the jobs'
part-steps share launches and jobs join and leave the batch between sweeps.
"""
import numpy as np
import pytest

from paper_1506_01418_gb300 import psgld as P
from paper_1506_01418_gb300 import serving

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _jobs():
    return [serving.Job(job_id=0, I=513, J=1200, K=16, B=8, p=1.0, sweeps=6, burn_in=2, seed=11,
                        data_seed=1),
            serving.Job(job_id=1, I=257, J=3000, K=64, B=8, p=1.5, sweeps=6, burn_in=2, seed=12,
                        data_seed=2),
            serving.Job(job_id=2, I=1025, J=800, K=16, B=8, p=1.0, sweeps=6, burn_in=2, seed=13,
                        data_seed=3)]


def _serve(jobs, budget, executor=serving.GpuExecutor):
    ex = executor()
    srv = serving.Server(ex, hbm_budget=budget)
    try:
        srv.run(jobs, idle_sleep=0)
    finally:
        srv.close()
        if hasattr(ex, "shutdown"):
            ex.shutdown()
    assert srv.used == 0 and not srv.active
    return {j.job_id: j.result for j in jobs}


def test_job_result_is_the_same_alone_and_in_the_mix():
    try:
        alone = _serve([_jobs()[0]], budget=8 << 30)
        mix = _serve(_jobs(), budget=8 << 30)
        ex = serving.GpuExecutor()
        e = [ex.estimate(j) for j in _jobs()]
        tight = max(e[0] + e[1], e[2])          # jobs 0 and 1 together; job 2 waits for them
        queued = _serve(_jobs(), budget=tight)
        for got in (mix[0], queued[0]):
            assert np.array_equal(alone[0]["Wmean"], got["Wmean"])
            assert np.array_equal(alone[0]["Hmean"], got["Hmean"])
        for k in (1, 2):
            assert np.array_equal(mix[k]["Wmean"], queued[k]["Wmean"])
        # the same chain straight through the library (legacy stream, cudaMalloc)
        P.psgld_set_allocator(None)
        job = _jobs()[0]
        V, W0, Ht0 = ex._data(job)
        ch = P.PSGLD(job.I, job.J, job.K, job.B, job.p, job.phi, seed=job.seed, eps=job.eps,
                     burn_in_sweeps=job.burn_in, dense_path=job.dense_path, lambda_w=job.lam,
                     lambda_h=job.lam)
        ch.set_data_dense(V)
        ch.set_factors(W0, Ht0)
        ch.sweep(job.sweeps)
        Wm, _, Hm, _, n = ch.posterior_mean()
        ch.close()
        assert n == job.sweeps - job.burn_in
        assert np.array_equal(alone[0]["Wmean"], Wm) and np.array_equal(alone[0]["Hmean"], Hm)
    finally:
        P.psgld_set_allocator(None)


def test_estimate_covers_what_a_context_holds():
    """psgld_estimate_device_bytes against the device memory a context really
    takes (cudaMalloc path, measured with cudaMemGetInfo)."""
    P.psgld_set_allocator(None)
    torch.cuda.synchronize()
    for (I, J, K, B, dp, vb) in ((1025, 3000, 64, 8, 1, 0), (700, 900, 200, 3, 2, 1), (513, 800, 16, 8, 3, 0)):
        V = torch.rand((I, J), device="cuda")
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        ch = P.PSGLD(I, J, K, B, 1.0, 1.0, dense_path=dp, dense_v_bf16=vb)
        ch.set_data_dense(V)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        used = free0 - free1
        est = P.psgld_estimate_device_bytes(I, J, K, B, 0, dp, vb)
        ch.close()
        # cudaMalloc rounds each buffer up (2 MB pages for large ones)
        assert est <= used + (8 << 20) and used <= est + 40 * (2 << 20), (I, J, K, B, dp, est, used)


def test_batched_serving_result_is_the_same_alone_and_in_the_mix():
    try:
        B = serving.BatchedGpuExecutor
        jobs = _jobs()
        jobs[1].arrival = 0.05                   # joins the batch a few sweeps later
        alone = _serve([_jobs()[0]], budget=8 << 30, executor=B)
        mix = _serve(jobs, budget=8 << 30, executor=B)
        ex = B()
        e = [ex.estimate(j) for j in _jobs()]
        queued = _serve(_jobs(), budget=max(e[0] + e[1], e[2]), executor=B)
        for got in (mix[0], queued[0]):
            assert np.array_equal(alone[0]["Wmean"], got["Wmean"])
            assert np.array_equal(alone[0]["Hmean"], got["Hmean"])
        for k in (1, 2):
            assert np.array_equal(mix[k]["Wmean"], queued[k]["Wmean"])
            assert mix[k]["n_samples"] == _jobs()[k].sweeps - _jobs()[k].burn_in
        # job 0 swept alone through the library on the same kernel
        P.psgld_set_allocator(None)
        job = _jobs()[0]
        V, W0, Ht0 = ex._data(job)
        ch = P.PSGLD(job.I, job.J, job.K, job.B, job.p, job.phi, seed=job.seed, eps=job.eps,
                     burn_in_sweeps=job.burn_in, dense_path=job.dense_path, lambda_w=job.lam,
                     lambda_h=job.lam)
        ch.set_data_dense(V)
        ch.set_factors(W0, Ht0)
        ch.sweep(job.sweeps)
        Wm, _, Hm, _, n = ch.posterior_mean()
        ch.close()
        assert np.array_equal(alone[0]["Wmean"], Wm) and np.array_equal(alone[0]["Hmean"], Hm)
    finally:
        P.psgld_set_allocator(None)
