"""The library's native serving loop (psgld_server_*): a job's result is the
same alone, in a mix, and under a memory budget that makes jobs wait, and
equal to the same chain run directly through the library; a job larger than
the whole budget is refused; latencies are reported for every job."""
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
            serving.Job(job_id=2, I=1025, J=800, K=16, B=8, p=1.0, sweeps=5, burn_in=1, seed=13,
                        data_seed=3)]


def _inputs(ex, job):
    V, W0, Ht0 = ex._data(job)
    torch.cuda.synchronize()
    return V, W0, Ht0


def _serve(jobs, budget):
    ex = serving.GpuExecutor()
    srv = P.NativeServer(budget)
    ids = {}
    for job in jobs:
        V, W0, Ht0 = _inputs(ex, job)
        ids[srv.submit(job.I, job.J, job.K, job.B, job.p, job.phi, V, W0, Ht0, job.sweeps,
                       lambda_w=job.lam, lambda_h=job.lam, seed=job.seed, eps=job.eps,
                       burn_in_sweeps=job.burn_in, dense_path=job.dense_path)] = job.job_id
    srv.wait_idle(300.0)
    done = srv.poll()
    assert sorted(i for i, _ in done) == sorted(ids)
    assert all(lat > 0 for _, lat in done), srv.last_error()
    out = {ids[i]: srv.results(i) for i, _ in done}
    st = srv.stats()
    srv.close()
    return out, st


def test_native_server_result_is_the_same_alone_and_in_the_mix():
    try:
        alone, _ = _serve([_jobs()[0]], 8 << 30)
        mix, st = _serve(_jobs(), 8 << 30)
        assert st["sweeps"] >= 6 and st["jobs_per_sweep"] >= 1.0   # batching depends on timing
        e = [P.psgld_estimate_device_bytes(j.I, j.J, j.K, j.B, 0, j.dense_path, 0) for j in _jobs()]
        queued, stq = _serve(_jobs(), max(e[0] + e[1], e[2]))
        assert stq["peak_bytes"] <= max(e[0] + e[1], e[2])
        for got in (mix[0], queued[0]):
            assert np.array_equal(alone[0][0], got[0]) and np.array_equal(alone[0][1], got[1])
        for k in (1, 2):
            assert np.array_equal(mix[k][0], queued[k][0]) and np.array_equal(mix[k][1], queued[k][1])
        # the same chain straight through the library
        P.psgld_set_allocator(None)
        job = _jobs()[0]
        V, W0, Ht0 = _inputs(serving.GpuExecutor(), job)
        P.psgld_set_allocator(None)
        ch = P.PSGLD(job.I, job.J, job.K, job.B, job.p, job.phi, seed=job.seed, eps=job.eps,
                     burn_in_sweeps=job.burn_in, dense_path=job.dense_path, lambda_w=job.lam,
                     lambda_h=job.lam)
        ch.set_data_dense(V)
        ch.set_factors(W0, Ht0)
        ch.sweep(job.sweeps)
        Wm, _, Hm, _, n = ch.posterior_mean()
        ch.close()
        assert n == job.sweeps - job.burn_in
        assert np.array_equal(alone[0][0], Wm) and np.array_equal(alone[0][1], Hm)
    finally:
        P.psgld_set_allocator(None)


def test_native_server_refuses_a_job_larger_than_the_budget():
    job = _jobs()[0]
    V, W0, Ht0 = _inputs(serving.GpuExecutor(), job)
    P.psgld_set_allocator(None)
    srv = P.NativeServer(1 << 20)
    with pytest.raises(P.PsgldError) as ex:
        srv.submit(job.I, job.J, job.K, job.B, job.p, job.phi, V, W0, Ht0, job.sweeps,
                   dense_path=job.dense_path)
    assert ex.value.status == P.PSGLD_ERR_SIZE
    srv.close()
