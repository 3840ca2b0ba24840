"""Failure detection on the device, without faulting the GPU.

Every spin-wait in the library's kernels is bounded: a wait that runs out
sets the context's error flag, the kernel waits (bounded again, with the
normal limit) for its own copies in flight and returns, and the next
synchronising call reports PSGLD_ERR_TIMEOUT naming the kernel and the wait.
Here a test limit (the option debug_wait_polls) makes the sparse gradient
kernel's first wait for its row gathers give up after one poll, so the
timeout path runs for real; the drain wait keeps its normal limit.  The
test checks the status and the message, that the GPU and the context stay
usable, and that the next part-step, with the normal limit and fresh
factors, matches the oracle.
"""
import numpy as np
import pytest

from gpu_helpers import Pair, sparse_case
from paper_1506_01418_gb300 import datagen
from paper_1506_01418_gb300 import psgld as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_gather_wait_that_runs_out_reports_timeout_and_the_context_recovers():
    I, J, K, B = 300, 200, 50, 3
    i, j, v = sparse_case(I, J, 20000, 5, seed=I + J)
    W0, H0 = datagen.init_factors(I, J, K, seed=3, scale=0.3, nonneg=False)
    pr = Pair(I, J, K, B, 0.0, 1.0, i, j, v, W0, H0, prior_kind=1, seed=7, eps=1e-3)
    pr.gpu.set_options(debug_wait_polls=1)
    pr.gpu.part_step(1)
    torch.cuda.synchronize()                 # no fault: the kernels returned
    with pytest.raises(P.PsgldError) as e:
        pr.gpu.log_lik()
    assert e.value.status == P.PSGLD_ERR_TIMEOUT
    assert "sparse gradient kernel (wait for the row gathers)" in str(e.value)
    # the flag was cleared by the report; with the normal limit and fresh
    # factors the next part-step is the oracle's
    pr.gpu.set_options(debug_wait_polls=0)
    pr.set_factors(W0, H0)
    pr.step_and_check(1)
    assert np.isfinite(pr.gpu.log_lik())
    # and a second timeout is reported again (nothing was left stuck)
    pr.gpu.set_options(debug_wait_polls=1)
    pr.gpu.part_step(2)
    with pytest.raises(P.PsgldError) as e:
        pr.gpu.posterior_mean()
    assert e.value.status == P.PSGLD_ERR_TIMEOUT
    pr.gpu.close()


def test_debug_wait_polls_is_validated():
    c = P.PSGLD(10, 10, 4, 2, 1.0, 1.0)
    with pytest.raises(P.PsgldError) as e:
        c.set_options(debug_wait_polls=-1)
    assert e.value.status == P.PSGLD_ERR_ARG
    c.close()
