"""psgld_log_lik_static: the log-likelihood for callers that cannot allocate.

Callers whose device memory belongs to another allocator, or who run where an
allocation would synchronise the device, can still evaluate the Tweedie
log-likelihood of their factors: this entry point takes plain entry and
factor arrays and keeps its scratch in a fixed array inside the library.  The
test checks it through the C ABI against the context-based psgld_log_lik on
two different problems, one call right after the other (the second call
reuses the scratch the first one left behind), and that an input beyond the
fixed maximum is refused with PSGLD_ERR_SIZE.

It also checks what the entry point promises beyond the value: repeated
calls leave the device's free memory and PyTorch's reserved memory exactly
as they were (nothing is allocated), a call on a side stream and one for the
compound Poisson model (p = 1.5) give the same value as the context's,
zero entries give 0, and an entry index outside the factors gives NaN
without reading outside the caller's arrays.

This file is collected last on purpose: it must pass on its own in a fresh
process and after every other test.
"""
import numpy as np
import pytest

from paper_1506_01418_gb300 import datagen
from paper_1506_01418_gb300 import psgld as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _problem(I, J, nnz, K, p, seed):
    dev = "cuda"
    i, j, v = datagen.sparse_ratings(I, J, nnz, 6, seed)
    nonneg = p > 0
    W0, H0 = datagen.init_factors(I, J, K, seed, scale=0.4, nonneg=nonneg)
    chain = P.PSGLD(I, J, K, 3, p, 1.3, prior_kind=0 if nonneg else 1, seed=seed, eps=1e-3)
    ti = torch.as_tensor(i, device=dev)
    tj = torch.as_tensor(j, device=dev)
    tv = torch.as_tensor(v, device=dev)
    chain.set_data_coo(ti, tj, tv)
    chain.set_factors(torch.from_numpy(W0).to(dev), torch.from_numpy(H0.T.copy()).to(dev))
    chain.sweep(1)                                  # factors away from their start
    W, Ht = chain.get_factors()
    torch.cuda.synchronize()
    return chain, ti, tj, tv, W, Ht


def test_static_log_lik_matches_context_log_lik_twice_in_a_row():
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    cases = [(3000, 2000, 60000, 50, 0.0, 3),       # 15 blocks of entries
             (700, 400, 5000, 13, 1.0, 4)]          # 2 blocks: stale slots must not leak
    for I, J, nnz, K, p, seed in cases:
        chain, i, j, v, W, Ht = _problem(I, J, nnz, K, p, seed)
        want = chain.log_lik()
        P.psgld_log_lik_static(i, j, v, W, Ht, p, 1.3, out)
        torch.cuda.synchronize()
        got = float(out.item())
        assert got == pytest.approx(want, rel=1e-9, abs=1e-9), (I, J, nnz, got, want)
        chain.close()


def test_static_log_lik_refuses_inputs_beyond_its_scratch():
    n = P.PSGLD_STATIC_MAX_NNZ + 1
    lib = P.load()
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = lib.psgld_log_lik_static(n, dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                                  dummy.data_ptr(), dummy.data_ptr(), 2, 2, 1, 0.0, 1.0, 1e-10,
                                  out.data_ptr(), None)
    assert st == P.PSGLD_ERR_SIZE


def test_static_log_lik_allocates_nothing_and_follows_the_stream():
    chain, i, j, v, W, Ht = _problem(900, 600, 20000, 24, 1.5, 5)
    want = chain.log_lik()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    P.psgld_log_lik_static(i, j, v, W, Ht, 1.5, 1.3, out)      # the first call may set up
    torch.cuda.synchronize()
    with torch.cuda.stream(side):                              # the side stream used once
        P.psgld_log_lik_static(i, j, v, W, Ht, 1.5, 1.3, out, stream=side.cuda_stream)
    side.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    res0 = torch.cuda.memory_reserved()
    for n in range(6):
        out.zero_()
        torch.cuda.synchronize()
        if n % 2:
            with torch.cuda.stream(side):
                P.psgld_log_lik_static(i, j, v, W, Ht, 1.5, 1.3, out, stream=side.cuda_stream)
            side.synchronize()
        else:
            P.psgld_log_lik_static(i, j, v, W, Ht, 1.5, 1.3, out)
            torch.cuda.synchronize()
        assert float(out.item()) == pytest.approx(want, rel=1e-9, abs=1e-9), n
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_reserved() == res0
    assert free1 == free0
    chain.close()


def test_static_log_lik_of_no_entries_is_zero_and_bad_indices_give_nan():
    chain, i, j, v, W, Ht = _problem(500, 300, 9000, 8, 1.0, 6)
    out = torch.full((1,), 123.0, dtype=torch.float64, device="cuda")
    P.psgld_log_lik_static(i[:0], j[:0], v[:0], W, Ht, 1.0, 1.3, out)
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0
    for which, bad in (("i", 500), ("i", -1), ("j", 300), ("j", -7)):
        ii, jj = i.clone(), j.clone()
        (ii if which == "i" else jj)[4100] = bad            # in the second block of entries
        P.psgld_log_lik_static(ii, jj, v, W, Ht, 1.0, 1.3, out)
        torch.cuda.synchronize()
        assert np.isnan(float(out.item())), (which, bad)
    # and a clean call afterwards is exact again: nothing carries over
    P.psgld_log_lik_static(i, j, v, W, Ht, 1.0, 1.3, out)
    torch.cuda.synchronize()
    assert float(out.item()) == pytest.approx(chain.log_lik(), rel=1e-9, abs=1e-9)
    chain.close()
