"""Checkpoint and resume (psgld_get_state / psgld_set_state): a chain that
stops after some sweeps, whose factors, posterior sums and counters are
restored into a fresh context with the same options and data, ends bit for
bit where the same chain run straight through ends.  This holds because the
Langevin noise of iteration t depends only on (seed, t, matrix, index) --
Sec. 2's N(0, 2 eps) drawn from a counter-based stream -- and the
size-proportional part draw only on (seed, t).  Covered: the sparse path
with captured-graph sweeps, the size-proportional part order, the dense
two-sided tensor-core kernel with an odd B, and burn-in spanning the
checkpoint."""
import numpy as np
import pytest

from gpu_helpers import sparse_case
from paper_1506_01418_gb300 import datagen
from paper_1506_01418_gb300 import psgld as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

CASES = {
    # name: (I, J, K, B, p, prior_kind, dense, options)
    "sparse_gauss_graphs": (300, 200, 13, 3, 0.0, 1, False, dict(use_graphs=1)),
    "sparse_poisson_size_proportional": (240, 180, 8, 4, 1.0, 0, False, dict(part_mode=1)),
    "dense_two_sided_odd_B": (300, 260, 40, 3, 1.0, 0, True, dict(dense_path=2)),
}


def _inputs(name):
    I, J, K, B, p, kind, dense, _ = CASES[name]
    nonneg = kind == 0
    W0, H0 = datagen.init_factors(I, J, K, seed=4, scale=0.4 if nonneg else 0.3, nonneg=nonneg)
    if dense:
        V, _, _ = datagen.dense_poisson(I, J, 3, 2)
        return (torch.from_numpy(np.ascontiguousarray(V, np.float32)).cuda(),), W0, H0
    i, j, v = sparse_case(I, J, 4000, 5, seed=I + J)
    if p >= 1:
        v = v.astype(np.float32) + np.float32(0.25)
    return tuple(torch.as_tensor(x, device="cuda") for x in (i, j, v)), W0, H0


def _chain(name, data, W0, H0):
    I, J, K, B, p, kind, dense, opts = CASES[name]
    ch = P.PSGLD(I, J, K, B, p, 1.0, prior_kind=kind, lambda_w=0.8, lambda_h=1.2, sigma_w=0.9,
                 sigma_h=1.1, seed=77, eps=1e-4, burn_in_sweeps=3, **opts)
    if dense:
        ch.set_data_dense(*data)
    else:
        ch.set_data_coo(*data)
    ch.set_factors(torch.from_numpy(np.ascontiguousarray(W0, np.float32)).cuda(),
                   torch.from_numpy(np.ascontiguousarray(H0.T, np.float32)).cuda())
    return ch


def _factors(ch):
    W, Ht = ch.get_factors()
    torch.cuda.synchronize()
    return W.cpu().numpy(), Ht.cpu().numpy()


@pytest.mark.parametrize("name", sorted(CASES))
def test_resumed_chain_equals_the_chain_run_straight_through(name):
    data, W0, H0 = _inputs(name)
    straight = _chain(name, data, W0, H0)
    straight.sweep(5)

    first = _chain(name, data, W0, H0)
    first.sweep(2)                       # stops before the end of burn-in
    Wc, Htc = _factors(first)
    state = first.get_state()
    assert list(state[4]) == [2 * CASES[name][3], 2, 0]
    first.close()

    resumed = _chain(name, data, W0, H0)
    resumed.set_factors(torch.from_numpy(Wc).cuda(), torch.from_numpy(Htc).cuda())
    resumed.set_state(state)
    resumed.sweep(1)
    # a second checkpoint, now with samples kept, restored into the same context
    W1, Ht1 = _factors(resumed)
    s1 = resumed.get_state()
    assert list(s1[4]) == [3 * CASES[name][3], 3, 0]
    resumed.set_factors(torch.from_numpy(W1).cuda(), torch.from_numpy(Ht1).cuda())
    resumed.set_state(s1)
    resumed.sweep(2)

    Wa, Ha = _factors(straight)
    Wb, Hb = _factors(resumed)
    assert np.array_equal(Wa, Wb) and np.array_equal(Ha, Hb)
    sa, sb = straight.get_state(), resumed.get_state()
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)
    assert list(sb[4]) == [5 * CASES[name][3], 5, 2]
    ma, mb = straight.posterior_mean(), resumed.posterior_mean()
    for x, y in zip(ma[:4], mb[:4]):
        assert np.array_equal(x, y)
    assert ma[4] == mb[4] == 2
    straight.close()
    resumed.close()


def test_set_state_refusals():
    data, W0, H0 = _inputs("sparse_gauss_graphs")
    I, J, K = CASES["sparse_gauss_graphs"][:3]
    ch = _chain("sparse_gauss_graphs", data, W0, H0)
    z = [np.zeros((n, K)) for n in (I, I, J, J)]
    for bad in ([-1, 0, 0], [0, -1, 0], [3, 1, 2], [3, 1, -1]):
        with pytest.raises(P.PsgldError) as ex:
            ch.set_state((*z, np.array(bad, np.int64)))
        assert ex.value.status == P.PSGLD_ERR_ARG
    fresh = P.PSGLD(I, J, K, 3, 0.0, 1.0, prior_kind=1)
    fresh.set_data_coo(*data)
    with pytest.raises(P.PsgldError) as ex:
        fresh.set_state((*z, np.array([0, 0, 0], np.int64)))
    assert ex.value.status == P.PSGLD_ERR_STATE
    ch.close()
    fresh.close()
