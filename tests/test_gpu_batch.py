"""Many dense chains sweeping in shared launches (psgld_batch_sweep).

At every part of a sweep one tensor-core gradient launch per kernel variant
covers the blocks of all the chains on it (the two-sided kernel as one
persistent launch over all their items) and one update launch covers all
the chains' rows (Sec. 3's part-step, run for many independent chains at
once).  Each chain reads only its own parameters, so a chain swept in a
batch must end bit for bit where the same chain swept alone ends (alone
through the captured-graph sweep): factors, posterior sums and iteration
counter.  The batch mixes sizes (ragged blocks, blocks over one 128-row
tile), ranks of every K class, Tweedie powers, both priors and both step
size schedules, GEMM1 in BF16 and in E4M3, and both tensor-core kernels
(the two-sided one with FP32 and BF16 V, K widths 64 and 256).
"""
import numpy as np
import pytest

from paper_1506_01418_gb300 import datagen
from paper_1506_01418_gb300 import psgld as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

# (I, J, K, p, prior_kind, eps_mode, kernel options)
SP = dict(dense_path=3)
MIX = [
    (300, 700, 8, 1.0, 0, 0, SP),
    (513, 900, 16, 2.0, 0, 0, SP),    # blocks of 128 and 129 rows: two M-tiles
    (257, 4000, 32, 1.0, 0, 0, SP),
    (640, 1000, 32, 1.5, 0, 1, SP),   # second chain of the K = 32 class, eps_t = (a/t)^b
    (1025, 300, 64, 0.0, 1, 0, SP),   # Gaussian likelihood and priors
    (90, 61, 13, 3.0, 0, 0, SP),
    (200, 500, 100, 1.0, 0, 1, SP),
    (400, 800, 32, 1.0, 0, 0, dict(dense_path=3, dense_fp8=1)),   # E4M3 GEMM1: a launch of its own
    (130, 333, 12, 2.0, 0, 0, dict(dense_path=3, dense_fp8=1)),
    # two-sided kernel: one persistent launch per (K width, V type, power)
    (300, 700, 8, 1.0, 0, 0, dict(dense_path=2)),
    (513, 2000, 50, 1.0, 0, 1, dict(dense_path=2)),   # blocks over 128 rows
    (260, 390, 200, 1.0, 0, 0, dict(dense_path=2)),   # K width 256
    (700, 450, 40, 2.0, 0, 0, dict(dense_path=2, dense_v_bf16=1)),
    (333, 777, 64, 2.0, 0, 0, dict(dense_path=2, dense_v_bf16=1)),
    # columns items taking E from the rows items, in the same launches as
    # contexts whose columns items form their own mu
    (513, 2000, 50, 1.0, 0, 1, dict(dense_path=2, dense_share_e=1)),
    (700, 450, 40, 2.0, 0, 0, dict(dense_path=2, dense_v_bf16=1, dense_share_e=1)),
]
B = 4


def _chain(idx, I, J, K, p, kind, eps_mode, kopts, use_graphs, burn_in=1, B=B):
    dev = torch.device("cuda", 0)
    if p == 1.0:
        V, _, _ = datagen.dense_poisson(I, J, 3, idx)
    else:
        V, _, _ = datagen.dense_gamma(I, J, 3, idx)
    if p >= 2:
        V = V + np.float32(0.5)
    nonneg = kind == 0
    W0, H0 = datagen.init_factors(I, J, K, seed=idx + 50, scale=0.4 if nonneg else 0.3,
                                  nonneg=nonneg)
    opts = dict(seed=1000 + idx, eps=1e-4, burn_in_sweeps=burn_in, use_graphs=use_graphs, **kopts)
    if eps_mode:
        opts.update(eps_mode=P.PSGLD_EPS_POLY, eps_a=0.02, eps_b=0.55)
    ch = P.PSGLD(I, J, K, B, p, 1.0, prior_kind=kind, lambda_w=0.8, lambda_h=1.2, sigma_w=0.9,
                 sigma_h=1.1, **opts)
    ch.set_data_dense(torch.from_numpy(np.ascontiguousarray(V, np.float32)).to(dev))
    ch.set_factors(torch.from_numpy(W0).to(dev), torch.from_numpy(H0.T.copy()).to(dev))
    return ch


def _state(ch):
    W, Ht = ch.get_factors()
    torch.cuda.synchronize()
    return W.cpu().numpy(), Ht.cpu().numpy(), ch.posterior_mean(), ch.iterations_done


def _assert_same(a, b):
    Wa, Ha, ma, ta = _state(a)
    Wb, Hb, mb, tb = _state(b)
    assert ta == tb
    assert np.array_equal(Wa, Wb) and np.array_equal(Ha, Hb)
    for x, y in zip(ma[:4], mb[:4]):
        assert np.array_equal(x, y)
    assert ma[4] == mb[4]


def test_batched_sweeps_equal_sweeps_alone():
    batch = [_chain(i, *m, use_graphs=0) for i, m in enumerate(MIX)]
    alone = [_chain(i, *m, use_graphs=1) for i, m in enumerate(MIX)]
    P.psgld_batch_sweep(batch, 2)
    P.psgld_batch_sweep(batch, 1)
    for ch in alone:
        ch.sweep(3)
    for a, b in zip(batch, alone):
        _assert_same(a, b)
        assert a.posterior_mean()[4] == 2
    # the chains moved and stayed valid
    for a, m in zip(batch, MIX):
        W, Ht, _, _ = _state(a)
        assert np.isfinite(W).all() and np.isfinite(Ht).all()
        if m[4] == 0:
            assert W.min() >= 0 and Ht.min() >= 0
    for ch in batch + alone:
        ch.close()


def test_batch_of_one_and_zero_sweeps():
    a = _chain(3, *MIX[3], use_graphs=0)
    b = _chain(3, *MIX[3], use_graphs=0)
    P.psgld_batch_sweep([a], 0)
    assert a.iterations_done == 0
    P.psgld_batch_sweep([a], 2)
    b.sweep(2)
    _assert_same(a, b)
    a.close()
    b.close()


def test_batch_refusals():
    good = _chain(0, *MIX[0], use_graphs=0)
    other = _chain(2, *MIX[2], use_graphs=0)
    # a context twice
    with pytest.raises(P.PsgldError) as ex:
        P.psgld_batch_sweep([good, other, good], 1)
    assert ex.value.status == P.PSGLD_ERR_ARG
    # not at a sweep boundary
    other.part_step(1)
    with pytest.raises(P.PsgldError) as ex:
        P.psgld_batch_sweep([good, other], 1)
    assert ex.value.status == P.PSGLD_ERR_STATE
    # a context on the sparse layout (dense V through the FP32 gather path)
    I, J, K = 300, 700, 8
    V, _, _ = datagen.dense_poisson(I, J, 3, 0)
    two = P.PSGLD(I, J, K, B, 1.0, 1.0, dense_path=0)
    two.set_data_dense(torch.from_numpy(V).cuda())
    W0, H0 = datagen.init_factors(I, J, K, seed=1, scale=0.4, nonneg=True)
    two.set_factors(torch.from_numpy(W0).cuda(), torch.from_numpy(H0.T.copy()).cuda())
    with pytest.raises(P.PsgldError) as ex:
        P.psgld_batch_sweep([good, two], 1)
    assert ex.value.status == P.PSGLD_ERR_STATE
    # another B
    I, J, K = 100, 80, 8
    V, _, _ = datagen.dense_poisson(I, J, 3, 0)
    b3 = P.PSGLD(I, J, K, 3, 1.0, 1.0, dense_path=3)
    b3.set_data_dense(torch.from_numpy(V).cuda())
    W0, H0 = datagen.init_factors(I, J, K, seed=1, scale=0.4, nonneg=True)
    b3.set_factors(torch.from_numpy(W0).cuda(), torch.from_numpy(H0.T.copy()).cuda())
    with pytest.raises(P.PsgldError) as ex:
        P.psgld_batch_sweep([good, b3], 1)
    assert ex.value.status == P.PSGLD_ERR_ARG
    # nothing ran on the refused calls
    assert good.iterations_done == 0
    for ch in (good, other, two, b3):
        ch.close()


def test_batched_sweeps_are_profiled_on_the_first_context():
    """profile = 1 on the first context: events around every part's
    launches, read with psgld_profile_read_split."""
    chains = [_chain(i, *m, use_graphs=0) for i, m in enumerate(MIX[:4])]
    chains[0].set_options(profile=1)
    P.psgld_batch_sweep(chains, 1)
    g, u, n = chains[0].profile_read_split()
    assert n == B and g > 0 and u > 0
    for ch in chains:
        ch.close()


def test_odd_b_alternates_the_buffers_between_sweeps():
    """With B odd the ping-pong buffers a sweep starts from alternate, so the
    call keeps two sets of tables; three sweeps (and a frozen H, whose
    buffer never flips) against the same chains swept alone."""
    mix = [MIX[0], MIX[9], MIX[12]]
    batch = [_chain(i, *m, use_graphs=0, B=3) for i, m in enumerate(mix)]
    alone = [_chain(i, *m, use_graphs=1, B=3) for i, m in enumerate(mix)]
    for ch in (batch[1], alone[1]):
        ch.set_options(freeze_H=1)
    P.psgld_batch_sweep(batch, 3)
    for ch in alone:
        ch.sweep(3)
    for a, b in zip(batch, alone):
        _assert_same(a, b)
    for ch in batch + alone:
        ch.close()


def test_batched_sweeps_from_captured_graphs_equal_sweeps_alone():
    """use_graphs on the first context: each batched sweep replays a captured
    graph (one per buffer parity and accumulation flag).  Calls of one and
    of two sweeps (replays of the same graphs), B even and odd, against the
    chains swept alone."""
    for b_ in (B, 3):
        mix = MIX if b_ == B else [MIX[0], MIX[9], MIX[12], MIX[3]]
        batch = [_chain(i, *m, use_graphs=1, B=b_) for i, m in enumerate(mix)]
        alone = [_chain(i, *m, use_graphs=1, B=b_) for i, m in enumerate(mix)]
        for n in (1, 2):          # a capture, then replays of the captured graphs
            P.psgld_batch_sweep(batch, n)
        for ch in alone:
            ch.sweep(3)
        for a, b in zip(batch, alone):
            _assert_same(a, b)
        for ch in batch + alone:
            ch.close()


def test_batch_graph_is_captured_again_when_the_list_changes():
    """The first context keeps the graphs of its batch; a list with another
    structure (a context more or less, another kernel variant, another first
    context) captures new ones on its second consecutive call, and every
    chain still ends where it ends alone."""
    idx = [0, 2, 9, 12]
    batch = {i: _chain(i, *MIX[i], use_graphs=1) for i in idx}
    alone = {i: _chain(i, *MIX[i], use_graphs=1) for i in idx}
    plan = [[0, 2, 9, 12]] * 2 + [[0, 2]] * 2 + [[0, 9, 12]] * 2 + [[2, 9, 12]] * 2
    done = {i: 0 for i in idx}
    for lst in plan:
        P.psgld_batch_sweep([batch[i] for i in lst], 1)
        for i in lst:
            done[i] += 1
    for i in idx:
        alone[i].sweep(done[i])
        _assert_same(batch[i], alone[i])
    for ch in list(batch.values()) + list(alone.values()):
        ch.close()


@pytest.mark.parametrize("ctas,blocks", [(76, 0), (112, 608), (0, 4864), (13, 1)])
def test_batch_launch_knobs_do_not_change_the_chains(ctas, blocks):
    """batch_ctas (CTAs of the persistent two-sided launches) and
    batch_update_blocks (blocks of the update launches) move work between
    CTAs only: chains end bit for bit as with the default launches."""
    mix = [MIX[i] for i in (0, 2, 9, 12, 13)]    # fixed step sizes: stable over many sweeps
    tuned = [_chain(i, *m, use_graphs=1) for i, m in enumerate(mix)]
    plain = [_chain(i, *m, use_graphs=1) for i, m in enumerate(mix)]
    tuned[0].set_options(batch_ctas=ctas, batch_update_blocks=blocks)
    P.psgld_batch_sweep(tuned, 2)
    P.psgld_batch_sweep(plain, 2)
    for a, b in zip(tuned, plain):
        _assert_same(a, b)
    for ch in tuned + plain:
        ch.close()


def test_autotuner_records_a_choice_and_its_sweeps_are_ordinary_sweeps():
    from paper_1506_01418_gb300 import autotune
    mix = [MIX[i] for i in (0, 2, 9, 12, 13)]    # fixed step sizes: stable over many sweeps
    tuned = [_chain(i, *m, use_graphs=1) for i, m in enumerate(mix)]
    plain = [_chain(i, *m, use_graphs=1) for i, m in enumerate(mix)]
    rec = autotune.tune_batch(tuned, sweeps_per_trial=1, repeats=1,
                              cta_candidates=(0, 76), update_candidates=(0, 608))
    assert rec["batch_ctas"] in (0, 76) and rec["batch_update_blocks"] in (0, 608)
    assert len(rec["ms_per_sweep"]) == 3 and all(v > 0 for v in rec["ms_per_sweep"].values())
    assert tuned[0].options.batch_ctas == rec["batch_ctas"]
    n = tuned[0].iterations_done // B
    assert n == 2 * 3          # one capture sweep and one timed sweep per trial
    P.psgld_batch_sweep(tuned, 1)
    for ch in plain:
        ch.sweep(n + 1)
    for a, b in zip(tuned, plain):
        _assert_same(a, b)
    for ch in tuned + plain:
        ch.close()
