"""A CPU model of the two-sided tensor-core kernel's barrier protocol
(`two_sided::chain_body` in psgld_dense.cu), run under random interleavings.

The kernel's roles -- a producer warp (bulk copies of the owned tile, the
walked tiles and the V tiles), an MMA warp (owned tile into TMEM, GEMM1 into
one of two mu buffers, GEMM2 of the previous tile from one of two E buffers)
and eight epilogue warps (mu + V -> E; the item's G rows at its end) -- are
modelled as coroutines that wait on mbarrier phases with the kernel's parity
rule (a wait for parity P passes once the phase with that parity has
completed), arrive with the kernel's counts, and issue asynchronous work:
copies that land in any order, and tensor-core operations (tcgen05.cp, MMAs,
commits) that run in issue order.  Every read checks that the slot holds the
tile it expects, so a wrong parity, a missing wait or a slot reused too early
fails; a deadlock fails too.  The slot and phase arithmetic follows the
kernel's (rings of NS walked and NV V slots advanced per tile across items,
mu / E buffer tc % 2 used for the (tc / 2)-th time).  CPU only.
"""
import random

import pytest

EPI_WARPS = 8


class Bar:
    """An mbarrier: `count` arrivals complete a phase."""

    def __init__(self, count):
        self.count, self.pending, self.phases = count, count, 0

    def arrive(self):
        self.pending -= 1
        if self.pending == 0:
            self.phases += 1
            self.pending = self.count

    def done(self, parity):
        # try_wait.parity: the phase with this parity has completed
        return (self.phases & 1) != parity


class Ring:
    def __init__(self):
        self.slot, self.phase = 0, 0

    def next(self, n):
        self.slot += 1
        if self.slot == n:
            self.slot, self.phase = 0, self.phase ^ 1


def run(items, NS, NV, seed, bug=None):
    """bug (for the model's own check): 'mu_parity' -- the epilogue waits
    for the wrong mu phase; 'skip_empty' -- the producer refills a walked
    slot without waiting for its release; 'early_release' -- GEMM2's slot is
    released before GEMM2 is issued."""
    rnd = random.Random(seed)
    full = [Bar(1) for _ in range(NS)]
    empty = [Bar(1) for _ in range(NS)]
    vfull = [Bar(1) for _ in range(NV)]
    vempty = [Bar(EPI_WARPS) for _ in range(NV)]
    mu_full = [Bar(1) for _ in range(2)]
    mu_empty = [Bar(EPI_WARPS) for _ in range(2)]
    e_full = [Bar(EPI_WARPS) for _ in range(2)]
    e_empty = [Bar(1) for _ in range(2)]
    a_full, a_empty, g_full, g_empty = Bar(1), Bar(1), Bar(1), Bar(EPI_WARPS)
    sA = [None]
    sB = [None] * NS
    sV = [None] * NV
    tmemA = [None]
    mu = [None, None]
    E = [[None] * EPI_WARPS for _ in range(2)]   # each warp writes its part of E
    G = {}
    copies, pipe = [], []

    def producer():
        rb, rv, ic = Ring(), Ring(), 0
        for nj in items:
            while not a_empty.done((ic & 1) ^ 1):
                yield
            copies.append((sA, 0, ("own", ic), a_full))
            for j in range(nj):
                st, sv = rb.slot, rv.slot
                while bug != "skip_empty" and not empty[st].done(rb.phase ^ 1):
                    yield
                copies.append((sB, st, ("B", ic, j), full[st]))
                while not vempty[sv].done(rv.phase ^ 1):
                    yield
                copies.append((sV, sv, ("V", ic, j), vfull[sv]))
                rb.next(NS)
                rv.next(NV)
            ic += 1

    def mma():
        tc, ic = 0, 0
        r1, r2 = Ring(), Ring()
        for nj in items:
            while not a_full.done(ic & 1):
                yield
            pipe.append(("cp", ic))
            pipe.append(("commit", a_empty))
            for j in range(nj + 1):
                if j < nj:
                    st, b = r1.slot, tc & 1
                    while not full[st].done(r1.phase):
                        yield
                    while not mu_empty[b].done(((tc >> 1) & 1) ^ 1):
                        yield
                    pipe.append(("gemm1", st, b, ic, j))
                    pipe.append(("commit", mu_full[b]))
                    tc += 1
                    r1.next(NS)
                if j > 0:
                    tp = tc - 2 if j < nj else tc - 1
                    b, st = tp & 1, r2.slot
                    while not e_full[b].done((tp >> 1) & 1):
                        yield
                    if j == 1:
                        while not g_empty.done((ic & 1) ^ 1):
                            yield
                    if bug == "early_release":
                        pipe.append(("commit", empty[st]))
                    pipe.append(("gemm2", st, b, ic, j - 1, j == 1))
                    pipe.append(("commit", e_empty[b]))
                    if bug != "early_release":
                        pipe.append(("commit", empty[st]))
                    r2.next(NS)
            pipe.append(("commit", g_full))
            ic += 1

    def epilogue(w):
        tc, ic, rv = 0, 0, Ring()
        for nj in items:
            for j in range(nj):
                b, sv, ph = tc & 1, rv.slot, (tc >> 1) & 1
                while not vfull[sv].done(rv.phase):
                    yield
                while not mu_full[b].done(ph ^ 1 if bug == "mu_parity" else ph):
                    yield
                while not e_empty[b].done(ph ^ 1):
                    yield
                assert mu[b] == (ic, j), ("mu", w, mu[b], ic, j)
                assert sV[sv] == ("V", ic, j), ("V", w, sV[sv], ic, j)
                E[b][w] = (ic, j)
                vempty[sv].arrive()
                mu_empty[b].arrive()
                e_full[b].arrive()
                tc += 1
                rv.next(NV)
            while not g_full.done(ic & 1):
                yield
            assert G.get(ic) == nj, ("G", w, G.get(ic), nj)
            g_empty.arrive()
            ic += 1

    def execute(op):
        kind = op[0]
        if kind == "commit":
            op[1].arrive()
        elif kind == "cp":
            assert sA[0] == ("own", op[1]), ("cp", sA[0], op)
            tmemA[0] = op[1]
        elif kind == "gemm1":
            _, st, b, ic, j = op
            assert sB[st] == ("B", ic, j) and tmemA[0] == ic, ("gemm1", sB[st], tmemA[0], op)
            mu[b] = (ic, j)
        else:
            _, st, b, ic, j, first = op
            assert sB[st] == ("B", ic, j), ("gemm2", sB[st], op)
            assert all(e == (ic, j) for e in E[b]), ("gemm2 E", E[b], op)
            G[ic] = 1 if first else G[ic] + 1

    roles = [producer(), mma()] + [epilogue(w) for w in range(EPI_WARPS)]
    alive = set(range(len(roles)))
    stalls = 0
    while alive or copies or pipe:
        choices = [("role", r) for r in alive]
        if copies:
            choices.append(("copy", None))
        if pipe:
            choices.append(("pipe", None))
        kind, r = rnd.choice(choices)
        if kind == "role":
            try:
                next(roles[r])
            except StopIteration:
                alive.discard(r)
            stalls += 1
            assert stalls < 200_000, "deadlock"
        elif kind == "copy":
            dst, idx, content, bar = copies.pop(rnd.randrange(len(copies)))
            dst[idx] = content
            bar.arrive()
            stalls = 0
        else:
            execute(pipe.pop(0))
            stalls = 0
    return G


@pytest.mark.parametrize("NS,NV", [(2, 2), (3, 2), (4, 3)])
def test_protocol_holds_under_random_interleavings(NS, NV):
    for seed in range(60):
        rnd = random.Random(1000 * NS + seed)
        items = [rnd.choice([1, 2, 3, 5, 8, 32]) for _ in range(rnd.randint(1, 5))]
        G = run(items, NS, NV, seed)
        assert G == {ic: nj for ic, nj in enumerate(items)}


@pytest.mark.parametrize("bug", ["mu_parity", "skip_empty", "early_release"])
def test_model_catches_planted_protocol_mistakes(bug):
    """The model has teeth: each planted slip makes some read see the wrong
    tile (or the roles deadlock) under some interleaving."""
    with pytest.raises(AssertionError) as ex:
        for seed in range(200):
            run([32, 5, 8], 3, 2, seed, bug=bug)
    assert "deadlock" not in str(ex.value), ex.value
