"""The serving scheduler's admission and accounting, on the CPU with a
stand-in executor (no GPU): jobs are admitted in arrival order while the
device memory they will hold fits the budget, finished jobs release it, and
latency is completion minus arrival."""
import pytest

from paper_1506_01418_gb300 import serving


class FakeExecutor:
    """Each job takes `ticks` polls after it starts; memory = I * J * 100 B."""

    def __init__(self, ticks=3):
        self.ticks = ticks
        self.started = []
        self.standing_steps = 0

    def estimate(self, job):
        return job.I * job.J * 100

    def start(self, job):
        self.started.append(job.job_id)
        return {"left": self.ticks}

    def done(self, h):
        h["left"] -= 1
        return h["left"] <= 0

    def step_standing(self, job, h):
        self.standing_steps += 1

    def finish(self, job, h):
        return {"ok": job.job_id}


def _job(i, I, J, arrival, sweeps=5):
    return serving.Job(job_id=i, I=I, J=J, K=8, B=4, p=1.0, sweeps=sweeps, arrival=arrival)


def test_admission_respects_budget_and_order():
    ex = FakeExecutor(ticks=2)
    srv = serving.Server(ex, hbm_budget=10 * 100 * 100 * 100, max_active=8)   # room for ten 100x100 jobs
    jobs = [_job(0, 100, 100, 0.0), _job(1, 100, 600, 0.0), _job(2, 100, 100, 0.0),
            _job(3, 100, 100, 0.0)]
    for j in jobs:
        srv.submit(j)
    t = 0.0
    trace = []
    while len(srv.done) < len(jobs):
        srv.poll(t)
        trace.append((t, sorted(srv.active), srv.used))
        assert srv.used <= srv.budget
        t += 1.0
        assert t < 50
    # in order: job 1 (6 units) fits beside job 0 (1 unit); then 2 and 3 (1 each): 9 <= 10
    assert ex.started == [0, 1, 2, 3]
    assert srv.peak_used <= srv.budget
    assert srv.used == 0
    assert all(j.result == {"ok": j.job_id} for j in jobs)


def test_head_of_line_waits_for_memory():
    ex = FakeExecutor(ticks=3)
    srv = serving.Server(ex, hbm_budget=8 * 100 * 100 * 100)
    a, b, c = _job(0, 100, 600, 0.0), _job(1, 100, 500, 0.0), _job(2, 100, 100, 0.0)
    for j in (a, b, c):
        srv.submit(j)
    srv.poll(0.0)
    # b (5 units) does not fit beside a (6 units); c stays behind b (arrival order)
    assert ex.started == [0]
    for t in (1.0, 2.0, 3.0):
        srv.poll(t)
    assert a.finished == 3.0 and ex.started == [0, 1, 2]


def test_job_larger_than_budget_is_refused():
    srv = serving.Server(FakeExecutor(), hbm_budget=1000)
    srv.submit(_job(0, 100, 100, 0.0))
    with pytest.raises(ValueError):
        srv.poll(0.0)


def test_run_replays_arrivals_and_reports_latency():
    ex = FakeExecutor(ticks=2)
    srv = serving.Server(ex, hbm_budget=10 ** 9)
    clock = {"t": 0.0}

    def tick():
        clock["t"] += 0.5
        return clock["t"]

    jobs = [_job(i, 50, 50, arrival=float(i)) for i in range(5)]
    standing = serving.Job(job_id=99, I=50, J=50, K=8, B=4, p=1.0, sweeps=None, arrival=0.0)
    srv.run(jobs + [standing], clock=tick, idle_sleep=0)
    lat = serving.latency_summary(jobs)
    assert lat["n"] == 5 and lat["p50_s"] > 0
    assert all(j.finished >= j.arrival for j in jobs)
    assert ex.standing_steps > 0 and 99 in srv.active
    out = srv.stop_standing()
    assert [j.job_id for j in out] == [99] and srv.used == 0


def test_poisson_trace_rate_and_mix():
    jobs = serving.poisson_trace(200.0, 5.0, seed=1, job_factory=serving.mixed_job_factory())
    assert 850 < len(jobs) < 1150
    assert {j.I for j in jobs} == {257, 513, 1025}
    assert {j.K for j in jobs} == {16, 64} and {j.p for j in jobs} == {1.0, 1.5}
    assert min(j.J for j in jobs) >= 500 and max(j.J for j in jobs) <= 20000
    assert all(a.arrival < b.arrival for a, b in zip(jobs, jobs[1:]))


class FakeBatchExecutor(FakeExecutor):
    """Continuous batching stand-in: every tick advances each unfinished
    admitted job by one sweep; records which jobs each tick covered."""

    def __init__(self):
        super().__init__()
        self.members = []
        self.tick_log = []

    def start(self, job):
        self.started.append(job.job_id)
        h = {"job": job, "left": job.sweeps}
        self.members.append(h)
        return h

    def tick(self):
        if not self.members:
            return
        self.tick_log.append(sorted(h["job"].job_id for h in self.members))
        for h in self.members:
            h["left"] -= 1
        self.members = [h for h in self.members if h["left"] > 0]

    def done(self, h):
        return h["left"] <= 0


def test_continuous_batching_joins_jobs_at_the_next_sweep():
    ex = FakeBatchExecutor()
    srv = serving.Server(ex, hbm_budget=100 * 100 * 100 * 100)
    jobs = [_job(0, 100, 100, 0.0, sweeps=3), _job(1, 100, 100, 1.0, sweeps=2),
            _job(2, 100, 100, 1.0, sweeps=4)]
    pending = list(jobs)
    t = 0.0
    while len(srv.done) < len(jobs):
        while pending and pending[0].arrival <= t:
            srv.submit(pending.pop(0))
        srv.poll(t)
        t += 1.0
        assert t < 20
    # job 0 alone in the first sweep, then 1 and 2 join; each job is in
    # exactly `sweeps` ticks
    assert ex.tick_log[0] == [0]
    assert ex.tick_log[1] == [0, 1, 2]
    for j in jobs:
        assert sum(j.job_id in tl for tl in ex.tick_log) == j.sweeps
    assert srv.used == 0
    assert max(len(tl) for tl in ex.tick_log) == 3


def test_close_releases_every_job_and_raises_the_first_error():
    class Failing(FakeExecutor):
        def finish(self, job, h):
            if job.job_id == 0:
                raise RuntimeError("boom")
            return {"ok": job.job_id}

    ex = Failing(ticks=100)
    srv = serving.Server(ex, hbm_budget=10 * 100 * 100 * 100)
    for k in range(3):
        srv.submit(_job(k, 100, 100, 0.0))
    srv.poll(0.0)
    assert len(srv.active) == 3
    with pytest.raises(RuntimeError):
        srv.close()
    assert not srv.active and srv.used == 0
