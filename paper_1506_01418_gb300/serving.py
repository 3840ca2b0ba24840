"""Serving loop: factorisation jobs admitted continuously under an HBM budget.

Each request is one dense non-negative factorisation job (a spectrogram-like
V of its own size, Tweedie power, rank K and number of sweeps).  The server
admits waiting jobs in arrival order whenever the device memory they will
hold (`psgld_estimate_device_bytes`) fits in what the budget has left and a
slot is free; an admitted job gets its own CUDA stream and library context,
its data and initial factors are put on the device, and all its sweeps are
enqueued at once, so jobs that arrive while others run overlap with them on
the device.  The loop only polls completion events; a finished job's
posterior means are read back and its context (and memory, through the
caching allocator) released, which lets the next jobs in.  A standing chain
(a job without an end) can share the device: the loop keeps one sweep of it
queued at all times.

With `BatchedGpuExecutor` the jobs' part-steps share launches instead
(continuous batching at sweep granularity): every admitted job joins the
next sweep of one shared batch, and each loop iteration that finds fewer
than three batch sweeps in flight enqueues one more over all unfinished jobs
(per part one tensor-core gradient launch per K class and one update
launch, through psgld_batch_sweep).  Jobs arriving meanwhile join at the
next sweep; a finished job leaves the batch and its memory is released.

The scheduler (`Server`) is separate from the executor that touches the GPU,
so its admission and accounting logic runs on the CPU with a stand-in
executor.  Latency of a job = completion time - arrival time on the host
clock.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time
from typing import Callable, Optional

import numpy as np


@dataclasses.dataclass
class Job:
    """One factorisation request."""
    job_id: int
    I: int
    J: int
    K: int
    B: int
    p: float
    phi: float = 1.0
    sweeps: Optional[int] = 20         # None: a standing chain that never ends
    burn_in: int = 10
    seed: int = 0
    eps: float = 1e-4
    lam: float = 1.0
    init_scale: float = 0.5
    dense_path: int = 1
    dense_v_bf16: int = 0
    max_sms: int = 0                   # > 0: SMs the two-sided kernel may hold (standing chains)
    dense_share_e: int = -1            # the two-sided kernel's mode (-1: the library's rule)
    arrival: float = 0.0               # seconds from the start of the trace
    data_seed: int = 0
    # filled in by the server
    admitted: Optional[float] = None
    finished: Optional[float] = None
    result: Optional[dict] = None

    @property
    def entries(self) -> int:
        return self.I * self.J


class Server:
    """Admission and accounting; `executor` does the device work.

    executor.estimate(job) -> bytes the job will hold on the device
    executor.start(job) -> handle          (enqueues all of the job's work)
    executor.done(handle) -> bool          (non-blocking)
    executor.finish(job, handle) -> dict   (results; frees the job's memory)
    executor.step_standing(job, handle)    (keep a standing chain's sweep queued)
    executor.tick()                        (optional: called once per poll, after
                                            admission; a batching executor
                                            advances its jobs here)
    """

    def __init__(self, executor, hbm_budget: int, max_active: int = 64):
        self.ex = executor
        self.budget = int(hbm_budget)
        self.max_active = int(max_active)
        self.waiting: collections.deque = collections.deque()
        self.active: dict = {}               # job_id -> (job, handle, bytes)
        self.done: list = []
        self.used = 0
        self.peak_used = 0

    def submit(self, job: Job):
        self.waiting.append(job)

    def poll(self, now: float):
        """Finish completed jobs, then admit waiting jobs in order while they
        fit.  Returns the jobs finished in this call."""
        finished = []
        for jid in list(self.active):
            job, h, nbytes = self.active[jid]
            if job.sweeps is None:
                self.ex.step_standing(job, h)
                continue
            if self.ex.done(h):
                job.result = self.ex.finish(job, h)
                job.finished = now
                del self.active[jid]
                self.used -= nbytes
                self.done.append(job)
                finished.append(job)
        tick = getattr(self.ex, "tick", None)
        while self.waiting and len(self.active) < self.max_active:
            job = self.waiting[0]
            nbytes = int(self.ex.estimate(job))
            if nbytes > self.budget:
                raise ValueError(f"job {job.job_id} needs {nbytes} bytes, more than the whole budget")
            if self.used + nbytes > self.budget:
                break                        # in order: wait for memory to free up
            self.waiting.popleft()
            job.admitted = now
            self.active[job.job_id] = (job, self.ex.start(job), nbytes)
            self.used += nbytes
            self.peak_used = max(self.peak_used, self.used)
        if tick is not None:
            tick()
        return finished

    def run(self, jobs, clock: Callable[[], float] = time.perf_counter, idle_sleep: float = 1e-4,
            timeout: float = 600.0):
        """Replay `jobs` (sorted by arrival) in real time until every finite
        job has finished.  Returns the wall time from the first arrival."""
        pending = collections.deque(sorted(jobs, key=lambda j: j.arrival))
        n_finite = sum(1 for j in jobs if j.sweeps is not None)
        t0 = clock()
        while True:
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                self.submit(pending.popleft())
            self.poll(now)
            if not pending and sum(1 for j in self.done if j.sweeps is not None) == n_finite:
                break
            if now > timeout:
                raise TimeoutError("serving trace did not finish")
            if idle_sleep:
                time.sleep(idle_sleep)
        return clock() - t0

    def close(self):
        """Release every active job (after an error, or at the end); the
        first error raised while releasing is raised after all are done."""
        first = None
        for jid in list(self.active):
            job, h, nbytes = self.active.pop(jid)
            try:
                self.ex.finish(job, h)
            except Exception as e:          # keep releasing the others
                first = first or e
            finally:
                self.used -= nbytes
        if first is not None:
            raise first

    def stop_standing(self):
        """Finish standing chains (after a trace); returns their results."""
        out = []
        for jid in list(self.active):
            job, h, nbytes = self.active[jid]
            if job.sweeps is None:
                job.result = self.ex.finish(job, h)
                del self.active[jid]
                self.used -= nbytes
                out.append(job)
        return out


def latency_summary(jobs) -> dict:
    lat = np.array([j.finished - j.arrival for j in jobs if j.finished is not None])
    if lat.size == 0:
        return {"n": 0}
    return {"n": int(lat.size), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
            "max_s": float(lat.max())}


def poisson_trace(rate: float, duration: float, seed: int, job_factory) -> list:
    """Arrival times of a Poisson process of `rate` per second over
    `duration` seconds; job_factory(index, arrival, rng) makes each job."""
    rng = np.random.Generator(np.random.Philox(seed))
    jobs, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        jobs.append(job_factory(len(jobs), t, rng))
    return jobs


def mixed_job_factory(sweeps: int = 20, burn_in: int = 10, B: int = 8, eps: float = 1e-4):
    """The serving workload's job mix: I in {257, 513, 1025}, J log-uniform
    on [500, 20000], Tweedie p in {1, 1.5}, K in {16, 64}."""
    def make(index, arrival, rng):
        I = int(rng.choice([257, 513, 1025]))
        J = int(round(math.exp(rng.uniform(math.log(500), math.log(20000)))))
        return Job(job_id=index, I=I, J=J, K=int(rng.choice([16, 64])), B=B,
                   p=float(rng.choice([1.0, 1.5])), sweeps=sweeps, burn_in=burn_in, eps=eps,
                   seed=1000 + index, data_seed=index, arrival=arrival)
    return make


class GpuExecutor:
    """Runs jobs on one GPU through the C ABI: one stream and one context per
    job, memory from PyTorch's caching allocator (a finished job's memory is
    reused without a device-wide wait)."""

    def __init__(self, device=None):
        import torch

        from . import psgld as P
        self.torch = torch
        self.P = P
        self.dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        P.use_torch_allocator(self.dev.index)

    def estimate(self, job: Job) -> int:
        nbytes = self.P.psgld_estimate_device_bytes(job.I, job.J, job.K, job.B, 0, job.dense_path,
                                                    job.dense_v_bf16)
        return nbytes + 4 * job.I * job.J          # the caller-side V the job is given

    def _data(self, job: Job):
        from . import datagen
        torch = self.torch
        if job.p == 1.0:
            V = datagen.dense_poisson_device(job.I, job.J, 8, job.data_seed, self.dev)
        elif 1.0 < job.p < 2.0:
            # the compound Poisson-gamma law of the job's own power and
            # dispersion (exact zeros included)
            V = datagen.dense_compound_poisson_device(job.I, job.J, 8, job.data_seed, self.dev,
                                                      p=job.p, phi=job.phi)
        else:
            V = datagen.dense_gamma_device(job.I, job.J, 8, job.data_seed, self.dev)
        W0, H0 = datagen.init_factors(job.I, job.J, job.K, job.seed, scale=job.init_scale, nonneg=True)
        return V, torch.from_numpy(W0).to(self.dev, non_blocking=True), \
            torch.from_numpy(H0.T.copy()).to(self.dev, non_blocking=True)

    def start(self, job: Job):
        torch = self.torch
        # finite jobs ahead of a standing chain when both have work queued
        stream = torch.cuda.Stream(self.dev, priority=0 if job.sweeps is None else -1)
        with torch.cuda.stream(stream):
            V, W0, Ht0 = self._data(job)
            ctx = self.P.PSGLD(job.I, job.J, job.K, job.B, job.p, job.phi,
                               prior_kind=self.P.PSGLD_PRIOR_EXPONENTIAL, lambda_w=job.lam,
                               lambda_h=job.lam, seed=job.seed, eps=job.eps, use_graphs=1,
                               burn_in_sweeps=job.burn_in, dense_path=job.dense_path,
                               dense_v_bf16=job.dense_v_bf16, max_sms=job.max_sms,
                               dense_share_e=job.dense_share_e)
            ctx.set_data_dense(V, stream.cuda_stream)
            ctx.set_factors(W0, Ht0, stream.cuda_stream)
            del V, W0, Ht0
            n = job.sweeps if job.sweeps is not None else 1
            ctx.sweep(n, stream.cuda_stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        return {"ctx": ctx, "stream": stream, "event": ev, "sweeps_queued": n}

    def done(self, h) -> bool:
        return h["event"].query()

    def step_standing(self, job: Job, h):
        if h["event"].query():
            torch = self.torch
            h["ctx"].sweep(1, h["stream"].cuda_stream)
            h["event"] = torch.cuda.Event()
            h["event"].record(h["stream"])
            h["sweeps_queued"] += 1

    def finish(self, job: Job, h) -> dict:
        h["event"].synchronize()
        Wm, Wv, Hm, Hv, n = h["ctx"].posterior_mean()
        out = {"Wmean": Wm, "Hmean": Hm, "n_samples": n, "sweeps": h["sweeps_queued"]}
        h["ctx"].close()
        return out


class BatchedGpuExecutor(GpuExecutor):
    """Continuous batching: the part-steps of all admitted jobs share
    launches.  Jobs run on one stream; each tick (when fewer than
    `max_inflight` batch sweeps are queued) enqueues one psgld_batch_sweep
    over every unfinished job that is set up, so each advances by one sweep
    per tick (each job on the tensor-core kernel its shape selects; jobs on
    the same kernel variant share its launches).  A job's set-up (device
    data, context, input checks) and its read-back and teardown run on two
    worker threads, so the loop that enqueues the batch sweeps does not wait
    for them.  Standing chains run on their own streams as in GpuExecutor."""

    def __init__(self, device=None, max_inflight: int = 3, sweeps_per_tick: int = 1):
        import concurrent.futures as cf
        super().__init__(device)
        self.sweeps_per_tick = int(sweeps_per_tick)
        torch = self.torch
        self.stream = torch.cuda.Stream(self.dev, priority=-1)   # the batch's sweeps
        self.adm = torch.cuda.Stream(self.dev, priority=-1)      # admitted jobs' data and set-up
        self.setup_pool = cf.ThreadPoolExecutor(max_workers=1)
        self.teardown_pool = cf.ThreadPoolExecutor(max_workers=1)
        self.members: list = []
        self.inflight: collections.deque = collections.deque()
        self.max_inflight = int(max_inflight)
        self.ticks = 0
        self.batch_sizes: list = []

    @staticmethod
    def batchable(job: Job) -> bool:
        return job.sweeps is not None and job.dense_path != 0

    def _setup(self, job: Job, h):
        torch = self.torch
        torch.cuda.set_device(self.dev)
        with torch.cuda.stream(self.adm):
            V, W0, Ht0 = self._data(job)
            ctx = self.P.PSGLD(job.I, job.J, job.K, job.B, job.p, job.phi,
                               prior_kind=self.P.PSGLD_PRIOR_EXPONENTIAL, lambda_w=job.lam,
                               lambda_h=job.lam, seed=job.seed, eps=job.eps, use_graphs=0,
                               burn_in_sweeps=job.burn_in, dense_path=job.dense_path,
                               dense_v_bf16=job.dense_v_bf16)
            ctx.set_data_dense(V, self.adm.cuda_stream)
            ctx.set_factors(W0, Ht0, self.adm.cuda_stream)
            del V, W0, Ht0
            ev = torch.cuda.Event()
            ev.record(self.adm)
        h["ctx"] = ctx
        h["ready_event"] = ev

    def _teardown(self, h) -> dict:
        self.torch.cuda.set_device(self.dev)
        h["event"].synchronize()
        Wm, Wv, Hm, Hv, n = h["ctx"].posterior_mean()
        out = {"Wmean": Wm, "Hmean": Hm, "n_samples": n, "sweeps": h["sweeps_queued"]}
        h["ctx"].close()
        return out

    def start(self, job: Job):
        if not self.batchable(job):
            return super().start(job)
        h = {"ctx": None, "left": job.sweeps, "batched": True, "event": None, "sweeps_queued": 0,
             "joined": False}
        h["setup"] = self.setup_pool.submit(self._setup, job, h)
        self.members.append(h)
        return h

    def tick(self):
        """One more batch sweep over every unfinished job that is set up,
        unless `max_inflight` are already queued.  (Topping the queue up on
        every call was measured worse: jobs admitted meanwhile joined later,
        and the standing chain lost the SMs to the always-busy batch
        stream.)"""
        while self.inflight and self.inflight[0].query():
            self.inflight.popleft()
        if len(self.inflight) >= self.max_inflight or not self.members:
            time.sleep(0)                         # let the worker threads run
            return
        live = []
        for h in self.members:
            f = h["setup"]
            if not f.done():
                continue
            f.result()                            # a failed set-up raises here
            if not h["joined"]:
                self.stream.wait_event(h["ready_event"])
                h["joined"] = True
            live.append(h)
        if not live:
            time.sleep(0)
            return
        torch = self.torch
        # up to sweeps_per_tick sweeps in one call, never past a member's last
        k = max(1, min([self.sweeps_per_tick] + [h["left"] for h in live]))
        self.P.psgld_batch_sweep([h["ctx"] for h in live], k, self.stream.cuda_stream)
        ev = torch.cuda.Event()
        ev.record(self.stream)
        for h in live:
            h["left"] -= k
            h["sweeps_queued"] += k
            if h["left"] == 0:
                h["event"] = ev
                h["teardown"] = self.teardown_pool.submit(self._teardown, h)
        self.members = [h for h in self.members if h["left"] > 0]
        self.inflight.append(ev)
        self.ticks += k
        self.batch_sizes.append(len(live))

    def done(self, h) -> bool:
        if not h.get("batched"):
            return super().done(h)
        return "teardown" in h and h["teardown"].done()

    def shutdown(self):
        """Stop the worker threads (after the server has released its jobs)."""
        self.setup_pool.shutdown(wait=True)
        self.teardown_pool.shutdown(wait=True)

    def finish(self, job: Job, h) -> dict:
        if not h.get("batched"):
            return super().finish(job, h)
        if "teardown" in h:
            return h["teardown"].result()
        # released before its last sweep (close after an error)
        self.members = [m for m in self.members if m is not h]
        h["setup"].result()                  # a failed set-up raises here (nothing to close)
        self.stream.synchronize()
        out = {"sweeps": h["sweeps_queued"]}
        h["ctx"].close()
        return out
