"""Host-side logic of the request loop (admission, ordering, retirement, failures, latency),
driven by a fake engine: no GPU."""

import numpy as np
import pytest

from paper_1903_04502_gb300.serve import Job, Server, device_footprint


class FakeClock:
    """Simulated time: every reading advances it by 0.1 ms (so idle waits end)."""

    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4
        return self.t


class FakeEngine:
    """Each resident job's relative change after i iterations is 1 / (i + 1)."""

    def __init__(self, clock, fail_sizes=()):
        self.clock = clock
        self.iters = {}
        self.fail_sizes = set(fail_sizes)
        self.started = []
        self.steps = []

    def start(self, job):
        if job.n_side in self.fail_sizes:
            raise ValueError("bad coverage")
        self.iters[job.job_id] = 0
        self.started.append(job.job_id)

    def step(self, k):
        self.steps.append((k, sorted(self.iters)))
        for j in self.iters:
            self.iters[j] += k
        self.clock.t += 0.001 * k

    def status(self, job):
        i = self.iters[job.job_id]
        return i, 1.0 / (i + 1)

    def finish(self, job):
        self.iters.pop(job.job_id)
        return np.zeros((job.n_side, job.n_side))

    def abort(self, job):
        self.iters.pop(job.job_id, None)


def job(n=64, M=1000, max_iter=50, rel_tol=0.0, arrival=0.0):
    return Job(uvw=np.zeros((M, 4), np.float32), y=np.zeros(M, np.complex64), n_side=n, eps=1.0,
               max_iter=max_iter, rel_tol=rel_tol, arrival=arrival)


def test_footprint_grows_with_size():
    assert device_footprint(64, 1000) < device_footprint(128, 1000) < device_footprint(128, 10**6)


def test_admission_respects_budget_and_arrival_order():
    clk = FakeClock()
    fp = device_footprint(64, 1000, 4, 9)
    eng = FakeEngine(clk)
    srv = Server(eng, hbm_budget=int(2.5 * fp), check_every=10, clock=clk)
    jobs = [srv.submit(job(max_iter=30)) for _ in range(5)]
    srv.tick()
    assert len(srv.active) == 2 and len(srv.queue) == 3          # only two fit
    while srv.queue or srv.active:
        srv.tick()
        assert srv.used <= srv.budget
        assert len(srv.active) <= 2
    assert eng.started == [j.job_id for j in jobs]                 # first come, first admitted
    assert all(j.iters == 30 for j in srv.done)
    assert srv.stats()["jobs"] == 5 and srv.max_resident == 2


def test_jobs_join_a_running_batch():
    clk = FakeClock()
    eng = FakeEngine(clk)
    srv = Server(eng, hbm_budget=10**12, check_every=5, clock=clk)
    a = srv.submit(job(max_iter=40))
    srv.tick()
    b = srv.submit(job(max_iter=40))
    srv.tick()
    # b joined while a was still running: they were stepped together
    assert eng.steps[1][1] == sorted([a.job_id, b.job_id])
    assert a in srv.active and b in srv.active


def test_convergence_retires_early_and_cap_is_exact():
    clk = FakeClock()
    srv = Server(FakeEngine(clk), hbm_budget=10**12, check_every=7, clock=clk)
    fast = srv.submit(job(max_iter=1000, rel_tol=0.05))   # 1/(i+1) < 0.05 once i >= 20
    capped = srv.submit(job(max_iter=23))
    while srv.active or srv.queue:
        srv.tick()
    assert fast.iters >= 20 and fast.iters < 30
    assert capped.iters == 23                               # steps never overshoot the cap


def test_failures_do_not_stop_the_server():
    clk = FakeClock()
    fp = device_footprint(64, 1000, 4, 9)
    srv = Server(FakeEngine(clk, fail_sizes={13}), hbm_budget=3 * fp, check_every=10, clock=clk)
    bad = srv.submit(job(n=13))
    huge = srv.submit(job(n=4096, M=10**9))
    good = srv.submit(job(max_iter=10))
    while srv.active or srv.queue:
        srv.tick()
    assert bad in srv.failed and "bad coverage" in bad.error
    assert huge in srv.failed and "budget" in huge.error
    assert good in srv.done and good.result.shape == (64, 64)
    assert srv.used == 0


def test_latency_from_arrival_to_result():
    clk = FakeClock()
    srv = Server(FakeEngine(clk), hbm_budget=10**12, check_every=10, clock=clk)
    arr = [job(max_iter=20, arrival=0.0), job(max_iter=20, arrival=0.005), job(max_iter=40, arrival=0.05)]
    done = srv.run(arr, idle_sleep=0.0)
    assert len(done) == 3
    for j in done:
        assert j.latency > 0 and j.done_at >= j.admitted_at >= j.arrival
    st = srv.stats()
    assert st["p50_ms"] <= st["p99_ms"]


class AsyncFakeEngine(FakeEngine):
    """Prepares a job over `delay` loop turns (as the GPU engine does on its worker thread);
    preparation of sizes in `fail_prepare` fails when the job is activated."""

    def __init__(self, clock, delay=3, fail_prepare=()):
        super().__init__(clock)
        self.delay = delay
        self.fail_prepare = set(fail_prepare)
        self.countdown = {}
        self.jobs = {}

    def start(self, job):
        self.countdown[job.job_id] = self.delay
        self.jobs[job.job_id] = job

    def poll_ready(self):
        ready = []
        for jid in list(self.countdown):
            self.countdown[jid] -= 1
            if self.countdown[jid] <= 0:
                ready.append(jid)
        return ready

    def activate(self, job):
        self.countdown.pop(job.job_id)
        if job.n_side in self.fail_prepare:
            raise MemoryError("gbri error -2: cudaMalloc: out of memory")
        super().start(job)


def test_asynchronous_preparation_and_failed_setup():
    clk = FakeClock()
    fp = device_footprint(64, 1000, 4, 9)
    eng = AsyncFakeEngine(clk, delay=3, fail_prepare={48})
    srv = Server(eng, hbm_budget=3 * fp, check_every=5, clock=clk)
    a = srv.submit(job(max_iter=20))
    bad = srv.submit(job(n=48, max_iter=20))
    b = srv.submit(job(max_iter=20))
    assert srv.tick() == -1                 # admitted, still being prepared: nothing to step
    assert len(srv.preparing) == 3 and not srv.active
    while srv.queue or srv.preparing or srv.active:
        srv.tick()
        assert srv.used <= srv.budget
    assert bad in srv.failed and "out of memory" in bad.error
    assert a in srv.done and b in srv.done and srv.used == 0
    assert all(j.admitted_at > 0 for j in (a, b))
