"""Request loop for imaging jobs: HBM-budget admission and continuous batching.

Jobs (one imaging problem each: coverage, data, dictionary, stopping rule) arrive
over time.  The server admits queued jobs in arrival order while their estimated
device footprint fits the HBM budget, keeps each admitted job's plan, data,
iterate and dual variables resident on the device, and advances every resident
job together: each step is one launch of the batch graph (``Batch.step``), so jobs
of different sizes share the GPU.  Every ``check_every`` iterations the server
reads each job's FP64 relative iterate change, retires the jobs that converged or
reached their iteration cap (image copied to the host), frees their memory and
admits waiting jobs at once -- jobs join and leave the running batch between
steps.  Latency is measured from arrival to result on the host.

The GPU engine prepares an admitted job (plan creation, the power method for
||Phi||^2, solver state) on a worker thread with its own CUDA stream, and tears
retired jobs down there too: the loop thread only launches batch steps, reads the
convergence scalars and copies finished images, so resident jobs keep running
while new ones are set up.  A job joins the batch at the first step after its
preparation has finished.  Job inputs may be host arrays or device tensors.

The device work is behind a small engine interface so that the scheduling logic
(admission, ordering, retirement, failures, latency bookkeeping) can be exercised
without a GPU.
"""

import collections
import time
from dataclasses import dataclass

import numpy as np


@dataclass(eq=False)
class Job:
    """One reconstruction request.  uvw: float32 [M, 4] {u, v, w, weight}; y: complex64 [M]."""
    uvw: np.ndarray
    y: np.ndarray
    n_side: int
    eps: float
    J: int = 4
    db_orders: tuple = (0, 1, 2, 3, 4, 5, 6, 7, 8)
    levels: int = 4
    max_iter: int = 300
    rel_tol: float = 1e-3
    op_norm_sq: float = 0.0
    gamma: float = 0.0
    deterministic: bool = False  # bitwise reproducible gridding (results equal alone and in the mix)
    arrival: float = 0.0
    job_id: int = -1
    # filled by the server
    result: object = None
    iters: int = 0
    rel_change: float = float("inf")
    error: str = ""
    admitted_at: float = 0.0
    done_at: float = 0.0

    @property
    def M(self):
        return int(self.uvw.shape[0])

    @property
    def latency(self):
        return self.done_at - self.arrival


def device_footprint(n_side, M, J=4, n_w=9, oversample=2, deterministic=False):
    """Upper estimate of the device bytes a resident job holds (plan, wavelets, solver state)."""
    K = oversample * n_side
    N = n_side * n_side
    # padded image 4 K^2, half spectrum 8 K (K/2 + 1), grid 8 K^2, the two cuFFT work areas
    # (bounded by 16 K^2 together: a plan at K = 4096, M = 2e6, J = 6 measured 534 MB in all
    # against this formula's 654 MB), tile tables, scalars
    plan = M * (8 + 4 + 8) + M // 2 * 8 + 20 * K * K + 8 * K + 16 * K * K + (8 * K * K // 64) + (1 << 20)
    plan_build = M * (16 + 4 + 4 + 4 + 8 + 4) + 8 * K * K  # transient during plan creation
    wav = 2 * max(1, n_w - 1) * 4 * N
    solver = M * 8 * 2 + N * 4 * (5 + n_w) + (1 << 20)
    if deterministic:  # one window slot per gridding work item (at most every tile plus the split pieces)
        plan += ((K // 16) ** 2 + M // 1024 + 1) * (16 + J - 1) ** 2 * 8 + 4 * (K // 16) ** 2
    return plan + max(plan_build - plan, 0) + wav + solver


class GpuEngine:
    """Device side of the server: resident solvers stepped together in one batch graph, with
    job set-up and teardown on a worker thread and its own CUDA stream."""

    def __init__(self, device=0, power_iters=50, power_tol=1e-4, workers=3, shared_pass=False):
        import concurrent.futures
        import threading
        import torch
        import paper_1903_04502_gb300 as g
        self.torch, self.g = torch, g
        self.device = torch.device("cuda", device)
        self.batch = g.Batch()
        # The batch's shared fused pass is off by default here: every change of membership would
        # rebuild it by a capture that waits for the workers' plan creation, stalling the
        # resident jobs (10 jobs/s: p50 379 ms, p99 684 ms with it against 207 / 462 ms without),
        # and it gains no throughput on this mix.
        self.shared_pass = bool(shared_pass)
        self.batch.set_shared_pass(self.shared_pass)
        self.state = {}
        self.pending = {}
        self.power_iters, self.power_tol = int(power_iters), float(power_tol)
        self._streams = threading.local()
        # plan creation and teardown free and synchronise device memory; a graph capture on
        # another thread (a job's iteration, or the batch's shared pass) must not overlap
        # them, so they take turns (the power method and
        # the solver state run concurrently on the workers' own streams)
        self._sync_lock = threading.Lock()
        self._rebuild = False  # the batch's membership changed since its last step
        self.worker = concurrent.futures.ThreadPoolExecutor(max_workers=max(1, int(workers)))

    def _stream(self):
        if not hasattr(self._streams, "s"):
            with self.torch.cuda.device(self.device):
                self._streams.s = self.torch.cuda.Stream(device=self.device)
        return self._streams.s

    def _prepare(self, job):
        torch, g = self.torch, self.g
        prep_stream = self._stream()
        with torch.cuda.device(self.device), torch.cuda.stream(prep_stream):
            if torch.is_tensor(job.uvw):
                uvw = job.uvw.to(self.device, torch.float32).contiguous()
            else:
                uvw = torch.from_numpy(np.ascontiguousarray(job.uvw, dtype=np.float32)).to(self.device)
            with self._sync_lock:
                plan = g.Plan(uvw, job.n_side, J=job.J, deterministic=job.deterministic)
            del uvw
            wav = g.Wavelet(job.n_side, job.levels, job.db_orders)
            if torch.is_tensor(job.y):
                y = job.y.to(self.device, torch.complex64).contiguous()
            else:
                y = torch.from_numpy(np.ascontiguousarray(job.y, dtype=np.complex64)).to(self.device)
            opn = job.op_norm_sq
            if opn <= 0:
                # step sizes need ||Phi||^2 to a few digits: the power method approaches it from
                # below, and stopping at 1e-4 relative change keeps tau (sigma1 + sigma2 ||Phi||^2) < 1
                opn, _ = g.op_norm(plan, self.power_iters, self.power_tol, seed=job.job_id)
            s = g.Solver(plan, wav, y, eps=job.eps, op_norm_sq=opn, gamma=job.gamma, max_iter=job.max_iter,
                         rel_tol=job.rel_tol)
            prep_stream.synchronize()
            # capture the iteration here: the loop thread then only composes captured graphs
            with self._sync_lock:
                s.capture()
            return plan, wav, s

    def start(self, job):
        """Begin preparing an admitted job (returns at once)."""
        self.pending[job.job_id] = self.worker.submit(self._prepare, job)

    def poll_ready(self):
        """Job ids whose preparation has finished (successfully or not)."""
        return [jid for jid, f in self.pending.items() if f.done()]

    def activate(self, job):
        """Add a prepared job to the running batch (raises if its preparation failed)."""
        plan, wav, s = self.pending.pop(job.job_id).result()
        self.state[job.job_id] = (plan, wav, s)
        self.batch.add(s)
        self._rebuild = True

    def step(self, n_iter):
        # after a change of membership the batch rebuilds its graph on this step, capturing the
        # shared pass's members: that capture takes its turn with plan creation and teardown
        if self._rebuild and self.shared_pass:
            with self._sync_lock:
                self.batch.step(n_iter)
        else:
            self.batch.step(n_iter)
        self._rebuild = False

    def status(self, job):
        return self.state[job.job_id][2].status()

    def _teardown(self, objs):
        with self._sync_lock:
            for o in objs:
                o.close()

    def finish(self, job):
        plan, wav, s = self.state.pop(job.job_id)
        x = s.x().cpu().numpy()
        self.batch.remove(s)
        self._rebuild = True
        self.worker.submit(self._teardown, (s, wav, plan))
        return x

    def abort(self, job):
        f = self.pending.pop(job.job_id, None)
        if f is not None:
            try:
                self.worker.submit(self._teardown, f.result()[::-1])
            except Exception:
                pass
            return
        st = self.state.pop(job.job_id, None)
        if st is None:
            return
        plan, wav, s = st
        try:
            self.batch.remove(s)
            self._rebuild = True
        except Exception:
            pass
        self.worker.submit(self._teardown, (s, wav, plan))

    def close(self):
        self.worker.shutdown(wait=True)


class Server:
    """Continuous-batching request loop with HBM-footprint admission (see the module docstring)."""

    def __init__(self, engine, hbm_budget, check_every=10, clock=time.perf_counter):
        self.engine = engine
        self.budget = int(hbm_budget)
        self.check_every = int(check_every)
        self.clock = clock
        self.queue = collections.deque()
        self.preparing = []          # admitted, set-up in progress (engines that prepare asynchronously)
        self.active = []
        self.done = []
        self.failed = []
        self.used = 0
        self.iterations = 0          # solver iterations run, summed over jobs
        self.vis_iterations = 0      # visibilities through Phi and Phi^dagger, summed
        self.max_resident = 0
        self._next_id = 0
        self._fp = {}

    def submit(self, job):
        job.job_id = self._next_id
        self._next_id += 1
        if not job.arrival:
            job.arrival = self.clock()
        self._fp[job.job_id] = device_footprint(job.n_side, job.M, job.J, len(job.db_orders),
                                                deterministic=job.deterministic)
        if self._fp[job.job_id] > self.budget:
            job.error = "job needs %d bytes, more than the whole budget of %d" % (self._fp[job.job_id], self.budget)
            job.done_at = self.clock()
            self.failed.append(job)
            return job
        self.queue.append(job)
        return job

    def _fail(self, job, e):
        job.error = "%s: %s" % (type(e).__name__, e)
        job.done_at = self.clock()
        self.failed.append(job)
        self.engine.abort(job)

    def _admit(self):
        # arrival order: the head of the queue waits until it fits (no overtaking); its memory
        # is reserved from admission on, while it is being prepared
        asynchronous = hasattr(self.engine, "poll_ready")
        while self.queue and self.used + self._fp[self.queue[0].job_id] <= self.budget:
            job = self.queue.popleft()
            try:
                self.engine.start(job)
            except Exception as e:  # bad input, allocation failure: the job fails, the server goes on
                self._fail(job, e)
                continue
            self.used += self._fp[job.job_id]
            if asynchronous:
                self.preparing.append(job)
            else:
                job.admitted_at = self.clock()
                self.active.append(job)
        if asynchronous and self.preparing:
            ready = set(self.engine.poll_ready())
            still = []
            for job in self.preparing:
                if job.job_id not in ready:
                    still.append(job)
                    continue
                try:
                    self.engine.activate(job)
                except Exception as e:  # set-up failed on the worker (allocation, bad input)
                    self.used -= self._fp[job.job_id]
                    self._fail(job, e)
                    continue
                job.admitted_at = self.clock()
                self.active.append(job)
            self.preparing = still
        self.max_resident = max(self.max_resident, len(self.active))

    def _retire(self):
        keep = []
        for job in self.active:
            it, rel = self.engine.status(job)
            job.iters, job.rel_change = it, rel
            if it >= job.max_iter or (job.rel_tol > 0 and rel < job.rel_tol):
                job.result = self.engine.finish(job)
                job.done_at = self.clock()
                self.used -= self._fp[job.job_id]
                self.done.append(job)
            else:
                keep.append(job)
        self.active = keep

    def tick(self):
        """Admit what fits, advance every resident job, retire finished ones.  Returns the
        number of iterations each resident job advanced (0 when idle, -1 while jobs are only
        being prepared)."""
        self._admit()
        if not self.active:
            if self.preparing:  # nothing to step until a prepared job is ready
                time.sleep(2e-4)
                return -1
            return 0
        k = min(self.check_every, min(j.max_iter - j.iters for j in self.active))
        k = max(1, k)
        self.engine.step(k)
        for j in self.active:
            self.iterations += k
            self.vis_iterations += k * j.M
        self._retire()
        return k

    def run(self, arrivals=(), idle_sleep=1e-3):
        """Serve ``arrivals`` (jobs with ``arrival`` times relative to the start, in order) and
        every job already queued, until all are done.  Returns the finished jobs."""
        pending = collections.deque(sorted(arrivals, key=lambda j: j.arrival))
        t0 = self.clock()
        for j in pending:
            j.arrival += t0
        while pending or self.queue or self.active or self.preparing:
            now = self.clock()
            while pending and pending[0].arrival <= now:
                self.submit(pending.popleft())
            if self.tick() == 0 and pending:
                time.sleep(min(idle_sleep, max(0.0, pending[0].arrival - self.clock())))
        return self.done

    def stats(self):
        lat = np.array([j.latency for j in self.done]) if self.done else np.zeros(0)
        return {
            "jobs": len(self.done),
            "failed": len(self.failed),
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
            "max_resident": self.max_resident,
        }
