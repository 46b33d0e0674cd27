"""Served simulation jobs with continuous batching.

Jobs (workloads.Job: model, L, T, Delta, seed, sweeps, arrival time) arrive
as a stream.  The server loop works in steps.  At every step boundary it
admits arrived jobs first-come-first-served while their device footprint
fits the memory budget (a job's lattice and per-job workspace stay resident
on the device until the job ends), then advances every resident job in one
runner launch (many lattices, one persistent kernel), each by as many
sweeps as fit the step's work budget without passing its next measurement
point.  Measurements follow section 3.3's log-spaced times in the form this
library uses: after 1, 2, 4, 8, ... completed sweeps a job's C(r) is taken
along both axes for r <= min(L/2, rmax_cap).  The exact (M, B, Q) of every
sweep are recorded.  A finished job releases its memory at once, so jobs
that arrived meanwhile are admitted at the next step and their work
overlaps with the jobs already on the device.

Every job's results equal those of the same job run alone on the plain
path (run_sequential), because the runner reproduces lat_sweep bit for bit.
The engine is a parameter so that the scheduling logic can be tested on the
CPU with a fake engine.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class JobResult:
    job: object
    admitted: float = -1.0
    completed: float = -1.0
    obs: list = field(default_factory=list)      # per-sweep record arrays, in order
    corr: dict = field(default_factory=dict)     # completed sweeps -> (cx, cy)
    final_hash: int = 0
    status: str = "done"                         # "done", "failed" or "cancelled"
    error: str = ""                              # why a job failed

    @property
    def latency(self) -> float:
        return self.completed - self.job.arrival


class Deferred:
    """A result the device writes asynchronously (a correlation or a final
    hash): settle() fills .value once the engine's stream has passed the
    work, and returns it."""

    __slots__ = ("value", "_fill")

    def __init__(self, fill):
        self.value, self._fill = None, fill

    def settle(self):
        if self._fill is not None:
            self.value, self._fill = self._fill(), None
        return self.value


def resolve(x):
    return x.settle() if isinstance(x, Deferred) else x


def next_measurement(done: int) -> int:
    """The next power of two strictly above `done` (measurement after 1, 2, 4, ... sweeps)."""
    p = 1
    while p <= done:
        p *= 2
    return p


def plan_step(active, budget_updates: float, max_sweeps: int, policy: str = "fair"):
    """Sweeps per resident job for one step.

    active: list of (L, sweeps_done, sweeps_total).  A job's cap is the
    smallest of max_sweeps, its remaining sweeps and the sweeps to its next
    measurement point.
      fair: every job gets the same quota q = budget / sum(L^2) (at least 1),
            capped.
      srpt: jobs are served in order of increasing remaining work
            (L^2 x remaining sweeps); each takes its cap while the budget
            lasts, and every job gets at least one sweep, so none starves."""
    if not active:
        return []
    caps = [max(0, min(max_sweeps, total - done, next_measurement(done) - done)) for (_, done, total) in active]
    if policy == "fair":
        tot = float(sum(L * L for (L, _, _) in active))
        q = int(max(1, min(max_sweeps, budget_updates // max(tot, 1.0))))
        return [min(q, c) for c in caps]
    if policy != "srpt":
        raise ValueError("unknown policy %r" % policy)
    order = sorted(range(len(active)), key=lambda i: (active[i][0] ** 2 * (active[i][2] - active[i][1]), i))
    out = [0] * len(active)
    left = float(budget_updates)
    for i in order:
        L2 = float(active[i][0]) ** 2
        k = min(caps[i], max(1, int(left // L2)))
        out[i] = k
        left -= k * L2
    return out


class GpuEngine:
    """The device side: lattices in torch-owned buffers, one runner, all on
    the runner's stream.  A step is submitted and collected; the
    measurements and final hashes of a step are only enqueued (results in
    page-locked buffers, returned as Deferred), so the device runs them while
    the host plans the next step, and the next step's collect, which waits
    for the stream, settles them.  A finished lattice is closed after that
    collect."""

    def __init__(self, max_jobs: int, max_step_sweeps: int, rmax_cap: int = 1024, tiles=None):
        from . import binding as b
        self.b = b
        self.runner = b.Runner(max_jobs, max_step_sweeps)
        if tiles:
            for (m, L), t in tiles.items():
                self.runner.set_tile(m, L, t)
        self.rmax_cap = rmax_cap
        self.launches = 0  # kernels launched: quench, runner runs, correlation, hash
        self.pending = []   # Deferred results written by enqueued work
        self.retired = []   # finished lattices, closed once their hash has landed
        self.pool = {}      # page-locked int64 buffers by length, for reuse

    def _pinned(self, n: int):
        import torch
        free = self.pool.setdefault(n, [])
        t = free.pop() if free else torch.empty(n, dtype=torch.int64, pin_memory=True)
        return t, t.numpy()

    def _release_pinned(self, n: int, t) -> None:
        self.pool[n].append(t)

    def settle(self) -> None:
        """Wait for the stream, fill every pending result and close retired lattices."""
        self.runner.stream.synchronize()
        self._settled()

    def _settled(self) -> None:
        for d in self.pending:
            d.settle()
        self.pending = []
        for h in self.retired:
            h.close()
        self.retired = []

    def footprint(self, job) -> int:
        return self.b.lat_footprint(self.b.make_params(job.model, job.L, job.T, job.seed, Delta=job.Delta))

    def create(self, job):
        self.launches += 1
        return self.b.Lattice(job.model, job.L, job.T, job.seed, Delta=job.Delta, stream=self.runner.stream)

    def advance(self, handles, nsweeps):
        self.launches += 1 if any(nsweeps) else 0
        self.runner.submit(handles, nsweeps)
        obs = self.runner.collect(nsweeps)
        self._settled()  # the collect waited for the stream: earlier measurements and hashes are in
        return obs

    def measure(self, h):
        rmax = min(h.L // 2, self.rmax_cap)
        self.launches += 1 if rmax <= 32 else 2
        n = 2 * (rmax + 1)
        t, buf = self._pinned(n)
        self.b.lat_correlation_async(h.handle, rmax, buf[:rmax + 1], buf[rmax + 1:])

        def fill():
            out = (buf[:rmax + 1].copy(), buf[rmax + 1:].copy())
            self._release_pinned(n, t)
            return out
        d = Deferred(fill)
        self.pending.append(d)
        return d

    def sweep(self, h, n: int):
        """The one-lattice path (sequential baseline): two phase launches per sweep."""
        self.launches += 2 * n
        return h.sweep(n)

    def finish(self, h):
        self.launches += 1
        t, buf = self._pinned(1)
        self.b.lat_hash_async(h.handle, buf.view(np.uint64))

        def fill():
            v = int(buf.view(np.uint64)[0])
            self._release_pinned(1, t)
            return v
        d = Deferred(fill)
        self.pending.append(d)
        self.retired.append(h)
        return d

    def abort(self, h) -> None:
        h.close()

    def close(self):
        self.settle()
        self.runner.close()


class Server:
    """Continuous batching: admits arriving jobs first-come-first-served while
    their device footprint fits mem_budget (at most max_batch resident), and
    advances every resident job in one engine step at a time.  The sweeps a
    job gets per step come from plan_step (policy "srpt" or "fair", at most
    max_step_sweeps); C(r) is measured after sweeps 1, 2, 4, ... and a job
    leaves, freeing its memory, when its sweeps are done."""

    def __init__(self, engine, mem_budget: int, max_batch: int, step_updates: float = 2e9,
                 max_step_sweeps: int = 16, clock=time.perf_counter, sleep=time.sleep, policy: str = "srpt"):
        self.engine = engine
        self.mem_budget = mem_budget
        self.max_batch = max_batch
        self.step_updates = step_updates
        self.max_step_sweeps = max_step_sweeps
        self.clock, self.sleep = clock, sleep
        self.policy = policy
        self.steps = 0
        self.peak_mem = 0
        self.peak_batch = 0

    def _release(self, h):
        """Close a job's lattice without reading a result (failure or cancel)."""
        abort = getattr(self.engine, "abort", None)
        try:
            if abort is not None:
                abort(h)
            else:
                self.engine.finish(h)
        except Exception:
            pass

    def run(self, jobs, cancels=None):
        """Serve `jobs`; cancels maps a job id to the time (seconds after the
        start) at which it is withdrawn, whether it is still waiting, running
        or not yet arrived.  A job whose lattice cannot be created, or whose
        step or measurement raises, ends with status "failed"; the other jobs
        go on."""
        jobs = sorted(jobs, key=lambda j: (j.arrival, j.id))
        arrivals = deque(jobs)
        pending = deque()
        active = []  # [result, handle, done, footprint]
        results = {}
        cancel_at = dict(cancels or {})
        used = 0
        t0 = self.clock()

        def end(r, status, error=""):
            r.status, r.error = status, error
            r.completed = self.clock() - t0

        while arrivals or pending or active:
            now = self.clock() - t0
            while arrivals and arrivals[0].arrival <= now:
                j = arrivals.popleft()
                results[j.id] = JobResult(j)
                pending.append(j)
            # withdrawals
            if cancel_at:
                for j in [j for j in pending if cancel_at.get(j.id, float("inf")) <= now]:
                    pending.remove(j)
                    end(results[j.id], "cancelled")
                keep = []
                for a in active:
                    if cancel_at.get(a[0].job.id, float("inf")) <= now:
                        self._release(a[1])
                        used -= a[3]
                        end(a[0], "cancelled")
                    else:
                        keep.append(a)
                active = keep
            # admission: first come, first served, by device footprint
            while pending and len(active) < self.max_batch:
                j = pending[0]
                fp = self.engine.footprint(j)
                if fp > self.mem_budget:
                    raise ValueError("job %d needs %d bytes, more than the whole budget" % (j.id, fp))
                if used + fp > self.mem_budget:
                    break
                pending.popleft()
                r = results[j.id]
                r.admitted = self.clock() - t0
                try:
                    h = self.engine.create(j)
                except Exception as e:  # e.g. the device allocation failed
                    end(r, "failed", repr(e))
                    continue
                used += fp
                self.peak_mem = max(self.peak_mem, used)
                active.append([r, h, 0, fp])
            if not active:
                if arrivals:
                    self.sleep(max(0.0, arrivals[0].arrival - (self.clock() - t0)))
                continue
            self.peak_batch = max(self.peak_batch, len(active))
            plan = plan_step([(a[0].job.L, a[2], a[0].job.sweeps) for a in active], self.step_updates,
                             self.max_step_sweeps, self.policy)
            try:
                obs = self.engine.advance([a[1] for a in active], plan)
            except Exception as e:  # e.g. a device wait timed out: these lattices are in doubt
                for a in active:
                    self._release(a[1])
                    used -= a[3]
                    end(a[0], "failed", repr(e))
                active = []
                self.steps += 1
                continue
            self.steps += 1
            keep = []
            for a, k, o in zip(active, plan, obs):
                r, h = a[0], a[1]
                if k:
                    r.obs.append(o)
                    a[2] += k
                try:
                    if a[2] > 0 and (a[2] & (a[2] - 1)) == 0 and a[2] not in r.corr:
                        r.corr[a[2]] = self.engine.measure(h)
                    if a[2] >= r.job.sweeps:
                        r.final_hash = self.engine.finish(h)
                        end(r, "done")
                        used -= a[3]
                        continue
                except Exception as e:
                    self._release(h)
                    used -= a[3]
                    end(r, "failed", repr(e))
                    continue
                keep.append(a)
            active = keep
        settle = getattr(self.engine, "settle", None)
        if settle is not None:
            settle()
        self.wall = self.clock() - t0
        out = [results[j.id] for j in jobs]
        for r in out:
            r.corr = {t: resolve(v) for t, v in r.corr.items()}
            r.final_hash = resolve(r.final_hash)
        return out


def run_sequential(engine, jobs, clock=time.perf_counter, sleep=time.sleep):
    """The plain baseline: jobs one at a time in arrival order, each alone on
    the one-lattice path (lat_sweep up to each measurement point)."""
    jobs = sorted(jobs, key=lambda j: (j.arrival, j.id))
    out = []
    t0 = clock()
    for j in jobs:
        now = clock() - t0
        if now < j.arrival:
            sleep(j.arrival - now)
        r = JobResult(j, admitted=clock() - t0)
        h = engine.create(j)
        done = 0
        while done < j.sweeps:
            k = min(j.sweeps, next_measurement(done)) - done
            r.obs.append(engine.sweep(h, k) if hasattr(engine, "sweep") else h.sweep(k))
            done += k
            if (done & (done - 1)) == 0:
                r.corr[done] = engine.measure(h)
        r.final_hash = engine.finish(h)
        settle = getattr(engine, "settle", None)
        if settle is not None:   # the job's results are in and its lattice is released
            settle()
        r.corr = {t: resolve(v) for t, v in r.corr.items()}
        r.final_hash = resolve(r.final_hash)
        r.completed = clock() - t0
        out.append(r)
    return out


def summarize(results, wall: float) -> dict:
    """Latency and throughput over the jobs that completed; counts of the others."""
    done = [r for r in results if r.status == "done"]
    lat = np.array([r.latency for r in done]) if done else np.zeros(1)
    updates = float(sum(r.job.L * r.job.L * r.job.sweeps for r in done))
    out = {"jobs": len(results), "p50_latency_s": float(np.percentile(lat, 50)),
           "p99_latency_s": float(np.percentile(lat, 99)), "wall_s": wall,
           "updates": updates, "flips_per_ns": updates / wall / 1e9}
    for status in ("failed", "cancelled"):
        n = sum(1 for r in results if r.status == status)
        if n:
            out[status] = n
    return out


def digest(r: JobResult) -> str:
    """SHA-256 over everything a job returns (status, per-sweep records,
    C(r) at every measurement point, final hash): two runs of a job are
    bit-identical iff their digests are equal (up to a hash collision).  Lets
    the served and the sequential runs be compared across processes."""
    import hashlib
    h = hashlib.sha256()
    h.update(r.status.encode())
    h.update(int(r.final_hash).to_bytes(8, "little"))
    for o in r.obs:
        h.update(np.ascontiguousarray(o).tobytes())
    for t in sorted(r.corr):
        h.update(int(t).to_bytes(8, "little"))
        for a in r.corr[t]:
            h.update(np.ascontiguousarray(a, dtype=np.int64).tobytes())
    return h.hexdigest()


def same_results(a: JobResult, b: JobResult) -> bool:
    """Bit-exact comparison of two runs of one job."""
    oa = np.concatenate(a.obs) if a.obs else np.zeros(0)
    ob = np.concatenate(b.obs) if b.obs else np.zeros(0)
    if a.final_hash != b.final_hash or not np.array_equal(oa, ob) or a.corr.keys() != b.corr.keys():
        return False
    return all(np.array_equal(a.corr[t][0], b.corr[t][0]) and np.array_equal(a.corr[t][1], b.corr[t][1])
               for t in a.corr)
