"""Host-side logic of the served loop, on the CPU with a fake engine and a
virtual clock: admission by footprint (first come, first served, never over
budget), continuous batching (jobs that arrive while others run are admitted
at the next step), measurement points at 1, 2, 4, ... sweeps, and step
plans that never pass a measurement point or a job's end."""
import numpy as np
import pytest

from paper_2502_18624_gb300 import serve, workloads


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 0.0)


class FakeHandle:
    def __init__(self, job):
        self.job, self.L, self.done, self.closed = job, job.L, 0, False


class FakeEngine:
    """Records everything the server asks for; time advances with the work."""

    def __init__(self, clock, rate_updates_per_s=1e11):
        self.clock, self.rate = clock, rate_updates_per_s
        self.live, self.peak_live, self.events = 0, 0, []

    def footprint(self, job):
        return workloads.footprint_bytes(job) + 4096

    def create(self, job):
        self.live += self.footprint(job)
        self.peak_live = max(self.peak_live, self.live)
        self.events.append(("create", job.id, self.clock()))
        return FakeHandle(job)

    def advance(self, handles, nsweeps):
        assert len(set(map(id, handles))) == len(handles)
        work = 0.0
        out = []
        for h, k in zip(handles, nsweeps):
            assert not h.closed and 0 <= k and h.done + k <= h.job.sweeps
            rec = np.zeros(k, dtype=[("sweep", np.uint64)])
            rec["sweep"] = np.arange(h.done + 1, h.done + k + 1)
            h.done += k
            work += h.L * h.L * k
            out.append(rec)
        self.clock.t += work / self.rate + 1e-4
        return out

    def measure(self, h):
        self.events.append(("measure", h.job.id, h.done))
        return (np.array([h.done]), np.array([h.done]))

    def finish(self, h):
        assert h.done == h.job.sweeps
        h.closed = True
        self.live -= self.footprint(h.job)
        return h.job.id * 7 + h.done


def _jobs(n=60, seed=5):
    return workloads.served_jobs(n=n, rate=50.0, seed=seed, kmin=6, kmax=10, smin=3, smax=300)


def test_all_jobs_finish_with_every_sweep_and_measurement():
    clock = Clock()
    eng = FakeEngine(clock)
    srv = serve.Server(eng, mem_budget=600_000, max_batch=16, step_updates=5e6, max_step_sweeps=64,
                       clock=clock, sleep=clock.sleep)
    jobs = _jobs()
    res = srv.run(jobs)
    for r in res:
        sweeps = np.concatenate(r.obs)["sweep"]
        assert list(sweeps) == list(range(1, r.job.sweeps + 1))
        expect = [2 ** k for k in range(0, 20) if 2 ** k <= r.job.sweeps]
        assert sorted(r.corr) == expect
        assert r.final_hash == r.job.id * 7 + r.job.sweeps
        assert r.completed >= r.admitted >= r.job.arrival - 1e-12
    assert eng.live == 0


def test_memory_budget_is_never_exceeded_and_admission_is_fifo():
    clock = Clock()
    eng = FakeEngine(clock)
    budget = 400_000
    srv = serve.Server(eng, mem_budget=budget, max_batch=64, step_updates=5e6, max_step_sweeps=64,
                       clock=clock, sleep=clock.sleep)
    jobs = _jobs(80, 9)
    srv.run(jobs)
    assert eng.peak_live <= budget
    created = [e[1] for e in eng.events if e[0] == "create"]
    assert created == [j.id for j in sorted(jobs, key=lambda j: (j.arrival, j.id))]


def test_jobs_arriving_during_work_join_running_batches():
    clock = Clock()
    eng = FakeEngine(clock, rate_updates_per_s=2e9)
    srv = serve.Server(eng, mem_budget=10**9, max_batch=64, step_updates=2e6, max_step_sweeps=32,
                       clock=clock, sleep=clock.sleep)
    res = srv.run(_jobs(40, 3))
    # some job was admitted while another, admitted earlier, was still running
    overlap = any(b.admitted < a.completed and b.admitted > a.admitted for a in res for b in res)
    assert overlap and srv.peak_batch > 1


def test_oversized_job_is_rejected():
    clock = Clock()
    srv = serve.Server(FakeEngine(clock), mem_budget=1000, max_batch=4, clock=clock, sleep=clock.sleep)
    with pytest.raises(ValueError):
        srv.run([workloads.Job(0, 0, 4096, 2.0, 0.0, 1, 5, 0.0)])


@pytest.mark.parametrize("done,total,expect_cap", [(0, 10, 1), (1, 10, 1), (2, 10, 2), (5, 100, 3), (64, 70, 6)])
def test_plan_step_respects_measurements_and_ends(done, total, expect_cap):
    k = serve.plan_step([(64, done, total)], budget_updates=1e12, max_sweeps=1000)[0]
    assert k == expect_cap
    assert serve.next_measurement(done) - done >= k and total - done >= k


def test_plan_step_shares_the_budget():
    ks = serve.plan_step([(1024, 0, 10**6 - 1), (2048, 3, 10**6 - 1)], budget_updates=1024**2 * 5 * 10, max_sweeps=64)
    # quota = budget / (1024^2 + 2048^2) = 10, capped by the next measurement points (1 and 1)
    assert ks == [1, 1]
    ks = serve.plan_step([(1024, 64, 10**6 - 1), (2048, 64, 10**6 - 1)], budget_updates=1024**2 * 5 * 10,
                         max_sweeps=64)
    assert ks == [10, 10]


def test_plan_step_srpt_serves_short_jobs_first():
    # two big jobs and one small one; the budget covers the small job's cap and a few big sweeps
    active = [(4096, 10, 1000), (256, 3, 50), (4096, 100, 5000)]
    ks = serve.plan_step(active, budget_updates=4096**2 * 6 + 256**2, max_sweeps=64, policy="srpt")
    assert ks[1] == 1                     # capped by its next measurement point (4)
    assert ks[0] == 6 and ks[2] == 1      # the shorter big job takes the rest; the other keeps one sweep
    fair = serve.plan_step(active, budget_updates=4096**2 * 6 + 256**2, max_sweeps=64, policy="fair")
    assert fair == [2, 1, 2]             # q = floor(budget / sum L^2) = 2, capped
    with pytest.raises(ValueError):
        serve.plan_step(active, 1e9, 64, policy="lifo")


@pytest.mark.parametrize("policy", ["fair", "srpt"])
def test_both_policies_run_every_sweep_and_measurement(policy):
    clock = Clock()
    eng = FakeEngine(clock)
    srv = serve.Server(eng, mem_budget=600_000, max_batch=16, step_updates=5e6, max_step_sweeps=64,
                       clock=clock, sleep=clock.sleep, policy=policy)
    res = srv.run(_jobs())
    for r in res:
        assert list(np.concatenate(r.obs)["sweep"]) == list(range(1, r.job.sweeps + 1))
        assert sorted(r.corr) == [2 ** k for k in range(0, 20) if 2 ** k <= r.job.sweeps]
        assert r.final_hash == r.job.id * 7 + r.job.sweeps
    assert eng.live == 0


def test_srpt_lowers_the_median_latency_of_a_burst():
    lat = {}
    for policy in ("fair", "srpt"):
        clock = Clock()
        srv = serve.Server(FakeEngine(clock), mem_budget=10**12, max_batch=256, step_updates=5e7, max_step_sweeps=256,
                           clock=clock, sleep=clock.sleep, policy=policy)
        res = srv.run(workloads.served_jobs(n=80, rate=1e6, seed=11, kmin=6, kmax=12, smin=10, smax=3000))
        lat[policy] = np.median([r.latency for r in res])
    assert lat["srpt"] < lat["fair"]


class FlakyEngine(FakeEngine):
    """Fails the creation of some jobs, and one whole step."""

    def __init__(self, clock, bad_create=(), bad_step=None):
        super().__init__(clock)
        self.bad_create, self.bad_step, self.nsteps, self.aborted = set(bad_create), bad_step, 0, []

    def create(self, job):
        if job.id in self.bad_create:
            raise MemoryError("device allocation failed for job %d" % job.id)
        return super().create(job)

    def advance(self, handles, nsweeps):
        self.nsteps += 1
        if self.nsteps == self.bad_step:
            raise RuntimeError("lat_runner_run failed: a bounded device-side wait gave up (-4)")
        return super().advance(handles, nsweeps)

    def abort(self, h):
        h.closed = True
        self.live -= self.footprint(h.job)
        self.aborted.append(h.job.id)


def _check_done(r):
    assert list(np.concatenate(r.obs)["sweep"]) == list(range(1, r.job.sweeps + 1))
    assert r.final_hash == r.job.id * 7 + r.job.sweeps


def test_failed_admission_fails_only_that_job():
    clock = Clock()
    jobs = _jobs(30, 4)
    bad = {jobs[3].id, jobs[10].id}
    eng = FlakyEngine(clock, bad_create=bad)
    res = serve.Server(eng, mem_budget=600_000, max_batch=16, step_updates=5e6, max_step_sweeps=64,
                       clock=clock, sleep=clock.sleep).run(jobs)
    for r in res:
        if r.job.id in bad:
            assert r.status == "failed" and "allocation" in r.error and not r.obs
        else:
            assert r.status == "done"
            _check_done(r)
    assert eng.live == 0
    s = serve.summarize(res, 1.0)
    assert s["failed"] == 2 and s["jobs"] == 30


def test_failed_step_fails_its_jobs_and_the_rest_go_on():
    clock = Clock()
    jobs = _jobs(40, 6)
    eng = FlakyEngine(clock, bad_step=5)
    res = serve.Server(eng, mem_budget=600_000, max_batch=8, step_updates=5e6, max_step_sweeps=16,
                       clock=clock, sleep=clock.sleep).run(jobs)
    failed = [r for r in res if r.status == "failed"]
    assert failed and all("wait gave up" in r.error for r in failed)
    assert sorted(r.job.id for r in failed) == sorted(eng.aborted)
    for r in res:
        if r.status == "done":
            _check_done(r)
    assert sum(r.status == "done" for r in res) == len(jobs) - len(failed)
    assert eng.live == 0


def test_cancellation_while_waiting_running_or_before_arrival():
    clock = Clock()
    jobs = _jobs(30, 8)
    first, late = jobs[0], jobs[-1]
    eng = FlakyEngine(clock)
    srv = serve.Server(eng, mem_budget=300_000, max_batch=4, step_updates=5e6, max_step_sweeps=8,
                       clock=clock, sleep=clock.sleep)
    res = srv.run(jobs, cancels={first.id: first.arrival + 1e-6, late.id: 0.0})
    by = {r.job.id: r for r in res}
    assert by[first.id].status == "cancelled" and by[late.id].status == "cancelled" and not by[late.id].obs
    for r in res:
        if r.job.id not in (first.id, late.id):
            assert r.status == "done"
            _check_done(r)
    assert eng.live == 0


class DeferringEngine(FakeEngine):
    """An engine whose measurements and final hashes arrive later (as the GPU
    engine's do): they are Deferred until the next step or settle()."""

    def __init__(self, clock):
        super().__init__(clock)
        self.pending = []
        self.settles = 0

    def measure(self, h):
        v = super().measure(h)
        d = serve.Deferred(lambda: v)
        self.pending.append(d)
        return d

    def finish(self, h):
        v = super().finish(h)
        d = serve.Deferred(lambda: v)
        self.pending.append(d)
        return d

    def advance(self, handles, nsweeps):
        out = super().advance(handles, nsweeps)
        for d in self.pending:
            d.settle()
        self.pending = []
        return out

    def sweep(self, h, n):
        return self.advance([h], [n])[0]

    def settle(self):
        self.settles += 1
        for d in self.pending:
            d.settle()
        self.pending = []


def test_deferred_results_are_resolved_in_every_job():
    clock = Clock()
    eng = DeferringEngine(clock)
    srv = serve.Server(eng, mem_budget=600_000, max_batch=16, step_updates=5e6, max_step_sweeps=64,
                       clock=clock, sleep=clock.sleep)
    res = srv.run(_jobs(40, 21))
    assert eng.settles >= 1 and not eng.pending
    for r in res:
        assert r.final_hash == r.job.id * 7 + r.job.sweeps
        assert all(isinstance(v, tuple) and int(v[0][0]) == t for t, v in r.corr.items())
    seq = serve.run_sequential(DeferringEngine(clock), _jobs(10, 22), clock=clock, sleep=clock.sleep)
    for r in seq:
        assert isinstance(r.final_hash, int) and all(isinstance(v, tuple) for v in r.corr.values())


def test_digest_separates_runs_that_differ():
    clock = Clock()
    res = serve.run_sequential(DeferringEngine(clock), _jobs(6, 23), clock=clock, sleep=clock.sleep)
    again = serve.run_sequential(DeferringEngine(clock), _jobs(6, 23), clock=clock, sleep=clock.sleep)
    assert [serve.digest(r) for r in res] == [serve.digest(r) for r in again]
    r = res[0]
    d0 = serve.digest(r)
    r.final_hash += 1
    assert serve.digest(r) != d0
    r.final_hash -= 1
    t = sorted(r.corr)[0]
    r.corr[t] = (r.corr[t][0] + 1, r.corr[t][1])
    assert serve.digest(r) != d0
