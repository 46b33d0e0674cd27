"""The served loop on the GPU: every job's per-sweep (M, B, Q), C(r) at
sweeps 2^k and final lattice are bit-identical to the same job run alone on
the plain path, while jobs share runner launches (continuous batching)."""
import pytest

from paper_2502_18624_gb300 import serve, workloads

pytestmark = pytest.mark.gpu


def test_served_results_equal_sequential_plain_runs(gpu):
    jobs = workloads.served_jobs(n=24, rate=400.0, seed=77, kmin=8, kmax=10, smin=10, smax=150)
    eng = serve.GpuEngine(max_jobs=16, max_step_sweeps=64, rmax_cap=256)
    srv = serve.Server(eng, mem_budget=96 << 20, max_batch=16, step_updates=3e7, max_step_sweeps=64)
    res = srv.run(jobs)
    eng.close()
    seq_eng = serve.GpuEngine(max_jobs=1, max_step_sweeps=1, rmax_cap=256)
    seq = serve.run_sequential(seq_eng, jobs)
    seq_eng.close()
    assert srv.peak_batch > 1 and srv.steps > 1
    for a, b in zip(res, seq):
        assert a.job.id == b.job.id
        assert serve.same_results(a, b), "job %d differs between served and plain runs" % a.job.id
        assert sorted(a.corr) == [2 ** k for k in range(16) if 2 ** k <= a.job.sweeps]


class StallOnceEngine(serve.GpuEngine):
    """A GpuEngine whose second step has one lattice's device waits stall, so
    the runner gives up after a short limit (no GPU fault, no hang)."""

    def advance(self, handles, nsweeps):
        self.nadv = getattr(self, "nadv", 0) + 1
        if self.nadv == 2:
            self.runner.set_timeout(200_000_000)  # 0.2 s
            self.runner.inject_stall(0)
            try:
                return super().advance(handles, nsweeps)
            finally:
                self.runner.inject_stall(0xFFFFFFFF)
                self.runner.set_timeout(10_000_000_000)
        return super().advance(handles, nsweeps)


def test_served_step_that_times_out_fails_only_its_jobs(gpu):
    jobs = workloads.served_jobs(n=16, rate=50.0, seed=78, kmin=8, kmax=9, smin=10, smax=80)
    eng = StallOnceEngine(max_jobs=8, max_step_sweeps=8, rmax_cap=128)
    srv = serve.Server(eng, mem_budget=64 << 20, max_batch=8, step_updates=1e7, max_step_sweeps=8)
    res = srv.run(jobs)
    eng.close()
    failed = [r for r in res if r.status == "failed"]
    done = [r for r in res if r.status == "done"]
    assert failed and all("-4" in r.error or "gave up" in r.error for r in failed)
    assert done, "the jobs after the failed step must complete"
    seq_eng = serve.GpuEngine(max_jobs=1, max_step_sweeps=1, rmax_cap=128)
    seq = {r.job.id: r for r in serve.run_sequential(seq_eng, [r.job for r in done])}
    seq_eng.close()
    for r in done:
        assert serve.same_results(r, seq[r.job.id]), "job %d differs after the failed step" % r.job.id
