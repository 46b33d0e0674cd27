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
