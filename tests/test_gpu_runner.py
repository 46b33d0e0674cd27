"""The runner (many lattices, one persistent launch) against the plain path.

Each lattice advanced by the runner must end bit-identical to the same
lattice advanced alone by lat_sweep, with identical per-sweep (M, B, Q) and
draw counts, for a mix of models, sizes (ragged word counts included),
temperatures (every acceptance mode) and sweep counts (zero included), over
chained runs and any tile schedule.  A wait that runs out must come back as
LAT_ETIMEDOUT and leave the runner usable.  The per-lattice tile counters
are 64-bit: started just below 2^32 they cross it inside a run with no
effect on any result, and a run whose counts could not fit is refused before
anything is launched.
"""
import numpy as np
import pytest

from paper_2502_18624_gb300 import binding as b

pytestmark = pytest.mark.gpu

TC = b.TC_ISING

JOBS = [  # (model, L, T, Delta, seed)
    (0, 64, TC, 0.0, 1), (0, 128, 0.9 * TC, 0.0, 2), (0, 192, 5.0, 0.0, 3), (0, 256, 1e-3, 0.0, 4),
    (0, 320, 1e15, 0.0, 5), (0, 512, TC, 0.0, 6), (0, 1024, 1.1 * TC, 0.0, 7), (0, 64, 2.0, 0.0, 8),
    (1, 64, 1.398, 1.0, 9), (1, 128, 1.69, 0.5, 10), (1, 192, 1.69, 1.5, 11), (1, 256, 3.0, -1.0, 12),
    (1, 512, 1e-3, 1.0, 13), (1, 64, 0.608, 1.966, 14), (0, 2048, TC, 0.0, 15), (1, 1024, 1.4, 1.0, 16),
]


def _make(jobs):
    return [b.Lattice(m, L, T, s, Delta=D) for (m, L, T, D, s) in jobs]


def _check_same(run_lats, ref_lats, obs, ref_obs):
    for i, (a, r) in enumerate(zip(run_lats, ref_lats)):
        assert a.sweep_index == r.sweep_index, i
        assert a.hash() == r.hash(), "lattice %d differs" % i
        if a.L <= 2048:
            assert np.array_equal(a.spins(), r.spins()), i
        assert np.array_equal(obs[i], ref_obs[i]), "per-sweep records of lattice %d differ" % i


def test_runner_matches_plain_path_over_chained_runs(gpu):
    runner = b.Runner(64, 64)
    lats, refs = _make(JOBS), _make(JOBS)
    rng = np.random.default_rng(0)
    for rnd in range(3):
        ns = rng.integers(0, 12, size=len(JOBS))
        ns[rnd] = 0
        obs = runner.run(lats, ns)
        ref_obs = [r.sweep(int(k)) for r, k in zip(refs, ns)]
        _check_same(lats, refs, obs, ref_obs)
    runner.close()


def test_runner_tile_schedule_does_not_change_results(gpu):
    jobs = [(0, 1024, TC, 0.0, 21), (0, 2048, 0.95 * TC, 0.0, 22), (1, 1024, 1.5, 1.0, 23), (0, 192, TC, 0.0, 24)]
    results = []
    for tiles in (None, 256, 1024, 16384):
        runner = b.Runner(8, 16)
        if tiles:
            for (m, L, _, _, _) in jobs:
                runner.set_tile(m, L, tiles)
        lats = _make(jobs)
        obs = runner.run(lats, [9, 7, 8, 11])
        results.append(([lt.hash() for lt in lats], [o.copy() for o in obs]))
        runner.close()
    for h, o in results[1:]:
        assert h == results[0][0]
        assert all(np.array_equal(x, y) for x, y in zip(o, results[0][1]))


def test_runner_wait_timeout_is_reported_and_recoverable(gpu):
    runner = b.Runner(4, 8)
    lats = _make([(0, 1024, TC, 0.0, 31), (0, 256, TC, 0.0, 32)])
    runner.set_timeout(200_000_000)  # 0.2 s
    runner.inject_stall(0)
    with pytest.raises(b.LatError) as e:
        runner.run(lats, [4, 4])
    assert e.value.code == b.LAT_ETIMEDOUT
    runner.inject_stall(0xFFFFFFFF)
    runner.set_timeout(10_000_000_000)
    fresh, ref = _make([(0, 512, TC, 0.0, 33)]), _make([(0, 512, TC, 0.0, 33)])
    obs = runner.run(fresh, [5])
    assert np.array_equal(obs[0], ref[0].sweep(5)) and fresh[0].hash() == ref[0].hash()
    runner.close()


def test_runner_rejects_bad_arguments(gpu):
    runner = b.Runner(2, 4)
    a, c, d = _make([(0, 64, TC, 0.0, 1), (0, 64, TC, 0.0, 2), (0, 64, TC, 0.0, 3)])
    for lats, ns in [([a, a], [1, 1]), ([a], [5]), ([a, c, d], [1, 1, 1])]:
        with pytest.raises(b.LatError) as e:
            runner.run(lats, ns)
        assert e.value.code == b.LAT_EINVAL
    with pytest.raises(b.LatError):
        runner.set_tile(0, 64, 100)   # not a multiple of 256
    runner.close()


def test_runner_on_the_batched_workload_sample(gpu):
    """A slice of the 512-replica workload, every replica bit-exact to its plain run."""
    from paper_2502_18624_gb300 import workloads
    jobs = workloads.batched_replicas()
    pick = [j for j in jobs if j.L <= 1024][:40] + [j for j in jobs if j.L >= 2048][:2]
    lats = [b.Lattice(j.model, j.L, j.T, j.seed, Delta=j.Delta) for j in pick]
    refs = [b.Lattice(j.model, j.L, j.T, j.seed, Delta=j.Delta) for j in pick]
    runner = b.Runner(len(pick), 32)
    obs = runner.run(lats, [20] * len(pick))
    ref_obs = [r.sweep(20) for r in refs]
    _check_same(lats, refs, obs, ref_obs)
    runner.close()


def test_runner_counters_cross_the_32_bit_boundary(gpu):
    jobs = [(0, 1024, TC, 0.0, 41), (1, 512, 1.4, 1.0, 42), (0, 2048, 0.9 * TC, 0.0, 43), (0, 192, TC, 0.0, 44)]
    ns = [9, 6, 7, 5]
    runner = b.Runner(4, 16)
    for (m, L, _, _, _) in jobs:
        runner.set_tile(m, L, 256)          # many tiles per phase, so the counts move fast
    runner.set_counter_base((1 << 32) - 3)  # every counter passes 2^32 within its first phase
    lats, refs = _make(jobs), _make(jobs)
    obs = runner.run(lats, ns)
    ref_obs = [r.sweep(k) for r, k in zip(refs, ns)]
    _check_same(lats, refs, obs, ref_obs)
    # a second run continues from the same base, chained on the same lattices
    obs = runner.run(lats, [3, 4, 2, 6])
    ref_obs = [r.sweep(k) for r, k in zip(refs, [3, 4, 2, 6])]
    _check_same(lats, refs, obs, ref_obs)
    # counts that would reach 2^64 - 1 are refused before launch; nothing changes
    before = [lt.hash() for lt in lats]
    runner.set_counter_base((1 << 64) - 4)
    with pytest.raises(b.LatError) as e:
        runner.run(lats, [1, 1, 1, 1])
    assert e.value.code == b.LAT_EINVAL
    assert [lt.hash() for lt in lats] == before and [lt.sweep_index for lt in lats] == [12, 10, 9, 11]
    with pytest.raises(b.LatError):
        runner.set_counter_base((1 << 64) - 1)
    runner.set_counter_base(0)
    obs = runner.run(lats, [2, 2, 2, 2])
    ref_obs = [r.sweep(2) for r in refs]
    _check_same(lats, refs, obs, ref_obs)
    runner.close()


def test_submit_collect_and_async_measurements(gpu):
    """lat_runner_submit / lat_runner_collect give what lat_runner_run gives;
    lat_correlation_async and lat_hash_async, enqueued behind a run on the
    runner's stream, give what the synchronous calls give once collected; a
    handle on another stream is ordered before the run by a device-side wait;
    and the call sequence is checked (LAT_ESTATE)."""
    import torch
    runner = b.Runner(8, 16)
    side = torch.cuda.Stream()
    jobs = [(0, 512, TC, 0.0, 51), (1, 256, 1.4, 1.0, 52), (0, 1024, 0.9 * TC, 0.0, 53)]
    lats = [b.Lattice(m, L, T, s, Delta=D, stream=runner.stream) for (m, L, T, D, s) in jobs[:2]]
    lats.append(b.Lattice(*[jobs[2][i] for i in (0, 1, 2, 4)], Delta=0.0, stream=side))
    refs = _make(jobs)
    ns = [6, 9, 4]
    with pytest.raises(b.LatError) as e:
        runner.collect(ns)
    assert e.value.code == b.LAT_ESTATE
    runner.submit(lats, ns)
    with pytest.raises(b.LatError) as e:
        runner.submit(lats, ns)
    assert e.value.code == b.LAT_ESTATE
    obs = runner.collect(ns)
    ref_obs = [r.sweep(k) for r, k in zip(refs, ns)]
    _check_same(lats, refs, obs, ref_obs)
    # measurements enqueued behind the next run, read after its collect
    runner.submit(lats[:2], [3, 5])
    pinned = [torch.zeros(2 * 257, dtype=torch.int64, pin_memory=True) for _ in range(2)]
    hashes = torch.zeros(2, dtype=torch.int64, pin_memory=True)
    for lt, buf in zip(lats[:2], pinned):
        a = buf.numpy()
        b.lat_correlation_async(lt.handle, 128, a[:129], a[129:258])
    for i, lt in enumerate(lats[:2]):
        b.lat_hash_async(lt.handle, hashes.numpy().view(np.uint64)[i:i + 1])
    runner.collect([3, 5])
    runner.stream.synchronize()
    for i, (lt, r, k) in enumerate(zip(lats[:2], refs[:2], [3, 5])):
        r.sweep(k, record=False)
        rx, ry = r.correlation(128)
        a = pinned[i].numpy()
        assert np.array_equal(a[:129], rx) and np.array_equal(a[129:258], ry)
        assert int(hashes.numpy().view(np.uint64)[i]) == r.hash() == lt.hash()
    runner.close()
