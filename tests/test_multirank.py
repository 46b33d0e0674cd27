"""bench.py's multi-rank plumbing on the CPU (gloo, world size 2): one
process per rank, independent replicas, a barrier and a max-over-ranks time
reduction only; the whole-job value counts every rank's work over the
slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    r, w, local = bench.dist_env()
    dist = bench.dist_init(w, "gloo")
    bench.barrier(dist)
    secs = 1.0 + r  # rank 1 is the slower one
    mx = bench.reduce_max(dist, secs)
    value = bench.whole_job(1e9, w, mx)
    q.put((r, mx, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_time_and_sum_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.0, 2.0]          # both ranks see the slowest time
    assert all(abs(o[2] - 1.0) < 1e-12 for o in out)  # 2 ranks x 1e9 updates / 2 s = 1 update/ns


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.dist_init(1, "gloo") is None
    assert bench.reduce_max(None, 3.5) == 3.5
    assert bench.whole_job(2e9, 1, 2.0) == pytest.approx(1.0)
