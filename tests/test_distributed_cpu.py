"""The multi-rank benchmark path (one independent factorization stream per
GPU, no data-path collective) on CPU: two gloo ranks agree on the slowest
rank's time, the barrier holds, and the whole-job rate counts every rank."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import time
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t0 = time.perf_counter()
    if rank == 1:
        time.sleep(0.3)          # the slow rank
    bench.dist_barrier()         # rank 0 waits here for rank 1
    waited = time.perf_counter() - t0
    ms_rank = 10.0 + 5.0 * rank
    ms = bench.dist_max(ms_rank)
    rate = bench.whole_job_rate(512, world, ms)
    q.put((rank, waited, ms, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_max_time_and_whole_job_rate():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res = {r: (w, ms, rate) for r, w, ms, rate in out}
    assert res[0][1] == res[1][1] == 15.0            # both see the slowest rank's time
    assert res[0][2] == res[1][2] == pytest.approx(2 * 512 / 0.015)
    assert res[0][0] >= 0.25                         # rank 0 waited for rank 1 at the barrier


def test_single_process_helpers_are_identities():
    import bench
    assert bench.dist_max(3.5) == 3.5
    bench.dist_barrier()
    assert bench.whole_job_rate(1, 1, 100.0) == pytest.approx(10.0)


def _worker_rank_dies(rank, world, port, q):
    import datetime
    import time
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=3))
    import bench
    bench.dist_barrier()                 # step 1: both ranks present
    if rank == 1:
        q.put((rank, "left", 0.0))
        q.close()
        q.join_thread()                  # the message is out before the process ends
        os._exit(0)                      # leaves between steps, with nothing in flight
    t0 = time.perf_counter()
    try:
        bench.dist_max(10.0)             # step 2: the collective rank 1 never joins
        q.put((rank, "returned", time.perf_counter() - t0))
    except Exception:                    # the process group's timeout ends it with an error
        q.put((rank, "error", time.perf_counter() - t0))


def test_a_rank_that_leaves_ends_the_next_collective_with_an_error():
    """Failure detection on the host: a rank exits between steps; the other
    rank's next collective ends with an error after the short process-group
    timeout instead of hanging."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_rank_dies, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        r, what, dt = q.get(timeout=120)
        out[r] = (what, dt)
    for p in procs:
        p.join(timeout=60)
    assert out[1][0] == "left"
    assert out[0][0] == "error" and out[0][1] < 60.0, out
