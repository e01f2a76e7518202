"""The multi-process path of bench.py on CPU: two ranks over gloo (127.0.0.1),
each solving its own replica.  Checks the host logic the N > 1 run relies on:
the rank environment, the per-rank Philox instance, the barrier, and the
whole-job rate = units of all ranks / the slowest rank's time (max over
ranks by all_reduce)."""
import queue
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import os
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ws, r, local = bench.dist_env()
        w = bench.rank_workload("cfg2", r)
        local_ms = 100.0 * (r + 1)                  # rank 1 is the slower one
        rate, max_ms = bench.whole_job_rate(w.path_steps(), ws, 3, local_ms)
        bench.barrier()
        q.put((r, ws, local, w.instance, w.path_steps(), rate, max_ms))
    finally:
        dist.destroy_process_group()


def test_two_replicas_over_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = []
    try:
        for _ in range(2):
            got.append(q.get(timeout=120))
    except queue.Empty:
        pytest.fail("a rank did not report")
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    got.sort()
    (r0, ws0, l0, inst0, units, rate0, max0), (r1, ws1, l1, inst1, _, rate1, max1) = got
    assert (r0, r1, ws0, ws1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert inst1 == inst0 + 1000                    # independent clouds per rank
    assert max0 == max1 == 200.0                    # the slowest rank's time
    assert rate0 == rate1 == pytest.approx(units * 2 * 3 / 0.2)
