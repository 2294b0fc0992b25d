"""The multi-rank host logic of bench.py on CPU with two gloo ranks: every
rank gets the element-wise maximum of the ranks' step times, the whole-job
rate counts every rank's units against the slowest rank, replicas get their
own scene seeds, and the reference arm does no work on ranks other than 0."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    # rank 0 is slower on the first value, rank 1 on the second
    times = bench.max_over_ranks([1.0 + r, 5.0 - r], w, "cpu")
    rate = bench.whole_job_rate(10, times[0], w)

    class Args:
        pass
    ref = bench.run_reference(Args(), r, w, r) if r != 0 else "skipped"
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, times, rate, bench.replica_seeds(r), ref))


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, times, rate, seeds, ref in out:
        assert times == [2.0, 5.0]                  # the slower rank's time, element-wise
        assert rate == pytest.approx(10.0)          # 2 ranks x 10 units / 2.0 s
        assert ref is None or ref == "skipped"      # no reference work off rank 0
    assert out[0][3] != out[1][3]                    # independent replicas


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, "cpu") == [3.0, 4.0]
    assert bench.whole_job_rate(30, 2.0, 1) == 15.0
