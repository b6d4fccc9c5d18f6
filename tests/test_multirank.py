"""Whole-job totals of the benchmark over two ranks, on the CPU (gloo).

Tracer boxes are independent, so a run on N GPUs gives each rank its own
boxes and exchanges nothing while stepping; the only collective is the final
reduction of the throughput inputs: the site updates of all ranks add up and
the time is the slowest rank's.
"""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, units, ms, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    q.put((rank,) + bench.whole_job(units[rank], ms[rank]))
    dist.barrier()
    dist.destroy_process_group()


def _run(world, units, ms):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, units, ms, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


def test_two_ranks_sum_units_max_time():
    # uneven batches (the ranks draw different box sizes) and uneven times
    units = [2_097_152 * 160, 1_900_000 * 160]
    ms = [12.5, 13.75]
    out = _run(2, units, ms)
    for rank, u, m in out:
        assert u == float(sum(units))
        assert m == max(ms)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(123, 4.5) == (123.0, 4.5)
