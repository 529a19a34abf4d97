"""bench.py's whole-job figure across ranks, checked with two gloo ranks on the
CPU: every rank reports the slowest rank's time, and the value counts the units
of all ranks over that time (weak scaling: each rank solves its own copy of the
workload, no data-path collective)."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, ms, units, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        q.put((rank, bench.whole_job_rate(ms[rank], units, world)))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, units, ms = 2, 4194304.0, [12.5, 20.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, ms, units, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for r in range(world):
        ms_max, value = got[r]
        assert ms_max == 20.0
        assert abs(value - world * units / 0.020) <= 1e-6 * value


def test_single_rank_rate_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms_max, value = bench.whole_job_rate(8.0, 1000.0, 1)
    assert ms_max == 8.0 and abs(value - 1000.0 / 0.008) < 1e-6
