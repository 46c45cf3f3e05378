"""The N-GPU bench path is N independent replicas (the correlation has no exchange step); its only
cross-rank logic is the max-over-ranks timing and the whole-job throughput.  Exercised here with
two gloo ranks on the CPU."""
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


def _rank(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = [0.75, 1.25][rank]   # per-rank timed seconds
    t_max = bench.max_over_ranks(t)
    value = bench.replica_throughput(cells_per_rank=1000, steps=4, world=world, t_max_s=t_max)
    out.put((rank, t_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, t_max, value in res:
        assert t_max == pytest.approx(1.25)
        assert value == pytest.approx(1000 * 4 * 2 / 1.25)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(2.5) == 2.5
