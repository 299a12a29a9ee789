"""The multi-GPU form of the path is replicas (independent instances per
rank, no data exchange): world_size-2 gloo ranks on the CPU check the host
logic bench.py uses -- disjoint Philox ranges per rank, the whole-job time as
the slowest rank's, and the whole-job rate."""
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


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = 1.5 + rank            # rank 1 is the slower one
    tmax = bench.max_over_ranks(t, world)
    rate = bench.whole_job_rate(152 * 5, world, tmax)
    off = bench.replica_offset(rank)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, tmax, rate, off))


def test_replica_host_logic_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, rate0, off0), (r1, t1, rate1, off1) = res
    assert t0 == t1 == 2.5
    assert rate0 == rate1 == pytest.approx(152 * 5 * 2 / 2.5)
    # each rank's instances (at most 10 million chain indices) do not overlap
    assert off1 - off0 >= 10_000_000


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0
