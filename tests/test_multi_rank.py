"""The N > 1 bench path on CPU ranks (gloo, world size 2): every rank
searches its own file (different seeds, hence different data), the job time
is the slowest rank's, and the whole-job value counts all ranks' trials.
No collective touches the search itself."""
import os
import socket
import sys
import zlib

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = bench.make_workload("small", seed_offset=rank)
    crc = zlib.crc32(wl.fil.data.tobytes())
    crcs = [None] * world
    dist.all_gather_object(crcs, crc)
    ms = bench.max_over_ranks(10.0 * (rank + 1), world)
    value = bench.job_value(world, 101, ms)
    dist.barrier()
    out.put((rank, crcs, ms, value))
    dist.destroy_process_group()


def test_two_cpu_ranks_shard_files_and_reduce_max():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=300) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    (_, crcs0, ms0, v0), (_, crcs1, ms1, v1) = res
    assert crcs0 == crcs1 and crcs0[0] != crcs0[1]  # each rank has its own file
    assert ms0 == ms1 == 20.0                       # the slowest rank's time
    assert abs(v0 - 2 * 101 / 0.020) < 1e-9 and v0 == v1
