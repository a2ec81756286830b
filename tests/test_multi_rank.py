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


def _shard_rank(rank, world, port, out):
    # contiguous DM shard of the small workload, searched by the oracle on this rank; the raw
    # detections are gathered on rank 0, which sifts once (the exchange of the multi-GPU plan:
    # KB of candidates to the host, no device collective)
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle import search as OSr
    from paper_1912_12807_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = synth.workload_small(nsamp=1 << 14)
    ndm = sum(s.n_dm for s in wl.stages)
    lo, hi = rank * ndm // world, (rank + 1) * ndm // world
    raw, _ = OSr.search(wl.fil, wl.stages, wl.cfg, dm_indices=range(lo, hi))
    gathered = [None] * world
    dist.all_gather_object(gathered, raw)
    if rank == 0:
        from oracle import sift as OSf
        merged = {}
        for part in gathered:
            merged.update(part)
        out.put(("sharded", sorted(merged), OSf.sift(merged, wl.cfg.dz, wl.cfg.min_dm_hits), merged))
    dist.barrier()
    dist.destroy_process_group()


def test_two_cpu_ranks_dm_shards_gather_and_sift_once():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    from oracle import search as OSr
    from paper_1912_12807_gb300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    tag, dms, sharded, merged = q.get(timeout=600)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    wl = synth.workload_small(nsamp=1 << 14)
    _, whole = OSr.search(wl.fil, wl.stages, wl.cfg)
    assert dms == list(range(sum(s.n_dm for s in wl.stages)))
    assert len(whole) > 0 and sharded == whole
    # the library's host sift of the gathered list (FP32 powers, as the device reports them)
    # equals the oracle's sift of the same list
    import numpy as np
    from oracle import sift as OSf
    from oracle import stats as OST
    from paper_1912_12807_gb300 import build, pss
    if not os.path.exists(pss.LIB_PATH):
        build.build()
    rows = [(c["dm_idx"], c["numharm"], c["h"], c["j"], np.float32(c["power"]), 0)
            for d in sorted(merged) for c in merged[d]]
    raw = np.array(rows, dtype=pss.RAW_DTYPE)
    plan = pss.Plan(pss.FilDesc.of(wl.fil), wl.stages)
    got = pss.pss_sift(plan, pss.cfg_of(wl.cfg), raw)
    by_dm = {}
    for c in raw:
        n, h, j = int(c["numharm"]), int(c["h"]), int(c["j"])
        r, z = OSf.fundamental(n, h, j, 0, wl.cfg.dz)
        by_dm.setdefault(int(c["dm_idx"]), []).append(dict(
            dm_idx=int(c["dm_idx"]), numharm=n, h=h, j=j, r=r, z=z, zq=OSf.zq(n, j, 0), power=float(c["power"]),
            sigma=OST.sigma_of(n, float(c["power"]))))
    ref = OSf.sift(by_dm, wl.cfg.dz, wl.cfg.min_dm_hits)
    assert len(got) == len(ref) > 0
    for g, r in zip(got, ref):
        assert (int(g["dm_idx"]), int(g["numharm"]), int(g["h"]), int(g["j"]), int(g["dm_hits"])) == \
               (r["dm_idx"], r["numharm"], r["h"], r["j"], r["dm_hits"])
