"""The multi-GPU form of the benchmark runs independent replicas: each rank
packs/unpacks its own data and the only collective is the max over ranks of
the timed region.  Checked here with two gloo ranks on the CPU: every rank
gets the slowest rank's time, the whole-job throughput counts every rank's
bytes, and the pack itself needs no exchange (each rank's result equals the
oracle's on its own data)."""
import os

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import inputs
    # each replica works on its own seeded shard of the same workload shape
    spec = inputs.strided_vector_spec(64, 4, 16)
    t = oracle.from_spec(spec)
    src = inputs.uniform_f32(2 * 64 * 16, 100 + rank).view(np.uint8)  # covers two elements
    assert src.size >= t.extent + t.true_extent
    packed = t.pack(src, 2)
    mine = 0.010 * (rank + 1)  # pretend timed seconds: rank 1 is slower
    slowest = bench.max_over_ranks(mine, world)
    gbs = bench.job_throughput(2 * packed.size, world, slowest)
    q.put((rank, slowest, gbs, packed.tobytes() == t.pack(src, 2).tobytes()))
    dist.destroy_process_group()


def test_two_gloo_replicas_reduce_time_only():
    world = 2
    port = 29500 + (os.getpid() % 1000)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [0.020, 0.020]  # both see the slowest rank
    per_rank = 2 * (2 * 64 * 4 * 4)               # read + write of two packed elements
    assert all(abs(r[2] - per_rank * world / 0.020 / 1e9) < 1e-12 for r in res)
    assert all(r[3] for r in res)
