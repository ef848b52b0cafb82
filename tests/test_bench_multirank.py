"""bench.py's multi-rank path on CPU: two ranks over gloo (rendezvous on
127.0.0.1), the way torchrun starts them.  The GPU path shards with no data
collective: every rank runs its own seeded workload, and the only exchange is
the reduction of the whole-job figures (units summed, time the slowest
rank's), which is what these tests check."""
import os
import socket
import types

import numpy as np

WORLD = 2


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(WORLD))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        import bench
        units, ms = bench.job_totals(1000 * (rank + 1), 5.0 + 2.5 * rank, WORLD)
        # a rank that is not 0 runs no reference work and prints nothing
        args = types.SimpleNamespace(seed=bench.W.DEFAULT_SEED, arena_gib=1, nreq=2000, steps=1, warmup=0)
        ref = bench.reference_arm(args, rank, WORLD) if rank else "skipped"
        q.put((rank, units, ms, ref))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_sum_units_and_take_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    got = {}
    try:
        for _ in range(WORLD):
            rank, units, ms, ref = q.get(timeout=180)
            got[rank] = (units, ms, ref)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert sorted(got) == [0, 1]
    for rank, (units, ms, ref) in got.items():
        assert units == 3000.0 and ms == 7.5, (rank, units, ms)
    assert got[1][2] is None
    assert all(p.exitcode == 0 for p in procs)


def test_single_rank_totals_are_local():
    import bench
    assert bench.job_totals(123, 4.5, 1) == (123.0, 4.5)


def test_ranks_get_independent_workloads():
    """Weak scaling: rank r's workload is the same recipe under its own seed."""
    import bench
    args = types.SimpleNamespace(seed=bench.W.DEFAULT_SEED, arena_gib=1, nreq=3000)
    img0, wl0, b0 = bench.build_workload(args, 0)
    img1, wl1, b1 = bench.build_workload(args, 1)
    assert len(wl0.reqs) == len(wl1.reqs) == 3000
    assert not np.array_equal(wl0.segs["gva"][:100], wl1.segs["gva"][:100])
    assert abs(wl0.payload_bytes / wl1.payload_bytes - 1) < 0.5
