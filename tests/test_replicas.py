"""The multi-GPU path of bench.py is independent replicas (one synthetic snapshot per rank, seed =
rank; no collective on the data path): the FEF solve of one snapshot does not shard further here.
Its only cross-rank step, the whole-job aggregation after the timed region, runs here on two CPU
ranks over gloo: the time is the slowest rank's, quartets and launches are summed."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    from synth import systems as S
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # replica inputs: one snapshot per rank, seeded by the rank
        system = S.water_box(8, seed=rank)
        ms, quartets, launches = bench.reduce_over_replicas(dist, 10.0 + 5.0 * rank, 1000 * (rank + 1), 3 + rank,
                                                            "cpu")
        out.put((rank, ms, quartets, launches, float(system.xyz.sum())))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, quartets, launches, _ in res:
        assert ms == 15.0 and quartets == 3000.0 and launches == 7
    assert res[0][4] != res[1][4]  # the replicas solve different snapshots
