"""The multi-GPU path of bench.py is independent replicas (one solve per
rank, no data-path collective); only the timings are combined, with a max
over ranks.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank-dependent per-rank timings: device time, end-to-end time, mixed time
    res = bench.max_over_ranks([1.0 + rank, 5.0 - rank, 0.5 * (rank + 1)], world, dist)
    out.put((rank, res))
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert got[r] == [2.0, 5.0, 1.0]


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]
