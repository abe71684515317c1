"""The N > 1 host logic of bench.py on CPU: two gloo ranks (127.0.0.1).

Each rank gets its own view (weak scaling over views, no collective on the
data path); the whole-job figures are the max step time and the summed
evals over the ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, ev = bench.reduce_over_ranks(1.5 + rank, 100.0 * (rank + 1))
        q.put((rank, ms, ev, bench.rank_camera_seeds(rank, 3000)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, ev, seeds in res:
        assert ms == pytest.approx(2.5)      # max over ranks
        assert ev == pytest.approx(300.0)    # sum over ranks
    assert res[0][3] != res[1][3]            # each rank renders its own view
