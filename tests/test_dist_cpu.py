"""bench.py's multi-rank host logic (process group set-up, barrier, max over ranks) with two
gloo ranks on the CPU; no GPU and no data-path collective involved."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), SMNN_DIST_BACKEND="gloo")
    import bench
    import torch.distributed as dist
    ws, r, local = bench.dist_setup()
    bench.barrier(ws)
    m = bench.max_over_ranks(float(10 * (rank + 1)), ws)
    out.put((r, ws, m))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=100) for _ in range(2))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert res == [(0, 2, 20.0), (1, 2, 20.0)]
