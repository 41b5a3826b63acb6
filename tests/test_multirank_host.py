"""The multi-GPU path of bench.py runs one independent replica per rank (the
maps do not share anything, so there is no data-path collective); the only
cross-rank steps are the barrier and the whole-job aggregation: units summed
over ranks, time the slowest rank's.  Checked here with two gloo ranks on
the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    bench._barrier(ws)
    # rank r processed 1000 * (r + 1) rays in 10 * (r + 1) ms
    total, max_ms, value = bench.whole_job(1000 * (rank + 1), 10.0 * (rank + 1), ws)
    mx = bench._max_over_ranks(float(rank), ws)
    sm = bench._sum_over_ranks(2.5, ws)
    bench._barrier(ws)
    dist.destroy_process_group()
    q.put((rank, total, max_ms, value, mx, sm))


@pytest.mark.parametrize("ws", [2])
def test_whole_job_aggregation_over_gloo_ranks(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, max_ms, value, mx, sm in out:
        assert total == 3000.0 and max_ms == 20.0  # every rank sees the same whole-job numbers
        assert value == pytest.approx(3000.0 / 0.020)
        assert mx == ws - 1 and sm == 2.5 * ws


def test_single_rank_needs_no_process_group():
    import bench
    total, max_ms, value = bench.whole_job(131072, 0.5, 1)
    assert (total, max_ms) == (131072.0, 0.5) and value == pytest.approx(131072 / 0.0005)
