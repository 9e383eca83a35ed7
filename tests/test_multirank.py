"""The multi-rank bench path on CPU: two gloo ranks, each with its own replica,
agree on the slowest rank's time and report the whole-job rate (weak scaling,
no data-path collective).  Rendezvous on 127.0.0.1."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    my_ms = [120.0, 150.0][rank]
    slow = bench.max_over_ranks(my_ms, dist, ws, device="cpu")
    rate = bench.whole_job_rate(1000, slow, ws)
    out[rank] = (slow, rate, bench.dist_env())
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_aggregate_rate():
    ws, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(ws):
        slow, rate, env = out[r]
        assert slow == 150.0
        assert rate == pytest.approx(2 * 1000 / 0.150)
        assert env == (2, r, 0)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(3.5, None, 1) == 3.5
    assert bench.whole_job_rate(10, 1000.0, 1) == pytest.approx(10.0)
