"""The multi-rank benchmark path on CPU: two gloo ranks, each with its own
field strength, timing reduced by max over ranks into whole-job steps/s."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = [12.0, 20.0][rank]
        ms_max, value = bench.aggregate_timing(ms_local, 5, world, dist)
        out[rank] = (ms_max, value, bench.rank_field_amplitude(0.001, rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_timing_by_max():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    assert res[0][0] == pytest.approx(20.0) and res[1][0] == pytest.approx(20.0)
    # whole-job throughput: 2 ranks x 5 steps in the slowest rank's 20 ms
    assert res[0][1] == pytest.approx(500.0) and res[1][1] == pytest.approx(500.0)
    assert res[0][2] != res[1][2]  # independent field strengths per rank


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.aggregate_timing(25.0, 10, 1)
    assert ms == 25.0 and value == pytest.approx(400.0)
