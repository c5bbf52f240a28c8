"""Host logic of bench.py's multi-GPU mode, run as two gloo ranks on the CPU.

With N ranks every rank channelizes its own beam (independent input, no
data-path collective); the job time is the slowest rank's and the reported
bandwidth counts every rank's spectra.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 25.0 * rank
        out[rank] = (bench.reduce_max(local_ms, dist, "cpu"), bench.beam_seed(rank))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_max_time_and_independent_beams():
    import bench
    mp = torch.multiprocessing.get_context("spawn")
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        procs = [mp.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 125.0          # slowest rank
    assert res[0][1] != res[1][1]                     # independent beams
    # whole-job bandwidth: both ranks' spectra over the slowest time
    assert bench.whole_job_ghz(2, 10, 1000, 32768, 125.0) == pytest.approx(2 * 10 * 1000 * 32768 / 0.125 / 1e9)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.reduce_max(42.0) == 42.0
