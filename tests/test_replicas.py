"""The multi-GPU form is replicas only (every rank evaluates its own copy of the box, no data-path
collective); what crosses ranks is the timing barrier and the max over ranks.  That host logic
(bench.Ranks, bench.whole_job_rate) runs here as world-size-2 gloo process groups on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    ranks = bench.Ranks("gloo", "cpu")
    ranks.barrier()
    seconds = [0.5, 2.0][rank]           # the slower replica decides
    out[rank] = (ranks.max(seconds), bench.whole_job_rate(1000.0, seconds, ranks), ranks.world)
    ranks.close()


def test_two_replicas_take_the_slowest_rank():
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    for rank in (0, 1):
        mx, rate, world = res[rank]
        assert world == 2 and mx == 2.0
        assert rate == pytest.approx(2 * 1000.0 / 2.0)


def test_single_process_without_torchrun(monkeypatch):
    import bench
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    r = bench.Ranks("gloo", "cpu")
    assert r.world == 1 and r.rank == 0 and r.dist is None
    assert r.max(3.5) == 3.5
    assert bench.whole_job_rate(100.0, 2.0, r) == 50.0
