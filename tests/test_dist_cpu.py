"""The benchmark's multi-rank path on the CPU: two gloo ranks on 127.0.0.1
run bench.py's process-group setup, barrier and max-over-ranks timing (the
N > 1 launch runs one independent replica per GPU; the only collectives are
these)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench

    ws, r, local = bench.dist_setup()
    assert (ws, r, local) == (world, rank, rank)
    bench.barrier(ws)
    # each rank reports its own time; every rank gets the maximum
    out[rank] = bench.max_over_ranks(ws, 10.0 + 5.0 * rank)
    import torch.distributed as dist

    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        assert dict(out) == {0: 15.0, 1: 15.0}


def test_reference_arm_prints_only_on_rank_0(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup = 1, 0

    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""
