"""The N > 1 launch of bench.py on CPU (gloo, world size 2): every rank advances its own
replica, so replicas draw different mode sets from the same seed (key word 1 is
seed_hi ^ replica), the job time is the slowest rank's, and only rank 0 reports."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    ws, r, local = bench.dist_info()
    t = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
    m, S = oracle.sample_k(11, 3, r, np.array([60.0, 60.0, 60.0]), 0.09, 64)
    ms = [None] * world
    dist.all_gather_object(ms, m.tolist())
    out[rank] = (ws, r, t, ms, S)
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_time():
    pytest.importorskip("torch.distributed")
    port = _free_port()
    # spawn, not fork: earlier tests may have started OpenMP threads in this process
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        ws, r, t, ms, S = res[rank]
        assert ws == 2 and r == rank
        assert t == 15.0  # the slowest rank's time on every rank
        assert ms[0] != ms[1]  # independent replicas: different mode sets
    assert res[0][3] == res[1][3]  # both ranks see the same pair of sets
    assert res[0][4] == res[1][4]  # S depends on the box, not the replica


def test_reference_arm_other_ranks_do_nothing(capsys, monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(type("A", (), {"steps": 1, "warmup": 0, "N": 64, "P": 8,
                                               "gpus": 2})()) is None
    assert capsys.readouterr().out == ""
