"""Host logic of the multi-GPU benchmark path, on CPU with gloo.

Each rank of `bench.py --gpus N` processes its own independently seeded
batch of datasets (weak scaling, no collective on the data path); the only
collective is the max of the step time over ranks, taken outside the timed
region.  These tests run that logic with two gloo ranks."""

import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    step_ms = 10.0 + 5.0 * rank          # rank 1 is the slowest
    mx = bench.reduce_max(step_ms)
    desc, sigma, g, k, sets = bench.make_workload("dna_toy", r)
    out[rank] = (ws, r, local, mx, int(sets[0][0][:64].sum()), len(sets[0][1]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_get_distinct_data():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][:3] == (2, 0, 0) and res[1][:3] == (2, 1, 1)
    assert res[0][3] == res[1][3] == 15.0        # max over ranks
    assert res[0][5] == res[1][5]                # same shapes (weak scaling)
    assert res[0][4] != res[1][4]                # independently seeded data


def test_reference_arm_is_rank0_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        workload, dna_sizes, steps, warmup, ref_rows, gpus = "dna_toy", None, 1, 0, 2, 2

    bench.run_reference(A)
    assert capsys.readouterr().out == ""
