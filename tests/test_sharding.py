"""Mask-sharded Gram computation on CPU ranks (gloo).

Every (level, mask) pass of countAndUpdate is independent and C_m is the
sum of the passes' contributions (Section 2.2 "Parallelization", S:5.3,
Eq. 8).  ``paper_1704_07468_gb300.shard`` splits a dataset's masks into
contiguous slices, one per rank, and adds the slices' C_0..C_M with one sum
all-reduce.  Here the ranks are gloo processes on CPU; each computes its
slice with the oracle's per-mask counting route (the GPU path uses
``gakco_gram_partial_device`` instead), and the reduced profiles, through
Eq. 9 and Eq. 7, must equal the oracle's brute-force N_m and K bit for bit
on every rank.
"""

import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_1704_07468_gb300 import shard, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("nmasks,world", [(29, 2), (29, 3), (386, 8), (3, 5), (1, 1), (0, 2)])
def test_slices_cover_every_mask_once(nmasks, world):
    sl = shard.mask_slices(nmasks, world)
    assert len(sl) == world
    assert sl[0][0] == 0 and sl[-1][1] == nmasks
    for (a, b), (c, d) in zip(sl, sl[1:]):
        assert a <= b == c <= d
    sizes = [b - a for a, b in sl]
    assert max(sizes) - min(sizes) <= 1


def test_weighted_slices_balance_the_weight():
    # Level-ordered masks of g = 10, M = 4 weighted by level (later levels
    # cost more): contiguous slices of near-equal weight.
    from math import comb
    w = [float(4 ** m) for m in range(5) for _ in range(comb(10, m))]
    sl = shard.mask_slices(len(w), 4, w)
    tot = [sum(w[a:b]) for a, b in sl]
    assert sum(tot) == sum(w)
    assert max(tot) - min(tot) <= 2 * max(w)
    with pytest.raises(ValueError):
        shard.mask_slices(3, 2, [1.0, -1.0, 1.0])


def _worker(rank, world, port, case, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    seed, n, sigma, lo, hi, g, k = case
    M = g - k
    codes, off = synth.random_small(seed, n, sigma, lo, hi)
    masks = oracle.position_masks(g, M)

    def partial(begin, end, C):
        part = oracle.cumulative_profile(codes, off, g, M, masks[begin:end])
        C.copy_(torch.from_numpy(part.astype(np.int32)))

    C = torch.full((M + 1, n, n), -7, dtype=torch.int32)
    span = shard.sharded_profile(partial, len(masks), C)
    out[rank] = (span, C.numpy().copy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_shard_one_dataset(world):
    case = (90, 9, 4, 0, 40, 6, 3)  # n = 9, g = 6, k = 3: 42 masks over 4 levels
    seed, n, sigma, lo, hi, g, k = case
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, case, out), nprocs=world, join=True)
        res = dict(out)
    spans = [res[r][0] for r in range(world)]
    assert spans == shard.mask_slices(len(oracle.position_masks(g, g - k)), world)
    assert all(b > a for a, b in spans)                      # every rank had work
    codes, off = synth.random_small(seed, n, sigma, lo, hi)
    ref = oracle.gram(codes, off, g, k)
    for r in range(world):
        C = res[r][1].astype(np.int64)
        np.testing.assert_array_equal(C, res[0][1])        # same result on every rank
        N = oracle.inclusion_exclusion(C, g)
        np.testing.assert_array_equal(N, ref["Nm"])
        np.testing.assert_array_equal(oracle.kernel_from_profile(N, g, k), ref["K"])
