"""The sharded Gram's device entry points on one GPU.

``gakco_gram_partial_device`` computes one slice of a dataset's masks into
C_0..C_M and ``gakco_combine_device`` finishes a summed C (Section 2.2
"Parallelization", S:5.3, Eq. 8, Eq. 9, Eq. 7).  The ranks of a sharded run
are emulated one after another on this GPU (no rank waits on another): the
slices' buffers are summed on the device, combined, and must equal the
regular Gram call and the oracle bit for bit (K, N_m; Khat within 1e-12).
Slices cut through dense and sparse levels alike.
"""

import numpy as np
import pytest

import oracle
import paper_1704_07468_gb300 as pkg
from paper_1704_07468_gb300 import shard, synth

pytestmark = pytest.mark.gpu
KHAT_RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_07468_gb300 import build as lib_build
    lib_build.build()
    oracle.build()


def _sharded(sigma, g, k, codes, off, world, opts=None, weights=None):
    import torch

    dev = torch.device("cuda:0")
    n, M = len(off) - 1, g - k
    d_codes = torch.from_numpy(codes if len(codes) else np.zeros(1, np.uint8)).to(dev)
    stream = torch.cuda.current_stream().cuda_stream
    with pkg.gakco_create(sigma, g, k) as ctx:
        for name, v in (opts or {}).items():
            ctx.set_option(name, v)
        total = torch.zeros((M + 1, n, n), dtype=torch.int32, device=dev)
        spans = shard.mask_slices(ctx.num_masks(), world, weights)
        for b, e in spans:
            C = torch.full((M + 1, n, n), -1, dtype=torch.int32, device=dev)
            ctx.gram_partial_device(d_codes.data_ptr(), off, b, e, C.data_ptr(), stream)
            low = torch.tril(torch.ones(n, n, dtype=torch.bool, device=dev), -1)
            assert not C[:, low].any(), "partial C must leave the lower triangles zero"
            total += C
        K = torch.empty((n, n), dtype=torch.int32, device=dev)
        Kh = torch.empty((n, n), dtype=torch.float64, device=dev)
        Nm = torch.empty((M + 1, n, n), dtype=torch.int32, device=dev)
        ctx.combine_device(total.data_ptr(), n, K.data_ptr(), Kh.data_ptr(), Nm.data_ptr(), stream)
        torch.cuda.synchronize()
        return {"K": K.cpu().numpy(), "Khat": Kh.cpu().numpy(), "Nm": Nm.cpu().numpy()}


def _check(out, ref):
    np.testing.assert_array_equal(out["K"], ref["K"])
    np.testing.assert_array_equal(out["Nm"], ref["Nm"])
    err = np.abs(out["Khat"] - ref["Khat"])
    assert np.all(err <= KHAT_RTOL * np.abs(ref["Khat"]) + 1e-300)


@pytest.mark.parametrize("case", [  # (seed, n, sigma, lo, hi, g, k, world, opts)
    (150, 60, 4, 0, 300, 10, 6, 2, {}),
    (151, 60, 4, 100, 300, 10, 6, 3, {"dense": 2}),        # slices cut the dense levels 2-4
    (152, 45, 20, 10, 400, 8, 4, 4, {}),
    (153, 40, 36, 5, 300, 8, 5, 7, {"heavy": 1}),
    (154, 25, 4, 0, 60, 5, 4, 9, {}),                         # more ranks than some levels' masks
])
def test_sharded_slices_sum_to_the_gram_matrix(case):
    seed, n, sigma, lo, hi, g, k, world, opts = case
    codes, off = synth.random_small(seed, n, sigma, lo, hi)
    ref = oracle.gram(codes, off, g, k)
    _check(_sharded(sigma, g, k, codes, off, world, opts), ref)


def test_one_slice_and_empty_slices():
    codes, off = synth.random_small(155, 30, 4, 50, 200)
    ref = oracle.gram(codes, off, 7, 5)
    _check(_sharded(4, 7, 5, codes, off, 1), ref)
    # Weights that put every mask on the last rank: the others' slices are empty.
    w = [0.0] * 28 + [1.0]
    _check(_sharded(4, 7, 5, codes, off, 3, weights=w), ref)


def test_partial_rejects_bad_slices():
    import torch

    codes, off = synth.random_small(156, 5, 4, 20, 40)
    d = torch.from_numpy(codes).to("cuda:0")
    C = torch.empty((3, 5, 5), dtype=torch.int32, device="cuda:0")
    with pkg.gakco_create(4, 7, 5) as ctx:
        nm = ctx.num_masks()
        assert nm == 1 + 7 + 21
        for b, e in ((-1, 3), (4, 2), (0, nm + 1)):
            with pytest.raises(pkg.GakcoError):
                ctx.gram_partial_device(d.data_ptr(), off, b, e, C.data_ptr())
        ctx.set_option("engine", 1)
        with pytest.raises(pkg.GakcoError):
            ctx.gram_partial_device(d.data_ptr(), off, 0, nm, C.data_ptr())
