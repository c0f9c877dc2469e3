"""The allocation-free Gram entry point against the regular one.

``gakco_gram_device_noalloc`` serves callers that may not let the library
allocate device memory (memory owned by a framework's pool or budget,
request paths that cannot take cudaMalloc's device-wide synchronisation,
plug-ins handed their buffers).  It keeps all intermediate data in a static
device array that every call reuses, so this test makes two calls in a row
with different inputs and checks each against ``gakco_gram_device``: K and
N_m bit-exact, the normalised kernel within 1e-12 relative.  The file name
makes pytest collect it last.
"""

import ctypes

import numpy as np
import pytest

import paper_1704_07468_gb300 as pkg
from paper_1704_07468_gb300 import synth

pytestmark = pytest.mark.gpu
KHAT_RTOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    from paper_1704_07468_gb300 import build as lib_build
    lib_build.build()
    return pkg.load_library()


def _buffers(torch, n, M):
    dev = torch.device("cuda:0")
    return (torch.full((n, n), -1, dtype=torch.int32, device=dev),
            torch.full((n, n), -1.0, dtype=torch.float64, device=dev),
            torch.full((M + 1, n, n), -1, dtype=torch.int32, device=dev))


def _regular(torch, sigma, g, k, d_codes, off):
    n = len(off) - 1
    K, Kh, Nm = _buffers(torch, n, g - k)
    with pkg.gakco_create(sigma, g, k) as ctx:
        ctx.gram_device(d_codes.data_ptr(), off, K.data_ptr(), Kh.data_ptr(), Nm.data_ptr(),
                        stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return K.cpu().numpy(), Kh.cpu().numpy(), Nm.cpu().numpy()


def _noalloc(torch, lib, sigma, g, k, d_codes, off):
    n = len(off) - 1
    K, Kh, Nm = _buffers(torch, n, g - k)
    off = np.ascontiguousarray(off, dtype=np.int64)
    err = ctypes.create_string_buffer(256)
    rc = lib.gakco_gram_device_noalloc(sigma, g, k, d_codes.data_ptr(), off.ctypes.data, n,
                                       K.data_ptr(), Kh.data_ptr(), Nm.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream, err, 256)
    assert rc == 0, err.value.decode()
    torch.cuda.synchronize()
    return K.cpu().numpy(), Kh.cpu().numpy(), Nm.cpu().numpy()


def test_noalloc_matches_regular_entry_point_on_two_calls_in_a_row(lib):
    import torch

    cases = [
        (20, 8, 4, synth.random_small(70, 90, 20, 0, 400)),
        (4, 7, 5, synth.random_small(71, 31, 4, 0, 150)),  # smaller: stale data must not leak
    ]
    for sigma, g, k, (codes, off) in cases:
        d_codes = torch.from_numpy(codes).to("cuda:0")
        K0, Kh0, Nm0 = _regular(torch, sigma, g, k, d_codes, off)
        K1, Kh1, Nm1 = _noalloc(torch, lib, sigma, g, k, d_codes, off)
        np.testing.assert_array_equal(K1, K0)
        np.testing.assert_array_equal(Nm1, Nm0)
        assert np.all(np.abs(Kh1 - Kh0) <= KHAT_RTOL * np.abs(Kh0) + 1e-300)


def test_noalloc_rejects_inputs_beyond_its_static_area(lib):
    import torch

    # 5000 short sequences: the two C_m planes alone need 200 MB.
    codes, off = synth.random_small(72, 5000, 4, 20, 20)
    d_codes = torch.from_numpy(codes).to("cuda:0")
    K = torch.empty((5000, 5000), dtype=torch.int32, device="cuda:0")
    err = ctypes.create_string_buffer(256)
    rc = lib.gakco_gram_device_noalloc(4, 5, 4, d_codes.data_ptr(), off.ctypes.data, 5000,
                                       K.data_ptr(), None, None, None, err, 256)
    assert rc == -3 and b"scratch" in err.value
