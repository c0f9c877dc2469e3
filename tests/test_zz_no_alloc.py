"""The allocation-free Gram entry point against the regular one and the
oracle.

``gakco_gram_device_noalloc`` serves callers that may not let the library
allocate device memory (memory owned by a framework's pool or budget,
request paths that cannot take cudaMalloc's device-wide synchronisation,
plug-ins handed their buffers).  It keeps all intermediate data in a static
device array that every call reuses, so this test makes two calls in a row
with different inputs and checks each against ``gakco_gram_device`` and the
CPU oracle: K and N_m bit-exact, the normalised kernel within 1e-12
relative.  It also checks that further calls leave the device's free
memory unchanged, and the case where no sequence has a window.  The file
name makes pytest collect it last.
"""

import ctypes

import numpy as np
import pytest

import oracle
import paper_1704_07468_gb300 as pkg
from paper_1704_07468_gb300 import synth

pytestmark = pytest.mark.gpu
KHAT_RTOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    from paper_1704_07468_gb300 import build as lib_build
    lib_build.build()
    oracle.build()
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


def _call(torch, lib, sigma, g, k, d_codes, off, K, Kh, Nm):
    n = len(off) - 1
    off = np.ascontiguousarray(off, dtype=np.int64)
    err = ctypes.create_string_buffer(256)
    rc = lib.gakco_gram_device_noalloc(sigma, g, k, d_codes.data_ptr(), off.ctypes.data, n,
                                       K.data_ptr(), Kh.data_ptr(), Nm.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream, err, 256)
    assert rc == 0, err.value.decode()


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
        ref = oracle.gram(codes, off, g, k)
        np.testing.assert_array_equal(K1, ref["K"])
        np.testing.assert_array_equal(Nm1, ref["Nm"])
        assert np.all(np.abs(Kh1 - ref["Khat"]) <= KHAT_RTOL * np.abs(ref["Khat"]) + 1e-300)


def test_noalloc_calls_leave_device_memory_unchanged(lib):
    import torch

    sigma, g, k = 20, 8, 4
    codes, off = synth.random_small(73, 120, sigma, 0, 500)
    d_codes = torch.from_numpy(codes).to("cuda:0")
    n = len(off) - 1
    K, Kh, Nm = _buffers(torch, n, g - k)
    _call(torch, lib, sigma, g, k, d_codes, off, K, Kh, Nm)  # warm: kernels loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    held0 = torch.cuda.memory_allocated()
    for _ in range(3):
        _call(torch, lib, sigma, g, k, d_codes, off, K, Kh, Nm)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
    assert torch.cuda.memory_allocated() == held0
    ref = oracle.gram(codes, off, g, k)
    np.testing.assert_array_equal(K.cpu().numpy(), ref["K"])


def test_noalloc_without_any_window(lib):
    """Every sequence shorter than g (and one empty): no window, so K, Khat
    and every N_m are zero; the call succeeds."""
    import torch

    codes, off = synth.random_small(74, 6, 4, 0, 6)
    codes, off = synth.pack([codes[off[i]:off[i + 1]] for i in range(6)] + [np.zeros(0, np.uint8)])
    assert np.all(np.diff(off) < 7) and off[-1] == off[-2]
    d_codes = torch.from_numpy(codes if len(codes) else np.zeros(1, np.uint8)).to("cuda:0")
    K, Kh, Nm = _noalloc(torch, lib, 4, 7, 5, d_codes, off)
    assert not K.any() and not Kh.any() and not Nm.any()
    ref = oracle.gram(codes, off, 7, 5)
    np.testing.assert_array_equal(K, ref["K"])
    np.testing.assert_array_equal(Kh, ref["Khat"])


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
