"""CPU oracle for the gapped k-mer string kernel (GaKCo, arXiv 1704.07468).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this package.  The product path never
does; it shares no code with the CUDA library.

The oracle computes the kernel from its plain definition:

* mismatch profile N_m(x, y): the number of window pairs (i, j), one g-mer
  of x and one of y, at Hamming distance exactly m (Definition 1 and Eq. 7,
  Section 2.1), by brute force over all pairs in C (``gakco_oracle.c``);
* h_m = C(g - m, k) if g - m >= k, else 0 (Eq. 6);
* K(x, y) = sum_{m=0}^{g-k} h_m N_m(x, y) (Eq. 7);
* normalised kernel K(x, y) / sqrt(K(x, x) K(y, y)), set to 0 when either
  diagonal entry is 0.  The paper does not normalise; this output is part of
  the library's interface and is stated here in fp64 exactly as
  ``K / sqrt(Kxx * Kyy)`` with IEEE double arithmetic.

Every integer is int64; floating point is fp64.
"""

from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
from collections import Counter
from math import comb

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gakco_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``gakco_oracle.c`` into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                        "-pthread", _SRC, "-o", tmp], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        p = ctypes.c_void_p
        i32 = ctypes.c_int32
        lib.oracle_profile.argtypes = [p, p, p, i32, p, p, i32, i32, i32,
                                       i32, p]
        lib.oracle_profile.restype = ctypes.c_int
        lib.oracle_self_profile.argtypes = [p, p, i32, i32, i32, p]
        lib.oracle_self_profile.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _as_dataset(codes, offsets):
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    if codes.size == 0:
        codes = np.zeros(1, dtype=np.uint8)  # valid pointer, never read
    return codes, offsets


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def mismatch_profile(xcodes, xoff, g, maxd, rows=None, ycodes=None, yoff=None,
                     threads=None):
    """N_d(x, y) for d = 0..maxd, rows x of X (all if ``rows`` is None)
    against every y of Y (Y = X if not given).  Shape (maxd+1, nrows, ny)."""
    xcodes, xoff = _as_dataset(xcodes, xoff)
    if ycodes is None:
        ycodes, yoff = xcodes, xoff
    else:
        ycodes, yoff = _as_dataset(ycodes, yoff)
    nx = len(xoff) - 1
    ny = len(yoff) - 1
    rows = np.arange(nx, dtype=np.int32) if rows is None else \
        np.ascontiguousarray(rows, dtype=np.int32)
    out = np.zeros((maxd + 1, len(rows), ny), dtype=np.int64)
    if len(rows) == 0 or ny == 0:
        return out
    rc = _load().oracle_profile(_ptr(xcodes), _ptr(xoff), _ptr(rows),
                                len(rows), _ptr(ycodes), _ptr(yoff), ny, g,
                                maxd, threads or default_threads(), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_profile rejected its arguments")
    return out


def self_profile(codes, offsets, g, maxd):
    """N_d(x, x) for every x; shape (maxd+1, n)."""
    codes, offsets = _as_dataset(codes, offsets)
    n = len(offsets) - 1
    out = np.zeros((maxd + 1, n), dtype=np.int64)
    if n == 0:
        return out
    rc = _load().oracle_self_profile(_ptr(codes), _ptr(offsets), n, g, maxd,
                                     _ptr(out))
    if rc != 0:
        raise ValueError("oracle_self_profile rejected its arguments")
    return out


def h_coefficients(g, k):
    """h_m for m = 0..g-k (Eq. 6): C(g - m, k) when g - m >= k, else 0."""
    return np.array([comb(g - m, k) if g - m >= k else 0
                     for m in range(g - k + 1)], dtype=np.int64)


def kernel_from_profile(nm, g, k):
    """K = sum_m h_m N_m over m = 0..g-k (Eq. 7); ``nm`` is indexed by m on
    its first axis and may hold more levels than g-k (they are ignored)."""
    h = h_coefficients(g, k)
    return np.tensordot(h, nm[: len(h)], axes=(0, 0))


def normalise(K, diag_rows, diag_cols):
    """K(x, y) / sqrt(K(x, x) K(y, y)) in fp64; 0 where a diagonal is 0."""
    dx = np.asarray(diag_rows, dtype=np.float64)[:, None]
    dy = np.asarray(diag_cols, dtype=np.float64)[None, :]
    prod = dx * dy
    with np.errstate(divide="ignore", invalid="ignore"):
        out = np.asarray(K, dtype=np.float64) / np.sqrt(prod)
    out[prod == 0] = 0.0
    return out


def position_masks(g, M):
    """The deleted-position sets of levels m = 0..M (Section 2.2, step 3):
    all C(g, m) sets of m of the g positions, level by level, each level in
    lexicographic order."""
    return [d for m in range(M + 1) for d in itertools.combinations(range(g), m)]


def cumulative_profile(codes, offsets, g, M, deleted_sets=None):
    """The contributions of the given masks (default: all of levels 0..M)
    to the cumulative mismatch profiles C_m (Eq. 8), by the counting route
    of Section 2.2 (Fig. 2, steps 3-5): delete the mask's positions from
    every g-mer, count each remaining (g-m)-mer per sequence, and add
    c_x * c_y to C_m(x, y) over the (g-m)-mers x and y share.  Plain Python
    (tiny inputs only); shape (M+1, n, n), int64."""
    codes, offsets = np.asarray(codes), np.asarray(offsets, dtype=np.int64)
    n = len(offsets) - 1
    seqs = [codes[offsets[i]:offsets[i + 1]] for i in range(n)]
    wins = [[tuple(int(c) for c in s[i:i + g]) for i in range(len(s) - g + 1)] for s in seqs]
    C = np.zeros((M + 1, n, n), dtype=np.int64)
    for dele in (position_masks(g, M) if deleted_sets is None else deleted_sets):
        m = len(dele)
        keep = [p for p in range(g) if p not in dele]
        cnt = [Counter(tuple(w[p] for p in keep) for w in ws) for ws in wins]
        for x in range(n):
            for y in range(n):
                C[m, x, y] += sum(v * cnt[y].get(f, 0) for f, v in cnt[x].items())
    return C


def inclusion_exclusion(C, g):
    """Eq. 9: N_m = C_m - sum_{j<m} C(g-j, m-j) N_j for m = 0..M."""
    C = np.asarray(C, dtype=np.int64)
    N = np.zeros_like(C)
    for m in range(C.shape[0]):
        N[m] = C[m] - sum(comb(g - j, m - j) * N[j] for j in range(m))
    return N


def _check_gk(g, k):
    if not (1 <= k <= g):
        raise ValueError("need 1 <= k <= g")


def gram(codes, offsets, g, k, rows=None, threads=None):
    """Gram kernel of one dataset.

    Returns a dict with ``Nm`` (M+1, nrows, n), ``K`` (nrows, n), ``diag``
    (n,) = K(y, y) for every y, and ``Khat`` (nrows, n).
    """
    _check_gk(g, k)
    M = g - k
    n = len(offsets) - 1
    rows = np.arange(n, dtype=np.int32) if rows is None else \
        np.asarray(rows, dtype=np.int32)
    nm = mismatch_profile(codes, offsets, g, M, rows=rows, threads=threads)
    K = kernel_from_profile(nm, g, k)
    diag = kernel_from_profile(self_profile(codes, offsets, g, M), g, k)
    return {"Nm": nm, "K": K, "diag": diag,
            "Khat": normalise(K, diag[rows], diag)}


def cross(test_codes, test_off, train_codes, train_off, g, k, rows=None,
          threads=None):
    """Cross kernel K(test, train).  The test diagonal K(t, t) comes from
    each test sequence alone, the train diagonal from each train sequence.

    Returns ``Nm`` (M+1, nrows, ntrain), ``K``, ``Khat``, ``diag_test``
    (nt,), ``diag_train`` (ntrain,).
    """
    _check_gk(g, k)
    M = g - k
    nt = len(test_off) - 1
    rows = np.arange(nt, dtype=np.int32) if rows is None else \
        np.asarray(rows, dtype=np.int32)
    nm = mismatch_profile(test_codes, test_off, g, M, rows=rows,
                          ycodes=train_codes, yoff=train_off, threads=threads)
    K = kernel_from_profile(nm, g, k)
    dt = kernel_from_profile(self_profile(test_codes, test_off, g, M), g, k)
    dr = kernel_from_profile(self_profile(train_codes, train_off, g, M), g, k)
    return {"Nm": nm, "K": K, "diag_test": dt, "diag_train": dr,
            "Khat": normalise(K, dt[rows], dr)}
