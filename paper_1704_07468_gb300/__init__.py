"""GB300-native gapped k-mer string kernel (GaKCo, arXiv 1704.07468).

Thin Python binding over the C ABI declared in ``include/gakco.h``: argument
marshalling only, every step of the computation runs in the CUDA library
``_lib/libgakco.so``.  The names mirror the C functions:

    ctx = gakco_create(sigma, g, k)
    out = ctx.gram(codes, offsets, khat=True, nm=False)      # host buffers
    ctx.gram_device(codes_ptr, offsets, n, K_ptr, ...)       # device buffers

Loading fails loudly (``RuntimeError``) when the library is missing; there
is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["gakco_create", "gakco_gram_device_noalloc", "gakco_measure_smem_atomics", "Context", "GakcoError", "load_library",
           "library_path", "OPT", "STAT", "ERRORS"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libgakco.so")
_lib = None

GAKCO_OK = 0
GAKCO_E_PENDING = -6
ERRORS = {
    -1: "GAKCO_E_INVALID", -2: "GAKCO_E_OOM", -3: "GAKCO_E_OVERFLOW",
    -4: "GAKCO_E_CUDA", -5: "GAKCO_E_TIMEOUT", -6: "GAKCO_E_PENDING",
    -7: "GAKCO_E_INTERNAL",
}
OPT = {"engine": 1, "radix_bits": 2, "chunk_elems": 3, "graph": 4,
       "accum_threads": 5, "profile": 6, "smem_cols": 7,
       "fail_alloc_after": 8, "group_bytes": 9, "serve_slots": 10,
       "serve_max_seqs": 11, "serve_max_windows": 12, "serve_mem_bytes": 13,
       "dense": 14, "dense_bytes": 15, "dense_overflow": 16,
       "dense_run_cols": 17, "kernel_only": 18, "overlap": 19, "dense_sms": 20,
       "heavy": 21, "heavy_bytes": 22, "direct_d2h": 23,
       "dense_round_sum": 24, "dense_wait_cycles": 25, "sort": 26,
       "accum_variant": 27, "rle_items": 28,
       "level_radix_bits": 29, "dense_split": 30,
       "dense_late": 31}
STAT = {"launches": 1, "mask_passes": 2, "device_bytes": 3,
        "graph_replay": 4, "pair_updates": 5, "entries_visited": 6,
        "windows_visited": 7, "served_batches": 8, "served_requests": 9,
        "dense_problems": 10, "dense_flops": 11, "dense_issued_flops": 12,
        "dense_bytes": 13, "sort_bytes": 14, "heavy_columns": 15,
        "heavy_flops": 16, "rle_bytes": 17, "pack_bytes": 18, "combine_bytes": 19,
        "masks": 20}


class GakcoError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"{ERRORS.get(code, code)}: {message}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


def library_path() -> str:
    return _LIB_PATH


def load_library(build_if_missing: bool = False):
    """Load the CUDA library.  Raises RuntimeError if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from . import build as _build
        _build.build()
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(
            f"GaKCo CUDA library not found at {_LIB_PATH}; build it with "
            "`python -m paper_1704_07468_gb300.build` (there is no CPU fallback)")
    lib = ctypes.CDLL(_LIB_PATH)
    p, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "gakco_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, pp], ctypes.c_int),
        "gakco_destroy": ([p], None),
        "gakco_last_error": ([p], ctypes.c_char_p),
        "gakco_set_option": ([p, ctypes.c_int, i64], ctypes.c_int),
        "gakco_get_stat": ([p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "gakco_kernel_timing": ([p, ctypes.c_int, ctypes.c_char_p, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "gakco_gram": ([p, p, p, i32, p, p, p], ctypes.c_int),
        "gakco_gram_batch": ([p, i32, p, p, p, p, p, p], ctypes.c_int),
        "gakco_gram_device": ([p, p, p, i32, p, p, p, p], ctypes.c_int),
        "gakco_gram_batch_device": ([p, i32, p, p, p, p, p, p, p], ctypes.c_int),
        "gakco_autotune": ([p, i32, p, p, p, p, ctypes.c_char_p, ctypes.c_int], ctypes.c_int),
        "gakco_fit": ([p, p, p, i32], ctypes.c_int),
        "gakco_fit_device": ([p, p, p, i32, p], ctypes.c_int),
        "gakco_cross_fitted": ([p, p, p, i32, p, p], ctypes.c_int),
        "gakco_cross_fitted_device": ([p, p, p, i32, p, p, p], ctypes.c_int),
        "gakco_cross": ([p, p, p, i32, p, p, i32, p, p], ctypes.c_int),
        "gakco_submit": ([p, p, p, i32, p, p, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "gakco_poll": ([p, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_double)],
                       ctypes.c_int),
        "gakco_set_svm": ([p, p, i32, ctypes.c_double, ctypes.c_int], ctypes.c_int),
        "gakco_extend": ([p, p, p, i32, p, p], ctypes.c_int),
        "gakco_decision": ([p, p, p, i32, p], ctypes.c_int),
        "gakco_submit_svm": ([p, p, p, i32, p, p, p, ctypes.POINTER(ctypes.c_uint64)],
                             ctypes.c_int),
        "gakco_gram_partial_device": ([p, p, p, i32, i32, i32, p, p], ctypes.c_int),
        "gakco_combine_device": ([p, p, i32, p, p, p, p], ctypes.c_int),
        "gakco_measure_smem_atomics": ([p, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "gakco_measure_smem_atomics_pattern": ([p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)],
                                               ctypes.c_int),
        "gakco_gram_device_noalloc": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, p, p, i32,
                                       p, p, p, p, ctypes.c_char_p, ctypes.c_int],
                                      ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * max(1, len(ptrs)))()
    for i, v in enumerate(ptrs):
        arr[i] = v
    return arr


def _dataset(codes, offsets):
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    return codes, offsets


class Context:
    """A GaKCo engine context for one (sigma, g, k)."""

    def __init__(self, sigma: int, g: int, k: int):
        self._lib = load_library()
        h = ctypes.c_void_p()
        rc = self._lib.gakco_create(int(sigma), int(g), int(k), ctypes.byref(h))
        if rc != GAKCO_OK:
            raise GakcoError(rc, f"gakco_create(sigma={sigma}, g={g}, k={k}) failed")
        self._h = h
        self.sigma, self.g, self.k, self.M = int(sigma), int(g), int(k), int(g) - int(k)
        self._ntrain = 0
        self._inflight = {}

    # -- lifetime --------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.gakco_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- helpers ---------------------------------------------------------
    def last_error(self) -> str:
        return self._lib.gakco_last_error(self._h).decode()

    def _check(self, rc):
        if rc != GAKCO_OK:
            raise GakcoError(rc, self.last_error())

    def set_option(self, name, value):
        key = OPT[name] if isinstance(name, str) else int(name)
        self._check(self._lib.gakco_set_option(self._h, key, int(value)))
        return self

    def get_stat(self, name) -> float:
        key = STAT[name] if isinstance(name, str) else int(name)
        v = ctypes.c_double()
        self._check(self._lib.gakco_get_stat(self._h, key, ctypes.byref(v)))
        return v.value

    def kernel_timings(self):
        """{kernel name: (total ms, launches)} of the last profiled call."""
        out = {}
        buf = ctypes.create_string_buffer(64)
        ms, n = ctypes.c_double(), ctypes.c_int64()
        i = 0
        while self._lib.gakco_kernel_timing(self._h, i, buf, 64, ctypes.byref(ms),
                                            ctypes.byref(n)) == GAKCO_OK:
            out[buf.value.decode()] = (ms.value, n.value)
            i += 1
        return out

    # -- host-buffer calls -----------------------------------------------
    def gram(self, codes, offsets, khat=True, nm=False, K=True, out=None):
        """Gram kernel of one dataset (host arrays).  Returns a dict with
        ``K`` (n, n) int32, ``Khat`` (n, n) float64, ``Nm`` (M+1, n, n).
        ``out``: such a dict to write into instead of new arrays."""
        return self.gram_batch([(codes, offsets)], khat=khat, nm=nm, K=K,
                               out=None if out is None else [out])[0]

    def gram_batch(self, datasets, khat=True, nm=False, K=True, out=None):
        """Gram kernels of several datasets in one batched call.  ``out``:
        one dict per dataset (keys ``K``, ``Khat``, ``Nm``, C-contiguous
        arrays of the shapes and dtypes above) that the call writes into, so
        that repeated calls reuse their host buffers; returned as given."""
        ds = [_dataset(c, o) for c, o in datasets]
        nd = len(ds)
        ns = np.array([len(o) - 1 for _, o in ds], dtype=np.int32)
        if out is not None:
            if len(out) != nd:
                raise ValueError("out needs one dict per dataset")
            specs = (("K", K, np.int32, lambda n: (n, n)), ("Khat", khat, np.float64, lambda n: (n, n)),
                     ("Nm", nm, np.int32, lambda n: (self.M + 1, n, n)))
            for o, n in zip(out, ns):
                for key, want, dt, shape in specs:
                    a = o.get(key) if want else None
                    if want and (a is None or a.dtype != dt or a.shape != shape(int(n))
                                 or not a.flags.c_contiguous or not a.flags.writeable):
                        raise ValueError(f"out[{key!r}] must be a writable C-contiguous "
                                         f"{np.dtype(dt).name} array of shape {shape(int(n))}")
                    o[key] = a
            outs = out
        else:
            outs = []
            for (c, o), n in zip(ds, ns):
                outs.append({
                    "K": np.empty((n, n), np.int32) if K else None,
                    "Khat": np.empty((n, n), np.float64) if khat else None,
                    "Nm": np.empty((self.M + 1, n, n), np.int32) if nm else None,
                })
        keep = [c if c.size else np.zeros(1, np.uint8) for c, _ in ds]
        rc = self._lib.gakco_gram_batch(
            self._h, nd,
            _ptr_array([k.ctypes.data for k in keep]),
            _ptr_array([o.ctypes.data for _, o in ds]),
            ns.ctypes.data_as(ctypes.c_void_p),
            _ptr_array([o["K"].ctypes.data if o["K"] is not None else None for o in outs]),
            _ptr_array([o["Khat"].ctypes.data if o["Khat"] is not None else None for o in outs]),
            _ptr_array([o["Nm"].ctypes.data if o["Nm"] is not None else None for o in outs]))
        self._check(rc)
        return outs

    def autotune_device(self, codes_ptrs, offsets, stream=None):
        """Tune speed options on these datasets (device codes); returns the
        library's report of the choice."""
        offs = [np.ascontiguousarray(o, dtype=np.int64) for o in offsets]
        ns = np.array([len(o) - 1 for o in offs], dtype=np.int32)
        rep = ctypes.create_string_buffer(256)
        self._check(self._lib.gakco_autotune(
            self._h, len(offs), _ptr_array(codes_ptrs), _ptr_array([o.ctypes.data for o in offs]),
            ns.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(stream) if stream else None,
            rep, 256))
        return rep.value.decode()

    # -- device-buffer calls ---------------------------------------------
    def gram_device(self, codes_ptr, offsets, K_ptr, Khat_ptr=None, Nm_ptr=None,
                    stream=None):
        """Device form: pointers are device addresses (ints), ``offsets`` a
        host int64 array, ``stream`` a cudaStream_t as int (None = default)."""
        return self.gram_batch_device([codes_ptr], [offsets], [K_ptr], [Khat_ptr],
                                      [Nm_ptr], stream)

    def gram_batch_device(self, codes_ptrs, offsets, K_ptrs, Khat_ptrs=None,
                          Nm_ptrs=None, stream=None):
        nd = len(codes_ptrs)
        offs = [np.ascontiguousarray(o, dtype=np.int64) for o in offsets]
        ns = np.array([len(o) - 1 for o in offs], dtype=np.int32)
        Khat_ptrs = Khat_ptrs or [None] * nd
        Nm_ptrs = Nm_ptrs or [None] * nd
        rc = self._lib.gakco_gram_batch_device(
            self._h, nd, _ptr_array(codes_ptrs),
            _ptr_array([o.ctypes.data for o in offs]),
            ns.ctypes.data_as(ctypes.c_void_p), _ptr_array(K_ptrs),
            _ptr_array(Khat_ptrs), _ptr_array(Nm_ptrs),
            ctypes.c_void_p(stream) if stream else None)
        self._check(rc)

    def gram_partial_device(self, codes_ptr, offsets, mask_begin, mask_end, C_ptr, stream=None):
        """Contribution of masks [mask_begin, mask_end) to C_0..C_M (C:
        ``gakco_gram_partial_device``): ``C_ptr`` is a device buffer of
        (M+1) x n x n uint32, upper triangles written, lower ones zero."""
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        rc = self._lib.gakco_gram_partial_device(
            self._h, ctypes.c_void_p(codes_ptr), off.ctypes.data_as(ctypes.c_void_p),
            len(off) - 1, int(mask_begin), int(mask_end), ctypes.c_void_p(C_ptr),
            ctypes.c_void_p(stream) if stream else None)
        self._check(rc)

    def combine_device(self, C_ptr, n, K_ptr, Khat_ptr=None, Nm_ptr=None, stream=None):
        """Eq. 9, Eq. 7 and the normalisation on a summed C (C:
        ``gakco_combine_device``)."""
        rc = self._lib.gakco_combine_device(
            self._h, ctypes.c_void_p(C_ptr), int(n), ctypes.c_void_p(K_ptr),
            ctypes.c_void_p(Khat_ptr) if Khat_ptr else None,
            ctypes.c_void_p(Nm_ptr) if Nm_ptr else None,
            ctypes.c_void_p(stream) if stream else None)
        self._check(rc)

    def num_masks(self) -> int:
        """c_gk, the position masks of all levels (a sharded Gram's units)."""
        return int(self.get_stat("masks"))


def _add_cross_methods(cls):
    """Cross-kernel and serving methods (C: gakco_fit, gakco_cross_fitted,
    gakco_cross, gakco_submit, gakco_poll)."""

    def fit(self, codes, offsets):
        codes, offsets = _dataset(codes, offsets)
        keep = codes if codes.size else np.zeros(1, np.uint8)
        self._check(self._lib.gakco_fit(self._h, keep.ctypes.data, offsets.ctypes.data,
                                        len(offsets) - 1))
        self._ntrain = len(offsets) - 1
        return self

    def fit_device(self, codes_ptr, offsets, stream=None):
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self._check(self._lib.gakco_fit_device(self._h, codes_ptr, offsets.ctypes.data,
                                               len(offsets) - 1,
                                               ctypes.c_void_p(stream) if stream else None))
        self._ntrain = len(offsets) - 1
        return self

    def cross_fitted(self, codes, offsets, khat=True, K=True):
        codes, offsets = _dataset(codes, offsets)
        nt = len(offsets) - 1
        out = {"K": np.empty((nt, self._ntrain), np.int32) if K else None,
               "Khat": np.empty((nt, self._ntrain), np.float64) if khat else None}
        keep = codes if codes.size else np.zeros(1, np.uint8)
        self._check(self._lib.gakco_cross_fitted(
            self._h, keep.ctypes.data, offsets.ctypes.data, nt,
            _ptr(out["K"]), _ptr(out["Khat"])))
        return out

    def cross_fitted_device(self, codes_ptr, offsets, K_ptr, Khat_ptr=None, stream=None):
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self._check(self._lib.gakco_cross_fitted_device(
            self._h, codes_ptr, offsets.ctypes.data, len(offsets) - 1, K_ptr, Khat_ptr,
            ctypes.c_void_p(stream) if stream else None))

    def cross(self, test, train, khat=True):
        """K(test, train) for host datasets (fit + cross_fitted)."""
        self.fit(*train)
        return self.cross_fitted(*test, khat=khat)

    def extend(self, codes, offsets, khat=True):
        """Add sequences to the fitted set; returns the new rows of the
        union's Gram matrix (old sequences first), nb x (n + nb)."""
        codes, offsets = _dataset(codes, offsets)
        nb = len(offsets) - 1
        N = self._ntrain + nb
        out = {"K": np.empty((nb, N), np.int32), "Khat": np.empty((nb, N), np.float64) if khat else None}
        keep = codes if codes.size else np.zeros(1, np.uint8)
        self._check(self._lib.gakco_extend(self._h, keep.ctypes.data, offsets.ctypes.data, nb,
                                           _ptr(out["K"]) if nb else None,
                                           _ptr(out["Khat"]) if nb else None))
        self._ntrain = N
        return out

    def set_svm(self, coef, bias=0.0, kind=0):
        """Coefficients alpha_i * y_i of the fitted training set and the bias
        for decision values (Eq. 1); kind 0 uses Khat, 1 uses K."""
        coef = np.ascontiguousarray(coef, dtype=np.float64)
        self._check(self._lib.gakco_set_svm(self._h, _ptr(coef) if coef.size else None, len(coef),
                                            float(bias), int(kind)))
        return self

    def decision(self, codes, offsets):
        """SVM decision values of test sequences against the fitted set."""
        codes, offsets = _dataset(codes, offsets)
        nt = len(offsets) - 1
        f = np.empty(nt, np.float64)
        keep = codes if codes.size else np.zeros(1, np.uint8)
        self._check(self._lib.gakco_decision(self._h, keep.ctypes.data, offsets.ctypes.data, nt,
                                             _ptr(f) if nt else None))
        return f

    def submit(self, codes, offsets, khat=True, K=True, decision=False):
        """Queue a cross-kernel request; returns its ticket.  The output
        arrays are kept alive by the context until poll() reports done."""
        codes, offsets = _dataset(codes, offsets)
        nt = len(offsets) - 1
        out = {"K": np.empty((nt, self._ntrain), np.int32) if K else None,
               "Khat": np.empty((nt, self._ntrain), np.float64) if khat else None,
               "decision": np.empty(nt, np.float64) if decision else None}
        keep = codes if codes.size else np.zeros(1, np.uint8)
        t = ctypes.c_uint64()
        rc = self._lib.gakco_submit_svm(self._h, keep.ctypes.data, offsets.ctypes.data, nt,
                                        _ptr(out["K"]), _ptr(out["Khat"]), _ptr(out["decision"]),
                                        ctypes.byref(t))
        self._check(rc)
        self._inflight[t.value] = out
        return t.value

    def poll(self, ticket, timeout_ms=0):
        """None while pending; else the result dict with ``latency_ms``."""
        lat = ctypes.c_double()
        rc = self._lib.gakco_poll(self._h, ctypes.c_uint64(ticket), int(timeout_ms),
                                  ctypes.byref(lat))
        if rc == GAKCO_E_PENDING:
            return None
        out = self._inflight.pop(ticket, None)
        self._check(rc)
        out["latency_ms"] = lat.value
        return out

    for f in (fit, fit_device, cross_fitted, cross_fitted_device, cross, extend, set_svm, decision, submit,
              poll):
        setattr(cls, f.__name__, f)
    return cls


def gakco_gram_device_noalloc(sigma, g, k, codes_ptr, offsets, K_ptr, Khat_ptr=None,
                              Nm_ptr=None, stream=None):
    """Gram kernel without any allocation (C: ``gakco_gram_device_noalloc``).

    For callers that may not let the library allocate device memory (memory
    owned by a framework's pool or budget, allocation-free request paths,
    plug-ins handed their buffers).  Intermediate data lives in the
    library's 64 MiB static device array; calls must not overlap on the GPU.
    Pointers are device addresses (ints); ``offsets`` is a host int64 array.
    """
    lib = load_library()
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    err = ctypes.create_string_buffer(256)
    rc = lib.gakco_gram_device_noalloc(int(sigma), int(g), int(k), codes_ptr,
                                       offsets.ctypes.data, len(offsets) - 1, K_ptr,
                                       Khat_ptr, Nm_ptr, stream, err, 256)
    if rc != GAKCO_OK:
        raise GakcoError(rc, err.value.decode())


_add_cross_methods(Context)


def gakco_measure_smem_atomics(stream=None, random_columns=False) -> float:
    """Shared-memory atomic adds per second of the current GPU, conflict-free
    or at random columns of a 4096-word row (C:
    ``gakco_measure_smem_atomics_pattern``)."""
    lib = load_library()
    v = ctypes.c_double()
    rc = lib.gakco_measure_smem_atomics_pattern(ctypes.c_void_p(stream) if stream else None,
                                                int(bool(random_columns)), ctypes.byref(v))
    if rc != GAKCO_OK:
        raise GakcoError(rc, "shared-memory atomic probe failed")
    return v.value


def gakco_create(sigma: int, g: int, k: int) -> Context:
    """Create an engine context (C: ``gakco_create``)."""
    return Context(sigma, g, k)
