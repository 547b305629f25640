"""Thin ctypes binding over ``libzoomsvd.so`` (the C ABI in include/zoomsvd.h).

Argument marshalling only: every step of the range-SVD path runs in the
library's CUDA kernels.  PyTorch supplies device memory for results and the
current CUDA stream.  If the library is missing, importing this module raises
— there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libzoomsvd.so")

ZS_F64, ZS_F32, ZS_BF16 = 0, 1, 2
ZS_FLAG_FP64_REFINE = 1
ZS_FLAG_EXACT_GRAM = 2
ZS_FLAG_ROW_APPEND = 4
DTYPES = {"f64": ZS_F64, "f32": ZS_F32, "bf16": ZS_BF16}
STATUS = {0: "ZS_OK", 1: "ZS_EINVAL", 2: "ZS_ERANGE", 3: "ZS_ENOMEM", 4: "ZS_EBUSY",
          5: "ZS_ETIMEDOUT", 6: "ZS_EDTYPE", 7: "ZS_ECUDA", 8: "ZS_EINTERNAL", 9: "ZS_ENOTFOUND",
          10: "ZS_ENOCONV"}


class ZsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class StoreConfig(C.Structure):
    _fields_ = [("n", C.c_int64), ("b", C.c_int64), ("k", C.c_int32), ("in_dtype", C.c_int32),
                ("capacity_rows", C.c_int64), ("device", C.c_int32), ("flags", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("U", C.c_void_p), ("ldu", C.c_int64), ("S", C.c_void_p), ("V", C.c_void_p),
                ("ldv", C.c_int64), ("rank", C.c_void_p)]


class ServeConfig(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("max_inflight", C.c_int32), ("queue_capacity", C.c_int32),
                ("memory_budget", C.c_int64)]


class ServeStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("rejected", C.c_int64), ("batches", C.c_int64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("max_ms", C.c_double),
                ("mean_ms", C.c_double), ("wall_s", C.c_double), ("queries_per_s", C.c_double),
                ("mean_batch", C.c_double)]


# name -> (restype, argtypes); exactly the functions include/zoomsvd.h declares
SIGNATURES = {
    "zs_store_create": (C.c_int, [C.POINTER(StoreConfig), C.POINTER(C.c_void_p)]),
    "zs_store_destroy": (None, [C.c_void_p]),
    "zs_store_append": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_void_p]),
    "zs_store_reset": (C.c_int, [C.c_void_p]),
    "zs_store_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "zs_store_fault": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "zs_store_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int64)]),
    "zs_store_set_xi": (C.c_int, [C.c_void_p, C.c_double]),
    "zs_store_block_stats": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                       C.POINTER(C.c_double)]),
    "zs_similar_ranges": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                                    C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_int32),
                                    C.c_void_p]),
    "zs_store_export_block": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_void_p]),
    "zs_compress_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_int64, C.c_int64,
                                      C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "zs_noalloc_status": (C.c_int, [C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "zs_query": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.POINTER(Result), C.c_void_p]),
    "zs_store_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "zs_query_batch_factored": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_int32,
                                          C.c_int32, C.POINTER(Result), C.c_void_p, C.c_int64, C.c_void_p]),
    "zs_query_batch": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_int32, C.c_int32,
                                 C.POINTER(Result), C.c_void_p]),
    "zs_serve_start": (C.c_int, [C.c_void_p, C.POINTER(ServeConfig), C.POINTER(C.c_void_p)]),
    "zs_serve_submit": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.POINTER(Result),
                                  C.POINTER(C.c_uint64)]),
    "zs_serve_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "zs_serve_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int64, C.POINTER(C.c_int32)]),
    "zs_serve_stop": (C.c_int, [C.c_void_p, C.POINTER(ServeStats)]),
    "zs_status_str": (C.c_char_p, [C.c_int]),
    "zs_last_error": (C.c_char_p, []),
    "zs_launch_count": (C.c_int64, []),
    "zs_profile_enable": (None, [C.c_int32]),
    "zs_profile_reset": (None, []),
    "zs_profile_count": (C.c_int32, []),
    "zs_profile_get": (C.c_int, [C.c_int32, C.POINTER(C.c_char_p), C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
}


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libzoomsvd.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _check(status: int):
    if status != 0:
        raise ZsError(status, lib().zs_last_error().decode())


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def factor_dtype(dtype: str) -> torch.dtype:
    return torch.float64 if dtype == "f64" else torch.float32


class QueryOut:
    """Device tensors of one range-SVD result."""

    def __init__(self, rows: int, n: int, k_out: int, dtype: torch.dtype, device):
        self.U = torch.empty((rows, k_out), dtype=dtype, device=device)
        self.S = torch.empty((k_out,), dtype=dtype, device=device)
        self.V = torch.empty((n, k_out), dtype=dtype, device=device)
        self.rank = torch.zeros((1,), dtype=torch.int32, device=device)

    def as_c(self) -> Result:
        return Result(self.U.data_ptr(), self.U.stride(0), self.S.data_ptr(), self.V.data_ptr(),
                      self.V.stride(0), self.rank.data_ptr())


class Store:
    """A compressed range-SVD store on one GPU (the sets U, S, V of Def. 2)."""

    def __init__(self, n: int, b: int, k: int, dtype: str = "f32", capacity_rows: int = 1 << 20,
                 device: int = 0, fp64_refine: bool = False, exact_gram: bool = False, xi: float | None = None,
                 row_append: bool = False):
        self.n, self.b, self.k, self.dtype = n, b, k, dtype
        self.device = torch.device("cuda", device)
        self.fdtype = factor_dtype(dtype)
        flags = (ZS_FLAG_FP64_REFINE if fp64_refine else 0) | (ZS_FLAG_EXACT_GRAM if exact_gram else 0) | \
            (ZS_FLAG_ROW_APPEND if row_append else 0)
        cfg = StoreConfig(n, b, k, DTYPES[dtype], capacity_rows, device, flags)
        h = C.c_void_p()
        _check(lib().zs_store_create(C.byref(cfg), C.byref(h)))
        self._h = h
        if xi is not None:
            self.set_xi(xi)

    def set_xi(self, xi: float):
        """Energy rule (Eq. 1) for blocks compressed from now on; 0 = fixed k."""
        _check(lib().zs_store_set_xi(self._h, float(xi)))

    def close(self):
        if getattr(self, "_h", None):
            lib().zs_store_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def append(self, rows, stream=None):
        """Append rows (torch CUDA tensor, or numpy/CPU tensor copied by the library).

        bf16 rows are given as int16/uint16 bit patterns or torch.bfloat16.
        """
        if isinstance(rows, np.ndarray):
            arr = np.ascontiguousarray(rows)
            ld = arr.strides[0] // arr.itemsize
            _check(lib().zs_store_append(self._h, arr.ctypes.data, arr.shape[0], ld, 0, _stream_ptr(stream)))
            return
        t = rows
        if t.dim() != 2 or t.stride(1) != 1:
            t = t.contiguous()
        on_dev = 1 if t.is_cuda else 0
        _check(lib().zs_store_append(self._h, t.data_ptr(), t.shape[0], t.stride(0), on_dev, _stream_ptr(stream)))

    def autotune(self, nq: int = 64, stream=None):
        _check(lib().zs_store_autotune(self._h, nq, _stream_ptr(stream)))

    def reset(self):
        _check(lib().zs_store_reset(self._h))

    def info(self):
        T, nb, by = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().zs_store_info(self._h, C.byref(T), C.byref(nb), C.byref(by)))
        return T.value, nb.value, by.value

    def fault(self) -> int:
        """The store's device fault word: 1 once a kernel gave up a bounded wait."""
        f = C.c_int32()
        _check(lib().zs_store_fault(self._h, C.byref(f)))
        return f.value

    def status(self, check: bool = True):
        """(unconverged blocks, unconverged query results) since creation;
        synchronises the device.  With check, a nonzero count raises ZsError
        (ZS_ENOCONV) and a set fault word ZS_ETIMEDOUT."""
        return self.status_counts(check)[:2]

    def status_counts(self, check: bool = True):
        """(unconverged blocks, unconverged queries, refined blocks, refined
        queries) since creation, as zs_store_status reports them."""
        v = [C.c_int64() for _ in range(4)]
        st = lib().zs_store_status(self._h, *[C.byref(x) for x in v])
        if check or st not in (0, 5, 10):
            _check(st)
        return tuple(x.value for x in v)

    def block_stats(self):
        """(ranks k_i, kept energies, block energies or -1) of every block,
        as numpy arrays (zs_store_block_stats)."""
        nb = self.info()[1]
        r = np.zeros(nb, dtype=np.int32)
        kept = np.zeros(nb)
        en = np.zeros(nb)
        _check(lib().zs_store_block_stats(self._h, nb, r.ctypes.data_as(C.POINTER(C.c_int32)),
                                          kept.ctypes.data_as(C.POINTER(C.c_double)),
                                          en.ctypes.data_as(C.POINTER(C.c_double))))
        return r, kept, en

    def export_block(self, i: int, stream=None):
        U = torch.empty((self.b, self.k), dtype=self.fdtype, device=self.device)
        s = torch.empty((self.k,), dtype=self.fdtype, device=self.device)
        Vt = torch.empty((self.k, self.n), dtype=self.fdtype, device=self.device)
        r, kk = C.c_int32(), C.c_int32()
        _check(lib().zs_store_export_block(self._h, i, U.data_ptr(), s.data_ptr(), Vt.data_ptr(),
                                           C.byref(r), C.byref(kk), _stream_ptr(stream)))
        return U[: r.value], s, Vt, kk.value

    def new_result(self, ts: int, te: int, k_out: int) -> QueryOut:
        return QueryOut(te - ts + 1, self.n, k_out, self.fdtype, self.device)

    def query(self, ts: int, te: int, k_out: int | None = None, out: QueryOut | None = None, stream=None):
        k_out = self.k if k_out is None else k_out
        out = out or self.new_result(ts, te, k_out)
        r = out.as_c()
        _check(lib().zs_query(self._h, ts, te, k_out, C.byref(r), _stream_ptr(stream)))
        return out

    def similar_ranges(self, base, stride: int, max_windows: int | None = None, stream=None):
        """Windows of the base range's length starting stride, 2 stride, ...
        rows before it, scored by the cosine of their first left singular
        vector with the base's (Section 6): [(start, cosine), ...]."""
        t_s, t_e = int(base[0]), int(base[1])
        cap = max(0, t_s // max(int(stride), 1)) if max_windows is None else int(max_windows)
        starts = np.zeros(max(cap, 1), dtype=np.int64)
        cos = np.zeros(max(cap, 1), dtype=np.float64)
        nw = C.c_int32()
        _check(lib().zs_similar_ranges(self._h, t_s, t_e, int(stride), cap,
                                       starts.ctypes.data_as(C.POINTER(C.c_int64)),
                                       cos.ctypes.data_as(C.POINTER(C.c_double)), C.byref(nw),
                                       _stream_ptr(stream)))
        return [(int(starts[j]), float(cos[j])) for j in range(nw.value)]

    def query_batch_factored(self, ts, te, k_out: int | None = None, out: "FactoredBatch | None" = None,
                             stream=None):
        """Batch with U left factored (zs_query_batch_factored)."""
        k_out = self.k if k_out is None else k_out
        ts = np.ascontiguousarray(ts, dtype=np.int64)
        te = np.ascontiguousarray(te, dtype=np.int64)
        out = out or FactoredBatch(self, ts, te, k_out)
        res = (Result * len(ts))(*out.results())
        _check(lib().zs_query_batch_factored(self._h, ts.ctypes.data_as(C.POINTER(C.c_int64)),
                                             te.ctypes.data_as(C.POINTER(C.c_int64)), len(ts), k_out, res,
                                             out.coef.data_ptr(), out.coef.shape[0], _stream_ptr(stream)))
        return out

    def query_batch(self, ts, te, k_out: int | None = None, outs=None, stream=None):
        k_out = self.k if k_out is None else k_out
        ts = np.ascontiguousarray(ts, dtype=np.int64)
        te = np.ascontiguousarray(te, dtype=np.int64)
        nq = ts.shape[0]
        if outs is None:
            outs = [self.new_result(int(a), int(z), k_out) for a, z in zip(ts, te)]
        res = (Result * nq)(*[o.as_c() for o in outs])
        _check(lib().zs_query_batch(self._h, ts.ctypes.data_as(C.POINTER(C.c_int64)),
                                    te.ctypes.data_as(C.POINTER(C.c_int64)), nq, k_out, res,
                                    _stream_ptr(stream)))
        return outs


class FactoredBatch:
    """Device tensors of a batch answered with U factored: S (nq x k_out),
    V (nq x n x k_out), rank (nq), and coef (sum of the queries' covered
    blocks x k rows, k_out columns); offsets[q] is query q's first
    coefficient row."""

    def __init__(self, store, ts, te, k_out):
        b, k = store.b, store.k
        nblk = te // b - ts // b + 1
        self.offsets = np.concatenate([[0], np.cumsum(nblk)])[:-1] * k
        self.rows = int(np.sum(nblk)) * k
        dev, dt = store.device, store.fdtype
        nq = len(ts)
        self.S = torch.empty((nq, k_out), dtype=dt, device=dev)
        self.V = torch.empty((nq, store.n, k_out), dtype=dt, device=dev)
        self.rank = torch.zeros((nq,), dtype=torch.int32, device=dev)
        self.coef = torch.empty((max(self.rows, 1), k_out), dtype=dt, device=dev)
        self.k_out = k_out

    def results(self):
        es = self.S.element_size()
        return [Result(0, self.k_out, self.S.data_ptr() + q * self.k_out * es,
                       self.V.data_ptr() + q * self.V.shape[1] * self.k_out * es, self.k_out,
                       self.rank.data_ptr() + 4 * q) for q in range(self.S.shape[0])]


class Server:
    """Continuous-batching query server over a Store."""

    def __init__(self, store: Store, max_batch=256, max_inflight=2, queue_capacity=1 << 16,
                 memory_budget=4 << 30):
        self.store = store
        cfg = ServeConfig(max_batch, max_inflight, queue_capacity, memory_budget)
        h = C.c_void_p()
        _check(lib().zs_serve_start(store.handle, C.byref(cfg), C.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, ts: int, te: int, k_out: int | None = None, out: QueryOut | None = None):
        k_out = self.store.k if k_out is None else k_out
        out = out or self.store.new_result(ts, te, k_out)
        r = out.as_c()
        t = C.c_uint64()
        st = lib().zs_serve_submit(self._h, ts, te, k_out, C.byref(r), C.byref(t))
        if st != 0:
            raise ZsError(st, lib().zs_last_error().decode())
        self._keep[t.value] = out
        return t.value, out

    def poll(self, ticket: int):
        d, s = C.c_int32(), C.c_int32()
        _check(lib().zs_serve_poll(self._h, ticket, C.byref(d), C.byref(s)))
        if d.value:
            self._keep.pop(ticket, None)
        return bool(d.value), s.value

    def wait(self, ticket: int, timeout_ms: int = 60_000):
        s = C.c_int32()
        _check(lib().zs_serve_wait(self._h, ticket, timeout_ms, C.byref(s)))
        self._keep.pop(ticket, None)
        return s.value

    def stop(self) -> dict:
        st = ServeStats()
        _check(lib().zs_serve_stop(self._h, C.byref(st)))
        self._h = None
        return {f: getattr(st, f) for f, _ in ServeStats._fields_}


def launch_count() -> int:
    return int(lib().zs_launch_count())


def profile(on: bool = True):
    lib().zs_profile_enable(1 if on else 0)


def profile_reset():
    lib().zs_profile_reset()


def profile_table() -> dict:
    """{kernel name: (launches, total device ms)} of the launches profiled so far."""
    out = {}
    for i in range(lib().zs_profile_count()):
        name, n, ms = C.c_char_p(), C.c_int64(), C.c_double()
        _check(lib().zs_profile_get(i, C.byref(name), C.byref(n), C.byref(ms)))
        out[name.value.decode()] = (n.value, ms.value)
    return out


def noalloc_status(check: bool = True):
    """(fault word, unconverged blocks) of the last zs_compress_noalloc call on
    the current device; synchronises the device.  With check, a set fault word
    raises ZS_ETIMEDOUT and unconverged blocks ZS_ENOCONV."""
    f, u = C.c_int32(), C.c_int32()
    st = lib().zs_noalloc_status(C.byref(f), C.byref(u))
    if check or st not in (0, 5, 10):
        _check(st)
    return f.value, u.value
