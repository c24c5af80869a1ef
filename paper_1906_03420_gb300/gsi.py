"""Thin ctypes binding of libgsi.so (include/gsi.h).

Argument marshalling only: every step of the matching path runs in the
library's CUDA kernels.  The library must be built (``_build.build()``); if it
is missing or cannot load, importing raises -- there is no fallback.
PyTorch is used for device buffers and streams (``torch.cuda`` tensors and
``torch.cuda.Stream.cuda_stream`` handles).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

GSI_OK, GSI_EINVAL, GSI_ENOMEM, GSI_ECAPPED, GSI_ETIMEOUT, GSI_ECANCELLED, GSI_ECUDA, GSI_EBUSY = range(8)
GSI_ISOMORPHISM, GSI_HOMOMORPHISM = 0, 1
GSI_EDGE_HOST_ONLY = 1
GSI_ISECT_BSEARCH, GSI_ISECT_MERGE, GSI_ISECT_BITMAP = 0, 1, 2
STATUS_NAMES = {0: "GSI_OK", 1: "GSI_EINVAL", 2: "GSI_ENOMEM", 3: "GSI_ECAPPED", 4: "GSI_ETIMEOUT",
                5: "GSI_ECANCELLED", 6: "GSI_ECUDA", 7: "GSI_EBUSY"}
MAX_QUERY_VERTICES = 32
SIG_WORDS = 16

EXPORTED = [
    "gsi_graph_create", "gsi_graph_destroy", "gsi_graph_get_info", "gsi_graph_export", "gsi_graph_label_freq",
    "gsi_query_run", "gsi_result_count", "gsi_result_columns", "gsi_result_copy", "gsi_result_copy_async", "gsi_result_destroy", "gsi_server_estimate",
    "gsi_filter", "gsi_query_signatures", "gsi_join_step", "gsi_join_step_noalloc", "gsi_plan_order",
    "gsi_batch_run", "gsi_batch_autotune", "gsi_batch_autotune_full", "gsi_batch_prepare", "gsi_batch_replay", "gsi_batch_destroy", "gsi_server_create", "gsi_server_submit", "gsi_server_poll", "gsi_server_cancel",
    "gsi_server_destroy", "gsi_last_error", "gsi_version", "gsi_selftest_wait_timeout",
    "gsi_edge_graph_create", "gsi_edge_graph_destroy", "gsi_edge_graph_line", "gsi_edge_graph_device",
    "gsi_edge_query_line", "gsi_edge_query_run",
]


class GsiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class c_graph_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class c_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_elabels", ctypes.c_int32), ("n_vlabels", ctypes.c_int32),
                ("m", ctypes.c_int64), ("device_bytes", ctypes.c_uint64), ("build_ms", ctypes.c_double),
                ("off", ctypes.c_void_p), ("ci", ctypes.c_void_p), ("cl", ctypes.c_void_p), ("sig", ctypes.c_void_p)]


class c_stats(ctypes.Structure):
    _fields_ = [("filter_ms", ctypes.c_double), ("join_ms", ctypes.c_double), ("other_ms", ctypes.c_double),
                ("filter_launches", ctypes.c_uint64), ("join_launches", ctypes.c_uint64),
                ("other_launches", ctypes.c_uint64), ("filter_bytes", ctypes.c_uint64),
                ("join_bytes", ctypes.c_uint64), ("join_items", ctypes.c_uint64), ("tiles", ctypes.c_uint64),
                ("peak_bytes", ctypes.c_uint64), ("kernels", ctypes.c_uint64), ("host_driven", ctypes.c_uint64),
                ("cand", ctypes.c_uint64 * 32), ("order", ctypes.c_int32 * 32),
                ("k", ctypes.c_int32), ("join_bytes_listwise", ctypes.c_uint64),
                ("batch_ms", ctypes.c_double), ("batch_bytes", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("cand", "order")}
        d["cand"] = list(self.cand)[: self.k]
        d["order"] = list(self.order)[: self.k]
        return d


class c_query_opts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("row_cap", ctypes.c_uint64), ("mem_budget", ctypes.c_uint64),
                ("count_only", ctypes.c_int32), ("semantics", ctypes.c_int32),
                ("order", ctypes.POINTER(ctypes.c_int32)), ("stats", ctypes.POINTER(c_stats)),
                ("host_driven", ctypes.c_int32), ("listwise_bytes", ctypes.c_int32), ("no_dedup", ctypes.c_int32),
                ("tight_rows", ctypes.c_int32)]


class c_query_desc(ctypes.Structure):
    _fields_ = [("vlab", ctypes.POINTER(ctypes.c_int32)), ("k", ctypes.c_int32),
                ("src", ctypes.POINTER(ctypes.c_int32)), ("dst", ctypes.POINTER(ctypes.c_int32)),
                ("elab", ctypes.POINTER(ctypes.c_int32)), ("qm", ctypes.c_int32)]


class c_batch_opts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("row_cap", ctypes.c_uint64), ("mem_budget", ctypes.c_uint64),
                ("count_only", ctypes.c_int32), ("stats", ctypes.POINTER(c_stats)),
                ("seeds_per_item", ctypes.c_int32), ("item_rows", ctypes.c_int32), ("isect", ctypes.c_int32),
                ("rows_per_thread", ctypes.c_int32), ("block_threads", ctypes.c_int32)]


class c_server_opts(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_uint64), ("n_streams", ctypes.c_int32), ("row_cap", ctypes.c_uint64),
                ("count_only", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("seeds_per_item", ctypes.c_int32),
                ("item_rows", ctypes.c_int32), ("min_batch", ctypes.c_int32), ("isect", ctypes.c_int32),
                ("rows_per_thread", ctypes.c_int32), ("block_threads", ctypes.c_int32)]


_lib = None
I32P = ctypes.POINTER(ctypes.c_int32)
U32P = ctypes.POINTER(ctypes.c_uint32)
U64P = ctypes.POINTER(ctypes.c_uint64)
VP = ctypes.c_void_p


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libgsi.so; raises if it is absent (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise ImportError(f"libgsi.so not built at {path}; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    st = ctypes.c_int
    L.gsi_graph_create.argtypes = [I32P, ctypes.c_int32, I32P, I32P, I32P, ctypes.c_int64,
                                   ctypes.POINTER(c_graph_opts), ctypes.POINTER(VP)]
    L.gsi_graph_create.restype = st
    L.gsi_graph_destroy.argtypes = [VP]
    L.gsi_graph_destroy.restype = None
    L.gsi_graph_get_info.argtypes = [VP, ctypes.POINTER(c_graph_info)]
    L.gsi_graph_get_info.restype = st
    L.gsi_graph_export.argtypes = [VP, VP, VP, VP, VP]
    L.gsi_graph_export.restype = st
    L.gsi_graph_label_freq.argtypes = [VP, U64P, ctypes.c_int32]
    L.gsi_graph_label_freq.restype = st
    L.gsi_query_run.argtypes = [VP, I32P, ctypes.c_int32, I32P, I32P, I32P, ctypes.c_int32,
                                ctypes.POINTER(c_query_opts), ctypes.POINTER(VP)]
    L.gsi_query_run.restype = st
    L.gsi_result_count.argtypes = [VP, U64P]
    L.gsi_result_count.restype = st
    L.gsi_result_columns.argtypes = [VP, I32P]
    L.gsi_result_columns.restype = st
    L.gsi_result_copy.argtypes = [VP, VP, ctypes.c_uint64, U64P]
    L.gsi_result_copy.restype = st
    L.gsi_result_copy_async.argtypes = [VP, VP, ctypes.c_uint64, U64P, VP]
    L.gsi_result_copy_async.restype = st
    L.gsi_result_destroy.argtypes = [VP]
    L.gsi_result_destroy.restype = None
    L.gsi_filter.argtypes = [VP, I32P, ctypes.c_int32, I32P, I32P, I32P, ctypes.c_int32, VP, VP, VP]
    L.gsi_filter.restype = st
    L.gsi_query_signatures.argtypes = [I32P, ctypes.c_int32, I32P, I32P, I32P, ctypes.c_int32, U32P]
    L.gsi_query_signatures.restype = st
    L.gsi_join_step.argtypes = [VP, VP, ctypes.c_uint64, ctypes.c_int32, VP, ctypes.c_int32, I32P, I32P,
                                ctypes.c_int32, VP, ctypes.c_uint64, U64P, VP]
    L.gsi_join_step.restype = st
    L.gsi_join_step_noalloc.argtypes = L.gsi_join_step.argtypes
    L.gsi_join_step_noalloc.restype = st
    L.gsi_plan_order.argtypes = [ctypes.c_int32, I32P, I32P, I32P, ctypes.c_int32, U64P, U64P, ctypes.c_int32,
                                 I32P, I32P]
    L.gsi_plan_order.restype = st
    L.gsi_batch_run.argtypes = [VP, ctypes.POINTER(c_query_desc), ctypes.c_int32, ctypes.POINTER(c_batch_opts),
                                ctypes.POINTER(VP), I32P]
    L.gsi_batch_run.restype = st
    L.gsi_batch_autotune.argtypes = [VP, ctypes.POINTER(c_query_desc), ctypes.c_int32, ctypes.POINTER(c_batch_opts),
                                     I32P, I32P, ctypes.POINTER(ctypes.c_double)]
    L.gsi_batch_autotune_full.argtypes = [VP, ctypes.POINTER(c_query_desc), ctypes.c_int32,
                                          ctypes.POINTER(c_batch_opts), ctypes.POINTER(c_batch_opts),
                                          ctypes.POINTER(ctypes.c_double), I32P]
    L.gsi_batch_autotune_full.restype = st
    L.gsi_batch_autotune.restype = st
    L.gsi_batch_prepare.argtypes = [VP, ctypes.POINTER(c_query_desc), ctypes.c_int32, ctypes.POINTER(c_batch_opts),
                                    ctypes.POINTER(VP), I32P]
    L.gsi_batch_prepare.restype = st
    L.gsi_batch_replay.argtypes = [VP, ctypes.POINTER(VP), I32P, ctypes.POINTER(c_stats)]
    L.gsi_batch_replay.restype = st
    L.gsi_batch_destroy.argtypes = [VP]
    L.gsi_batch_destroy.restype = None
    L.gsi_server_create.argtypes = [VP, ctypes.POINTER(c_server_opts), ctypes.POINTER(VP)]
    L.gsi_server_create.restype = st
    L.gsi_server_submit.argtypes = [VP, ctypes.POINTER(c_query_desc), U64P]
    L.gsi_server_submit.restype = st
    L.gsi_server_poll.argtypes = [VP, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(VP),
                                  ctypes.POINTER(ctypes.c_double)]
    L.gsi_server_poll.restype = st
    L.gsi_server_cancel.argtypes = [VP, ctypes.c_uint64]
    L.gsi_server_cancel.restype = st
    L.gsi_server_estimate.argtypes = [VP, ctypes.POINTER(c_query_desc), U64P]
    L.gsi_server_estimate.restype = st
    L.gsi_server_destroy.argtypes = [VP]
    L.gsi_server_destroy.restype = None
    L.gsi_edge_graph_create.argtypes = [I32P, ctypes.c_int32, I32P, I32P, I32P, ctypes.c_int64,
                                        ctypes.POINTER(c_graph_opts), ctypes.c_int32, ctypes.POINTER(VP)]
    L.gsi_edge_graph_create.restype = st
    L.gsi_edge_graph_destroy.argtypes = [VP]
    L.gsi_edge_graph_destroy.restype = None
    L.gsi_edge_graph_line.argtypes = [VP, I32P, I32P, I32P, I32P, ctypes.c_int64, I32P,
                                      ctypes.POINTER(ctypes.c_int64)]
    L.gsi_edge_graph_line.restype = st
    L.gsi_edge_graph_device.argtypes = [VP, ctypes.POINTER(VP)]
    L.gsi_edge_graph_device.restype = st
    L.gsi_edge_query_line.argtypes = [VP, I32P, ctypes.c_int32, I32P, I32P, I32P, ctypes.c_int32, I32P, I32P, I32P,
                                      I32P, ctypes.c_int32, I32P, I32P]
    L.gsi_edge_query_line.restype = st
    L.gsi_edge_query_run.argtypes = [VP, I32P, ctypes.c_int32, I32P, I32P, I32P, ctypes.c_int32,
                                     ctypes.POINTER(c_query_opts), ctypes.POINTER(VP)]
    L.gsi_edge_query_run.restype = st
    L.gsi_last_error.argtypes = []
    L.gsi_last_error.restype = ctypes.c_char_p
    L.gsi_selftest_wait_timeout.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
    L.gsi_selftest_wait_timeout.restype = st
    L.gsi_version.argtypes = []
    L.gsi_version.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc: int, what: str, ok=(GSI_OK,)):
    if rc not in ok:
        msg = (_lib.gsi_last_error() or b"").decode()
        raise GsiError(rc, f"{what}: {msg}")
    return rc


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


def _p32(a: np.ndarray):
    return a.ctypes.data_as(I32P)


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


@dataclass
class QueryArrays:
    vlab: np.ndarray
    src: np.ndarray
    dst: np.ndarray
    elab: np.ndarray

    @classmethod
    def of(cls, q) -> "QueryArrays":
        return cls(_i32(q.vlab), _i32(q.src), _i32(q.dst), _i32(q.elab))

    @property
    def k(self):
        return int(self.vlab.shape[0])

    @property
    def qm(self):
        return int(self.src.shape[0])

    def desc(self) -> c_query_desc:
        return c_query_desc(_p32(self.vlab), self.k, _p32(self.src), _p32(self.dst), _p32(self.elab), self.qm)


class Result:
    """Owner of a gsi_result handle."""

    def __init__(self, handle: int):
        self._h = handle

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "_h", None):
            load().gsi_result_destroy(self._h)
            self._h = None

    @property
    def count(self) -> int:
        c = ctypes.c_uint64()
        _check(load().gsi_result_count(self._h, ctypes.byref(c)), "gsi_result_count")
        return int(c.value)

    @property
    def k(self) -> int:
        k = ctypes.c_int32()
        _check(load().gsi_result_columns(self._h, ctypes.byref(k)), "gsi_result_columns")
        return int(k.value)

    def copy_to(self, ptr: int, max_rows: int) -> tuple[int, bool]:
        """Copy into host or device memory at ptr; returns (rows, capped)."""
        rows = ctypes.c_uint64()
        rc = _check(load().gsi_result_copy(self._h, ptr, max_rows, ctypes.byref(rows)), "gsi_result_copy",
                    ok=(GSI_OK, GSI_ECAPPED))
        return int(rows.value), rc == GSI_ECAPPED

    def copy_to_async(self, ptr: int, max_rows: int, stream=None) -> tuple[int, bool]:
        """Enqueue the copy on `stream` (torch stream or handle); returns (rows,
        capped) at once.  Keep the result alive until the copy has completed."""
        rows = ctypes.c_uint64()
        rc = _check(load().gsi_result_copy_async(self._h, ptr, max_rows, ctypes.byref(rows), _stream_handle(stream)),
                    "gsi_result_copy_async", ok=(GSI_OK, GSI_ECAPPED))
        return int(rows.value), rc == GSI_ECAPPED

    def rows(self, max_rows: int | None = None) -> np.ndarray:
        """Materialised rows as a host int32 array [rows, k] (unordered)."""
        n = self.count if max_rows is None else max_rows
        out = np.empty((max(n, 1), self.k), np.int32)
        got, _ = self.copy_to(out.ctypes.data, n)
        return out[:got]


class Graph:
    """A labelled data graph resident on one GPU (gsi_graph_create)."""

    def __init__(self, vlab, src, dst, elab, device: int = 0, stream=None):
        L = load()
        self._keep = [_i32(vlab), _i32(src), _i32(dst), _i32(elab)]
        vl, s, d, e = self._keep
        h = VP()
        opts = c_graph_opts(device, _stream_handle(stream))
        _check(L.gsi_graph_create(_p32(vl), vl.shape[0], _p32(s), _p32(d), _p32(e), s.shape[0],
                                  ctypes.byref(opts), ctypes.byref(h)), "gsi_graph_create")
        self._h = h.value
        self._keep = None
        self.device = device

    @classmethod
    def from_synth(cls, g, device: int = 0, stream=None) -> "Graph":
        return cls(g.vlab, g.src, g.dst, g.elab, device, stream)

    @classmethod
    def _borrowed(cls, handle: int, device: int, owner) -> "Graph":
        """A view of a graph that `owner` holds (not destroyed by close())."""
        g = cls.__new__(cls)
        g._h = handle
        g._keep = None
        g.device = device
        g._owner = owner
        return g

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owner", None) is None:
                load().gsi_graph_destroy(self._h)
            self._h = None

    @property
    def handle(self) -> int:
        return self._h

    def info(self) -> c_graph_info:
        i = c_graph_info()
        _check(load().gsi_graph_get_info(self._h, ctypes.byref(i)), "gsi_graph_get_info")
        return i

    def export(self) -> tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
        """(off uint32[n*L+1], ci int32[2m], cl uint16[2m], sig uint32[16, n]) copied to the host."""
        i = self.info()
        off = np.zeros(i.n * i.n_elabels + 1, np.uint32)
        ci = np.zeros(max(2 * i.m, 1), np.int32)
        cl = np.zeros(max(2 * i.m, 1), np.uint16)
        sig = np.zeros((SIG_WORDS, i.n), np.uint32)
        _check(load().gsi_graph_export(self._h, off.ctypes.data, ci.ctypes.data, cl.ctypes.data, sig.ctypes.data),
               "gsi_graph_export")
        return off, ci[: 2 * i.m], cl[: 2 * i.m], sig

    def label_freq(self) -> np.ndarray:
        L = self.info().n_elabels
        out = np.zeros(L, np.uint64)
        _check(load().gsi_graph_label_freq(self._h, out.ctypes.data_as(U64P), L), "gsi_graph_label_freq")
        return out

    def query(self, q, stream=None, row_cap: int = 0, mem_budget: int = 0, count_only: bool = False,
              order=None, stats: c_stats | None = None, host_driven: bool = False, semantics: int = 0,
              listwise_bytes: bool = False, no_dedup: bool = False, tight_rows: bool = False) -> Result:
        qa = q if isinstance(q, QueryArrays) else QueryArrays.of(q)
        o = c_query_opts()
        o.stream = _stream_handle(stream)
        o.row_cap = row_cap
        o.mem_budget = mem_budget
        o.count_only = int(count_only)
        o.semantics = int(semantics)
        o.host_driven = int(host_driven)
        o.listwise_bytes = int(listwise_bytes)
        o.no_dedup = int(no_dedup)
        o.tight_rows = int(tight_rows)
        ordr = None
        if order is not None:
            ordr = _i32(order)
            o.order = _p32(ordr)
        if stats is not None:
            o.stats = ctypes.pointer(stats)
        h = VP()
        _check(load().gsi_query_run(self._h, _p32(qa.vlab), qa.k, _p32(qa.src), _p32(qa.dst), _p32(qa.elab), qa.qm,
                                    ctypes.byref(o), ctypes.byref(h)), "gsi_query_run")
        return Result(h.value)

    def filter(self, q, stream=None) -> tuple[np.ndarray, np.ndarray]:
        """(bitmaps uint32[k, ceil(n/32)], counts uint64[k]) on the host."""
        qa = q if isinstance(q, QueryArrays) else QueryArrays.of(q)
        n = self.info().n
        words = (n + 31) // 32
        bm = np.zeros((qa.k, words), np.uint32)
        cnt = np.zeros(qa.k, np.uint64)
        _check(load().gsi_filter(self._h, _p32(qa.vlab), qa.k, _p32(qa.src), _p32(qa.dst), _p32(qa.elab), qa.qm,
                                 bm.ctypes.data, cnt.ctypes.data, _stream_handle(stream)), "gsi_filter")
        return bm, cnt

    def join_step(self, M_ptr: int, R: int, t: int, cand_ptr: int, ulabel: int, cols, labs, out_ptr: int,
                  out_cap: int, stream=None) -> int:
        """One join iteration on device buffers (pointers); returns the survivor count."""
        c = _i32(cols)
        l = _i32(labs)
        cnt = ctypes.c_uint64()
        _check(load().gsi_join_step(self._h, M_ptr, R, t, cand_ptr, ulabel, _p32(c), _p32(l), c.shape[0], out_ptr,
                                    out_cap, ctypes.byref(cnt), _stream_handle(stream)), "gsi_join_step")
        return int(cnt.value)

    def join_step_noalloc(self, M_ptr: int, R: int, t: int, cand_ptr: int, ulabel: int, cols, labs, out_ptr: int,
                          out_cap: int, stream=None) -> int:
        """join_step with the library's static scratch array: no device allocation
        (for callers that may not allocate); returns the survivor count."""
        c = _i32(cols)
        l = _i32(labs)
        cnt = ctypes.c_uint64()
        _check(load().gsi_join_step_noalloc(self._h, M_ptr, R, t, cand_ptr, ulabel, _p32(c), _p32(l), c.shape[0],
                                            out_ptr, out_cap, ctypes.byref(cnt), _stream_handle(stream)),
               "gsi_join_step_noalloc")
        return int(cnt.value)

    def batch(self, queries, stream=None, row_cap: int = 0, mem_budget: int = 0, count_only: bool = False,
              stats: c_stats | None = None, seeds_per_item: int = 0, item_rows: int = 0, isect: int = 0,
              rows_per_thread: int = 0, block_threads: int = 0) -> list:
        qas = [q if isinstance(q, QueryArrays) else QueryArrays.of(q) for q in queries]
        descs = (c_query_desc * len(qas))(*[qa.desc() for qa in qas])
        outs = (VP * len(qas))()
        sts = (ctypes.c_int32 * len(qas))()
        o = c_batch_opts(_stream_handle(stream), row_cap, mem_budget, int(count_only),
                         ctypes.pointer(stats) if stats is not None else None, seeds_per_item, item_rows, isect,
                         rows_per_thread, block_threads)
        _check(load().gsi_batch_run(self._h, descs, len(qas), ctypes.byref(o), outs, sts), "gsi_batch_run")
        res = []
        for i in range(len(qas)):
            res.append(Result(outs[i]) if sts[i] == GSI_OK else GsiError(sts[i], "batched query failed"))
        return res


class EdgeGraph:
    """Edge isomorphism (Sec. VII-A) by the line-graph transform
    (gsi_edge_graph_*): G's line graph G' on the device; queries are
    transformed to Q' and matched in G'.  Result rows hold data edge ids
    (positions in this graph's edge list), column j for query edge j."""

    def __init__(self, vlab, src, dst, elab, device: int = 0, stream=None, host_only: bool = False):
        L = load()
        vl, s, d, e = _i32(vlab), _i32(src), _i32(dst), _i32(elab)
        h = VP()
        opts = c_graph_opts(device, _stream_handle(stream))
        _check(L.gsi_edge_graph_create(_p32(vl), vl.shape[0], _p32(s), _p32(d), _p32(e), s.shape[0],
                                       ctypes.byref(opts), GSI_EDGE_HOST_ONLY if host_only else 0, ctypes.byref(h)),
               "gsi_edge_graph_create")
        self._h = h.value
        self.device = device
        self.m = int(s.shape[0])

    @classmethod
    def from_synth(cls, g, device: int = 0, stream=None, host_only: bool = False) -> "EdgeGraph":
        return cls(g.vlab, g.src, g.dst, g.elab, device, stream, host_only)

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "_h", None):
            load().gsi_edge_graph_destroy(self._h)
            self._h = None

    def line_graph(self) -> tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
        """G' on the host: (vlab int32[m], src, dst, elab int32[|E(G')|])."""
        L = load()
        ln = ctypes.c_int32()
        lm = ctypes.c_int64()
        _check(L.gsi_edge_graph_line(self._h, None, None, None, None, 0, ctypes.byref(ln), ctypes.byref(lm)),
               "gsi_edge_graph_line")
        vl = np.zeros(max(ln.value, 1), np.int32)
        s, d, e = (np.zeros(max(lm.value, 1), np.int32) for _ in range(3))
        _check(L.gsi_edge_graph_line(self._h, _p32(vl), _p32(s), _p32(d), _p32(e), lm.value, None, None),
               "gsi_edge_graph_line")
        return vl[: ln.value], s[: lm.value], d[: lm.value], e[: lm.value]

    def line_query(self, q) -> QueryArrays:
        """Q' against this graph's label tables (host only)."""
        qa = q if isinstance(q, QueryArrays) else QueryArrays.of(q)
        L = load()
        cap = 32 * 31 // 2
        vl = np.zeros(max(qa.qm, 1), np.int32)
        s, d, e = (np.zeros(cap, np.int32) for _ in range(3))
        lk = ctypes.c_int32()
        lqm = ctypes.c_int32()
        _check(L.gsi_edge_query_line(self._h, _p32(qa.vlab), qa.k, _p32(qa.src), _p32(qa.dst), _p32(qa.elab), qa.qm,
                                     _p32(vl), _p32(s), _p32(d), _p32(e), cap, ctypes.byref(lk), ctypes.byref(lqm)),
               "gsi_edge_query_line")
        return QueryArrays(vl[: lk.value].copy(), s[: lqm.value].copy(), d[: lqm.value].copy(),
                           e[: lqm.value].copy())

    def line(self) -> Graph:
        """G' as a Graph view (owned by this object) for batches and servers of line queries."""
        g = VP()
        _check(load().gsi_edge_graph_device(self._h, ctypes.byref(g)), "gsi_edge_graph_device")
        if not g.value:
            raise GsiError(GSI_EINVAL, "host-only edge graph has no device line graph")
        return Graph._borrowed(g.value, self.device, self)

    def query(self, q, stream=None, row_cap: int = 0, mem_budget: int = 0, count_only: bool = False,
              order=None, stats: c_stats | None = None, host_driven: bool = False,
              listwise_bytes: bool = False, no_dedup: bool = False, tight_rows: bool = False) -> Result:
        qa = q if isinstance(q, QueryArrays) else QueryArrays.of(q)
        o = c_query_opts()
        o.stream = _stream_handle(stream)
        o.row_cap = row_cap
        o.mem_budget = mem_budget
        o.count_only = int(count_only)
        o.host_driven = int(host_driven)
        o.listwise_bytes = int(listwise_bytes)
        o.no_dedup = int(no_dedup)
        o.tight_rows = int(tight_rows)
        ordr = None
        if order is not None:
            ordr = _i32(order)
            o.order = _p32(ordr)
        if stats is not None:
            o.stats = ctypes.pointer(stats)
        h = VP()
        _check(load().gsi_edge_query_run(self._h, _p32(qa.vlab), qa.k, _p32(qa.src), _p32(qa.dst), _p32(qa.elab),
                                         qa.qm, ctypes.byref(o), ctypes.byref(h)), "gsi_edge_query_run")
        return Result(h.value)

    def batch(self, queries, **kw) -> list:
        """Edge queries as one batch on the line graph (Graph.batch on the Q')."""
        return self.line().batch([self.line_query(q) for q in queries], **kw)


class PreparedBatch:
    """A batch planned once and replayed from a captured CUDA graph (gsi_batch_prepare / gsi_batch_replay)."""

    def __init__(self, graph: "Graph", queries, stream=None, row_cap: int = 0, mem_budget: int = 0,
                 count_only: bool = False, seeds_per_item: int = 0, item_rows: int = 0, counters: bool = False,
                 isect: int = 0, rows_per_thread: int = 0, block_threads: int = 0):
        self._graph = graph
        self._qas = [q if isinstance(q, QueryArrays) else QueryArrays.of(q) for q in queries]
        self._descs = (c_query_desc * len(self._qas))(*[qa.desc() for qa in self._qas])
        self.statuses = (ctypes.c_int32 * len(self._qas))()
        self._probe = c_stats() if counters else None
        o = c_batch_opts(_stream_handle(stream), row_cap, mem_budget, int(count_only),
                         ctypes.pointer(self._probe) if counters else None, seeds_per_item, item_rows, isect,
                         rows_per_thread, block_threads)
        h = VP()
        _check(load().gsi_batch_prepare(graph.handle, self._descs, len(self._qas), ctypes.byref(o), ctypes.byref(h),
                                        self.statuses), "gsi_batch_prepare")
        self._h = h.value

    def __len__(self):
        return len(self._qas)

    def run(self, stats: c_stats | None = None) -> list:
        n = len(self._qas)
        outs = (VP * n)()
        sts = (ctypes.c_int32 * n)()
        _check(load().gsi_batch_replay(self._h, outs, sts, ctypes.pointer(stats) if stats is not None else None),
               "gsi_batch_replay")
        return [Result(outs[i]) if sts[i] == GSI_OK else GsiError(sts[i], "batched query failed") for i in range(n)]

    def close(self):
        if getattr(self, "_h", None):
            load().gsi_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def batch_autotune(graph: "Graph", queries, stream=None, mem_budget: int = 0) -> tuple[int, int, float]:
    """Pick the batch work-unit sizes on a calibration batch: (seeds_per_item, item_rows, ms)."""
    qas = [q if isinstance(q, QueryArrays) else QueryArrays.of(q) for q in queries]
    descs = (c_query_desc * len(qas))(*[qa.desc() for qa in qas])
    o = c_batch_opts(_stream_handle(stream), 0, mem_budget, 0, None, 0, 0, 0, 0, 0)
    spi = ctypes.c_int32()
    rows = ctypes.c_int32()
    ms = ctypes.c_double()
    _check(load().gsi_batch_autotune(graph.handle, descs, len(qas), ctypes.byref(o), ctypes.byref(spi),
                                     ctypes.byref(rows), ctypes.byref(ms)), "gsi_batch_autotune")
    return int(spi.value), int(rows.value), float(ms.value)


def batch_autotune_full(graph: "Graph", queries, stream=None, mem_budget: int = 0) -> dict:
    """Every batch knob tuned on a calibration batch (gsi_batch_autotune_full):
    seeds_per_item, item_rows, isect, rows_per_thread, block_threads, ms, trials."""
    qas = [q if isinstance(q, QueryArrays) else QueryArrays.of(q) for q in queries]
    descs = (c_query_desc * len(qas))(*[qa.desc() for qa in qas])
    o = c_batch_opts(_stream_handle(stream), 0, mem_budget, 0, None, 0, 0, 0, 0, 0)
    best = c_batch_opts()
    ms = ctypes.c_double()
    trials = ctypes.c_int32()
    _check(load().gsi_batch_autotune_full(graph.handle, descs, len(qas), ctypes.byref(o), ctypes.byref(best),
                                          ctypes.byref(ms), ctypes.byref(trials)), "gsi_batch_autotune_full")
    return {"seeds_per_item": best.seeds_per_item, "item_rows": best.item_rows, "isect": best.isect,
            "rows_per_thread": best.rows_per_thread, "block_threads": best.block_threads,
            "ms": float(ms.value), "trials": int(trials.value)}


def query_signatures(q) -> np.ndarray:
    qa = q if isinstance(q, QueryArrays) else QueryArrays.of(q)
    out = np.zeros((qa.k, SIG_WORDS), np.uint32)
    _check(load().gsi_query_signatures(_p32(qa.vlab), qa.k, _p32(qa.src), _p32(qa.dst), _p32(qa.elab), qa.qm,
                                       out.ctypes.data_as(U32P)), "gsi_query_signatures")
    return out


def plan_order(q, cand, freq) -> tuple[np.ndarray, np.ndarray]:
    qa = q if isinstance(q, QueryArrays) else QueryArrays.of(q)
    cand = np.ascontiguousarray(cand, np.uint64)
    freq = np.ascontiguousarray(freq, np.uint64)
    order = np.zeros(qa.k, np.int32)
    first = np.zeros(qa.k, np.int32)
    _check(load().gsi_plan_order(qa.k, _p32(qa.src), _p32(qa.dst), _p32(qa.elab), qa.qm, cand.ctypes.data_as(U64P),
                                 freq.ctypes.data_as(U64P), freq.shape[0], _p32(order), _p32(first)),
           "gsi_plan_order")
    return order, first


class Server:
    """Continuous-batching server over a resident graph (gsi_server_*)."""

    def __init__(self, graph: Graph, mem_budget: int = 0, n_streams: int = 2, row_cap: int = 0,
                 count_only: bool = False, max_batch: int = 0, seeds_per_item: int = 0, item_rows: int = 0,
                 min_batch: int = 0, isect: int = 0, rows_per_thread: int = 0, block_threads: int = 0):
        self._graph = graph
        h = VP()
        o = c_server_opts(mem_budget, n_streams, row_cap, int(count_only), max_batch, seeds_per_item, item_rows,
                          min_batch, isect, rows_per_thread, block_threads)
        _check(load().gsi_server_create(graph.handle, ctypes.byref(o), ctypes.byref(h)), "gsi_server_create")
        self._h = h.value

    def submit(self, q) -> int:
        qa = q if isinstance(q, QueryArrays) else QueryArrays.of(q)
        t = ctypes.c_uint64()
        d = qa.desc()
        _check(load().gsi_server_submit(self._h, ctypes.byref(d), ctypes.byref(t)), "gsi_server_submit")
        return int(t.value)

    def poll(self, ticket: int, timeout_ms: int = -1):
        """(Result, latency_ms), or None if not finished within timeout_ms."""
        h = VP()
        lat = ctypes.c_double()
        rc = load().gsi_server_poll(self._h, ticket, timeout_ms, ctypes.byref(h), ctypes.byref(lat))
        if rc == GSI_EBUSY:
            return None
        _check(rc, "gsi_server_poll")
        return Result(h.value), float(lat.value)

    def cancel(self, ticket: int):
        _check(load().gsi_server_cancel(self._h, ticket), "gsi_server_cancel")

    def estimate(self, q) -> int:
        """Admission estimate of a query's intermediate-table bytes."""
        qa = q if isinstance(q, QueryArrays) else QueryArrays.of(q)
        b = ctypes.c_uint64()
        d = qa.desc()
        _check(load().gsi_server_estimate(self._h, ctypes.byref(d), ctypes.byref(b)), "gsi_server_estimate")
        return int(b.value)

    def close(self):
        if getattr(self, "_h", None):
            load().gsi_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def selftest_wait_timeout(device: int = 0, spin_limit: int = 4096) -> tuple[int, float]:
    """Run the bounded-wait self-test; returns (status, elapsed ms); GSI_ETIMEOUT is the expected status."""
    ms = ctypes.c_double()
    rc = load().gsi_selftest_wait_timeout(device, spin_limit, ctypes.byref(ms))
    return int(rc), float(ms.value)


def version() -> str:
    return load().gsi_version().decode()


def last_error() -> str:
    return (load().gsi_last_error() or b"").decode()
