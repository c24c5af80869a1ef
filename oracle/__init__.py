"""ORACLE -- test infrastructure only.

Plain, slow CPU statement of the subgraph-isomorphism path (``oracle.c``):
enumeration by definition (Defs. 1-3), brute force, homomorphism and edge
isomorphism (Sec. VII-A), the Sec. III-A signature filter and the result of
one Alg. 3 join iteration.  Only ``tests/``,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline / reference legs
may import this package; the CUDA library never does, and the two share no
code.  Built with gcc into ``liboracle.so`` by :func:`build`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

SIG_WORDS = 16


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, src, "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i64p = ctypes.POINTER(ctypes.c_int64)
        vp = ctypes.c_void_p
        lib.oracle_graph_new.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, i32p]
        lib.oracle_graph_new.restype = vp
        lib.oracle_graph_free.argtypes = [vp]
        lib.oracle_edge_label.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
        lib.oracle_edge_label.restype = ctypes.c_int32
        q = [ctypes.c_int32, i32p, i32p, i32p, i32p, ctypes.c_int32]
        lib.oracle_enumerate.argtypes = [vp] + q + [i32p, ctypes.c_int64, ctypes.c_int32, u64p]
        lib.oracle_enumerate.restype = ctypes.c_int64
        lib.oracle_order.argtypes = q + [i32p]
        lib.oracle_order.restype = ctypes.c_int32
        lib.oracle_bruteforce.argtypes = [vp] + q + [i32p, ctypes.c_int64]
        lib.oracle_bruteforce.restype = ctypes.c_int64
        lib.oracle_enumerate_hom.argtypes = [vp] + q + [i32p, ctypes.c_int64, ctypes.c_int32, u64p]
        lib.oracle_enumerate_hom.restype = ctypes.c_int64
        lib.oracle_bruteforce_hom.argtypes = [vp] + q + [i32p, ctypes.c_int64]
        lib.oracle_bruteforce_hom.restype = ctypes.c_int64
        lib.oracle_enumerate_edge.argtypes = [vp] + q + [i32p, ctypes.c_int64, ctypes.c_int32, u64p]
        lib.oracle_enumerate_edge.restype = ctypes.c_int64
        lib.oracle_bruteforce_edge.argtypes = [vp] + q + [i32p, ctypes.c_int64]
        lib.oracle_bruteforce_edge.restype = ctypes.c_int64
        lib.oracle_murmur3_32.argtypes = [u8p, ctypes.c_int32, ctypes.c_uint32]
        lib.oracle_murmur3_32.restype = ctypes.c_uint32
        lib.oracle_data_signatures.argtypes = [vp, u32p]
        lib.oracle_query_signatures.argtypes = q + [u32p]
        lib.oracle_query_signatures.restype = ctypes.c_int32
        lib.oracle_filter.argtypes = [vp] + q + [u8p, i64p]
        lib.oracle_filter.restype = ctypes.c_int32
        lib.oracle_join_step.argtypes = [vp, i32p, ctypes.c_int64, ctypes.c_int32, u8p, i32p, i32p,
                                         ctypes.c_int32, i32p, ctypes.c_int64]
        lib.oracle_join_step.restype = ctypes.c_int64
        lib.oracle_fingerprint.argtypes = [i32p, ctypes.c_int64, ctypes.c_int32, u64p]
        _lib = lib
    return _lib


def _i32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _c(a, dtype=np.int32):
    return np.ascontiguousarray(a, dtype=dtype)


def _threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


class OracleGraph:
    """The oracle's own adjacency of an undirected labelled graph."""

    def __init__(self, vlab, src, dst, elab):
        self.vlab = _c(vlab)
        self.src = _c(src)
        self.dst = _c(dst)
        self.elab = _c(elab)
        self.n = int(self.vlab.shape[0])
        self.m = int(self.src.shape[0])
        self._h = _load().oracle_graph_new(self.n, self.m, _i32(self.vlab), _i32(self.src), _i32(self.dst),
                                           _i32(self.elab))

    @classmethod
    def from_synth(cls, g) -> "OracleGraph":
        return cls(g.vlab, g.src, g.dst, g.elab)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.oracle_graph_free(self._h)
            self._h = None

    def edge_label(self, u: int, v: int) -> int:
        return int(_load().oracle_edge_label(self._h, u, v))


def _qargs(q):
    vl, s, d, e = _c(q.vlab), _c(q.src), _c(q.dst), _c(q.elab)
    return (vl, s, d, e), [int(vl.shape[0]), _i32(vl), _i32(s), _i32(d), _i32(e), int(s.shape[0])]


def _enum_fn(hom: bool):
    lib = _load()
    return lib.oracle_enumerate_hom if hom else lib.oracle_enumerate


def enumerate_rows(g: OracleGraph, q, max_rows: int | None = None, hom: bool = False) -> np.ndarray:
    """All embeddings (homomorphisms with hom=True; rows in query-vertex
    order), sorted lexicographically."""
    keep, a = _qargs(q)
    k = a[0]
    fn = _enum_fn(hom)
    if max_rows is None:
        cnt = fn(g._h, *a, None, 0, 1, None)
        if cnt < 0:
            raise ValueError("invalid query")
        max_rows = cnt
    out = np.empty((max(max_rows, 1), k), np.int32)
    cnt = fn(g._h, *a, _i32(out), max_rows, 1, None)
    if cnt < 0:
        raise ValueError("invalid query")
    rows = out[:min(cnt, max_rows)]
    return sort_rows(rows)


def count(g: OracleGraph, q, nthreads: int | None = None, hom: bool = False) -> tuple[int, tuple[int, int, int]]:
    """(count, fingerprint) with nthreads workers over the first position's candidates."""
    keep, a = _qargs(q)
    fp = (ctypes.c_uint64 * 3)()
    nt = _threads() if nthreads is None else nthreads
    cnt = _enum_fn(hom)(g._h, *a, None, 0, nt, fp)
    if cnt < 0:
        raise ValueError("invalid query")
    return int(cnt), (int(fp[0]), int(fp[1]), int(fp[2]))


def order(q) -> np.ndarray:
    keep, a = _qargs(q)
    out = np.empty(a[0], np.int32)
    if _load().oracle_order(*a, _i32(out)) != 0:
        raise ValueError("invalid query")
    return out


def bruteforce_rows(g: OracleGraph, q, hom: bool = False) -> np.ndarray:
    keep, a = _qargs(q)
    k = a[0]
    lib = _load()
    fn = lib.oracle_bruteforce_hom if hom else lib.oracle_bruteforce
    cnt = fn(g._h, *a, None, 0)
    if cnt < 0:
        raise ValueError("invalid query")
    out = np.empty((max(cnt, 1), k), np.int32)
    fn(g._h, *a, _i32(out), cnt)
    return sort_rows(out[:cnt])


def enumerate_edge_rows(g: OracleGraph, q) -> np.ndarray:
    """All edge-isomorphic matches (Sec. VII-A): rows of data edge ids, column
    j = query edge j, sorted lexicographically."""
    keep, a = _qargs(q)
    fn = _load().oracle_enumerate_edge
    cnt = fn(g._h, *a, None, 0, 1, None)
    if cnt < 0:
        raise ValueError("invalid query")
    out = np.empty((max(cnt, 1), a[5]), np.int32)
    fn(g._h, *a, _i32(out), cnt, 1, None)
    return sort_rows(out[:cnt])


def count_edge(g: OracleGraph, q, nthreads: int | None = None) -> tuple[int, tuple[int, int, int]]:
    """(count, fingerprint) of the edge-isomorphic matches."""
    keep, a = _qargs(q)
    fp = (ctypes.c_uint64 * 3)()
    nt = _threads() if nthreads is None else nthreads
    cnt = _load().oracle_enumerate_edge(g._h, *a, None, 0, nt, fp)
    if cnt < 0:
        raise ValueError("invalid query")
    return int(cnt), (int(fp[0]), int(fp[1]), int(fp[2]))


def bruteforce_edge_rows(g: OracleGraph, q) -> np.ndarray:
    """Edge-isomorphic matches by checking every map of query edges to data
    edges (tiny inputs only)."""
    keep, a = _qargs(q)
    fn = _load().oracle_bruteforce_edge
    cnt = fn(g._h, *a, None, 0)
    if cnt < 0:
        raise ValueError("invalid query")
    out = np.empty((max(cnt, 1), a[5]), np.int32)
    fn(g._h, *a, _i32(out), cnt)
    return sort_rows(out[:cnt])


def murmur3_32(data: bytes, seed: int) -> int:
    buf = (ctypes.c_uint8 * max(1, len(data))).from_buffer_copy(data if data else b"\0")
    return int(_load().oracle_murmur3_32(buf, len(data), seed))


def data_signatures(g: OracleGraph) -> np.ndarray:
    """uint32[n, 16], vertex-major."""
    out = np.empty((g.n, SIG_WORDS), np.uint32)
    _load().oracle_data_signatures(g._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return out


def query_signatures(q) -> np.ndarray:
    keep, a = _qargs(q)
    out = np.empty((a[0], SIG_WORDS), np.uint32)
    if _load().oracle_query_signatures(*a, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))) != 0:
        raise ValueError("invalid query")
    return out


def filter_sets(g: OracleGraph, q) -> tuple[np.ndarray, np.ndarray]:
    """(member bool[k, n], counts int64[k])."""
    keep, a = _qargs(q)
    member = np.empty((a[0], g.n), np.uint8)
    counts = np.empty(a[0], np.int64)
    r = _load().oracle_filter(g._h, *a, member.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                              counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if r != 0:
        raise ValueError("invalid query")
    return member.astype(bool), counts


def join_step(g: OracleGraph, M: np.ndarray, in_c: np.ndarray, cols, labs) -> np.ndarray:
    """Rows (m || w) of one join iteration, sorted."""
    M = _c(M)
    nrows, t = (M.shape[0], M.shape[1]) if M.ndim == 2 else (0, 0)
    in_c = _c(in_c, np.uint8)
    cols = _c(cols)
    labs = _c(labs)
    lib = _load()
    u8 = in_c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    cnt = lib.oracle_join_step(g._h, _i32(M), nrows, t, u8, _i32(cols), _i32(labs), len(cols), None, 0)
    if cnt < 0:
        raise ValueError("invalid step")
    out = np.empty((max(cnt, 1), t + 1), np.int32)
    lib.oracle_join_step(g._h, _i32(M), nrows, t, u8, _i32(cols), _i32(labs), len(cols), _i32(out), cnt)
    return sort_rows(out[:cnt])


def fingerprint(rows: np.ndarray) -> tuple[int, int, int]:
    rows = _c(rows)
    k = rows.shape[1] if rows.ndim == 2 else 0
    fp = (ctypes.c_uint64 * 3)()
    _load().oracle_fingerprint(_i32(rows), rows.shape[0], k, fp)
    return int(fp[0]), int(fp[1]), int(fp[2])


def sort_rows(rows: np.ndarray) -> np.ndarray:
    """Rows sorted lexicographically (first column most significant)."""
    rows = np.ascontiguousarray(rows, np.int32)
    if rows.shape[0] <= 1:
        return rows
    idx = np.lexsort(rows.T[::-1])
    return rows[idx]
