"""Seeded synthetic inputs: data graphs, labels, query graphs and workloads.

This module is shared by the CUDA library's tests/benchmark and by the CPU
oracle's tests.  It holds none of the matching method's arithmetic: it draws
graphs (Erdos-Renyi, R-MAT), labels (Zipf, uniform) and queries (random walks
from the data graph, as in the paper's experimental setup, Sec. VIII-A), and
returns plain numpy arrays.  The sampling code is C (``synth.c``), built by
:func:`build` with gcc into ``libsynth.so`` next to this file.

Workload recipes (``workload(name)``) fix every seed:

* ``tiny``     Erdos-Renyi n=1000, m=5000, vertex/edge labels uniform in {0..3};
               five 4-vertex shape queries (path, star, triangle+pendant, C4,
               K4 minus an edge), each an occurrence found in G.
* ``medium``   R-MAT scale 20 (a,b,c,d)=(.57,.19,.19,.05), 16M distinct
               undirected non-loop edges, ids permuted; 64 Zipf(1.1) vertex
               labels, 8 uniform edge labels; 100 random-walk queries with
               k ~ U{6..12}, alternately sparse (walk edges) and dense
               (walk edges plus induced edges up to |E| = 2k).
* ``scale``    R-MAT scale 24, 256M edges, 256 Zipf vertex labels, 16 edge
               labels; 20 queries with k ~ U{8..16}.
* ``batched``  the medium graph; 4,096 queries with k ~ U{4..16}, rare-label
               walks (below).
* ``served``   R-MAT scale 22, 64M edges, 128 Zipf vertex labels, 8 edge
               labels; 20,000 queries, k = 4 + Geometric(mean 4) clipped to
               [4, 16] (mean 8), rare-label walks, Poisson arrivals.
* ``edge``     Erdos-Renyi n=2^20, m=4M (degree at most a few dozen, so its
               line graph stays small: 4M vertices, about 30M edges); 4
               uniform vertex labels, 2 uniform edge labels; 100 random-walk
               queries with k ~ U{4..8}, asked as edge-isomorphism queries
               (Sec. VII-A).  The admission bound counts vertex
               homomorphisms, which bound the edge matches only roughly
               (they run 1-4x the embeddings here).

Random walks on these R-MAT graphs often hit hubs, and with only 8-16 edge
labels a tree-shaped walk query can have 10^9-10^13 embeddings.  Each walk
workload therefore carries an admission bound: a walk whose labelled
spanning-tree homomorphism count (an upper bound on its embedding count)
exceeds ``max_bound`` is redrawn with the next attempt counter.  This is a
deterministic stand-in for the paper's 100 s per-query timeout.  On these
graphs almost no uniform walk of 8 or more vertices passes 10^6 (the median
bound of a 10-vertex walk is about 4e11), so the batched and served
workloads, which stand for many small requests of 4..16 vertices, draw
rare-label walks: the walk starts at and steps to vertices whose label is 8
or above only (outside the eight most frequent Zipf labels, about 60% of the
vertices), as most labels of a real labelled graph are rare.  Such walks pass
the 10^6 bound within a few attempts at every size.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so (gcc, portable flags)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, src, "-lpthread", "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.synth_er.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, i32p, i32p]
        lib.synth_er.restype = ctypes.c_int64
        lib.synth_rmat.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int32, i32p, i32p]
        lib.synth_rmat.restype = ctypes.c_int64
        lib.synth_labels_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, i32p]
        lib.synth_labels_zipf.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_double, i32p]
        lib.synth_adj_build.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, i32p]
        lib.synth_adj_build.restype = ctypes.c_void_p
        lib.synth_adj_free.argtypes = [ctypes.c_void_p]
        lib.synth_adj_degree.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        lib.synth_adj_degree.restype = ctypes.c_int64
        lib.synth_walk_query.argtypes = [ctypes.c_void_p, i32p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, i32p, i32p, i32p, i32p, i32p,
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]
        lib.synth_walk_query.restype = ctypes.c_int32
        lib.synth_shape_query.argtypes = [ctypes.c_void_p, i32p, ctypes.c_uint64, ctypes.c_int32,
                                          i32p, i32p, i32p, i32p, i32p]
        lib.synth_shape_query.restype = ctypes.c_int32
        lib.synth_tree_hom_bound.argtypes = [ctypes.c_void_p, ctypes.c_int32, i32p, i32p, i32p, i32p,
                                             ctypes.c_int32, ctypes.c_int32]
        lib.synth_tree_hom_bound.restype = ctypes.c_double
        lib.synth_uniform_int.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_int32]
        lib.synth_uniform_int.restype = ctypes.c_int32
        lib.synth_unit.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64]
        lib.synth_unit.restype = ctypes.c_double
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


@dataclass
class Graph:
    """Undirected labelled data graph; each edge stored once with src < dst."""
    vlab: np.ndarray          # int32[n]
    src: np.ndarray           # int32[m]
    dst: np.ndarray           # int32[m]
    elab: np.ndarray          # int32[m]
    n_elabels: int
    name: str = ""
    _adj: int | None = field(default=None, repr=False)

    @property
    def n(self) -> int:
        return int(self.vlab.shape[0])

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    def adj(self):
        if self._adj is None:
            lib = _load()
            self._adj = lib.synth_adj_build(self.n, self.m, _p(self.src), _p(self.dst), _p(self.elab),
                                            _p(self.vlab))
        return self._adj

    def __del__(self):
        if self._adj is not None and _lib is not None:
            _lib.synth_adj_free(self._adj)
            self._adj = None


@dataclass
class Query:
    """Labelled query graph: k vertices, edges (src[i], dst[i]) with label elab[i]."""
    vlab: np.ndarray          # int32[k]
    src: np.ndarray           # int32[qm]
    dst: np.ndarray           # int32[qm]
    elab: np.ndarray          # int32[qm]
    occurrence: np.ndarray    # int32[k]: data vertices of one occurrence in G
    dense: bool = False
    bound: float = 0.0        # spanning-tree homomorphism bound (0 if not computed)
    attempts: int = 1         # walks drawn until this one was admitted

    @property
    def k(self) -> int:
        return int(self.vlab.shape[0])

    @property
    def qm(self) -> int:
        return int(self.src.shape[0])


def erdos_renyi(seed: int, n: int, m: int) -> tuple[np.ndarray, np.ndarray]:
    lib = _load()
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    r = lib.synth_er(seed, n, m, _threads(), _p(src), _p(dst))
    if r != m:
        raise ValueError("erdos_renyi: invalid size")
    return src, dst


def rmat(seed: int, scale: int, m: int, a=0.57, b=0.19, c=0.19) -> tuple[np.ndarray, np.ndarray]:
    lib = _load()
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    r = lib.synth_rmat(seed, scale, m, a, b, c, _threads(), _p(src), _p(dst))
    if r != m:
        raise ValueError("rmat: invalid size or out of memory")
    return src, dst


def labels_uniform(seed: int, stream: int, count: int, nlabels: int) -> np.ndarray:
    out = np.empty(count, np.int32)
    _load().synth_labels_uniform(seed, stream, count, nlabels, _p(out))
    return out


def labels_zipf(seed: int, stream: int, count: int, nlabels: int, s: float = 1.1) -> np.ndarray:
    out = np.empty(count, np.int32)
    _load().synth_labels_zipf(seed, stream, count, nlabels, s, _p(out))
    return out


def make_graph(vlab, src, dst, elab, n_elabels, name="") -> Graph:
    return Graph(np.ascontiguousarray(vlab, np.int32), np.ascontiguousarray(src, np.int32),
                 np.ascontiguousarray(dst, np.int32), np.ascontiguousarray(elab, np.int32), int(n_elabels), name)


def walk_query(g: Graph, seed: int, index: int, k: int, dense: bool, max_bound: float = 0.0,
               max_attempts: int = 0, min_label: int = 0) -> Query:
    """Random-walk query; with max_bound > 0, walks whose labelled spanning-tree
    homomorphism count (an upper bound on the embedding count) exceeds
    max_bound are redrawn.  With min_label > 0 the walk starts at and steps to
    vertices labelled min_label or above only (a rare-label walk)."""
    lib = _load()
    qvlab = np.empty(k, np.int32)
    cap = max(2 * k, k * (k - 1) // 2) + 1
    qsrc = np.empty(cap, np.int32)
    qdst = np.empty(cap, np.int32)
    qelab = np.empty(cap, np.int32)
    occ = np.empty(k, np.int32)
    bound = ctypes.c_double(0.0)
    attempts = ctypes.c_int32(0)
    ne = lib.synth_walk_query(g.adj(), _p(g.vlab), seed, index, k, int(dense), float(max_bound), 1,
                              int(max_attempts), int(min_label), _p(qvlab), _p(qsrc), _p(qdst), _p(qelab), _p(occ),
                              ctypes.byref(bound), ctypes.byref(attempts))
    if ne < 0:
        raise RuntimeError(f"walk_query: no admissible walk reached {k} vertices")
    return Query(qvlab, qsrc[:ne].copy(), qdst[:ne].copy(), qelab[:ne].copy(), occ, dense, bound.value,
                 int(attempts.value))


def tree_hom_bound(g: Graph, q: Query) -> float:
    return float(_load().synth_tree_hom_bound(g.adj(), q.k, _p(q.vlab), _p(q.src), _p(q.dst), _p(q.elab),
                                              q.qm, _threads()))


SHAPES = ("path", "star", "paw", "c4", "diamond")


def shape_query(g: Graph, seed: int, shape: int) -> Query:
    lib = _load()
    qvlab = np.empty(4, np.int32)
    qsrc = np.empty(6, np.int32)
    qdst = np.empty(6, np.int32)
    qelab = np.empty(6, np.int32)
    occ = np.empty(4, np.int32)
    ne = lib.synth_shape_query(g.adj(), _p(g.vlab), seed, shape, _p(qvlab), _p(qsrc), _p(qdst), _p(qelab), _p(occ))
    if ne < 0:
        raise RuntimeError(f"shape_query: no occurrence of {SHAPES[shape]}")
    return Query(qvlab, qsrc[:ne].copy(), qdst[:ne].copy(), qelab[:ne].copy(), occ, shape >= 2)


def uniform_int(seed: int, stream: int, idx: int, lo: int, hi: int) -> int:
    return int(_load().synth_uniform_int(seed, stream, idx, lo, hi))


def unit(seed: int, stream: int, idx: int) -> float:
    return float(_load().synth_unit(seed, stream, idx))


# ----------------------------------------------------------------- recipes
@dataclass
class GraphSpec:
    kind: str                 # "er" or "rmat"
    n: int
    m: int
    n_vlabels: int
    n_elabels: int
    vlab_dist: str            # "uniform" or "zipf"
    seed: int
    scale: int = 0


@dataclass
class WorkloadSpec:
    name: str
    graph: GraphSpec
    n_queries: int
    k_lo: int
    k_hi: int
    k_dist: str               # "shapes", "uniform" or "geometric"
    query_seed: int
    row_cap: int = 0          # 0 = no cap on materialised rows
    max_bound: float = 0.0    # admission bound on the spanning-tree homomorphism count
    description: str = ""
    min_label: int = 0        # > 0: queries of rare_from_k or more vertices are rare-label walks
    rare_from_k: int = 0      #      (vertices labelled min_label or above only)


GRAPHS = {
    "er1k": GraphSpec("er", 1000, 5000, 4, 4, "uniform", 1001),
    "rmat20": GraphSpec("rmat", 1 << 20, 16_000_000, 64, 8, "zipf", 1002, scale=20),
    "rmat24": GraphSpec("rmat", 1 << 24, 256_000_000, 256, 16, "zipf", 1003, scale=24),
    "rmat22": GraphSpec("rmat", 1 << 22, 64_000_000, 128, 8, "zipf", 1005, scale=22),
    "er20": GraphSpec("er", 1 << 20, 4_000_000, 4, 2, "uniform", 1006),
}

WORKLOADS = {
    "tiny": WorkloadSpec("tiny", GRAPHS["er1k"], 5, 4, 4, "shapes", 2001,
                         description="ER n=1000 m=5000, 4x4 uniform labels, 5 shape queries k=4"),
    "medium": WorkloadSpec("medium", GRAPHS["rmat20"], 100, 6, 12, "uniform", 2002, max_bound=1e8,
                           description="R-MAT 2^20 / 16M edges, 64 Zipf vlabels, 8 elabels, 100 walk queries k=6..12"),
    "scale": WorkloadSpec("scale", GRAPHS["rmat24"], 20, 8, 16, "uniform", 2003, row_cap=1_000_000_000,
                          max_bound=1e10,
                          description="R-MAT 2^24 / 256M edges, 256 Zipf vlabels, 16 elabels, 20 queries k=8..16"),
    "batched": WorkloadSpec("batched", GRAPHS["rmat20"], 4096, 4, 16, "uniform", 2004, max_bound=1e6,
                            description="R-MAT 2^20 graph, 4096 rare-label walk queries k=4..16",
                            min_label=8, rare_from_k=4),
    "served": WorkloadSpec("served", GRAPHS["rmat22"], 20000, 4, 16, "geometric", 2005, max_bound=1e6,
                           description="R-MAT 2^22 / 64M edges, 20000 rare-label walk queries k=4+Geom (mean 8), "
                                       "clipped to 16",
                           min_label=8, rare_from_k=4),
    "edge": WorkloadSpec("edge", GRAPHS["er20"], 100, 4, 8, "uniform", 2006, max_bound=1e7,
                         description="ER 2^20 / 4M edges, 4 vlabels, 2 elabels, 100 walk queries k=4..8 "
                                     "asked as edge-isomorphism queries"),
}

_GRAPH_CACHE: dict[str, Graph] = {}


def graph(name: str) -> Graph:
    """Build (and memoise) one of the named data graphs."""
    if name in _GRAPH_CACHE:
        return _GRAPH_CACHE[name]
    s = GRAPHS[name]
    if s.kind == "er":
        src, dst = erdos_renyi(s.seed, s.n, s.m)
    else:
        src, dst = rmat(s.seed, s.scale, s.m)
    if s.vlab_dist == "zipf":
        vlab = labels_zipf(s.seed, 1, s.n, s.n_vlabels, 1.1)
    else:
        vlab = labels_uniform(s.seed, 1, s.n, s.n_vlabels)
    elab = labels_uniform(s.seed, 2, s.m, s.n_elabels)
    g = make_graph(vlab, src, dst, elab, s.n_elabels, name)
    _GRAPH_CACHE[name] = g
    return g


def query_size(w: WorkloadSpec, i: int) -> int:
    if w.k_dist == "geometric":
        # k = 4 + G, G geometric on {0,1,...} with mean 4 (p = 1/5), so that k
        # has mean 8, clipped to k_hi
        u = unit(w.query_seed, 7, i)
        p = 1.0 / 5.0
        g = int(math.floor(math.log1p(-u) / math.log1p(-p)))
        return max(w.k_lo, min(w.k_hi, 4 + g))
    return uniform_int(w.query_seed, 5, i, w.k_lo, w.k_hi)


def drawn_size(w: WorkloadSpec, i: int) -> int:
    return query_size(w, i)


def queries(name: str, count: int | None = None, start: int = 0) -> list[Query]:
    """Queries of a named workload (index range [start, start+count)).

    Walk queries are drawn in parallel threads (each query is a pure function
    of its index, so the result does not depend on the thread count)."""
    w = WORKLOADS[name]
    g = graph(_graph_name(w))
    count = w.n_queries - start if count is None else count
    idx = list(range(start, start + count))
    if w.k_dist == "shapes":
        return [shape_query(g, w.query_seed, i % 5) for i in idx]
    g.adj()
    from concurrent.futures import ThreadPoolExecutor

    def one(i):
        k = drawn_size(w, i)
        rare = w.min_label if (w.min_label and k >= w.rare_from_k) else 0
        return walk_query(g, w.query_seed, i, k, dense=(i % 2 == 1), max_bound=w.max_bound, min_label=rare)

    with ThreadPoolExecutor(max_workers=_threads()) as ex:
        return list(ex.map(one, idx))


def _graph_name(w: WorkloadSpec) -> str:
    for k, v in GRAPHS.items():
        if v is w.graph:
            return k
    raise KeyError(w.name)


def workload_graph(name: str) -> Graph:
    return graph(_graph_name(WORKLOADS[name]))


def poisson_arrivals(seed: int, count: int, rate: float) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    u = np.array([unit(seed, 9, i) for i in range(count)])
    gaps = -np.log1p(-u) / rate
    return np.cumsum(gaps)
