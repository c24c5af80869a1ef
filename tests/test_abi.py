"""C-ABI library checks that need no GPU: it loads, exports every declared
symbol, and its host-only logic (query signatures, Alg. 2 planner, query
validation) behaves as the paper states."""
import os
import re

import numpy as np
import pytest

import oracle
from tests import helpers as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1906_03420_gb300 as p
    p.load()
    return p


def declared_functions():
    text = open(os.path.join(ROOT, "include", "gsi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gsi_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(pkg):
    lib = pkg.load()
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(pkg.EXPORTED)
    assert pkg.version().startswith("gsi-gb300")


def test_library_is_built_for_sm103a(pkg):
    from paper_1906_03420_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
    assert os.path.exists(pkg.lib_path())


def test_no_cpu_fallback_without_gpu(pkg):
    """Without a usable GPU the library reports GSI_ECUDA instead of computing on the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    g = H.complete(4)
    with pytest.raises(pkg.GsiError) as e:
        pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    assert e.value.status == pkg.GSI_ECUDA


@pytest.mark.parametrize("seed", range(4))
def test_query_signatures_match_oracle(pkg, seed):
    """Sec. III-A signatures: the library's host encoder equals the oracle's, bit for bit."""
    rng = np.random.default_rng(seed)
    for _ in range(40):
        k = int(rng.integers(1, 12))
        q = H.random_connected_query(rng, k, int(rng.integers(0, 6)), int(rng.integers(1, 70)),
                                     int(rng.integers(1, 20)))
        assert np.array_equal(pkg.query_signatures(q), oracle.query_signatures(q))


def _q(k, edges, labels=None):
    return H.query(k, edges, None, labels if labels is not None else [0] * len(edges))


def test_plan_first_vertex_is_min_score(pkg):
    """Alg. 2: start at argmin |C(u)| / deg(u)."""
    q = _q(4, [(0, 1), (1, 2), (2, 3), (1, 3)])
    # deg = [1, 3, 2, 2]; scores = [10, 10, 20, 4]
    order, first = pkg.plan_order(q, [10, 30, 40, 8], [5])
    assert order[0] == 3 and first[0] == -1


def test_plan_follows_frequency_weighted_scores(pkg):
    """Alg. 2: after a pick, neighbours' scores are multiplied by freq(edge label)."""
    # path 0-1-2 plus 0-3; labels: 0-1 -> a (freq 100), 0-3 -> b (freq 1)
    q = _q(4, [(0, 1), (1, 2), (0, 3)], [0, 0, 1])
    order, first = pkg.plan_order(q, [1, 50, 50, 60], [100, 1])
    # start at 0 (score 1/2); then 1: 50*100/2 = 2500, 3: 60*1 = 60 -> 3
    assert list(order[:2]) == [0, 3]
    assert order[2] == 1 and order[3] == 2


def test_plan_ties_take_lowest_id(pkg):
    q = _q(3, [(0, 1), (1, 2), (0, 2)])
    order, _ = pkg.plan_order(q, [7, 7, 7], [3])
    assert list(order) == [0, 1, 2]


def test_plan_first_edge_is_least_frequent_label(pkg):
    """Alg. 4: among linking edges, e0 has the least frequent label (ties: lowest id)."""
    q = _q(3, [(0, 2), (1, 2), (0, 1)], [3, 1, 0])
    order, first = pkg.plan_order(q, [1, 2, 100], [50, 10, 7, 40])
    assert list(order) == [0, 1, 2]
    assert first[1] == 0
    # vertex 2 links to 0 (label 3, freq 40) and 1 (label 1, freq 10)
    assert first[2] == 1


def test_plan_order_is_connected(pkg):
    rng = np.random.default_rng(5)
    for _ in range(100):
        k = int(rng.integers(2, 16))
        q = H.random_connected_query(rng, k, int(rng.integers(0, 8)), 4, 4)
        cand = rng.integers(1, 1000, k)
        order, first = pkg.plan_order(q, cand, rng.integers(1, 100, 4))
        assert sorted(order.tolist()) == list(range(k))
        adj = set()
        for a, b in zip(q.src, q.dst):
            adj.add((int(a), int(b))); adj.add((int(b), int(a)))
        for p in range(1, k):
            assert (int(order[p]), int(first[p])) in adj
            assert int(first[p]) in order[:p].tolist()


@pytest.mark.parametrize("bad", [
    dict(k=0, edges=[]),
    dict(k=33, edges=[(i, i + 1) for i in range(32)]),
    dict(k=3, edges=[(0, 1)]),                  # disconnected
    dict(k=3, edges=[(0, 1), (1, 1), (1, 2)]),  # self-loop
    dict(k=3, edges=[(0, 1), (1, 0), (1, 2)]),  # repeated pair
    dict(k=2, edges=[(0, 2)]),                  # id out of range
])
def test_invalid_queries_rejected(pkg, bad):
    q = _q(bad["k"], bad["edges"]) if bad["k"] > 0 else H.Q(np.zeros(0, np.int32), np.zeros(0, np.int32),
                                                                np.zeros(0, np.int32), np.zeros(0, np.int32))
    with pytest.raises(pkg.GsiError) as e:
        pkg.plan_order(q, [1] * max(q.k, 1), [1])
    assert e.value.status == pkg.GSI_EINVAL


def test_negative_query_label_rejected(pkg):
    q = _q(2, [(0, 1)], [-1])
    with pytest.raises(pkg.GsiError) as e:
        pkg.plan_order(q, [1, 1], [1])
    assert e.value.status == pkg.GSI_EINVAL


def test_header_constants_match_the_binding(pkg):
    """Status codes, semantics values and fixed sizes in include/gsi.h agree
    with the constants and struct layouts of the Python binding."""
    import ctypes
    import re
    from paper_1906_03420_gb300 import gsi as b
    text = open(os.path.join(ROOT, "include", "gsi.h")).read()
    enums = dict((k, int(v)) for k, v in re.findall(r"\b(GSI_[A-Z_]+)\s*=\s*(\d+)", text))
    for name in ("GSI_OK", "GSI_EINVAL", "GSI_ENOMEM", "GSI_ECAPPED", "GSI_ETIMEOUT", "GSI_ECANCELLED", "GSI_ECUDA",
                 "GSI_EBUSY", "GSI_ISOMORPHISM", "GSI_HOMOMORPHISM"):
        assert getattr(pkg, name) == enums[name], name
    defines = dict((k, int(v)) for k, v in re.findall(r"#define\s+(GSI_[A-Z_]+)\s+(\d+)", text))
    assert defines["GSI_MAX_QUERY_VERTICES"] == 32 and defines["GSI_SIG_WORDS"] == b.SIG_WORDS
    assert defines["GSI_EDGE_HOST_ONLY"] == pkg.GSI_EDGE_HOST_ONLY
    # every struct the binding passes by pointer has the header's field order and types
    fields = lambda name: [f[0] for f in getattr(b, name)._fields_]
    assert fields("c_query_opts") == ["stream", "row_cap", "mem_budget", "count_only", "semantics", "order", "stats",
                                      "host_driven", "listwise_bytes", "no_dedup", "tight_rows"]
    assert fields("c_batch_opts") == ["stream", "row_cap", "mem_budget", "count_only", "stats", "seeds_per_item",
                                      "item_rows", "isect", "rows_per_thread", "block_threads"]
    assert fields("c_server_opts") == ["mem_budget", "n_streams", "row_cap", "count_only", "max_batch",
                                       "seeds_per_item", "item_rows", "min_batch", "isect", "rows_per_thread",
                                       "block_threads"]
    for name in ("GSI_ISECT_BSEARCH", "GSI_ISECT_MERGE", "GSI_ISECT_BITMAP"):
        assert defines[name] == getattr(pkg, name), name
    for st, members in (("gsi_query_opts", fields("c_query_opts")), ("gsi_batch_opts", fields("c_batch_opts")),
                        ("gsi_server_opts", fields("c_server_opts")), ("gsi_graph_opts", fields("c_graph_opts")),
                        ("gsi_graph_info", fields("c_graph_info")), ("gsi_stats", fields("c_stats")),
                        ("gsi_query_desc", fields("c_query_desc"))):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + st + ";", text).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        declared = []
        for decl in body.split(";"):                    # "int32_t a, b" and "T *x[32]" forms
            decl = re.sub(r"\[[^\]]*\]", "", decl).strip()
            if not decl:
                continue
            names = decl.split(",")
            declared.append(re.findall(r"(\w+)\s*$", names[0])[0])
            declared += [n.strip().lstrip("*").strip() for n in names[1:]]
        assert declared == members, (st, declared)
