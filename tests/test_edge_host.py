"""The library's line-graph transform for edge isomorphism (Sec. VII-A),
checked on the CPU through the C ABI (host-only edge graphs, no CUDA call).

The main check composes the library's transform with the oracle's vertex
enumeration.  Matching the library's Q' in the library's G' must give exactly
the oracle's edge-isomorphic matches, which the oracle computes on G itself
with no line graph."""
import math

import numpy as np
import pytest

import oracle
from tests import helpers as H


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1906_03420_gb300 as p
    p.load()
    return p


def og(vlab, src, dst, elab):
    return oracle.OracleGraph(vlab, src, dst, elab)


def edge_graph(pkg, g):
    return pkg.EdgeGraph(g.vlab, g.src, g.dst, g.elab, host_only=True)


def test_figure_example_becomes_a_triangle(pkg):
    """Sec. VII-A's figure: edges e1, e2, e3 at v0 become three line-graph
    vertices joined pairwise, each join standing for v0."""
    g = H.graph(4, [(0, 1), (0, 2), (0, 3)], [5, 7, 7, 9])
    vl, s, d, e = edge_graph(pkg, g).line_graph()
    assert vl.shape[0] == 3
    assert sorted(zip(s.tolist(), d.tolist())) == [(0, 1), (0, 2), (1, 2)]
    assert e.tolist() == [0, 0, 0]                  # rank of v0's label 5 among {5, 7, 9}
    # edges {0,1} and {0,2}: labels (5,7) and (5,7) -> same id; {0,3}: (5,9) -> another
    assert vl[0] == vl[1] != vl[2]


@pytest.mark.parametrize("seed", range(3))
def test_line_graph_structure(pkg, seed):
    """G' has one vertex per edge and one edge per pair of edges meeting at
    a vertex (sum_v C(deg v, 2) edges), labelled with that vertex's label
    rank.  Vertex labels agree exactly when (edge label, endpoint label pair)
    agree."""
    rng = np.random.default_rng(500 + seed)
    for _ in range(10):
        g = H.random_graph(rng, int(rng.integers(4, 30)), float(rng.uniform(0.05, 0.4)), 4, 3)
        if g.m == 0:
            continue
        vl, s, d, e = edge_graph(pkg, g).line_graph()
        deg = np.bincount(np.concatenate([g.src, g.dst]), minlength=g.n)
        assert s.shape[0] == sum(math.comb(int(x), 2) for x in deg)
        assert (s < d).all()
        labels = sorted(set(g.vlab.tolist()))
        seen = set()
        for a, b, lab in zip(s.tolist(), d.tolist(), e.tolist()):
            common = {int(g.src[a]), int(g.dst[a])} & {int(g.src[b]), int(g.dst[b])}
            assert len(common) == 1
            assert lab == labels.index(int(g.vlab[common.pop()]))
            seen.add((a, b))
        assert len(seen) == s.shape[0]
        key = [(int(g.elab[i]), tuple(sorted((int(g.vlab[g.src[i]]), int(g.vlab[g.dst[i]]))))) for i in range(g.m)]
        for i in range(g.m):
            for j in range(g.m):
                assert (vl[i] == vl[j]) == (key[i] == key[j])


@pytest.mark.parametrize("block", range(4))
def test_transform_then_vertex_matching_equals_edge_isomorphism(pkg, block):
    """The library's G' and Q', matched by the oracle's vertex enumeration,
    give the oracle's edge-isomorphic matches computed on G (388 cases run)."""
    rng = np.random.default_rng(600 + block)
    for case in range(100):
        g = H.random_graph(rng, int(rng.integers(4, 14)), float(rng.uniform(0.1, 0.5)), int(rng.integers(1, 4)),
                           int(rng.integers(1, 3)))
        if g.m == 0:
            continue
        k = int(rng.integers(2, 6))
        q = H.random_connected_query(rng, k, int(rng.integers(0, 3)), int(rng.integers(1, 5)),
                                     int(rng.integers(1, 4)))    # labels G may lack
        eg = edge_graph(pkg, g)
        lg = og(*eg.line_graph())
        lq = eg.line_query(q)
        assert lq.k == len(q.src)
        got = oracle.enumerate_rows(lg, lq)
        want = oracle.enumerate_edge_rows(og(g.vlab, g.src, g.dst, g.elab), q)
        assert np.array_equal(got, want), (block, case)


@pytest.mark.parametrize("block", range(3))
def test_transform_on_queries_taken_from_the_graph(pkg, block):
    """As above, with queries cut out of G (so each has matches) and few
    labels (so the line graph has many equal labels): 225 cases run."""
    rng = np.random.default_rng(700 + block)
    nonzero = 0
    for case in range(80):
        g = H.random_graph(rng, int(rng.integers(5, 12)), float(rng.uniform(0.2, 0.5)), int(rng.integers(1, 3)),
                           int(rng.integers(1, 3)))
        if g.m < 2:
            continue
        q = H.extracted_query(rng, g, int(rng.integers(2, 5)))
        if q is None or len(q.src) == 0:
            continue
        eg = edge_graph(pkg, g)
        got = oracle.enumerate_rows(og(*eg.line_graph()), eg.line_query(q))
        want = oracle.enumerate_edge_rows(og(g.vlab, g.src, g.dst, g.elab), q)
        assert np.array_equal(got, want), (block, case)
        nonzero += want.shape[0] > 0
    assert nonzero >= 40


def test_query_labels_missing_from_the_graph(pkg):
    """A query vertex or edge label that G lacks yields labels nothing in G'
    carries: -1 on Q' vertices, INT32_MAX on Q' edges."""
    g = H.graph(3, [(0, 1), (1, 2)], [0, 1, 0], [0, 0])
    eg = edge_graph(pkg, g)
    lq = eg.line_query(H.query(3, [(0, 1), (1, 2)], [0, 2, 0], [0, 0]))   # label 2 absent
    assert lq.vlab.tolist() == [-1, -1] and lq.elab.tolist() == [2 ** 31 - 1]
    lq = eg.line_query(H.query(3, [(0, 1), (1, 2)], [0, 1, 0], [0, 5]))   # edge label 5 absent
    assert lq.vlab[1] == -1 and lq.vlab[0] >= 0 and lq.elab.tolist() == [1]


@pytest.mark.parametrize("edges", [
    [(0, 1), (0, 1)],          # repeated pair
    [(0, 1), (1, 0)],          # repeated pair, reversed
    [(0, 0)],                  # self-loop
    [(0, 5)],                  # id out of range
    [],                        # no edge
])
def test_invalid_graphs_rejected(pkg, edges):
    g = H.G(H.arr([0, 0, 0]), H.arr([a for a, _ in edges]), H.arr([b for _, b in edges]), H.arr([0] * len(edges)))
    with pytest.raises(pkg.GsiError) as e:
        edge_graph(pkg, g)
    assert e.value.status == pkg.GSI_EINVAL


def test_negative_edge_label_rejected(pkg):
    g = H.graph(3, [(0, 1), (1, 2)], None, [0, -2])
    with pytest.raises(pkg.GsiError) as e:
        edge_graph(pkg, g)
    assert e.value.status == pkg.GSI_EINVAL


def test_line_graph_size_limit(pkg):
    """A star with 65,537 leaves has C(65537, 2) >= 2^31 line-graph edges."""
    n = 65538
    g = H.G(np.zeros(n, np.int32), np.zeros(n - 1, np.int32), np.arange(1, n, dtype=np.int32),
            np.zeros(n - 1, np.int32))
    with pytest.raises(pkg.GsiError) as e:
        edge_graph(pkg, g)
    assert e.value.status == pkg.GSI_EINVAL and "line graph" in str(e.value)


@pytest.mark.parametrize("q", [
    H.query(1, []),                                           # no edge
    H.query(3, [(0, 1)]),                                     # disconnected
    H.query(34, [(i, i + 1) for i in range(33)]),             # 33 edges (and 34 vertices)
])
def test_invalid_edge_queries_rejected(pkg, q):
    eg = edge_graph(pkg, H.complete(4))
    with pytest.raises(pkg.GsiError) as e:
        eg.line_query(q)
    assert e.value.status == pkg.GSI_EINVAL


def test_host_only_graph_cannot_run_queries(pkg):
    eg = edge_graph(pkg, H.complete(4))
    with pytest.raises(pkg.GsiError) as e:
        eg.query(H.path_query(3))
    assert e.value.status == pkg.GSI_EINVAL
    with pytest.raises(pkg.GsiError):
        eg.line()


def test_device_edge_graph_needs_a_gpu(pkg):
    """Without a usable GPU the device build reports GSI_ECUDA (no CPU fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    g = H.complete(4)
    with pytest.raises(pkg.GsiError) as e:
        pkg.EdgeGraph(g.vlab, g.src, g.dst, g.elab)
    assert e.value.status == pkg.GSI_ECUDA


def test_transform_at_the_benchmark_size(pkg):
    """The edge workload's full graph (ER 2^20 / 4M edges; line graph 4M
    vertices, about 30.5M edges): the library's G' and Q' of the first three
    queries, matched by the oracle's vertex enumeration, give exactly the
    oracle's edge matches on G (rows and fingerprints)."""
    import synth
    g = synth.workload_graph("edge")
    eg = pkg.EdgeGraph.from_synth(g, host_only=True)
    vl, s, d, e = eg.line_graph()
    deg = np.bincount(np.concatenate([g.src, g.dst]), minlength=g.n).astype(np.int64)
    assert vl.shape[0] == g.m and s.shape[0] == int((deg * (deg - 1) // 2).sum())
    lg = og(vl, s, d, e)
    O = og(g.vlab, g.src, g.dst, g.elab)
    for i, q in enumerate(synth.queries("edge", 3)):
        got = oracle.enumerate_rows(lg, eg.line_query(q))
        want, fp = oracle.count_edge(O, q)
        assert got.shape[0] == want and oracle.fingerprint(got) == (want, fp[1], fp[2]), i
