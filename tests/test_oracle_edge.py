"""Pins for the oracle's edge-isomorphism mode (Sec. VII-A), independent of it.

Edge isomorphism maps query edges to data edges injectively.  Two query
edges that share a vertex must go to data edges that share a vertex.  The
oracle also keeps edge labels, endpoint labels and the label of each shared
vertex.  It works on G directly.  The checks here:

- exhaustive search over every edge map;
- networkx's line graph with its VF2 subgraph monomorphisms, which is the
  transform the paper describes, done by a library;
- closed-form counts on unlabelled graphs, including Whitney's exception
  (a triangle and a 3-star have the same line graph);
- the invariant that every vertex embedding induces an edge match.
"""
import math

import numpy as np
import pytest

import oracle
from tests import helpers as H


def og(g):
    return oracle.OracleGraph(g.vlab, g.src, g.dst, g.elab)


@pytest.mark.parametrize("block", range(6))
def test_edge_backtracking_equals_bruteforce(block):
    """Random labelled cases (566 run): backtracking over query edges equals the
    exhaustive check of all m^|E(Q)| maps, rows and fingerprints."""
    rng = np.random.default_rng(4000 + block)
    for case in range(100):
        n = int(rng.integers(3, 8))
        g = H.random_graph(rng, n, float(rng.uniform(0.2, 0.7)), int(rng.integers(1, 3)), int(rng.integers(1, 3)))
        if g.m == 0:
            continue
        qm_max = 3 if g.m > 8 else 4
        k = int(rng.integers(2, qm_max + 2))
        q = H.random_connected_query(rng, k, 0, int(rng.integers(1, 3)), int(rng.integers(1, 3)))
        if len(q.src) > qm_max:
            continue
        G = og(g)
        got = oracle.enumerate_edge_rows(G, q)
        want = oracle.bruteforce_edge_rows(G, q)
        assert got.shape == want.shape and np.array_equal(got, want), (block, case)
        c, fp = oracle.count_edge(G, q, nthreads=3)
        assert c == want.shape[0] and fp == oracle.fingerprint(want)


def test_edge_bruteforce_with_cycles_in_the_query():
    """Queries with cycles (triangle, 4-cycle, triangle with a tail), labelled."""
    rng = np.random.default_rng(4100)
    shapes = [[(0, 1), (1, 2), (0, 2)], [(0, 1), (1, 2), (2, 3), (0, 3)], [(0, 1), (1, 2), (0, 2), (2, 3)]]
    for case in range(60):
        g = H.random_graph(rng, 6, float(rng.uniform(0.4, 0.8)), int(rng.integers(1, 3)), 1)
        edges = shapes[case % 3]
        k = 1 + max(max(e) for e in edges)
        q = H.query(k, edges, rng.integers(0, 2, k), [0] * len(edges))
        G = og(g)
        assert np.array_equal(oracle.enumerate_edge_rows(G, q), oracle.bruteforce_edge_rows(G, q)), case


def _line_graph_matches(g, q):
    """Rows of data edge ids from networkx: VF2 subgraph monomorphisms of
    L(Q) into L(G), vertices of the line graphs labelled by (edge label,
    endpoint label pair) and their edges by the shared vertex's label."""
    nx = pytest.importorskip("networkx")
    from networkx.algorithms import isomorphism as iso

    def line(vlab, src, dst, elab):
        base = nx.Graph()
        ids = {}
        for i, (a, b) in enumerate(zip(src.tolist(), dst.tolist())):
            base.add_edge(a, b)
            ids[frozenset((a, b))] = i
        L = nx.line_graph(base)
        out = nx.Graph()
        for node in L.nodes:
            i = ids[frozenset(node)]
            a, b = int(src[i]), int(dst[i])
            out.add_node(i, key=(int(elab[i]), tuple(sorted((int(vlab[a]), int(vlab[b]))))))
        for x, y in L.edges:
            common = set(x) & set(y)
            assert len(common) == 1
            out.add_edge(ids[frozenset(x)], ids[frozenset(y)], key=int(vlab[common.pop()]))
        return out

    LG = line(g.vlab, g.src, g.dst, g.elab)
    LQ = line(q.vlab, q.src, q.dst, q.elab)
    gm = iso.GraphMatcher(LG, LQ, node_match=lambda a, b: a["key"] == b["key"],
                          edge_match=lambda a, b: a["key"] == b["key"])
    rows = []
    for mapping in gm.subgraph_monomorphisms_iter():
        row = [0] * len(q.src)
        for data_edge, query_edge in mapping.items():
            row[query_edge] = data_edge
        rows.append(row)
    return oracle.sort_rows(np.array(rows, np.int32).reshape(-1, len(q.src)))


@pytest.mark.parametrize("seed", range(3))
def test_edge_matches_equal_networkx_line_graph_monomorphisms(seed):
    """Sec. VII-A's transform done by a library: the oracle's matches on G
    equal networkx's monomorphisms of L(Q) into L(G)."""
    rng = np.random.default_rng(4200 + seed)
    for case in range(25):
        g = H.random_graph(rng, int(rng.integers(5, 12)), float(rng.uniform(0.15, 0.5)),
                           int(rng.integers(1, 3)), int(rng.integers(1, 3)))
        if g.m == 0:
            continue
        k = int(rng.integers(2, 6))
        q = H.random_connected_query(rng, k, int(rng.integers(0, 2)), int(rng.integers(1, 3)),
                                     int(rng.integers(1, 3)))
        want = _line_graph_matches(g, q)
        got = oracle.enumerate_edge_rows(og(g), q)
        assert np.array_equal(got, want), (seed, case)


def test_edge_closed_forms():
    """Unlabelled graphs:
    one edge -> m;
    2-path -> sum_v deg(v)(deg(v)-1);
    3-star and triangle -> 6 (sum_v C(deg(v), 3) + triangles of G), because
    three pairwise adjacent edges form a star or a triangle (Whitney);
    3-path -> sum over edges xy of a(a-1), where a = deg(x) + deg(y) - 2
    counts the edges adjacent to xy."""
    rng = np.random.default_rng(4300)
    for _ in range(6):
        g = H.random_graph(rng, 16, float(rng.uniform(0.15, 0.5)), 1, 1)
        G = og(g)
        A = np.zeros((g.n, g.n), np.int64)
        A[g.src, g.dst] = 1
        A[g.dst, g.src] = 1
        deg = A.sum(axis=1)
        tri = int(np.trace(np.linalg.matrix_power(A, 3))) // 6
        assert oracle.count_edge(G, H.path_query(2))[0] == g.m
        assert oracle.count_edge(G, H.path_query(3))[0] == int((deg * (deg - 1)).sum())
        three = 6 * (sum(math.comb(int(d), 3) for d in deg) + tri)
        assert oracle.count_edge(G, H.star_query(3))[0] == three
        assert oracle.count_edge(G, H.clique_query(3))[0] == three
        a = deg[g.src] + deg[g.dst] - 2
        assert oracle.count_edge(G, H.path_query(4))[0] == int((a * (a - 1)).sum())


def test_edge_figure_example():
    """Sec. VII-A's figure: three edges at one vertex become three pairwise
    adjacent line-graph vertices, so a triangle query matches them in all
    3! orders, as does the 3-star."""
    g = H.graph(4, [(0, 1), (0, 2), (0, 3)])
    G = og(g)
    want = oracle.sort_rows(np.array([[0, 1, 2], [0, 2, 1], [1, 0, 2], [1, 2, 0], [2, 0, 1], [2, 1, 0]], np.int32))
    assert np.array_equal(oracle.enumerate_edge_rows(G, H.clique_query(3)), want)
    assert np.array_equal(oracle.enumerate_edge_rows(G, H.star_query(3)), want)


def test_edge_labels_select():
    """Edge labels, endpoint labels and the shared vertex's label all count."""
    # path 0-1-2 with vertex labels A B A and edge labels 0, 1
    g = H.graph(3, [(0, 1), (1, 2)], [0, 1, 0], [0, 1])
    G = og(g)
    assert oracle.count_edge(G, H.query(3, [(0, 1), (1, 2)], [0, 1, 0], [0, 1]))[0] == 1
    assert oracle.count_edge(G, H.query(3, [(0, 1), (1, 2)], [0, 1, 0], [1, 0]))[0] == 1   # mirror
    assert oracle.count_edge(G, H.query(3, [(0, 1), (1, 2)], [0, 1, 0], [0, 0]))[0] == 0   # edge label
    assert oracle.count_edge(G, H.query(3, [(0, 1), (1, 2)], [1, 0, 1], [0, 1]))[0] == 0   # endpoint labels
    # two edges labelled A-B meeting at an A vertex cannot stand for two
    # A-B edges meeting at a B vertex
    g2 = H.graph(3, [(0, 1), (0, 2)], [0, 1, 1], [0, 0])
    G2 = og(g2)
    assert oracle.count_edge(G2, H.query(3, [(0, 1), (0, 2)], [0, 1, 1], [0, 0]))[0] == 2
    assert oracle.count_edge(G2, H.query(3, [(0, 1), (0, 2)], [1, 0, 0], [0, 0]))[0] == 0


def test_vertex_embeddings_induce_edge_matches():
    """For a connected query with at least three vertices, each embedding f
    gives the edge match h(ab) = f(a)f(b), and distinct f give distinct h."""
    rng = np.random.default_rng(4400)
    for case in range(40):
        g = H.random_graph(rng, 9, float(rng.uniform(0.2, 0.6)), int(rng.integers(1, 3)), int(rng.integers(1, 3)))
        if g.m == 0:
            continue
        k = int(rng.integers(3, 5))
        q = H.random_connected_query(rng, k, int(rng.integers(0, 2)), int(rng.integers(1, 3)),
                                     int(rng.integers(1, 3)))
        G = og(g)
        ids = {frozenset((int(a), int(b))): i for i, (a, b) in enumerate(zip(g.src, g.dst))}
        emb = oracle.enumerate_rows(G, q)
        induced = {tuple(ids[frozenset((int(f[a]), int(f[b])))] for a, b in zip(q.src, q.dst)) for f in emb}
        assert len(induced) == emb.shape[0]
        edge_rows = {tuple(r) for r in oracle.enumerate_edge_rows(G, q).tolist()}
        assert induced <= edge_rows, case


def test_edge_invalid_queries():
    g = H.complete(4)
    G = og(g)
    with pytest.raises(ValueError):
        oracle.count_edge(G, H.query(1, []))                       # no edge
    with pytest.raises(ValueError):
        oracle.count_edge(G, H.query(3, [(0, 1), (1, 0)]))         # repeated pair
