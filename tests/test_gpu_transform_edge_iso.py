"""Edge isomorphism (Sec. VII-A) on the GPU: the line graph built by the
library, matched by the ordinary path, against the oracle's edge mode (which
works on G itself) and closed forms."""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1906_03420_gb300 as p
    p.load()
    torch.cuda.init()
    return p


def og(g):
    return oracle.OracleGraph(g.vlab, g.src, g.dst, g.elab)


@pytest.mark.parametrize("seed", range(4))
def test_edge_matches_equal_oracle(pkg, seed):
    """Random labelled graphs; queries cut out of G and random ones: rows
    (data edge ids per query edge) equal the oracle's, on the device-driven
    and the host-driven path, and count-only counts agree."""
    rng = np.random.default_rng(800 + seed)
    for case in range(12):
        g = H.random_graph(rng, int(rng.integers(20, 80)), float(rng.uniform(0.05, 0.25)), int(rng.integers(1, 3)),
                           int(rng.integers(1, 3)))
        if g.m < 2:
            continue
        if case % 2 == 0:
            q = H.extracted_query(rng, g, int(rng.integers(2, 6)))
        else:
            q = H.random_connected_query(rng, int(rng.integers(2, 6)), int(rng.integers(0, 2)),
                                         int(rng.integers(1, 3)), int(rng.integers(1, 3)))
        if q is None or len(q.src) == 0:
            continue
        E = pkg.EdgeGraph(g.vlab, g.src, g.dst, g.elab)
        want = oracle.enumerate_edge_rows(og(g), q)
        for host_driven in (False, True):
            r = E.query(q, host_driven=host_driven)
            assert r.count == want.shape[0], (seed, case, host_driven)
            assert r.k == len(q.src)
            assert np.array_equal(oracle.sort_rows(r.rows()), want), (seed, case, host_driven)
        assert E.query(q, count_only=True).count == want.shape[0]


def test_edge_closed_forms_on_rmat(pkg):
    """Unlabelled R-MAT graph (2^11 vertices, 8,000 edges): one edge -> m;
    2-path -> sum deg(deg-1); 3-star and triangle -> 6 (sum C(deg,3) +
    triangles); 3-path -> sum over edges of a(a-1), a = deg(x) + deg(y) - 2."""
    import scipy.sparse as sp
    s, d = synth.rmat(71, 11, 8_000)
    n = 1 << 11
    g = H.G(np.zeros(n, np.int32), s, d, np.zeros(s.shape[0], np.int32))
    E = pkg.EdgeGraph(g.vlab, g.src, g.dst, g.elab)
    deg = np.bincount(np.concatenate([g.src, g.dst]), minlength=n).astype(np.int64)
    A = sp.coo_matrix((np.ones(2 * g.m, np.int64), (np.concatenate([g.src, g.dst]), np.concatenate([g.dst, g.src]))),
                      shape=(n, n)).tocsr()
    tri = int((A @ A).multiply(A).sum()) // 6
    count = lambda q: E.query(q, count_only=True).count
    assert count(H.path_query(2)) == g.m
    assert count(H.path_query(3)) == int((deg * (deg - 1)).sum())
    three = 6 * (sum(math.comb(int(x), 3) for x in deg) + tri)
    assert count(H.star_query(3)) == three
    assert count(H.clique_query(3)) == three
    a = deg[g.src] + deg[g.dst] - 2
    assert count(H.path_query(4)) == int((a * (a - 1)).sum())


def test_edge_batch_equals_single_queries(pkg):
    """Edge queries as one batch on the line graph equal one-at-a-time runs."""
    rng = np.random.default_rng(900)
    g = H.random_graph(rng, 60, 0.12, 2, 2)
    E = pkg.EdgeGraph(g.vlab, g.src, g.dst, g.elab)
    qs = [q for q in (H.extracted_query(rng, g, int(rng.integers(2, 5))) for _ in range(24))
          if q is not None and len(q.src) > 0]
    res = E.batch(qs)
    O = og(g)
    for q, r in zip(qs, res):
        want = oracle.enumerate_edge_rows(O, q)
        assert r.count == want.shape[0]
        assert np.array_equal(oracle.sort_rows(r.rows()), want)


def test_edge_query_semantics_and_row_cap(pkg):
    """Row cap keeps the count exact; edge queries take isomorphism semantics only."""
    import ctypes
    g = H.complete(6)
    E = pkg.EdgeGraph(g.vlab, g.src, g.dst, g.elab)
    full = E.query(H.path_query(3))
    assert full.count == 6 * 5 * 4                       # ordered pairs of adjacent edges: sum_v deg(deg-1)
    capped = E.query(H.path_query(3), row_cap=10)
    assert capped.count == full.count and capped.rows().shape[0] == 10
    o = pkg.gsi.c_query_opts()
    o.semantics = pkg.GSI_HOMOMORPHISM
    q = pkg.QueryArrays.of(H.path_query(3))
    h = pkg.gsi.VP()
    rc = pkg.load().gsi_edge_query_run(E._h, pkg.gsi._p32(q.vlab), q.k, pkg.gsi._p32(q.src), pkg.gsi._p32(q.dst),
                                       pkg.gsi._p32(q.elab), q.qm, ctypes.byref(o), ctypes.byref(h))
    assert rc == pkg.GSI_EINVAL


def test_edge_workload_full_size(pkg):
    """The edge workload the benchmark times: ER 2^20 / 4M edges (line graph
    4M vertices, about 30.5M edges), 100 walk queries of 4..8 vertices asked
    as edge-isomorphism queries, one at a time.  Every query's count and
    full-set fingerprint equal the oracle's, which enumerates on G itself."""
    g = synth.workload_graph("edge")
    assert g.n == 1 << 20 and g.m == 4_000_000
    E = pkg.EdgeGraph.from_synth(g)
    O = og(g)
    for i, q in enumerate(synth.queries("edge")):
        want, fp = oracle.count_edge(O, q)
        r = E.query(q)
        assert r.count == want, i
        rows = r.rows()
        assert rows.shape == (want, len(q.src)), i
        assert oracle.fingerprint(rows) == (want, fp[1], fp[2]), i
        r.close()
