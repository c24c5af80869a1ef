"""Seeded input generators: determinism and structural validity (no method arithmetic)."""
import numpy as np

import oracle
import synth


def test_er_graph_is_simple_and_deterministic():
    g = synth.graph("er1k")
    assert g.n == 1000 and g.m == 5000
    assert (g.src < g.dst).all()
    keys = g.src.astype(np.int64) * g.n + g.dst
    assert np.unique(keys).shape[0] == g.m
    s2, d2 = synth.erdos_renyi(1001, 1000, 5000)
    assert np.array_equal(s2, g.src) and np.array_equal(d2, g.dst)
    assert g.vlab.min() >= 0 and g.vlab.max() <= 3 and g.elab.max() <= 3


def test_rmat_small_is_simple():
    s, d = synth.rmat(5, 12, 20000)
    assert (s < d).all() and s.min() >= 0 and d.max() < 4096
    keys = s.astype(np.int64) * 4096 + d
    assert np.unique(keys).shape[0] == 20000
    s2, d2 = synth.rmat(5, 12, 20000)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)


def test_zipf_shares():
    lab = synth.labels_zipf(1, 1, 200000, 64, 1.1)
    h = sum(1 / (i ** 1.1) for i in range(1, 65))
    assert abs((lab == 0).mean() - 1 / h) < 0.01
    assert lab.max() < 64


def test_shape_queries_are_occurrences():
    g = synth.graph("er1k")
    og = oracle.OracleGraph.from_synth(g)
    for i, q in enumerate(synth.queries("tiny")):
        assert q.k == 4
        occ = q.occurrence
        assert len(set(occ.tolist())) == 4
        assert (g.vlab[occ] == q.vlab).all()
        for a, b, l in zip(q.src, q.dst, q.elab):
            assert og.edge_label(int(occ[a]), int(occ[b])) == l
        assert oracle.count(og, q)[0] >= 1


def test_walk_query_small_graph():
    s, d = synth.rmat(9, 10, 6000)
    g = synth.make_graph(synth.labels_zipf(9, 1, 1024, 8), s, d, synth.labels_uniform(9, 2, 6000, 3), 3)
    og = oracle.OracleGraph.from_synth(g)
    for i in range(10):
        q = synth.walk_query(g, 77, i, 5, dense=bool(i % 2), max_bound=1e6)
        assert q.k == 5 and q.qm >= 4 and q.bound <= 1e6
        occ = q.occurrence
        for a, b, l in zip(q.src, q.dst, q.elab):
            assert og.edge_label(int(occ[a]), int(occ[b])) == l
        c = oracle.count(og, q)[0]
        assert 1 <= c <= q.bound
