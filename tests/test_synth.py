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


def test_rare_label_walks_visit_only_rare_labels():
    """Rare-label walks (the batched and served workloads' queries of 8 or
    more vertices) start at and step to vertices labelled min_label or above
    only; the query is still an occurrence in G with its labels."""
    s, d = synth.rmat(9, 11, 16000)
    g = synth.make_graph(synth.labels_zipf(9, 1, 2048, 16), s, d, synth.labels_uniform(9, 2, 16000, 3), 3)
    og = oracle.OracleGraph.from_synth(g)
    for i in range(8):
        q = synth.walk_query(g, 78, i, 8, dense=bool(i % 2), max_bound=1e6, min_label=4)
        occ = q.occurrence
        assert len(set(occ.tolist())) == 8 and q.attempts >= 1
        assert (g.vlab[occ] >= 4).all() and (q.vlab >= 4).all()
        for a, b, l in zip(q.src, q.dst, q.elab):
            assert og.edge_label(int(occ[a]), int(occ[b])) == l
        c = oracle.count(og, q)[0]
        assert 1 <= c <= q.bound <= 1e6


def test_batched_and_served_sizes_span_4_to_16():
    for name in ("batched", "served"):
        w = synth.WORKLOADS[name]
        ks = [synth.drawn_size(w, i) for i in range(2000)]
        assert min(ks) == 4 and max(ks) == 16
    w = synth.WORKLOADS["served"]
    ks = [synth.drawn_size(w, i) for i in range(20000)]
    assert 7.0 < sum(ks) / len(ks) < 8.2          # geometric with mean 8, clipped at 16
