"""Batched execution (one persistent launch over a queue of (query, seed-range)
items) against the plain per-query path and the oracle."""
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


@pytest.fixture(scope="module")
def world(pkg):
    s, d = synth.rmat(41, 13, 70_000)
    n = 1 << 13
    g = H.G(synth.labels_zipf(41, 1, n, 8, 1.1), s, d, synth.labels_uniform(41, 2, 70_000, 3))
    sg = synth.make_graph(g.vlab, g.src, g.dst, g.elab, 3)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    O = oracle.OracleGraph(g.vlab, g.src, g.dst, g.elab)
    qs = [synth.walk_query(sg, 90, i, 3 + i % 5, dense=bool(i % 2), max_bound=1e6) for i in range(48)]
    return g, G, O, qs


def test_batch_matches_oracle(pkg, world):
    g, G, O, qs = world
    res = G.batch(qs)
    assert len(res) == len(qs)
    for q, r in zip(qs, res):
        want = oracle.enumerate_rows(O, q)
        assert r.count == want.shape[0]
        assert np.array_equal(oracle.sort_rows(r.rows()), want)


def test_batch_equals_plain_alone_and_in_mix(pkg, world):
    """Each query's result is the same alone (plain path) and inside a batch."""
    g, G, O, qs = world
    rng = np.random.default_rng(3)
    order = rng.permutation(len(qs))
    mixed = [qs[i] for i in order]
    res = G.batch(mixed)
    for i, r in zip(order, res):
        alone = G.query(qs[i])
        assert r.count == alone.count
        assert np.array_equal(oracle.sort_rows(r.rows()), oracle.sort_rows(alone.rows()))


def test_batch_statuses_and_empty_queries(pkg, world):
    g, G, O, qs = world
    bad = H.query(3, [(0, 1)])                       # disconnected
    absent_v = H.query(2, [(0, 1)], [999, 0], [0])  # vertex label not in G
    absent_e = H.query(2, [(0, 1)], [0, 0], [99])   # edge label not in G
    single = H.query(1, [], [int(g.vlab[0])], [])
    res = G.batch([qs[0], bad, absent_v, absent_e, single, qs[1]])
    assert isinstance(res[1], pkg.GsiError) and res[1].status == pkg.GSI_EINVAL
    assert res[2].count == 0 and res[3].count == 0
    assert res[4].count == int((g.vlab == g.vlab[0]).sum())
    assert res[0].count == oracle.count(O, qs[0])[0]
    assert res[5].count == oracle.count(O, qs[1])[0]


def test_batch_count_only_and_row_cap(pkg, world):
    g, G, O, qs = world
    counts = [oracle.count(O, q)[0] for q in qs[:16]]
    res = G.batch(qs[:16], count_only=True)
    assert [r.count for r in res] == counts
    assert all(r.rows().shape[0] == 0 for r in res)
    res = G.batch(qs[:16], row_cap=5)
    for q, r, c in zip(qs[:16], res, counts):
        assert r.count == c
        rows = r.rows()
        assert rows.shape[0] == min(5, c)
        want = {tuple(x) for x in oracle.enumerate_rows(O, q)}
        assert all(tuple(x) in want for x in rows)
        assert np.unique(rows, axis=0).shape[0] == rows.shape[0]


def test_batch_small_budget_falls_back(pkg, world):
    """A budget too small for some items: those queries run again on the plain path."""
    g, G, O, qs = world
    st = pkg.c_stats()
    res = G.batch(qs[:24], mem_budget=64 << 20, stats=st)
    for q, r in zip(qs[:24], res):
        want = oracle.enumerate_rows(O, q)
        assert r.count == want.shape[0]
        assert np.array_equal(oracle.sort_rows(r.rows()), want)


def test_batch_tiny_budget_runs_everything_on_the_plain_path(pkg, world):
    g, G, O, qs = world
    st = pkg.c_stats()
    res = G.batch(qs[:6], mem_budget=2 << 20, stats=st)
    for q, r in zip(qs[:6], res):
        assert r.count == oracle.count(O, q)[0]
    assert st.host_driven >= 1


def test_batch_results_outlive_each_other(pkg, world):
    """Results of one batch share an arena; destroying some keeps the others valid."""
    g, G, O, qs = world
    res = G.batch(qs[:10])
    keep = res[7]
    want = oracle.enumerate_rows(O, qs[7])
    for i, r in enumerate(res):
        if i != 7:
            r.close()
    del res
    assert np.array_equal(oracle.sort_rows(keep.rows()), want)


def test_batch_autotune_and_item_sizes(pkg, world):
    """The autotuner returns one of its candidate sizes; every item size gives the same results."""
    g, G, O, qs = world
    best, rows, ms = pkg.batch_autotune(G, qs[:16])
    assert best in (32, 64, 128) and rows in (512, 1024, 2048) and ms > 0
    ref = [oracle.count(O, q)[0] for q in qs[:16]]
    for spi in (1, 7, 32, 4096):
        res = G.batch(qs[:16], seeds_per_item=spi)
        assert [r.count for r in res] == ref
    # splitting: units that grow past item_rows rows hand pieces to other
    # CTAs; the results are the same with tiny, default and no splitting
    units = {}
    for ir in (-1, 0, 64, 7):
        st = pkg.c_stats()
        res = G.batch(qs[:16], item_rows=ir, stats=st)
        assert [r.count for r in res] == ref
        for q, r in zip(qs[:4], res[:4]):
            assert np.array_equal(oracle.sort_rows(r.rows()), oracle.sort_rows(G.query(q).rows()))
        units[ir] = st.tiles
    assert units[7] > units[-1] and units[64] > units[-1]


def test_batch_filter_many_query_vertices(pkg, world):
    """A batch with more query vertices than the filter's shared-memory
    counters hold (> 24,576) counts through global atomics; counts and sets
    still match the plain path on a sample."""
    g, G, O, qs = world
    big = [qs[i % len(qs)] for i in range(6200)]          # about 31,000 query vertices
    assert sum(len(np.asarray(q.vlab)) for q in big) > 24576
    res = G.batch(big, count_only=True)
    ref = [G.query(q, count_only=True).count for q in qs]
    for i in range(0, len(big), 97):
        assert res[i].count == ref[i % len(qs)]


def test_prepared_batch_replays(pkg, world):
    """A prepared batch replayed from its captured graph gives the oracle's
    sets on every replay; results outlive later replays and the batch."""
    import torch
    g, G, O, qs = world
    want = [oracle.enumerate_rows(O, q) for q in qs[:24]]
    s = torch.cuda.Stream()
    for stream in (None, s):
        pb = pkg.PreparedBatch(G, qs[:24], stream=stream, counters=True)
        assert list(pb.statuses) == [0] * 24
        first = pb.run()
        for _ in range(2):
            st = pkg.c_stats()
            again = pb.run(stats=st)
            assert st.join_launches == 1 and st.filter_launches == 1 and st.join_bytes > 0
            for r, w in zip(again, want):
                assert np.array_equal(oracle.sort_rows(r.rows()), w)
        pb.close()
        for r, w in zip(first, want):                      # still valid
            assert r.count == w.shape[0]
            assert np.array_equal(oracle.sort_rows(r.rows()), w)


def test_prepared_batch_statuses_caps_and_small_budget(pkg, world):
    g, G, O, qs = world
    bad = H.query(3, [(0, 1)])                               # disconnected
    mix = [qs[0], bad, qs[1]]
    pb = pkg.PreparedBatch(G, mix)
    assert list(pb.statuses) == [0, pkg.GSI_EINVAL, 0]
    res = pb.run()
    assert isinstance(res[1], pkg.GsiError) and res[1].status == pkg.GSI_EINVAL
    assert res[0].count == oracle.count(O, qs[0])[0] and res[2].count == oracle.count(O, qs[2 - 1])[0]
    pb.close()
    ref = [oracle.count(O, q)[0] for q in qs[:12]]
    pb = pkg.PreparedBatch(G, qs[:12], count_only=True)
    assert [r.count for r in pb.run()] == ref
    pb.close()
    pb = pkg.PreparedBatch(G, qs[:12], row_cap=5)
    for r, c in zip(pb.run(), ref):
        assert r.count == c and r.rows().shape[0] == min(5, c)
    pb.close()
    pb = pkg.PreparedBatch(G, qs[:12], mem_budget=1 << 20)  # no slice fits: every query on the plain path
    assert [r.count for r in pb.run()] == ref
    pb.close()


@pytest.fixture(scope="module")
def dense_world(pkg):
    """Dense walk queries (|E| up to 2k) on a small R-MAT graph: most join
    steps have two or more linking edges, so short rows go through the
    intersection strategies."""
    s, d = synth.rmat(43, 12, 40_000)
    n = 1 << 12
    g = H.G(synth.labels_zipf(43, 1, n, 8, 1.1), s, d, synth.labels_uniform(43, 2, 40_000, 3))
    sg = synth.make_graph(g.vlab, g.src, g.dst, g.elab, 3)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    O = oracle.OracleGraph(g.vlab, g.src, g.dst, g.elab)
    qs = [synth.walk_query(sg, 92, i, 5 + i % 4, dense=True, max_bound=1e6) for i in range(24)]
    assert sum(q.qm > q.k for q in qs) >= 10
    wants = [oracle.enumerate_rows(O, q) for q in qs]
    return G, qs, wants


@pytest.mark.parametrize("isect", [0, 1, 2])
@pytest.mark.parametrize("block_threads,rows_per_thread", [(256, 2), (256, 1), (128, 2), (128, 1)])
def test_batch_knobs_give_the_oracle_sets(pkg, dense_world, isect, block_threads, rows_per_thread):
    """Every intersection strategy (binary search, merge, candidate-position
    bitmap) under every block shape of the batch kernel gives the oracle's
    embedding sets."""
    G, qs, wants = dense_world
    res = G.batch(qs, isect=isect, rows_per_thread=rows_per_thread, block_threads=block_threads)
    assert sum(w.shape[0] > 0 for w in wants) >= 20
    for q, r, want in zip(qs, res, wants):
        assert r.count == want.shape[0]
        assert np.array_equal(oracle.sort_rows(r.rows()), want)


def test_batch_knobs_rejected_when_invalid(pkg, world):
    g, G, O, qs = world
    for kw in ({"block_threads": 64}, {"rows_per_thread": 3}, {"isect": 7}):
        with pytest.raises(pkg.GsiError) as e:
            G.batch(qs[:2], **kw)
        assert e.value.status == pkg.GSI_EINVAL


def test_full_autotuner_returns_a_valid_setting(pkg, dense_world):
    G, qs, wants = dense_world
    best = pkg.batch_autotune_full(G, qs)
    assert best["seeds_per_item"] in (32, 64, 128) and best["item_rows"] in (512, 1024, 2048)
    assert best["isect"] in (0, 1, 2) and best["rows_per_thread"] in (1, 2) and best["block_threads"] in (128, 256)
    assert best["ms"] > 0 and best["trials"] >= 2 * 10
    res = G.batch(qs, **{k: best[k] for k in ("seeds_per_item", "item_rows", "isect", "rows_per_thread",
                                              "block_threads")})
    assert [r.count for r in res] == [w.shape[0] for w in wants]
