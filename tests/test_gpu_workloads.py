"""The medium, batched and served configurations at full size, in the launch
configurations the benchmark times.

- medium: R-MAT 2^20 vertices / 16M edges, 64 Zipf vertex labels, 8 edge
  labels, 100 walk queries of 6..12 vertices, one at a time on the plain path.
  Every query's count and full-set fingerprint equal the oracle's, computed
  once on the CPU into tests/golden/medium_counts.json.
- batched: the same graph, 4,096 walk queries of 4..16 vertices (rare-label
  walks from 8 vertices) as one prepared batch replayed from its captured
  CUDA graph: every count equals the plain path's, and a seeded 256-query
  sample equals the oracle (counts and full-set fingerprints).
- served: the 2^22 graph; the first 256 arrivals through a continuous-
  batching server equal the plain path, a 32-query sample the oracle.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

ROW_SAMPLE = 50_000


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
def medium(pkg):
    g = synth.workload_graph("medium")
    G = pkg.Graph.from_synth(g)
    O = oracle.OracleGraph.from_synth(g)
    a = np.minimum(g.src, g.dst).astype(np.int64)
    b = np.maximum(g.src, g.dst).astype(np.int64)
    key = a * g.n + b
    order = np.argsort(key, kind="stable")
    return g, G, O, key[order], g.elab[order]


def check_rows(g, q, rows, keys, labs):
    """Every row is an embedding (labels, injectivity, every query edge with
    its label) and no row repeats."""
    if rows.shape[0] == 0:
        return
    assert (g.vlab[rows] == np.asarray(q.vlab)[None, :]).all()
    s = np.sort(rows, axis=1)
    assert (s[:, 1:] != s[:, :-1]).all()
    for e in range(len(q.src)):
        u, v, lab = int(q.src[e]), int(q.dst[e]), int(q.elab[e])
        a = np.minimum(rows[:, u], rows[:, v]).astype(np.int64)
        b = np.maximum(rows[:, u], rows[:, v]).astype(np.int64)
        k = a * g.n + b
        idx = np.minimum(np.searchsorted(keys, k), keys.shape[0] - 1)
        assert (keys[idx] == k).all() and (labs[idx] == lab).all()
    assert np.unique(rows, axis=0).shape[0] == rows.shape[0]


def oracle_sample(qs, n=8, max_bound=2e7):
    return [i for i, q in enumerate(qs) if q.bound <= max_bound][:n]


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FP_CHUNK = 1 << 22


def golden_counts(workload):
    """Per-query oracle counts and fingerprints written by
    tests/golden/make_counts.py (CPU oracle only)."""
    with open(os.path.join(GOLDEN, f"{workload}_counts.json")) as f:
        rec = json.load(f)
    return {q["index"]: q for q in rec["queries"]}


def result_fingerprint(r, k):
    """The oracle's order-independent fingerprint of a whole result: rows are
    copied device to device, then fingerprinted on the host chunk by chunk
    (the fingerprint's sum and xor combine over chunks)."""
    import torch
    c = r.count
    buf = torch.empty((max(c, 1), k), dtype=torch.int32, device="cuda")
    rows, _ = r.copy_to(buf.data_ptr(), c)
    s = x = 0
    for a in range(0, rows, FP_CHUNK):
        n, s1, x1 = oracle.fingerprint(buf[a:a + FP_CHUNK].cpu().numpy())
        s = (s + s1) % (1 << 64)
        x ^= x1
    first = buf[:min(rows, ROW_SAMPLE)].cpu().numpy()
    del buf
    return rows, s, x, first


def test_medium_plain_path_full_size(pkg, medium):
    """Every one of the 100 queries: exact count and full-set fingerprint
    equal to the oracle's (tests/golden/medium_counts.json), and the first
    rows satisfy the definition."""
    g, G, O, keys, labs = medium
    assert g.n == 1 << 20 and g.m == 16_000_000
    qs = synth.queries("medium")
    want = golden_counts("medium")
    assert sorted(want) == list(range(len(qs)))
    for i, q in enumerate(qs):
        assert want[i]["k"] == q.k and want[i]["edges"] == q.qm
        r = G.query(q)
        c = r.count
        assert c == want[i]["count"], i
        rows, s, x, first = result_fingerprint(r, q.k)
        assert rows == c
        assert (c, s, x) == tuple(int(v) for v in want[i]["fingerprint"]), i
        check_rows(g, q, first, keys, labs)
        r.close()


def test_medium_results_kept_alive(pkg, medium):
    """Results keep their table region while a quarter of the device's memory
    allows, then move to tight copies: 24 results of the medium workload held
    at once (more than that allowance holds), each one's count and full-set
    fingerprint equal to the oracle's after all were made."""
    g, G, O, keys, labs = medium
    qs = synth.queries("medium")
    want = golden_counts("medium")
    small = sorted((i for i in range(len(qs)) if 0 < want[i]["count"] * qs[i].k * 4 < 1 << 30),
                   key=lambda i: want[i]["count"])[:24]
    assert len(small) == 24
    held = [(i, G.query(qs[i])) for i in small]
    for i, r in held:
        assert r.count == want[i]["count"], i
        rows, s, x, _ = result_fingerprint(r, qs[i].k)
        assert (rows, s, x) == tuple(int(v) for v in want[i]["fingerprint"]), i
    for _, r in held:
        r.close()


def test_medium_tight_rows(pkg, medium):
    """gsi_query_opts.tight_rows (the bench's end-to-end loop): the rows move
    to a buffer of their own size, large results included; ten medium
    queries, count and full-set fingerprint against the oracle's."""
    g, G, O, keys, labs = medium
    qs = synth.queries("medium")
    want = golden_counts("medium")
    for i in range(5, len(qs), 10):
        r = G.query(qs[i], tight_rows=True)
        assert r.count == want[i]["count"], i
        rows, s, x, _ = result_fingerprint(r, qs[i].k)
        assert (rows, s, x) == tuple(int(v) for v in want[i]["fingerprint"]), i
        r.close()


def test_medium_without_duplicate_removal(pkg, medium):
    """The join without duplicate removal (gsi_query_opts.no_dedup, the
    bench's --no-dedup line) gives the same sets: ten medium queries, count
    and full-set fingerprint against the oracle's."""
    g, G, O, keys, labs = medium
    qs = synth.queries("medium")
    want = golden_counts("medium")
    for i in range(0, len(qs), 10):
        r = G.query(qs[i], no_dedup=True)
        assert r.count == want[i]["count"], i
        rows, s, x, _ = result_fingerprint(r, qs[i].k)
        assert (rows, s, x) == tuple(int(v) for v in want[i]["fingerprint"]), i
        r.close()


def test_batched_prepared_batch_full_size(pkg, medium):
    g, G, O, keys, labs = medium
    qs = synth.queries("batched")
    assert len(qs) == 4096
    pb = pkg.PreparedBatch(G, qs)
    assert list(pb.statuses) == [0] * len(qs)
    res = pb.run()
    counts = [r.count for r in res]
    assert counts == [G.query(q, count_only=True).count for q in qs]     # every query: batch == plain path
    rng = np.random.default_rng(2004)
    for i in sorted(rng.choice(len(qs), 256, replace=False).tolist()):
        want, fp = oracle.count(O, qs[i])
        assert counts[i] == want, i
        assert oracle.fingerprint(res[i].rows()) == (want, fp[1], fp[2]), i
    for i in range(0, len(qs), 97):                                       # the definition on other queries
        check_rows(g, qs[i], res[i].rows(max_rows=ROW_SAMPLE), keys, labs)
    pb.close()


def test_served_full_size(pkg):
    """Served configuration: R-MAT 2^22 vertices / 64M edges, 128 Zipf vertex
    labels, 8 edge labels; the first 256 queries of the arrival stream all
    submitted to a continuous-batching server (2 slots, 40 GB budget, as the
    benchmark).  Every result equals the plain path's; a seeded 32-query
    sample equals the oracle (counts and full-set fingerprints)."""
    g = synth.workload_graph("served")
    assert g.n == 1 << 22 and g.m == 64_000_000
    G = pkg.Graph.from_synth(g)
    qs = synth.queries("served", 256)
    S = pkg.Server(G, mem_budget=40 << 30, n_streams=2, max_batch=0)
    tickets = [S.submit(q) for q in qs]
    served = []
    for t in tickets:
        r, lat = S.poll(t, -1)
        assert lat >= 0
        served.append(r)
    S.close()
    assert [r.count for r in served] == [G.query(q, count_only=True).count for q in qs]
    O = oracle.OracleGraph.from_synth(g)
    rng = np.random.default_rng(2005)
    for i in sorted(rng.choice(len(qs), 32, replace=False).tolist()):
        want, fp = oracle.count(O, qs[i])
        assert served[i].count == want, i
        assert oracle.fingerprint(served[i].rows()) == (want, fp[1], fp[2]), i
