"""The scale configuration at full size: R-MAT 2^24 vertices / 256M undirected
edges, 256 Zipf vertex labels, 16 edge labels, 20 random-walk queries of 8..16
vertices, at most 10^9 rows kept per query with exact counts.

Too large for the oracle to enumerate every query, so parity is checked by what
holds at any size: a closed form (labelled stars, counted per vertex from the
edge list), the definition checked on materialised rows (labels, injectivity,
every query edge present with its label, no duplicates), the count's
independence of the join order, the admission bound, and the oracle's own count
on the queries it finishes in seconds."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SAMPLE_ROWS = 200_000


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
def scale(pkg):
    w = synth.WORKLOADS["scale"]
    g = synth.workload_graph("scale")
    qs = synth.queries("scale")
    G = pkg.Graph.from_synth(g)
    a = np.minimum(g.src, g.dst).astype(np.int64)
    b = np.maximum(g.src, g.dst).astype(np.int64)
    key = a * g.n + b
    order = np.argsort(key, kind="stable")
    return w, g, G, qs, key[order], g.elab[order]


def check_rows(g, q, rows, keys, labs):
    """Every row is an embedding (Def. 2-3 as read here) and no row repeats."""
    assert (g.vlab[rows] == np.asarray(q.vlab)[None, :]).all()
    s = np.sort(rows, axis=1)
    assert (s[:, 1:] != s[:, :-1]).all()                       # injective
    for e in range(q.qm):
        u, v, lab = int(q.src[e]), int(q.dst[e]), int(q.elab[e])
        a = np.minimum(rows[:, u], rows[:, v]).astype(np.int64)
        b = np.maximum(rows[:, u], rows[:, v]).astype(np.int64)
        k = a * g.n + b
        idx = np.minimum(np.searchsorted(keys, k), keys.shape[0] - 1)
        assert (keys[idx] == k).all()                          # the edge exists
        assert (labs[idx] == lab).all()                        # with the query's label
    assert np.unique(rows, axis=0).shape[0] == rows.shape[0]


def bfs_order(q, start):
    adj = {u: set() for u in range(q.k)}
    for a, b in zip(q.src, q.dst):
        adj[int(a)].add(int(b))
        adj[int(b)].add(int(a))
    order, seen = [start], {start}
    i = 0
    while i < len(order):
        for w in sorted(adj[order[i]]):
            if w not in seen:
                seen.add(w)
                order.append(w)
        i += 1
    return order


def test_scale_workload_counts_rows_and_orders(pkg, scale):
    w, g, G, qs, keys, labs = scale
    assert g.n == 1 << 24 and g.m == 256_000_000
    for q in qs:
        r = G.query(q, row_cap=w.row_cap)
        c = r.count
        assert c <= q.bound * (1 + 1e-9) + 1                   # the spanning-tree bound caps the count
        kept = min(c, w.row_cap)
        rows = r.rows(max_rows=SAMPLE_ROWS)
        assert rows.shape[0] == min(kept, SAMPLE_ROWS)
        if rows.shape[0]:
            check_rows(g, q, rows, keys, labs)
        r.close()
        # another connected join order gives the same count
        alt = bfs_order(q, q.k - 1)
        assert G.query(q, count_only=True, order=alt).count == c


def test_scale_oracle_counts_on_small_queries(pkg, scale):
    w, g, G, qs, keys, labs = scale
    small = [q for q in qs if q.bound <= 5e5]
    assert small
    O = oracle.OracleGraph.from_synth(g)
    for q in small:
        want, fp = oracle.count(O, q)
        r = G.query(q)
        assert r.count == want
        assert oracle.fingerprint(r.rows()) == (want, fp[1], fp[2])


def test_scale_labelled_star_closed_form(pkg, scale):
    """Star with centre label c and leaves (edge label e_i, leaf label l_i):
    sum over vertices v with label c of the product, over distinct leaf keys,
    of the falling factorial (count of v's neighbours with that key) over the
    key's multiplicity."""
    from tests import helpers as H
    w, g, G, qs, keys, labs = scale
    deg = np.bincount(g.src, minlength=g.n) + np.bincount(g.dst, minlength=g.n)
    rng = np.random.default_rng(7)
    done = 0
    for attempt in range(40):
        if done == 3:
            break
        s = 2 + done % 2
        v0 = int(rng.choice(np.flatnonzero(deg >= 8)))
        m_nb = (g.src == v0) | (g.dst == v0)
        nb = np.where(g.src[m_nb] == v0, g.dst[m_nb], g.src[m_nb])
        el = g.elab[m_nb]
        pick = rng.choice(nb.shape[0], s, replace=False)
        leaf_keys = [(int(el[i]), int(g.vlab[nb[i]])) for i in pick]
        c_lab = int(g.vlab[v0])
        prod = np.ones(g.n, dtype=np.uint64)
        for key in sorted(set(leaf_keys)):
            mult = leaf_keys.count(key)
            e, l = key
            me = g.elab == e
            u, v = g.src[me], g.dst[me]
            cnt = (np.bincount(u[g.vlab[v] == l], minlength=g.n) +
                   np.bincount(v[g.vlab[u] == l], minlength=g.n)).astype(np.int64)
            ff = np.ones(g.n, dtype=np.int64)
            for j in range(mult):
                ff *= np.maximum(cnt - j, 0)
            prod *= ff.astype(np.uint64)
        want = int(sum(int(x) for x in prod[(g.vlab == c_lab) & (prod > 0)]))
        if want > 10**10:                                      # keep the enumeration to seconds
            continue
        edges = [(0, i + 1) for i in range(s)]
        q = H.query(s + 1, edges, vlab=[c_lab] + [k[1] for k in leaf_keys], elab=[k[0] for k in leaf_keys])
        assert G.query(q, count_only=True).count == want
        done += 1
    assert done == 3
