"""GPU parity: every stage of the CUDA path against the CPU oracle, through the C ABI.

Integer work throughout, so the bar is bit-exact: layouts and bitmaps equal
element by element, embedding sets equal as sorted row sets (the GPU emits rows
in atomic-reservation order, so only the set is unique).
"""
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


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bitmap_of(member: np.ndarray) -> np.ndarray:
    """bool[n] -> uint32 words, bit v of word v/32 (little-endian bit order)."""
    n = member.shape[0]
    words = (n + 31) // 32
    padded = np.zeros(words * 32, bool)
    padded[:n] = member
    return np.packbits(padded, bitorder="little").view(np.uint32)


def og(g):
    return oracle.OracleGraph(g.vlab, g.src, g.dst, g.elab)


def rmat_graph(seed, scale, m, nvl, nel):
    s, d = synth.rmat(seed, scale, m)
    n = 1 << scale
    return H.G(synth.labels_zipf(seed, 1, n, nvl, 1.1), s, d, synth.labels_uniform(seed, 2, m, nel))


# ------------------------------------------------------------------ layout
def expected_layout(g, L):
    """Entries sorted by (vertex, edge label, label rank of the neighbour, neighbour)."""
    uniq = np.unique(g.vlab)
    rank = np.searchsorted(uniq, g.vlab).astype(np.int64)
    v = np.concatenate([g.src, g.dst]).astype(np.int64)
    w = np.concatenate([g.dst, g.src]).astype(np.int64)
    l = np.concatenate([g.elab, g.elab]).astype(np.int64)
    idx = np.lexsort((w, rank[w], l, v))
    seg = v[idx] * L + l[idx]
    off = np.searchsorted(seg, np.arange(g.n * L + 1), side="left").astype(np.uint32)
    return off, w[idx].astype(np.int32), rank[w[idx]].astype(np.uint16)


@pytest.mark.parametrize("case", ["random", "er1k", "rmat14", "isolated"])
def test_layout_matches_oracle_adjacency(pkg, case):
    rng = np.random.default_rng(4)
    if case == "random":
        g = H.random_graph(rng, 60, 0.2, 5, 7)
    elif case == "er1k":
        g = synth.graph("er1k")
    elif case == "rmat14":
        g = rmat_graph(14, 14, 200_000, 16, 8)
    else:
        g = H.graph(10, [(0, 9), (3, 4)], vlab=list(range(10)), elab=[2, 0])
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    info = G.info()
    L = int(g.elab.max()) + 1 if g.m else 1
    assert info.n == g.n and info.m == g.m and info.n_elabels == L
    off, ci, cl, sig = G.export()
    eoff, eci, ecl = expected_layout(g, L)
    assert info.n_vlabels == np.unique(g.vlab).shape[0]
    assert np.array_equal(off, eoff)
    assert np.array_equal(ci, eci)
    assert np.array_equal(cl, ecl)
    assert np.array_equal(sig.T, oracle.data_signatures(og(g)))
    assert np.array_equal(G.label_freq(), np.bincount(g.elab, minlength=L).astype(np.uint64))


@pytest.mark.parametrize("bad", ["self_loop", "dup_pair", "dup_pair_other_label", "id_range", "neg_label"])
def test_invalid_graphs_rejected(pkg, bad):
    edges = {"self_loop": ([0, 1], [1, 1], [0, 0]), "dup_pair": ([0, 1], [1, 0], [0, 0]),
             "dup_pair_other_label": ([0, 2], [2, 0], [0, 1]), "id_range": ([0], [5], [0]),
             "neg_label": ([0], [1], [-1])}[bad]
    with pytest.raises(pkg.GsiError) as e:
        pkg.Graph([0, 0, 0], *edges)
    assert e.value.status == pkg.GSI_EINVAL


def test_graph_without_edges(pkg):
    G = pkg.Graph([3, 3, 4], np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    r = G.query(H.query(1, [], [3], []))
    assert r.count == 2
    assert sorted(r.rows().ravel().tolist()) == [0, 1]
    assert G.query(H.query(2, [(0, 1)], [3, 3], [0])).count == 0


# ------------------------------------------------------------------ filter
@pytest.mark.parametrize("seed", range(3))
def test_filter_matches_oracle(pkg, seed):
    rng = np.random.default_rng(40 + seed)
    g = rmat_graph(100 + seed, 13, 60_000, 8, 4) if seed == 2 else H.random_graph(rng, 300, 0.05, 4, 3)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    O = og(g)
    sg = synth.make_graph(g.vlab, g.src, g.dst, g.elab, int(g.elab.max()) + 1)
    for i in range(12):
        q = synth.walk_query(sg, 9 + seed, i, int(rng.integers(1, 9)), dense=bool(i % 2))
        bm, cnt = G.filter(q)
        member, ocnt = oracle.filter_sets(O, q)
        assert np.array_equal(cnt.astype(np.int64), ocnt)
        for u in range(q.k):
            assert np.array_equal(bm[u], bitmap_of(member[u])), (i, u)


# --------------------------------------------------------------- join step
def _prefix_tables(O, g, q, order):
    """Oracle tables M_t along `order` (t = 1..k), filter sets as candidates."""
    member, _ = oracle.filter_sets(O, q)
    qadj = {}
    for a, b, l in zip(q.src, q.dst, q.elab):
        qadj[(int(a), int(b))] = qadj[(int(b), int(a))] = int(l)
    M = np.nonzero(member[order[0]])[0].astype(np.int32)[:, None]
    tables, steps = [M], []
    for t in range(1, q.k):
        u = order[t]
        cols = [c for c in range(t) if (order[c], u) in qadj]
        labs = [qadj[(order[c], u)] for c in cols]
        steps.append((u, cols, labs))
        M = oracle.join_step(O, M, member[u], cols, labs)
        tables.append(M)
    return member, tables, steps


def _gpu_step(pkg, G, M, member_u, ulabel, cols, labs, out_cap=None):
    import torch
    t = M.shape[1]
    R = M.shape[0]
    Md = dev(M if R else np.zeros((1, t), np.int32))
    cd = dev(bitmap_of(member_u).view(np.int32))
    cap = out_cap if out_cap is not None else max(1, R * 64)
    out = torch.full((max(cap, 1), t + 1), -7, dtype=torch.int32, device="cuda")
    cnt = G.join_step(Md.data_ptr(), R, t, cd.data_ptr(), int(ulabel), cols, labs, out.data_ptr(), cap)
    torch.cuda.synchronize()
    return cnt, out[: min(cnt, cap)].cpu().numpy()


@pytest.mark.parametrize("seed", range(4))
def test_join_step_matches_oracle(pkg, seed):
    """Alg. 3 step by step: same M, same C(u), same linking edges -> same M'."""
    rng = np.random.default_rng(70 + seed)
    g = rmat_graph(200 + seed, 12, 30_000, 8, 3)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    O = og(g)
    sg = synth.make_graph(g.vlab, g.src, g.dst, g.elab, int(g.elab.max()) + 1)
    checked = 0
    for i in range(10):
        q = synth.walk_query(sg, 50 + seed, i, int(rng.integers(3, 7)), dense=bool(i % 2), max_bound=1e6)
        order = oracle.order(q)
        member, tables, steps = _prefix_tables(O, g, q, list(order))
        for t, (u, cols, labs) in enumerate(steps, start=1):
            M = tables[t - 1]
            if M.shape[0] > 400_000:
                break
            # e0 may be any linking edge: rotate it
            rot = int(rng.integers(0, len(cols)))
            cols_r = cols[rot:] + cols[:rot]
            labs_r = labs[rot:] + labs[:rot]
            cnt, rows = _gpu_step(pkg, G, M, member[u], q.vlab[u], cols_r, labs_r)
            want = tables[t]
            assert cnt == want.shape[0]
            assert np.array_equal(oracle.sort_rows(rows), want)
            checked += 1
    assert checked >= 10


def test_join_step_skewed_hub(pkg):
    """A hub row whose candidate list spans many tiles, beside many one-candidate rows."""
    hub_deg = 50_000
    edges = [(0, i) for i in range(1, hub_deg + 1)]
    edges += [(i, i + 1) for i in range(1, hub_deg)]
    n = hub_deg + 1
    g = H.graph(n, edges, vlab=[0] * n, elab=[0] * len(edges))
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    O = og(g)
    # rows: the hub first, then a ragged number of leaf rows
    M = np.concatenate([[0], np.arange(1, 3001, dtype=np.int32)]).astype(np.int32)[:, None]
    everyone = np.ones(n, bool)
    cnt, rows = _gpu_step(pkg, G, M, everyone, 0, [0], [0], out_cap=hub_deg + 10_000)
    want = oracle.join_step(O, M, everyone, [0], [0])
    assert cnt == want.shape[0]
    assert np.array_equal(oracle.sort_rows(rows), want)
    # two-column rows (hub, leaf) extended by a vertex adjacent to both (a triangle closer)
    M2 = want[want[:, 0] == 0][:5000]
    cnt2, rows2 = _gpu_step(pkg, G, M2, everyone, 0, [0, 1], [0, 0])
    want2 = oracle.join_step(O, M2, everyone, [0, 1], [0, 0])
    assert cnt2 == want2.shape[0] and np.array_equal(oracle.sort_rows(rows2), want2)


def test_join_step_edge_cases(pkg):
    g = H.graph(6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (0, 5), (0, 2)], vlab=[0] * 6, elab=[0, 1, 0, 1, 0, 1, 0])
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    O = og(g)
    everyone = np.ones(6, bool)
    # empty M
    assert G.join_step(0, 0, 1, 0, 0, [0], [0], 0, 0) == 0
    # edge label beyond the graph's labels, or a vertex label no vertex has: no candidates
    M = np.arange(6, dtype=np.int32)[:, None]
    cnt, _ = _gpu_step(pkg, G, M, everyone, 0, [0], [5])
    assert cnt == 0
    cnt, _ = _gpu_step(pkg, G, M, everyone, 3, [0], [0])
    assert cnt == 0
    # rows with repeated values (injectivity applies to every column)
    M = np.array([[0, 0], [1, 1], [2, 0]], np.int32)
    cnt, rows = _gpu_step(pkg, G, M, everyone, 0, [1], [0])
    want = oracle.join_step(O, M, everyone, [1], [0])
    assert cnt == want.shape[0] and np.array_equal(oracle.sort_rows(rows), want)
    # out_cap smaller than the count: count exact, rows valid and distinct
    M = np.repeat(np.arange(6, dtype=np.int32), 40)[:, None]
    full = oracle.join_step(O, M, everyone, [0], [0])
    cnt, rows = _gpu_step(pkg, G, M, everyone, 0, [0], [0], out_cap=7)
    assert cnt == full.shape[0] and rows.shape[0] == 7
    fs = {tuple(r) for r in full}
    assert all(tuple(r) in fs for r in rows)
    # invalid arguments
    with pytest.raises(pkg.GsiError):
        G.join_step(0, 1, 1, 0, 0, [1], [0], 0, 0)     # column outside [0, t)
    with pytest.raises(pkg.GsiError):
        G.join_step(0, 1, 1, 0, 0, [0, 0], [0, 0], 0, 0)   # d > t


# ------------------------------------------------------------ full queries
def _check_query(pkg, G, O, q, **kw):
    r = G.query(q, **kw)
    want = oracle.enumerate_rows(O, q)
    assert r.count == want.shape[0]
    got = oracle.sort_rows(r.rows())
    assert np.array_equal(got, want)
    return r.count


def test_tiny_workload_full_sets(pkg):
    g = synth.graph("er1k")
    G = pkg.Graph.from_synth(g)
    O = oracle.OracleGraph.from_synth(g)
    for q in synth.queries("tiny"):
        assert _check_query(pkg, G, O, q) >= 1


@pytest.mark.parametrize("seed", range(6))
def test_random_small_queries_full_sets(pkg, seed):
    rng = np.random.default_rng(500 + seed)
    for _ in range(25):
        n = int(rng.integers(5, 40))
        g = H.random_graph(rng, n, float(rng.uniform(0.1, 0.6)), int(rng.integers(1, 4)), int(rng.integers(1, 3)))
        if g.m == 0:
            continue
        G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
        O = og(g)
        for _ in range(4):
            q = H.extracted_query(rng, g, int(rng.integers(1, 7)))
            if q is None:
                q = H.random_connected_query(rng, 3, 1, 2, 2)
            _check_query(pkg, G, O, q)


def test_closed_form_counts_on_gpu(pkg):
    """Clique in K_n: n!/(n-k)!;  triangle in C_n: 0;  path P_k in C_n: 2n."""
    import math
    G = pkg.Graph(*(lambda g: (g.vlab, g.src, g.dst, g.elab))(H.complete(9)))
    for k in range(1, 7):
        assert G.query(H.clique_query(k)).count == math.perm(9, k)
    C = pkg.Graph(*(lambda g: (g.vlab, g.src, g.dst, g.elab))(H.cycle(50)))
    assert C.query(H.clique_query(3)).count == 0
    for k in (2, 5, 9):
        assert C.query(H.path_query(k)).count == 100


def test_orders_give_same_result(pkg):
    """The result does not depend on the join order (three forced orders + Alg. 2)."""
    rng = np.random.default_rng(8)
    g = rmat_graph(31, 11, 12_000, 6, 3)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    O = og(g)
    sg = synth.make_graph(g.vlab, g.src, g.dst, g.elab, int(g.elab.max()) + 1)
    for i in range(6):
        q = synth.walk_query(sg, 3, i, 5, dense=bool(i % 2), max_bound=1e6)
        want = oracle.enumerate_rows(O, q)
        qadj = {(int(a), int(b)) for a, b in zip(q.src, q.dst)} | {(int(b), int(a)) for a, b in zip(q.src, q.dst)}
        for _ in range(3):
            order = [int(rng.integers(0, q.k))]
            while len(order) < q.k:
                cand = sorted({b for (a, b) in qadj if a in order and b not in order})
                order.append(int(rng.choice(cand)))
            r = G.query(q, order=order)
            assert r.count == want.shape[0]
            assert np.array_equal(oracle.sort_rows(r.rows()), want)


def test_memory_budget_splits_give_same_result(pkg):
    g = rmat_graph(32, 12, 40_000, 6, 3)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    O = og(g)
    sg = synth.make_graph(g.vlab, g.src, g.dst, g.elab, int(g.elab.max()) + 1)
    split_seen = False
    for i in range(4):
        q = synth.walk_query(sg, 4, i, 5, dense=False, max_bound=2e6)
        want = oracle.enumerate_rows(O, q)
        st = pkg.c_stats()
        budget = 1 << 20
        r = G.query(q, mem_budget=budget, stats=st, host_driven=True)
        assert r.count == want.shape[0]
        assert np.array_equal(oracle.sort_rows(r.rows()), want)
        assert st.peak_bytes <= budget
        split_seen = split_seen or st.tiles > q.k - 1
    assert split_seen


def test_device_driven_overflow_falls_back(pkg):
    """A budget too small for the device-driven arena's tables: the host-driven path takes over."""
    g = rmat_graph(34, 12, 40_000, 6, 3)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    O = og(g)
    sg = synth.make_graph(g.vlab, g.src, g.dst, g.elab, int(g.elab.max()) + 1)
    for i in range(3):
        q = synth.walk_query(sg, 6, i, 5, dense=False, max_bound=2e6)
        want = oracle.enumerate_rows(O, q)
        for budget in (1 << 18, 1 << 20, 1 << 30):
            r = G.query(q, mem_budget=budget)
            assert r.count == want.shape[0]
            assert np.array_equal(oracle.sort_rows(r.rows()), want)


def test_host_and_device_driven_agree(pkg):
    g = rmat_graph(35, 13, 80_000, 8, 3)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    sg = synth.make_graph(g.vlab, g.src, g.dst, g.elab, int(g.elab.max()) + 1)
    for i in range(8):
        q = synth.walk_query(sg, 7, i, int(4 + i % 5), dense=bool(i % 2), max_bound=5e6)
        a = G.query(q)
        b = G.query(q, host_driven=True)
        assert a.count == b.count
        assert np.array_equal(oracle.sort_rows(a.rows()), oracle.sort_rows(b.rows()))
        for cap in (1, 17):
            c = G.query(q, row_cap=cap)
            assert c.count == a.count and c.rows().shape[0] == min(cap, a.count)
        assert G.query(q, count_only=True).count == a.count


def test_budget_too_small_is_enomem(pkg):
    g = H.complete(30)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    with pytest.raises(pkg.GsiError) as e:
        G.query(H.path_query(3), mem_budget=64, host_driven=True)
    assert e.value.status == pkg.GSI_ENOMEM


def test_row_cap_and_count_only(pkg):
    g = H.complete(12)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    O = og(g)
    q = H.path_query(4)
    want = oracle.enumerate_rows(O, q)
    r = G.query(q, row_cap=1000)
    assert r.count == want.shape[0] == 11880
    rows = r.rows()
    assert rows.shape[0] == 1000
    assert np.unique(rows, axis=0).shape[0] == 1000
    ws = {tuple(x) for x in want}
    assert all(tuple(x) in ws for x in rows)
    r2 = G.query(q, count_only=True)
    assert r2.count == want.shape[0] and r2.rows().shape[0] == 0


def test_absent_labels_give_empty_results(pkg):
    g = H.graph(4, [(0, 1), (1, 2)], vlab=[0, 1, 0, 1], elab=[0, 1])
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    assert G.query(H.query(2, [(0, 1)], [0, 1], [7])).count == 0      # edge label absent
    assert G.query(H.query(2, [(0, 1)], [9, 1], [0])).count == 0      # vertex label absent
    assert G.query(H.query(1, [], [1], [])).count == 2


def test_invalid_query_rejected_before_gpu_work(pkg):
    g = H.complete(5)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    with pytest.raises(pkg.GsiError) as e:
        G.query(H.query(3, [(0, 1)]))
    assert e.value.status == pkg.GSI_EINVAL


def test_relabelling_invariance(pkg):
    """Permuting data-vertex ids permutes the result and nothing else."""
    rng = np.random.default_rng(12)
    g = rmat_graph(33, 10, 6000, 6, 3)
    perm = rng.permutation(g.n).astype(np.int32)
    g2 = H.G(g.vlab[np.argsort(perm)], perm[g.src], perm[g.dst], g.elab)
    G1 = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    G2 = pkg.Graph(g2.vlab, np.minimum(g2.src, g2.dst), np.maximum(g2.src, g2.dst), g2.elab)
    sg = synth.make_graph(g.vlab, g.src, g.dst, g.elab, int(g.elab.max()) + 1)
    for i in range(4):
        q = synth.walk_query(sg, 5, i, 5, dense=True, max_bound=1e6)
        a = oracle.sort_rows(G1.query(q).rows())
        b = oracle.sort_rows(np.argsort(perm).astype(np.int32)[G2.query(q).rows()])
        assert np.array_equal(a, b)


def test_worked_example_on_gpu(pkg):
    """The worked example of Secs. III-B and V (tests/golden): one join step from
    M = {(v0, v_i)} leaves (v0, v100, v201); the full query finds the single
    printed match."""
    facts, g, q = H.worked_example()
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    assert G.query(q).rows().tolist() == [facts["match"]]
    M = np.array([(0, i) for i in range(1, 101)], np.int32)
    cnt, rows = _gpu_step(pkg, G, M, g.vlab == 2, 2, [1, 0], [0, 1])   # linking edges u1u2:a, u0u2:b
    assert cnt == 1 and rows.tolist() == [[0, 100] + facts["buf99_final"]]


def test_shared_first_edge_rows_on_a_hub_graph(pkg):
    """Duplicate removal (Sec. VI-B) in the row pass: rows of a step that share
    their first-edge vertex share one sub-list lookup and one set of bitmap
    probes (warp groups found with __match_any_sync, and the per-step memo).
    On a graph of few hubs with hundreds of leaves each, nearly every warp
    holds such groups, mixed with rows of other vertices and with long rows
    (more than 16 candidates) that go to the slot tiles.  Counts and
    full-set fingerprints equal the oracle's; paths, stars and a triangle
    with a pendant, so both single- and multi-edge steps run."""
    rng = np.random.default_rng(606)
    n, hubs = 2400, 6
    edges = set()
    for h in range(hubs):
        for leaf in rng.choice(np.arange(hubs, n), 70, replace=False):
            edges.add((h, int(leaf)))
    while len(edges) < 9000:
        a, b = (int(x) for x in rng.integers(hubs, n, 2))
        if a != b:
            edges.add((min(a, b), max(a, b)))
    edges = sorted(edges)
    vlab = np.where(np.arange(n) < hubs, 0, 1 + rng.integers(0, 2, n)).astype(np.int32)
    elab = rng.integers(0, 2, len(edges)).astype(np.int32)
    g = H.graph(n, edges, vlab=vlab, elab=elab)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    O = oracle.OracleGraph(g.vlab, g.src, g.dst, g.elab)
    queries = [
        H.query(3, [(0, 1), (1, 2)], vlab=[1, 0, 1], elab=[0, 1]),                 # leaf-hub-leaf
        H.query(4, [(0, 1), (0, 2), (0, 3)], vlab=[0, 1, 2, 1], elab=[0, 0, 1]),   # hub star
        H.query(4, [(0, 1), (1, 2), (2, 3)], vlab=[2, 0, 1, 2], elab=[1, 0, 1]),   # path through a hub
        H.query(4, [(0, 1), (1, 2), (0, 2), (2, 3)], vlab=[0, 1, 2, 1], elab=[0, 1, 0, 1]),
        H.query(5, [(0, 1), (0, 2), (0, 3), (3, 4)], vlab=[0, 1, 1, 2, 1], elab=[1, 1, 0, 0]),
    ]
    nonzero = 0
    for q in queries:
        want, fp = oracle.count(O, q)
        for no_dedup in (False, True):      # with and without duplicate removal: the same set
            r = G.query(q, no_dedup=no_dedup)
            assert r.count == want
            assert oracle.fingerprint(r.rows()) == (want, fp[1], fp[2])
        nonzero += want > 0
    assert nonzero >= 4
