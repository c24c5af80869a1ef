"""Pins for the CPU oracle, independent of the oracle itself.

Each check is something the paper or mathematics fixes: exhaustive brute force
over every injective map (Defs. 2-3), closed-form embedding counts, counts from
a library routine (numpy matrix powers), a published hash's reference
implementation (scikit-learn's MurmurHash3), the necessary-condition property
of the Sec. III-A signature filter, and the composition of Alg. 3 join
iterations into the full result.
"""
import itertools
import math
import struct

import numpy as np
import pytest

import oracle
from tests import helpers as H

pytestmark = pytest.mark.filterwarnings("ignore")


def og(g):
    return oracle.OracleGraph(g.vlab, g.src, g.dst, g.elab)


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("block", range(12))
def test_backtracking_equals_bruteforce(block):
    """Defs. 2-3: the backtracking enumerator equals exhaustive search (1200 cases)."""
    rng = np.random.default_rng(1000 + block)
    for case in range(100):
        n = int(rng.integers(3, 10))
        g = H.random_graph(rng, n, float(rng.uniform(0.2, 0.8)), int(rng.integers(1, 4)), int(rng.integers(1, 4)))
        k = int(rng.integers(1, min(5, n) + 1))
        if case % 2 == 0 and g.m > 0:
            q = H.extracted_query(rng, g, k) or H.random_connected_query(rng, k, int(rng.integers(0, 3)), 3, 3)
        else:
            q = H.random_connected_query(rng, k, int(rng.integers(0, 3)), int(rng.integers(1, 4)),
                                         int(rng.integers(1, 4)))
        G = og(g)
        got = oracle.enumerate_rows(G, q)
        want = oracle.bruteforce_rows(G, q)
        assert got.shape == want.shape and np.array_equal(got, want), (block, case)
        c, fp = oracle.count(G, q, nthreads=3)
        assert c == want.shape[0]
        assert fp == oracle.fingerprint(want)


def test_bruteforce_disconnected_query():
    """The oracle also evaluates a disconnected query (two disjoint edges)."""
    rng = np.random.default_rng(7)
    for _ in range(30):
        g = H.random_graph(rng, 7, 0.5, 2, 2)
        q = H.query(4, [(0, 1), (2, 3)], rng.integers(0, 2, 4), rng.integers(0, 2, 2))
        G = og(g)
        assert np.array_equal(oracle.enumerate_rows(G, q), oracle.bruteforce_rows(G, q))


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n,k", [(5, 1), (5, 3), (6, 4), (7, 5), (8, 3), (9, 4)])
def test_clique_in_complete_graph(n, k):
    """Unlabelled k-clique in K_n: n!/(n-k)! embeddings."""
    c, _ = oracle.count(og(H.complete(n)), H.clique_query(k))
    assert c == math.perm(n, k)


@pytest.mark.parametrize("n,k", [(6, 3), (7, 4), (9, 5)])
def test_any_query_in_complete_graph(n, k):
    """Any unlabelled k-vertex query in K_n: n!/(n-k)! (every injective map works)."""
    for q in (H.path_query(k), H.star_query(k - 1)):
        c, _ = oracle.count(og(H.complete(n)), q)
        assert c == math.perm(n, k)


@pytest.mark.parametrize("n", [4, 5, 9, 20])
def test_triangle_in_cycle_is_zero(n):
    c, _ = oracle.count(og(H.cycle(n)), H.clique_query(3))
    assert c == 0


@pytest.mark.parametrize("n,k", [(5, 2), (6, 4), (10, 6), (12, 12)])
def test_path_in_cycle(n, k):
    """P_k in C_n (n >= k >= 2): 2n embeddings."""
    c, _ = oracle.count(og(H.cycle(n)), H.path_query(k))
    assert c == 2 * n


def test_edge_count_and_stars():
    """Single edge: 2|E|; star K_{1,s}: sum_v deg(v)!/(deg(v)-s)!."""
    rng = np.random.default_rng(3)
    for _ in range(10):
        g = H.random_graph(rng, 30, 0.2, 1, 1)
        deg = np.bincount(np.concatenate([g.src, g.dst]), minlength=g.n)
        G = og(g)
        assert oracle.count(G, H.path_query(2))[0] == 2 * g.m
        for s in (2, 3, 4):
            assert oracle.count(G, H.star_query(s))[0] == sum(H.falling(int(d), s) for d in deg)


def test_labelled_star():
    """Labelled star: sum over centres of prod over (edge label, leaf label) keys of falling factorials."""
    rng = np.random.default_rng(11)
    for _ in range(10):
        g = H.random_graph(rng, 40, 0.3, 3, 2)
        G = og(g)
        s = int(rng.integers(1, 5))
        cl = int(rng.integers(0, 3))
        leaf_vl = rng.integers(0, 3, s)
        leaf_el = rng.integers(0, 2, s)
        q = H.star_query(s, [cl] + list(leaf_vl), leaf_el)
        need = {}
        for a, b in zip(leaf_el, leaf_vl):
            need[(int(a), int(b))] = need.get((int(a), int(b)), 0) + 1
        nbrs = {v: [] for v in range(g.n)}
        for a, b, l in zip(g.src, g.dst, g.elab):
            nbrs[int(a)].append((int(l), int(g.vlab[b])))
            nbrs[int(b)].append((int(l), int(g.vlab[a])))
        want = 0
        for v in range(g.n):
            if g.vlab[v] != cl:
                continue
            prod = 1
            for key, mk in need.items():
                prod *= H.falling(sum(1 for x in nbrs[v] if x == key), mk)
            want += prod
        assert oracle.count(G, q)[0] == want


def test_triangles_match_matrix_trace():
    """Unlabelled triangle embeddings = trace(A^3) (numpy matrix product)."""
    rng = np.random.default_rng(5)
    for _ in range(8):
        g = H.random_graph(rng, 25, float(rng.uniform(0.1, 0.5)), 1, 1)
        A = np.zeros((g.n, g.n), np.int64)
        A[g.src, g.dst] = 1
        A[g.dst, g.src] = 1
        assert oracle.count(og(g), H.clique_query(3))[0] == int(np.trace(A @ A @ A))


@pytest.mark.parametrize("a,b", [(2, 2), (3, 4), (5, 3)])
def test_four_cycle_in_complete_bipartite(a, b):
    """C4 in K_{a,b}: 2 a(a-1) b(b-1)."""
    q = H.query(4, [(0, 1), (1, 2), (2, 3), (0, 3)])
    assert oracle.count(og(H.complete_bipartite(a, b)), q)[0] == 2 * a * (a - 1) * b * (b - 1)


def test_labels_select():
    """A vertex-label mismatch or an edge-label mismatch removes the embedding."""
    g = H.graph(3, [(0, 1), (1, 2)], vlab=[0, 1, 0], elab=[5, 6])
    G = og(g)
    assert oracle.count(G, H.query(2, [(0, 1)], [0, 1], [5]))[0] == 1
    assert oracle.count(G, H.query(2, [(0, 1)], [0, 1], [6]))[0] == 1
    assert oracle.count(G, H.query(2, [(0, 1)], [0, 1], [7]))[0] == 0
    assert oracle.count(G, H.query(2, [(0, 1)], [1, 1], [5]))[0] == 0


def test_non_induced():
    """Matches are not induced: a path query matches inside a triangle (6 ways)."""
    assert oracle.count(og(H.complete(3)), H.path_query(3))[0] == 6


# ------------------------------------------------------------------ signature
def test_murmur3_matches_library():
    """The oracle's hash is MurmurHash3 x86_32: compare with scikit-learn's implementation."""
    sk = pytest.importorskip("sklearn.utils")
    rng = np.random.default_rng(9)
    for _ in range(300):
        a, b = (int(x) for x in rng.integers(-2**31, 2**31, 2))
        key = struct.pack("<ii", a, b)
        seed = int(rng.integers(0, 2**32))
        assert oracle.murmur3_32(key, seed) == sk.murmurhash3_32(key, seed=seed, positive=True)
    for ln in range(0, 13):
        data = bytes(rng.integers(0, 256, ln).astype(np.uint8))
        assert oracle.murmur3_32(data, 0x9747B28C) == sk.murmurhash3_32(data, seed=0x9747B28C, positive=True)


def _group(el, nl):
    return oracle.murmur3_32(struct.pack("<ii", el, nl), 0x9747B28C) % 240


def test_signature_states():
    """Sec. III-A: label stored in the first 32 bits; group states 00/01/11 for 0/1/>=2 pairs."""
    # centre 0 (label 9): neighbours 1, 2 share key (edge 3, label 4); neighbour 3 has key (edge 1, label 2)
    g = H.graph(4, [(0, 1), (0, 2), (0, 3)], vlab=[9, 4, 4, 2], elab=[3, 3, 1])
    sig = oracle.data_signatures(og(g))
    s0 = sig[0]
    assert s0[0] == 9
    g1, g2 = _group(3, 4), _group(1, 2)
    bits = np.unpackbits(s0[1:].view(np.uint8), bitorder="little")
    assert bits[2 * g1] == 1 and bits[2 * g1 + 1] == 1
    if g2 != g1:
        assert bits[2 * g2] == 1 and bits[2 * g2 + 1] == 0
    assert bits.sum() == (2 if g1 == g2 else 3)
    # a leaf: one pair (3, 9)
    s1 = np.unpackbits(sig[1][1:].view(np.uint8), bitorder="little")
    assert sig[1][0] == 4 and s1.sum() == 1 and s1[2 * _group(3, 9)] == 1


def test_isolated_vertex_signature():
    g = H.graph(3, [(0, 1)], vlab=[1, 2, 7], elab=[0])
    sig = oracle.data_signatures(og(g))
    assert sig[2][0] == 7 and not sig[2][1:].any()


@pytest.mark.parametrize("seed", range(6))
def test_filter_is_sound(seed):
    """Sec. III-A: every data vertex used at u by some embedding passes the filter for u."""
    rng = np.random.default_rng(200 + seed)
    for _ in range(25):
        g = H.random_graph(rng, 12, 0.4, 2, 2)
        G = og(g)
        q = H.extracted_query(rng, g, int(rng.integers(2, 6)))
        if q is None:
            continue
        rows = oracle.enumerate_rows(G, q)
        member, counts = oracle.filter_sets(G, q)
        assert np.array_equal(counts, member.sum(axis=1))
        for u in range(q.k):
            assert member[u, rows[:, u]].all()
            # the label part is exact equality
            assert not member[u, g.vlab != q.vlab[u]].any()


def test_filter_prunes_by_neighbourhood():
    """A vertex with the right label but too few matching neighbours is pruned."""
    # data: 0 - 1 (labels 0,1), query: centre label 0 with two leaves labelled 1 (same key twice -> state 11)
    g = H.graph(3, [(0, 1), (0, 2)], vlab=[0, 1, 2], elab=[0, 0])
    q = H.star_query(2, [0, 1, 1], [0, 0])
    member, _ = oracle.filter_sets(og(g), q)
    assert not member[0, 0]


# ------------------------------------------------------------------ join step
@pytest.mark.parametrize("seed", range(6))
def test_join_steps_compose_to_full_result(seed):
    """Alg. 2/3: seeding M with C(u_first) and applying one join per vertex yields every embedding."""
    rng = np.random.default_rng(300 + seed)
    for _ in range(15):
        g = H.random_graph(rng, 14, 0.35, 2, 2)
        G = og(g)
        q = H.extracted_query(rng, g, int(rng.integers(2, 6)))
        if q is None:
            continue
        want = oracle.enumerate_rows(G, q)
        member, _ = oracle.filter_sets(G, q)
        qadj = {}
        for a, b, l in zip(q.src, q.dst, q.elab):
            qadj[(int(a), int(b))] = qadj[(int(b), int(a))] = int(l)
        # any connected order: random BFS-like growth
        order = [int(rng.integers(0, q.k))]
        while len(order) < q.k:
            cand = sorted({b for (a, b) in qadj if a in order and b not in order})
            order.append(int(rng.choice(cand)))
        for use_filter in (True, False):
            M = np.nonzero(member[order[0]] if use_filter else g.vlab == q.vlab[order[0]])[0].astype(np.int32)[:, None]
            for t in range(1, q.k):
                u = order[t]
                cols = [c for c in range(t) if (order[c], u) in qadj]
                labs = [qadj[(order[c], u)] for c in cols]
                inC = member[u] if use_filter else (g.vlab == q.vlab[u])
                M = oracle.join_step(G, M, inC, cols, labs)
            # back to query-vertex order
            if M.shape[0]:
                out = np.empty_like(M)
                out[:, order] = M
            else:
                out = np.empty((0, q.k), np.int32)
            assert np.array_equal(oracle.sort_rows(out), want)


def test_join_step_rules():
    """One step: injectivity (set subtraction), candidate set and every linking edge apply."""
    # triangle 0-1-2 plus pendant 2-3; all labels 0
    g = H.graph(4, [(0, 1), (1, 2), (0, 2), (2, 3)])
    G = og(g)
    M = np.array([[0, 1], [1, 0], [2, 3]], np.int32)
    everyone = np.ones(4, bool)
    # extend by a vertex adjacent to column 0 only
    got = oracle.join_step(G, M, everyone, [0], [0])
    assert [tuple(r) for r in got] == [(0, 1, 2), (1, 0, 2), (2, 3, 0), (2, 3, 1)]
    # adjacent to both columns
    got = oracle.join_step(G, M, everyone, [0, 1], [0, 0])
    assert [tuple(r) for r in got] == [(0, 1, 2), (1, 0, 2)]
    # candidate set excludes vertex 2
    inC = np.array([1, 1, 0, 1], bool)
    assert oracle.join_step(G, M, inC, [0, 1], [0, 0]).shape[0] == 0


@pytest.mark.parametrize("seed", range(3))
def test_join_step_output_within_the_alg4_bound(seed):
    """Alg. 4's preallocation bound, stated in Sec. V: row i's output never
    exceeds |N(v'_i, l0)| for whichever linking edge is taken as the first
    edge.  So the preallocated area, the sum of those bounds (|GBA|, the last
    offset of their exclusive scan), holds every survivor."""
    rng = np.random.default_rng(3000 + seed)
    for case in range(30):
        n = int(rng.integers(8, 40))
        g = H.random_graph(rng, n, float(rng.uniform(0.1, 0.5)), 2, 2)
        if g.m == 0:
            continue
        G = og(g)
        t = int(rng.integers(1, 4))
        M = np.unique(np.array([rng.choice(n, t, replace=False) for _ in range(int(rng.integers(1, 30)))],
                               np.int32), axis=0)                     # distinct rows, as in a table
        d = int(rng.integers(1, t + 1))
        cols = rng.choice(t, d, replace=False).tolist()
        labs = rng.integers(0, 2, d).tolist()
        in_c = rng.random(n) < 0.7
        out = oracle.join_step(G, M, in_c, cols, labs)
        nbrs = lambda v, l: sum(G.edge_label(int(v), w) == l for w in range(n))
        for j in range(d):
            caps = [nbrs(m[cols[j]], labs[j]) for m in M]
            per_row = [int((out[:, :t] == m).all(axis=1).sum()) for m in M] if out.shape[0] else [0] * len(M)
            assert all(c <= b for c, b in zip(per_row, caps)), (seed, case, j)
            assert out.shape[0] <= sum(caps)


def test_fingerprint_is_order_independent():
    rng = np.random.default_rng(1)
    rows = rng.integers(0, 1000, (500, 6)).astype(np.int32)
    fp = oracle.fingerprint(rows)
    assert fp == oracle.fingerprint(rows[rng.permutation(500)])
    assert fp != oracle.fingerprint(rows[:-1])
    assert fp[0] == 500


def test_fingerprint_separates_sets_that_additive_mixes_confuse():
    """The full-size parity tests compare fingerprints, so a wrong result must
    change them even where column sums, per-column value multisets and the
    row count stay the same: a column swap (a transposed operand), a +1/-1
    shift of two ids (an off-by-one that cancels in any additive hash), and
    two rows trading a value (right values, wrong rows)."""
    rng = np.random.default_rng(7)
    rows = np.unique(rng.integers(0, 5000, (2000, 5)).astype(np.int32), axis=0)
    fp = oracle.fingerprint(rows)
    for trial in range(20):
        a, b = rng.choice(rows.shape[1], 2, replace=False)
        swapped = rows.copy()
        swapped[:, [a, b]] = swapped[:, [b, a]]
        assert oracle.fingerprint(swapped) != fp
        one = rows.copy()
        r = rng.integers(rows.shape[0])
        one[r, [a, b]] = one[r, [b, a]]
        if not np.array_equal(one[r], rows[r]):
            assert oracle.fingerprint(one) != fp
        shifted = rows.copy()
        r1, r2 = rng.choice(rows.shape[0], 2, replace=False)
        c = rng.integers(rows.shape[1])
        shifted[r1, c] += 1
        shifted[r2, c] -= 1
        assert shifted[:, c].sum() == rows[:, c].sum()
        assert oracle.fingerprint(shifted) != fp
        traded = rows.copy()
        if traded[r1, c] != traded[r2, c]:
            traded[r1, c], traded[r2, c] = rows[r2, c], rows[r1, c]
            assert np.array_equal(np.sort(traded[:, c]), np.sort(rows[:, c]))
            assert oracle.fingerprint(traded) != fp


# ------------------------------------------------- homomorphism (Sec. VII-A)
@pytest.mark.parametrize("block", range(4))
def test_homomorphism_backtracking_equals_bruteforce(block):
    """Sec. VII-A: without injectivity, backtracking equals the exhaustive
    check of all n^k maps (400 cases)."""
    rng = np.random.default_rng(2000 + block)
    for case in range(100):
        n = int(rng.integers(3, 8))
        g = H.random_graph(rng, n, float(rng.uniform(0.2, 0.8)), int(rng.integers(1, 3)), int(rng.integers(1, 3)))
        k = int(rng.integers(1, 5))
        q = H.random_connected_query(rng, k, int(rng.integers(0, 3)), int(rng.integers(1, 3)),
                                     int(rng.integers(1, 3)))
        G = og(g)
        got = oracle.enumerate_rows(G, q, hom=True)
        want = oracle.bruteforce_rows(G, q, hom=True)
        assert np.array_equal(got, want), (block, case)
        c, fp = oracle.count(G, q, nthreads=3, hom=True)
        assert c == want.shape[0] and fp == oracle.fingerprint(want)
        # every embedding is a homomorphism; a clique query has no others
        iso = oracle.enumerate_rows(G, q)
        assert iso.shape[0] <= want.shape[0]
        if len(q.src) == k * (k - 1) // 2:
            assert np.array_equal(iso, want)


def test_homomorphism_closed_forms():
    """Unlabelled: hom(edge) = 2|E|, hom(path of k vertices) = 1^T A^(k-1) 1
    (walks), hom(star K_1,s) = sum_v deg(v)^s, hom(C4) = trace(A^4)."""
    rng = np.random.default_rng(11)
    for _ in range(6):
        g = H.random_graph(rng, 18, float(rng.uniform(0.1, 0.5)), 1, 1)
        G = og(g)
        A = np.zeros((g.n, g.n), np.int64)
        A[g.src, g.dst] = 1
        A[g.dst, g.src] = 1
        one = np.ones(g.n, np.int64)
        deg = A.sum(axis=1)
        assert oracle.count(G, H.path_query(2), hom=True)[0] == 2 * g.m
        for k in (3, 4, 5):
            want = int(one @ np.linalg.matrix_power(A, k - 1) @ one)
            assert oracle.count(G, H.path_query(k), hom=True)[0] == want
        for s in (2, 3):
            assert oracle.count(G, H.star_query(s), hom=True)[0] == int((deg ** s).sum())
        c4 = H.query(4, [(0, 1), (1, 2), (2, 3), (0, 3)])
        assert oracle.count(G, c4, hom=True)[0] == int(np.trace(np.linalg.matrix_power(A, 4)))


# ------------------------------------------- worked example (Secs. III-B, IV, V)
def test_worked_example_fixture_holds_the_printed_facts():
    """The constructed graph satisfies every Prealloc fact Sec. V prints."""
    facts, g, q = H.worked_example()
    G = og(g)
    nbr = lambda v, l: sorted(w for w in range(g.n) if w != v and G.edge_label(v, w) == l)
    rows = [(0, i) for i in range(1, 101)]                     # matches of u0u1 (label a)
    caps_a = [len(nbr(v1, 0)) for _, v1 in rows]               # first edge u1u2, label a
    caps_b = [len(nbr(v0, 1)) for v0, _ in rows]               # first edge u0u2, label b
    assert sum(caps_a) == facts["gba_u1u2"][0]
    assert sum(caps_a[:99]) == facts["buf99_offset"][0] and caps_a[99] == facts["num_L99_a"][0]
    assert sum(caps_b) == facts["gba_u0u2"][0]
    assert [w for w in nbr(100, 0) if w not in (0, 100)] == facts["buf99_subtracted"]


def test_worked_example_fixture_holds_the_other_printed_facts():
    """Facts printed about the same graph outside the Prealloc example:
    - Sec. III-B's candidate sets are the vertex-label classes.  The
      signature filter keeps a subset of each (a reading: the text lists
      candidates by label);
    - Sec. IV's P(G,b) has two edges, on v0, v1, v101 and v201;
    - Sec. IV's PCSR example gives N(v0,a) 100 entries."""
    facts, g, q = H.worked_example()
    G = og(g)
    member, _ = oracle.filter_sets(G, q)
    for u in range(q.k):
        lo, hi = facts[f"cand_u{u}"]
        printed = list(range(lo, hi + 1))
        assert np.flatnonzero(g.vlab == q.vlab[u]).tolist() == printed
        assert set(np.flatnonzero(member[u]).tolist()) <= set(printed)
    b = g.elab == 1
    assert int(b.sum()) == facts["pgb_edges"][0]
    assert sorted(set(g.src[b].tolist()) | set(g.dst[b].tolist())) == facts["pgb_vertices"]
    assert sum(G.edge_label(0, w) == 0 for w in range(g.n)) == facts["n_v0_a"][0]


def test_worked_example_oracle_join_and_match():
    """Alg. 3 on the example: joining u2 to M = {(v0, v_i)} leaves only
    buf99 = {v201}; the full search returns the single printed match."""
    facts, g, q = H.worked_example()
    G = og(g)
    M = np.array([(0, i) for i in range(1, 101)], np.int32)
    in_c = np.array(g.vlab == 2, np.uint8)                     # C(u2) = the label-C vertices
    got = oracle.join_step(G, M, in_c, [1, 0], [0, 1])         # linking edges u1u2:a, u0u2:b
    assert got.tolist() == [[0, 100] + facts["buf99_final"]]
    assert oracle.enumerate_rows(G, q).tolist() == [facts["match"]]
    member, _ = oracle.filter_sets(G, q)                       # the match survives the filter
    assert all(member[u, v] for u, v in enumerate(facts["match"]))
