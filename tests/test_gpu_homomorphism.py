"""Homomorphism semantics (Sec. VII-A: the set subtraction of Alg. 3 dropped)
on the plain path, against the oracle's homomorphism mode and closed forms."""
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
def test_homomorphism_sets_match_oracle(pkg, seed):
    rng = np.random.default_rng(300 + seed)
    for case in range(12):
        n = int(rng.integers(20, 120))
        g = H.random_graph(rng, n, float(rng.uniform(0.05, 0.3)), int(rng.integers(1, 4)), int(rng.integers(1, 3)))
        if g.m == 0:
            continue
        k = int(rng.integers(2, 6))
        q = H.random_connected_query(rng, k, int(rng.integers(0, 3)), int(rng.integers(1, 4)),
                                     int(rng.integers(1, 3)))
        G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
        want = oracle.enumerate_rows(og(g), q, hom=True)
        for host_driven in (False, True):
            r = G.query(q, semantics=pkg.GSI_HOMOMORPHISM, host_driven=host_driven)
            assert r.count == want.shape[0], (seed, case, host_driven)
            assert np.array_equal(oracle.sort_rows(r.rows()), want), (seed, case, host_driven)
        # isomorphism results are the injective subset
        iso = oracle.enumerate_rows(og(g), q)
        assert G.query(q).count == iso.shape[0]


def test_homomorphism_closed_forms_on_rmat(pkg):
    """Unlabelled R-MAT graph: walks (paths), sum deg^s (stars), and
    homomorphisms equal embeddings for a clique (triangle)."""
    s, d = synth.rmat(61, 12, 20_000)
    n = 1 << 12
    g = H.G(np.zeros(n, np.int32), s, d, np.zeros(s.shape[0], np.int32))
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    deg = np.bincount(g.src, minlength=n) + np.bincount(g.dst, minlength=n)
    x = np.ones(n, dtype=object)

    def adj_mul(v):
        out = np.zeros(n, dtype=object)
        np.add.at(out, g.src, v[g.dst])
        np.add.at(out, g.dst, v[g.src])
        return out

    y = x.copy()
    for k in (2, 3, 4):
        y = adj_mul(y)                                     # y = A^(k-1) 1
        want = int(sum(y))
        assert G.query(H.path_query(k), count_only=True, semantics=pkg.GSI_HOMOMORPHISM).count == want
    for sdeg in (2, 3):
        want = int(sum(int(v) ** sdeg for v in deg))
        assert G.query(H.star_query(sdeg), count_only=True, semantics=pkg.GSI_HOMOMORPHISM).count == want
    tri = H.clique_query(3)
    assert (G.query(tri, count_only=True, semantics=pkg.GSI_HOMOMORPHISM).count ==
            G.query(tri, count_only=True).count)


def test_unknown_semantics_rejected(pkg):
    g = H.complete(5)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    with pytest.raises(pkg.GsiError) as e:
        G.query(H.path_query(3), semantics=2)
    assert e.value.status == pkg.GSI_EINVAL
