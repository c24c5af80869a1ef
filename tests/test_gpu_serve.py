"""Served execution (continuous batching over slots) and bounded device waits."""
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
    s, d = synth.rmat(51, 13, 70_000)
    n = 1 << 13
    g = H.G(synth.labels_zipf(51, 1, n, 8, 1.1), s, d, synth.labels_uniform(51, 2, 70_000, 3))
    sg = synth.make_graph(g.vlab, g.src, g.dst, g.elab, 3)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    qs = [synth.walk_query(sg, 91, i, 3 + i % 5, dense=bool(i % 2), max_bound=1e6) for i in range(40)]
    return g, G, qs


def _serve_all(S, qs):
    tickets = [S.submit(q) for q in qs]
    out = []
    for t in tickets:
        got = S.poll(t, -1)
        assert got is not None
        out.append(got)
    return out


@pytest.mark.parametrize("n_streams,max_batch,min_batch", [(2, 0, 1), (3, 4, 2), (1, 1, 0), (2, 0, 0), (1, 0, 16)])
def test_served_result_equals_alone(pkg, world, n_streams, max_batch, min_batch):
    """Each query's result is the same alone (plain path) and served in the mix,
    whether the slots batch, run one at a time, or switch by queue length."""
    g, G, qs = world
    S = pkg.Server(G, mem_budget=8 << 30, n_streams=n_streams, max_batch=max_batch, min_batch=min_batch)
    served = _serve_all(S, qs)
    for q, (r, lat) in zip(qs, served):
        alone = G.query(q)
        assert r.count == alone.count
        assert np.array_equal(oracle.sort_rows(r.rows()), oracle.sort_rows(alone.rows()))
        assert lat >= 0
    S.close()


def test_served_cancel_and_invalid(pkg, world):
    g, G, qs = world
    S = pkg.Server(G, mem_budget=4 << 30, n_streams=1, max_batch=1)
    tickets = [S.submit(q) for q in qs]
    S.cancel(tickets[-1])
    for t in tickets[:-1]:
        assert S.poll(t, -1) is not None
    try:
        got = S.poll(tickets[-1], -1)
        assert got is not None            # it had already started: a normal result
    except pkg.GsiError as e:
        assert e.status == pkg.GSI_ECANCELLED
    with pytest.raises(pkg.GsiError) as e:
        S.submit(H.query(3, [(0, 1)]))
    assert e.value.status == pkg.GSI_EINVAL
    with pytest.raises(pkg.GsiError):
        S.poll(10**9, 0)                  # unknown ticket
    S.close()


def test_bounded_device_wait_runs_out(pkg):
    """A grid barrier that can never complete gives up, reports GSI_ETIMEOUT, and the device stays usable."""
    import torch
    rc, ms = pkg.selftest_wait_timeout(0, 4096)
    assert rc == pkg.GSI_ETIMEOUT
    assert ms < 5000
    x = torch.arange(1000, device="cuda").sum().item()   # the context still works
    assert x == 499500


def test_served_workspace_reuse(pkg, world):
    """A slot's batch workspace is reused by batches of changing composition;
    every batch must see only its own data (a missing barrier between the
    seed writes and the first join step once let stale seeds through)."""
    g, G, qs = world
    alone = [G.query(q).count for q in qs]
    for i in range(20):
        S = pkg.Server(G, mem_budget=8 << 30, n_streams=1, max_batch=0, min_batch=1, item_rows=16 if i % 2 else 0)
        served = _serve_all(S, qs)
        S.close()
        assert [r.count for r, _ in served] == alone


def test_server_estimate_is_the_fewest_matching_edges(pkg, world):
    """The admission estimate of a query is 8 bytes (two int32 columns) times
    the fewest directed data edges that match one of its query edges by the
    labels of both ends and the edge label: counted here with numpy from the
    edge list."""
    g, G, qs = world
    S = pkg.Server(G, mem_budget=8 << 30, n_streams=1)
    src = np.concatenate([g.src, g.dst])
    dst = np.concatenate([g.dst, g.src])
    el = np.concatenate([g.elab, g.elab])
    for q in qs:
        want = min(int(((g.vlab[src] == q.vlab[a]) & (g.vlab[dst] == q.vlab[b]) & (el == l)).sum())
                   for a, b, l in zip(q.src, q.dst, q.elab))
        assert S.estimate(q) == 8 * want
    # a label no data vertex carries: nothing can match
    q = H.query(2, [(0, 1)], vlab=[0, 99], elab=[0])
    assert S.estimate(q) == 0
    S.close()


@pytest.mark.parametrize("budget", [1 << 30, 4 << 30, 12 << 30])
def test_served_under_tight_memory_budgets(pkg, world, budget):
    """Batches reserve their estimated memory from the budget (at least 4 GiB
    or the whole budget): with room for one batch at a time, or for three,
    every served result equals the plain path's."""
    g, G, qs = world
    alone = [G.query(q).count for q in qs]
    S = pkg.Server(G, mem_budget=budget, n_streams=3, max_batch=0, min_batch=1)
    served = _serve_all(S, qs * 3)
    S.close()
    assert [r.count for r, _ in served] == alone * 3
