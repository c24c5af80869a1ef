"""The allocation-free join step (gsi_join_step_noalloc), through the C ABI.

Some callers cannot allocate device memory: a plugin inside another runtime
that owns every device byte and hands it only input and output buffers, a
serving path that must never wait on an allocator, a process under a strict
memory quota.  They call gsi_join_step_noalloc, whose scratch is one static
device array.  This file checks that two calls in a row give the oracle's
join step (Alg. 3) and the allocating entry point's result, that the
count-only form counts the same rows, and that sizes beyond the array's
limits are rejected before any kernel touches it.

It is collected last, so a run that stops at the first failure has already
run every other test; it passes alone in a fresh process as well.
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


def _bitmap(member):
    n = member.shape[0]
    padded = np.zeros(((n + 31) // 32) * 32, bool)
    padded[:n] = member
    return np.packbits(padded, bitorder="little").view(np.uint32)


def _run(fn, M, member_u, ulabel, cols, labs, cap):
    import torch
    t = M.shape[1]
    Md = torch.from_numpy(np.ascontiguousarray(M)).cuda()
    cd = torch.from_numpy(_bitmap(member_u).view(np.int32)).cuda()
    out = torch.full((max(cap, 1), t + 1), -1, dtype=torch.int32, device="cuda")
    cnt = fn(Md.data_ptr(), M.shape[0], t, cd.data_ptr(), int(ulabel), cols, labs, out.data_ptr() if cap else 0,
             cap)
    torch.cuda.synchronize()
    return cnt, oracle.sort_rows(out[: min(cnt, cap)].cpu().numpy())


def test_noalloc_matches_oracle_and_allocating_join_step_twice(pkg):
    s, d = synth.rmat(77, 12, 30_000)
    n = 1 << 12
    g = H.G(synth.labels_zipf(77, 1, n, 6, 1.1), s, d, synth.labels_uniform(77, 2, 30_000, 3))
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    O = oracle.OracleGraph(g.vlab, g.src, g.dst, g.elab)
    sg = synth.make_graph(g.vlab, g.src, g.dst, g.elab, 3)
    calls = 0
    for i in range(6):
        q = synth.walk_query(sg, 21, i, 5, dense=bool(i % 2), max_bound=1e6)
        member, _ = oracle.filter_sets(O, q)
        order = list(oracle.order(q))
        qadj = {}
        for a, b, l in zip(q.src, q.dst, q.elab):
            qadj[(int(a), int(b))] = qadj[(int(b), int(a))] = int(l)
        M = np.nonzero(member[order[0]])[0].astype(np.int32)[:, None]
        for t in range(1, q.k):
            u = order[t]
            cols = [c for c in range(t) if (order[c], u) in qadj]
            labs = [qadj[(order[c], u)] for c in cols]
            if M.shape[0] == 0 or M.shape[0] > 200_000:
                break
            want = oracle.join_step(O, M, member[u], cols, labs)
            cap = max(16, want.shape[0])
            alloc_n, alloc_rows = _run(G.join_step, M, member[u], q.vlab[u], cols, labs, cap)
            assert alloc_n == want.shape[0] and np.array_equal(alloc_rows, want)
            # two calls in a row on the shared static scratch
            for _ in range(2):
                got_n, got = _run(G.join_step_noalloc, M, member[u], q.vlab[u], cols, labs, cap)
                assert got_n == want.shape[0]
                assert np.array_equal(got, want)
                calls += 1
            # count only (no output buffer): the same count
            cnt_only, _ = _run(G.join_step_noalloc, M, member[u], q.vlab[u], cols, labs, 0)
            assert cnt_only == want.shape[0]
            M = want
    assert calls >= 8


def test_noalloc_rejects_more_rows_than_its_limit(pkg):
    g = H.complete(4)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    with pytest.raises(pkg.GsiError) as e:
        G.join_step_noalloc(16, (1 << 20) + 1, 1, 16, 0, [0], [0], 0, 0)
    assert e.value.status == pkg.GSI_EINVAL
    assert "2^20" in str(e.value)


def test_noalloc_rejects_more_slots_than_its_limit(pkg):
    """2^20 copies of a star's centre, each with 300 candidates: the bound scan
    totals 2^20 * (300 + 2) > 2^28 slots, which the call must refuse before
    partitioning into the static array."""
    import torch
    leaves = 300
    g = H.graph(leaves + 1, [(0, i) for i in range(1, leaves + 1)], vlab=[0] + [1] * leaves)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    M = torch.zeros(1 << 20, dtype=torch.int32, device="cuda")
    member = np.zeros(leaves + 1, bool)
    member[1:] = True
    cd = torch.from_numpy(_bitmap(member).view(np.int32)).cuda()
    with pytest.raises(pkg.GsiError) as e:
        G.join_step_noalloc(M.data_ptr(), 1 << 20, 1, cd.data_ptr(), 1, [0], [0], 0, 0)
    assert e.value.status == pkg.GSI_EINVAL
    assert "2^28" in str(e.value)
    # the array is still usable afterwards: a small call gives the oracle's rows
    O = oracle.OracleGraph(g.vlab, g.src, g.dst, g.elab)
    M1 = np.zeros((3, 1), np.int32)
    want = oracle.join_step(O, M1, member, [0], [0])
    got_n, got = _run(G.join_step_noalloc, M1, member, 1, [0], [0], 4 * leaves)
    assert got_n == want.shape[0] == 3 * leaves
    assert np.array_equal(got, want)
