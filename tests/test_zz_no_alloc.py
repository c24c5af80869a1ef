"""The allocation-free join step (gsi_join_step_noalloc) against gsi_join_step.

Some callers cannot allocate device memory (a plugin inside a runtime that
owns all device memory, a serving path that must not wait on an allocator, a
process under a strict memory quota).  They call gsi_join_step_noalloc, whose
scratch is one static device array.  This file checks, through the C ABI,
that two calls in a row give the same result as the allocating entry point,
and that sizes beyond the array's limits are rejected.
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


def _run(G, fn, M, member_u, ulabel, cols, labs, cap):
    import torch
    t = M.shape[1]
    Md = torch.from_numpy(np.ascontiguousarray(M)).cuda()
    cd = torch.from_numpy(_bitmap(member_u).view(np.int32)).cuda()
    out = torch.full((cap, t + 1), -1, dtype=torch.int32, device="cuda")
    cnt = fn(Md.data_ptr(), M.shape[0], t, cd.data_ptr(), int(ulabel), cols, labs, out.data_ptr(), cap)
    torch.cuda.synchronize()
    return cnt, oracle.sort_rows(out[: min(cnt, cap)].cpu().numpy())


def test_noalloc_matches_allocating_join_step_twice(pkg):
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
            cap = max(16, 64 * M.shape[0])
            want_n, want = _run(G, G.join_step, M, member[u], q.vlab[u], cols, labs, cap)
            # two calls in a row on the shared static scratch
            for _ in range(2):
                got_n, got = _run(G, G.join_step_noalloc, M, member[u], q.vlab[u], cols, labs, cap)
                assert got_n == want_n
                assert np.array_equal(got, want)
                calls += 1
            M = want
    assert calls >= 8


def test_noalloc_rejects_sizes_beyond_its_limit(pkg):
    g = H.complete(4)
    G = pkg.Graph(g.vlab, g.src, g.dst, g.elab)
    with pytest.raises(pkg.GsiError) as e:
        G.join_step_noalloc(16, (1 << 20) + 1, 1, 16, 0, [0], [0], 0, 0)
    assert e.value.status == pkg.GSI_EINVAL
    assert "2^20" in str(e.value)
