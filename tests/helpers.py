"""Small seeded graph/query builders for tests (plain numpy; no method arithmetic)."""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np


@dataclass
class Q:
    vlab: np.ndarray
    src: np.ndarray
    dst: np.ndarray
    elab: np.ndarray

    @property
    def k(self):
        return int(self.vlab.shape[0])


@dataclass
class G:
    vlab: np.ndarray
    src: np.ndarray
    dst: np.ndarray
    elab: np.ndarray

    @property
    def n(self):
        return int(self.vlab.shape[0])

    @property
    def m(self):
        return int(self.src.shape[0])


def arr(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32).reshape(-1))


def graph(n, edges, vlab=None, elab=None) -> G:
    edges = [(min(a, b), max(a, b)) for a, b in edges]
    vlab = arr(vlab if vlab is not None else [0] * n)
    el = arr(elab if elab is not None else [0] * len(edges))
    s = arr([a for a, _ in edges])
    d = arr([b for _, b in edges])
    return G(vlab, s, d, el)


def query(k, edges, vlab=None, elab=None) -> Q:
    vlab = arr(vlab if vlab is not None else [0] * k)
    el = arr(elab if elab is not None else [0] * len(edges))
    return Q(vlab, arr([a for a, _ in edges]), arr([b for _, b in edges]), el)


def complete(n):
    return graph(n, list(itertools.combinations(range(n), 2)))


def cycle(n):
    return graph(n, [(i, (i + 1) % n) for i in range(n)])


def complete_bipartite(a, b):
    return graph(a + b, [(i, a + j) for i in range(a) for j in range(b)])


def path_query(k):
    return query(k, [(i, i + 1) for i in range(k - 1)])


def clique_query(k):
    return query(k, list(itertools.combinations(range(k), 2)))


def star_query(s, vlab=None, elab=None):
    return query(s + 1, [(0, i) for i in range(1, s + 1)], vlab, elab)


def random_graph(rng, n, p, n_vl, n_el) -> G:
    edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
    return graph(n, edges, rng.integers(0, n_vl, n), rng.integers(0, n_el, len(edges)))


def random_connected_query(rng, k, extra, n_vl, n_el) -> Q:
    """Random spanning tree on k vertices plus `extra` random extra edges."""
    edges = set()
    for v in range(1, k):
        u = int(rng.integers(0, v))
        edges.add((u, v))
    allp = [(i, j) for i in range(k) for j in range(i + 1, k) if (i, j) not in edges]
    rng.shuffle(allp)
    for e in allp[:extra]:
        edges.add(e)
    edges = sorted(edges)
    return query(k, edges, rng.integers(0, n_vl, k), rng.integers(0, n_el, len(edges)))


def extracted_query(rng, g: G, k):
    """Query = a connected k-vertex piece of g (BFS from a random vertex), with g's labels."""
    adj = {v: [] for v in range(g.n)}
    lab = {}
    for a, b, l in zip(g.src, g.dst, g.elab):
        adj[int(a)].append(int(b)); adj[int(b)].append(int(a)); lab[(int(a), int(b))] = lab[(int(b), int(a))] = int(l)
    for _ in range(50):
        start = int(rng.integers(0, g.n))
        seen = [start]
        frontier = [start]
        while frontier and len(seen) < k:
            v = frontier.pop(0)
            nb = adj[v][:]
            rng.shuffle(nb)
            for w in nb:
                if w not in seen and len(seen) < k:
                    seen.append(w); frontier.append(w)
        if len(seen) == k:
            idx = {v: i for i, v in enumerate(seen)}
            edges, el = [], []
            for i, v in enumerate(seen):
                for w in adj[v]:
                    if w in idx and idx[w] > i and rng.random() < 0.8:
                        edges.append((i, idx[w])); el.append(lab[(v, w)])
            # keep connected: add BFS tree edges back if needed
            parent_edges = _spanning(seen, adj)
            es = set(edges)
            for a, b in parent_edges:
                e = (min(idx[a], idx[b]), max(idx[a], idx[b]))
                if e not in es:
                    es.add(e); edges.append(e); el.append(lab[(a, b)])
            return query(k, edges, g.vlab[seen], el)
    return None


def _spanning(verts, adj):
    vs = set(verts)
    seen = {verts[0]}
    out = []
    stack = [verts[0]]
    while stack:
        v = stack.pop()
        for w in adj[v]:
            if w in vs and w not in seen:
                seen.add(w); out.append((v, w)); stack.append(w)
    return out


def falling(x, k):
    r = 1
    for i in range(k):
        r *= (x - i)
    return r if x >= k else 0


def worked_example():
    """(printed facts, graph, query) of the worked-example fixture (Secs. III-B, IV, V)."""
    import os
    facts, vl, E, qvl, QE = {}, None, [], None, []
    path = os.path.join(os.path.dirname(__file__), "golden", "worked_example.txt")
    for line in open(path):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "fact":
            facts[f[1]] = [int(x) for x in f[2:]]
        elif f[0] == "vlab":
            vl = [int(x) for x in f[1:]]
        elif f[0] == "e":
            E.append(tuple(int(x) for x in f[1:]))
        elif f[0] == "qvlab":
            qvl = [int(x) for x in f[1:]]
        elif f[0] == "qe":
            QE.append(tuple(int(x) for x in f[1:]))
    g = graph(len(vl), [(a, b) for a, b, _ in E], vl, [l for _, _, l in E])
    q = query(len(qvl), [(a, b) for a, b, _ in QE], qvl, [l for _, _, l in QE])
    return facts, g, q
