"""Small hand-built graph families for the tests (constructions from first
principles, each with its known minimum cut).  No minimum-cut arithmetic."""
from __future__ import annotations

import itertools

import numpy as np


def from_edges(n, edges, weights=None):
    """Symmetric CSR (rows sorted) from an undirected edge list.  Parallel
    edges are kept as separate entries (callers that want a canonical graph
    pass distinct pairs)."""
    edges = list(edges)
    if weights is None:
        weights = [1] * len(edges)
    src, dst, ww = [], [], []
    for (u, v), c in zip(edges, weights):
        src += [u, v]
        dst += [v, u]
        ww += [c, c]
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    ww = np.asarray(ww, np.int64)
    order = np.lexsort((dst, src)) if len(src) else np.zeros(0, np.int64)
    src, dst, ww = src[order], dst[order], ww[order]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, src + 1, 1)
    rp = np.cumsum(rp)
    return rp, dst.astype(np.int32), ww


def cycle(n, weights=None):
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], weights)


def complete(n, w=1):
    e = list(itertools.combinations(range(n), 2))
    return from_edges(n, e, [w] * len(e))


def complete_bipartite(a, b):
    e = [(i, a + j) for i in range(a) for j in range(b)]
    return from_edges(a + b, e)


def hypercube(d):
    n = 1 << d
    e = [(v, v ^ (1 << k)) for v in range(n) for k in range(d) if v < v ^ (1 << k)]
    return from_edges(n, e)


def grid(a, b):
    idx = lambda i, j: i * b + j
    e = []
    for i in range(a):
        for j in range(b):
            if i + 1 < a:
                e.append((idx(i, j), idx(i + 1, j)))
            if j + 1 < b:
                e.append((idx(i, j), idx(i, j + 1)))
    return from_edges(a * b, e)


def random_tree(n, rng, wlo=1, whi=20):
    e = [(int(rng.integers(0, v)), v) for v in range(1, n)]
    w = [int(x) for x in rng.integers(wlo, whi + 1, size=n - 1)]
    return from_edges(n, e, w), min(w)


def two_cliques(k5, path_w, clique_w, links):
    """Two K_k5 with weight clique_w joined by `links` distinct edges of weight
    path_w between vertex i of the first clique and vertex i of the second."""
    e, w = [], []
    for base in (0, k5):
        for i, j in itertools.combinations(range(k5), 2):
            e.append((base + i, base + j))
            w.append(clique_w)
    for i in range(links):
        e.append((i, k5 + i))
        w.append(path_w)
    return from_edges(2 * k5, e, w)


def random_graph(n, p, rng, wlo=1, whi=10, connected=False):
    while True:
        e = [(i, j) for i, j in itertools.combinations(range(n), 2) if rng.random() < p]
        w = [int(x) for x in rng.integers(wlo, whi + 1, size=len(e))]
        g = from_edges(n, e, w)
        if not connected or is_connected(n, g[0], g[1]):
            return g


def is_connected(n, rp, col):
    seen = np.zeros(n, bool)
    seen[0] = True
    st = [0]
    while st:
        v = st.pop()
        for y in col[rp[v]:rp[v + 1]]:
            if not seen[y]:
                seen[y] = True
                st.append(int(y))
    return bool(seen.all())


def to_nx(n, rp, col, w):
    import networkx as nx
    G = nx.Graph()
    G.add_nodes_from(range(n))
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            v = int(col[e])
            if u < v:
                if G.has_edge(u, v):
                    G[u][v]["weight"] += int(w[e])
                else:
                    G.add_edge(u, v, weight=int(w[e]))
    return G


def csr_checksum(g) -> str:
    """Order-dependent 64-bit checksum of a graph's (row_ptr, col, w), as hex:
    ties a stored value to the exact generator output it was computed on."""
    h = np.uint64(1469598103934665603)
    with np.errstate(over="ignore"):
        for a in (g.row_ptr.astype(np.uint64), g.col.astype(np.uint64), g.w.astype(np.uint64)):
            idx = np.arange(1, a.size + 1, dtype=np.uint64)
            h = np.uint64(h * np.uint64(1099511628211)) ^ np.uint64(
                np.bitwise_xor.reduce(a * np.uint64(0x9E3779B97F4A7C15) +
                                      idx * np.uint64(0xBF58476D1CE4E5B9)))
            h = np.uint64(h + np.uint64(a.size))
    return f"{int(h):016x}"
