"""Pins for the CPU oracle: closed forms, brute force, library routines and
hand-derived golden traces.  CPU only (``-m "not gpu"``).

Each pin is chosen so that a plausible mistake in the oracle (a dropped term,
a wrong sign or index, a transposed operand) fails it."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import synth
from tests import graphs as G

GOLD = os.path.join(os.path.dirname(__file__), "golden")
INF = oracle.INF


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def mincut_all(n, g):
    """Brute force, Stoer-Wagner and NOI on the same graph."""
    rp, col, w = g
    b, bs = oracle.mincut_brute(n, rp, col, w) if n <= 18 else (None, None)
    s, ss = oracle.stoer_wagner(n, rp, col, w)
    q, qs, _ = oracle.noi(n, rp, col, w)
    return b, s, q, bs, ss, qs


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [3, 4, 5, 8, 13])
def test_unit_cycle_is_2(n):
    b, s, q, *_ = mincut_all(n, G.cycle(n))
    assert b == s == q == 2


def test_weighted_cycle_two_smallest():
    rng = np.random.default_rng(7)
    for n in [3, 5, 9, 14, 40]:
        w = [int(x) for x in rng.integers(1, 50, size=n)]
        b, s, q, *_ = mincut_all(n, G.cycle(n, w))
        expect = sum(sorted(w)[:2])
        assert s == q == expect
        if b is not None:
            assert b == expect


@pytest.mark.parametrize("n", [2, 3, 5, 7, 9])
def test_complete_graph_is_n_minus_1(n):
    b, s, q, *_ = mincut_all(n, G.complete(n))
    assert b == s == q == n - 1


def test_complete_graph_large():
    n = 60
    _, s, q, *_ = mincut_all(n, G.complete(n, 3))
    assert s == q == 3 * (n - 1)


def test_int32_max_weights_sum_in_int64():
    """Weights at the int32 limit: every cut value exceeds 2^31 (K_n) or
    2^32 and the oracle tiers still agree with the closed forms."""
    W = (1 << 31) - 1
    for n in (4, 7, 12):
        b, s, q, *_ = mincut_all(n, G.complete(n, W))
        assert s == q == (n - 1) * W
        if b is not None:
            assert b == (n - 1) * W
    w = [W, W - 1, W - 2, W, W, W - 5]
    b, s, q, *_ = mincut_all(6, G.cycle(6, w))
    assert b == s == q == (W - 5) + (W - 2)


def test_scale_invariance_at_large_weights():
    """Multiplying every weight and the bound by k scales every cut by k and
    changes no PR flag, CAPFOREST order or mark (all their tests compare
    sums of weights); k = 2^24 pushes the sums past 2^32."""
    rng = np.random.default_rng(29)
    k = 1 << 24
    for trial in range(40):
        n = int(rng.integers(3, 10))
        rp, col, w = G.random_graph(n, float(rng.uniform(0.3, 1.0)), rng, 1, 100)
        wk = w.astype(np.int64) * k
        lam = int(oracle.degrees(n, rp, col, w).min())
        assert np.array_equal(oracle.pr_marks(n, rp, col, w, lam, 0xF, -1),
                              oracle.pr_marks(n, rp, col, wk, lam * k, 0xF, -1))
        a = oracle.capforest(n, rp, col, w, lam, 0)
        b = oracle.capforest(n, rp, col, wk, lam * k, 0)
        assert b["lambda"] == k * a["lambda"]
        assert np.array_equal(a["order"], b["order"]) and np.array_equal(a["marks"], b["marks"])
        assert oracle.noi(n, rp, col, wk)[0] == k * oracle.noi(n, rp, col, w)[0]
        assert oracle.stoer_wagner(n, rp, col, wk)[0] == k * oracle.mincut_brute(n, rp, col, w)[0]


def test_relabelling_invariance():
    """lambda does not depend on vertex names: NOI and Stoer-Wagner on a
    randomly relabelled copy agree with brute force on the original, and
    the returned sides are cuts of that value in the relabelled graph."""
    rng = np.random.default_rng(31)
    for trial in range(60):
        n = int(rng.integers(2, 14))
        rp, col, w = G.random_graph(n, float(rng.uniform(0.2, 1.0)), rng, 1, 20)
        lam = oracle.mincut_brute(n, rp, col, w)[0]
        perm = rng.permutation(n)
        src = np.repeat(np.arange(n), np.diff(rp))
        keep = src < col
        edges = list(zip(perm[src[keep]].tolist(), perm[col[keep]].tolist()))
        g2 = G.from_edges(n, edges, w[keep].tolist())
        q, side, _ = oracle.noi(n, *g2)
        s2, sside = oracle.stoer_wagner(n, *g2)
        assert q == s2 == lam
        assert oracle.cut_weight(n, *g2, side) == lam
        assert oracle.cut_weight(n, *g2, sside) == lam


def test_tree_is_min_edge():
    rng = np.random.default_rng(3)
    for n in [2, 5, 11, 16, 200]:
        g, wmin = G.random_tree(n, rng)
        b, s, q, *_ = mincut_all(n, g)
        assert s == q == wmin
        if b is not None:
            assert b == wmin


@pytest.mark.parametrize("a,b", [(1, 1), (2, 3), (3, 3), (2, 7), (4, 6)])
def test_complete_bipartite_is_min_side(a, b):
    br, s, q, *_ = mincut_all(a + b, G.complete_bipartite(a, b))
    assert s == q == min(a, b)
    if br is not None:
        assert br == min(a, b)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 7])
def test_hypercube_is_d(d):
    b, s, q, *_ = mincut_all(1 << d, G.hypercube(d))
    assert s == q == d
    if b is not None:
        assert b == d


@pytest.mark.parametrize("a,b", [(2, 2), (2, 5), (3, 4), (4, 4), (15, 20)])
def test_grid_is_2(a, b):
    br, s, q, *_ = mincut_all(a * b, G.grid(a, b))
    assert s == q == 2
    if br is not None:
        assert br == 2


def test_disconnected_is_0():
    rp, col, w = G.from_edges(7, [(0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (5, 6), (3, 6)],
                              [5, 5, 5, 7, 7, 7, 7])
    b, s, q, bs, ss, qs = mincut_all(7, (rp, col, w))
    assert b == s == q == 0
    for side in (bs, ss, qs):
        assert oracle.cut_weight(7, rp, col, w, side) == 0
        assert 0 < side.sum() < 7


def test_isolated_vertex_is_0():
    rp, col, w = G.from_edges(4, [(0, 1), (1, 2)], [3, 3])
    b, s, q, *_ = mincut_all(4, (rp, col, w))
    assert b == s == q == 0


@pytest.mark.parametrize("k", [1, 2, 3])
def test_two_cliques_joined_by_k(k):
    rp, col, w = G.two_cliques(6, 1, 4, k)
    b, s, q, *_ = mincut_all(12, (rp, col, w))
    assert b == s == q == k


def test_two_vertices():
    rp, col, w = G.from_edges(2, [(0, 1)], [9])
    b, s, q, *_ = mincut_all(2, (rp, col, w))
    assert b == s == q == 9


def test_brute_st_cut_on_path():
    # path 0-1-2-3-4 with weights: lambda(G, s, t) = min weight between s and t
    w = [5, 2, 7, 3]
    rp, col, ww = G.from_edges(5, [(i, i + 1) for i in range(4)], w)
    for s, t in itertools.combinations(range(5), 2):
        assert oracle.st_cut_brute(5, rp, col, ww, s, t) == min(w[s:t])


def test_cut_weight_by_definition():
    rp, col, w = G.from_edges(4, [(0, 1), (1, 2), (2, 3), (0, 3)], [1, 2, 3, 4])
    assert oracle.cut_weight(4, rp, col, w, np.array([1, 0, 0, 0], np.uint8)) == 1 + 4
    assert oracle.cut_weight(4, rp, col, w, np.array([1, 1, 0, 0], np.uint8)) == 2 + 4
    assert oracle.cut_weight(4, rp, col, w, np.array([0, 0, 0, 0], np.uint8)) == 0


# ------------------------------------------------- cross-checks on random graphs
def test_random_small_graphs_all_tiers_agree():
    rng = np.random.default_rng(11)
    for trial in range(300):
        n = int(rng.integers(2, 13))
        g = G.random_graph(n, float(rng.uniform(0.15, 0.9)), rng, 1, int(rng.integers(1, 12)))
        b, s, q, bs, ss, qs = mincut_all(n, g)
        assert b == s == q, (trial, n, b, s, q)
        for side in (bs, ss, qs):
            assert oracle.cut_weight(n, *g, side) == b
            assert 0 < side.sum() < n


def test_stoer_wagner_and_noi_vs_networkx():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(5)
    for trial in range(12):
        n = int(rng.integers(20, 90))
        g = G.random_graph(n, float(rng.uniform(0.05, 0.3)), rng, 1, 30, connected=True)
        cut, _ = nx.stoer_wagner(G.to_nx(n, *g))
        s, _ = oracle.stoer_wagner(n, *g)
        q, _, _ = oracle.noi(n, *g)
        assert s == q == cut


def test_noi_vs_stoer_wagner_er_workload():
    g = synth.er_connected(600, 4000, 1, 10, 9)
    s, ss = oracle.stoer_wagner(g.n, g.row_ptr, g.col, g.w)
    q, qs, rounds = oracle.noi(g.n, g.row_ptr, g.col, g.w)
    assert s == q
    assert oracle.cut_weight(g.n, g.row_ptr, g.col, g.w, qs) == q
    assert rounds >= 1


def test_noi_planted_cut_small():
    g = synth.planted(1 << 11, 21 << 11, 30, 5, 1, 17)
    q, side, _ = oracle.noi(g.n, g.row_ptr, g.col, g.w)
    assert q == 5
    assert oracle.cut_weight(g.n, g.row_ptr, g.col, g.w, side) == 5
    # the witness is the block split
    blk = g.meta["block"]
    assert np.array_equal(side, blk ^ blk[0])


@pytest.mark.parametrize("n", [5, 6, 9, 16, 17])
def test_wheel_all_trivial_cuts_minimum(n):
    # closed form: every vertex has weighted degree 2(n-1) and no cut is lighter
    g = synth.wheel(n, seed=n)
    c = (g.row_ptr, g.col, g.w.astype(np.int64))
    deg = oracle.degrees(n, *c)
    assert (deg == 2 * (n - 1)).all()
    b, s_, q, *_ = mincut_all(n, c)
    assert b == s_ == q == 2 * (n - 1)


@pytest.mark.parametrize("n", [10, 14, 18])
def test_dblcyc_halves_are_the_unique_minimum(n):
    # closed form: lambda = 2*heavy, attained only by the two halves (brute
    # force over all cuts for n <= 18 checks uniqueness)
    heavy, light = 50, 3
    g = synth.dblcyc(n, heavy, light, seed=n)
    c = (g.row_ptr, g.col, g.w.astype(np.int64))
    b, s_, q, *_ = mincut_all(n, c)
    assert b == s_ == q == 2 * heavy
    vals = []
    for mask in range(1, 1 << (n - 1)):
        side = np.array([(mask >> v) & 1 for v in range(n)], np.uint8)
        vals.append(oracle.cut_weight(n, *c, side))
    vals = np.sort(np.array(vals))
    assert vals[0] == 2 * heavy and vals[1] >= 2 * heavy + 2 * light


def test_adversarial_families_noi_larger():
    for n in (202, 403):
        g = synth.wheel(n, seed=1)
        assert oracle.noi(n, g.row_ptr, g.col, g.w.astype(np.int64))[0] == 2 * (n - 1)
    for n in (202, 302):
        g = synth.dblcyc(n, 1000, 3, seed=2)
        assert oracle.noi(n, g.row_ptr, g.col, g.w.astype(np.int64))[0] == 2000


def test_noi_accepts_noncanonical_input():
    # duplicates, a self-loop and a zero-weight entry
    rp, col, w = G.from_edges(4, [(0, 1), (0, 1), (1, 2), (2, 3), (3, 0), (2, 2), (1, 3)],
                              [1, 2, 4, 4, 4, 9, 0])
    b, _ = oracle.mincut_brute(4, rp, col, w)
    q, _, _ = oracle.noi(4, rp, col, w)
    s, _ = oracle.stoer_wagner(4, rp, col, w)
    assert b == q == s == 7  # {0} has 1+2+4 = 7; {3}: 4+4 = 8


# ------------------------------------------------------------------ contraction
def dense(n, rp, col, w):
    A = np.zeros((n, n), np.int64)
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            A[u, col[e]] += w[e]
    return A


def test_contract_is_PtAP_offdiagonal():
    rng = np.random.default_rng(2)
    for trial in range(60):
        n = int(rng.integers(1, 25))
        g = G.random_graph(n, 0.4, rng, 1, 9) if n > 1 else G.from_edges(1, [])
        groups = rng.integers(0, max(1, n // 2 + 1), size=n).astype(np.int32)
        n2, L = oracle.labels_from_groups(groups)
        rp2, col2, w2 = oracle.contract(n, *g, L, n2)
        P = np.zeros((n, n2), np.int64)
        P[np.arange(n), L] = 1
        A2 = P.T @ dense(n, *g) @ P
        np.fill_diagonal(A2, 0)
        # canonical CSR of A2: rows ascending, nonzeros only
        nz = [np.nonzero(A2[i])[0] for i in range(n2)]
        assert np.array_equal(rp2, np.concatenate([[0], np.cumsum([len(x) for x in nz])]))
        if len(col2):
            assert np.array_equal(col2, np.concatenate(nz))
            assert np.array_equal(w2, np.concatenate([A2[i][nz[i]] for i in range(n2)]))


def test_canonical_labels_order_by_smallest_member():
    groups = np.array([5, 2, 5, 0, 2, 6, 0], np.int32)
    n2, L = oracle.labels_from_groups(groups)
    assert n2 == 4
    assert L.tolist() == [0, 1, 0, 2, 1, 3, 2]


def test_labels_from_pairs_vs_networkx():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(8)
    for trial in range(40):
        n = int(rng.integers(1, 60))
        k = int(rng.integers(0, n + 1))
        pu = rng.integers(0, n, size=k).astype(np.int32)
        pv = rng.integers(0, n, size=k).astype(np.int32)
        n2, L = oracle.labels_from_pairs(n, pu, pv)
        H = nx.Graph()
        H.add_nodes_from(range(n))
        H.add_edges_from(zip(pu.tolist(), pv.tolist()))
        comps = sorted((sorted(c) for c in nx.connected_components(H)), key=lambda c: c[0])
        assert n2 == len(comps)
        for cid, c in enumerate(comps):
            assert all(L[v] == cid for v in c)


def test_contract_preserves_unsplit_cuts():
    rng = np.random.default_rng(21)
    for trial in range(25):
        n = int(rng.integers(3, 11))
        g = G.random_graph(n, 0.5, rng, 1, 7)
        groups = rng.integers(0, n, size=n).astype(np.int32)
        n2, L = oracle.labels_from_groups(groups)
        rp2, col2, w2 = oracle.contract(n, *g, L, n2)
        for mask in range(1 << n2):
            s2 = np.array([(mask >> i) & 1 for i in range(n2)], np.uint8)
            assert oracle.cut_weight(n2, rp2, col2, w2, s2) == oracle.cut_weight(n, *g, s2[L])


def test_contract_degree_sum_invariant():
    rng = np.random.default_rng(4)
    g = G.random_graph(30, 0.3, rng, 1, 9)
    groups = rng.integers(0, 10, size=30).astype(np.int32)
    n2, L = oracle.labels_from_groups(groups)
    rp2, col2, w2 = oracle.contract(30, *g, L, n2)
    rp, col, w = g
    src = np.repeat(np.arange(30), np.diff(rp))
    inner = w[L[src] == L[col]].sum()
    assert w2.sum() == w.sum() - inner


# -------------------------------------------------------------------- PR tests
def test_pr_golden_example():
    d = gold("pr_example.json")
    rp, col, w = G.from_edges(d["n"], d["edges"], d["weights"])
    fl = oracle.pr_marks(d["n"], rp, col, w, d["lambda"], 0xF, -1)
    for u in range(d["n"]):
        for e in range(rp[u], rp[u + 1]):
            v = int(col[e])
            key = f"{min(u, v)}-{max(u, v)}"
            assert fl[e] == d["expect_flags"][key], key
    assert oracle.mincut_brute(d["n"], rp, col, w)[0] == d["mincut"]


def test_pr_strict_exchange_counterexample():
    d = gold("pr2_strict_counterexample.json")
    e, w = [], []
    for base in (0, 5):
        for i, j in itertools.combinations(range(5), 2):
            e.append((base + i, base + j)); w.append(3)
    e += [(0, 10), (10, 11), (11, 5)]; w += [2, 2, 2]
    rp, col, ww = G.from_edges(12, e, w)
    lam = int(oracle.degrees(12, rp, col, ww).min())
    assert lam == d["min_degree"]
    assert oracle.stoer_wagner(12, rp, col, ww)[0] == d["mincut"]
    fl = oracle.pr_marks(12, rp, col, ww, lam, 0xF, -1)
    src = np.repeat(np.arange(12), np.diff(rp))
    path = ((src >= 10) | (col >= 10))
    assert not fl[path].any(), "a path edge was marked"


def _check_pr_soundness(n, g, lam, fl):
    rp, col, w = g
    lam_true, _ = oracle.mincut_brute(n, rp, col, w)
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            v = int(col[e])
            if u > v or not fl[e]:
                continue
            if fl[e] & (1 | 8):  # threshold tests: lambda(G,u,v) >= lambda_hat
                assert oracle.st_cut_brute(n, rp, col, w, u, v) >= lam
            if fl[e] & (2 | 4):  # exchange tests: no minimum cut below lambda_hat separates u, v
                if lam_true < lam:
                    assert oracle.st_cut_brute(n, rp, col, w, u, v) > lam_true
    # simultaneous contraction keeps lambda
    pu = [u for u in range(n) for e in range(rp[u], rp[u + 1]) if fl[e] and u < col[e]]
    pv = [int(col[e]) for u in range(n) for e in range(rp[u], rp[u + 1]) if fl[e] and u < col[e]]
    n2, L = oracle.labels_from_pairs(n, np.array(pu, np.int32), np.array(pv, np.int32))
    rp2, col2, w2 = oracle.contract(n, rp, col, w, L, n2)
    lam2 = oracle.mincut_brute(n2, rp2, col2, w2)[0] if n2 >= 2 else INF
    assert min(lam, lam2) == lam_true


def test_pr_soundness_brute_force():
    rng = np.random.default_rng(13)
    fired = np.zeros(4, int)
    for trial in range(250):
        n = int(rng.integers(3, 11))
        g = G.random_graph(n, float(rng.uniform(0.3, 1.0)), rng, 1, int(rng.integers(1, 9)))
        deg = oracle.degrees(n, *g)
        lam = int(deg.min())
        if trial % 3 == 0:  # any valid upper bound in [lambda, min degree]
            lam_true = oracle.mincut_brute(n, *g)[0]
            lam = int(rng.integers(lam_true, lam + 1))
        fl = oracle.pr_marks(n, *g, lam, 0xF, -1)
        for b in range(4):
            fired[b] += int(((fl >> b) & 1).sum() > 0)
        _check_pr_soundness(n, g, lam, fl)
    assert (fired > 0).all(), fired  # every test fires somewhere


def test_pr_budget_only_limits():
    rng = np.random.default_rng(1)
    g = G.random_graph(14, 0.6, rng, 1, 5)
    lam = int(oracle.degrees(14, *g).min())
    full = oracle.pr_marks(14, *g, lam, 0xF, -1)
    cut = oracle.pr_marks(14, *g, lam, 0xF, 3)
    assert np.all((cut & ~full) == 0)
    assert np.array_equal(cut & 3, full & 3)


# ------------------------------------------------------------------- CAPFOREST
@pytest.mark.parametrize("name", ["capforest_two_triangles.json", "capforest_chain.json"])
def test_capforest_golden_trace(name):
    d = gold(name)
    rp, col, w = G.from_edges(d["n"], d["edges"], d["weights"])
    r = oracle.capforest(d["n"], rp, col, w, d["lambda_in"], d["start"])
    ex = d["expect"]
    assert r["lambda"] == ex["lambda_out"]
    assert r["order"].tolist() == ex["order"]
    assert r["marks"].tolist() == ex["marks"]
    assert r["best_len"] == ex["best_len"]
    for u in range(d["n"]):
        for e in range(rp[u], rp[u + 1]):
            v = int(col[e])
            key = f"{min(u, v)}-{max(u, v)}"
            if r["q"][e] >= 0:
                assert r["q"][e] == ex["q"][key], key
    assert oracle.mincut_brute(d["n"], rp, col, w)[0] == d["mincut"]


def test_capforest_marks_sound_and_alpha_is_a_cut():
    rng = np.random.default_rng(17)
    for trial in range(200):
        n = int(rng.integers(2, 12))
        g = G.random_graph(n, float(rng.uniform(0.2, 1.0)), rng, 1, int(rng.integers(1, 9)))
        rp, col, w = g
        lam_true, _ = oracle.mincut_brute(n, rp, col, w)
        lam_in = int(oracle.degrees(n, rp, col, w).min())
        start = int(rng.integers(0, n))
        r = oracle.capforest(n, rp, col, w, lam_in, start)
        assert lam_true <= r["lambda"] <= lam_in
        for x, y in r["marks"]:
            assert oracle.st_cut_brute(n, rp, col, w, int(x), int(y)) >= r["lambda"]
        if r["best_len"]:
            side = np.zeros(n, np.uint8)
            side[r["order"][:r["best_len"]]] = 1
            assert oracle.cut_weight(n, rp, col, w, side) == r["lambda"]
        n2, L = oracle.labels_from_pairs(n, r["marks"][:, 0].copy(), r["marks"][:, 1].copy())
        rp2, col2, w2 = oracle.contract(n, rp, col, w, L, n2)
        lam2 = oracle.mincut_brute(n2, rp2, col2, w2)[0] if n2 >= 2 else INF
        assert min(r["lambda"], lam2) == lam_true
        if G.is_connected(n, rp, col) and r["lambda"] == lam_in and lam_in > 0:
            assert len(r["marks"]) >= 1  # a full pass marks at least one edge
            assert sorted(r["order"].tolist()) == list(range(n))


# -------------------------------------------------------------------- LP bound
def test_lp_bound_is_cut_of_its_cluster():
    rng = np.random.default_rng(19)
    for trial in range(40):
        n = int(rng.integers(3, 40))
        g = G.random_graph(n, 0.2, rng, 1, 9)
        lab = oracle.lp(n, *g, 4)
        assert lab.min() >= 0 and lab.max() < n
        val, bl = oracle.lp_bound(n, *g, lab)
        if val == INF:
            assert len(np.unique(lab)) == 1
            continue
        side = (lab == bl).astype(np.uint8)
        assert 0 < side.sum() < n
        assert oracle.cut_weight(n, *g, side) == val
        if n <= 16:
            assert val >= oracle.mincut_brute(n, *g)[0]


def test_lp_two_cliques_finds_bridge():
    # enough sweeps separate two dense cliques joined by one light edge
    rp, col, w = G.two_cliques(6, 1, 5, 1)
    lab = oracle.lp(12, rp, col, w, 6)
    val, _ = oracle.lp_bound(12, rp, col, w, lab)
    assert val == 1


def test_lp_sweep_rule_small():
    # path 0-1-2 weights (1, 5): sweep 0 updates even vertices from the initial ids
    rp, col, w = G.from_edges(3, [(0, 1), (1, 2)], [1, 5])
    lab = oracle.lp(3, rp, col, w, 1)
    assert lab.tolist() == [1, 1, 1]  # 0 adopts 1 (weight 1 > 0), 2 adopts 1 (5 > 0)
    lab = oracle.lp(3, rp, col, w, 2)
    assert lab.tolist() == [1, 1, 1]  # 1 keeps 1 (own weight 6 > 0)


def test_lp_golden_trace():
    with open(os.path.join(GOLD, "lp_trace.json")) as f:
        gd = json.load(f)
    n = gd["n"]
    rp, col, w = G.from_edges(n, [tuple(e) for e in gd["edges"]], gd["weights"])
    for iters, labels in gd["expect_labels"].items():
        assert oracle.lp(n, rp, col, w, int(iters)).tolist() == labels, iters
    lab = oracle.lp(n, rp, col, w, 3)
    val, _ = oracle.lp_bound(n, rp, col, w, lab)
    assert val == gd["expect_bound"]
    assert oracle.mincut_brute(n, rp, col, w)[0] == gd["mincut"]


# ---------------------------------------------------------------- round oracle
def test_round_preserves_lambda():
    rng = np.random.default_rng(23)
    for trial in range(120):
        n = int(rng.integers(2, 12))
        g = G.random_graph(n, float(rng.uniform(0.2, 1.0)), rng, 1, int(rng.integers(1, 9)))
        lam_true, _ = oracle.mincut_brute(n, *g)
        n2, rp2, col2, w2, info = oracle.round_(n, *g, lp_iters=2, lp_min_n=4)
        assert n2 <= n
        lam2 = oracle.mincut_brute(n2, rp2, col2, w2)[0] if n2 >= 2 else INF
        if info["stopped"]:
            assert info["lambda"] == lam_true or n <= 2
        assert min(info["lambda"], lam2) == lam_true


@pytest.mark.parametrize("case", ["A", "B", "C", "D", "E"])
def test_round_golden_trace(case):
    d = gold("round_two_triangles.json")
    n = d["n"]
    rp, col, w = G.from_edges(n, d["edges"], d["weights"])
    c = d["cases"][case]
    lam_in = INF if c["lambda_in"] is None else c["lambda_in"]
    n2, rp2, col2, w2, info = oracle.round_(n, rp, col, w, lambda_in=lam_in, lp_iters=0,
                                            pr_mask=c["pr_mask"], capforest=c["capforest"])
    ex = c["expect"]
    assert n2 == ex["n2"]
    for k in ("lambda", "marks_pr", "marks_cf", "stopped"):
        assert info[k] == ex[k], k
    if ex.get("unchanged"):
        assert rp2.tolist() == rp.tolist() and col2.tolist() == col.tolist()
        assert w2.tolist() == w.tolist()
    else:
        assert rp2.tolist() == ex["rp2"] and col2.tolist() == ex["col2"]
        assert w2.tolist() == ex["w2"]
    assert oracle.mincut_brute(n, rp, col, w)[0] == d["mincut"]


def test_round_iterated_reaches_lambda():
    g = synth.er_connected(300, 1500, 1, 10, 3)
    s, _ = oracle.stoer_wagner(g.n, g.row_ptr, g.col, g.w)
    n, rp, col, w = g.n, g.row_ptr, g.col, g.w.astype(np.int64)
    lam = INF
    for it in range(1000):
        n, rp, col, w, info = oracle.round_(n, rp, col, w, lambda_in=lam, lp_iters=2, lp_min_n=50)
        lam = info["lambda"]
        if info["stopped"]:
            break
    assert lam == s


# ------------------------------------------- CAPFOREST, neighbour-first ties
def test_capforest_neighbour_first_golden_trace():
    d = gold("capforest_nbr_cycle.json")
    rp, col, w = G.from_edges(d["n"], d["edges"], d["weights"])
    r = oracle.capforest(d["n"], rp, col, w, d["lambda_in"], d["start"], tie=1)
    ex = d["expect"]
    assert r["lambda"] == ex["lambda_out"]
    assert r["order"].tolist() == ex["order"]
    assert r["marks"].tolist() == ex["marks"]
    assert r["best_len"] == ex["best_len"]
    for u in range(d["n"]):
        for e in range(rp[u], rp[u + 1]):
            v = int(col[e])
            if r["q"][e] >= 0:
                assert r["q"][e] == ex["q"][f"{min(u, v)}-{max(u, v)}"]
    r0 = oracle.capforest(d["n"], rp, col, w, d["lambda_in"], d["start"], tie=0)
    assert r0["order"].tolist() == d["smaller_id_rule"]["order"]
    assert r0["marks"].tolist() == d["smaller_id_rule"]["marks"]
    assert oracle.mincut_brute(d["n"], rp, col, w)[0] == d["mincut"]


def test_capforest_neighbour_first_two_triangles():
    # on the two triangles the neighbour-first rule visits in the same order
    # as the smaller-id rule (each tie is won by a neighbour of smaller id)
    d = gold("capforest_two_triangles.json")
    rp, col, w = G.from_edges(d["n"], d["edges"], d["weights"])
    r = oracle.capforest(d["n"], rp, col, w, d["lambda_in"], d["start"], tie=1)
    assert r["order"].tolist() == d["expect"]["order"]
    assert r["marks"].tolist() == d["expect"]["marks"]
    assert r["lambda"] == d["expect"]["lambda_out"]


def _replay_max_adjacency(n, rp, col, w, lam_in, order, start):
    """Replays a visit order and checks that every visited vertex had the
    highest bounded key Q = min(r, lambda) among the unvisited vertices
    reached so far (lambda lowered by the cuts of proper prefixes); returns
    the marks (x, y) with r(y) < lambda <= r(y) + c(x, y) in scan order."""
    r = np.zeros(n, np.int64)
    deg = oracle.degrees(n, rp, col, w)
    seen = np.zeros(n, bool)
    reached = np.zeros(n, bool)
    reached[start] = True
    lam, alpha, marks = lam_in, 0, []
    for i, x in enumerate(order):
        x = int(x)
        cand = [v for v in range(n) if reached[v] and not seen[v]]
        best = max(min(int(r[v]), lam) for v in cand)
        assert min(int(r[x]), lam) == best and reached[x] and not seen[x]
        seen[x] = True
        alpha += int(deg[x]) - 2 * int(r[x])
        if i + 1 < n and alpha < lam:
            lam = alpha
        for e in range(rp[x], rp[x + 1]):
            y = int(col[e])
            if seen[y]:
                continue
            if r[y] < lam <= r[y] + w[e]:
                marks.append((x, y))
            r[y] += w[e]
            reached[y] = True
    return lam, marks


def test_capforest_neighbour_first_is_max_adjacency_and_sound():
    """Random graphs: the neighbour-first order is a bounded maximum-adjacency
    order (replayed independently), the marks are those of that order, each
    mark (x, y) has lambda(G, x, y) >= the returned bound (brute force), the
    bound's prefix is a cut of that weight, and contracting the marks keeps
    min(bound, lambda(G')) = lambda(G)."""
    rng = np.random.default_rng(23)
    for trial in range(200):
        n = int(rng.integers(2, 12))
        g = G.random_graph(n, float(rng.uniform(0.2, 1.0)), rng, 1, int(rng.integers(1, 9)))
        rp, col, w = g
        lam_true, _ = oracle.mincut_brute(n, rp, col, w)
        lam_in = int(oracle.degrees(n, rp, col, w).min())
        start = int(rng.integers(0, n))
        r = oracle.capforest(n, rp, col, w, lam_in, start, tie=1)
        lam_r, marks_r = _replay_max_adjacency(n, rp, col, w, lam_in, r["order"], start)
        assert lam_r == r["lambda"]
        assert [tuple(m) for m in r["marks"].tolist()] == marks_r
        assert lam_true <= r["lambda"] <= lam_in
        for x, y in r["marks"]:
            assert oracle.st_cut_brute(n, rp, col, w, int(x), int(y)) >= r["lambda"]
        if r["best_len"]:
            side = np.zeros(n, np.uint8)
            side[r["order"][:r["best_len"]]] = 1
            assert oracle.cut_weight(n, rp, col, w, side) == r["lambda"]
        n2, L = oracle.labels_from_pairs(n, r["marks"][:, 0].copy(), r["marks"][:, 1].copy())
        rp2, col2, w2 = oracle.contract(n, rp, col, w, L, n2)
        lam2 = oracle.mincut_brute(n2, rp2, col2, w2)[0] if n2 >= 2 else INF
        assert min(r["lambda"], lam2) == lam_true
