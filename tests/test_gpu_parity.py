"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work, so the bar is bit-exact: canonical CSRs, PR flags, the
deterministic CAPFOREST pass (visit order, mark set, bound), label
propagation bounds and every cut value.  Where several answers are correct
(the side of a minimum cut, the marks of concurrent passes) the tests check
what is unique (the value) and that the rest is valid (the side's cut weight
equals the value; every contraction keeps min(bound, lambda(G')) = lambda(G)).
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from tests import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2609_07204_gb300 as mc  # noqa: E402

INF = mc.INT64_MAX


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mc.load_library()


def canon(n, rp, col, w):
    return oracle.canonicalize(n, rp, col, w)


def make(n, rp, col, w, **kw):
    return mc.mincut_graph_from_csr(n, np.asarray(rp, np.int64), np.asarray(col, np.int32),
                                    np.asarray(w, np.int32), **kw)


def assert_csr_equal(a, b):
    assert np.array_equal(a[0], b[0]), "row_ptr differs"
    assert np.array_equal(a[1], b[1]), "col differs"
    assert np.array_equal(np.asarray(a[2], np.int64), np.asarray(b[2], np.int64)), "w differs"


def noncanonical(n, rng, m, wmax=9):
    """Symmetric multigraph with duplicates, self-loops, zero weights, rows
    in random order."""
    e = [(int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(m)]
    w = [int(x) for x in rng.integers(0, wmax + 1, size=m)]
    rp, col, ww = G.from_edges(n, e, w)
    # shuffle inside rows
    col = col.copy()
    ww = ww.copy()
    for u in range(n):
        b, en = rp[u], rp[u + 1]
        perm = rng.permutation(en - b)
        col[b:en] = col[b:en][perm]
        ww[b:en] = ww[b:en][perm]
    return rp, col, ww


# ----------------------------------------------------------- canonical input
@pytest.mark.parametrize("n,m,seed", [(2, 1, 0), (17, 60, 1), (300, 3000, 2), (5000, 90000, 3)])
def test_from_csr_canonicalises_like_oracle(n, m, seed):
    rng = np.random.default_rng(seed)
    rp, col, w = noncanonical(n, rng, m)
    g = make(n, rp, col, w)
    got = mc.mincut_graph_export_csr(g)
    assert_csr_equal(got, canon(n, rp, col, w))


def test_from_csr_large_multi_tile_multi_pass():
    # ~1.3M raw entries: many sort tiles, 4 radix passes (n = 2^17 -> 34 key bits)
    rng = np.random.default_rng(4)
    n, m = 1 << 17, 650_000
    u = rng.integers(0, n, size=m)
    v = rng.integers(0, n, size=m)
    w = rng.integers(1, 5, size=m)
    src = np.concatenate([u, v]); dst = np.concatenate([v, u]); ww = np.concatenate([w, w])
    order = rng.permutation(src.size)  # rows out of order inside
    src, dst, ww = src[order], dst[order], ww[order]
    o2 = np.argsort(src, kind="stable")
    src, dst, ww = src[o2], dst[o2], ww[o2]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, src + 1, 1)
    rp = np.cumsum(rp)
    g = make(n, rp, dst, ww)
    assert_csr_equal(mc.mincut_graph_export_csr(g), canon(n, rp, dst.astype(np.int32), ww))


def test_from_csr_above_the_scan_fold():
    """More than 2048 scan blocks (8.4 M values): the exclusive scans of the
    canonicalisation take their three-launch form (a separate partials pass)
    instead of the two-launch one.  10 M raw entries, rows out of order,
    duplicates; against the oracle's canonical form."""
    rng = np.random.default_rng(44)
    n, m = 1 << 20, 5_000_000
    u = rng.integers(0, n, size=m)
    v = rng.integers(0, n, size=m)
    w = rng.integers(1, 9, size=m)
    src = np.concatenate([u, v]); dst = np.concatenate([v, u]); ww = np.concatenate([w, w])
    order = rng.permutation(src.size)
    src, dst, ww = src[order], dst[order], ww[order]
    o2 = np.argsort(src, kind="stable")
    src, dst, ww = src[o2], dst[o2], ww[o2]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, src + 1, 1)
    rp = np.cumsum(rp)
    assert rp[-1] > 2048 * 4096
    g = make(n, rp, dst, ww)
    assert_csr_equal(mc.mincut_graph_export_csr(g), canon(n, rp, dst.astype(np.int32), ww))


@pytest.mark.parametrize("defect", ["none", "self", "zero", "swap", "swap_tile_edge"])
@pytest.mark.parametrize("big", [False, True])
def test_from_csr_canonical_input_and_single_defects(defect, big):
    """A canonical input is taken as is; one defect (a self-loop, a zero
    weight, two neighbours out of order -- also across an entry tile
    boundary) sends it through the canonicalisation sort.  Both give the
    oracle's canonical form and the exact minimum cut."""
    rng = np.random.default_rng(31 + big)
    n = 1200
    lo, hi = ((1 << 22), (1 << 31) - 1) if big else (1, 50)
    g0 = G.random_graph(n, 0.02, rng, lo, hi, connected=True)
    rp, col, w = (np.array(x) for x in canon(n, *g0))
    M = int(rp[-1])
    assert M > 4 * 2048
    col = col.astype(np.int32)
    w = w.astype(np.int64)
    if defect == "self":
        u = int(np.searchsorted(rp, M // 3, "right")) - 1
        b = int(rp[u])
        col = np.insert(col, b, u).astype(np.int32)
        w = np.insert(w, b, 7)
        rp[u + 1:] += 1
    elif defect == "zero":
        u = int(np.searchsorted(rp, M // 3, "right")) - 1
        b = int(rp[u])
        v = int(col[b])
        j = int(rp[v]) + int(np.searchsorted(col[rp[v]:rp[v + 1]], u))
        w[b] = 0
        w[j] = 0
    elif defect.startswith("swap"):
        i = 2047 if defect == "swap_tile_edge" else M // 2
        u = int(np.searchsorted(rp, i, "right")) - 1
        if i + 1 >= int(rp[u + 1]):  # keep both entries inside row u
            i = int(rp[u + 1]) - 2
        assert int(rp[u]) <= i
        col[i], col[i + 1] = col[i + 1], col[i]
        w[i], w[i + 1] = w[i + 1], w[i]
    g = make(n, rp, col, w)
    c = canon(n, rp, col, w)
    assert_csr_equal(mc.mincut_graph_export_csr(g), c)
    v, _, _ = mc.mincut_solve(g, bitmap=False)
    assert v == oracle.stoer_wagner(n, *c)[0]


def test_graphs_reuse_pooled_memory_and_release():
    """Graphs created one after another (library pool, pinned state mirrors
    reused) give the same results; releasing the cached blocks between
    graphs changes nothing."""
    rng = np.random.default_rng(8)
    rp, col, w = noncanonical(700, rng, 9000)
    c = canon(700, rp, col, w)
    exp = oracle.stoer_wagner(700, *c)[0]
    for i in range(6):
        g = make(700, rp, col, w)
        assert_csr_equal(mc.mincut_graph_export_csr(g), c)
        assert mc.mincut_solve(g, bitmap=False)[0] == exp
        g.destroy()
        if i % 2:
            mc.mincut_release_cached(torch.cuda.current_device())


def test_from_csr_device_pointers_and_torch_allocator():
    rng = np.random.default_rng(5)
    rp, col, w = noncanonical(400, rng, 5000)
    t = [torch.from_numpy(np.asarray(x)).cuda() for x in (rp, col.astype(np.int32), w.astype(np.int32))]
    g = mc.mincut_graph_from_csr(400, t[0], t[1], t[2], use_torch_allocator=True)
    assert_csr_equal(mc.mincut_graph_export_csr(g), canon(400, rp, col, w))
    v, bm, _ = mc.mincut_solve(g)
    c = canon(400, rp, col, w)
    assert v == oracle.stoer_wagner(400, *c)[0]
    g.destroy()


@pytest.mark.parametrize("case", ["asym", "neg", "range", "weight_asym", "unpaired_lower"])
def test_from_csr_rejects_malformed(case):
    rp, col, w = G.from_edges(4, [(0, 1), (1, 2), (2, 3)], [1, 2, 3])
    col = col.copy(); w = w.copy()
    if case == "unpaired_lower":
        # every entry u -> v with u < v has its mirror, but 3 -> 0 has none
        rp = np.array([0, 1, 3, 5, 7], np.int64)
        col = np.array([1, 0, 2, 1, 3, 0, 2], np.int32)
        w = np.array([1, 1, 2, 2, 3, 4, 3], np.int64)
    if case == "asym":
        col[0] = 3  # 0->3 without 3->0
    elif case == "neg":
        w[0] = -1
    elif case == "range":
        col[0] = 7
    elif case == "weight_asym":
        w[0] = 5
    with pytest.raises(mc.MincutError) as e:
        make(4, rp, col, w)
    assert e.value.status == mc.MINCUT_ERR_INVALID


@pytest.mark.parametrize("case", ["swap_weights", "two_vertex", "moved_mirror"])
def test_from_csr_rejects_asymmetry_with_balanced_counts(case):
    """Asymmetric canonical inputs whose (u < v) and (u > v) entry counts
    agree: only the triples differ (caught by the symmetry fingerprint of
    the input pass; the exact check covers non-canonical inputs)."""
    if case == "swap_weights":
        # 0-1 and 0-2 with weights 1, 2; mirrors carry them swapped
        rp, col, w = [0, 2, 3, 4], [1, 2, 0, 0], [1, 2, 2, 1]
        n = 3
    elif case == "two_vertex":
        rp, col, w = [0, 1, 2], [1, 0], [1, 2]
        n = 2
    else:
        # 0-1 present both ways; 0->2 is answered by 3->1 instead of 2->0
        rp, col, w = [0, 2, 3, 3, 4], [1, 2, 0, 1], [1, 1, 1, 1]
        n = 4
    for where in ("pageable", "pinned", "device"):
        args = [np.asarray(rp, np.int64), np.asarray(col, np.int32), np.asarray(w, np.int32)]
        if where == "pinned":
            args = [torch.from_numpy(a).pin_memory().numpy() for a in args]
        elif where == "device":
            args = [torch.from_numpy(a).cuda() for a in args]
        with pytest.raises(mc.MincutError) as e:
            mc.mincut_graph_from_csr(n, *args)
        assert e.value.status == mc.MINCUT_ERR_INVALID
    g = mc.mincut_graph_from_csr(n, np.asarray(rp, np.int64), np.asarray(col, np.int32),
                                 np.asarray(w, np.int32), skip_validate=True)
    g.destroy()


@pytest.mark.parametrize("canonical", [True, False])
def test_from_csr_pinned_host_matches_pageable_and_device(canonical):
    """Entries in pinned host memory are read in place by the input pass;
    the graph equals the one built from pageable host arrays and from device
    tensors, and so do the solves."""
    rng = np.random.default_rng(21)
    if canonical:
        g0 = synth.core_lcc(synth.rmat(13, 8, wlo=1, whi=9, seed=21), 3)
        rp, col, w = g0.row_ptr, g0.col, g0.w
        n = g0.n
    else:
        n = 900
        rp, col, w = noncanonical(n, rng, 12000)
    rp = np.asarray(rp, np.int64); col = np.asarray(col, np.int32); w = np.asarray(w, np.int32)
    c = canon(n, rp, col, w)
    pin = [torch.from_numpy(a).pin_memory() for a in (rp, col, w)]
    dev = [torch.from_numpy(a).cuda() for a in (rp, col, w)]
    ref = None
    for kind in ("pageable", "pinned", "device"):
        if kind == "pageable":
            g = mc.mincut_graph_from_csr(n, rp, col, w)
        elif kind == "pinned":
            g = mc.mincut_graph_from_csr(n, *(t.numpy() for t in pin))
        else:
            g = mc.mincut_graph_from_csr(n, *dev)
        assert_csr_equal(mc.mincut_graph_export_csr(g), c)
        v = mc.mincut_solve(g, bitmap=False)[0]
        if ref is None:
            ref = v
        assert v == ref
        g.destroy()
    if n <= 1000:
        assert ref == oracle.stoer_wagner(n, *c)[0]


# -------------------------------------------------------------- contraction
@pytest.mark.parametrize("n,p,seed", [(3, 0.9, 0), (60, 0.2, 1), (700, 0.05, 2), (3000, 0.01, 3)])
def test_contract_by_groups_bit_exact(n, p, seed):
    rng = np.random.default_rng(seed)
    g0 = synth.er(n, int(p * n * (n - 1) / 2), 1, 50, seed + 10)
    groups = rng.integers(0, max(1, n // 3), size=n).astype(np.int32)
    g = make(n, g0.row_ptr, g0.col, g0.w)
    ro = mc.default_round_options()
    ro.groups = groups.ctypes.data
    res = mc.mincut_contract_round(g, ro)
    n2, L = oracle.labels_from_groups(groups)
    exp = oracle.contract(n, g0.row_ptr, g0.col, g0.w, L, n2)
    assert res["n_out"] == n2
    assert_csr_equal(mc.mincut_graph_export_csr(g), exp)


def test_contract_by_pairs_bit_exact_and_chained():
    rng = np.random.default_rng(8)
    g0 = synth.er(4000, 40000, 1, 20, 8)
    g = make(g0.n, g0.row_ptr, g0.col, g0.w)
    n, rp, col, w = g0.n, g0.row_ptr, g0.col, g0.w.astype(np.int64)
    for step in range(4):
        k = n // 2
        pu = rng.integers(0, n, size=k).astype(np.int32)
        pv = rng.integers(0, n, size=k).astype(np.int32)
        ro = mc.default_round_options()
        ro.npairs = k
        ro.pair_u = pu.ctypes.data
        ro.pair_v = pv.ctypes.data
        res = mc.mincut_contract_round(g, ro)
        n2, L = oracle.labels_from_pairs(n, pu, pv)
        rp, col, w = oracle.contract(n, rp, col, w, L, n2)
        n = n2
        assert res["n_out"] == n2
        assert_csr_equal(mc.mincut_graph_export_csr(g), (rp, col, w))
    mc.mincut_graph_reset(g)
    assert mc.mincut_graph_info(g) == (g0.n, g0.M)


def _singleton_entry_share(n, rp, L):
    cnt = np.bincount(L)
    deg = np.diff(rp)
    return float(deg[cnt[L] == 1].sum()) / max(int(rp[-1]), 1)


@pytest.mark.parametrize("weights,scale", [("unit", 15), ("int64_totals", 15), ("unit", 13)])
def test_contract_rowwise_bit_exact(weights, scale):
    """Rounds where most groups are single vertices take the row-wise path:
    singleton rows rebuilt in place with the labels of multi-member groups
    merged in (duplicates summed), rows longer than 4096 entries and rows
    with more than 32 distinct multi-member neighbours through the sort.
    The scale-15 graphs hold more than 2^18 entries: their singleton rows go
    through the entry tiles (rows that cross tile boundaries included), those
    with several moved labels through the warp-per-row kernels; the scale-13
    ones (fewer entries) take one warp per singleton row.  Three chained
    contractions, each against the oracle's contraction."""
    rng = np.random.default_rng(21)
    s = synth.workload_rmat_core(scale=scale, k=8, seed=9)
    n, rp, col = s.n, s.row_ptr.copy(), s.col.copy()
    w = s.w.astype(np.int64)
    if weights == "int64_totals":
        w = _sym_weights(n, rp, col, 1 << 22, 1 << 23)
    deg = np.diff(rp)
    if scale == 15:
        assert deg.max() > 4096 and rp[-1] >= 1 << 18
    else:
        assert rp[-1] < 1 << 18
    g = make(n, rp, col, w)
    n0, rp0, col0, w0 = n, rp, col, w
    for step in range(3):
        pu, pv = [], []
        # groups of 2-6 random vertices
        for _ in range(60):
            mem = rng.choice(n, size=int(rng.integers(2, 7)), replace=False)
            pu += [int(mem[0])] * (len(mem) - 1)
            pv += [int(x) for x in mem[1:]]
        # one group of the highest-degree vertices: its rows hold more than a
        # quarter of n entries (the dense-accumulator path)
        d = np.diff(rp)
        top = np.argsort(-d, kind="stable")[:5]
        pu += [int(top[0])] * 4
        pv += [int(x) for x in top[1:]]
        # a row of 64..4096 entries whose neighbours fall into 40 groups
        cand = np.flatnonzero((d >= 64) & (d <= 4096))
        h = int(cand[rng.integers(0, len(cand))])
        nb = col[rp[h]:rp[h + 1]][:40]
        others = rng.choice(n, size=40, replace=False)
        pu += [int(x) for x in nb]
        pv += [int(x) for x in others]
        # rows whose neighbours fall into 2..6 groups (the worklist of the
        # warp-per-row kernels on large graphs)
        for _ in range(4):
            h = int(cand[rng.integers(0, len(cand))])
            k = int(rng.integers(2, 7))
            nb = col[rp[h]:rp[h + 1]][-k:]
            others = rng.choice(n, size=k, replace=False)
            pu += [int(x) for x in nb]
            pv += [int(x) for x in others]
        pu = np.asarray(pu, np.int32)
        pv = np.asarray(pv, np.int32)
        n2, L = oracle.labels_from_pairs(n, pu, pv)
        assert _singleton_entry_share(n, rp, np.asarray(L)) >= 0.25
        La = np.asarray(L)
        assert np.bincount(La, weights=d, minlength=n2).max() >= max(n2 / 4, 1024)
        ro = mc.default_round_options()
        ro.npairs = len(pu)
        ro.pair_u = pu.ctypes.data
        ro.pair_v = pv.ctypes.data
        res = mc.mincut_contract_round(g, ro)
        rp, col, w = oracle.contract(n, rp, col, w, L, n2)
        n = n2
        assert res["n_out"] == n2
        assert_csr_equal(mc.mincut_graph_export_csr(g), (rp, col, w))
    # a solve starts again from the input graph; its own rounds contract
    # row-wise too
    v, _, _ = mc.mincut_solve(g, bitmap=False)
    assert v == oracle.noi(n0, rp0, col0, w0)[0]


def test_contract_rowwise_full_size_rmat20():
    """The contraction at the size the bench times: the R-MAT scale-20
    10-core graph (29 M directed entries) contracted by groups that exercise
    every part of the entry-tiled path -- 20,000 random pairs, one group of
    the 64 highest-degree vertices (a dense accumulator), and 200 rows whose
    neighbours fall into 2..40 groups -- compared entry by entry with the
    oracle's contraction."""
    rng = np.random.default_rng(2020)
    s = synth.workload_rmat_core(20, 10, 2)
    n, rp, col, w = s.n, s.row_ptr, s.col, s.w.astype(np.int64)
    d = np.diff(rp)
    groups = np.arange(n, dtype=np.int32)
    pick = rng.choice(n, size=40000, replace=False)
    groups[pick[:20000]] = pick[20000:]
    top = np.argsort(-d, kind="stable")[:64]
    groups[top] = int(top[0])
    cand = np.flatnonzero((d >= 64) & (d <= 4096))
    for h in rng.choice(cand, size=200, replace=False):
        k = int(rng.integers(2, 41))
        nb = col[rp[h]:rp[h + 1]][-k:]
        groups[nb] = rng.choice(n, size=k, replace=False).astype(np.int32)
    n2, L = oracle.labels_from_groups(groups)
    exp = oracle.contract(n, rp, col, w, L, n2)
    g = make(n, rp, col, w)
    ro = mc.default_round_options()
    ro.groups = groups.ctypes.data
    res = mc.mincut_contract_round(g, ro)
    assert res["n_out"] == n2
    assert_csr_equal(mc.mincut_graph_export_csr(g), exp)


def test_contract_rowwise_short_rows_bit_exact():
    """Entry tiles that cover more rows than their shared-memory row table
    (rows of about two entries) find rows in the global row offsets; the
    moved labels come from about 3000 pairs and one group of 40.  Against the
    oracle's contraction."""
    rng = np.random.default_rng(31)
    s = synth.cycle_plus(150000, 0.2, 1, 9, 11)
    n, rp, col, w = s.n, s.row_ptr, s.col, s.w.astype(np.int64)
    assert rp[-1] >= 1 << 18
    assert np.diff(rp).mean() < 4
    groups = np.arange(n, dtype=np.int32)
    pick = rng.choice(n, size=6000, replace=False)
    groups[pick[:3000]] = pick[3000:]          # 3000 pairs
    groups[pick[:40]] = int(pick[0])           # one group of 40 (with their pair mates)
    n2, L = oracle.labels_from_groups(groups)
    g = make(n, rp, col, w)
    ro = mc.default_round_options()
    ro.groups = groups.ctypes.data
    res = mc.mincut_contract_round(g, ro)
    exp = oracle.contract(n, rp, col, w, L, n2)
    assert res["n_out"] == n2
    assert_csr_equal(mc.mincut_graph_export_csr(g), exp)


def test_contract_rowwise_empty_rows_bit_exact():
    """Isolated vertices (empty rows) spread through a graph large enough for
    the entry tiles: the row walks of the counting and writing passes step
    over them, and their groups stay empty rows of the contracted graph."""
    rng = np.random.default_rng(41)
    s = synth.cycle_plus(140000, 1.0, 1, 9, 13)
    n0, rp0, col0, w0 = s.n, s.row_ptr, s.col, s.w.astype(np.int64)
    # every 97th new id is an isolated vertex
    n = n0 + n0 // 90 + 10
    keep = np.ones(n, bool)
    keep[::97] = False
    new_ids = np.flatnonzero(keep)[:n0]
    n = int(new_ids[-1]) + 1
    new_of_old = new_ids
    deg_new = np.zeros(n, np.int64)
    deg_new[new_of_old] = np.diff(rp0)
    rp = np.concatenate([[0], np.cumsum(deg_new)])
    row_old = np.repeat(np.arange(n0), np.diff(rp0))
    u = new_of_old[row_old]
    v = new_of_old[col0]
    order = np.lexsort((v, u))
    col = v[order].astype(np.int32)
    w = w0[order]
    assert rp[-1] >= 1 << 18 and (np.diff(rp) == 0).sum() > 1000
    groups = np.arange(n, dtype=np.int32)
    pick = rng.choice(np.flatnonzero(np.diff(rp) > 0), size=8000, replace=False)
    groups[pick[:4000]] = pick[4000:]
    n2, L = oracle.labels_from_groups(groups)
    g = make(n, rp, col, w)
    ro = mc.default_round_options()
    ro.groups = groups.ctypes.data
    res = mc.mincut_contract_round(g, ro)
    assert res["n_out"] == n2
    assert_csr_equal(mc.mincut_graph_export_csr(g), oracle.contract(n, rp, col, w, L, n2))


# ------------------------------------------------------------------ PR flags
@pytest.mark.parametrize("budget", [-1, 3])
def test_pr_flags_bit_exact(budget):
    rng = np.random.default_rng(12)
    for trial in range(6):
        n = int(rng.integers(30, 400))
        g0 = G.random_graph(n, float(rng.uniform(0.02, 0.3)), rng, 1, int(rng.integers(1, 20)))
        c = canon(n, *g0)
        lam = int(oracle.degrees(n, *c).min())
        g = make(n, c[0], c[1], c[2])
        M = int(c[0][-1])
        flags = np.zeros(max(M, 1), np.uint8)
        ro = mc.default_round_options()
        ro.capforest = 0
        ro.lp_iters = 0
        ro.pr_budget = budget
        ro.pr_flags_out = flags.ctypes.data
        res = mc.mincut_contract_round(g, ro)
        if res["stopped"]:
            continue
        exp = oracle.pr_marks(n, *c, lam, 0xF, budget)
        assert np.array_equal(flags[:M], exp)
        src = np.repeat(np.arange(n), np.diff(c[0]))
        assert res["marks_pr"] == int(((exp != 0) & (src < c[1])).sum())


@pytest.mark.parametrize("budget,big", [(-1, False), (3, False), (-1, True)])
def test_pr_flags_bit_exact_hub_rows(budget, big):
    """Rows longer than two entry tiles (whole tiles inside one row take the
    shared-memory row index), with common neighbours among the leaves."""
    rng = np.random.default_rng(77 + budget + 5 * big)
    n = 9000
    hubs = [0, 1, 2, 4500]
    edges = set()
    for h in hubs:
        for x in rng.choice(n, size=int(rng.integers(4300, 8000)), replace=False):
            if x != h:
                edges.add((min(h, int(x)), max(h, int(x))))
    edges.update((i, i + 1) for i in range(n - 1))
    for _ in range(12000):
        a, b = (int(t) for t in rng.integers(0, n, 2))
        if a != b:
            edges.add((min(a, b), max(a, b)))
    edges = sorted(edges)
    lo, hi = ((1 << 20), (1 << 31) - 1) if big else (1, 40)  # big: int64 totals
    wts = [int(t) for t in rng.integers(lo, hi, len(edges))]
    c = canon(n, *G.from_edges(n, edges, wts))
    lam = int(oracle.degrees(n, *c).min())
    g = make(n, c[0], c[1], c[2])
    M = int(c[0][-1])
    assert int(np.diff(c[0]).max()) > 2 * 2048
    flags = np.zeros(M, np.uint8)
    ro = mc.default_round_options()
    ro.capforest = 0
    ro.lp_iters = 0
    ro.pr_budget = budget
    ro.pr_flags_out = flags.ctypes.data
    res = mc.mincut_contract_round(g, ro)
    assert not res["stopped"]
    exp = oracle.pr_marks(n, *c, lam, 0xF, budget)
    assert np.array_equal(flags, exp)
    src = np.repeat(np.arange(n), np.diff(c[0]))
    assert res["marks_pr"] == int(((exp != 0) & (src < c[1])).sum())


def _pr_clustered_graph(rng, n, big):
    """Rows of two to four heavy entries (they set the degree bound above the
    light edges' weights), rows whose ids sit in two narrow windows at both
    ends of the id range, and a light clique over one window (many common
    neighbours), so that the PR3/PR4 searches meet short and long rows,
    uneven id spreads and several search steps per lane."""
    win = list(range(0, 40)) + list(range(n - 40, n))
    hubs = [n // 2, n // 2 + 1, n // 3]
    light, heavy = {}, {}
    for h in hubs:
        for x in win:
            light[(min(h, x), max(h, x))] = int(rng.integers(1, 13))
    for i in range(40):
        for j in range(i + 1, 40):
            if rng.random() < 0.6:
                light[(i, j)] = int(rng.integers(1, 13))
    for v in range(40, n - 40):
        if v in hubs:
            continue
        for k in rng.choice(len(win), 2 + v % 3, replace=False):
            x = win[int(k)]
            heavy[(min(v, x), max(v, x))] = int(rng.integers(20, 41))
    edges = sorted(set(light) | set(heavy))
    scale = 1 << 25 if big else 1  # big: 64-bit totals
    wts = [scale * heavy.get(e, light.get(e, 0)) for e in edges]
    return canon(n, *G.from_edges(n, edges, wts))


@pytest.mark.parametrize("budget,big", [(-1, False), (16, False), (3, False), (-1, True)])
def test_pr_clustered_ids_flags_and_round_bit_exact(budget, big):
    """PR flags entry by entry, then a PR-only round without a flags output
    (the early-exit form the solve runs) contracted exactly like the
    oracle's round with the same bound and budget."""
    rng = np.random.default_rng(5 + budget + 7 * big)
    for n in (300, 2500):
        c = _pr_clustered_graph(rng, n, big)
        M = int(c[0][-1])
        lam = int(oracle.degrees(n, *c).min())
        flags = np.zeros(M, np.uint8)
        g = make(n, c[0], c[1], c[2])
        ro = mc.default_round_options()
        ro.capforest = 0
        ro.lp_iters = 0
        ro.pr_budget = budget
        ro.pr_flags_out = flags.ctypes.data
        res = mc.mincut_contract_round(g, ro)
        assert not res["stopped"]
        exp = oracle.pr_marks(n, *c, lam, 0xF, budget)
        assert np.array_equal(flags, exp)
        # the intersections decide marks that PR1/PR2 do not
        assert int(((exp & 12 != 0) & (exp & 3 == 0)).sum()) > 0
        g.destroy()
        g = make(n, c[0], c[1], c[2])
        ro = mc.default_round_options()
        ro.capforest = 0
        ro.lp_iters = 0
        ro.pr_budget = budget
        res = mc.mincut_contract_round(g, ro)
        n2, rp2, col2, w2, info = oracle.round_(n, *c, lambda_in=INF, lp_iters=0,
                                                pr_mask=0xF, pr_budget=budget, capforest=False)
        assert res["lambda_out"] == info["lambda"]
        assert res["n_out"] == n2
        assert_csr_equal(mc.mincut_graph_export_csr(g), (rp2, col2, w2))
        g.destroy()


# ------------------------------------------------ deterministic CAPFOREST pass
def _det_round(n, c, lam_in=INF, start=0, lp_iters=0, lp_min_n=10000, pr_mask=0xF,
               capforest=2):
    g = make(n, c[0], c[1], c[2])
    M = int(c[0][-1])
    order = np.zeros(n, np.int32)
    marks = np.zeros(2 * (M // 2 + 1), np.int32)
    ro = mc.default_round_options()
    ro.lambda_in = lam_in
    ro.capforest = capforest
    ro.cf_start = start
    ro.lp_iters = lp_iters
    ro.lp_min_n = lp_min_n
    ro.pr_mask = pr_mask
    ro.pr_budget = -1
    ro.cf_order_out = order.ctypes.data
    ro.cf_marks_out = marks.ctypes.data
    ro.cf_marks_cap = M // 2 + 1
    res = mc.mincut_contract_round(g, ro)
    return g, res, order[:res["cf_nscanned"]], marks[:2 * res["cf_nmarks"]].reshape(-1, 2)


@pytest.mark.parametrize("name", ["capforest_two_triangles.json", "capforest_chain.json"])
def test_sequential_pass_golden(name):
    import json, os
    d = json.load(open(os.path.join(os.path.dirname(__file__), "golden", name)))
    c = G.from_edges(d["n"], d["edges"], d["weights"])
    g, res, order, marks = _det_round(d["n"], c, d["lambda_in"], d["start"], pr_mask=0)
    assert order.tolist() == d["expect"]["order"]
    assert sorted(map(tuple, marks.tolist())) == sorted(map(tuple, d["expect"]["marks"]))
    assert res["lambda_out"] == d["expect"]["lambda_out"]


def test_sequential_pass_bit_exact_random():
    rng = np.random.default_rng(31)
    for trial in range(25):
        n = int(rng.integers(3, 3000))
        p = min(0.9, float(rng.uniform(2, 20)) / n)
        g0 = G.random_graph(n, p, rng, 1, int(rng.integers(1, 30))) if n < 200 else None
        if g0 is None:
            s = synth.er(n, int(p * n * (n - 1) / 2), 1, int(rng.integers(1, 30)), trial)
            g0 = (s.row_ptr, s.col, s.w)
        c = canon(n, *g0)
        deg = oracle.degrees(n, *c)
        lam = int(deg.min()) if n >= 2 else INF
        start = int(rng.integers(0, n))
        g, res, order, marks = _det_round(n, c, INF, start, pr_mask=0)
        if res["stopped"]:
            assert lam == 0 or n <= 2
            continue
        r = oracle.capforest(n, *c, lam, start)
        assert order.tolist() == r["order"].tolist(), trial
        assert sorted(map(tuple, marks.tolist())) == sorted(map(tuple, r["marks"].tolist())), trial
        assert res["lambda_out"] == r["lambda"]


def test_deterministic_round_bit_exact_with_pr_and_lp():
    rng = np.random.default_rng(41)
    for trial in range(12):
        n = int(rng.integers(40, 2500))
        s = synth.er_connected(n, int(n * rng.uniform(2, 8)), 1, int(rng.integers(1, 40)), trial + 100)
        c = (s.row_ptr, s.col, s.w.astype(np.int64))
        lp_iters = int(rng.integers(0, 4))
        g, res, _, _ = _det_round(n, c, INF, 0, lp_iters=lp_iters, lp_min_n=10)
        n2, rp2, col2, w2, info = oracle.round_(n, *c, lambda_in=INF, lp_iters=lp_iters,
                                                lp_min_n=10, pr_mask=0xF, pr_budget=-1,
                                                capforest=True, cf_start=0)
        assert res["lambda_out"] == info["lambda"], trial
        assert res["n_out"] == n2
        assert_csr_equal(mc.mincut_graph_export_csr(g), (rp2, col2, w2))


# --------------------------------------------------------- label propagation
def _lp_case(c, n, iters):
    g = make(n, c[0], c[1], c[2])
    lab = np.full(n, -1, np.int32)
    ro = mc.default_round_options()
    ro.lp_iters = iters
    ro.lp_min_n = 2
    ro.pr_mask = 0
    ro.capforest = 0
    ro.lp_labels_out = lab.ctypes.data
    res = mc.mincut_contract_round(g, ro)
    assert not res["stopped"]
    exp = oracle.lp(n, *c, iters)
    assert np.array_equal(lab, exp)
    deg = oracle.degrees(n, *c)
    val, _ = oracle.lp_bound(n, *c, exp)
    assert res["lambda_out"] == min(int(deg.min()), val)


def test_lp_labels_bit_exact_short_rows():
    rng = np.random.default_rng(81)
    for trial in range(6):
        n = int(rng.integers(50, 3000))
        s = synth.er_connected(n, int(n * rng.uniform(2, 6)), 1, int(rng.integers(1, 20)), trial)
        _lp_case((s.row_ptr, s.col, s.w.astype(np.int64)), n, int(rng.integers(1, 5)))


def _sym_weights(n, rp, col, lo, span):
    """Symmetric pseudo-random weights in [lo, lo + span) keyed by the edge."""
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    a = np.minimum(src, col.astype(np.int64))
    b = np.maximum(src, col.astype(np.int64))
    return lo + (a * 1000003 + b * 7919) % span


@pytest.mark.parametrize("weights", ["unit", "small", "int64_totals"])
def test_lp_labels_bit_exact_medium_and_long_rows(weights):
    # R-MAT cores have rows of every length class (warp table, small and large
    # block tables, pooled tables for rows longer than 4096)
    s = synth.workload_rmat_core(scale=15, k=8, seed=9)
    d = np.diff(s.row_ptr)
    assert ((d > 128) & (d <= 1024)).any() and ((d > 1024) & (d <= 4096)).any()
    assert (d > 4096).any()
    w = s.w.astype(np.int64)
    if weights == "small":
        w = _sym_weights(s.n, s.row_ptr, s.col, 1, 100)
    elif weights == "int64_totals":
        w = _sym_weights(s.n, s.row_ptr, s.col, 1 << 22, 1 << 23)
        assert int(w.sum()) > 2 ** 31
    for iters in (1, 2, 3):
        _lp_case((s.row_ptr, s.col, w), s.n, iters)


def test_lp_two_communities_bound():
    s = synth.planted(1 << 10, 21 << 10, 30, 3, 1, 7)
    _lp_case((s.row_ptr, s.col, s.w.astype(np.int64)), s.n, 8)


# ---------------------------------------------------------- concurrent passes
@pytest.mark.parametrize("mode", [1, 3])  # shared / private visit sets
def test_concurrent_round_sound_brute_force(mode):
    rng = np.random.default_rng(51 + mode)
    for trial in range(60):
        n = int(rng.integers(4, 15))
        g0 = G.random_graph(n, float(rng.uniform(0.2, 1.0)), rng, 1, int(rng.integers(1, 9)))
        c = canon(n, *g0)
        lam_true, _ = oracle.mincut_brute(n, *c)
        g = make(n, c[0], c[1], c[2])
        ro = mc.default_round_options()
        ro.capforest = mode
        ro.passes = int(rng.integers(1, 8))
        ro.seed = trial
        ro.lp_min_n = 4
        res = mc.mincut_contract_round(g, ro)
        rp2, col2, w2 = mc.mincut_graph_export_csr(g)
        n2 = res["n_out"]
        lam2 = oracle.mincut_brute(n2, rp2, col2, w2)[0] if n2 >= 2 else INF
        assert min(res["lambda_out"], lam2) == lam_true, trial


# ---------------------------------------------------------------- full solve
def _check_solve(n, c, opts=None, expect=None):
    g = make(n, c[0], c[1], c[2])
    v, bm, st = mc.mincut_solve(g, opts)
    if expect is None:
        expect = oracle.stoer_wagner(n, *c)[0]
    assert v == expect, (v, expect, st)
    side = mc.bitmap_to_side(bm, n)
    assert side[0] == 0 and 0 < side.sum() < n
    assert oracle.cut_weight(n, *c, side) == v
    g.destroy()
    return st


@pytest.mark.parametrize("variant", ["private", "alternate", "coarsen", "coarsen_private"])
def test_solve_paper_variants(variant):
    """The variants of Sec. 4 (visit arrays private to each pass, or the two
    settings alternated over the first rounds) and the coarsening heuristic
    of Sec. 2.1 for the first bound give the exact minimum cut and a witness
    of that weight on random, planted and R-MAT inputs."""
    kw = {"private": dict(cf_visit=1), "alternate": dict(cf_visit=2),
          "coarsen": dict(init_bound=1, lp_min_n=200),
          "coarsen_private": dict(init_bound=1, cf_visit=1, lp_min_n=200)}[variant]
    rng = np.random.default_rng(17)
    cases = []
    for trial in range(4):
        n = int(rng.integers(300, 900))
        g0 = G.random_graph(n, float(rng.uniform(0.01, 0.05)), rng, 1, 30, connected=True)
        cases.append((n, canon(n, *g0), None))
    s = synth.planted(1 << 10, 21 << 10, 30, 3, 1, 7)
    c = (s.row_ptr, s.col, s.w.astype(np.int64))
    cases.append((s.n, c, oracle.noi(s.n, *c)[0]))
    s = synth.workload_rmat_core(scale=13, k=6, seed=4)
    c = (s.row_ptr, s.col, s.w.astype(np.int64))
    cases.append((s.n, c, oracle.noi(s.n, *c)[0]))
    for n, c, exp in cases:
        st = _check_solve(n, c, mc.default_options(seed=3, **kw), expect=exp)
        if variant.startswith("coarsen") and n >= 200:
            assert st["lambda_source"] in (1, 2, 3, 4)


@pytest.mark.parametrize("kind", ["wheel", "dblcyc"])
@pytest.mark.parametrize("seq_passes,cf_visit", [(1, 0), (0, 0), (0, 1), (0, 2)])
def test_solve_adversarial_families(kind, seq_passes, cf_visit):
    """Families that defeat the PR tests (all trivial cuts minimum; a hidden
    unique minimum below many near-minimum cuts) solved exactly with the
    single sequential pass of Algorithm 2 or several whole passes at once."""
    n = 257 if kind == "wheel" else 258
    g = synth.wheel(n, seed=3) if kind == "wheel" else synth.dblcyc(n, 1000, 3, seed=3)
    c = (g.row_ptr, g.col, g.w.astype(np.int64))
    st = _check_solve(n, c, mc.default_options(seq_passes=seq_passes, cf_visit=cf_visit),
                      expect=g.meta["lambda"])
    if kind == "dblcyc" and seq_passes == 1 and cf_visit == 0:
        assert st["rounds"] > n // 4  # one merge per round: Theta(n) rounds


def test_solve_dblcyc_private_passes_then_sequential_passes():
    """Private concurrent passes that lower the bound without marking, then
    several sequential passes that do not lower it further: the witness of
    the bound stays the concurrent pass's prefix."""
    g = synth.dblcyc(1026, 1000, 3, seed=7)
    c = (g.row_ptr, g.col, g.w.astype(np.int64))
    _check_solve(g.n, c, mc.default_options(cf_visit=1, seq_passes=0), expect=2000)


def test_solve_closed_forms():
    cases = [(G.cycle(50), 50, 2), (G.complete(12), 12, 11), (G.hypercube(6), 64, 6),
             (G.grid(9, 11), 99, 2), (G.complete_bipartite(3, 9), 12, 3),
             (G.two_cliques(8, 1, 5, 3), 16, 3)]
    for c, n, lam in cases:
        _check_solve(n, canon(n, *c), expect=lam)


def test_solve_disconnected_and_isolated():
    rp, col, w = G.from_edges(9, [(0, 1), (1, 2), (3, 4), (4, 5), (5, 3), (6, 7)], [4, 4, 2, 2, 2, 9])
    _check_solve(9, canon(9, rp, col, w), expect=0)


def test_solve_random_small_vs_stoer_wagner():
    rng = np.random.default_rng(61)
    for trial in range(40):
        n = int(rng.integers(2, 60))
        g0 = G.random_graph(n, float(rng.uniform(0.05, 0.8)), rng, 1, int(rng.integers(1, 50)))
        c = canon(n, *g0)
        if int(c[0][-1]) == 0:
            continue
        opts = mc.default_options(lp_min_n=8, seed=trial, deterministic=trial % 3 == 0)
        _check_solve(n, c, opts)


def test_solve_er2000_workload():
    s = synth.workload_er2000()
    c = (s.row_ptr, s.col, s.w.astype(np.int64))
    sw = oracle.stoer_wagner(s.n, *c)[0]
    st = _check_solve(s.n, c, mc.default_options(), expect=sw)
    st2 = _check_solve(s.n, c, mc.default_options(deterministic=1), expect=sw)
    assert st["rounds"] >= 1 and st2["rounds"] >= 1


def test_solve_int64_weights():
    rng = np.random.default_rng(71)
    for trial in range(4):
        n = 120
        g0 = G.random_graph(n, 0.1, rng, 2 ** 28, 2 ** 31 - 1, connected=True)
        c = canon(n, *g0)
        assert int(c[2].sum()) > 2 ** 31
        _check_solve(n, c, mc.default_options(lp_min_n=10, seed=trial))


def test_solve_rmat_core_small():
    s = synth.workload_rmat_core(scale=14, k=10, seed=2)
    c = (s.row_ptr, s.col, s.w.astype(np.int64))
    lam, _, _ = oracle.noi(s.n, *c)
    _check_solve(s.n, c, mc.default_options(lp_min_n=1000), expect=lam)


def test_solve_planted_small():
    s = synth.planted(1 << 12, 21 << 12, 30, 25, 1, 5)
    c = (s.row_ptr, s.col, s.w.astype(np.int64))
    _check_solve(s.n, c, mc.default_options(lp_min_n=1000), expect=25)


# ------------------------------------------------------- full-size workloads
def test_solve_er2000_full_size_bitmap():
    s = synth.workload_er2000()
    c = (s.row_ptr, s.col, s.w.astype(np.int64))
    _check_solve(s.n, c, mc.default_options(), expect=oracle.noi(s.n, *c)[0])


def test_solve_rmat20_core_full_size():
    """The benchmark workload at full size, in the benchmark's configuration
    (default options): the value equals the oracle's NOI and the returned
    side's cut weight equals the value."""
    s = synth.workload_rmat_core(20, 10, 2)
    c = (s.row_ptr, s.col, s.w)
    lam, _, _ = oracle.noi(s.n, *c)
    _check_solve(s.n, c, mc.default_options(), expect=lam)


@pytest.mark.slow
def test_solve_planted21_full_size():
    """Two 2^21-vertex blocks, 25 unit cross edges (~85 M edges): the value
    equals the oracle's NOI value stored in tests/golden/planted21_noi.json
    (computed on this exact graph, identified by its CSR checksum) and the
    returned side's cut weight equals the value."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "planted21_noi.json")) as f:
        gold = json.load(f)
    s = synth.workload_planted(21, 42, 30, 25, 3)
    assert (s.n, s.m) == (gold["n"], gold["m"])
    assert G.csr_checksum(s) == gold["csr_checksum"]
    c = (s.row_ptr, s.col, s.w)
    st = _check_solve(s.n, c, mc.default_options(), expect=gold["lambda"])
    assert st["rounds"] >= 1
