"""Pins for the seeded input generators shared by the oracle tests, the GPU
tests and the benchmark: SplitMix64's published outputs, the CSR form every
generator promises, and the structure each workload recipe states (sizes,
weight ranges, degree closed forms, the planted blocks, k-cores checked
against networkx, the batched workload's size distribution).  CPU only."""
import math

import numpy as np
import pytest

import synth



def _edges(g):
    """Undirected edges (u < v) with weights, from the symmetric CSR."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    keep = src < g.col
    return src[keep], g.col[keep].astype(np.int64), g.w[keep].astype(np.int64)


def _nx(g, weight_filter=None):
    nx = pytest.importorskip("networkx")
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    for u, v, w in zip(*_edges(g)):
        if weight_filter is None or weight_filter(w):
            G.add_edge(int(u), int(v), weight=int(w))
    return G


def _wdeg(g):
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    return np.bincount(src, weights=g.w.astype(np.int64), minlength=g.n).astype(np.int64)


def _same(a, b):
    return (a.n == b.n and np.array_equal(a.row_ptr, b.row_ptr)
            and np.array_equal(a.col, b.col) and np.array_equal(a.w, b.w))


def test_splitmix64_published_outputs():
    """The first outputs of SplitMix64 from state 0, as printed by the
    generator's public-domain reference implementation (S. Vigna)."""
    s = 0
    out = []
    for _ in range(3):
        v, s = synth.splitmix64(s)
        out.append(v)
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # the state advances by the golden-ratio increment
    assert s == (3 * 0x9E3779B97F4A7C15) % (1 << 64)


def test_er_exact_size_weights_and_determinism():
    g = synth.er(300, 2000, 3, 9, 11)
    synth.check_csr(g)
    assert g.n == 300 and len(g.col) == 4000
    assert g.w.min() == 3 and g.w.max() == 9
    assert set(np.unique(g.w)) == set(range(3, 10))
    assert abs(g.w.mean() - 6.0) < 0.2
    assert _same(g, synth.er(300, 2000, 3, 9, 11))
    assert not _same(g, synth.er(300, 2000, 3, 9, 12))
    # the complete graph is the largest G(n, m)
    k = synth.er(12, 66, 1, 1, 5)
    assert np.all(np.diff(k.row_ptr) == 11)


def test_rmat_is_skewed_and_core_lcc_matches_networkx():
    nx = pytest.importorskip("networkx")
    g = synth.rmat(12, 16, 0.57, 0.19, 0.19, 1, 1, 5)
    synth.check_csr(g)
    assert g.n == 4096 and np.all(g.w == 1)
    deg = np.diff(g.row_ptr)
    assert deg.max() > 20 * deg.mean()  # heavy-tailed degrees
    c = synth.core_lcc(g, 10, True)
    synth.check_csr(c)
    # the 10-core by networkx, then its largest component
    K = nx.k_core(_nx(g), 10)
    big = max(nx.connected_components(K), key=len)
    H = K.subgraph(big)
    assert c.n == H.number_of_nodes() and len(c.col) == 2 * H.number_of_edges()
    assert np.diff(c.row_ptr).min() >= 10
    assert nx.is_connected(_nx(c))
    # relabelled densely in increasing old id: the degree sequences agree
    old = sorted(big)
    assert np.array_equal(np.diff(c.row_ptr), [H.degree(v) for v in old])


def test_planted_blocks_cross_edges_and_cores():
    cross, cross_w, k = 25, 3, 30
    g = synth.planted(1 << 10, 21 << 10, k, cross, cross_w, 3)
    synth.check_csr(g)
    block = g.meta["block"]
    assert block.shape == (g.n,) and set(np.unique(block)) == {0, 1}
    u, v, w = _edges(g)
    x = block[u] != block[v]
    # the cross edges carry cross * cross_w in total (a repeated pair sums)
    assert w[x].sum() == cross * cross_w and 1 <= x.sum() <= cross
    assert np.all(w[~x] == 1)
    # inside its block every vertex keeps at least k neighbours (k-core)
    inside = np.bincount(np.concatenate([u[~x], v[~x]]), minlength=g.n)
    assert inside.min() >= k
    # with unit cross edges (the planted workload) the block split is
    # lighter than every single-vertex cut
    g1 = synth.planted(1 << 10, 21 << 10, k, cross, 1, 3)
    assert cross < k <= _wdeg(g1).min()


def test_wheel_degrees_closed_form():
    for n in (5, 9, 64):
        g = synth.wheel(n, seed=n)
        synth.check_csr(g)
        assert len(g.col) == 4 * (n - 1)
        assert np.all(_wdeg(g) == 2 * (n - 1))
        deg = np.diff(g.row_ptr)
        assert sorted(deg.tolist()) == [3] * (n - 1) + [n - 1]


def test_dblcyc_heavy_hamiltonian_and_light_half_cycles():
    nx = pytest.importorskip("networkx")
    for n, heavy, light in ((10, 1000, 3), (22, 7, 2), (102, 50, 1)):
        h = n // 2
        g = synth.dblcyc(n, heavy, light, seed=n)
        synth.check_csr(g)
        assert len(g.col) == 4 * n
        assert np.all(_wdeg(g) == 2 * heavy + 2 * light)
        Hh = _nx(g, lambda w: w == heavy)
        assert Hh.number_of_edges() == n and nx.is_connected(Hh)
        assert all(d == 2 for _, d in Hh.degree())  # one Hamiltonian cycle
        Hl = _nx(g, lambda w: w == light)
        comps = [c for c in nx.connected_components(Hl)]
        assert sorted(len(c) for c in comps) == [h, h]  # one cycle per half
        assert all(d == 2 for _, d in Hl.degree())
    with pytest.raises(ValueError):
        synth.dblcyc(12)  # the half must be odd


def test_cycle_plus_size_connectivity_and_weights():
    nx = pytest.importorskip("networkx")
    for n, d in ((3, 10.0), (50, 3.0), (500, 6.0), (800, 11.5)):
        g = synth.cycle_plus(n, d, 1, 100, 9 + n)
        synth.check_csr(g)
        m = min(max(n, math.ceil(n * d / 2)), n * (n - 1) // 2)
        assert len(g.col) == 2 * m
        assert np.diff(g.row_ptr).min() >= 2  # the Hamiltonian cycle
        assert nx.is_connected(_nx(g))
        assert g.w.min() >= 1 and g.w.max() <= 100


def test_batched_workload_distribution():
    """4096 graphs: n log-uniform on [20, 2000], average degree uniform on
    [3, 12]; the totals of the batched workload with seed 4."""
    ns, ds, ms = [], [], []
    for i in range(4096):
        n, d, _ = synth.batch_params(4, i)
        assert 20 <= n <= 2000 and 3.0 <= d <= 12.0
        ns.append(n)
        ds.append(d)
        ms.append(min(max(n, math.ceil(n * d / 2)), n * (n - 1) // 2))
    assert sum(ns) == 1_781_764 and sum(ms) == 6_751_902
    # E[ln n] = (ln 20 + ln 2000) / 2 and E[d] = 7.5, within four standard errors
    mid = (math.log(20) + math.log(2000)) / 2
    assert abs(np.mean(np.log(ns)) - mid) < 4 * math.log(100) / math.sqrt(12 * 4096)
    assert abs(np.mean(ds) - 7.5) < 4 * 9 / math.sqrt(12 * 4096)
    g = synth.batch_graph(4, 7)
    n, d, _ = synth.batch_params(4, 7)
    assert g.n == n and g.meta["batch_index"] == 7


def test_serving_requests_connected_and_mixed():
    nx = pytest.importorskip("networkx")
    kinds = set()
    for i in range(40):
        g = synth.serving_request(5, i, 100, 3000)
        synth.check_csr(g)
        assert 2 <= g.n <= g.meta["n_drawn"] <= 3000
        assert g.w.min() >= 1 and g.w.max() <= 100
        assert nx.is_connected(_nx(g))
        kinds.add(g.meta["kind"])
    assert kinds == {"rmat", "er"}


def test_workload_sizes_as_documented():
    """The single-solve workloads: G(2000, 16000) connected with weights in
    [1, 10]; the R-MAT scale-20 10-core with n = 247,314 and m = 14,515,608."""
    nx = pytest.importorskip("networkx")
    c1 = synth.workload_er2000()
    synth.check_csr(c1)
    assert c1.n == 2000 and len(c1.col) == 32000
    assert c1.w.min() == 1 and c1.w.max() == 10
    assert nx.is_connected(_nx(c1))
    c2 = synth.workload_rmat_core()
    assert c2.n == 247_314 and len(c2.col) == 2 * 14_515_608
    assert np.diff(c2.row_ptr).min() >= 10 and np.all(c2.w == 1)
