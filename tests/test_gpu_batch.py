"""Packed batch solve (many independent graphs in one CSR) against the oracle:
every graph's value equals the oracle's, and every graph's side (from the
shared bitmap) has that cut weight with both sides non-empty."""
import numpy as np
import pytest

import oracle
import synth
from tests import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2609_07204_gb300 as mc  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mc.load_library()


def _check_batch(graphs, expect, opts=None):
    vo, rp, col, w = mc.pack_graphs(graphs)
    B = mc.mincut_batch_from_csr(vo, rp, col, w)
    vals, bm, st = mc.mincut_batch_solve(B, opts)
    side_all = mc.bitmap_to_side(bm, int(vo[-1]))
    for i, (n, grp, gcol, gw) in enumerate(graphs):
        assert vals[i] == expect[i], (i, n, vals[i], expect[i])
        side = side_all[vo[i]:vo[i + 1]]
        assert side[0] == 0 and 0 < side.sum() < n, i
        assert oracle.cut_weight(n, grp, gcol, gw, side) == vals[i], i
    B.destroy()
    return st


def test_batch_random_small_graphs():
    rng = np.random.default_rng(91)
    graphs, expect = [], []
    for i in range(300):
        n = int(rng.integers(2, 50))
        g = G.random_graph(n, float(rng.uniform(0.05, 0.9)), rng, 1, int(rng.integers(1, 60)))
        c = oracle.canonicalize(n, *g)
        graphs.append((n, c[0], c[1], c[2]))
        expect.append(oracle.stoer_wagner(n, *c)[0])
    _check_batch(graphs, expect)
    _check_batch(graphs, expect, mc.default_options(deterministic=1))
    # every graph in the shared round kernels; every graph on its own warp;
    # both at once
    for small in (-1, 2048, 20):
        _check_batch(graphs, expect, mc.default_options(batch_small_n=small))


def test_batch_closed_forms_and_disconnected():
    cases = [(G.cycle(30), 30, 2), (G.complete(9), 9, 8), (G.hypercube(5), 32, 5),
             (G.grid(6, 7), 42, 2), (G.two_cliques(7, 1, 6, 2), 14, 2),
             (G.from_edges(5, [(0, 1), (2, 3)], [4, 4]), 5, 0),
             (G.from_edges(2, [(0, 1)], [7]), 2, 7)]
    graphs = []
    for c, n, lam in cases:
        cc = oracle.canonicalize(n, *c)
        graphs.append((n, cc[0], cc[1], cc[2]))
    for small in (0, -1, 2048, 10):
        _check_batch(graphs, [lam for _, _, lam in cases], mc.default_options(batch_small_n=small))


def test_batch_workload_subset_vs_noi():
    graphs, expect = [], []
    for i in range(256):
        s = synth.batch_graph(4, i)
        graphs.append((s.n, s.row_ptr, s.col, s.w.astype(np.int64)))
        expect.append(oracle.noi(s.n, s.row_ptr, s.col, s.w)[0])
    _check_batch(graphs, expect)  # threshold chosen by timing
    st = _check_batch(graphs, expect, mc.default_options(batch_small_n=-1))
    assert st["rounds"] >= 1
    st = _check_batch(graphs, expect, mc.default_options(batch_small_n=2048))
    assert st["rounds"] == 0  # every graph solved by its own warp
    _check_batch(graphs, expect, mc.default_options(batch_small_n=300))


def test_batch_warp_path_weighted_and_pr_variants():
    """The one-warp-per-graph solver on weighted graphs up to its size
    limit, with and without the PR tests (it applies PR1 / PR2 of the mask),
    against Stoer-Wagner."""
    rng = np.random.default_rng(17)
    graphs, expect = [], []
    for i in range(24):
        n = int(rng.integers(100, 700)) if i % 4 else 2048
        s = synth.er_connected(n, int(n * rng.uniform(2.0, 7.0)), 1, 100, 300 + i)
        c = (s.row_ptr, s.col, s.w.astype(np.int64))
        graphs.append((n, *c))
        expect.append(oracle.stoer_wagner(n, *c)[0])
    for mask in (0xF, 0x1, 0x0):
        _check_batch(graphs, expect, mc.default_options(batch_small_n=2048, pr_mask=mask))


def _solve_and_check(B, vo, graphs, expect, opts):
    vals, bm, st = mc.mincut_batch_solve(B, opts)
    side_all = mc.bitmap_to_side(bm, int(vo[-1]))
    for i, (n, grp, gcol, gw) in enumerate(graphs):
        assert vals[i] == expect[i], (i, n, vals[i], expect[i])
        side = side_all[vo[i]:vo[i + 1]]
        assert side[0] == 0 and 0 < side.sum() < n, i
        assert oracle.cut_weight(n, grp, gcol, gw, side) == vals[i], i
    return st


@pytest.mark.parametrize("own_stream", [False, True])
def test_batch_repeated_solves_replay_captured_launches(own_stream):
    """Solving the same batch again (every graph on its own warp) replays the
    launches captured as a CUDA graph at the second solve; a changed PR mask,
    a round-kernel solve in between (which swaps the offsets buffer) and a
    profiled solve take the direct launches or a new capture.  Every solve
    matches the oracle."""
    graphs, expect = [], []
    for i in range(160):
        s = synth.batch_graph(4, 1000 + i)
        graphs.append((s.n, s.row_ptr, s.col, s.w.astype(np.int64)))
        expect.append(oracle.noi(s.n, s.row_ptr, s.col, s.w)[0])
    vo, rp, col, w = mc.pack_graphs(graphs)
    strm = torch.cuda.Stream() if own_stream else None
    B = mc.mincut_batch_from_csr(vo, rp, col, w, stream=strm)
    warp = mc.default_options(batch_small_n=2048)
    launches = set()
    for _ in range(4):
        launches.add(_solve_and_check(B, vo, graphs, expect, warp)["kernel_launches"])
    assert len(launches) == 1  # the replayed graph launches the same kernels
    for _ in range(3):
        _solve_and_check(B, vo, graphs, expect, mc.default_options(batch_small_n=2048, pr_mask=0x1))
    _solve_and_check(B, vo, graphs, expect, mc.default_options(batch_small_n=-1))
    for _ in range(3):
        _solve_and_check(B, vo, graphs, expect, warp)
    _solve_and_check(B, vo, graphs, expect, mc.default_options(batch_small_n=2048, profile=1))
    _solve_and_check(B, vo, graphs, expect, warp)
    B.destroy()


def test_batch_rejects_cross_graph_edge_and_tiny_graph():
    c1 = oracle.canonicalize(3, *G.cycle(3))
    c2 = oracle.canonicalize(3, *G.cycle(3))
    vo, rp, col, w = mc.pack_graphs([(3, *c1), (3, *c2)])
    col = col.copy()
    col[0] = 4  # 0 -> 4 crosses into the second graph (and breaks symmetry)
    with pytest.raises(mc.MincutError) as e:
        mc.mincut_batch_from_csr(vo, rp, col, w, skip_validate=True)
    assert e.value.status == mc.MINCUT_ERR_INVALID
    vo2 = np.array([0, 1, 6], np.int64)
    with pytest.raises(mc.MincutError):
        mc.mincut_batch_from_csr(vo2, rp, col, w)
