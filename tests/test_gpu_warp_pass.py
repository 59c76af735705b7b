"""The warp-driven whole-graph CAPFOREST pass (the sequential pass of
Algorithm 2, one warp per pass, neighbour-first ties) against the oracle's
CAPFOREST with the same tie rule (oracle.capforest(..., tie=1)): visit
order, marks (in scan order) and the returned bound are equal entry by entry
(integers).  The cases cover every key width (8-, 16-, 32-bit priorities),
r[] and the tree levels in shared or global memory, rows longer than one
batch of 128 entries, 64-bit weights, a bound lowered by alpha and a
disconnected graph.  Full solves on the default path (several such passes
per round) are checked against Stoer-Wagner / NOI in test_gpu_parity.py."""
import numpy as np
import pytest

import oracle
import synth
from tests import graphs as G
from tests.test_gpu_parity import INF, _check_solve, _det_round, canon

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2609_07204_gb300 as mc  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mc.load_library()


def _compare(n, c, start, tag):
    deg = oracle.degrees(n, *c)
    lam = int(deg.min())
    g, res, order, marks = _det_round(n, c, INF, start, pr_mask=0, capforest=4)
    g.destroy()
    if res["stopped"]:
        assert lam == 0 or n <= 2, tag
        return None
    r = oracle.capforest(n, *c, lam, start, tie=1)
    assert res["seq_pass"] == 1, tag
    assert order.tolist() == r["order"].tolist(), tag
    assert marks.tolist() == r["marks"].tolist(), tag
    assert res["lambda_out"] == r["lambda"], tag
    return r


def test_warp_pass_small_graphs_bit_exact():
    """n < 3000: r[], the tree and (when it fits) the CSR in shared memory."""
    rng = np.random.default_rng(61)
    for trial in range(30):
        n = int(rng.integers(3, 3000))
        p = min(0.9, float(rng.uniform(2, 20)) / n)
        if n < 200:
            g0 = G.random_graph(n, p, rng, 1, int(rng.integers(1, 30)))
        else:
            s = synth.er(n, int(p * n * (n - 1) / 2), 1, int(rng.integers(1, 30)), trial)
            g0 = (s.row_ptr, s.col, s.w)
        c = canon(n, *g0)
        _compare(n, c, int(rng.integers(0, n)), trial)


@pytest.mark.parametrize("wlo,whi,key_bytes", [(1, 1, 1), (100, 300, 2), (1, 200000, 4)])
def test_warp_pass_key_widths_global_r(wlo, whi, key_bytes):
    """60,000 vertices (r[] in global memory): unit weights keep the bound
    under 255 (8-bit keys), weights in [100, 300] under 65,535 (16-bit),
    weights to 200,000 need 32-bit keys."""
    n = 60000
    s = synth.er(n, 8 * n, wlo, whi, 7 + whi)
    c = (s.row_ptr, s.col, s.w.astype(np.int64))
    lam = int(oracle.degrees(n, *c).min())
    assert {1: lam <= 254, 2: 254 < lam <= 65534, 4: 65534 < lam}[key_bytes], lam
    r = _compare(n, c, 123, (wlo, whi, key_bytes))
    assert r is not None and len(r["marks"]) > 0


def test_warp_pass_global_tree_level():
    """1.8 M vertices with 32-bit keys: the lowest tree level (225 KB) does
    not fit in shared memory and lives in global memory."""
    n = 1_800_000
    s = synth.er(n, 10 * n, 100000, 300000, 11)
    c = (s.row_ptr, s.col, s.w.astype(np.int64))
    assert int(oracle.degrees(n, *c).min()) > 65534
    r = _compare(n, c, 5, "global level 1")
    assert r is not None and len(r["order"]) == n


def test_warp_pass_long_rows_and_alpha():
    """A planted cut between two dense blocks with a hub of 600 neighbours:
    rows longer than a 128-entry batch, and alpha lowers the bound to the
    planted cut during the pass."""
    s = synth.planted(1 << 11, 24 << 11, 20, 3, 1, 9)
    n = s.n
    rp, col, w = s.row_ptr, s.col, s.w.astype(np.int64)
    # add a hub: vertex 0 joined to 600 others of its block (weight 1)
    block = np.asarray(s.meta["block"])
    others = [v for v in range(1, n) if block[v] == block[0]][:600]
    edges = set()
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            if u < col[e]:
                edges.add((u, int(col[e]), int(w[e])))
    have = {(a, b) for a, b, _ in edges}
    for v in others:
        if (0, v) not in have:
            edges.add((0, v, 1))
    el = sorted(edges)
    rp2, col2, w2 = G.from_edges(n, [(a, b) for a, b, _ in el], [c for _, _, c in el])
    c = canon(n, rp2, col2, w2)
    assert int(np.diff(c[0]).max()) > 512
    r = _compare(n, c, 0, "hub")
    assert r["lambda"] == 3 and r["best_len"] > 0


def test_warp_pass_int64_weights():
    """Total weight above 2^31: 64-bit sums; the bound still fits 32-bit keys."""
    n = 3000
    s = synth.er(n, 6 * n, 100000, 1000000, 13)
    c = (s.row_ptr, s.col, s.w.astype(np.int64))
    assert int(c[2].sum()) > (1 << 31)
    _compare(n, c, 17, "int64")


def test_warp_pass_disconnected():
    """Two components: the pass stops when its component is exhausted; the
    visited prefix is a cut of weight 0."""
    a = synth.er(500, 3000, 1, 9, 21)
    b = synth.er(400, 2000, 1, 9, 22)
    n = 900
    rp = np.concatenate([a.row_ptr, a.row_ptr[-1] + b.row_ptr[1:]])
    col = np.concatenate([a.col, b.col + 500])
    w = np.concatenate([a.w, b.w]).astype(np.int64)
    r = _compare(n, (rp, col, w), 3, "disconnected")
    assert r["lambda"] == 0 and len(r["order"]) == 500


def test_solve_default_and_block_pass_kernels_agree():
    """Full solves on the default path (warp passes) and with the block
    passes (seq_kernel = 1) give the oracle's value on graphs that need the
    sequential pass."""
    rng = np.random.default_rng(71)
    for trial in range(6):
        n = int(rng.integers(200, 2500))
        s = synth.er_connected(n, int(n * rng.uniform(3, 8)), 1, 20, 300 + trial)
        c = (s.row_ptr, s.col, s.w.astype(np.int64))
        want = oracle.stoer_wagner(n, *c)[0]
        for kern in (0, 1):
            for sp in (0, 1, 3):
                _check_solve(n, c, mc.default_options(seq_kernel=kern, seq_passes=sp),
                             expect=want)
