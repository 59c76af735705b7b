"""The allocation-free contraction entry point (mincut_contract_csr_noalloc).

It exists for callers that cannot allocate device memory (a plug-in inside a
host application that owns the device pool, or a latency-critical loop that
cannot pay for cudaMalloc); all its scratch lives in a fixed device array
inside the library.  These tests call it through the C ABI several times in
a row -- a small graph, a larger one, then a smaller one again, so that a
call finds the previous, larger call's data in the shared array -- and check
every result entry by entry against the oracle's canonical contraction
(oracle.contract) and against the allocating path (mincut_graph_from_csr +
mincut_contract_round with the same groups): integers, so bit-exact.  Each
malformed input is rejected before any kernel reads it.  The file is named to
be collected last."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2609_07204_gb300 as mc  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mc.load_library()


def _reference(g, groups):
    G = mc.mincut_graph_from_csr(g.n, g.row_ptr, g.col, g.w)
    ro = mc.default_round_options()
    ro.groups = groups.ctypes.data
    res = mc.mincut_contract_round(G, ro)
    out = mc.mincut_graph_export_csr(G)
    G.destroy()
    return res["n_out"], out


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.device("cuda"))


def _call(g, labels, n2, *, m_directed=None, col=None, w=None, rp=None):
    dev = torch.device("cuda")
    rp_d = _dev(g.row_ptr if rp is None else rp)
    col_d = _dev(g.col if col is None else col)
    w_d = _dev(g.w if w is None else w)
    cap = max(int(col_d.numel()), 1)
    rp_out = torch.full((n2 + 1,), -7, dtype=torch.int64, device=dev)
    col_out = torch.full((cap,), -7, dtype=torch.int32, device=dev)
    w_out = torch.full((cap,), -7, dtype=torch.int32, device=dev)
    m2 = mc.mincut_contract_csr_noalloc(g.n, rp_d, col_d, w_d, _dev(labels), n2, rp_out, col_out,
                                        w_out, m_directed=m_directed)
    torch.cuda.synchronize()
    return m2, rp_out.cpu().numpy(), col_out[:m2].cpu().numpy(), w_out[:m2].cpu().numpy()


def test_noalloc_matches_oracle_and_allocating_path_several_calls():
    rng = np.random.default_rng(2024)
    # small, larger, then smaller again: the third call meets the second's
    # (larger) leftovers in the shared scratch
    for call, (n, m, seed) in enumerate([(3000, 40000, 1), (20000, 120000, 2), (900, 5000, 3)]):
        g = synth.er(n, m, 1, 50, seed)
        groups = rng.integers(0, max(n // 4, 1), size=n).astype(np.int32)
        n2, labels = oracle.labels_from_groups(groups)  # numbered by smallest member
        rp_o, col_o, w_o = oracle.contract(n, g.row_ptr, g.col, g.w, labels, n2)
        n2_ref, (rp_ref, col_ref, w_ref) = _reference(g, groups)
        assert n2 == n2_ref
        m2, rp_out, col_out, w_out = _call(g, labels, n2)
        assert m2 == int(rp_o[-1]), call
        assert np.array_equal(rp_out, rp_o), call
        assert np.array_equal(col_out, col_o), call
        assert np.array_equal(w_out.astype(np.int64), w_o), call
        # the allocating path agrees as well
        assert np.array_equal(rp_ref, rp_o) and np.array_equal(col_ref, col_o), call
        assert np.array_equal(w_ref, w_o), call


def test_noalloc_one_group_gives_empty_graph():
    g = synth.er(500, 3000, 1, 9, 5)
    labels = np.zeros(g.n, np.int32)
    m2, rp_out, col_out, _ = _call(g, labels, 1)
    assert m2 == 0 and col_out.size == 0
    assert np.array_equal(rp_out, np.zeros(2, np.int64))


def test_noalloc_identity_labels_keep_the_graph():
    g = synth.er(700, 4000, 1, 30, 6)
    labels = np.arange(g.n, dtype=np.int32)
    m2, rp_out, col_out, w_out = _call(g, labels, g.n)
    assert m2 == g.M
    assert np.array_equal(rp_out, g.row_ptr)
    assert np.array_equal(col_out, g.col) and np.array_equal(w_out, g.w)


def test_noalloc_no_entries():
    g = synth.Graph(4, np.zeros(5, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32), {})
    labels = np.array([0, 1, 1, 0], np.int32)
    m2, rp_out, _, _ = _call(g, labels, 2)
    assert m2 == 0 and np.array_equal(rp_out, np.zeros(3, np.int64))


def _rejects(status, g, labels, n2, **kw):
    with pytest.raises(mc.MincutError) as e:
        _call(g, labels, n2, **kw)
    assert e.value.status == status, mc.mincut_last_error()


def test_noalloc_rejects_malformed_inputs():
    g = synth.er(400, 2000, 1, 20, 7)
    labels = (np.arange(g.n) % 10).astype(np.int32)
    n2 = 10
    # label outside [0, n2)
    bad = labels.copy()
    bad[123] = n2
    _rejects(mc.MINCUT_ERR_INVALID, g, bad, n2)
    bad[123] = -1
    _rejects(mc.MINCUT_ERR_INVALID, g, bad, n2)
    # column outside [0, n)
    col = g.col.copy()
    col[77] = g.n
    _rejects(mc.MINCUT_ERR_INVALID, g, labels, n2, col=col)
    # negative weight
    w = g.w.copy()
    w[5] = -1
    _rejects(mc.MINCUT_ERR_INVALID, g, labels, n2, w=w)
    # row_ptr[n] != m_directed (a column buffer with spare capacity)
    _rejects(mc.MINCUT_ERR_INVALID, g, labels, n2, m_directed=g.M - 2)
    # row_ptr[0] != 0
    rp = g.row_ptr.copy()
    rp[0] = 1
    _rejects(mc.MINCUT_ERR_INVALID, g, labels, n2, rp=rp)
    # decreasing row offsets (ends still right)
    rp = g.row_ptr.copy()
    rp[200] = rp[202] + 1
    _rejects(mc.MINCUT_ERR_INVALID, g, labels, n2, rp=rp)
    # weights whose sum exceeds 2^31 - 1 (the contracted weights are int32)
    w = np.full(g.M, (1 << 31) // g.M + 1, np.int32)
    _rejects(mc.MINCUT_ERR_OVERFLOW, g, labels, n2, w=w)
    # after the rejections a valid call still works
    m2, rp_out, col_out, w_out = _call(g, labels, n2)
    rp_o, col_o, w_o = oracle.contract(g.n, g.row_ptr, g.col, g.w, labels, n2)
    assert np.array_equal(rp_out, rp_o) and np.array_equal(col_out, col_o)
    assert np.array_equal(w_out.astype(np.int64), w_o)


def test_noalloc_rejects_oversized_graph():
    dev = torch.device("cuda")
    n = (1 << 18) + 1
    rp = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    z = torch.zeros(1, dtype=torch.int32, device=dev)
    lab = torch.zeros(n, dtype=torch.int32, device=dev)
    rp_out = torch.zeros(2, dtype=torch.int64, device=dev)
    with pytest.raises(mc.MincutError) as e:
        mc.mincut_contract_csr_noalloc(n, rp, z, z, lab, 1, rp_out, z, z)
    assert e.value.status == mc.MINCUT_ERR_OVERFLOW
    assert "262144" in mc.mincut_last_error()
