"""The allocation-free contraction entry point (mincut_contract_csr_noalloc).

It exists for callers that cannot allocate device memory (a plug-in inside a
host application that owns the device pool, or a latency-critical loop that
cannot pay for cudaMalloc); all its scratch lives in a fixed device array
inside the library.  This test calls it through the C ABI twice in a row and
checks each result against the allocating path (mincut_graph_from_csr +
mincut_contract_round with the same groups): integers, so bit-exact.  The
file is named to be collected last."""
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


def test_noalloc_matches_allocating_path_two_calls():
    rng = np.random.default_rng(2024)
    for call, (n, m, seed) in enumerate([(3000, 40000, 1), (20000, 120000, 2)]):
        g = synth.er(n, m, 1, 50, seed)
        groups = rng.integers(0, n // 4, size=n).astype(np.int32)
        n2, labels = oracle.labels_from_groups(groups)  # numbered by smallest member
        n2_ref, (rp_ref, col_ref, w_ref) = _reference(g, groups)
        assert n2 == n2_ref
        dev = torch.device("cuda")
        rp = torch.from_numpy(g.row_ptr).to(dev)
        col = torch.from_numpy(g.col).to(dev)
        w = torch.from_numpy(g.w).to(dev)
        lab = torch.from_numpy(labels).to(dev)
        rp_out = torch.empty(n2 + 1, dtype=torch.int64, device=dev)
        col_out = torch.empty(g.M, dtype=torch.int32, device=dev)
        w_out = torch.empty(g.M, dtype=torch.int32, device=dev)
        m2 = mc.mincut_contract_csr_noalloc(n, rp, col, w, lab, n2, rp_out, col_out, w_out)
        torch.cuda.synchronize()
        assert m2 == int(rp_ref[-1]), call
        assert np.array_equal(rp_out.cpu().numpy(), rp_ref), call
        assert np.array_equal(col_out[:m2].cpu().numpy(), col_ref), call
        assert np.array_equal(w_out[:m2].cpu().numpy().astype(np.int64), w_ref), call


def test_noalloc_rejects_oversized_graph():
    dev = torch.device("cuda")
    n = (1 << 18) + 1
    rp = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    z = torch.zeros(1, dtype=torch.int32, device=dev)
    lab = torch.zeros(n, dtype=torch.int32, device=dev)
    with pytest.raises(mc.MincutError) as e:
        mc.mincut_contract_csr_noalloc(n, rp, z, z, lab, 1, rp, z, z)
    assert e.value.status == mc.MINCUT_ERR_OVERFLOW
    assert "262144" in mc.mincut_last_error()
