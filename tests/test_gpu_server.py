"""Serving loop (continuous batching): requests submitted together are
admitted as workers and memory free up, small ones solved as packed batches.
Every served value equals the oracle's Stoer-Wagner value of that request
(the independent exact check of App. C) and its value solved alone (exact
integers, tolerance 0); each returned side has that cut weight."""
from concurrent.futures import ThreadPoolExecutor

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


@pytest.fixture(scope="module")
def requests_small():
    return [synth.serving_request(5, i, 100, 3000) for i in range(96)]


@pytest.fixture(scope="module")
def oracle_values(requests_small):
    # the oracle's C code runs with the GIL released: one request per thread
    with ThreadPoolExecutor(max_workers=16) as ex:
        return list(ex.map(lambda g: oracle.stoer_wagner(g.n, g.row_ptr, g.col, g.w)[0],
                           requests_small))


def _alone(g):
    G = mc.mincut_graph_from_csr(g.n, g.row_ptr, g.col, g.w)
    v, _, _ = mc.mincut_solve(G)
    G.destroy()
    return v


def test_server_results_equal_oracle_and_alone(requests_small, oracle_values):
    S = mc.Server(workers=4, pack_max_n=1500, pack_max_requests=32)
    ids = [S.submit(g.n, g.row_ptr, g.col, g.w) for g in requests_small]
    res = [S.wait(i) for i in ids]
    st = S.stats()
    S.close()
    assert st["completed"] == len(requests_small)
    assert st["packed_batches"] >= 1 and st["single_solves"] >= 1
    assert st["peak_inflight"] > 1
    for g, want, (v, lat, bm) in zip(requests_small, oracle_values, res):
        assert v == want
        assert v == _alone(g)
        side = mc.bitmap_to_side(bm, g.n)
        assert side[0] == 0 and 0 < side.sum() < g.n
        assert oracle.cut_weight(g.n, g.row_ptr, g.col, g.w, side) == v
        assert lat >= 0


def test_server_admission_cap_serialises(requests_small, oracle_values):
    sub = requests_small[:12]
    S = mc.Server(workers=4, hbm_cap_bytes=1, pack_max_requests=1)
    ids = [S.submit(g.n, g.row_ptr, g.col, g.w) for g in sub]
    vals = [S.wait(i)[0] for i in ids]
    st = S.stats()
    S.close()
    assert st["peak_inflight"] == 1  # every request exceeds the cap: one at a time
    assert vals == oracle_values[:12]
    assert vals == [_alone(g) for g in sub]


def test_server_rejects_bad_request():
    S = mc.Server(workers=1)
    with pytest.raises(mc.MincutError):
        S.submit(1, np.zeros(2, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32))
    S.close()


def test_server_borrowed_pinned_requests_equal_oracle(requests_small, oracle_values):
    """Requests submitted without a copy (the server reads the caller's pinned
    arrays in place until wait returns) give the oracle's values."""
    sub = requests_small[:40]
    pinned = [(g.n, torch.from_numpy(g.row_ptr).pin_memory().numpy(),
               torch.from_numpy(g.col).pin_memory().numpy(),
               torch.from_numpy(g.w).pin_memory().numpy()) for g in sub]
    S = mc.Server(workers=4, pack_max_n=1500, pack_max_requests=16)
    ids = [S.submit(n, rp, col, w, borrow=True) for (n, rp, col, w) in pinned]
    vals = [S.wait(i)[0] for i in ids]
    S.close()
    assert vals == oracle_values[:40]
