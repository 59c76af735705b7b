"""Host-side checks of the C ABI (CPU only): the library loads, exports every
function include/mincut.h declares, and rejects bad arguments before any
device work."""
import ctypes
import os

import numpy as np
import pytest

import paper_2609_07204_gb300 as mc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(mc.LIB_PATH):
        from paper_2609_07204_gb300 import _build
        _build.build()
    return mc.load_library()


def test_exports_every_declared_symbol(lib):
    syms = mc.exported_symbols()
    assert "mincut_graph_from_csr" in syms and "mincut_solve" in syms
    assert "mincut_contract_round" in syms
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_struct_sizes_match_header(lib):
    # the ctypes mirrors must match the C layout field by field
    assert ctypes.sizeof(mc.MincutOptions) == 88
    assert ctypes.sizeof(mc.MincutStats) == 64
    o = mc.default_options()
    assert (o.lp_iters, o.lp_min_n, o.lp_every_round, o.pr_mask, o.pr_budget) == (2, 10000, 0, 0xF, 16)
    assert (o.init_bound, o.cf_visit, o.seq_passes, o.batch_small_n, o.seq_kernel) == (0, 0, 0, 0, 0)
    ro = mc.default_round_options()
    assert ro.lambda_in == mc.INT64_MAX and ro.capforest == 1


def test_status_strings(lib):
    for s in range(-6, 1):
        assert mc.mincut_status_string(s)
    assert mc.mincut_status_string(-99) == "unknown status"


def test_rejects_n_below_2_without_device_work(lib):
    rp = np.zeros(2, np.int64)
    with pytest.raises(mc.MincutError) as e:
        mc.mincut_graph_from_csr(1, rp, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert e.value.status == mc.MINCUT_ERR_INVALID
    assert "n >= 2" in mc.mincut_last_error()


def test_rejects_bad_row_ptr_start(lib):
    rp = np.array([1, 1, 1], np.int64)
    with pytest.raises(mc.MincutError) as e:
        mc.mincut_graph_from_csr(2, rp, np.zeros(1, np.int32), np.zeros(1, np.int32))
    assert e.value.status == mc.MINCUT_ERR_INVALID


def test_null_arguments(lib):
    out = ctypes.c_void_p(0)
    rc = lib.mincut_graph_from_csr(4, None, None, None, 0, None, None, ctypes.byref(out))
    assert rc == mc.MINCUT_ERR_INVALID
    v = ctypes.c_int64(0)
    assert lib.mincut_solve(None, None, ctypes.byref(v), None, None) == mc.MINCUT_ERR_INVALID
    assert lib.mincut_graph_reset(None) == mc.MINCUT_ERR_INVALID
    lib.mincut_graph_destroy(None)  # ignored


def test_release_cached_rejects_bad_device(lib):
    assert lib.mincut_release_cached(-1) == mc.MINCUT_ERR_INVALID
    assert lib.mincut_release_cached(64) == mc.MINCUT_ERR_INVALID


def test_package_fails_loudly_without_library(tmp_path):
    with pytest.raises(RuntimeError, match="missing"):
        mc.load_library(str(tmp_path / "nope.so"))


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2609_07204_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "oracle.c" not in text and "liboracle" not in text, f


def test_batch_rejects_bad_offsets_before_device_work(lib):
    rp = np.array([0, 1, 2, 3, 4], np.int64)
    col = np.array([1, 0, 3, 2], np.int32)
    w = np.ones(4, np.int32)
    for vo, what in (([1, 2, 4], "vertex_offsets[0]"), ([0, 1, 4], "fewer than 2"),
                     ([0, 2, 2, 4], "fewer than 2")):
        with pytest.raises(mc.MincutError) as e:
            mc.mincut_batch_from_csr(np.array(vo, np.int64), rp, col, w)
        assert e.value.status == mc.MINCUT_ERR_INVALID
        assert what in mc.mincut_last_error()
    out = ctypes.c_void_p(0)
    vo = np.array([0], np.int64)
    assert lib.mincut_batch_from_csr(0, vo.ctypes.data, rp.ctypes.data, col.ctypes.data,
                                     w.ctypes.data, 0, None, None,
                                     ctypes.byref(out)) == mc.MINCUT_ERR_INVALID
    assert lib.mincut_batch_from_csr(1, None, None, None, None, 0, None, None,
                                     ctypes.byref(out)) == mc.MINCUT_ERR_INVALID


def test_server_rejects_bad_options_and_requests(lib):
    for kw in ({"workers": 0}, {"workers": 65}, {"hbm_cap_bytes": 0}):
        o = mc.server_default_options(**kw)
        out = ctypes.c_void_p(0)
        assert lib.mincut_server_create(ctypes.byref(o), ctypes.byref(out)) == mc.MINCUT_ERR_INVALID
        assert not out.value
    rid = ctypes.c_uint64(0)
    rp = np.array([0, 1, 2], np.int64)
    assert lib.mincut_server_submit(None, 2, rp.ctypes.data, None, None,
                                    ctypes.byref(rid)) == mc.MINCUT_ERR_INVALID


def test_footprint_estimate(lib):
    """The admission estimate: -1 for negative sizes, monotone in both sizes,
    and at least the input CSR and its two contracted copies."""
    assert mc.mincut_graph_footprint(-1, 10) == -1
    assert mc.mincut_graph_footprint(10, -1) == -1
    prev = 0
    for n, M in ((2, 2), (1000, 16000), (247_314, 29_031_216), (4 << 20, 170 << 20)):
        f = mc.mincut_graph_footprint(n, M)
        assert f > prev and f >= 3 * (8 * (n + 1) + 8 * M)
        assert mc.mincut_graph_footprint(n + 1, M) > f
        assert mc.mincut_graph_footprint(n, M + 1) > f
        prev = f


def test_size_limits_rejected_before_device_work(lib):
    out = ctypes.c_void_p(0)
    one = np.zeros(4, np.int32)
    rp = np.zeros(4, np.int64)
    rc = lib.mincut_graph_from_csr(1 << 31, rp.ctypes.data, one.ctypes.data, one.ctypes.data,
                                   mc.MINCUT_HOST_PTRS, None, None, ctypes.byref(out))
    assert rc == mc.MINCUT_ERR_OVERFLOW and "2^31-2" in mc.mincut_last_error()
    rp = np.array([0, 0, 1 << 31], np.int64)  # M = 2^31 entries
    rc = lib.mincut_graph_from_csr(2, rp.ctypes.data, one.ctypes.data, one.ctypes.data,
                                   mc.MINCUT_HOST_PTRS, None, None, ctypes.byref(out))
    assert rc == mc.MINCUT_ERR_OVERFLOW and "2^31-1" in mc.mincut_last_error()
    assert not out.value


def test_plain_c_program_links_and_calls_the_abi(lib, tmp_path):
    """The header is plain C99 (no C++), and a C program linked against the
    library calls it without a GPU: default options, status strings, the
    n >= 2 rejection and the footprint estimate."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "mincut.h"
int main(void) {
    mincut_options o;
    mincut_default_options(&o);
    if (o.lp_iters != 2 || o.pr_mask != 0xF) return 1;
    if (strcmp(mincut_status_string(-99), "unknown status") != 0) return 2;
    int64_t rp[2] = {0, 0};
    int32_t c[1] = {0}, w[1] = {0};
    mincut_graph* g = NULL;
    if (mincut_graph_from_csr(1, rp, c, w, MINCUT_HOST_PTRS, NULL, NULL, &g) != MINCUT_ERR_INVALID)
        return 3;
    if (g != NULL) return 4;
    if (mincut_graph_footprint(-1, 0) != -1) return 5;
    printf("ok\n");
    return 0;
}
''')
    exe = tmp_path / "abi"
    libdir = os.path.dirname(mc.LIB_PATH)
    subprocess.check_call([gcc, "-std=c99", "-Wall", "-Werror", "-pedantic",
                           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                           "-L", libdir, "-lmincut", f"-Wl,-rpath,{libdir}"])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stderr[-500:])
