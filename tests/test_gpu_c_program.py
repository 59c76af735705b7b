"""The C ABI used from a plain C99 program on the GPU: the program builds a
weighted cycle (host CSR), solves it with the library defaults and reports
the value, the weight of the cut its side bitmap names and the side's size.
A weighted cycle's minimum cut is the sum of its two lightest edges (Sec. 2:
every proper cut of a cycle crosses at least two of its edges)."""
import os
import shutil
import subprocess

import pytest

import paper_2609_07204_gb300 as mc

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r'''
#include <stdio.h>
#include <stdlib.h>
#include "mincut.h"
static int32_t weight(int64_t i) { return (int32_t)(3 + (i * 7919) % 97); }
int main(int argc, char** argv) {
    const int64_t n = argc > 1 ? atoll(argv[1]) : 1000;
    int64_t* rp = malloc((size_t)(n + 1) * sizeof(int64_t));
    int32_t* col = malloc((size_t)(2 * n) * sizeof(int32_t));
    int32_t* w = malloc((size_t)(2 * n) * sizeof(int32_t));
    uint64_t* bm = calloc((size_t)((n + 63) / 64), sizeof(uint64_t));
    for (int64_t i = 0; i < n; ++i) {  /* row i: i-1 and i+1 (mod n), sorted */
        const int64_t a = (i + n - 1) % n, b = (i + 1) % n;
        const int32_t wa = weight(a), wb = weight(i);
        rp[i] = 2 * i;
        col[2 * i] = (int32_t)(a < b ? a : b);
        w[2 * i] = a < b ? wa : wb;
        col[2 * i + 1] = (int32_t)(a < b ? b : a);
        w[2 * i + 1] = a < b ? wb : wa;
    }
    rp[n] = 2 * n;
    mincut_graph* g = NULL;
    int rc = mincut_graph_from_csr(n, rp, col, w, MINCUT_HOST_PTRS, NULL, NULL, &g);
    if (rc != MINCUT_OK) { fprintf(stderr, "create: %s\n", mincut_last_error()); return 1; }
    int64_t lambda = -1;
    mincut_stats st;
    rc = mincut_solve(g, NULL, &lambda, bm, &st);
    if (rc != MINCUT_OK) { fprintf(stderr, "solve: %s\n", mincut_last_error()); return 2; }
    int64_t cutw = 0, ones = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t j = (i + 1) % n;
        const int si = (int)((bm[i / 64] >> (i % 64)) & 1), sj = (int)((bm[j / 64] >> (j % 64)) & 1);
        if (si != sj) cutw += weight(i);
        ones += si;
    }
    printf("%lld %lld %lld %d\n", (long long)lambda, (long long)cutw, (long long)ones,
           (int)(bm[0] & 1));
    mincut_graph_destroy(g);
    free(rp); free(col); free(w); free(bm);
    return 0;
}
'''


@pytest.mark.parametrize("n", [3, 1000, 70001])
def test_c_program_solves_weighted_cycle(tmp_path, n):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    mc.load_library()
    src = tmp_path / "cycle.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "cycle"
    libdir = os.path.dirname(mc.LIB_PATH)
    subprocess.check_call([gcc, "-std=c99", "-O2", "-Wall", "-Werror", "-I",
                           os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                           "-L", libdir, "-lmincut", f"-Wl,-rpath,{libdir}"])
    r = subprocess.run([str(exe), str(n)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-1000:]
    lam, cutw, ones, bit0 = (int(x) for x in r.stdout.split())
    ws = sorted(3 + (i * 7919) % 97 for i in range(n))
    assert lam == ws[0] + ws[1]
    assert cutw == lam and 0 < ones < n and bit0 == 0
