"""Seeded synthetic inputs shared by the CPU oracle tests, the CUDA parity tests
and the benchmark.

Input construction only: this module draws graphs (Erdos-Renyi, R-MAT, k-core
and largest-component reductions, the planted two-block cut, the small graphs
of the batched workload) and contains none of the minimum-cut arithmetic.
The generators are plain C (``synth.c``) reached through ctypes; the shared
object is compiled with gcc on first use (or by ``__graft_entry__.build()``).

Every graph is returned as a symmetric CSR ``(row_ptr int64[n+1], col
int32[M], w int32[M])`` with sorted rows, no duplicates and no self-loops.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_SO = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


class _CGraph(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("m", ctypes.c_int64),
        ("row_ptr", ctypes.POINTER(ctypes.c_int64)),
        ("col", ctypes.POINTER(ctypes.c_int32)),
        ("w", ctypes.POINTER(ctypes.c_int32)),
    ]


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so next to it (gcc, -O2)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.check_call(
                ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        G = ctypes.POINTER(_CGraph)
        i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
        lib.synth_er.argtypes = [i64, i64, i32, i32, u64, G]
        lib.synth_rmat.argtypes = [ctypes.c_int, i64, dbl, dbl, dbl, i32, i32, u64, G]
        lib.synth_core_lcc.argtypes = [G, i64, ctypes.c_int, G, ctypes.POINTER(ctypes.POINTER(i32))]
        lib.synth_planted.argtypes = [i64, i64, i64, i64, i32, u64, G,
                                      ctypes.POINTER(ctypes.POINTER(ctypes.c_uint8))]
        lib.synth_cycle_plus.argtypes = [i64, dbl, i32, i32, u64, G]
        lib.synth_wheel.argtypes = [i64, u64, G]
        lib.synth_dblcyc.argtypes = [i64, i32, i32, u64, G]
        lib.synth_truncate_lcc.argtypes = [G, i64, ctypes.c_int, G]
        lib.synth_batch_params.argtypes = [u64, i64, i64, i64, dbl, dbl, ctypes.POINTER(i64),
                                           ctypes.POINTER(dbl), ctypes.POINTER(u64)]
        lib.synth_splitmix64.argtypes = [u64, ctypes.POINTER(u64)]
        lib.synth_splitmix64.restype = u64
        lib.synth_free.argtypes = [G]
        libc = ctypes.CDLL(None)
        libc.free.argtypes = [ctypes.c_void_p]
        lib._libc = libc
        _lib = lib
    return _lib


@dataclass
class Graph:
    """A symmetric CSR graph: ``row_ptr`` int64[n+1], ``col`` int32[M], ``w`` int32[M]."""
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    meta: dict

    @property
    def M(self) -> int:
        return int(self.col.shape[0])

    @property
    def m(self) -> int:
        return self.M // 2


def _take(g: _CGraph, meta: dict) -> Graph:
    lib = _load()
    n = int(g.n)
    M = int(g.row_ptr[n]) if n >= 0 else 0
    rp = np.ctypeslib.as_array(g.row_ptr, shape=(n + 1,)).copy()
    col = np.ctypeslib.as_array(g.col, shape=(max(M, 1),))[:M].copy()
    w = np.ctypeslib.as_array(g.w, shape=(max(M, 1),))[:M].copy()
    lib.synth_free(ctypes.byref(g))
    return Graph(n, rp, col, w, meta)


def splitmix64(state: int) -> tuple[int, int]:
    """One SplitMix64 step: returns (value, next_state)."""
    nxt = ctypes.c_uint64(0)
    v = _load().synth_splitmix64(ctypes.c_uint64(state), ctypes.byref(nxt))
    return int(v), int(nxt.value)


def er(n: int, m: int, wlo: int = 1, whi: int = 1, seed: int = 1) -> Graph:
    """G(n, m): m distinct uniform pairs, weights uniform in [wlo, whi]."""
    g = _CGraph()
    rc = _load().synth_er(n, m, wlo, whi, seed, ctypes.byref(g))
    if rc != 0:
        raise ValueError(f"synth_er({n}, {m}) failed: {rc}")
    return _take(g, {"kind": "er", "n": n, "m": m, "seed": seed})


def _reduce(g0: Graph, k: int, lcc: bool) -> tuple[Graph, np.ndarray]:
    lib = _load()
    cg = _CGraph()
    cg.n = g0.n
    cg.m = g0.m
    cg.row_ptr = g0.row_ptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    cg.col = g0.col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    cg.w = g0.w.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    out = _CGraph()
    old = ctypes.POINTER(ctypes.c_int32)()
    lib.synth_core_lcc(ctypes.byref(cg), k, 1 if lcc else 0, ctypes.byref(out), ctypes.byref(old))
    n2 = int(out.n)
    old_ids = np.ctypeslib.as_array(old, shape=(max(n2, 1),))[:n2].copy()
    lib._libc.free(ctypes.cast(old, ctypes.c_void_p))
    return _take(out, dict(g0.meta)), old_ids


def core_lcc(g: Graph, k: int, lcc: bool = True) -> Graph:
    """k-core (edge-count peeling) then the largest connected component."""
    g2, _ = _reduce(g, k, lcc)
    g2.meta.update({"kcore": k, "lcc": lcc})
    return g2


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         wlo: int = 1, whi: int = 1, seed: int = 2) -> Graph:
    """R-MAT with a random id permutation, deduplicated, self-loops removed."""
    g = _CGraph()
    rc = _load().synth_rmat(scale, edge_factor, a, b, c, wlo, whi, seed, ctypes.byref(g))
    if rc != 0:
        raise ValueError("synth_rmat failed")
    return _take(g, {"kind": "rmat", "scale": scale, "edge_factor": edge_factor, "seed": seed})


def planted(nb: int, mb: int, kcore: int, cross: int, cross_w: int = 1, seed: int = 3) -> Graph:
    """Two G(nb, mb) unit-weight blocks, each reduced to its kcore-core, joined
    by ``cross`` random edges of weight ``cross_w``; ids randomly permuted.
    ``meta['block']`` is the 0/1 block of every vertex."""
    lib = _load()
    g = _CGraph()
    bl = ctypes.POINTER(ctypes.c_uint8)()
    rc = lib.synth_planted(nb, mb, kcore, cross, cross_w, seed, ctypes.byref(g), ctypes.byref(bl))
    if rc != 0:
        raise ValueError(f"synth_planted failed: {rc}")
    n = int(g.n)
    block = np.ctypeslib.as_array(bl, shape=(n,)).copy()
    lib._libc.free(ctypes.cast(bl, ctypes.c_void_p))
    out = _take(g, {"kind": "planted", "nb": nb, "mb": mb, "kcore": kcore, "cross": cross,
                    "seed": seed})
    out.meta["block"] = block
    return out


def wheel(n: int, seed: int = 6) -> Graph:
    """Hub plus a rim cycle of n-1 vertices, spokes 2, rim edges n-2: every
    vertex has weighted degree 2(n-1) = lambda (all trivial cuts minimum)."""
    g = _CGraph()
    if _load().synth_wheel(n, seed, ctypes.byref(g)) != 0:
        raise ValueError(f"synth_wheel({n}) failed")
    return _take(g, {"kind": "wheel", "n": n, "seed": seed, "lambda": 2 * (n - 1)})


def dblcyc(n: int, heavy: int = 1000, light: int = 3, seed: int = 7) -> Graph:
    """Hamiltonian cycle of weight `heavy` plus a stride-2 cycle of weight
    `light` on each half (n = 2h, h odd): lambda = 2*heavy, the halves."""
    g = _CGraph()
    if _load().synth_dblcyc(n, heavy, light, seed, ctypes.byref(g)) != 0:
        raise ValueError(f"synth_dblcyc({n}) failed")
    return _take(g, {"kind": "dblcyc", "n": n, "seed": seed, "lambda": 2 * heavy})


def cycle_plus(n: int, d: float, wlo: int = 1, whi: int = 100, seed: int = 4) -> Graph:
    """Random Hamiltonian cycle plus random extra pairs up to ceil(n*d/2) edges."""
    g = _CGraph()
    rc = _load().synth_cycle_plus(n, d, wlo, whi, seed, ctypes.byref(g))
    if rc != 0:
        raise ValueError("synth_cycle_plus failed")
    return _take(g, {"kind": "cycle_plus", "n": n, "d": d, "seed": seed})


def batch_params(seed: int, i: int, nlo: int = 20, nhi: int = 2000, dlo: float = 3.0,
                 dhi: float = 12.0) -> tuple[int, float, int]:
    """(n, avg degree, graph seed) of graph i of a batched workload."""
    n = ctypes.c_int64(0)
    d = ctypes.c_double(0)
    s = ctypes.c_uint64(0)
    _load().synth_batch_params(seed, i, nlo, nhi, dlo, dhi, ctypes.byref(n), ctypes.byref(d),
                               ctypes.byref(s))
    return int(n.value), float(d.value), int(s.value)


def batch_graph(seed: int, i: int, nlo: int = 20, nhi: int = 2000) -> Graph:
    """Graph i of the batched workload (cycle plus extras, weights in [1, 100])."""
    n, d, s = batch_params(seed, i, nlo, nhi)
    g = cycle_plus(n, d, 1, 100, s)
    g.meta.update({"batch_index": i})
    return g


def truncate_lcc(g: Graph, nkeep: int, lcc: bool = True) -> Graph:
    """Induced subgraph on the vertices with id < nkeep, then the largest
    connected component."""
    lib = _load()
    cg = _CGraph()
    cg.n = g.n
    cg.m = g.m
    cg.row_ptr = g.row_ptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    cg.col = g.col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    cg.w = g.w.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    out = _CGraph()
    lib.synth_truncate_lcc(ctypes.byref(cg), nkeep, 1 if lcc else 0, ctypes.byref(out))
    return _take(out, dict(g.meta))


def serving_request(seed: int, i: int, nlo: int = 100, nhi: int = 1 << 20, wlo: int = 1,
                    whi: int = 100) -> Graph:
    """Request i of a serving stream: n log-uniform in [nlo, nhi]; with
    probability 1/2 R-MAT (a=.57, b=.19, c=.19) of scale ceil(log2 n), edge
    factor 16, truncated to n vertices, else G(n, 8n) (average degree 16);
    weights uniform in [wlo, whi]; the largest connected component is kept."""
    v, s = splitmix64(seed ^ (0xA0761D6478BD642F * (i + 1) & ((1 << 64) - 1)))
    u, s = splitmix64(s)
    kind, s = splitmix64(s)
    sub, s = splitmix64(s)
    x = (u >> 11) / float(1 << 53)
    n = int(math.floor(math.exp(math.log(nlo) + x * (math.log(nhi) - math.log(nlo)))))
    n = max(nlo, min(nhi, n))
    if kind & 1:
        scale = max(1, int(math.ceil(math.log2(n))))
        g = rmat(scale, 16, 0.57, 0.19, 0.19, wlo, whi, sub)
        g = truncate_lcc(g, n, True)
        kind_s = "rmat"
    else:
        m = min(8 * n, n * (n - 1) // 2)
        g = truncate_lcc(er(n, m, wlo, whi, sub), n, True)
        kind_s = "er"
    g.meta.update({"kind": kind_s, "request": i, "n_drawn": n})
    return g


# ---------------------------------------------------------------- workloads
def er_connected(n: int, m: int, wlo: int, whi: int, seed: int) -> Graph:
    """G(n, m) with the first seed >= ``seed`` whose graph is connected."""
    s = seed
    while True:
        g = er(n, m, wlo, whi, s)
        g2, _ = _reduce(g, 0, True)
        if g2.n == n:
            g.meta["seed"] = s
            return g
        s += 1


def workload_er2000(seed: int = 1) -> Graph:
    """Connected G(n=2000, m=16000), weights uniform in [1, 10]."""
    g = er_connected(2000, 16000, 1, 10, seed)
    g.meta["workload"] = "er_n2000_m16000_w1-10"
    return g


def workload_rmat_core(scale: int = 20, k: int = 10, seed: int = 2) -> Graph:
    """R-MAT(a=.57, b=.19, c=.19), edge factor 16, unit weights, k-core, LCC."""
    g = rmat(scale, 16, 0.57, 0.19, 0.19, 1, 1, seed)
    g = core_lcc(g, k, True)
    g.meta["workload"] = f"rmat{scale}_ef16_{k}core_lcc"
    return g


def workload_planted(log_nb: int = 21, avg_deg: int = 42, kcore: int = 30, cross: int = 25,
                     seed: int = 3) -> Graph:
    """Two G(2^log_nb, avg_deg/2 * 2^log_nb) blocks, each kcore-pruned, joined by
    ``cross`` unit cross edges (lambda = cross when both blocks stay dense).
    The 30-core of G(n, p) appears only above an average degree of about 40,
    so at 40 a small block's core can vanish; 42 keeps most of each block."""
    nb = 1 << log_nb
    g = planted(nb, nb * avg_deg // 2, kcore, cross, 1, seed)
    g.meta["workload"] = f"planted_2x2^{log_nb}_deg{avg_deg}_{kcore}core_cross{cross}"
    return g


def check_csr(g: Graph) -> None:
    """Assert the CSR invariants the generators promise (sorted, symmetric)."""
    n, rp, col, w = g.n, g.row_ptr, g.col, g.w
    assert rp.shape == (n + 1,) and rp[0] == 0 and rp[-1] == col.shape[0]
    assert np.all(np.diff(rp) >= 0)
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    assert np.all(col >= 0) and np.all(col < n)
    assert np.all(src != col)
    key = src * n + col
    assert np.all(np.diff(key) > 0), "rows not strictly sorted"
    rkey = col.astype(np.int64) * n + src
    order = np.argsort(rkey, kind="stable")
    assert np.array_equal(rkey[order], key), "not symmetric"
    assert np.array_equal(w[order], w), "weights not symmetric"
    assert np.all(w > 0)
