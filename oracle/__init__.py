"""CPU oracle for the exact minimum-cut contraction round -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library in
``paper_2609_07204_gb300`` and its binding) never does; the two share no code.

The arithmetic lives in plain C (``oracle.c``, int64 throughout, compiled with
gcc on first use).  This module only marshals numpy arrays through ctypes.
Functions and the passages of the paper they follow:

* ``cut_weight``        -- cut capacity (Sec. 2, Basic Concepts)
* ``mincut_brute``      -- lambda by enumerating all 2^(n-1)-1 cuts (Sec. 2)
* ``st_cut_brute``      -- lambda(G, s, t) by enumeration (Sec. 2)
* ``stoer_wagner``      -- Stoer-Wagner (App. A; the independent check of App. C)
* ``degrees``           -- weighted degree (Sec. 2)
* ``labels_from_groups`` / ``labels_from_pairs`` -- canonical contracted ids
* ``contract``          -- contraction with parallel edges summed (Sec. 2)
* ``pr_marks``          -- Padberg-Rinaldi tests PR1-PR4 (Sec. 2.1, App. A; reading)
* ``capforest``         -- one CAPFOREST pass (Algorithm 1, one process; Sec. 2.1)
* ``lp`` / ``lp_bound`` -- label propagation and its cluster bound (Sec. 2.1; reading)
* ``round_``            -- one deterministic contraction round (Algorithms 1-2)
* ``noi``               -- the sequential exact algorithm (Algorithm 2, one process)

Parity status: every function above is pinned by tests/test_oracle_*.py; the
labels produced by ``lp`` only by hand-traced sweeps (tests/golden/lp_trace.json)
and small rule checks, since no closed form fixes them on larger graphs (the
bound derived from them is pinned as the cut value of an explicit set).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None
INF = (1 << 63) - 1

_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")


class RoundOpts(ctypes.Structure):
    _fields_ = [("lambda_in", ctypes.c_int64), ("lp_iters", ctypes.c_int32),
                ("lp_min_n", ctypes.c_int32), ("pr_mask", ctypes.c_uint32),
                ("pr_budget", ctypes.c_int64), ("capforest", ctypes.c_int32),
                ("cf_start", ctypes.c_int32)]


class RoundRes(ctypes.Structure):
    _fields_ = [("lambda_out", ctypes.c_int64), ("n2", ctypes.c_int32), ("M2", ctypes.c_int64),
                ("marks_pr", ctypes.c_int64), ("marks_cf", ctypes.c_int64),
                ("stopped", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc -O2, plain C11)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
            os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_SO)
    i32, i64, u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    vp = ctypes.c_void_p
    lib.orc_degrees.argtypes = [i32, _i64p, _i32p, _i64p, _i64p]
    lib.orc_cut_weight.argtypes = [i32, _i64p, _i32p, _i64p, _u8p]
    lib.orc_cut_weight.restype = i64
    lib.orc_mincut_brute.argtypes = [i32, _i64p, _i32p, _i64p, _u8p]
    lib.orc_mincut_brute.restype = i64
    lib.orc_st_cut_brute.argtypes = [i32, _i64p, _i32p, _i64p, i32, i32]
    lib.orc_st_cut_brute.restype = i64
    lib.orc_stoer_wagner.argtypes = [i32, _i64p, _i32p, _i64p, _u8p]
    lib.orc_stoer_wagner.restype = i64
    lib.orc_labels_from_groups.argtypes = [i32, _i32p, _i32p]
    lib.orc_labels_from_groups.restype = i32
    lib.orc_labels_from_pairs.argtypes = [i32, i64, _i32p, _i32p, _i32p]
    lib.orc_labels_from_pairs.restype = i32
    lib.orc_contract.argtypes = [i32, _i64p, _i32p, _i64p, _i32p, i32, _i64p, _i32p, _i64p]
    lib.orc_contract.restype = i64
    lib.orc_pr_marks.argtypes = [i32, _i64p, _i32p, _i64p, i64, u32, i64, _u8p]
    lib.orc_capforest.argtypes = [i32, _i64p, _i32p, _i64p, i64, i32, vp, vp, vp, vp, vp, vp, vp]
    lib.orc_capforest.restype = i64
    lib.orc_capforest_tie.argtypes = [i32, _i64p, _i32p, _i64p, i64, i32, i32, vp, vp, vp, vp,
                                      vp, vp, vp]
    lib.orc_capforest_tie.restype = i64
    lib.orc_lp.argtypes = [i32, _i64p, _i32p, _i64p, i32, _i32p]
    lib.orc_lp_bound.argtypes = [i32, _i64p, _i32p, _i64p, _i32p, vp]
    lib.orc_lp_bound.restype = i64
    lib.orc_round.argtypes = [i32, _i64p, _i32p, _i64p, ctypes.POINTER(RoundOpts), _i64p, _i32p,
                              _i64p, ctypes.POINTER(RoundRes)]
    lib.orc_round.restype = ctypes.c_int
    lib.orc_noi.argtypes = [i32, _i64p, _i32p, _i64p, _u8p, vp]
    lib.orc_noi.restype = i64
    _lib = lib
    return lib


def _csr(rp, col, w):
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.int64)
    if col.size == 0:
        col = np.zeros(1, np.int32)
        w = np.zeros(1, np.int64)
    return rp, col, w


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def degrees(n, rp, col, w):
    rp, col, w = _csr(rp, col, w)
    out = np.zeros(max(n, 1), np.int64)
    _load().orc_degrees(n, rp, col, w, out)
    return out[:n]


def cut_weight(n, rp, col, w, side):
    rp, col, w = _csr(rp, col, w)
    side = np.ascontiguousarray(side, dtype=np.uint8)
    return int(_load().orc_cut_weight(n, rp, col, w, side))


def mincut_brute(n, rp, col, w):
    """(lambda, side) by enumeration; n <= 26."""
    rp, col, w = _csr(rp, col, w)
    side = np.zeros(max(n, 1), np.uint8)
    v = int(_load().orc_mincut_brute(n, rp, col, w, side))
    return v, side[:n]


def st_cut_brute(n, rp, col, w, s, t):
    rp, col, w = _csr(rp, col, w)
    return int(_load().orc_st_cut_brute(n, rp, col, w, s, t))


def stoer_wagner(n, rp, col, w):
    """(lambda, side) by Stoer-Wagner."""
    rp, col, w = _csr(rp, col, w)
    side = np.zeros(max(n, 1), np.uint8)
    v = int(_load().orc_stoer_wagner(n, rp, col, w, side))
    return v, side[:n]


def labels_from_groups(group):
    group = np.ascontiguousarray(group, dtype=np.int32)
    n = group.shape[0]
    L = np.zeros(max(n, 1), np.int32)
    n2 = int(_load().orc_labels_from_groups(n, group if n else np.zeros(1, np.int32), L))
    return n2, L[:n]


def labels_from_pairs(n, pu, pv):
    pu = np.ascontiguousarray(pu, dtype=np.int32)
    pv = np.ascontiguousarray(pv, dtype=np.int32)
    k = pu.shape[0]
    L = np.zeros(max(n, 1), np.int32)
    n2 = int(_load().orc_labels_from_pairs(n, k, pu if k else np.zeros(1, np.int32),
                                           pv if k else np.zeros(1, np.int32), L))
    return n2, L[:n]


def contract(n, rp, col, w, L, n2):
    """Canonical contraction by dense labels L (values in [0, n2))."""
    rp, col, w = _csr(rp, col, w)
    L = np.ascontiguousarray(L, dtype=np.int32)
    M = int(rp[n])
    rp2 = np.zeros(n2 + 1, np.int64)
    col2 = np.zeros(max(M, 1), np.int32)
    w2 = np.zeros(max(M, 1), np.int64)
    M2 = int(_load().orc_contract(n, rp, col, w, L if n else np.zeros(1, np.int32), n2, rp2,
                                  col2, w2))
    return rp2, col2[:M2].copy(), w2[:M2].copy()


def canonicalize(n, rp, col, w):
    """Contraction with identity labels: sorted rows, duplicates summed,
    self-loops and zero weights dropped."""
    return contract(n, rp, col, w, np.arange(n, dtype=np.int32), n)


def pr_marks(n, rp, col, w, lam, mask=0xF, budget=-1):
    rp, col, w = _csr(rp, col, w)
    M = int(rp[n])
    fl = np.zeros(max(M, 1), np.uint8)
    _load().orc_pr_marks(n, rp, col, w, int(min(lam, INF)), mask, budget, fl)
    return fl[:M]


def capforest(n, rp, col, w, lam, start=0, tie=0):
    """One CAPFOREST pass.  Returns dict(lambda, marks (k,2), order, q, best_len).
    tie 0: ties of highest priority to the smaller vertex id; tie 1: to the
    first unvisited vertex of the last scanned row, else the smaller id."""
    rp, col, w = _csr(rp, col, w)
    M = int(rp[n])
    mu = np.zeros(M // 2 + 1, np.int32)
    mv = np.zeros(M // 2 + 1, np.int32)
    nm = np.zeros(1, np.int64)
    order = np.zeros(max(n, 1), np.int32)
    ns = np.zeros(1, np.int32)
    q = np.zeros(max(M, 1), np.int64)
    bl = np.zeros(1, np.int32)
    lam2 = int(_load().orc_capforest_tie(n, rp, col, w, int(min(lam, INF)), start, int(tie),
                                         _ptr(mu), _ptr(mv), _ptr(nm), _ptr(order), _ptr(ns),
                                         _ptr(q), _ptr(bl)))
    k = int(nm[0])
    return {"lambda": lam2, "marks": np.stack([mu[:k], mv[:k]], axis=1),
            "order": order[:int(ns[0])].copy(), "q": q[:M].copy(), "best_len": int(bl[0])}


def lp(n, rp, col, w, iters):
    rp, col, w = _csr(rp, col, w)
    lab = np.zeros(max(n, 1), np.int32)
    _load().orc_lp(n, rp, col, w, iters, lab)
    return lab[:n]


def lp_bound(n, rp, col, w, label):
    rp, col, w = _csr(rp, col, w)
    label = np.ascontiguousarray(label, dtype=np.int32)
    bl = np.zeros(1, np.int32)
    v = int(_load().orc_lp_bound(n, rp, col, w, label, _ptr(bl)))
    return v, int(bl[0])


def round_(n, rp, col, w, lambda_in=INF, lp_iters=0, lp_min_n=10000, pr_mask=0xF, pr_budget=-1,
           capforest=True, cf_start=0):
    """One deterministic round.  Returns (n2, rp2, col2, w2, info dict)."""
    rp, col, w = _csr(rp, col, w)
    M = int(rp[n])
    o = RoundOpts(int(min(lambda_in, INF)), lp_iters, lp_min_n, pr_mask, pr_budget,
                  1 if capforest else 0, cf_start)
    res = RoundRes()
    rp2 = np.zeros(n + 1, np.int64)
    col2 = np.zeros(max(M, 1), np.int32)
    w2 = np.zeros(max(M, 1), np.int64)
    _load().orc_round(n, rp, col, w, ctypes.byref(o), rp2, col2, w2, ctypes.byref(res))
    n2, M2 = int(res.n2), int(res.M2)
    info = {"lambda": int(res.lambda_out), "marks_pr": int(res.marks_pr),
            "marks_cf": int(res.marks_cf), "stopped": bool(res.stopped)}
    return n2, rp2[:n2 + 1].copy(), col2[:M2].copy(), w2[:M2].copy(), info


def noi(n, rp, col, w):
    """(lambda, side, rounds) by sequential NOI."""
    rp, col, w = _csr(rp, col, w)
    side = np.zeros(max(n, 1), np.uint8)
    rounds = np.zeros(1, np.int32)
    v = int(_load().orc_noi(n, rp, col, w, side, _ptr(rounds)))
    return v, side[:n], int(rounds[0])
