"""Python binding of libmincut.so, the GB300 exact minimum-cut library.

Argument marshalling only: every step of a solve runs in the CUDA kernels of
``libmincut.so`` (see ``include/mincut.h``).  The names follow the C ABI:

    g = mincut_graph_from_csr(n, row_ptr, col, w)     # numpy (host) or torch CUDA tensors
    value, side_bitmap, stats = mincut_solve(g)
    res = mincut_contract_round(g, round_options)
    n, M = mincut_graph_info(g); rp, col, w = mincut_graph_export_csr(g)
    mincut_graph_reset(g); mincut_graph_destroy(g)

PyTorch supplies device memory (optionally through its caching allocator,
``use_torch_allocator=True``) and the CUDA stream.  There is no CPU fallback:
importing works anywhere, but every call raises if libmincut.so is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import Any, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmincut.so")
INT64_MAX = (1 << 63) - 1

MINCUT_OK = 0
MINCUT_ERR_INVALID = -1
MINCUT_ERR_OOM = -2
MINCUT_ERR_OVERFLOW = -3
MINCUT_ERR_DEVICE_TIMEOUT = -4
MINCUT_ERR_CUDA = -5
MINCUT_ERR_INTERNAL = -6

MINCUT_HOST_PTRS = 0
MINCUT_DEVICE_PTRS = 1
MINCUT_SKIP_VALIDATE = 2


class MincutError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mincut status {status}: {msg}")
        self.status = status


class MincutOptions(ctypes.Structure):
    _fields_ = [("lp_iters", ctypes.c_int32), ("lp_min_n", ctypes.c_int32),
                ("lp_every_round", ctypes.c_int32), ("pr_mask", ctypes.c_uint32),
                ("pr_budget", ctypes.c_int64), ("passes", ctypes.c_int32),
                ("pass_table", ctypes.c_int32), ("waves", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("deterministic", ctypes.c_int32),
                ("max_rounds", ctypes.c_int32), ("spin_limit", ctypes.c_int64),
                ("profile", ctypes.c_int32), ("init_bound", ctypes.c_int32),
                ("cf_visit", ctypes.c_int32), ("seq_passes", ctypes.c_int32),
                ("batch_small_n", ctypes.c_int32), ("seq_kernel", ctypes.c_int32)]


class MincutStats(ctypes.Structure):
    _fields_ = [("n_input", ctypes.c_int64), ("m_input", ctypes.c_int64),
                ("rounds", ctypes.c_int32), ("seq_passes", ctypes.c_int32),
                ("marks_pr", ctypes.c_int64), ("marks_cf", ctypes.c_int64),
                ("entries_processed", ctypes.c_int64), ("lambda_source", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int32), ("ms_total", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class MincutRoundOptions(ctypes.Structure):
    _fields_ = [("lambda_in", ctypes.c_int64), ("lp_iters", ctypes.c_int32),
                ("lp_min_n", ctypes.c_int32), ("pr_mask", ctypes.c_uint32),
                ("pr_budget", ctypes.c_int64), ("capforest", ctypes.c_int32),
                ("cf_start", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("pass_table", ctypes.c_int32), ("waves", ctypes.c_int32),
                ("seed", ctypes.c_uint64),
                ("groups", ctypes.c_void_p), ("npairs", ctypes.c_int64),
                ("pair_u", ctypes.c_void_p), ("pair_v", ctypes.c_void_p),
                ("pr_flags_out", ctypes.c_void_p), ("cf_order_out", ctypes.c_void_p),
                ("cf_marks_out", ctypes.c_void_p), ("cf_marks_cap", ctypes.c_int64),
                ("lp_labels_out", ctypes.c_void_p)]


class MincutRoundResult(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int64), ("m_in", ctypes.c_int64), ("n_out", ctypes.c_int64),
                ("m_out", ctypes.c_int64), ("lambda_out", ctypes.c_int64),
                ("marks_pr", ctypes.c_int64), ("marks_cf", ctypes.c_int64),
                ("stopped", ctypes.c_int32), ("seq_pass", ctypes.c_int32),
                ("cf_nscanned", ctypes.c_int64), ("cf_nmarks", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                            ctypes.c_void_p)


class MincutAllocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", ctypes.c_void_p)]


class MincutProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64),
                ("units", ctypes.c_int64), ("ms", ctypes.c_double)]


class MincutServerOptions(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("pack_max_requests", ctypes.c_int32),
                ("hbm_cap_bytes", ctypes.c_int64), ("pack_max_n", ctypes.c_int64),
                ("pack_max_vertices", ctypes.c_int64), ("want_bitmap", ctypes.c_int32),
                ("device", ctypes.c_int32), ("solve", MincutOptions)]


class MincutServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("packed_batches", ctypes.c_int64), ("packed_requests", ctypes.c_int64),
                ("single_solves", ctypes.c_int64), ("peak_inflight_bytes", ctypes.c_int64),
                ("inflight_bytes", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("peak_inflight", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load_library(path: Optional[str] = None) -> ctypes.CDLL:
    """Load libmincut.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is missing; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(p)
    vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    lib.mincut_default_options.argtypes = [ctypes.POINTER(MincutOptions)]
    lib.mincut_default_round_options.argtypes = [ctypes.POINTER(MincutRoundOptions)]
    lib.mincut_graph_from_csr.argtypes = [i64, vp, vp, vp, u32, vp,
                                          ctypes.POINTER(MincutAllocator),
                                          ctypes.POINTER(vp)]
    lib.mincut_graph_from_csr.restype = ctypes.c_int
    lib.mincut_solve.argtypes = [vp, ctypes.POINTER(MincutOptions), ctypes.POINTER(i64), vp,
                                 ctypes.POINTER(MincutStats)]
    lib.mincut_solve.restype = ctypes.c_int
    lib.mincut_contract_round.argtypes = [vp, ctypes.POINTER(MincutRoundOptions),
                                          ctypes.POINTER(MincutRoundResult)]
    lib.mincut_contract_round.restype = ctypes.c_int
    lib.mincut_graph_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.mincut_graph_info.restype = ctypes.c_int
    lib.mincut_graph_export_csr.argtypes = [vp, vp, vp, vp]
    lib.mincut_graph_export_csr.restype = ctypes.c_int
    lib.mincut_graph_reset.argtypes = [vp]
    lib.mincut_graph_reset.restype = ctypes.c_int
    lib.mincut_graph_destroy.argtypes = [vp]
    lib.mincut_graph_destroy.restype = None
    lib.mincut_status_string.argtypes = [ctypes.c_int]
    lib.mincut_status_string.restype = ctypes.c_char_p
    lib.mincut_last_error.argtypes = []
    lib.mincut_last_error.restype = ctypes.c_char_p
    lib.mincut_profile_read.argtypes = [vp, ctypes.POINTER(MincutProfileEntry), i32,
                                        ctypes.POINTER(i32), i32]
    lib.mincut_profile_read.restype = ctypes.c_int
    lib.mincut_batch_from_csr.argtypes = [i64, vp, vp, vp, vp, u32, vp,
                                          ctypes.POINTER(MincutAllocator), ctypes.POINTER(vp)]
    lib.mincut_batch_from_csr.restype = ctypes.c_int
    lib.mincut_batch_solve.argtypes = [vp, ctypes.POINTER(MincutOptions), vp, vp,
                                       ctypes.POINTER(MincutStats)]
    lib.mincut_batch_solve.restype = ctypes.c_int
    lib.mincut_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(i64)]
    lib.mincut_batch_info.restype = ctypes.c_int
    lib.mincut_graph_footprint.argtypes = [i64, i64]
    lib.mincut_graph_footprint.restype = i64
    lib.mincut_release_cached.argtypes = [ctypes.c_int]
    lib.mincut_release_cached.restype = ctypes.c_int
    lib.mincut_server_default_options.argtypes = [ctypes.POINTER(MincutServerOptions)]
    lib.mincut_server_create.argtypes = [ctypes.POINTER(MincutServerOptions), ctypes.POINTER(vp)]
    lib.mincut_server_create.restype = ctypes.c_int
    lib.mincut_server_submit.argtypes = [vp, i64, vp, vp, vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.mincut_server_submit.restype = ctypes.c_int
    lib.mincut_server_submit_borrowed.argtypes = [vp, i64, vp, vp, vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.mincut_server_submit_borrowed.restype = ctypes.c_int
    lib.mincut_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(i64),
                                       ctypes.POINTER(ctypes.c_double), vp]
    lib.mincut_server_wait.restype = ctypes.c_int
    lib.mincut_server_stats_read.argtypes = [vp, ctypes.POINTER(MincutServerStats)]
    lib.mincut_server_stats_read.restype = ctypes.c_int
    lib.mincut_server_destroy.argtypes = [vp]
    lib.mincut_server_destroy.restype = None
    lib.mincut_contract_csr_noalloc.argtypes = [i64, vp, vp, vp, i64, vp, i64, vp, vp, vp,
                                                ctypes.POINTER(i64), vp]
    lib.mincut_contract_csr_noalloc.restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def _check(rc: int) -> None:
    if rc != MINCUT_OK:
        lib = load_library()
        msg = (lib.mincut_last_error() or b"").decode() or lib.mincut_status_string(rc).decode()
        raise MincutError(rc, msg)


def default_options(**kw) -> MincutOptions:
    o = MincutOptions()
    load_library().mincut_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def default_round_options(**kw) -> MincutRoundOptions:
    o = MincutRoundOptions()
    load_library().mincut_default_round_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _is_torch_cuda(x: Any) -> bool:
    return hasattr(x, "is_cuda") and bool(getattr(x, "is_cuda"))


class _TorchAllocator:
    """Routes the library's device allocations through torch's caching allocator."""

    def __init__(self, device: int):
        import torch
        self.torch = torch
        self.device = device
        self.live: dict[int, int] = {}

        def _alloc(nbytes, stream, ctx):
            try:
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                         stream if stream else None)
            except Exception:
                return None
            self.live[int(ptr)] = int(nbytes)
            return int(ptr)

        def _free(ptr, nbytes, stream, ctx):
            if ptr and int(ptr) in self.live:
                del self.live[int(ptr)]
                torch.cuda.caching_allocator_delete(int(ptr))

        self._alloc = _ALLOC_FN(_alloc)
        self._free = _FREE_FN(_free)
        self.struct = MincutAllocator(self._alloc, self._free, None)


class Graph:
    """Owning handle of a device graph (destroyed with mincut_graph_destroy)."""

    def __init__(self, handle: int, n: int, keep: list, allocator=None):
        self.handle = ctypes.c_void_p(handle)
        self.n = n
        self._keep = keep
        self._allocator = allocator

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def destroy(self) -> None:
        if self.handle and self.handle.value:
            load_library().mincut_graph_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)


def mincut_graph_from_csr(n: int, row_ptr, col, w, *, stream: Any = None,
                          skip_validate: bool = False, use_torch_allocator: bool = False
                          ) -> Graph:
    """Build a device graph from a symmetric CSR (numpy host arrays or torch
    CUDA tensors: int64 row_ptr[n+1], int32 col[M], int32 w[M])."""
    lib = load_library()
    keep = []
    if _is_torch_cuda(row_ptr):
        import torch
        assert row_ptr.dtype == torch.int64 and col.dtype == torch.int32 and w.dtype == torch.int32
        row_ptr, col, w = row_ptr.contiguous(), col.contiguous(), w.contiguous()
        keep += [row_ptr, col, w]
        ptrs = (row_ptr.data_ptr(), col.data_ptr(), w.data_ptr())
        flags = MINCUT_DEVICE_PTRS
        if stream is None:
            stream = torch.cuda.current_stream(row_ptr.device).cuda_stream
        device = row_ptr.device.index or 0
    else:
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.int32)
        if col.size == 0:
            col = np.zeros(1, np.int32)
            w = np.zeros(1, np.int32)
        keep += [row_ptr, col, w]
        ptrs = (row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data)
        flags = MINCUT_HOST_PTRS
        device = 0
    if skip_validate:
        flags |= MINCUT_SKIP_VALIDATE
    if hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    alloc = _TorchAllocator(device) if use_torch_allocator else None
    out = ctypes.c_void_p(0)
    rc = lib.mincut_graph_from_csr(n, ptrs[0], ptrs[1], ptrs[2], flags,
                                   ctypes.c_void_p(stream or 0),
                                   ctypes.byref(alloc.struct) if alloc else None,
                                   ctypes.byref(out))
    _check(rc)
    return Graph(out.value, n, keep, alloc)


def pack_graphs(graphs) -> tuple:
    """Pack (n, row_ptr, col, w) graphs into one CSR with per-graph vertex
    offsets: returns (vertex_offsets int64[G+1], row_ptr, col, w)."""
    offs = [0]
    rps, cols, ws = [], [], []
    ebase = 0
    for (n, rp, col, w) in graphs:
        rp = np.asarray(rp, np.int64)
        rps.append(rp[:-1] + ebase)
        cols.append(np.asarray(col, np.int64) + offs[-1])
        ws.append(np.asarray(w, np.int64))
        ebase += int(rp[-1])
        offs.append(offs[-1] + int(n))
    row_ptr = np.concatenate(rps + [np.array([ebase], np.int64)])
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    w = np.concatenate(ws).astype(np.int32) if ws else np.zeros(0, np.int32)
    return np.asarray(offs, np.int64), row_ptr, col, w


def mincut_batch_from_csr(vertex_offsets, row_ptr, col, w, *, stream: Any = None,
                          skip_validate: bool = False) -> Graph:
    """Build a packed batch of graphs (host numpy arrays; see pack_graphs)."""
    lib = load_library()
    vo = np.ascontiguousarray(vertex_offsets, dtype=np.int64)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, np.int32)
        w = np.zeros(1, np.int32)
    flags = MINCUT_HOST_PTRS | (MINCUT_SKIP_VALIDATE if skip_validate else 0)
    if hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    out = ctypes.c_void_p(0)
    rc = lib.mincut_batch_from_csr(len(vo) - 1, vo.ctypes.data, row_ptr.ctypes.data,
                                   col.ctypes.data, w.ctypes.data, flags,
                                   ctypes.c_void_p(stream or 0), None, ctypes.byref(out))
    _check(rc)
    gr = Graph(out.value, int(vo[-1]), [vo, row_ptr, col, w])
    gr.G = len(vo) - 1
    gr.vertex_offsets = vo
    return gr


def mincut_batch_solve(g: Graph, opts: Optional[MincutOptions] = None, *, bitmap: bool = True):
    """Exact minimum cut of every graph of a batch: (values int64[G],
    bitmap uint64[ceil(n/64)] or None, stats)."""
    lib = load_library()
    vals = np.zeros(g.G, np.int64)
    st = MincutStats()
    bm = np.zeros((g.n + 63) // 64, np.uint64) if bitmap else None
    rc = lib.mincut_batch_solve(g.handle, ctypes.byref(opts) if opts is not None else None,
                                vals.ctypes.data, bm.ctypes.data if bm is not None else None,
                                ctypes.byref(st))
    _check(rc)
    return vals, bm, st.as_dict()


def mincut_batch_info(g: Graph) -> tuple[int, int]:
    """(vertex threshold of the one-warp-per-graph solver used by the last
    batch solve, number of graphs it solved)."""
    t = ctypes.c_int32(0)
    k = ctypes.c_int64(0)
    _check(load_library().mincut_batch_info(g.handle, ctypes.byref(t), ctypes.byref(k)))
    return int(t.value), int(k.value)


def mincut_solve(g: Graph, opts: Optional[MincutOptions] = None, *, bitmap: bool = True,
                 side_bitmap_out=None):
    """Exact minimum cut.  Returns (value, bitmap uint64[ceil(n/64)] or None,
    stats dict).  side_bitmap_out may be a torch CUDA tensor (int64) or a
    numpy uint64 array to write into."""
    lib = load_library()
    val = ctypes.c_int64(0)
    st = MincutStats()
    bm = None
    ptr = None
    if side_bitmap_out is not None:
        bm = side_bitmap_out
        ptr = bm.data_ptr() if _is_torch_cuda(bm) else bm.ctypes.data
    elif bitmap:
        bm = np.zeros((g.n + 63) // 64, np.uint64)
        ptr = bm.ctypes.data
    rc = lib.mincut_solve(g.handle, ctypes.byref(opts) if opts is not None else None,
                          ctypes.byref(val), ctypes.c_void_p(ptr) if ptr else None,
                          ctypes.byref(st))
    _check(rc)
    return int(val.value), bm, st.as_dict()


def bitmap_to_side(bm: np.ndarray, n: int) -> np.ndarray:
    """uint8[n] side flags from a solve bitmap (bit v of word v // 64)."""
    bits = np.unpackbits(np.asarray(bm, dtype=np.uint64).view(np.uint8), bitorder="little")
    return bits[:n].astype(np.uint8)


def mincut_contract_round(g: Graph, ro: Optional[MincutRoundOptions] = None) -> dict:
    """One contraction round on the graph's current state (see the header)."""
    lib = load_library()
    if ro is None:
        ro = default_round_options()
    res = MincutRoundResult()
    _check(lib.mincut_contract_round(g.handle, ctypes.byref(ro), ctypes.byref(res)))
    return res.as_dict()


def mincut_graph_info(g: Graph) -> tuple[int, int]:
    n = ctypes.c_int64(0)
    m = ctypes.c_int64(0)
    _check(load_library().mincut_graph_info(g.handle, ctypes.byref(n), ctypes.byref(m)))
    return int(n.value), int(m.value)


def mincut_graph_export_csr(g: Graph):
    """Current canonical CSR as numpy arrays (row_ptr int64, col int32, w int64)."""
    n, M = mincut_graph_info(g)
    rp = np.zeros(n + 1, np.int64)
    col = np.zeros(max(M, 1), np.int32)
    w = np.zeros(max(M, 1), np.int64)
    _check(load_library().mincut_graph_export_csr(g.handle, rp.ctypes.data, col.ctypes.data,
                                                  w.ctypes.data))
    return rp, col[:M], w[:M]


def mincut_graph_reset(g: Graph) -> None:
    _check(load_library().mincut_graph_reset(g.handle))


def mincut_graph_destroy(g: Graph) -> None:
    g.destroy()


def mincut_profile_read(g: Graph, reset: bool = False) -> dict:
    """Per-kernel-category device time of profiled solves:
    {name: {"launches", "units", "ms"}}."""
    lib = load_library()
    buf = (MincutProfileEntry * 32)()
    cnt = ctypes.c_int32(0)
    _check(lib.mincut_profile_read(g.handle, buf, 32, ctypes.byref(cnt), 1 if reset else 0))
    return {buf[i].name.decode(): {"launches": int(buf[i].launches), "units": int(buf[i].units),
                                   "ms": float(buf[i].ms)} for i in range(cnt.value)}


def mincut_contract_csr_noalloc(n: int, row_ptr, col, w, labels, n2: int, row_ptr_out, col_out,
                                w_out, *, m_directed: Optional[int] = None,
                                stream: Any = None) -> int:
    """Contract a device CSR (torch CUDA tensors) by labels without any device
    allocation inside the library; the caller supplies the output tensors
    (row_ptr_out int64[n2+1], col_out/w_out int32 with capacity M).  M is
    row_ptr[n] unless m_directed is given (the library rejects a mismatch).
    Returns the number of entries written.  See include/mincut.h for the
    limits."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(row_ptr.device).cuda_stream
    if hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    if row_ptr.numel() < n + 1 or labels.numel() < n or row_ptr_out.numel() < n2 + 1:
        raise ValueError("row_ptr needs n + 1, labels n and row_ptr_out n2 + 1 entries")
    M = int(row_ptr[n].item()) if m_directed is None else int(m_directed)
    if min(col.numel(), w.numel(), col_out.numel(), w_out.numel()) < M:
        raise ValueError(f"col, w, col_out and w_out need capacity for M = {M} entries")
    m = ctypes.c_int64(0)
    _check(load_library().mincut_contract_csr_noalloc(
        n, row_ptr.data_ptr(), col.data_ptr(), w.data_ptr(), M, labels.data_ptr(), n2,
        row_ptr_out.data_ptr(), col_out.data_ptr(), w_out.data_ptr(), ctypes.byref(m),
        ctypes.c_void_p(stream or 0)))
    return int(m.value)


def mincut_release_cached(device: int = 0) -> None:
    """Return the unused blocks of the library's device memory pool to the
    driver (graphs created without a user allocator draw from that pool)."""
    _check(load_library().mincut_release_cached(int(device)))


def mincut_graph_footprint(n: int, m_directed: int) -> int:
    return int(load_library().mincut_graph_footprint(n, m_directed))


def server_default_options(**kw) -> MincutServerOptions:
    o = MincutServerOptions()
    load_library().mincut_server_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Server:
    """Continuous-batching solve server (mincut_server_* in the C ABI)."""

    def __init__(self, opts: Optional[MincutServerOptions] = None, **kw):
        lib = load_library()
        if opts is None:
            opts = server_default_options(**kw)
        h = ctypes.c_void_p(0)
        _check(lib.mincut_server_create(ctypes.byref(opts), ctypes.byref(h)))
        self.handle = h
        self.sizes: dict[int, int] = {}
        self.keep: dict[int, tuple] = {}  # arrays of borrowed requests, until wait()

    def submit(self, n: int, row_ptr, col, w, *, borrow: bool = False) -> int:
        """Queue a request.  borrow=True: the server reads these arrays in
        place (pinned ones directly from the device) instead of copying them;
        they are kept referenced here until wait() returns."""
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        c = np.ascontiguousarray(col, dtype=np.int32)
        ww = np.ascontiguousarray(w, dtype=np.int32)
        rid = ctypes.c_uint64(0)
        fn = (load_library().mincut_server_submit_borrowed if borrow
              else load_library().mincut_server_submit)
        _check(fn(self.handle, n, rp.ctypes.data, c.ctypes.data if c.size else None,
                  ww.ctypes.data if ww.size else None, ctypes.byref(rid)))
        self.sizes[int(rid.value)] = n
        if borrow:
            self.keep[int(rid.value)] = (rp, c, ww)
        return int(rid.value)

    def wait(self, rid: int, bitmap: bool = True):
        """(value, latency_ms, bitmap or None) of a submitted request."""
        n = self.sizes.pop(rid)
        val = ctypes.c_int64(0)
        lat = ctypes.c_double(0)
        bm = np.zeros((n + 63) // 64, np.uint64) if bitmap else None
        try:
            _check(load_library().mincut_server_wait(self.handle, rid, ctypes.byref(val),
                                                     ctypes.byref(lat),
                                                     bm.ctypes.data if bm is not None else None))
        finally:
            self.keep.pop(rid, None)
        return int(val.value), float(lat.value), bm

    def stats(self) -> dict:
        st = MincutServerStats()
        _check(load_library().mincut_server_stats_read(self.handle, ctypes.byref(st)))
        return st.as_dict()

    def close(self) -> None:
        if self.handle and self.handle.value:
            load_library().mincut_server_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mincut_status_string(status: int) -> str:
    return load_library().mincut_status_string(status).decode()


def mincut_last_error() -> str:
    return (load_library().mincut_last_error() or b"").decode()


def exported_symbols() -> list[str]:
    """Function names declared in include/mincut.h (parsed from the header)."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "mincut.h")
    with open(hdr) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(mincut_[a-z_]+)\s*\(", text)))
