"""ctypes binding of libgrx (include/grx.h), with the same names as the C ABI.

This module only marshals arguments: every step of every traversal runs in
the CUDA kernels of libgrx.so.  PyTorch provides device memory (the library's
allocations go through torch's caching allocator) and streams.  There is no
CPU fallback: if libgrx.so is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import inputs as _inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgrx.so")

GRX_OK, GRX_EINVAL, GRX_ENOMEM, GRX_ECUDA, GRX_ETIMEOUT, GRX_ERANGE, GRX_EBUSY = 0, -1, -2, -3, -4, -5, -6
GRX_HOST_PTRS, GRX_DEVICE_PTRS, GRX_VALIDATE, GRX_OFFSETS64 = 0x0, 0x1, 0x2, 0x4
GRX_DIR_AUTO, GRX_DIR_PUSH, GRX_DIR_PULL = 0, 1, 2
GRX_LOOP_PERSISTENT, GRX_LOOP_HOST, GRX_LOOP_GRAPH = 0, 1, 2
GRX_MAX_LEVELS_STATS = 16384
_STATUS_NAMES = {0: "GRX_OK", -1: "GRX_EINVAL", -2: "GRX_ENOMEM", -3: "GRX_ECUDA",
                 -4: "GRX_ETIMEOUT", -5: "GRX_ERANGE", -6: "GRX_EBUSY"}


class GrxError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class grx_opts(ctypes.Structure):
    _fields_ = [("direction", ctypes.c_int), ("alpha", ctypes.c_float), ("beta", ctypes.c_float),
                ("loop", ctypes.c_int), ("grid_blocks", ctypes.c_int),
                ("block_threads", ctypes.c_int), ("timeout_s", ctypes.c_double),
                ("collect_stats", ctypes.c_int), ("exact_fv", ctypes.c_int),
                ("ev_begin", ctypes.c_void_p),
                ("ev_end", ctypes.c_void_p), ("push_bitmap", ctypes.c_float),
                ("sssp_delta", ctypes.c_uint)]


class grx_trav_stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32),
                ("dir", ctypes.c_int32 * GRX_MAX_LEVELS_STATS),
                ("frontier", ctypes.c_int64 * GRX_MAX_LEVELS_STATS),
                ("edges_examined", ctypes.c_int64 * GRX_MAX_LEVELS_STATS),
                ("vertices_scanned", ctypes.c_int64 * GRX_MAX_LEVELS_STATS),
                ("discovered", ctypes.c_int64 * GRX_MAX_LEVELS_STATS),
                ("level_ns", ctypes.c_int64 * GRX_MAX_LEVELS_STATS)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class grx_allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", ctypes.c_void_p)]


# (name, restype, argtypes) of every exported entry point
_P, _I, _I64, _U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
SIGNATURES = [
    ("grx_ctx_create", _I, [_P, _P]),
    ("grx_ctx_destroy", _I, [_P]),
    ("grx_last_error", ctypes.c_char_p, []),
    ("graph_load_csr", _I, [_P, _I64, _I64, _P, _I, _P, _P, _I, _P, _P]),
    ("graph_free", _I, [_P]),
    ("grx_graph_info", _I, [_P, _P, _P]),
    ("grx_graph_status", _I, [_P, _P]),
    ("grx_opts_default", None, [_P]),
    ("bfs", _I, [_P, ctypes.c_int32, _P, _P, _P, _P]),
    ("sssp", _I, [_P, ctypes.c_int32, _P, _P, _P]),
    ("cc", _I, [_P, _P, _P]),
    ("bc", _I, [_P, _P, _I, _P, _P, _P, _P]),
    ("bc_multi", _I, [_P, _P, _I, _P, _P, _P]),
    ("pagerank", _I, [_P, ctypes.c_float, _I, _P, _P]),
    ("grx_pagerank_block", _I, [_P, _I]),
    ("grx_last_stats", _I, [_P, _P, _P]),
    ("bfs_multi", _I, [_P, _P, _I, _P, _P, _P]),
    ("sssp_multi", _I, [_P, _P, _I, _P, _P, _P]),
    ("bfs_noalloc", _I, [_I64, _I64, _P, _P, ctypes.c_int32, _P, _P, _P, _P, _P]),
    ("grx_batch_open", _I, [_P, _I, _P, _P]),
    ("grx_batch_close", _I, [_P]),
    ("grx_batch_admit", _I, [_P, ctypes.c_int32, _P, _P]),
    ("grx_batch_step", _I, [_P, _I]),
    ("grx_batch_poll", _I, [_P, _P]),
    ("grx_batch_footprint", _I, [_P, _I, _P]),
    ("grx_multi_footprint", _I, [_P, _I, _P]),
    ("graph_load_csr64", _I, [_P, _I64, _I64, _P, _P, _I, _P, _P]),
    ("bfs64", _I, [_P, _I64, _P, _P, _P, _P]),
    ("grx_rmat_edges", _I, [_I, _I64, _U64, _U64, _U64, _U64, _P, _P, _P]),
    ("grx_edge_weights", _I, [_I64, _I64, _P, _P, ctypes.c_uint32, _U64, _P, _P]),
    ("grx_grid_edges", _I, [_I64, _I64, _U64, _U64, _P, _P, _P, _P]),
]

_lib = None
_lib_lock = threading.Lock()


def lib():
    """The loaded libgrx.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lib_lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "paper_1504_04804_gb300.build.build() (needs nvcc)")
            h = ctypes.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                fn = getattr(h, name)
                fn.restype = res
                fn.argtypes = args
            _lib = h
    return _lib


def _check(rc: int, what: str):
    if rc != GRX_OK:
        msg = lib().grx_last_error()
        raise GrxError(rc, f"{what}: {msg.decode() if msg else ''}")


def _stream_ptr(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


# ---------------------------------------------------------------------------
# context: one per (thread, device), allocating through torch
# ---------------------------------------------------------------------------
class _Ctx:
    def __init__(self, device: int):
        self.device = device

        def _alloc(nbytes, stream, user):
            try:
                with torch.cuda.device(self.device):
                    return torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                              int(stream or 0) or None)
            except Exception:          # out of memory -> NULL -> GRX_ENOMEM
                return None

        def _free(ptr, nbytes, stream, user):
            try:
                torch.cuda.caching_allocator_delete(ptr)
            except Exception:
                pass

        self._alloc_cb = _ALLOC_FN(_alloc)
        self._free_cb = _FREE_FN(_free)
        self._allocator = grx_allocator(self._alloc_cb, self._free_cb, None)
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            _check(lib().grx_ctx_create(ctypes.byref(self._allocator), ctypes.byref(h)),
                   "grx_ctx_create")
        self.handle = h


_tls = threading.local()


def _ctx(device: int | None = None) -> _Ctx:
    if not torch.cuda.is_available():
        raise RuntimeError("libgrx needs a CUDA GPU; none is visible")
    dev = torch.cuda.current_device() if device is None else int(device)
    cache = getattr(_tls, "ctxs", None)
    if cache is None:
        cache = _tls.ctxs = {}
    if dev not in cache:
        cache[dev] = _Ctx(dev)
    return cache[dev]


# ---------------------------------------------------------------------------
# graphs
# ---------------------------------------------------------------------------
def _as_contig(x, dtype_np, dtype_t):
    if isinstance(x, torch.Tensor):
        return x.contiguous().to(dtype_t)
    return torch.from_numpy(np.ascontiguousarray(x, dtype=dtype_np))


class Graph:
    """A CSR graph resident on the GPU (owned by libgrx)."""

    def __init__(self, handle, nv: int, ne: int, device: int, weighted: bool, name: str = ""):
        self.handle = handle
        self.nv = nv
        self.ne = ne
        self.device = device
        self.weighted = weighted
        self.name = name

    def free(self):
        if self.handle:
            torch.cuda.synchronize(self.device)
            lib().graph_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def graph_load_csr(row_offsets, col_indices, weights=None, validate: bool = False,
                   stream=None, name: str = "", offsets64: bool = False) -> Graph:
    """Copy a symmetric CSR (numpy arrays or torch tensors, host or device) to
    the GPU.  row_offsets int32 or int64 [nv+1], col_indices int32 [ne],
    weights uint32 [ne] or None.  offsets64 keeps 64-bit offsets on the device
    even when they would fit in 32 bits."""
    ctx = _ctx()
    ro = row_offsets
    ro64 = (ro.dtype == torch.int64) if isinstance(ro, torch.Tensor) else (np.asarray(ro).dtype == np.int64)
    ro = _as_contig(ro, np.int64 if ro64 else np.int32, torch.int64 if ro64 else torch.int32)
    col = _as_contig(col_indices, np.int32, torch.int32)
    w = None
    if weights is not None:
        if isinstance(weights, torch.Tensor):
            w = weights.contiguous().view(torch.int32) if weights.dtype != torch.int32 else weights.contiguous()
        else:
            w = torch.from_numpy(np.ascontiguousarray(weights, dtype=np.uint32).view(np.int32))
    nv = ro.numel() - 1
    ne = col.numel()
    on_dev = ro.is_cuda
    if on_dev != col.is_cuda or (w is not None and w.is_cuda != on_dev):
        raise ValueError("row_offsets, col_indices and weights must all be on the host or all on the GPU")
    flags = (GRX_DEVICE_PTRS if on_dev else GRX_HOST_PTRS) | (GRX_VALIDATE if validate else 0) | \
        (GRX_OFFSETS64 if offsets64 else 0)
    h = ctypes.c_void_p()
    if w is not None and ne == 0:          # weighted graph without edges: any non-NULL pointer
        w = torch.zeros(1, dtype=torch.int32, device=ro.device)
    _check(lib().graph_load_csr(ctx.handle, nv, ne, ro.data_ptr(), 1 if ro64 else 0,
                                col.data_ptr() if ne else None,
                                w.data_ptr() if w is not None else None,
                                flags, _stream_ptr(stream), ctypes.byref(h)), "graph_load_csr")
    if not on_dev:
        torch.cuda.current_stream().synchronize() if stream is None else torch.cuda.synchronize()
    return Graph(h, nv, ne, ctx.device, weights is not None, name)


def graph_free(g: Graph):
    g.free()


def graph_load_csr64(row_offsets, col_indices, validate: bool = False, stream=None, name: str = "") -> Graph:
    """Copy a symmetric CSR with 64-bit vertex ids (int64 row_offsets [nv+1] and
    col_indices [ne], numpy arrays or torch tensors, host or device) to the
    GPU; only bfs64 traverses it."""
    ctx = _ctx()
    ro = _as_contig(row_offsets, np.int64, torch.int64)
    col = _as_contig(col_indices, np.int64, torch.int64)
    nv, ne = ro.numel() - 1, col.numel()
    if ro.is_cuda != col.is_cuda:
        raise ValueError("row_offsets and col_indices must both be on the host or both on the GPU")
    flags = (GRX_DEVICE_PTRS if ro.is_cuda else GRX_HOST_PTRS) | (GRX_VALIDATE if validate else 0)
    h = ctypes.c_void_p()
    _check(lib().graph_load_csr64(ctx.handle, nv, ne, ro.data_ptr(), col.data_ptr() if ne else None,
                                  flags, _stream_ptr(stream), ctypes.byref(h)), "graph_load_csr64")
    if not ro.is_cuda:
        torch.cuda.current_stream().synchronize() if stream is None else torch.cuda.synchronize()
    return Graph(h, nv, ne, ctx.device, False, name)


def bfs64(g: Graph, src: int, depth_out=None, parent_out=None, opts: grx_opts | None = None,
          stream=None, parent: bool = False):
    """Depths (int32 [nv], -1 = unreached) on a graph_load_csr64 graph; with
    parent=True also int64 parents."""
    d = _out(depth_out, g.nv, torch.int32, g.device)
    p = None
    if parent or parent_out is not None:
        p = _out(parent_out, g.nv, torch.int64, g.device)
    _check(lib().bfs64(g.handle, int(src), d.data_ptr(), p.data_ptr() if p is not None else None,
                       ctypes.byref(opts) if opts is not None else None, _stream_ptr(stream)), "bfs64")
    return (d, p) if p is not None else d


def load(graph: "_inputs.Graph", validate: bool = False, stream=None, offsets64: bool = False) -> Graph:
    """Load an inputs.Graph (host CSR) onto the GPU."""
    return graph_load_csr(graph.row_offsets, graph.col_indices, graph.weights, validate=validate,
                          stream=stream, name=graph.name, offsets64=offsets64)


def opts(**kw) -> grx_opts:
    o = grx_opts()
    lib().grx_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _out(t, n, dtype, device):
    if t is None:
        return torch.empty(n, dtype=dtype, device=f"cuda:{device}")
    if not t.is_cuda or t.numel() < n or not t.is_contiguous():
        raise ValueError("output must be a contiguous CUDA tensor of sufficient size")
    return t


def bfs(g: Graph, src: int, depth_out=None, parent_out=None, opts: grx_opts | None = None,
        stream=None, parent: bool = False):
    """Depths (int32 [nv], -1 = unreached); with parent=True also parents."""
    d = _out(depth_out, g.nv, torch.int32, g.device)
    p = _out(parent_out, g.nv, torch.int32, g.device) if (parent or parent_out is not None) else None
    _check(lib().bfs(g.handle, int(src), d.data_ptr(), p.data_ptr() if p is not None else None,
                     ctypes.byref(opts) if opts is not None else None, _stream_ptr(stream)), "bfs")
    return (d, p) if p is not None else d


def sssp(g: Graph, src: int, dist_out=None, opts: grx_opts | None = None, stream=None):
    """Distances as an int32 tensor holding uint32 bits (UINT32_MAX = unreached);
    use ``as_uint32`` to read them."""
    d = _out(dist_out, g.nv, torch.int32, g.device)
    _check(lib().sssp(g.handle, int(src), d.data_ptr(),
                      ctypes.byref(opts) if opts is not None else None, _stream_ptr(stream)), "sssp")
    return d


def _srcs_arg(srcs):
    arr = np.ascontiguousarray(np.asarray(srcs, dtype=np.int32))
    return arr, arr.ctypes.data_as(ctypes.c_void_p), int(arr.shape[0])


def bfs_multi(g: Graph, srcs, depth_out=None, opts: grx_opts | None = None, stream=None):
    """Depths of up to 64 sources in one traversal: int32 [n, nv] (lane-major)."""
    arr, p, n = _srcs_arg(srcs)
    d = _out(depth_out, n * g.nv, torch.int32, g.device)
    _check(lib().bfs_multi(g.handle, p, n, d.data_ptr(),
                           ctypes.byref(opts) if opts is not None else None, _stream_ptr(stream)),
           "bfs_multi")
    return d[: n * g.nv].view(n, g.nv)


def sssp_multi(g: Graph, srcs, dist_out=None, opts: grx_opts | None = None, stream=None):
    """Distances of up to 64 sources, int32 tensor [n, nv] holding uint32 bits."""
    arr, p, n = _srcs_arg(srcs)
    d = _out(dist_out, n * g.nv, torch.int32, g.device)
    _check(lib().sssp_multi(g.handle, p, n, d.data_ptr(),
                            ctypes.byref(opts) if opts is not None else None, _stream_ptr(stream)),
           "sssp_multi")
    return d[: n * g.nv].view(n, g.nv)


def bc(g: Graph, srcs, bc_out=None, sigma_out=None, opts: grx_opts | None = None, stream=None,
       want_sigma: bool = False):
    """Sum over the sources of Brandes' dependencies, float64 tensor [nv];
    with ``want_sigma`` (or ``sigma_out``) also the shortest-path counts of
    the last source: returns (bc, sigma)."""
    arr = np.ascontiguousarray(np.atleast_1d(np.asarray(srcs, dtype=np.int32)))
    out = _out(bc_out, g.nv, torch.float64, g.device)
    sig = _out(sigma_out, g.nv, torch.float64, g.device) if (want_sigma or sigma_out is not None) else None
    _check(lib().bc(g.handle, arr.ctypes.data_as(ctypes.c_void_p), int(arr.shape[0]), out.data_ptr(),
                    sig.data_ptr() if sig is not None else None,
                    ctypes.byref(opts) if opts is not None else None, _stream_ptr(stream)), "bc")
    return (out, sig) if sig is not None else out


def bc_multi(g: Graph, srcs, bc_out=None, opts: grx_opts | None = None, stream=None):
    """The sum over up to 64 sources of Brandes' dependencies, computed in
    one shared sweep; float64 tensor [nv]."""
    arr, p, n = _srcs_arg(srcs)
    out = _out(bc_out, g.nv, torch.float64, g.device)
    _check(lib().bc_multi(g.handle, p, n, out.data_ptr(),
                          ctypes.byref(opts) if opts is not None else None, _stream_ptr(stream)), "bc_multi")
    return out


def cc(g: Graph, label_out=None, stream=None):
    lab = _out(label_out, g.nv, torch.int32, g.device)
    _check(lib().cc(g.handle, lab.data_ptr(), _stream_ptr(stream)), "cc")
    return lab


def pagerank(g: Graph, damping: float = 0.85, iters: int = 20, rank_out=None, stream=None):
    r = _out(rank_out, g.nv, torch.float32, g.device)
    _check(lib().pagerank(g.handle, float(damping), int(iters), r.data_ptr(), _stream_ptr(stream)),
           "pagerank")
    return r


def pagerank_block(g: Graph, shift: int):
    """Column-block width (2^shift vertices) of pagerank's gathers; <= 0 =
    no blocks (the default)."""
    _check(lib().grx_pagerank_block(g.handle, int(shift)), "grx_pagerank_block")


GRX_NOALLOC_MAX_NV = 1 << 19
GRX_NOALLOC_SCRATCH_BYTES = 23413632


def _noalloc_tensor(name: str, t, numel: int | None = None):
    """Argument checks of bfs_noalloc: an int32, contiguous CUDA tensor on the
    current device (the library reads it as a raw device pointer, and its
    scratch array is the current device's)."""
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"bfs_noalloc: {name} must be a torch.Tensor")
    if t.dtype != torch.int32:
        raise ValueError(f"bfs_noalloc: {name} must be int32 (got {t.dtype})")
    if not t.is_cuda:
        raise ValueError(f"bfs_noalloc: {name} must be a CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"bfs_noalloc: {name} is on cuda:{t.device.index}, the current device is "
                         f"cuda:{torch.cuda.current_device()}")
    if not t.is_contiguous():
        raise ValueError(f"bfs_noalloc: {name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"bfs_noalloc: {name} must have {numel} elements (got {t.numel()})")


def bfs_noalloc(row_offsets: torch.Tensor, col_indices: torch.Tensor, src: int, depth_out=None,
                parent_out=None, status_out=None, opts: grx_opts | None = None, stream=None):
    """BFS over caller-owned device CSR arrays (int32 offsets) without any
    device allocation by the library: for callers that cannot allocate.  The
    output tensors, if not given, are created here by torch (the library
    itself allocates nothing).  Limited to GRX_NOALLOC_MAX_NV vertices; calls
    share one fixed scratch array, so calls overlapping on the GPU race.
    Every tensor must be int32, contiguous and on the current CUDA device
    (ValueError otherwise)."""
    _noalloc_tensor("row_offsets", row_offsets)
    _noalloc_tensor("col_indices", col_indices)
    nv = row_offsets.numel() - 1
    for name, t in (("depth_out", depth_out), ("parent_out", parent_out)):
        if t is not None:
            _noalloc_tensor(name, t, nv)
    if status_out is not None:
        _noalloc_tensor("status_out", status_out, 1)
    dev = row_offsets.device.index
    d = _out(depth_out, nv, torch.int32, dev)
    _check(lib().bfs_noalloc(nv, col_indices.numel(), row_offsets.data_ptr(),
                             col_indices.data_ptr() if col_indices.numel() else None, int(src),
                             d.data_ptr(), parent_out.data_ptr() if parent_out is not None else None,
                             status_out.data_ptr() if status_out is not None else None,
                             ctypes.byref(opts) if opts is not None else None, _stream_ptr(stream)),
           "bfs_noalloc")
    return d


GRX_KIND_BFS, GRX_KIND_SSSP = 0, 1


def batch_footprint(g: Graph, kind: int) -> int:
    n = ctypes.c_size_t()
    _check(lib().grx_batch_footprint(g.handle, int(kind), ctypes.byref(n)), "grx_batch_footprint")
    return int(n.value)


def multi_footprint(g: Graph, kind: int) -> int:
    """Workspace bytes the next bfs_multi / sssp_multi on g will allocate (0 once it has)."""
    n = ctypes.c_size_t()
    _check(lib().grx_multi_footprint(g.handle, int(kind), ctypes.byref(n)), "grx_multi_footprint")
    return int(n.value)


class Batch:
    """A resident 64-lane traversal of one graph that queries join and leave
    between level steps (continuous batching; see grx_batch_* in grx.h)."""

    def __init__(self, g: Graph, kind: int, stream=None):
        self.g = g
        self.kind = int(kind)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=g.device)
        h = ctypes.c_void_p()
        _check(lib().grx_batch_open(g.handle, self.kind, _stream_ptr(self.stream), ctypes.byref(h)),
               "grx_batch_open")
        self.handle = h
        self.outs = {}

    def admit(self, src: int, out: torch.Tensor) -> int:
        """Put a query into a free lane; raises GrxError(GRX_EBUSY) when full."""
        lane = ctypes.c_int()
        _check(lib().grx_batch_admit(self.handle, int(src), out.data_ptr(), ctypes.byref(lane)),
               "grx_batch_admit")
        self.outs[lane.value] = out
        return lane.value

    def step(self, steps: int = 1):
        _check(lib().grx_batch_step(self.handle, int(steps)), "grx_batch_step")

    def poll(self) -> int:
        m = ctypes.c_uint64()
        _check(lib().grx_batch_poll(self.handle, ctypes.byref(m)), "grx_batch_poll")
        for lane in range(64):
            if m.value >> lane & 1:
                self.outs.pop(lane, None)
        return int(m.value)

    def close(self):
        if self.handle:
            lib().grx_batch_close(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def graph_status(g: Graph, stream=None):
    """Synchronise and raise GrxError if a device-side wait timed out or a
    distance overflowed in the graph's traversals since the last check."""
    _check(lib().grx_graph_status(g.handle, _stream_ptr(stream)), "device status")


def last_stats(g: Graph, stream=None) -> dict:
    st = grx_trav_stats()
    _check(lib().grx_last_stats(g.handle, _stream_ptr(stream), ctypes.byref(st)), "grx_last_stats")
    n = min(st.levels, GRX_MAX_LEVELS_STATS)
    return {"levels": st.levels,
            "dir": list(st.dir[:n]),
            "frontier": list(st.frontier[:n]),
            "edges_examined": list(st.edges_examined[:n]),
            "vertices_scanned": list(st.vertices_scanned[:n]),
            "discovered": list(st.discovered[:n]),
            "level_ns": list(st.level_ns[:n])}


def as_uint32(t: torch.Tensor) -> np.ndarray:
    """Host numpy uint32 view of an int32 tensor that holds uint32 bits."""
    return t.cpu().numpy().view(np.uint32)


# ---------------------------------------------------------------------------
# device twins of the input generators
# ---------------------------------------------------------------------------
def rmat_edges(scale: int, edge_factor: int, seed: int, abcd=_inputs.RMAT_ABCD, stream=None):
    """Directed R-MAT edge list on the GPU, bit-identical to inputs.rmat_edges."""
    m = edge_factor << scale
    t0, t1, t2 = _inputs.rmat_thresholds(abcd)
    dev = torch.cuda.current_device()
    u = torch.empty(m, dtype=torch.int32, device=f"cuda:{dev}")
    v = torch.empty(m, dtype=torch.int32, device=f"cuda:{dev}")
    _check(lib().grx_rmat_edges(scale, m, seed & (2**64 - 1), t0, t1, t2, u.data_ptr(), v.data_ptr(),
                                _stream_ptr(stream)), "grx_rmat_edges")
    return u, v


def edge_weights(row_offsets: torch.Tensor, col_indices: torch.Tensor, wmax: int, seed: int,
                 stream=None) -> torch.Tensor:
    """Symmetric uint32 weights (returned as int32 bits) on the GPU,
    bit-identical to inputs.edge_weights."""
    ro = row_offsets.to(torch.int64).contiguous()
    nv = ro.numel() - 1
    ne = col_indices.numel()
    w = torch.empty(max(ne, 1), dtype=torch.int32, device=ro.device)
    _check(lib().grx_edge_weights(nv, ne, ro.data_ptr(), col_indices.data_ptr(), int(wmax),
                                  seed & (2**64 - 1), w.data_ptr(), _stream_ptr(stream)),
           "grx_edge_weights")
    return w[:ne]


def build_csr_device(nv: int, u: torch.Tensor, v: torch.Tensor):
    """Symmetrise, drop self-loops and duplicates and build a sorted CSR on the
    GPU (input preparation, not timed): returns (row_offsets int64, col int32).
    Produces the same CSR as inputs.build_csr."""
    u = u.to(torch.int64)
    v = v.to(torch.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    keys = torch.cat([u * nv + v, v * nv + u])
    del u, v, keep
    keys = torch.unique(keys, sorted=True)
    rows = keys // nv
    col = (keys - rows * nv).to(torch.int32)
    del keys
    counts = torch.bincount(rows, minlength=nv)
    del rows
    ro = torch.zeros(nv + 1, dtype=torch.int64, device=col.device)
    torch.cumsum(counts, 0, out=ro[1:])
    return ro, col


def grid_graph_device(width: int, height: int, p_del: float = 0.1, seed: int | None = None,
                      wmax: int | None = None, weight_seed: int | None = None, stream=None):
    """Grid graph generated and built on the GPU (same CSR and weights as
    inputs.grid_graph).  Returns (row_offsets, col_indices, weights|None)."""
    from fractions import Fraction
    seed = width if seed is None else seed
    total = height * (width - 1) + (height - 1) * width
    dev = torch.cuda.current_device()
    u = torch.empty(max(total, 1), dtype=torch.int32, device=f"cuda:{dev}")
    v = torch.empty_like(u)
    keep = torch.empty(max(total, 1), dtype=torch.uint8, device=f"cuda:{dev}")
    t_del = int(Fraction(str(p_del)) * (1 << 53))
    _check(lib().grx_grid_edges(width, height, seed & (2**64 - 1), t_del, u.data_ptr(), v.data_ptr(),
                                keep.data_ptr(), _stream_ptr(stream)), "grx_grid_edges")
    k = keep[:total].bool()
    ro, col = build_csr_device(width * height, u[:total][k], v[:total][k])
    w = None
    if wmax is not None:
        w = edge_weights(ro, col, wmax, 100 + seed if weight_seed is None else weight_seed)
    return ro, col, w


def rmat_graph_device(scale: int, edge_factor: int = 16, seed: int | None = None,
                      wmax: int | None = None, weight_seed: int | None = None):
    """R-MAT graph generated and built on the GPU (same CSR and weights as
    inputs.rmat_graph).  Returns (row_offsets, col_indices, weights|None) as
    CUDA tensors."""
    seed = scale if seed is None else seed
    u, v = rmat_edges(scale, edge_factor, seed)
    ro, col = build_csr_device(1 << scale, u, v)
    del u, v
    w = None
    if wmax is not None:
        w = edge_weights(ro, col, wmax, 100 + seed if weight_seed is None else weight_seed)
    return ro, col, w
