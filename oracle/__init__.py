"""Plain CPU oracle for the traversal primitives of arXiv 1504.04804.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library (``paper_1504_04804_gb300``) and never imports it.

The arithmetic lives in ``oracle.c`` (plain C, one routine per primitive, each
citing the passage it follows); this module only compiles it with gcc and
marshals numpy arrays through ctypes.

* ``bfs``      -- FIFO-queue BFS: hop distance, -1 if unreached (Algorithm 1).
* ``sssp``     -- Dijkstra with a binary heap, uint64 accumulation, uint32
                  output, UINT32_MAX if unreached (Table 1, Sec. 7 weights).
* ``cc``       -- union-find, label = minimum vertex id of the component
                  (Table 1, Soman et al.'s hooking).
* ``pagerank`` -- float64 power iteration with dangling mass spread evenly,
                  exactly ``iters`` updates from r = 1/N (Algorithm 3 and the
                  normalised-with-compensation mode of Sec. 7).
* ``bc``       -- Brandes' dependency accumulation in float64: forward BFS
                  counting shortest paths (sigma), backward pass in reverse
                  BFS order (Table 1's BC, McLaughlin and Bader's scheme).
* ``check_bfs`` / ``check_sssp`` / ``check_cc`` -- invariant checkers that
  hold at any size.

Parity status: every function above is pinned by ``tests/test_oracle.py``
(exhaustive 6-vertex graphs against Floyd-Warshall / transitive closure,
closed forms, a dense-matrix PageRank and printed fixtures).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (portable flags only)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    p = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.oracle_bfs.argtypes = [i64, p, p, ctypes.c_int32, p]
    lib.oracle_bfs.restype = ctypes.c_int
    lib.oracle_sssp.argtypes = [i64, p, p, p, ctypes.c_int32, p]
    lib.oracle_sssp.restype = ctypes.c_int
    lib.oracle_cc.argtypes = [i64, p, p, p]
    lib.oracle_cc.restype = ctypes.c_int
    lib.oracle_pagerank.argtypes = [i64, p, p, ctypes.c_double, ctypes.c_int, p]
    lib.oracle_pagerank.restype = ctypes.c_int
    lib.oracle_bc.argtypes = [i64, p, p, p, i64, p, p]
    lib.oracle_bc.restype = ctypes.c_int
    lib.oracle_check_bfs.argtypes = [i64, p, p, ctypes.c_int32, p, p]
    lib.oracle_check_bfs.restype = ctypes.c_int64
    lib.oracle_check_sssp.argtypes = [i64, p, p, p, ctypes.c_int32, p]
    lib.oracle_check_sssp.restype = ctypes.c_int64
    lib.oracle_check_cc.argtypes = [i64, p, p, p]
    lib.oracle_check_cc.restype = ctypes.c_int64
    _lib = lib
    return lib


class OracleError(RuntimeError):
    pass


def _csr(row_offsets, col_indices):
    ro = np.ascontiguousarray(row_offsets, dtype=np.int64)
    col = np.ascontiguousarray(col_indices, dtype=np.int32)
    nv = ro.shape[0] - 1
    if nv < 0 or ro[0] != 0 or ro[-1] != col.shape[0]:
        raise OracleError("malformed CSR")
    return nv, ro, col


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def bfs(row_offsets, col_indices, src: int) -> np.ndarray:
    nv, ro, col = _csr(row_offsets, col_indices)
    depth = np.empty(nv, dtype=np.int32)
    rc = _load().oracle_bfs(nv, _ptr(ro), _ptr(col), int(src), _ptr(depth))
    if rc != 0:
        raise OracleError(f"oracle_bfs failed ({rc})")
    return depth


def sssp(row_offsets, col_indices, weights, src: int) -> np.ndarray:
    nv, ro, col = _csr(row_offsets, col_indices)
    w = np.ascontiguousarray(weights, dtype=np.uint32)
    if w.shape[0] != col.shape[0]:
        raise OracleError("weights must have one entry per CSR edge")
    dist = np.empty(nv, dtype=np.uint32)
    rc = _load().oracle_sssp(nv, _ptr(ro), _ptr(col), _ptr(w), int(src), _ptr(dist))
    if rc != 0:
        raise OracleError(f"oracle_sssp failed ({rc})")
    return dist


def cc(row_offsets, col_indices) -> np.ndarray:
    nv, ro, col = _csr(row_offsets, col_indices)
    label = np.empty(nv, dtype=np.int32)
    rc = _load().oracle_cc(nv, _ptr(ro), _ptr(col), _ptr(label))
    if rc != 0:
        raise OracleError(f"oracle_cc failed ({rc})")
    return label


def pagerank(row_offsets, col_indices, damping: float = 0.85, iters: int = 20) -> np.ndarray:
    nv, ro, col = _csr(row_offsets, col_indices)
    rank = np.empty(nv, dtype=np.float64)
    rc = _load().oracle_pagerank(nv, _ptr(ro), _ptr(col), float(damping), int(iters), _ptr(rank))
    if rc != 0:
        raise OracleError(f"oracle_pagerank failed ({rc})")
    return rank


def bc(row_offsets, col_indices, srcs, want_sigma: bool = False):
    """Sum over ``srcs`` of Brandes' dependencies (float64 [nv]); with
    ``want_sigma`` also the shortest-path counts of the last source."""
    nv, ro, col = _csr(row_offsets, col_indices)
    s = np.ascontiguousarray(np.atleast_1d(np.asarray(srcs, dtype=np.int32)))
    out = np.empty(nv, dtype=np.float64)
    sig = np.empty(nv, dtype=np.float64) if want_sigma else None
    rc = _load().oracle_bc(nv, _ptr(ro), _ptr(col), _ptr(s), int(s.shape[0]), _ptr(out),
                           None if sig is None else _ptr(sig))
    if rc != 0:
        raise OracleError(f"oracle_bc failed ({rc})")
    return (out, sig) if want_sigma else out


def check_bfs(row_offsets, col_indices, src: int, depth, parent=None) -> int:
    nv, ro, col = _csr(row_offsets, col_indices)
    d = np.ascontiguousarray(depth, dtype=np.int32)
    par = None if parent is None else np.ascontiguousarray(parent, dtype=np.int32)
    return int(_load().oracle_check_bfs(nv, _ptr(ro), _ptr(col), int(src), _ptr(d),
                                        None if par is None else _ptr(par)))


def check_sssp(row_offsets, col_indices, weights, src: int, dist) -> int:
    nv, ro, col = _csr(row_offsets, col_indices)
    w = np.ascontiguousarray(weights, dtype=np.uint32)
    d = np.ascontiguousarray(dist, dtype=np.uint32)
    return int(_load().oracle_check_sssp(nv, _ptr(ro), _ptr(col), _ptr(w), int(src), _ptr(d)))


def check_cc(row_offsets, col_indices, label) -> int:
    nv, ro, col = _csr(row_offsets, col_indices)
    lab = np.ascontiguousarray(label, dtype=np.int32)
    return int(_load().oracle_check_cc(nv, _ptr(ro), _ptr(col), _ptr(lab)))
