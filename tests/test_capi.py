"""Host-side checks of the C ABI: the library builds, loads and exports every
entry point include/grx.h declares, and the binding declares each of them.
No compute calls (no GPU here)."""
import ctypes
import os
import re

import pytest

from paper_1504_04804_gb300 import build, grx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def _declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b([A-Za-z_]\w*)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof", "defined"):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libgrx():
    build.build()
    return ctypes.CDLL(grx.LIB_PATH)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("graph_load_csr", "graph_free", "bfs", "sssp", "cc", "pagerank"):
        assert required in names


def test_library_exports_every_declared_symbol(libgrx):
    for name in _declared_functions():
        assert hasattr(libgrx, name), f"libgrx.so does not export {name}"


def test_binding_covers_every_declared_symbol():
    bound = {name for name, _, _ in grx.SIGNATURES}
    assert set(_declared_functions()) == bound


def test_opts_struct_layout_matches_defaults(libgrx):
    o = grx.grx_opts()
    libgrx.grx_opts_default(ctypes.byref(o))
    assert o.direction == grx.GRX_DIR_AUTO
    assert abs(o.alpha - 0.01) < 1e-7 and abs(o.beta - 0.1) < 1e-7
    assert o.loop == grx.GRX_LOOP_PERSISTENT and o.timeout_s == 5.0
    assert o.push_bitmap == 0.0 and o.sssp_delta == 0      # library defaults: V/8 rule, no bands


def test_argument_errors_without_gpu():
    """Calls that fail argument checks return an error code before touching
    the device."""
    lib = grx.lib()
    assert lib.bfs(None, 0, None, None, None, None) == grx.GRX_EINVAL
    assert b"NULL graph" in lib.grx_last_error()
    assert lib.sssp(None, 0, None, None, None) == grx.GRX_EINVAL
    assert lib.cc(None, None, None) == grx.GRX_EINVAL
    assert lib.pagerank(None, 0.85, 20, None, None) == grx.GRX_EINVAL
    assert lib.bc(None, None, 1, None, None, None, None) == grx.GRX_EINVAL
    assert lib.bc_multi(None, None, 1, None, None, None) == grx.GRX_EINVAL
    assert lib.bfs_multi(None, None, 1, None, None, None) == grx.GRX_EINVAL
    assert lib.sssp_multi(None, None, 1, None, None, None) == grx.GRX_EINVAL
    out = ctypes.c_void_p()
    assert lib.graph_load_csr(None, 4, 0, None, 0, None, None, 0, None, ctypes.byref(out)) == grx.GRX_EINVAL
    assert lib.grx_rmat_edges(0, 10, 1, 0, 0, 0, None, None, None) == grx.GRX_EINVAL


def test_noalloc_argument_checks_without_gpu():
    """bfs_noalloc refuses the CUDA-graph loop (it would allocate) before any
    CUDA call, and its binding refuses tensors the library cannot read."""
    import torch
    lib = grx.lib()
    o = grx.opts(loop=grx.GRX_LOOP_GRAPH)
    # the pointers are never dereferenced: the option check comes first
    rc = lib.bfs_noalloc(16, 0, 16, None, 0, 16, None, None, ctypes.byref(o), None)
    assert rc == grx.GRX_EINVAL
    assert b"GRX_LOOP_GRAPH" in lib.grx_last_error()
    o = grx.opts(loop=7)
    assert lib.bfs_noalloc(16, 0, 16, None, 0, 16, None, None, ctypes.byref(o), None) == grx.GRX_EINVAL
    ro = torch.zeros(17, dtype=torch.int32)
    col = torch.zeros(0, dtype=torch.int32)
    with pytest.raises(ValueError, match="int32"):
        grx.bfs_noalloc(ro.to(torch.int64), col, 0)
    with pytest.raises(ValueError, match="CUDA"):
        grx.bfs_noalloc(ro, col, 0)
    with pytest.raises(ValueError, match="Tensor"):
        grx.bfs_noalloc([0] * 17, col, 0)
    assert grx.GRX_NOALLOC_SCRATCH_BYTES == _header_define("GRX_NOALLOC_SCRATCH_BYTES")
    assert grx.GRX_NOALLOC_MAX_NV == eval(_header_define("GRX_NOALLOC_MAX_NV", raw=True))


def _header_define(name, raw=False):
    for h in HEADERS:
        m = re.search(rf"^#define {name} (.+)$", open(h).read(), flags=re.M)
        if m:
            return m.group(1).strip() if raw else int(m.group(1))
    raise KeyError(name)


def test_64bit_vertex_id_entry_points_check_arguments_without_gpu():
    lib = grx.lib()
    out = ctypes.c_void_p()
    assert lib.graph_load_csr64(None, 4, 0, None, None, 0, None, ctypes.byref(out)) == grx.GRX_EINVAL
    assert lib.bfs64(None, 0, None, None, None, None) == grx.GRX_EINVAL
    assert b"NULL graph" in lib.grx_last_error()
