"""bfs_noalloc: the BFS entry point for callers that cannot allocate device
memory (a host framework that owns the GPU's memory pool, a loop where
cudaMalloc/cudaFree would synchronise the device, a request path that must
not run out of memory half-way).  It keeps all scratch in one fixed device
array inside the library, so two calls in a row must each clear what the
previous one left there.  The check: called through the C ABI, twice in a row
(different sources, then the first again), it returns exactly the depths the
regular, allocating bfs() entry point returns.

This file is collected last on purpose; it also passes alone in a fresh
process (it sets up everything it needs)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1504_04804_gb300 import build, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def grx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_1504_04804_gb300 import grx as g
    return g


def _call_noalloc(grx, ro32, col, src, depth, parent, status, opts=None):
    """Direct C-ABI call of bfs_noalloc on device tensors."""
    lib = grx.lib()
    rc = lib.bfs_noalloc(ro32.numel() - 1, col.numel(), ro32.data_ptr(), col.data_ptr(), int(src),
                         depth.data_ptr(), parent.data_ptr() if parent is not None else None,
                         status.data_ptr(), ctypes.byref(opts) if opts is not None else None,
                         torch.cuda.current_stream().cuda_stream)
    assert rc == grx.GRX_OK, lib.grx_last_error()


@pytest.mark.parametrize("scale", [14, 18])
def test_noalloc_matches_bfs_on_consecutive_calls(grx, scale):
    ro64, col, _ = grx.rmat_graph_device(scale, 16, seed=scale)
    assert ro64.numel() - 1 <= grx.GRX_NOALLOC_MAX_NV
    ro32 = ro64.to(torch.int32)
    g = grx.graph_load_csr(ro64, col)
    srcs = [int(s) for s in inputs.pick_sources(ro64.cpu().numpy(), 2, seed=scale)]
    nv = g.nv
    depth = torch.empty(nv, dtype=torch.int32, device="cuda")
    parent = torch.empty(nv, dtype=torch.int32, device="cuda")
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    for mode in (grx.GRX_DIR_AUTO, grx.GRX_DIR_PUSH):
        o = grx.opts(direction=mode)
        for s in (srcs[0], srcs[1], srcs[0]):           # consecutive calls share the scratch
            _call_noalloc(grx, ro32, col, s, depth, parent, status, o)
            want = grx.bfs(g, s, opts=o).cpu().numpy()
            got = depth.cpu().numpy()
            assert np.array_equal(got, want), (scale, mode, s)
            assert int(status.item()) == 0
            p = parent.cpu().numpy()
            assert p[s] == s and np.all((p >= 0) == (want >= 0))
            reached = np.flatnonzero((want > 0))
            assert np.all(want[p[reached]] == want[reached] - 1)


def test_noalloc_rejects_graphs_beyond_its_fixed_scratch(grx):
    lib = grx.lib()
    nv = grx.GRX_NOALLOC_MAX_NV + 1
    ro = torch.zeros(nv + 1, dtype=torch.int32, device="cuda")
    depth = torch.empty(nv, dtype=torch.int32, device="cuda")
    rc = lib.bfs_noalloc(nv, 0, ro.data_ptr(), None, 0, depth.data_ptr(), None, None, None,
                         torch.cuda.current_stream().cuda_stream)
    assert rc == grx.GRX_ERANGE
    assert b"at most" in lib.grx_last_error()
