"""bfs_noalloc: the BFS entry point for callers that cannot allocate device
memory (a host framework that owns the GPU's memory pool, a loop where
cudaMalloc/cudaFree would synchronise the device, a request path that must
not run out of memory half-way).  It keeps all scratch in one fixed device
array inside the library, so two calls in a row must each clear what the
previous one left there.  The checks, through the C ABI: called several
times in a row (different sources, then the first again), in both level
loops that allocate nothing and in every direction mode, it returns exactly
the depths of the oracle's BFS and of the regular, allocating bfs() entry
point, with parents the oracle's checker accepts; an edgeless graph gives
the source alone; the CUDA-graph loop (which would allocate) and graphs
beyond the fixed scratch are refused.

This file is collected last on purpose; it also passes alone in a fresh
process (it sets up everything it needs)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1504_04804_gb300 import build, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def grx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    from paper_1504_04804_gb300 import grx as g
    return g


def _call_noalloc(grx, ro32, col, src, depth, parent, status, opts=None):
    """Direct C-ABI call of bfs_noalloc on device tensors; returns the status."""
    lib = grx.lib()
    return lib.bfs_noalloc(ro32.numel() - 1, col.numel(), ro32.data_ptr(),
                           col.data_ptr() if col.numel() else None, int(src),
                           depth.data_ptr(), parent.data_ptr() if parent is not None else None,
                           status.data_ptr() if status is not None else None,
                           ctypes.byref(opts) if opts is not None else None,
                           torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("scale", [14, 18])
def test_noalloc_matches_oracle_and_bfs_on_consecutive_calls(grx, scale):
    ro64, col, _ = grx.rmat_graph_device(scale, 16, seed=scale)
    assert ro64.numel() - 1 <= grx.GRX_NOALLOC_MAX_NV
    ro32 = ro64.to(torch.int32)
    g = grx.graph_load_csr(ro64, col)
    ro_h, col_h = ro64.cpu().numpy(), col.cpu().numpy()
    srcs = [int(s) for s in inputs.pick_sources(ro_h, 2, seed=scale)]
    want = {s: oracle.bfs(ro_h, col_h, s) for s in srcs}
    nv = g.nv
    depth = torch.empty(nv, dtype=torch.int32, device="cuda")
    parent = torch.empty(nv, dtype=torch.int32, device="cuda")
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    for loop in (grx.GRX_LOOP_PERSISTENT, grx.GRX_LOOP_HOST):
        for mode in (grx.GRX_DIR_AUTO, grx.GRX_DIR_PUSH, grx.GRX_DIR_PULL):
            o = grx.opts(direction=mode, loop=loop)
            for s in (srcs[0], srcs[1], srcs[0]):       # consecutive calls share the scratch
                depth.fill_(-7)
                parent.fill_(-7)
                rc = _call_noalloc(grx, ro32, col, s, depth, parent, status, o)
                assert rc == grx.GRX_OK, grx.lib().grx_last_error()
                got = depth.cpu().numpy()
                assert np.array_equal(got, want[s]), (scale, loop, mode, s)
                assert np.array_equal(got, grx.bfs(g, s, opts=o).cpu().numpy())
                assert int(status.item()) == 0
                assert oracle.check_bfs(ro_h, col_h, s, got, parent.cpu().numpy()) == 0


def test_noalloc_edgeless_graph(grx):
    nv = 1000
    ro = torch.zeros(nv + 1, dtype=torch.int32, device="cuda")
    col = torch.empty(0, dtype=torch.int32, device="cuda")
    depth = torch.empty(nv, dtype=torch.int32, device="cuda")
    parent = torch.empty(nv, dtype=torch.int32, device="cuda")
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    for loop in (grx.GRX_LOOP_PERSISTENT, grx.GRX_LOOP_HOST):
        for s in (3, 999):
            rc = _call_noalloc(grx, ro, col, s, depth, parent, status, grx.opts(loop=loop))
            assert rc == grx.GRX_OK, grx.lib().grx_last_error()
            want = np.full(nv, -1, np.int32)
            want[s] = 0
            assert np.array_equal(depth.cpu().numpy(), want)
            p = np.full(nv, -1, np.int32)
            p[s] = s
            assert np.array_equal(parent.cpu().numpy(), p)
            assert int(status.item()) == 0


def test_noalloc_refuses_the_graph_loop_and_stays_usable(grx):
    ro64, col, _ = grx.rmat_graph_device(12, 16, seed=12)
    ro32 = ro64.to(torch.int32)
    ro_h, col_h = ro64.cpu().numpy(), col.cpu().numpy()
    s = int(inputs.pick_sources(ro_h, 1, seed=3)[0])
    nv = ro32.numel() - 1
    depth = torch.empty(nv, dtype=torch.int32, device="cuda")
    rc = _call_noalloc(grx, ro32, col, s, depth, None, None, grx.opts(loop=grx.GRX_LOOP_GRAPH))
    assert rc == grx.GRX_EINVAL
    assert b"GRX_LOOP_GRAPH" in grx.lib().grx_last_error()
    with pytest.raises(grx.GrxError):
        grx.bfs_noalloc(ro32, col, s, opts=grx.opts(loop=grx.GRX_LOOP_GRAPH))
    # the next call runs normally
    got = grx.bfs_noalloc(ro32, col, s, depth_out=depth)
    assert np.array_equal(got.cpu().numpy(), oracle.bfs(ro_h, col_h, s))
    with pytest.raises(ValueError):
        grx.bfs_noalloc(ro64, col, s)                   # int64 offsets are refused


def test_noalloc_rejects_graphs_beyond_its_fixed_scratch(grx):
    lib = grx.lib()
    nv = grx.GRX_NOALLOC_MAX_NV + 1
    ro = torch.zeros(nv + 1, dtype=torch.int32, device="cuda")
    depth = torch.empty(nv, dtype=torch.int32, device="cuda")
    rc = lib.bfs_noalloc(nv, 0, ro.data_ptr(), None, 0, depth.data_ptr(), None, None, None,
                         torch.cuda.current_stream().cuda_stream)
    assert rc == grx.GRX_ERANGE
    assert b"at most" in lib.grx_last_error()
