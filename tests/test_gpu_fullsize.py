"""GPU parity at the benchmarked size: R-MAT scale 22 (ef 16, seed 22,
weights U[1,64] with seed 122), generated on the device and loaded with int32
offsets exactly as the benchmark's default workload, with the library's
launch configuration.  Every primitive is compared with the CPU oracle on
seeded sources of the benchmark's own source list: BFS depths, SSSP
distances and CC labels bit-exact, PageRank within 1e-5 relative, BC within
1e-9 relative, and two lanes of a 64-lane multi-source BFS."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1504_04804_gb300 import build, inputs

pytestmark = pytest.mark.gpu

SCALE, EF, SEED, WMAX, WSEED = 22, 16, 22, 64, 122


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_1504_04804_gb300 import grx
    ro, col, w = grx.rmat_graph_device(SCALE, EF, seed=SEED, wmax=WMAX, weight_seed=WSEED)
    g = grx.graph_load_csr(ro, col, w, validate=False)
    host = (ro.cpu().numpy().astype(np.int64), col.cpu().numpy(), w.cpu().numpy().view(np.uint32))
    srcs = [int(s) for s in inputs.pick_sources(host[0], 16, 1)]
    return grx, g, host, srcs


def test_bfs_and_multi_source_bfs_at_scale_22(big):
    grx, g, (ro, col, _), srcs = big
    for s in srcs[:2]:
        want = oracle.bfs(ro, col, s)
        for kw in ({}, {"alpha": 1e-5, "beta": 0.01}, {"direction": 1}):
            assert np.array_equal(grx.bfs(g, s, opts=grx.opts(**kw)).cpu().numpy(), want), (s, kw)
    lanes = [int(x) for x in inputs.pick_sources(ro, 64, 5)]
    d = grx.bfs_multi(g, lanes)
    for b in (0, 63):
        assert np.array_equal(d[b].cpu().numpy(), oracle.bfs(ro, col, lanes[b]))


def test_sssp_cc_pagerank_at_scale_22(big):
    grx, g, (ro, col, w), srcs = big
    want = oracle.sssp(ro, col, w, srcs[0])
    for delta in (0, 64):
        got = grx.as_uint32(grx.sssp(g, srcs[0], opts=grx.opts(sssp_delta=delta)))
        assert np.array_equal(got, want), delta
    assert np.array_equal(grx.cc(g).cpu().numpy(), oracle.cc(ro, col))
    r = grx.pagerank(g, 0.85, 20).cpu().numpy().astype(np.float64)
    pr = oracle.pagerank(ro, col, 0.85, 20)
    assert np.max(np.abs(r - pr) / pr) <= 1e-5


def test_bc_at_scale_22(big):
    grx, g, (ro, col, _), srcs = big
    want, wsig = oracle.bc(ro, col, [srcs[0]], want_sigma=True)
    for mode in (0, 1, 2):
        got, sig = grx.bc(g, [srcs[0]], want_sigma=True, opts=grx.opts(direction=mode))
        np.testing.assert_allclose(got.cpu().numpy(), want, rtol=1e-9, atol=0, err_msg=str(mode))
        np.testing.assert_allclose(sig.cpu().numpy(), wsig, rtol=1e-12, atol=0, err_msg=str(mode))


def test_bc_multi_at_scale_22(big):
    grx, g, (ro, col, _), srcs = big
    lanes = [int(x) for x in inputs.pick_sources(ro, 16, 5)]       # the oracle takes ~1.5 s per source
    got = grx.bc_multi(g, lanes).cpu().numpy()
    grx.graph_status(g)
    np.testing.assert_allclose(got, oracle.bc(ro, col, lanes), rtol=1e-9, atol=0)
