"""GPU parity at the benchmarked size: R-MAT scale 22 (ef 16, seed 22,
weights U[1,64] with seed 122), generated on the device and loaded with int32
offsets exactly as the benchmark's default workload, with the library's
launch configuration.  Every primitive is compared with the CPU oracle on
seeded sources of the benchmark's own source list: BFS depths, SSSP
distances and CC labels bit-exact, PageRank within 1e-5 relative, BC within
1e-9 relative, and two lanes of a 64-lane multi-source BFS.  R-MAT 24 and 26
check PageRank's 20-iteration result at every vertex."""
import os

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


# ---- the other benchmarked configurations at full size

def test_bfs_rmat16_sixteen_sources():
    """R-MAT scale 16 (65,536 vertices): plain BFS from the 16 seeded sources, bit-exact."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_1504_04804_gb300 import grx
    g = inputs.rmat_graph(16, 16, seed=16)
    dg = grx.load(g)
    for s in inputs.pick_sources(g.row_offsets, 16, 1):
        for mode in (0, 1):
            assert np.array_equal(grx.bfs(dg, int(s), opts=grx.opts(direction=mode)).cpu().numpy(),
                                  oracle.bfs(g.row_offsets, g.col_indices, int(s))), (int(s), mode)


def test_grid_4096_bfs_loops_and_sssp():
    """The 4096 x 4096 grid (10 % of edges deleted, weights U[1,1000]): BFS with
    the three level loops and SSSP (plain and near-far) from a bench source."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_1504_04804_gb300 import autotune, grx
    ro, col, w = grx.grid_graph_device(4096, 4096, p_del=0.1, seed=4096, wmax=1000, weight_seed=4196)
    g = grx.graph_load_csr(ro, col, w)
    roh, colh, wh = ro.cpu().numpy().astype(np.int64), col.cpu().numpy(), w.cpu().numpy().view(np.uint32)
    s = int(inputs.pick_sources(roh, 4, 1)[0])
    want = oracle.bfs(roh, colh, s)
    for loop in (grx.GRX_LOOP_PERSISTENT, grx.GRX_LOOP_HOST, grx.GRX_LOOP_GRAPH):
        assert np.array_equal(grx.bfs(g, s, opts=grx.opts(loop=loop)).cpu().numpy(), want), loop
    dist = oracle.sssp(roh, colh, wh, s)
    tuned = autotune.tune_sssp_delta(g, roh, wh, cache=None)
    for delta in (0, 20000, tuned["sssp_delta"]):
        assert np.array_equal(grx.as_uint32(grx.sssp(g, s, opts=grx.opts(sssp_delta=delta))), dist), delta
    grx.graph_status(g)


def check_lanes_parallel(ro, col, lanes, row_of, chunk=16):
    """oracle.check_bfs on every lane, `chunk` lanes at a time on host
    threads (the oracle's C calls release the GIL); row_of(b) gives lane b's
    depths as a host array.  Returns the violation count of each lane."""
    from concurrent.futures import ThreadPoolExecutor
    counts = []
    with ThreadPoolExecutor(max_workers=min(chunk, os.cpu_count() or 1)) as pool:
        for b0 in range(0, len(lanes), chunk):
            idx = range(b0, min(len(lanes), b0 + chunk))
            rows = [row_of(b) for b in idx]
            counts += list(pool.map(lambda br: oracle.check_bfs(ro, col, lanes[br[0]], br[1]),
                                    zip(idx, rows)))
    return counts


def _pr_max_rel_err(got, want):
    got = np.asarray(got, dtype=np.float64)
    rel = np.abs(got - want) / want
    v = int(np.argmax(rel))
    return float(rel[v]), v


def test_pagerank_rmat24_twenty_iterations():
    """R-MAT scale 24 (16.8M vertices, ~520M directed edges): the FP32 ranks
    after 20 iterations against the oracle's FP64 20-iteration result at every
    vertex, max relative error <= 1e-5 (hubs here sum over a million terms)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_1504_04804_gb300 import grx
    ro, col, _ = grx.rmat_graph_device(24, 16, seed=24)
    g = grx.graph_load_csr(ro, col, None)
    roh, colh = ro.cpu().numpy().astype(np.int64), col.cpu().numpy()
    got = grx.pagerank(g, 0.85, 20).cpu().numpy()
    grx.graph_status(g)
    want = oracle.pagerank(roh, colh, 0.85, 20)
    err, v = _pr_max_rel_err(got, want)
    assert err <= 1e-5, f"max relative error {err:.3e} at vertex {v} (degree {roh[v + 1] - roh[v]})"
    print(f"pagerank R-MAT 24: max relative error {err:.3e} at vertex {v}")


def test_rmat26_dobfs_multi_source_and_pagerank():
    """R-MAT scale 26 with int64 offsets, as the benchmark loads it: one
    DOBFS source and two of the 64 multi-source lanes bit-exact against the
    oracle, every lane against the BFS invariants on host threads, and nine
    lanes against single-source BFS on the GPU; the DOBFS source again with
    64-bit vertex ids (bfs64) equal to it; PageRank after 20 iterations
    against the oracle's FP64 20-iteration result at every vertex (max
    relative error <= 1e-5; the oracle runs on a host thread meanwhile)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if torch.cuda.mem_get_info()[0] < 60e9:
        pytest.skip("needs 60 GB of free device memory")
    build.build()
    from concurrent.futures import ThreadPoolExecutor
    from paper_1504_04804_gb300 import grx
    ro, col, _ = grx.rmat_graph_device(26, 16, seed=26)
    g = grx.graph_load_csr(ro, col, None, offsets64=True)
    roh, colh = ro.cpu().numpy().astype(np.int64), col.cpu().numpy()
    pool = ThreadPoolExecutor(max_workers=1)
    pr_want = pool.submit(oracle.pagerank, roh, colh, 0.85, 20)   # ~minutes of one core
    try:
        src = int(inputs.pick_sources(roh, 16, 1)[0])
        assert np.array_equal(grx.bfs(g, src).cpu().numpy(), oracle.bfs(roh, colh, src))
        lanes = [int(x) for x in inputs.pick_sources(roh, 64, 5)]
        d = grx.bfs_multi(g, lanes)
        for b in (0, 63):
            assert np.array_equal(d[b].cpu().numpy(), oracle.bfs(roh, colh, lanes[b])), b
        for b in range(1, 63, 7):
            assert torch.equal(d[b], grx.bfs(g, lanes[b])), b
        # every lane against the BFS invariants (multithreaded host checker)
        assert check_lanes_parallel(roh, colh, lanes, lambda b: d[b].cpu().numpy()) == [0] * 64
        del d
        # the same traversal with 64-bit vertex ids (every id, offset and count int64)
        g64 = grx.graph_load_csr64(ro.to(torch.int64), col.to(torch.int64))
        assert torch.equal(grx.bfs64(g64, src), grx.bfs(g, src))
        grx.graph_status(g64)
        g64.free()
        del g64
        torch.cuda.empty_cache()
        r20 = grx.pagerank(g, 0.85, 20).cpu().numpy()
        grx.graph_status(g)
        assert abs(r20.astype(np.float64).sum() - 1.0) < 1e-3
        err, v = _pr_max_rel_err(r20, pr_want.result())
        assert err <= 1e-5, f"max relative error {err:.3e} at vertex {v} (degree {roh[v + 1] - roh[v]})"
        print(f"pagerank R-MAT 26: max relative error {err:.3e} at vertex {v}")
    finally:
        pool.shutdown(wait=True)
