"""Continuous batching: the admission policy (host logic) and, on the GPU,
that every query's result is the same alone and in the mix -- lanes joining
a traversal already in flight, several graphs and both kinds at once."""
import numpy as np
import pytest

import oracle
from paper_1504_04804_gb300 import inputs, serving


def _req(rid, graph, kind="bfs"):
    return serving.Request(rid, graph, kind, 0, 0.0)


def test_plan_admission_lanes_and_memory():
    fp = {("a", "bfs"): 1000, ("b", "bfs"): 5000}
    ob = {("a", "bfs"): 10, ("b", "bfs"): 10}
    pend = [_req(0, "a"), _req(1, "b"), _req(2, "a")]
    # a has one free lane, b has none and no room for a new batch
    admit, new, wait = serving.plan_admission(pend, {("a", "bfs"): 1}, 2000, fp, ob, {})
    assert [r.rid for r in admit] == [0, 2] and new == [("a", "bfs")] and [r.rid for r in wait] == [1]
    # plenty of memory: one new batch per key, lanes reused afterwards
    admit, new, wait = serving.plan_admission(pend, {}, 10**9, fp, ob, {})
    assert [r.rid for r in admit] == [0, 1, 2] and sorted(new) == [("a", "bfs"), ("b", "bfs")]
    assert wait == []
    # no memory at all: nothing is admitted
    admit, new, wait = serving.plan_admission(pend, {}, 5, fp, ob, {})
    assert admit == [] and new == [] and len(wait) == 3


def test_make_requests_poisson_and_seeded():
    g = inputs.rmat_graph(10, 8, seed=1)
    graphs = {"g1": (g.row_offsets, True), "g2": (g.row_offsets, False)}
    r1 = serving.make_requests(graphs, 500, rate_qps=1000.0, seed=3)
    r2 = serving.make_requests(graphs, 500, rate_qps=1000.0, seed=3)
    assert [(r.graph, r.kind, r.src, r.arrival) for r in r1] == [(r.graph, r.kind, r.src, r.arrival) for r in r2]
    gaps = np.diff([r.arrival for r in r1])
    assert abs(gaps.mean() - 1e-3) < 2.5e-4                     # exponential, mean 1/rate
    assert all(r.kind == "bfs" for r in r1 if r.graph == "g2")  # unweighted: BFS only
    assert np.all(np.diff(g.row_offsets)[[r.src for r in r1]] > 0)


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_04804_gb300 import build, grx
    build.build()
    return torch, grx


def _graphs():
    return {
        "r11": inputs.rmat_graph(11, 16, seed=11, wmax=64, weight_seed=111),
        "r12": inputs.rmat_graph(12, 8, seed=12, wmax=64, weight_seed=112),
        "grid": inputs.grid_graph(40, 30, p_del=0.1, seed=40, wmax=1000, weight_seed=4),
    }


@pytest.mark.gpu
def test_batch_lanes_joining_mid_traversal(gpu):
    torch, grx = gpu
    g = _graphs()["grid"]
    dg = grx.load(g)
    for kind in (grx.GRX_KIND_BFS, grx.GRX_KIND_SSSP):
        b = grx.Batch(dg, kind)
        srcs = [int(s) for s in inputs.pick_sources(g.row_offsets, 5, seed=kind + 3)]
        outs, done = {}, 0
        for i, s in enumerate(srcs):                   # one new lane every 7 levels
            out = torch.empty(g.nv, dtype=torch.int32, device="cuda")
            lane = b.admit(s, out)
            outs[lane] = (s, out)
            b.step(7)
            done |= b.poll()
        for _ in range(10000):
            if done == sum(1 << l for l in outs):
                break
            b.step(4)
            done |= b.poll()
        assert done == sum(1 << l for l in outs)
        for lane, (s, out) in outs.items():
            if kind == grx.GRX_KIND_BFS:
                assert np.array_equal(out.cpu().numpy(), oracle.bfs(g.row_offsets, g.col_indices, s))
            else:
                assert np.array_equal(out.cpu().numpy().view(np.uint32),
                                      oracle.sssp(g.row_offsets, g.col_indices, g.weights, s))
        # the freed lanes serve new queries correctly
        s = srcs[0]
        out = torch.empty(g.nv, dtype=torch.int32, device="cuda")
        b.admit(s, out)
        while not b.poll():
            b.step(8)
        want = (oracle.bfs(g.row_offsets, g.col_indices, s) if kind == grx.GRX_KIND_BFS
                else oracle.sssp(g.row_offsets, g.col_indices, g.weights, s).view(np.int32))
        assert np.array_equal(out.cpu().numpy(), want)
        b.close()


@pytest.mark.gpu
def test_server_results_same_alone_and_in_the_mix(gpu):
    torch, grx = gpu
    hg = _graphs()
    graphs = {k: grx.load(v) for k, v in hg.items()}
    degrees = {k: torch.from_numpy(np.diff(v.row_offsets).astype(np.int32)).cuda() for k, v in hg.items()}
    reqs = serving.make_requests({k: (v.row_offsets, True) for k, v in hg.items()}, 300,
                                 rate_qps=20000.0, seed=5)
    srv = serving.Server(graphs, degrees, steps_per_poll=1, keep_results=True)
    stats = srv.run(reqs)
    srv.close()
    assert stats["queries"] == 300 and stats["p99_ms"] >= stats["p50_ms"] > 0
    joined_late = 0
    for r in reqs:
        g = hg[r.graph]
        got = r.result.cpu().numpy()
        if r.kind == "bfs":
            want = oracle.bfs(g.row_offsets, g.col_indices, r.src)
            assert np.array_equal(got, want), r
            assert r.edges == int(np.diff(g.row_offsets)[want >= 0].sum())
        else:
            want = oracle.sssp(g.row_offsets, g.col_indices, g.weights, r.src)
            assert np.array_equal(got.view(np.uint32), want), r
        joined_late += r.admitted > 0
    assert joined_late > 0
    # a sample of queries run alone through the single-source entry points
    for r in reqs[:20]:
        alone = grx.bfs(graphs[r.graph], r.src) if r.kind == "bfs" else grx.sssp(graphs[r.graph], r.src)
        assert np.array_equal(alone.cpu().numpy(), r.result.cpu().numpy())


@pytest.mark.gpu
def test_server_rejects_when_nothing_fits(gpu):
    torch, grx = gpu
    g = inputs.rmat_graph(10, 8, seed=2)
    graphs = {"g": grx.load(g)}
    degrees = {"g": torch.from_numpy(np.diff(g.row_offsets).astype(np.int32)).cuda()}
    reqs = serving.make_requests({"g": (g.row_offsets, False)}, 3, rate_qps=0, seed=1)
    srv = serving.Server(graphs, degrees, budget_bytes=1024)
    with pytest.raises(RuntimeError, match="admission impossible"):
        srv.run(reqs, realtime=False)


def test_plan_job_oldest_key_first_and_batch_thresholds():
    def reqs(key, times, base):
        return [serving.Request(base + i, key[0], key[1], 0, t) for i, t in enumerate(times)]
    pend = {("a", "bfs"): reqs(("a", "bfs"), [0.3, 0.4], 0),
            ("b", "sssp"): reqs(("b", "sssp"), [0.1, 0.2, 0.5], 10),
            ("c", "bfs"): []}
    key, batch, multi = serving.plan_job(pend, sssp_multi_min=3)
    assert key == ("b", "sssp") and multi and [r.rid for r in batch] == [10, 11, 12]
    key, batch, multi = serving.plan_job(pend, sssp_multi_min=4)
    assert key == ("b", "sssp") and not multi and [r.rid for r in batch] == [10]
    pend[("b", "sssp")] = []
    key, batch, multi = serving.plan_job(pend)
    assert key == ("a", "bfs") and multi and len(batch) == 2
    pend[("a", "bfs")] = reqs(("a", "bfs"), [0.3], 0)
    assert serving.plan_job(pend)[2] is False                     # one BFS request runs alone
    many = {("a", "bfs"): reqs(("a", "bfs"), [i * 1e-3 for i in range(100)], 0)}
    assert len(serving.plan_job(many)[1]) == 64                   # at most 64 lanes
    assert serving.plan_job({("a", "bfs"): []}) is None


@pytest.mark.gpu
def test_traversal_server_results_same_alone_and_in_the_mix(gpu):
    torch, grx = gpu
    hg = _graphs()
    graphs = {k: grx.load(v) for k, v in hg.items()}
    degrees = {k: torch.from_numpy(np.diff(v.row_offsets).astype(np.int32)).cuda() for k, v in hg.items()}
    reqs = serving.make_requests({k: (v.row_offsets, True) for k, v in hg.items()}, 300,
                                 rate_qps=20000.0, seed=6)
    srv = serving.TraversalServer(graphs, degrees, sssp_multi_min=4, keep_results=True)
    stats = srv.run(reqs)
    assert stats["queries"] == 300 and stats["p99_ms"] >= stats["p50_ms"] > 0
    for r in reqs:
        g = hg[r.graph]
        got = r.result.cpu().numpy()
        if r.kind == "bfs":
            want = oracle.bfs(g.row_offsets, g.col_indices, r.src)
            assert np.array_equal(got, want), r
            assert r.edges == int(np.diff(g.row_offsets)[want >= 0].sum())
        else:
            want = oracle.sssp(g.row_offsets, g.col_indices, g.weights, r.src)
            assert np.array_equal(got.view(np.uint32), want), r
    for r in reqs[:20]:
        alone = grx.bfs(graphs[r.graph], r.src) if r.kind == "bfs" else grx.sssp(graphs[r.graph], r.src)
        assert np.array_equal(alone.cpu().numpy(), r.result.cpu().numpy())


def test_plan_job_skips_graphs_with_a_traversal_in_flight():
    pend = {("a", "bfs"): [serving.Request(0, "a", "bfs", 0, 0.1)],
            ("b", "bfs"): [serving.Request(1, "b", "bfs", 0, 0.2)]}
    assert serving.plan_job(pend)[0] == ("a", "bfs")
    assert serving.plan_job(pend, busy={"a"})[0] == ("b", "bfs")
    assert serving.plan_job(pend, busy={"a", "b"}) is None


def test_plan_lanes_admits_by_free_memory():
    # everything fits
    assert serving.plan_lanes(64, 1000, 10, 10**6, others_running=True) == 64
    assert serving.plan_lanes(64, 1000, 10, 1000 + 640, others_running=False) == 64
    # does not fit while others run: wait for their memory
    assert serving.plan_lanes(64, 1000, 10, 1000 + 639, others_running=True) == 0
    # nothing else runs: as many lanes as fit
    assert serving.plan_lanes(64, 1000, 10, 1000 + 639, others_running=False) == 63
    assert serving.plan_lanes(64, 0, 10, 15, others_running=False) == 1
    assert serving.plan_lanes(0, 0, 10, 15, others_running=False) == 0
    with pytest.raises(MemoryError):
        serving.plan_lanes(64, 1000, 10, 1005, others_running=False)


@pytest.mark.gpu
def test_multi_footprint_matches_what_the_first_call_allocates(gpu):
    torch, grx = gpu
    hg = inputs.rmat_graph(13, 16, seed=13, wmax=64, weight_seed=113)
    for kind, fn in ((grx.GRX_KIND_BFS, grx.bfs_multi), (grx.GRX_KIND_SSSP, grx.sssp_multi)):
        g = grx.load(hg)
        srcs = [int(s) for s in inputs.pick_sources(hg.row_offsets, 8, seed=2)]
        out = torch.empty(8 * g.nv, dtype=torch.int32, device="cuda")
        want = grx.multi_footprint(g, kind)
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        fn(g, srcs, out)
        torch.cuda.synchronize()
        got = torch.cuda.memory_allocated() - before
        # torch's caching allocator rounds each block up to 512 bytes
        assert want <= got <= want + 512 * 40, (kind, want, got)
        assert grx.multi_footprint(g, kind) == 0
        g.free()


@pytest.mark.gpu
def test_traversal_server_under_a_tiny_memory_budget(gpu):
    """A budget that holds the workspace and only a few lanes' outputs: the
    server starts smaller traversals (and waits for memory while one runs),
    and every result is still the query's own single-source result."""
    torch, grx = gpu
    hg = {"r11": inputs.rmat_graph(11, 16, seed=11, wmax=64, weight_seed=111)}
    graphs = {k: grx.load(v) for k, v in hg.items()}
    degrees = {k: torch.from_numpy(np.diff(v.row_offsets).astype(np.int32)).cuda() for k, v in hg.items()}
    g = graphs["r11"]
    ws = max(grx.multi_footprint(g, grx.GRX_KIND_BFS), grx.multi_footprint(g, grx.GRX_KIND_SSSP))
    lane = 9 * g.nv + 64
    budget = grx.multi_footprint(g, grx.GRX_KIND_BFS) + grx.multi_footprint(g, grx.GRX_KIND_SSSP) + 6 * lane
    reqs = serving.make_requests({k: (v.row_offsets, True) for k, v in hg.items()}, 120,
                                 rate_qps=0.0, seed=8)
    srv = serving.TraversalServer(graphs, degrees, sssp_multi_min=2, keep_results=True,
                                  budget_bytes=budget)
    stats = srv.run(reqs, realtime=False)
    assert stats["queries"] == 120 and stats["shrunk"] > 0
    assert srv.used <= budget and ws > 0
    h = hg["r11"]
    for r in reqs:
        got = r.result.cpu().numpy()
        if r.kind == "bfs":
            assert np.array_equal(got, oracle.bfs(h.row_offsets, h.col_indices, r.src)), r
        else:
            assert np.array_equal(got.view(np.uint32),
                                  oracle.sssp(h.row_offsets, h.col_indices, h.weights, r.src)), r


def test_batch_threshold_from_measured_times():
    # 8 lanes cost less than 8 single traversals: batch from 8, up to 64
    assert serving.batch_threshold(1.0, {8: 5.0, 64: 30.0}) == (8, 64)
    # only the full batch wins
    assert serving.batch_threshold(1.0, {8: 9.0, 64: 60.0}) == (64, 64)
    # never wins: never batch
    assert serving.batch_threshold(1.0, {8: 40.0, 64: 240.0}) == (65, 64)
    # a latency bound: batches of up to 16 lanes take at most 12 ms
    assert serving.batch_threshold(1.0, {8: 5.0, 16: 9.0, 64: 30.0}, max_ms=12.0) == (8, 16)
    assert serving.batch_threshold(1.0, {8: 5.0, 64: 30.0}, max_ms=4.0) == (65, 64)
    pend = {("a", "sssp"): [serving.Request(i, "a", "sssp", 0, 0.1 * i) for i in range(20)]}
    assert serving.plan_job(pend, thresholds={("a", "sssp"): (65, 64)})[2] is False
    key, reqs, multi = serving.plan_job(pend, thresholds={("a", "sssp"): (8, 16)})
    assert multi and len(reqs) == 16
