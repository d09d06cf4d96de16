"""GPU parity: every libgrx entry point against the CPU oracle on the same
seeded inputs.  BFS depths, SSSP distances and CC labels must match
bit-for-bit; FP32 PageRank within a max relative error of 1e-5 per vertex
against the FP64 oracle.  Parents (several valid answers) are checked by the
oracle's invariant checker."""
import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1504_04804_gb300 import build, inputs

pytestmark = pytest.mark.gpu

PR_TOL = 1e-5
MODES = {"auto": 0, "push": 1, "pull": 2}


@pytest.fixture(scope="module")
def grx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_1504_04804_gb300 import grx as g
    return g


def _ragged_edges(nh):
    edges, leaf = [], nh
    for h in range(nh):
        if h + 1 < nh:
            edges.append((h, h + 1))
        for _ in range(h + 1):
            edges.append((h, leaf))
            leaf += 1
    return edges


def _graphs():
    gs = {
        "rmat10": inputs.rmat_graph(10, 16, seed=10, wmax=64, weight_seed=110),
        "rmat13": inputs.rmat_graph(13, 16, seed=13, wmax=64, weight_seed=113),
        "rmat14_ef4": inputs.rmat_graph(14, 4, seed=7, wmax=1000, weight_seed=3),
        "grid64": inputs.grid_graph(64, 48, p_del=0.1, seed=64, wmax=1000, weight_seed=9),
        "path": inputs.csr_from_edges(3000, [(i, i + 1) for i in range(2999)]),
        "star": inputs.csr_from_edges(5001, [(0, i) for i in range(1, 5001)]),
        "disconnected": inputs.csr_from_edges(
            40, [(1, 2), (2, 3), (3, 1), (5, 6), (10, 11), (11, 12), (12, 13), (30, 31)]),
        # rows of every length from 1 to 600 (hub h owns a block of h + 1 leaves, the
        # hubs chained): row boundaries fall at every offset of the per-thread,
        # per-lane and per-warp edge runs of the tiled kernels
        "ragged": inputs.csr_from_edges(600 + 600 * 601 // 2, _ragged_edges(600)),
    }
    for name in ("path", "star", "disconnected", "ragged"):
        g = gs[name]
        rows = np.repeat(np.arange(g.nv), np.diff(g.row_offsets))
        lo = np.minimum(rows, g.col_indices).astype(np.uint64)
        hi = np.maximum(rows, g.col_indices).astype(np.uint64)
        g.weights = (1 + inputs.draw(5, lo * np.uint64(g.nv) + hi) % np.uint64(50)).astype(np.uint32)
    return gs


GRAPHS = _graphs()


def _sources(g, n, seed=1):
    n = min(n, int(np.count_nonzero(np.diff(g.row_offsets))))
    return [int(s) for s in inputs.pick_sources(g.row_offsets, n, seed)]


@pytest.fixture(scope="module")
def loaded(grx):
    return {name: grx.load(g, validate=True) for name, g in GRAPHS.items()}


# push levels: library default threshold, bitmap marking on every push
# level, queue push only
PUSH_BITMAP = {"pbdefault": 0.0, "pbalways": 1e-9, "pbnever": -1.0}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("pb", list(PUSH_BITMAP))
def test_bfs_matches_oracle(grx, loaded, name, mode, pb):
    g, dg = GRAPHS[name], loaded[name]
    o = grx.opts(direction=MODES[mode], push_bitmap=PUSH_BITMAP[pb])
    for s in _sources(g, 4) + [g.nv - 1]:
        for want_parent in (True, False):
            if want_parent:
                d, p = grx.bfs(dg, s, opts=o, parent=True)
            else:
                d = grx.bfs(dg, s, opts=o)
            grx.graph_status(dg)
            want = oracle.bfs(g.row_offsets, g.col_indices, s)
            got = d.cpu().numpy()
            assert np.array_equal(got, want), (name, mode, pb, s, np.flatnonzero(got != want)[:10])
            if want_parent:
                assert oracle.check_bfs(g.row_offsets, g.col_indices, s, got, p.cpu().numpy()) == 0


@pytest.mark.parametrize("alpha,beta,exact", [(0.01, 0.1, 0), (1e-4, 1e-3, 0), (0.5, 0.05, 0),
                                              (1e-6, 10.0, 0), (0.01, 0.1, 1), (0.2, 0.5, 1)])
def test_dobfs_independent_of_switch_parameters(grx, loaded, alpha, beta, exact):
    g, dg = GRAPHS["rmat13"], loaded["rmat13"]
    o = grx.opts(alpha=alpha, beta=beta, exact_fv=exact, collect_stats=1)
    for s in _sources(g, 3, seed=4):
        d = grx.bfs(dg, s, opts=o)
        st = grx.last_stats(dg)
        assert np.array_equal(d.cpu().numpy(), oracle.bfs(g.row_offsets, g.col_indices, s))
        assert st["levels"] >= 1 and st["frontier"][0] == 1


def test_dobfs_switches_direction(grx, loaded):
    g, dg = GRAPHS["rmat13"], loaded["rmat13"]
    o = grx.opts(collect_stats=1)
    s = _sources(g, 1)[0]
    grx.bfs(dg, s, opts=o)
    st = grx.last_stats(dg)
    assert 1 in st["dir"], st["dir"]
    want = oracle.bfs(g.row_offsets, g.col_indices, s)
    assert st["levels"] == want.max() + 1
    # newly discovered per level equals the oracle's level sizes
    sizes = np.bincount(want[want >= 0])
    assert st["discovered"][: len(sizes) - 1] == list(sizes[1:])


@pytest.mark.parametrize("loop", ["host", "graph"])
def test_bfs_host_stepped_and_cuda_graph_loops(grx, loaded, loop):
    mode = grx.GRX_LOOP_HOST if loop == "host" else grx.GRX_LOOP_GRAPH
    for name in ("rmat10", "path", "grid64", "star", "disconnected"):
        g, dg = GRAPHS[name], loaded[name]
        for direction, pb in itertools.product((0, 1, 2), (0.0, 1e-9, -1.0)):
            o = grx.opts(loop=mode, direction=direction, push_bitmap=pb)
            for s in _sources(g, 2, seed=2) + [g.nv - 1]:
                d, p = grx.bfs(dg, s, opts=o, parent=True)
                grx.graph_status(dg)
                want = oracle.bfs(g.row_offsets, g.col_indices, s)
                assert np.array_equal(d.cpu().numpy(), want), (loop, name, direction, pb, s)
                assert oracle.check_bfs(g.row_offsets, g.col_indices, s, d.cpu().numpy(),
                                        p.cpu().numpy()) == 0


def test_bfs_small_grids(grx, loaded):
    g, dg = GRAPHS["rmat13"], loaded["rmat13"]
    for blocks in (1, 2, 7, 152):
        o = grx.opts(grid_blocks=blocks)
        s = _sources(g, 1, seed=blocks)[0]
        d = grx.bfs(dg, s, opts=o)
        assert np.array_equal(d.cpu().numpy(), oracle.bfs(g.row_offsets, g.col_indices, s))


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("pb", list(PUSH_BITMAP))
@pytest.mark.parametrize("delta", [0, 1, 7, 300])
def test_sssp_matches_oracle(grx, loaded, name, pb, delta):
    g, dg = GRAPHS[name], loaded[name]
    o = grx.opts(push_bitmap=PUSH_BITMAP[pb], sssp_delta=delta)
    for s in _sources(g, 3) + [g.nv - 1]:
        d = grx.sssp(dg, s, opts=o)
        grx.graph_status(dg)
        got = grx.as_uint32(d)
        want = oracle.sssp(g.row_offsets, g.col_indices, g.weights, s)
        assert np.array_equal(got, want), (name, pb, delta, s)


@pytest.mark.parametrize("name", list(GRAPHS))
def test_cc_matches_oracle(grx, loaded, name):
    g, dg = GRAPHS[name], loaded[name]
    lab = grx.cc(dg)
    grx.graph_status(dg)
    assert np.array_equal(lab.cpu().numpy(), oracle.cc(g.row_offsets, g.col_indices))


@pytest.mark.parametrize("name", list(GRAPHS))
def test_pagerank_matches_oracle(grx, loaded, name):
    g, dg = GRAPHS[name], loaded[name]
    for iters in (0, 1, 20):
        r = grx.pagerank(dg, 0.85, iters).cpu().numpy().astype(np.float64)
        want = oracle.pagerank(g.row_offsets, g.col_indices, 0.85, iters)
        rel = np.max(np.abs(r - want) / want)
        assert rel <= PR_TOL, (name, iters, rel)
        assert abs(r.sum() - 1.0) < 1e-4


@pytest.mark.parametrize("name", list(GRAPHS))
def test_pagerank_column_blocks_match_oracle(grx, loaded, name):
    """Column-blocked gathers (forced small blocks: many passes per
    iteration, rows split into many segments) within the same tolerance."""
    g, dg = GRAPHS[name], loaded[name]
    finest = max(1, int(np.ceil(np.log2(g.nv / 256))))      # at most 256 blocks
    try:
        for shift in sorted({finest, max(finest, int(np.log2(g.nv)) - 2)}):
            if (g.nv >> shift) < 1:
                continue
            grx.pagerank_block(dg, shift)
            for iters in (1, 20):
                r = grx.pagerank(dg, 0.85, iters).cpu().numpy().astype(np.float64)
                want = oracle.pagerank(g.row_offsets, g.col_indices, 0.85, iters)
                rel = np.max(np.abs(r - want) / want)
                assert rel <= PR_TOL, (name, shift, iters, rel)
        if g.nv > 2 * 256:
            with pytest.raises(grx.GrxError):
                grx.pagerank_block(dg, 1)                     # too many blocks
    finally:
        grx.pagerank_block(dg, 0)


def test_exhaustive_6_vertex_graphs_as_one_union(grx):
    """All 2^15 labelled graphs on 6 vertices as one disjoint union: CC over
    the union, BFS/SSSP from a vertex of a seeded sample of the graphs."""
    pairs = list(itertools.combinations(range(6), 2))
    edges = []
    for gi in range(1 << 15):
        base = 6 * gi
        edges += [(base + a, base + b) for i, (a, b) in enumerate(pairs) if gi >> i & 1]
    u = inputs.csr_from_edges(6 << 15, edges)
    rows = np.repeat(np.arange(u.nv), np.diff(u.row_offsets))
    lo = np.minimum(rows, u.col_indices).astype(np.uint64)
    hi = np.maximum(rows, u.col_indices).astype(np.uint64)
    u.weights = (1 + inputs.draw(66, lo * np.uint64(u.nv) + hi) % np.uint64(3)).astype(np.uint32)
    du = grx.load(u, validate=True)
    assert np.array_equal(grx.cc(du).cpu().numpy(), oracle.cc(u.row_offsets, u.col_indices))
    rng = np.random.default_rng(6)
    for gi in rng.choice(1 << 15, size=64, replace=False):
        s = int(6 * gi + rng.integers(0, 6))
        for mode, pb in itertools.product((0, 1, 2), (0.0, 1e-9)):
            d = grx.bfs(du, s, opts=grx.opts(direction=mode, push_bitmap=pb)).cpu().numpy()
            assert np.array_equal(d, oracle.bfs(u.row_offsets, u.col_indices, s))
        for delta in (0, 2):
            dist = grx.as_uint32(grx.sssp(du, s, opts=grx.opts(sssp_delta=delta)))
            assert np.array_equal(dist, oracle.sssp(u.row_offsets, u.col_indices, u.weights, s))


def test_graph_without_edges_and_isolated_source(grx):
    g = inputs.csr_from_edges(100, [])
    g.weights = np.zeros(0, dtype=np.uint32)
    dg = grx.load(g)
    d = grx.bfs(dg, 7).cpu().numpy()
    assert d[7] == 0 and np.all(np.delete(d, 7) == -1)
    dist = grx.as_uint32(grx.sssp(dg, 7))
    assert dist[7] == 0 and np.all(np.delete(dist, 7) == 0xFFFFFFFF)
    assert np.array_equal(grx.cc(dg).cpu().numpy(), np.arange(100))
    r = grx.pagerank(dg, 0.85, 20).cpu().numpy()
    assert np.allclose(r, 0.01, rtol=1e-6)
    # isolated source in a graph with edges
    g2 = GRAPHS["disconnected"]
    d2 = grx.bfs(grx.load(g2), 0).cpu().numpy()
    assert d2[0] == 0 and np.all(d2[1:] == -1)


def test_invalid_arguments_raise(grx, loaded):
    dg = loaded["rmat10"]
    with pytest.raises(grx.GrxError):
        grx.bfs(dg, -1)
    with pytest.raises(grx.GrxError):
        grx.bfs(dg, dg.nv)
    with pytest.raises(grx.GrxError):
        grx.sssp(grx.load(inputs.csr_from_edges(4, [(0, 1)])), 0)     # no weights
    bad = inputs.csr_from_edges(4, [(0, 1), (1, 2)])
    col = bad.col_indices.copy()
    col[0] = 3                                                          # breaks symmetry
    with pytest.raises(grx.GrxError):
        grx.graph_load_csr(bad.row_offsets, col, validate=True)


def test_device_generators_match_host(grx):
    for scale, ef, seed in ((10, 16, 1), (14, 16, 14), (12, 3, 99)):
        u, v = inputs.rmat_edges(scale, ef, seed)
        du, dv = grx.rmat_edges(scale, ef, seed)
        assert np.array_equal(du.cpu().numpy(), u) and np.array_equal(dv.cpu().numpy(), v)
    g = inputs.rmat_graph(12, 16, seed=12, wmax=64, weight_seed=77)
    ro, col, w = grx.rmat_graph_device(12, 16, seed=12, wmax=64, weight_seed=77)
    assert np.array_equal(ro.cpu().numpy(), g.row_offsets)
    assert np.array_equal(col.cpu().numpy(), g.col_indices)
    assert np.array_equal(grx.as_uint32(w), g.weights)
    for wd, ht in ((64, 48), (1, 5), (7, 1), (300, 211)):
        gg = inputs.grid_graph(wd, ht, p_del=0.1, seed=wd, wmax=1000, weight_seed=9)
        ro, col, w = grx.grid_graph_device(wd, ht, p_del=0.1, seed=wd, wmax=1000, weight_seed=9)
        assert np.array_equal(ro.cpu().numpy(), gg.row_offsets)
        assert np.array_equal(col.cpu().numpy(), gg.col_indices)
        assert np.array_equal(grx.as_uint32(w), gg.weights)


def test_load_from_device_arrays_int64_offsets(grx):
    g = GRAPHS["rmat13"]
    ro = torch.from_numpy(g.row_offsets).cuda()
    col = torch.from_numpy(g.col_indices).cuda()
    w = torch.from_numpy(g.weights.view(np.int32)).cuda()
    dg = grx.graph_load_csr(ro, col, w, validate=True)
    s = _sources(g, 1, seed=9)[0]
    assert np.array_equal(grx.bfs(dg, s).cpu().numpy(), oracle.bfs(g.row_offsets, g.col_indices, s))
    dg32 = grx.graph_load_csr(g.row_offsets.astype(np.int32), g.col_indices, g.weights)
    assert np.array_equal(grx.as_uint32(grx.sssp(dg32, s)),
                          oracle.sssp(g.row_offsets, g.col_indices, g.weights, s))


def test_timeout_status_is_reported_and_context_survives(grx, loaded):
    """A bounded wait that runs out sets GRX_ETIMEOUT on the host side and
    leaves the context usable (no fault, no hang: the wait limit is tiny)."""
    g, dg = GRAPHS["path"], loaded["path"]
    o = grx.opts(timeout_s=1e-9, direction=grx.GRX_DIR_PUSH)
    grx.bfs(dg, 0, opts=o)
    try:
        grx.graph_status(dg)
    except grx.GrxError as e:
        assert e.status == grx.GRX_ETIMEOUT
    d = grx.bfs(dg, 0)
    grx.graph_status(dg)
    assert np.array_equal(d.cpu().numpy(), oracle.bfs(g.row_offsets, g.col_indices, 0))


@pytest.mark.parametrize("name", ["rmat10", "rmat13", "rmat14_ef4", "grid64", "path", "star", "disconnected"])
@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("pb", ["pbdefault", "pbalways", "pbnever"])
def test_bfs_multi_lanes_match_oracle(grx, loaded, name, mode, pb):
    g, dg = GRAPHS[name], loaded[name]
    srcs = _sources(g, 61, seed=7) if name != "disconnected" else [1, 5, 10, 30, 0, 2]
    srcs = (srcs + [srcs[0], g.nv - 1, srcs[-1]])[:64]          # duplicates and an isolated/last vertex
    o = grx.opts(direction=MODES[mode], push_bitmap=PUSH_BITMAP[pb])
    d = grx.bfs_multi(dg, srcs, opts=o).cpu().numpy()
    grx.graph_status(dg)
    for b, s in enumerate(srcs):
        assert np.array_equal(d[b], oracle.bfs(g.row_offsets, g.col_indices, s)), (name, mode, pb, b, s)


def test_bfs_multi_after_an_interrupted_traversal(grx, loaded):
    """A multi-source traversal cut short by its wait limit leaves scratch
    state behind; the next one must clear it and still be exact."""
    for name, mode in (("path", 2), ("rmat13", 0), ("grid64", 1)):
        g, dg = GRAPHS[name], loaded[name]
        srcs = _sources(g, 40, seed=11)
        grx.bfs_multi(dg, srcs, opts=grx.opts(timeout_s=1e-9, direction=mode))
        try:
            grx.graph_status(dg)
        except grx.GrxError as e:
            assert e.status == grx.GRX_ETIMEOUT
        d = grx.bfs_multi(dg, srcs, opts=grx.opts(direction=mode)).cpu().numpy()
        grx.graph_status(dg)
        for b, s in enumerate(srcs):
            assert np.array_equal(d[b], oracle.bfs(g.row_offsets, g.col_indices, s)), (name, b, s)


def test_bfs_multi_few_lanes_and_stats(grx, loaded):
    g, dg = GRAPHS["rmat13"], loaded["rmat13"]
    for n in (1, 2, 31, 33):
        srcs = _sources(g, n, seed=n)
        d = grx.bfs_multi(dg, srcs, opts=grx.opts(collect_stats=1)).cpu().numpy()
        st = grx.last_stats(dg)
        want = [oracle.bfs(g.row_offsets, g.col_indices, s) for s in srcs]
        for b in range(n):
            assert np.array_equal(d[b], want[b])
        # discovered (vertex, lane) pairs per level equal the oracle's level sizes summed over lanes
        total = sum(int((w >= 0).sum()) for w in want)
        assert sum(st["discovered"]) + n == total


@pytest.mark.parametrize("name", ["rmat10", "rmat13", "rmat14_ef4", "grid64", "path", "star", "disconnected"])
@pytest.mark.parametrize("pb", list(PUSH_BITMAP))
@pytest.mark.parametrize("nl", [5, 8, 13, 16, 42])      # lane groups of 8, of 16, one lane per thread
def test_sssp_multi_lanes_match_oracle(grx, loaded, name, pb, nl):
    g, dg = GRAPHS[name], loaded[name]
    srcs = _sources(g, 40, seed=3) if name != "disconnected" else [1, 5, 10, 30, 0]
    srcs = (srcs + [srcs[0], g.nv - 1] + srcs)[:nl]
    d = grx.sssp_multi(dg, srcs, opts=grx.opts(push_bitmap=PUSH_BITMAP[pb])).cpu().numpy().view(np.uint32)
    grx.graph_status(dg)
    for b, s in enumerate(srcs):
        want = oracle.sssp(g.row_offsets, g.col_indices, g.weights, s)
        assert np.array_equal(d[b], want), (name, pb, b, s)


def test_multi_source_on_the_6_vertex_union(grx):
    pairs = list(itertools.combinations(range(6), 2))
    edges = []
    for gi in range(1 << 15):
        base = 6 * gi
        edges += [(base + a, base + b) for i, (a, b) in enumerate(pairs) if gi >> i & 1]
    u = inputs.csr_from_edges(6 << 15, edges)
    rows = np.repeat(np.arange(u.nv), np.diff(u.row_offsets))
    lo = np.minimum(rows, u.col_indices).astype(np.uint64)
    hi = np.maximum(rows, u.col_indices).astype(np.uint64)
    u.weights = (1 + inputs.draw(67, lo * np.uint64(u.nv) + hi) % np.uint64(3)).astype(np.uint32)
    du = grx.load(u)
    rng = np.random.default_rng(9)
    for rep in range(3):
        srcs = [int(6 * gi + rng.integers(0, 6)) for gi in rng.choice(1 << 15, size=64, replace=False)]
        d = grx.bfs_multi(du, srcs).cpu().numpy()
        dist = grx.sssp_multi(du, srcs).cpu().numpy().view(np.uint32)
        for b, s in enumerate(srcs):
            assert np.array_equal(d[b], oracle.bfs(u.row_offsets, u.col_indices, s))
            assert np.array_equal(dist[b], oracle.sssp(u.row_offsets, u.col_indices, u.weights, s))


@pytest.mark.parametrize("name", ["rmat13", "grid64", "path", "disconnected"])
def test_int64_offsets_every_primitive(grx, name):
    """The 64-bit-offset instantiation of every kernel (used when ne >= 2^31,
    forced here on small graphs)."""
    g = GRAPHS[name]
    dg = grx.load(g, validate=True, offsets64=True)
    srcs = _sources(g, 3, seed=8) + [g.nv - 1]
    for s in srcs:
        want = oracle.bfs(g.row_offsets, g.col_indices, s)
        for mode in (0, 1, 2):
            for loop in (grx.GRX_LOOP_PERSISTENT, grx.GRX_LOOP_HOST, grx.GRX_LOOP_GRAPH):
                d = grx.bfs(dg, s, opts=grx.opts(direction=mode, loop=loop))
                assert np.array_equal(d.cpu().numpy(), want), (name, s, mode, loop)
        assert np.array_equal(grx.as_uint32(grx.sssp(dg, s)),
                              oracle.sssp(g.row_offsets, g.col_indices, g.weights, s))
    assert np.array_equal(grx.cc(dg).cpu().numpy(), oracle.cc(g.row_offsets, g.col_indices))
    r = grx.pagerank(dg, 0.85, 20).cpu().numpy().astype(np.float64)
    want = oracle.pagerank(g.row_offsets, g.col_indices, 0.85, 20)
    assert np.max(np.abs(r - want) / want) <= PR_TOL
    dm = grx.bfs_multi(dg, srcs).cpu().numpy()
    dd = grx.sssp_multi(dg, srcs).cpu().numpy().view(np.uint32)
    for b, s in enumerate(srcs):
        assert np.array_equal(dm[b], oracle.bfs(g.row_offsets, g.col_indices, s))
        assert np.array_equal(dd[b], oracle.sssp(g.row_offsets, g.col_indices, g.weights, s))
    for kind in (grx.GRX_KIND_BFS, grx.GRX_KIND_SSSP):
        b = grx.Batch(dg, kind)
        outs = {}
        for s in srcs:
            out = torch.empty(g.nv, dtype=torch.int32, device="cuda")
            outs[b.admit(s, out)] = (s, out)
            b.step(3)
        done = b.poll()
        for _ in range(20000):
            if done == sum(1 << l for l in outs):
                break
            b.step(8)
            done |= b.poll()
        for lane, (s, out) in outs.items():
            got = out.cpu().numpy()
            if kind == grx.GRX_KIND_BFS:
                assert np.array_equal(got, oracle.bfs(g.row_offsets, g.col_indices, s))
            else:
                assert np.array_equal(got.view(np.uint32),
                                      oracle.sssp(g.row_offsets, g.col_indices, g.weights, s))
        b.close()
    grx.graph_status(dg)


# ---- betweenness centrality: float64 sums of nonnegative terms, so the
# relative error of each value is bounded by (levels + log2 terms) * 2^-53
# times a small constant -- far below BC_TOL on these graphs (at most 3,000
# levels); path counts are integers, exact below 2^53.
BC_TOL = 1e-9


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("pb", list(PUSH_BITMAP))
@pytest.mark.parametrize("mode", list(MODES))
def test_bc_single_sources_match_oracle(grx, loaded, name, pb, mode):
    """mode: auto = direction per level by edge counts; push = forward push
    and backward pull only; pull = forward pull (after the source level) and
    backward push only."""
    g, dg = GRAPHS[name], loaded[name]
    o = grx.opts(push_bitmap=PUSH_BITMAP[pb], direction=MODES[mode])
    for s in _sources(g, 3, seed=4) + [0, g.nv - 1]:
        got, sig = grx.bc(dg, [s], want_sigma=True, opts=o)
        want, wsig = oracle.bc(g.row_offsets, g.col_indices, [s], want_sigma=True)
        np.testing.assert_allclose(got.cpu().numpy(), want, rtol=BC_TOL, atol=0, err_msg=f"{name} {s}")
        np.testing.assert_allclose(sig.cpu().numpy(), wsig, rtol=1e-12, atol=0, err_msg=f"{name} {s}")


@pytest.mark.parametrize("name", list(GRAPHS))
def test_bc_sums_over_sources_match_oracle(grx, loaded, name):
    g, dg = GRAPHS[name], loaded[name]
    srcs = _sources(g, 6, seed=5)
    srcs += srcs[:2]                                     # duplicates count twice
    want = oracle.bc(g.row_offsets, g.col_indices, srcs)
    for mode in MODES.values():
        got = grx.bc(dg, srcs, opts=grx.opts(direction=mode)).cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=BC_TOL, atol=0, err_msg=str(mode))


def test_bc_every_source_of_every_5_vertex_graph(grx):
    """All 1,024 labelled graphs on 5 vertices as one disjoint union, every
    vertex a source; a seeded sample of 6-vertex graphs likewise."""
    for n, count in ((5, None), (6, 400)):
        pairs = list(itertools.combinations(range(n), 2))
        masks = range(1 << len(pairs)) if count is None else \
            np.random.default_rng(n).choice(1 << len(pairs), size=count, replace=False)
        edges = []
        for gi, mask in enumerate(masks):
            edges += [(gi * n + a, gi * n + b) for pi, (a, b) in enumerate(pairs) if int(mask) >> pi & 1]
        u = inputs.csr_from_edges(n * len(masks), edges)
        du = grx.load(u, validate=True)
        srcs = np.arange(u.nv)
        want = oracle.bc(u.row_offsets, u.col_indices, srcs)
        for mode in MODES.values():
            np.testing.assert_allclose(grx.bc(du, srcs, opts=grx.opts(direction=mode)).cpu().numpy(),
                                       want, rtol=BC_TOL, atol=0, err_msg=str(mode))


def test_bc_int64_offsets_and_edge_cases(grx):
    g = GRAPHS["grid64"]
    dg = grx.load(g, validate=True, offsets64=True)
    srcs = _sources(g, 3, seed=6)
    got, sig = grx.bc(dg, srcs, want_sigma=True)
    want, wsig = oracle.bc(g.row_offsets, g.col_indices, srcs, want_sigma=True)
    np.testing.assert_allclose(got.cpu().numpy(), want, rtol=BC_TOL, atol=0)
    np.testing.assert_allclose(sig.cpu().numpy(), wsig, rtol=1e-12, atol=0)
    # isolated source, graph without edges, bad arguments
    dd = grx.load(GRAPHS["disconnected"])
    b, s = grx.bc(dd, [0], want_sigma=True)
    assert np.all(b.cpu().numpy() == 0) and s.cpu().numpy()[0] == 1 and np.all(s.cpu().numpy()[1:] == 0)
    de = grx.load(inputs.csr_from_edges(50, []))
    assert np.all(grx.bc(de, [3, 4]).cpu().numpy() == 0)
    with pytest.raises(RuntimeError):
        grx.bc(dd, [40])
    with pytest.raises(RuntimeError):
        grx.bc(dd, [])


# ---- batched BC: up to 64 sources in one sweep, same sums as bc()

@pytest.mark.parametrize("name", ["rmat10", "rmat13", "rmat14_ef4", "star", "disconnected"])
def test_bc_multi_matches_oracle(grx, loaded, name):
    g, dg = GRAPHS[name], loaded[name]
    for n in (1, 7, 64):
        srcs = _sources(g, n, seed=9)
        srcs += srcs[:2] if len(srcs) < 64 else []       # duplicates allowed
        srcs = srcs[:64]
        got = grx.bc_multi(dg, srcs).cpu().numpy()
        grx.graph_status(dg)
        np.testing.assert_allclose(got, oracle.bc(g.row_offsets, g.col_indices, srcs), rtol=BC_TOL, atol=0,
                                   err_msg=f"{name} n={len(srcs)}")


def test_bc_multi_every_source_of_every_5_vertex_graph(grx):
    n = 5
    pairs = list(itertools.combinations(range(n), 2))
    edges = []
    for gi in range(1 << len(pairs)):
        edges += [(gi * n + a, gi * n + b) for pi, (a, b) in enumerate(pairs) if gi >> pi & 1]
    u = inputs.csr_from_edges(n * (1 << len(pairs)), edges)
    du = grx.load(u, validate=True, offsets64=True)
    total = np.zeros(u.nv)
    out = torch.empty(u.nv, dtype=torch.float64, device="cuda")
    for b in range(0, u.nv, 64):
        total += grx.bc_multi(du, np.arange(b, min(u.nv, b + 64)), bc_out=out).cpu().numpy()
    grx.graph_status(du)
    np.testing.assert_allclose(total, oracle.bc(u.row_offsets, u.col_indices, np.arange(u.nv)),
                               rtol=BC_TOL, atol=0)


def test_bc_multi_too_deep_reports_range_and_recovers(grx, loaded):
    dg = loaded["path"]                                  # 3,000 levels
    grx.bc_multi(dg, [0, 5])
    with pytest.raises(RuntimeError):
        grx.graph_status(dg)
    g = GRAPHS["rmat10"]
    srcs = _sources(g, 4, seed=3)
    np.testing.assert_allclose(grx.bc_multi(loaded["rmat10"], srcs).cpu().numpy(),
                               oracle.bc(g.row_offsets, g.col_indices, srcs), rtol=BC_TOL, atol=0)
    with pytest.raises(RuntimeError):
        grx.bc_multi(dg, list(range(65)))


def test_bc_multi_isolated_source_lane_and_sssp_zero_weights(grx, loaded):
    g, dg = GRAPHS["disconnected"], loaded["disconnected"]
    srcs = [0, 1, 5, 0, 12]                              # vertex 0 is isolated
    np.testing.assert_allclose(grx.bc_multi(dg, srcs).cpu().numpy(),
                               oracle.bc(g.row_offsets, g.col_indices, srcs), rtol=BC_TOL, atol=0)
    de = grx.load(inputs.csr_from_edges(40, []))         # no edges at all
    assert np.all(grx.bc_multi(de, [0, 3, 39]).cpu().numpy() == 0)
    grx.graph_status(de)
    # near-far bands with zero-weight edges
    h = inputs.rmat_graph(11, 8, seed=21)
    rows = np.repeat(np.arange(h.nv), np.diff(h.row_offsets))
    lo = np.minimum(rows, h.col_indices).astype(np.uint64)
    hi = np.maximum(rows, h.col_indices).astype(np.uint64)
    h.weights = (inputs.draw(31, lo * np.uint64(h.nv) + hi) % np.uint64(4)).astype(np.uint32)
    dh = grx.load(h, validate=True)
    for s in _sources(h, 3, seed=4):
        want = oracle.sssp(h.row_offsets, h.col_indices, h.weights, s)
        for delta in (0, 1, 2):
            assert np.array_equal(grx.as_uint32(grx.sssp(dh, s, opts=grx.opts(sssp_delta=delta))), want), delta


# ---- 64-bit vertex ids (graph_load_csr64 + bfs64)

@pytest.fixture(scope="module")
def loaded64(grx):
    return {name: grx.graph_load_csr64(g.row_offsets.astype(np.int64), g.col_indices.astype(np.int64),
                                       validate=True) for name, g in GRAPHS.items()}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("mode", list(MODES))
def test_bfs64_matches_oracle(grx, loaded64, name, mode):
    """Every id, offset and count 64-bit (forced on small graphs): depths
    bit-exact, int64 parents accepted by the oracle's checker; the star's hub
    row (5,000 edges) goes through the long-row phase."""
    g, dg = GRAPHS[name], loaded64[name]
    srcs = _sources(g, 4, seed=2) + ([0] if name == "star" else [])
    for s in srcs:
        d, p = grx.bfs64(dg, s, parent=True, opts=grx.opts(direction=MODES[mode]))
        want = oracle.bfs(g.row_offsets, g.col_indices, s)
        got = d.cpu().numpy()
        assert np.array_equal(got, want), (name, mode, s)
        ph = p.cpu().numpy()
        assert ph.max() < g.nv
        assert oracle.check_bfs(g.row_offsets, g.col_indices, s, got, ph.astype(np.int32)) == 0
    grx.graph_status(dg)


def test_bfs64_switch_parameters_and_union(grx):
    pairs = list(itertools.combinations(range(6), 2))
    edges = []
    for mask in range(1 << len(pairs)):
        base = 6 * mask
        edges += [(base + a, base + b) for i, (a, b) in enumerate(pairs) if mask >> i & 1]
    u = inputs.csr_from_edges(6 << len(pairs), edges)
    du = grx.graph_load_csr64(u.row_offsets, u.col_indices.astype(np.int64))
    for s in (6 * 32767, 6 * 12345 + 3, 6 * 5 + 1):
        want = oracle.bfs(u.row_offsets, u.col_indices, s)
        for kw in ({}, {"alpha": 1e-6, "beta": 1.0, "exact_fv": 1}, {"alpha": 1e3}, {"direction": 2}):
            assert np.array_equal(grx.bfs64(du, s, opts=grx.opts(**kw)).cpu().numpy(), want), (s, kw)


def test_64bit_graphs_are_refused_by_the_other_primitives(grx, loaded64):
    dg = loaded64["rmat10"]
    for fn in (lambda: grx.bfs(dg, 1), lambda: grx.cc(dg), lambda: grx.pagerank(dg, 0.85, 5),
               lambda: grx.bfs_multi(dg, [1, 2]), lambda: grx.multi_footprint(dg, 0)):
        with pytest.raises(grx.GrxError) as e:
            fn()
        assert e.value.status == grx.GRX_EINVAL
    # and a 32-bit graph is refused by bfs64
    with pytest.raises(grx.GrxError):
        grx.bfs64(grx.load(GRAPHS["rmat10"]), 1)
