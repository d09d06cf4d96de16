"""Pins for the CPU oracle: each check rests on something other than the
oracle itself -- brute force on every 6-vertex graph, closed forms, a dense
matrix formulation of PageRank, and printed fixtures under tests/golden/."""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1504_04804_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
N6 = 6
PAIRS6 = list(itertools.combinations(range(N6), 2))      # 15 possible edges


def _all_graphs6():
    """Every labelled simple graph on 6 vertices as a 15-bit edge mask."""
    return range(1 << len(PAIRS6))


def _adj6(mask):
    return [PAIRS6[i] for i in range(len(PAIRS6)) if mask >> i & 1]


def _floyd_warshall_all(masks, weight_of):
    """Brute-force all-pairs distances for a batch of 6-vertex graphs.
    weight_of(mask_index, pair_index) -> weight.  inf where unreachable."""
    m = len(masks)
    d = np.full((m, N6, N6), np.inf)
    d[:, np.arange(N6), np.arange(N6)] = 0
    for gi, mask in enumerate(masks):
        for pi, (a, b) in enumerate(PAIRS6):
            if mask >> pi & 1:
                w = weight_of(gi, pi)
                d[gi, a, b] = d[gi, b, a] = w
    for k in range(N6):
        d = np.minimum(d, d[:, :, k:k + 1] + d[:, k:k + 1, :])
    return d


def test_splitmix64_published_vectors():
    """Counter-based SplitMix64 reproduces the published seed-0 sequence."""
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        want = [int(line.split()[0], 16) for line in f
                if line.strip() and not line.startswith("#")]
    got = inputs.draw(0, np.arange(len(want)))
    assert [int(x) for x in got] == want


def test_bfs_exhaustive_6_vertices():
    masks = list(_all_graphs6())
    fw = _floyd_warshall_all(masks, lambda g, p: 1.0)
    for gi, mask in enumerate(masks):
        g = inputs.csr_from_edges(N6, _adj6(mask))
        for s in range(N6):
            depth = oracle.bfs(g.row_offsets, g.col_indices, s)
            want = np.where(np.isinf(fw[gi, s]), -1, fw[gi, s]).astype(np.int32)
            assert np.array_equal(depth, want), (mask, s)


def test_sssp_exhaustive_6_vertices():
    masks = list(_all_graphs6())
    rng = np.random.default_rng(6)
    wtab = rng.integers(1, 4, size=(len(masks), len(PAIRS6)))   # weights in {1,2,3}
    # a few zero weights too: Dijkstra must still be exact
    wtab[::7, 3] = 0
    fw = _floyd_warshall_all(masks, lambda g, p: float(wtab[g, p]))
    for gi, mask in enumerate(masks):
        edges = _adj6(mask)
        g = inputs.csr_from_edges(N6, edges)
        wmap = {}
        for pi, (a, b) in enumerate(PAIRS6):
            if mask >> pi & 1:
                wmap[(a, b)] = wmap[(b, a)] = int(wtab[gi, pi])
        rows = np.repeat(np.arange(N6), np.diff(g.row_offsets))
        w = np.array([wmap[(int(r), int(c))] for r, c in zip(rows, g.col_indices)],
                     dtype=np.uint32)
        for s in range(N6):
            dist = oracle.sssp(g.row_offsets, g.col_indices, w, s)
            want = np.where(np.isinf(fw[gi, s]), 0xFFFFFFFF, fw[gi, s]).astype(np.uint32)
            assert np.array_equal(dist, want), (mask, s)


def test_cc_exhaustive_6_vertices():
    masks = list(_all_graphs6())
    fw = _floyd_warshall_all(masks, lambda g, p: 1.0)
    reach = np.isfinite(fw)                       # transitive closure
    for gi, mask in enumerate(masks):
        g = inputs.csr_from_edges(N6, _adj6(mask))
        label = oracle.cc(g.row_offsets, g.col_indices)
        want = np.array([np.flatnonzero(reach[gi, v]).min() for v in range(N6)])
        assert np.array_equal(label, want), mask


def test_bfs_closed_forms():
    n = 50
    path = inputs.csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    cyc = inputs.csr_from_edges(n, [(i, (i + 1) % n) for i in range(n)])
    for s in (0, 17, n - 1):
        assert np.array_equal(oracle.bfs(path.row_offsets, path.col_indices, s),
                              np.abs(np.arange(n) - s))
        k = np.abs(np.arange(n) - s)
        assert np.array_equal(oracle.bfs(cyc.row_offsets, cyc.col_indices, s),
                              np.minimum(k, n - k))
    # full grid (no deletions): depth = Manhattan distance
    w, h = 23, 17
    u, v = inputs.grid_edges(w, h, 0.0, seed=1)
    assert len(u) == (w - 1) * h + w * (h - 1)
    ro, col = inputs.build_csr(w * h, u, v)
    s = 5 * w + 7
    xs, ys = np.arange(w * h) % w, np.arange(w * h) // w
    man = np.abs(xs - 7) + np.abs(ys - 5)
    assert np.array_equal(oracle.bfs(ro, col, s), man)
    ones = np.ones(col.shape[0], dtype=np.uint32)
    assert np.array_equal(oracle.sssp(ro, col, ones, s), man.astype(np.uint32))
    assert np.all(oracle.cc(ro, col) == 0)


def test_sssp_path_prefix_sums_and_unreached():
    n = 40
    rng = np.random.default_rng(3)
    wts = rng.integers(0, 1000, size=n - 1)
    g = inputs.csr_from_edges(n + 2, [(i, i + 1) for i in range(n - 1)] + [(n, n + 1)])
    rows = np.repeat(np.arange(n + 2), np.diff(g.row_offsets))
    w = np.array([wts[min(r, c)] if max(r, c) < n else 9 for r, c in zip(rows, g.col_indices)],
                 dtype=np.uint32)
    dist = oracle.sssp(g.row_offsets, g.col_indices, w, 0)
    assert np.array_equal(dist[:n], np.concatenate([[0], np.cumsum(wts)]).astype(np.uint32))
    assert dist[n] == 0xFFFFFFFF and dist[n + 1] == 0xFFFFFFFF
    depth = oracle.bfs(g.row_offsets, g.col_indices, n)
    assert depth[n + 1] == 1 and np.all(depth[:n] == -1)


def test_sssp_overflow_is_reported():
    g = inputs.csr_from_edges(3, [(0, 1), (1, 2)])
    w = np.full(4, 0x90000000, dtype=np.uint32)
    with pytest.raises(oracle.OracleError):
        oracle.sssp(g.row_offsets, g.col_indices, w, 0)


def test_cc_components_and_isolated():
    # two triangles, an edge, and isolated vertices, ids shuffled
    edges = [(9, 4), (4, 7), (7, 9), (2, 8), (8, 6), (6, 2), (5, 3)]
    g = inputs.csr_from_edges(11, edges)
    lab = oracle.cc(g.row_offsets, g.col_indices)
    assert list(lab) == [0, 1, 2, 3, 4, 3, 2, 4, 2, 4, 10]
    # random graphs: the number of labels equals the number of BFS sweeps
    rng = np.random.default_rng(11)
    for _ in range(20):
        n = int(rng.integers(20, 200))
        m = int(rng.integers(0, n))
        e = rng.integers(0, n, size=(m, 2))
        g = inputs.csr_from_edges(n, [tuple(x) for x in e])
        lab = oracle.cc(g.row_offsets, g.col_indices)
        seen = np.full(n, -1)
        sweeps = 0
        for v in range(n):
            if seen[v] < 0:
                d = oracle.bfs(g.row_offsets, g.col_indices, v)
                assert np.all(seen[d >= 0] < 0)
                seen[d >= 0] = sweeps
                assert np.all(lab[d >= 0] == v)    # v is the min id of its component
                sweeps += 1
        assert len(np.unique(lab)) == sweeps


def _dense_pagerank(ro, col, d, iters):
    """Independent formulation: r <- (1-d)/N 1 + d (A D^-1 + 1 z^T / N) r, where
    z marks zero-degree columns (dangling vertices spread their rank evenly)."""
    n = ro.shape[0] - 1
    deg = np.diff(ro).astype(np.float64)
    M = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(ro))
    M[col, rows] = 1.0 / deg[rows]
    M[:, deg == 0] = 1.0 / n
    r = np.full(n, 1.0 / n)
    for _ in range(iters):
        r = (1 - d) / n + d * (M @ r)
    return r


def test_pagerank_dense_matrix():
    rng = np.random.default_rng(21)
    for _ in range(25):
        n = int(rng.integers(2, 60))
        m = int(rng.integers(0, 3 * n))
        e = rng.integers(0, n, size=(m, 2))
        g = inputs.csr_from_edges(n, [tuple(x) for x in e])
        for iters in (0, 1, 2, 20):
            got = oracle.pagerank(g.row_offsets, g.col_indices, 0.85, iters)
            want = _dense_pagerank(g.row_offsets, g.col_indices, 0.85, iters)
            assert np.max(np.abs(got - want) / want) < 1e-13
            assert abs(got.sum() - 1) < 1e-12
            assert np.all(got >= 0.15 / n * (1 - 1e-12))


def test_pagerank_regular_graph_is_uniform():
    for g in (inputs.csr_from_edges(31, [(i, (i + 1) % 31) for i in range(31)]),
              inputs.csr_from_edges(8, list(itertools.combinations(range(8), 2)))):
        r = oracle.pagerank(g.row_offsets, g.col_indices, 0.85, 20)
        assert np.max(np.abs(r * g.nv - 1)) < 1e-13


def test_pagerank_dangling_closed_form():
    """One edge {0,1} plus an isolated vertex 2.  By symmetry r0 = r1 = (1-b)/2
    and the isolated rank obeys b_k = (1-d)/3 + (d/3) b_{k-1}, b_0 = 1/3, so
    b_k = b* + (d/3)^k (1/3 - b*) with b* = ((1-d)/3) / (1 - d/3)."""
    d = 0.85
    g = inputs.csr_from_edges(3, [(0, 1)])
    bstar = ((1 - d) / 3) / (1 - d / 3)
    for k in (1, 5, 20):
        r = oracle.pagerank(g.row_offsets, g.col_indices, d, k)
        b = bstar + (d / 3) ** k * (1 / 3 - bstar)
        assert abs(r[2] - b) < 1e-15
        assert abs(r[0] - (1 - b) / 2) < 1e-15 and r[0] == r[1]


def test_pagerank_star_closed_form():
    """A star: hub 0 with n leaves (degree 1 each), no dangling vertex.  By
    symmetry every leaf holds the same rank l, and with N = n + 1 the update is
    h' = (1-d)/N + d*n*l,  l' = (1-d)/N + d*h/n  from h = l = 1/N: a
    two-variable recurrence evaluated here in exact rational arithmetic.  The
    oracle sums the hub's n terms in FP64: relative error within a few
    (n + iterations) units of 2^-53."""
    from fractions import Fraction
    d = Fraction(85, 100)
    for n in (1, 7, 5000):
        g = inputs.csr_from_edges(n + 1, [(0, i) for i in range(1, n + 1)])
        N = n + 1
        h = l = Fraction(1, N)
        tol = 4 * (n + 20) * 2.0 ** -53
        for k in range(1, 21):
            h, l = (1 - d) / N + d * n * l, (1 - d) / N + d * h / n
            if k in (1, 2, 20):
                r = oracle.pagerank(g.row_offsets, g.col_indices, 0.85, k)
                assert abs(r[0] - float(h)) <= tol * float(h), (n, k)
                assert np.max(np.abs(r[1:] - float(l))) <= tol * float(l), (n, k)


def _ragged_graph(nh):
    """600 hubs in a chain, hub h owning h + 1 private leaves."""
    edges, leaf = [], nh
    for h in range(nh):
        if h + 1 < nh:
            edges.append((h, h + 1))
        for _ in range(h + 1):
            edges.append((h, leaf))
            leaf += 1
    return inputs.csr_from_edges(leaf, edges)


def test_bfs_sssp_cc_ragged_closed_forms():
    """The chained-hub graph of the GPU parity set (rows of every length from 1
    to nh + 1): from hub s, hub h sits at |h - s| and its leaves one further;
    from a leaf of hub h everything is one further than from h; unit weights
    give the same distances; one component, labelled 0."""
    nh = 60
    g = _ragged_graph(nh)
    owner = np.concatenate([np.arange(nh)] + [np.full(h + 1, h) for h in range(nh)])
    is_leaf = np.arange(g.nv) >= nh
    ones = np.ones(g.col_indices.shape[0], dtype=np.uint32)
    for s in (0, 17, nh - 1):
        want = np.abs(owner - s) + is_leaf
        assert np.array_equal(oracle.bfs(g.row_offsets, g.col_indices, s), want)
        assert np.array_equal(oracle.sssp(g.row_offsets, g.col_indices, ones, s), want.astype(np.uint32))
    leaf_of_5 = nh + 5 * 6 // 2                 # first leaf of hub 5
    want = np.abs(owner - 5) + is_leaf + 1
    want[leaf_of_5] = 0
    assert np.array_equal(oracle.bfs(g.row_offsets, g.col_indices, leaf_of_5), want)
    assert np.all(oracle.cc(g.row_offsets, g.col_indices) == 0)


def test_golden_fixtures():
    """Hand-derived values for small named graphs (see each fixture's header)."""
    for name in sorted(os.listdir(GOLDEN)):
        if not name.startswith("graph_"):
            continue
        fx = _read_fixture(os.path.join(GOLDEN, name))
        g = inputs.csr_from_edges(fx["n"], fx["edges"])
        if "bfs" in fx:
            for s, want in fx["bfs"].items():
                assert list(oracle.bfs(g.row_offsets, g.col_indices, s)) == want, (name, s)
        if "cc" in fx:
            assert list(oracle.cc(g.row_offsets, g.col_indices)) == fx["cc"], name
        if "sssp" in fx:
            wmap = {}
            for (a, b), w in zip(fx["edges"], fx["weights"]):
                wmap[(a, b)] = wmap[(b, a)] = w
            rows = np.repeat(np.arange(fx["n"]), np.diff(g.row_offsets))
            w = np.array([wmap[(int(r), int(c))] for r, c in zip(rows, g.col_indices)],
                         dtype=np.uint32)
            for s, want in fx["sssp"].items():
                assert list(oracle.sssp(g.row_offsets, g.col_indices, w, s)) == want


def _read_fixture(path):
    fx = {"bfs": {}, "sssp": {}}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, _, val = line.partition(":")
            key = key.strip()
            nums = [int(x) for x in val.split()]
            if key == "n":
                fx["n"] = nums[0]
            elif key == "edges":
                fx["edges"] = list(zip(nums[0::2], nums[1::2]))
            elif key == "weights":
                fx["weights"] = nums
            elif key.startswith("bfs"):
                fx["bfs"][int(key[3:])] = nums
            elif key.startswith("sssp"):
                fx["sssp"][int(key[4:])] = nums
            elif key == "cc":
                fx["cc"] = nums
    if not fx["bfs"]:
        del fx["bfs"]
    if not fx["sssp"]:
        del fx["sssp"]
    return fx


# ---- invariant checkers: they accept the oracle's answers and reject planted mistakes

def _rmat_small():
    return inputs.rmat_graph(10, 16, seed=3, wmax=64, weight_seed=7)


def test_checkers_accept_oracle_results():
    g = _rmat_small()
    src = int(inputs.pick_sources(g.row_offsets, 1, seed=1)[0])
    depth = oracle.bfs(g.row_offsets, g.col_indices, src)
    assert oracle.check_bfs(g.row_offsets, g.col_indices, src, depth) == 0
    dist = oracle.sssp(g.row_offsets, g.col_indices, g.weights, src)
    assert oracle.check_sssp(g.row_offsets, g.col_indices, g.weights, src, dist) == 0
    lab = oracle.cc(g.row_offsets, g.col_indices)
    assert oracle.check_cc(g.row_offsets, g.col_indices, lab) == 0
    # a parent array built from the depths is accepted
    par = np.full(g.nv, -1, dtype=np.int32)
    par[src] = src
    rows = np.repeat(np.arange(g.nv), np.diff(g.row_offsets))
    for r, c in zip(rows, g.col_indices):
        if depth[r] > 0 and depth[c] == depth[r] - 1:
            par[r] = c
    assert oracle.check_bfs(g.row_offsets, g.col_indices, src, depth, par) == 0


def test_checkers_reject_planted_mistakes():
    g = _rmat_small()
    src = int(inputs.pick_sources(g.row_offsets, 1, seed=1)[0])
    depth = oracle.bfs(g.row_offsets, g.col_indices, src)
    reached = np.flatnonzero(depth > 0)
    for v in reached[:: max(1, len(reached) // 15)]:
        for delta in (-1, 1):
            bad = depth.copy()
            bad[v] += delta
            assert oracle.check_bfs(g.row_offsets, g.col_indices, src, bad) > 0
    dist = oracle.sssp(g.row_offsets, g.col_indices, g.weights, src)
    for v in reached[:: max(1, len(reached) // 15)]:
        for delta in (-1, 1):
            bad = dist.copy()
            bad[v] = np.uint32(int(bad[v]) + delta)
            assert oracle.check_sssp(g.row_offsets, g.col_indices, g.weights, src, bad) > 0
    lab = oracle.cc(g.row_offsets, g.col_indices)
    v = int(np.flatnonzero(lab != np.arange(g.nv))[0])
    bad = lab.copy()
    bad[v] = v          # not the minimum of its component
    assert oracle.check_cc(g.row_offsets, g.col_indices, bad) > 0
    # the whole component relabelled to its second-smallest member
    comp = np.flatnonzero(lab == lab[v])
    bad = lab.copy()
    bad[comp] = comp[1]
    assert oracle.check_cc(g.row_offsets, g.col_indices, bad) > 0


def test_checkers_reject_a_second_root_and_merged_components():
    """Mistakes a purely local check misses: a second depth-0 vertex (it
    needs no predecessor), a zero-weight island away from the source carrying
    distance 0 (every edge in it is tight), and two components merged under
    one label (labels agree across every edge)."""
    star = inputs.csr_from_edges(5, [(0, 1), (0, 2), (0, 3), (0, 4)])
    d = oracle.bfs(star.row_offsets, star.col_indices, 0)
    assert oracle.check_bfs(star.row_offsets, star.col_indices, 0, d) == 0
    bad = d.copy()
    bad[3] = 0
    assert oracle.check_bfs(star.row_offsets, star.col_indices, 0, bad) > 0
    # an unreached pair labelled as if it held its own source
    two = inputs.csr_from_edges(4, [(0, 1), (2, 3)])
    d = oracle.bfs(two.row_offsets, two.col_indices, 0)
    bad = d.copy()
    bad[2], bad[3] = 0, 1
    assert oracle.check_bfs(two.row_offsets, two.col_indices, 0, bad) > 0
    w = np.array([5, 5, 0, 0], dtype=np.uint32)          # rows 0,1,2,3: edge 2-3 weighs 0
    dist = oracle.sssp(two.row_offsets, two.col_indices, w, 0)
    assert oracle.check_sssp(two.row_offsets, two.col_indices, w, 0, dist) == 0
    bad = dist.copy()
    bad[2] = bad[3] = 0
    assert oracle.check_sssp(two.row_offsets, two.col_indices, w, 0, bad) > 0
    lab = oracle.cc(two.row_offsets, two.col_indices)
    assert list(lab) == [0, 0, 2, 2]
    assert oracle.check_cc(two.row_offsets, two.col_indices, lab) == 0
    assert oracle.check_cc(two.row_offsets, two.col_indices, np.zeros(4, np.int32)) > 0
    # one component split in two
    path = inputs.csr_from_edges(4, [(0, 1), (1, 2), (2, 3)])
    assert oracle.check_cc(path.row_offsets, path.col_indices, np.array([0, 0, 2, 2], np.int32)) > 0


N4 = 4
PAIRS4 = list(itertools.combinations(range(N4), 2))


def _graphs4():
    for mask in range(1 << len(PAIRS4)):
        yield mask, [PAIRS4[i] for i in range(len(PAIRS4)) if mask >> i & 1]


def _fw4(edges, wmap=None):
    d = np.full((N4, N4), np.inf)
    np.fill_diagonal(d, 0)
    for a, b in edges:
        d[a, b] = d[b, a] = 1.0 if wmap is None else wmap[(a, b)]
    for k in range(N4):
        d = np.minimum(d, d[:, k:k + 1] + d[k:k + 1, :])
    return d


def test_checkers_accept_exactly_the_right_answer_on_every_4_vertex_graph():
    """Brute force: on every labelled 4-vertex graph, among all candidate
    answers (BFS depths in {-1..3}^4, CC labels in {0..3}^4, SSSP distances
    in {0..6, inf}^4 with weights in {0,1,2}), the checkers accept exactly one,
    the Floyd-Warshall / transitive-closure answer.  So the invariants are
    complete, not merely necessary."""
    depth_cands = [np.array(c, dtype=np.int32) for c in itertools.product(range(-1, 4), repeat=N4)]
    label_cands = [np.array(c, dtype=np.int32) for c in itertools.product(range(N4), repeat=N4)]
    inf = 0xFFFFFFFF
    dist_cands = [np.array(c, dtype=np.uint32)
                  for c in itertools.product([0, 1, 2, 3, 4, 5, 6, inf], repeat=N4)]
    rng = np.random.default_rng(44)
    for mask, edges in _graphs4():
        g = inputs.csr_from_edges(N4, edges)
        fw = _fw4(edges)
        src = mask % N4
        want = np.where(np.isinf(fw[src]), -1, fw[src]).astype(np.int32)
        ok = [c for c in depth_cands if oracle.check_bfs(g.row_offsets, g.col_indices, src, c) == 0]
        assert len(ok) == 1 and np.array_equal(ok[0], want), (mask, src)
        reach = np.isfinite(fw)
        want_l = np.array([np.flatnonzero(reach[v]).min() for v in range(N4)], dtype=np.int32)
        ok = [c for c in label_cands if oracle.check_cc(g.row_offsets, g.col_indices, c) == 0]
        assert len(ok) == 1 and np.array_equal(ok[0], want_l), mask
        wmap = {}
        for a, b in edges:
            wmap[(a, b)] = wmap[(b, a)] = int(rng.integers(0, 3))
        rows = np.repeat(np.arange(N4), np.diff(g.row_offsets))
        w = np.array([wmap[(int(r), int(c))] for r, c in zip(rows, g.col_indices)], dtype=np.uint32)
        fww = _fw4(edges, wmap)
        want_d = np.where(np.isinf(fww[src]), inf, fww[src]).astype(np.uint32)
        ok = [c for c in dist_cands
              if oracle.check_sssp(g.row_offsets, g.col_indices, w, src, c) == 0]
        assert len(ok) == 1 and np.array_equal(ok[0], want_d), (mask, src, wmap)


def test_rmat_generator_shape():
    scale, ef = 12, 16
    u, v = inputs.rmat_edges(scale, ef, seed=12)
    assert len(u) == ef << scale
    # quadrant frequencies at the top bit level: P(row bit 0) = a + b = 0.76,
    # P(col bit 0) = a + c = 0.76; P(D at top) = 0.05
    top = scale - 1
    bu, bv = (u >> top) & 1, (v >> top) & 1
    n = len(u)
    for frac, p in ((np.mean(bu == 0), 0.76), (np.mean(bv == 0), 0.76),
                    (np.mean((bu == 1) & (bv == 1)), 0.05)):
        assert abs(frac - p) < 4 * np.sqrt(p * (1 - p) / n)
    ro, col = inputs.build_csr(1 << scale, u, v)
    ne = ro[-1]
    assert ne <= 2 * len(u)
    rows = np.repeat(np.arange(1 << scale), np.diff(ro))
    assert not np.any(rows == col)                                  # no self-loops
    keys = rows * (1 << scale) + col
    assert np.all(np.diff(keys) > 0)                                 # sorted, no duplicates
    rev = np.sort(col.astype(np.int64) * (1 << scale) + rows)
    assert np.array_equal(rev, keys)                                 # symmetric


def test_weights_symmetric_and_in_range():
    g = inputs.rmat_graph(9, 8, seed=5, wmax=64, weight_seed=9)
    rows = np.repeat(np.arange(g.nv), np.diff(g.row_offsets))
    w = {(int(r), int(c)): int(x) for r, c, x in zip(rows, g.col_indices, g.weights)}
    assert all(w[(c, r)] == x for (r, c), x in w.items())
    assert min(w.values()) >= 1 and max(w.values()) <= 64
    gg = inputs.grid_graph(30, 20, p_del=0.1, seed=4, wmax=1000, weight_seed=2)
    assert gg.weights.min() >= 1 and gg.weights.max() <= 1000
    kept = gg.ne // 2
    total = 29 * 20 + 30 * 19
    assert abs(kept / total - 0.9) < 0.05


def test_pick_sources_non_isolated_distinct():
    g = inputs.rmat_graph(10, 4, seed=2)
    s = inputs.pick_sources(g.row_offsets, 16, seed=1)
    assert len(set(s.tolist())) == 16
    assert np.all(np.diff(g.row_offsets)[s] > 0)


# ---- betweenness centrality (Table 1's BC; Brandes' dependencies)

def _union_csr(n, masks, pairs):
    """Disjoint union of small graphs (graph g owns vertices g*n .. g*n+n-1)."""
    edges = []
    for gi, mask in enumerate(masks):
        edges += [(gi * n + a, gi * n + b) for pi, (a, b) in enumerate(pairs) if mask >> pi & 1]
    return inputs.csr_from_edges(n * len(masks), edges)


def _bc_by_matrix_powers(n, masks, pairs):
    """Definition-level BC of every vertex over every source, per graph.
    sigma_st = (A^k)[s,t] for k = d(s,t), since every walk of minimal length
    is a shortest path; d(s,t) = first k with (A^k)[s,t] > 0.  Then
    bc(v) = sum over s != v != t, d(s,v) + d(v,t) = d(s,t), of
    sigma_sv * sigma_vt / sigma_st."""
    m = len(masks)
    A = np.zeros((m, n, n), dtype=np.int64)
    for gi, mask in enumerate(masks):
        for pi, (a, b) in enumerate(pairs):
            if mask >> pi & 1:
                A[gi, a, b] = A[gi, b, a] = 1
    D = np.full((m, n, n), np.inf)
    S = np.zeros((m, n, n))
    D[:, np.arange(n), np.arange(n)] = 0
    S[:, np.arange(n), np.arange(n)] = 1
    P = np.broadcast_to(np.eye(n, dtype=np.int64), (m, n, n)).copy()
    for k in range(1, n):
        P = P @ A
        new = np.isinf(D) & (P > 0)
        D[new] = k
        S[new] = P[new]
    Dsv, Dvt, Dst = D[:, :, :, None], D[:, None, :, :], D[:, :, None, :]
    on = np.isfinite(Dst) & (Dsv + Dvt == Dst)
    idx = np.arange(n)
    on &= (idx[:, None, None] != idx[None, :, None])          # v != s
    on &= (idx[None, :, None] != idx[None, None, :])          # v != t
    on &= (idx[:, None, None] != idx[None, None, :])          # t != s
    frac = np.where(on, S[:, :, :, None] * S[:, None, :, :] / np.where(on, S[:, :, None, :], 1.0), 0.0)
    return frac.sum(axis=(1, 3)), frac[:, 0, :, :].sum(axis=2)   # all sources; source 0 only


def test_bc_exhaustive_5_vertices_matches_matrix_power_definition():
    n = 5
    pairs = list(itertools.combinations(range(n), 2))
    masks = list(range(1 << len(pairs)))
    g = _union_csr(n, masks, pairs)
    want_all, want_src0 = _bc_by_matrix_powers(n, masks, pairs)
    got_all = oracle.bc(g.row_offsets, g.col_indices, np.arange(g.nv))
    np.testing.assert_allclose(got_all, want_all.reshape(-1), rtol=1e-12, atol=1e-12)
    got_src0 = oracle.bc(g.row_offsets, g.col_indices, np.arange(0, g.nv, n))
    np.testing.assert_allclose(got_src0, want_src0.reshape(-1), rtol=1e-12, atol=1e-12)


def test_bc_random_7_vertex_graphs_match_matrix_power_definition():
    n = 7
    pairs = list(itertools.combinations(range(n), 2))
    rng = np.random.default_rng(7)
    masks = [int(x) for x in rng.integers(0, 1 << len(pairs), size=400)]
    g = _union_csr(n, masks, pairs)
    want_all, want_src0 = _bc_by_matrix_powers(n, masks, pairs)
    np.testing.assert_allclose(oracle.bc(g.row_offsets, g.col_indices, np.arange(g.nv)),
                               want_all.reshape(-1), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.bc(g.row_offsets, g.col_indices, np.arange(0, g.nv, n)),
                               want_src0.reshape(-1), rtol=1e-12, atol=1e-12)


def test_bc_closed_forms():
    n = 31
    path = inputs.csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    i = np.arange(n, dtype=np.float64)
    # all ordered pairs: vertex i lies inside i * (n-1-i) unordered pairs
    assert np.array_equal(oracle.bc(path.row_offsets, path.col_indices, np.arange(n)),
                          2 * i * (n - 1 - i))
    # from vertex 0: vertex i >= 1 lies on the paths to the n-1-i vertices beyond it
    d0, sig = oracle.bc(path.row_offsets, path.col_indices, [0], want_sigma=True)
    assert np.array_equal(d0, np.where(i >= 1, n - 1 - i, 0.0)) and np.all(sig == 1.0)
    # star with L leaves: the centre is on every leaf-to-leaf path
    L = 12
    star = inputs.csr_from_edges(L + 1, [(0, k) for k in range(1, L + 1)])
    b = oracle.bc(star.row_offsets, star.col_indices, np.arange(L + 1))
    assert b[0] == L * (L - 1) and np.all(b[1:] == 0)
    b1 = oracle.bc(star.row_offsets, star.col_indices, [3])
    assert b1[0] == L - 1 and np.all(b1[1:] == 0)
    # complete graph: no vertex is strictly inside a shortest path
    K = 9
    comp = inputs.csr_from_edges(K, list(itertools.combinations(range(K), 2)))
    assert np.all(oracle.bc(comp.row_offsets, comp.col_indices, np.arange(K)) == 0)
    # cycles: every vertex equal; the values sum to sum over ordered pairs of (d - 1)
    for c in (10, 11):
        cyc = inputs.csr_from_edges(c, [(k, (k + 1) % c) for k in range(c)])
        b = oracle.bc(cyc.row_offsets, cyc.col_indices, np.arange(c))
        k = np.arange(1, c)
        total = c * np.minimum(k, c - k).astype(np.float64).__sub__(1).sum()
        np.testing.assert_allclose(b, np.full(c, total / c), rtol=1e-13)
    # full lattice: shortest-path counts from (x0, y0) are binomial coefficients
    from math import comb
    w, h = 9, 7
    u, v = inputs.grid_edges(w, h, 0.0, seed=1)
    ro, col = inputs.build_csr(w * h, u, v)
    x0, y0 = 3, 2
    _, sig = oracle.bc(ro, col, [y0 * w + x0], want_sigma=True)
    want = [comb(abs(x - x0) + abs(y - y0), abs(x - x0)) for y in range(h) for x in range(w)]
    assert np.array_equal(sig, np.array(want, dtype=np.float64))


def test_bc_dependency_sum_identity_and_unreached():
    """sum over v of delta_s(v) = sum over reached t != s of (d(s,t) - 1): each
    shortest s-t path has d(s,t) - 1 interior vertices.  Checked against the
    BFS oracle's distances on an R-MAT graph; vertices in other components and
    the source get nothing."""
    g = _rmat_small()
    for s in inputs.pick_sources(g.row_offsets, 4, seed=2):
        s = int(s)
        delta = oracle.bc(g.row_offsets, g.col_indices, [s])
        d = oracle.bfs(g.row_offsets, g.col_indices, s)
        reached = d > 0
        np.testing.assert_allclose(delta.sum(), float((d[reached] - 1).sum()), rtol=1e-12)
        assert delta[s] == 0 and np.all(delta[d < 0] == 0) and np.all(delta >= 0)
    two = inputs.csr_from_edges(6, [(0, 1), (1, 2), (3, 4), (4, 5)])
    assert np.array_equal(oracle.bc(two.row_offsets, two.col_indices, [0]),
                          np.array([0, 1, 0, 0, 0, 0], dtype=np.float64))
    with pytest.raises(oracle.OracleError):
        oracle.bc(two.row_offsets, two.col_indices, [6])
