"""Autotuner: fingerprints (host), and on the GPU a search whose choice keeps
BFS results identical to the oracle and is cached by graph fingerprint."""
import os

import numpy as np
import pytest

import oracle
from paper_1504_04804_gb300 import autotune, inputs


def test_fingerprint_distinguishes_graphs_and_is_stable():
    g1 = inputs.rmat_graph(10, 16, seed=1)
    g2 = inputs.rmat_graph(10, 16, seed=2)
    g3 = inputs.grid_graph(32, 32, seed=1)
    f1 = autotune.fingerprint(g1.row_offsets)
    assert f1 == autotune.fingerprint(g1.row_offsets.copy())
    assert len({f1, autotune.fingerprint(g2.row_offsets), autotune.fingerprint(g3.row_offsets)}) == 3
    assert f1.startswith(f"nv{g1.nv}_ne{g1.ne}_")


@pytest.mark.gpu
def test_tuned_parameters_keep_results_exact(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_04804_gb300 import build, grx
    build.build()
    g = inputs.rmat_graph(13, 16, seed=13)
    dg = grx.load(g)
    cache = os.path.join(tmp_path, "tune.json")
    t = autotune.tune_bfs(dg, g.row_offsets, cache=cache)
    assert not t["cached"] and t["tried"] >= 36 + len(autotune.PUSH_BITMAPS) - 1
    assert t["exact_fv"] in (0, 1) and t["alpha"] in autotune.ALPHAS and t["beta"] in autotune.BETAS
    assert t["push_bitmap"] in autotune.PUSH_BITMAPS
    again = autotune.tune_bfs(dg, g.row_offsets, cache=cache)
    assert again["cached"] and again["alpha"] == t["alpha"]
    o = autotune.opts_from(grx, t)
    for s in inputs.pick_sources(g.row_offsets, 4, seed=5):
        assert np.array_equal(grx.bfs(dg, int(s), opts=o).cpu().numpy(),
                              oracle.bfs(g.row_offsets, g.col_indices, int(s)))
    # every push_bitmap candidate gives the oracle's depths (the knob only moves work)
    s = int(inputs.pick_sources(g.row_offsets, 1, seed=9)[0])
    want = oracle.bfs(g.row_offsets, g.col_indices, s)
    for pb in autotune.PUSH_BITMAPS:
        for mode in (grx.GRX_DIR_AUTO, grx.GRX_DIR_PUSH):
            o = grx.opts(push_bitmap=pb, direction=mode)
            assert np.array_equal(grx.bfs(dg, s, opts=o).cpu().numpy(), want), (pb, mode)


@pytest.mark.gpu
def test_tuned_multi_source_knobs_keep_lanes_exact(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_04804_gb300 import build, grx
    build.build()
    g = inputs.rmat_graph(12, 16, seed=12)
    dg = grx.load(g)
    cache = os.path.join(tmp_path, "tune.json")
    t = autotune.tune_bfs_multi(dg, g.row_offsets, lanes=16, cache=cache)
    assert not t["cached"]
    assert t["tried"] == len(autotune.MULTI_ALPHAS) * len(autotune.MULTI_BETAS) + len(autotune.PUSH_BITMAPS) - 1
    assert t["alpha"] in autotune.MULTI_ALPHAS and t["beta"] in autotune.MULTI_BETAS
    assert t["push_bitmap"] in autotune.PUSH_BITMAPS
    assert autotune.tune_bfs_multi(dg, g.row_offsets, lanes=16, cache=cache)["cached"]
    lanes = [int(x) for x in inputs.pick_sources(g.row_offsets, 16, seed=6)]
    want = [oracle.bfs(g.row_offsets, g.col_indices, s) for s in lanes]
    # the chosen knobs and every other candidate of the search keep every lane exact
    cands = [dict(alpha=t["alpha"], beta=t["beta"], push_bitmap=t["push_bitmap"])]
    cands += [dict(alpha=a, beta=b) for a in autotune.MULTI_ALPHAS for b in autotune.MULTI_BETAS]
    cands += [dict(push_bitmap=pb) for pb in autotune.PUSH_BITMAPS]
    for kw in cands:
        d = grx.bfs_multi(dg, lanes, opts=grx.opts(**kw)).cpu().numpy()
        for b in range(len(lanes)):
            assert np.array_equal(d[b], want[b]), (kw, b)


@pytest.mark.gpu
def test_tuned_sssp_delta_keeps_distances_exact(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_04804_gb300 import build, grx
    build.build()
    g = inputs.grid_graph(64, 64, p_del=0.1, seed=64, wmax=1000, weight_seed=164)
    dg = grx.load(g)
    cache = os.path.join(tmp_path, "tune.json")
    t = autotune.tune_sssp_delta(dg, g.row_offsets, g.weights, cache=cache)
    mean_w = float(np.mean(g.weights))
    assert not t["cached"] and t["tried"] == len(autotune.DELTA_FACTORS)
    assert t["sssp_delta"] in [int(min(f * mean_w, 2 ** 31)) for f in autotune.DELTA_FACTORS]
    assert autotune.tune_sssp_delta(dg, g.row_offsets, g.weights, cache=cache)["cached"]
    o = grx.opts(sssp_delta=t["sssp_delta"])
    for s in inputs.pick_sources(g.row_offsets, 4, seed=5):
        assert np.array_equal(grx.as_uint32(grx.sssp(dg, int(s), opts=o)),
                              oracle.sssp(g.row_offsets, g.col_indices, g.weights, int(s)))
