"""The frozen algorithmic-byte models of bench.py (the roofline numerators),
checked against hand-computed counts: every byte each model counts is
written out here from the per-unit figures (a push level reads the queue
slot, two row offsets and writes depth and the next slot; a pull level
reads row offsets and the non-isolated word per scanned vertex, and so on),
so a change to a model's arithmetic fails here."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_bfs_bytes_push_and_pull_levels():
    # level 0: push, |Q| = 1, 40 edges examined; level 1: pull over 1,000
    # candidates, 2,500 edges examined, 900 found; V = 4,096 (o = 4 and 8)
    st = {"levels": 2, "dir": [0, 1], "frontier": [1, 40], "edges_examined": [40, 2500],
          "vertices_scanned": [1, 1000], "discovered": [40, 900]}
    for o in (4, 8):
        push = 1 * (o + o + 4 + 4 + 4) + 40 * (4 + 4)
        pull = 1000 * (o + o + 4) + 2500 * (4 + 4) + 900 * (4 + 4) + 4096 // 8
        assert bench.bfs_bytes(st, 4096, o) == push + pull


def test_sssp_pr_cc_bytes():
    st = {"levels": 2, "frontier": [1, 7], "edges_examined": [5, 90]}
    assert bench.sssp_bytes(st, 4) == (1 * (4 + 4 + 4 + 4) + 5 * (4 + 4 + 8)) + (7 * 16 + 90 * 16)
    # PageRank: per iteration row offset + c read + r write + c write per vertex, column + gather per edge
    assert bench.pr_bytes(100, 1000, 4, 20) == 20 * (100 * (4 + 4 + 4 + 4) + 1000 * (4 + 4))
    assert bench.pr_bytes(100, 1000, 8, 1) == 100 * (8 + 12) + 1000 * 8
    # CC: 12 bytes per hooked edge, three row passes and three jumps
    assert bench.cc_bytes(1000, 300, 4) == 300 * 12 + 3 * 1000 * (4 + 4) + 3 * 1000 * 8


def test_msbfs_bytes_includes_the_depth_output():
    st = {"dir": [0, 1], "frontier": [64, 10], "edges_examined": [700, 5000], "vertices_scanned": [64, 900]}
    want = 4 * 64 * 2000 + (64 * (2 * 4 + 8) + 700 * (4 + 8 + 8)) + (900 * (2 * 4 + 8) + 5000 * (4 + 12))
    assert bench.msbfs_bytes(st, 2000, 4, 64) == want


def test_bc_bytes():
    o = 8
    per_vertex = 2 * o + 2 * (8 + o) + 12 + (8 + o) + 32
    assert bench.bc_bytes(1000, 600, 5000, 1200, o) == \
        1000 * 16 + 3 * 1000 // 8 + 600 * per_vertex + 5000 * 8 + 1200 * 16
