"""Per-graph autotuner for the traversal knobs.

Sec. 6.1 observes that the best direction-switch parameters (do_a, do_b) are
consistent for graphs of a similar type; this module finds them per graph by
measurement instead of hand-setting them.  It searches, with CUDA-event
timings on a few seeded tuning sources (single-source BFS: each traversal
timed alone from a flushed L2, the benchmark's condition):

* the switch rule: the paper's estimate FV = |Q|*E/V, or the frontier's exact
  edge count (``exact_fv``), which the append counter provides for free;
* alpha (push->pull) and beta (pull->push);
* the persistent grid size (full occupancy or half of it);
* the load-balance threshold between the two push kinds (``push_bitmap``):
  levels whose frontier holds at least push_bitmap * nv edges mark targets in
  a bitmap and build the next queue in a second, word-owning pass; smaller
  ones claim each target with an atomic and append it at once.  Searched
  after the switch knobs (coordinate descent).  Edge tiles are balanced by
  construction, and the per-lane / per-group widths are compile-time
  constants;
* for the 64-lane multi-source BFS, its own alpha / beta / push_bitmap
  (``tune_bfs_multi``): the rule acts on lane popcounts there;
* for SSSP, the near-far band width delta (``tune_sssp_delta``).

Results do not depend on the parameters (the tests check this); only the
time does.  The choice is cached in a JSON file keyed by a fingerprint of the
graph (vertex and edge counts plus a hash of the log2 degree histogram).
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os
import statistics
import time

import numpy as np

ALPHAS = (1e-6, 1e-5, 1e-4, 1e-3, 5e-3, 0.01, 0.05, 0.2)
BETAS = (0.01, 0.1, 1.0)
RULES = (0, 1)
# push_bitmap candidates: 0 = the library default (1/8), < 0 = never
PUSH_BITMAPS = (0.0, 1.0 / 64, 1.0 / 32, 0.5, -1.0)
MULTI_ALPHAS = (1e-4, 1e-3, 0.01, 0.05, 0.2, 1.0)
MULTI_BETAS = (0.01, 0.1, 1.0)
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "grx_autotune.json")


def fingerprint(row_offsets) -> str:
    """nv, ne and a hash of the log2-bucketed degree histogram."""
    ro = np.asarray(row_offsets, dtype=np.int64)
    deg = np.diff(ro)
    buckets = np.bincount(np.floor(np.log2(deg[deg > 0])).astype(np.int64), minlength=40) \
        if np.any(deg > 0) else np.zeros(40, dtype=np.int64)
    h = hashlib.sha1(buckets.astype(np.int64).tobytes()).hexdigest()[:16]
    return f"nv{ro.shape[0] - 1}_ne{int(ro[-1])}_{h}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def _save(path, data):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _l2_flush(torch, device):
    """A 256 MiB device buffer (twice the GB300's L2); writing it before a
    timed traversal evicts the graph, as the benchmark does.  Held only for
    the duration of one tuning call."""
    return torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{device}")


def _time_config(grx, torch, g, sources, kw, reps, flush):
    """Median over sources of the per-traversal kernel time (ms) and the sum
    over sources of the mean time; every timed traversal starts from a
    flushed L2 (the benchmark's condition, `flush` written first), timed alone
    with CUDA events."""
    o = grx.opts(**kw)
    stream = torch.cuda.current_stream()
    depth = torch.empty(g.nv, dtype=torch.int32, device=f"cuda:{g.device}")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(len(sources) * reps)]
    i = 0
    for s in sources:
        grx.bfs(g, s, depth_out=depth, opts=o)           # warm
        for _ in range(reps):
            flush.fill_(i & 0xff)
            evs[i][0].record(stream)
            grx.bfs(g, s, depth_out=depth, opts=o)
            evs[i][1].record(stream)
            i += 1
    evs[-1][1].synchronize()
    ts = [sum(evs[k * reps + r][0].elapsed_time(evs[k * reps + r][1]) for r in range(reps)) / reps
          for k in range(len(sources))]
    return statistics.median(ts), sum(ts)


def tune_bfs(g, row_offsets, n_sources: int = 8, seed: int = 2, reps: int = 2,
             cache: str | None = DEFAULT_CACHE, force: bool = False) -> dict:
    """Search the knobs for direction-optimising BFS on a loaded graph.
    Returns {"alpha", "beta", "exact_fv", "grid_blocks", "push_bitmap", "ms",
    "tried", "seconds", "fingerprint", "cached"}."""
    import torch

    from . import grx, inputs
    fp = fingerprint(row_offsets)
    if cache and not force:
        hit = _load(cache).get(fp)
        if hit:
            return dict(hit, cached=True)
    t0 = time.time()
    sources = [int(s) for s in inputs.pick_sources(row_offsets, n_sources, seed)]
    flush = _l2_flush(torch, g.device)
    grids = (0, -1)          # full occupancy, half of it
    best = None
    tried = 0
    full = None
    for rule, a, b, gsel in itertools.product(RULES, ALPHAS, BETAS, grids):
        kw = {"exact_fv": rule, "alpha": a, "beta": b}
        if gsel == -1:
            if full is None:
                continue
            kw["grid_blocks"] = max(1, full // 2)
        med, tot = _time_config(grx, torch, g, sources, kw, reps, flush)
        tried += 1
        if best is None or tot < best[0]:
            best = (tot, kw, med)
        if full is None:
            full = _occupancy_grid(grx, g)
    # then the push-kind threshold with the chosen switch knobs
    base = dict(best[1])
    for pb in PUSH_BITMAPS[1:]:
        kw = dict(base, push_bitmap=pb)
        med, tot = _time_config(grx, torch, g, sources, kw, reps, flush)
        tried += 1
        if tot < best[0]:
            best = (tot, kw, med)
    tot, kw, med = best
    grx.graph_status(g)
    res = {"alpha": kw["alpha"], "beta": kw["beta"], "exact_fv": kw["exact_fv"],
           "grid_blocks": kw.get("grid_blocks", 0), "push_bitmap": kw.get("push_bitmap", 0.0),
           "ms": med, "tried": tried,
           "seconds": time.time() - t0, "fingerprint": fp, "tuning_sources": sources}
    if cache:
        data = _load(cache)
        data[fp] = res
        _save(cache, data)
    return dict(res, cached=False)


def tune_bfs_multi(g, row_offsets, lanes: int = 64, seed: int = 4, reps: int = 2,
                   cache: str | None = DEFAULT_CACHE, force: bool = False) -> dict:
    """alpha / beta (on lane popcounts) and then push_bitmap for the 64-lane
    multi-source BFS, timed on one batch of `lanes` seeded tuning sources.
    Returns {"alpha", "beta", "push_bitmap", "ms", "tried", "seconds",
    "fingerprint", "cached"}."""
    import torch

    from . import grx, inputs
    fp = fingerprint(row_offsets) + f"_multi{lanes}"
    if cache and not force:
        hit = _load(cache).get(fp)
        if hit:
            return dict(hit, cached=True)
    t0 = time.time()
    sources = [int(s) for s in inputs.pick_sources(row_offsets, lanes, seed)]
    out = torch.empty(len(sources) * g.nv, dtype=torch.int32, device=f"cuda:{g.device}")
    stream = torch.cuda.current_stream()

    def timed(kw):
        o = grx.opts(**kw)
        grx.bfs_multi(g, sources, depth_out=out, opts=o)            # warm
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(reps):
            grx.bfs_multi(g, sources, depth_out=out, opts=o)
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / reps

    best, tried = None, 0
    for a, b in itertools.product(MULTI_ALPHAS, MULTI_BETAS):
        kw = {"alpha": a, "beta": b}
        ms = timed(kw)
        tried += 1
        if best is None or ms < best[0]:
            best = (ms, kw)
    base = dict(best[1])
    for pb in PUSH_BITMAPS[1:]:
        kw = dict(base, push_bitmap=pb)
        ms = timed(kw)
        tried += 1
        if ms < best[0]:
            best = (ms, kw)
    ms, kw = best
    grx.graph_status(g)
    res = {"alpha": kw["alpha"], "beta": kw["beta"], "push_bitmap": kw.get("push_bitmap", 0.0),
           "ms": ms, "tried": tried, "seconds": time.time() - t0, "fingerprint": fp,
           "tuning_sources": sources}
    if cache:
        data = _load(cache)
        data[fp] = res
        _save(cache, data)
    return dict(res, cached=False)


DELTA_FACTORS = (0, 4, 16, 64, 256, 1024, 4096)


def tune_sssp_delta(g, row_offsets, weights, n_sources: int = 2, seed: int = 3,
                    cache: str | None = DEFAULT_CACHE, force: bool = False) -> dict:
    """Near-far band width for SSSP on a loaded weighted graph: 0 (plain
    label-correcting rounds) or the mean edge weight times 4 ... 4096
    (Davidson et al. scale the band with the weights), whichever gives the
    smallest total kernel time over the tuning sources.
    Returns {"sssp_delta", "ms", "tried", "seconds", "fingerprint", "cached"}."""
    import torch

    from . import grx, inputs
    w = weights.cpu().numpy() if hasattr(weights, "cpu") else np.asarray(weights)
    fp = fingerprint(row_offsets) + f"_w{int(w.sum()) if w.size else 0}_sssp"
    if cache and not force:
        hit = _load(cache).get(fp)
        if hit:
            return dict(hit, cached=True)
    t0 = time.time()
    mean_w = max(1.0, float(w.mean())) if w.size else 1.0
    sources = [int(s) for s in inputs.pick_sources(row_offsets, n_sources, seed)]
    stream = torch.cuda.current_stream()
    dist = torch.empty(g.nv, dtype=torch.int32, device=f"cuda:{g.device}")
    best = None
    for f in DELTA_FACTORS:
        delta = int(min(f * mean_w, 2 ** 31))
        o = grx.opts(sssp_delta=delta)
        tot = 0.0
        for s in sources:
            grx.sssp(g, s, dist_out=dist, opts=o)          # warm
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            grx.sssp(g, s, dist_out=dist, opts=o)
            ev1.record(stream)
            ev1.synchronize()
            tot += ev0.elapsed_time(ev1)
        if best is None or tot < best[0]:
            best = (tot, delta)
    grx.graph_status(g)
    res = {"sssp_delta": best[1], "ms": best[0] / len(sources), "tried": len(DELTA_FACTORS),
           "seconds": time.time() - t0, "fingerprint": fp, "tuning_sources": sources}
    if cache:
        data = _load(cache)
        data[fp] = res
        _save(cache, data)
    return dict(res, cached=False)


def _occupancy_grid(grx, g) -> int:
    """The persistent grid the library picks (SMs x resident blocks)."""
    import torch
    props = torch.cuda.get_device_properties(g.device)
    return props.multi_processor_count * 3


def opts_from(grx, tuned: dict, **extra):
    """grx_opts carrying a tuning result."""
    kw = {"alpha": tuned["alpha"], "beta": tuned["beta"], "exact_fv": tuned.get("exact_fv", 0),
          "grid_blocks": tuned.get("grid_blocks", 0), "push_bitmap": tuned.get("push_bitmap", 0.0)}
    kw.update(extra)
    return grx.opts(**kw)
