"""Continuous-batching query servers over resident graphs.

Graphs stay loaded on the GPU.  Requests (a BFS or SSSP query: graph, source)
arrive over time.  Each (graph, kind) pair has one or more 64-lane batches
(``grx.Batch``), each on its own CUDA stream, so batches of different graphs
run concurrently on the device.  The loop:

1. admit arrived requests, first come first served, into a free lane of a
   running batch of their graph and kind -- they join at the next level
   boundary of a traversal already in flight -- or open a new batch when the
   free device memory covers the batch's footprint (``grx_batch_footprint``)
   plus the outputs it will hold; otherwise the request waits;
2. enqueue a few level steps on every batch with work (asynchronous, one
   stream per batch);
3. poll every batch; a retired lane's query is complete: its latency is
   completion minus arrival time, and its TEPS numerator (edges of the
   reached component) is reduced on the device before the output is freed.

Each query's result is exactly its single-source result (tests check alone
vs. in the mix).  ``run_one_at_a_time`` is the baseline: the same requests
served FIFO by single-source calls on one stream of the same GPU.

``TraversalServer`` batches at traversal boundaries instead: requests that
arrive while a traversal runs join the next multi-source traversal of their
graph and kind (one persistent kernel for up to 64 lanes).  It admits by free
device memory too (``plan_lanes``): a traversal starts only when its
workspace (``grx_multi_footprint``, allocated on a handle's first multi-source
call) and its lanes' outputs fit; otherwise it waits for running traversals
to return memory, or, when none runs, starts with as many lanes as fit.
"""
from __future__ import annotations

import statistics
import time
from dataclasses import dataclass, field

import numpy as np

KINDS = {"bfs": 0, "sssp": 1}


@dataclass
class Request:
    rid: int
    graph: str
    kind: str
    src: int
    arrival: float                      # seconds from the start of the run
    admitted: float = -1.0
    done: float = -1.0
    edges: int = 0                      # TEPS numerator (edges of the reached component)
    result: object = None               # kept only when keep_results is set


def make_requests(graphs: dict, n: int, rate_qps: float, seed: int = 0,
                  kinds=("bfs", "sssp")) -> list[Request]:
    """n requests with Poisson arrivals (rate_qps per second), graph chosen
    uniformly, kind uniformly from kinds, source a seeded non-isolated vertex.
    graphs: name -> (row_offsets as numpy, weighted: bool)."""
    from . import inputs
    rng = np.random.default_rng(seed)
    names = sorted(graphs)
    gaps = rng.exponential(1.0 / rate_qps, size=n) if rate_qps > 0 else np.zeros(n)
    t = np.cumsum(gaps) - gaps[0]
    pools = {name: inputs.pick_sources(graphs[name][0], min(4096, int(np.count_nonzero(
        np.diff(graphs[name][0])))), seed=seed + 17 + i) for i, name in enumerate(names)}
    reqs = []
    for i in range(n):
        name = names[int(rng.integers(len(names)))]
        kind = kinds[int(rng.integers(len(kinds)))]
        if kind == "sssp" and not graphs[name][1]:
            kind = "bfs"
        pool = pools[name]
        reqs.append(Request(i, name, kind, int(pool[int(rng.integers(len(pool)))]), float(t[i])))
    return reqs


def plan_admission(pending: list, free_lanes: dict, free_bytes: int, footprints: dict,
                   out_bytes: dict, open_batches: dict):
    """Pure admission policy (host logic, testable without a GPU).

    pending: requests in arrival order; free_lanes: (graph, kind) -> free lanes
    over its open batches; free_bytes: device memory available; footprints /
    out_bytes: (graph, kind) -> bytes of a new batch / of one query's output.
    Returns (admit, new_batches, waiting): requests to admit now (in order),
    (graph, kind) keys of batches to open first, and the requests that wait."""
    lanes = dict(free_lanes)
    budget = free_bytes
    admit, new, waiting = [], [], []
    for r in pending:
        key = (r.graph, r.kind)
        if lanes.get(key, 0) > 0 and budget >= out_bytes[key]:
            lanes[key] -= 1
            budget -= out_bytes[key]
            admit.append(r)
        elif budget >= footprints[key] + out_bytes[key]:
            new.append(key)
            budget -= footprints[key] + out_bytes[key]
            lanes[key] = lanes.get(key, 0) + 63
            admit.append(r)
        else:
            waiting.append(r)
    return admit, new, waiting


@dataclass
class _Slot:
    batch: object
    key: tuple
    lanes: dict = field(default_factory=dict)   # lane -> (request, output tensor)
    ev: object = None                           # event after the last enqueued steps


class Server:
    def __init__(self, graphs: dict, degrees: dict, steps_per_poll: int = 2,
                 reserve_bytes: int = 1 << 30, budget_bytes: int | None = None,
                 keep_results: bool = False):
        """graphs: name -> grx.Graph (loaded); degrees: name -> device int32
        degree tensor (for the TEPS numerator).  budget_bytes caps the device
        memory the server may use for batches (default: what is free)."""
        import torch

        from . import grx
        self.torch, self.grx = torch, grx
        self.graphs = graphs
        self.degrees = degrees
        self.steps_per_poll = steps_per_poll
        self.reserve = reserve_bytes
        self.budget = budget_bytes
        self.keep = keep_results
        self.slots: list[_Slot] = []
        self.footprints = {}
        self.out_bytes = {}
        for name, g in graphs.items():
            for kind, k in KINDS.items():
                if kind == "sssp" and not g.weighted:
                    continue
                self.footprints[(name, kind)] = grx.batch_footprint(g, k)
                self.out_bytes[(name, kind)] = 4 * g.nv
        self.used = 0

    def _free_bytes(self) -> int:
        if self.budget is not None:
            return self.budget - self.used
        torch = self.torch
        free, _ = torch.cuda.mem_get_info()
        # memory torch's caching allocator holds but does not use is free too
        cached = torch.cuda.memory_reserved() - torch.cuda.memory_allocated()
        return free + cached - self.reserve

    def _admit(self, pending: list, now: float) -> list:
        free_lanes = {}
        for s in self.slots:
            free_lanes[s.key] = free_lanes.get(s.key, 0) + 64 - len(s.lanes)
        admit, new, waiting = plan_admission(pending, free_lanes, self._free_bytes(),
                                             self.footprints, self.out_bytes, {})
        for key in new:
            g = self.graphs[key[0]]
            b = self.grx.Batch(g, KINDS[key[1]])
            self.slots.append(_Slot(b, key))
            self.used += self.footprints[key]
        for r in admit:
            key = (r.graph, r.kind)
            slot = next(s for s in self.slots if s.key == key and len(s.lanes) < 64)
            g = self.graphs[r.graph]
            with self.torch.cuda.stream(slot.batch.stream):
                out = self.torch.empty(g.nv, dtype=self.torch.int32, device=f"cuda:{g.device}")
            lane = slot.batch.admit(r.src, out)
            slot.lanes[lane] = (r, out)
            self.used += self.out_bytes[key]
            r.admitted = now
        return waiting

    def _finish(self, slot: _Slot, mask: int, now: float, t0: float):
        torch = self.torch
        for lane in list(slot.lanes):
            if not (mask >> lane & 1):
                continue
            r, out = slot.lanes.pop(lane)
            deg = self.degrees[r.graph]
            with torch.cuda.stream(slot.batch.stream):
                if r.kind == "bfs":
                    reached = out >= 0
                else:
                    reached = out != -1                  # UINT32_MAX bits read as int32 -1
                r.edges = int((deg * reached).sum().item())
            r.done = now
            if self.keep:
                r.result = out
            self.used -= self.out_bytes[slot.key]

    def run(self, requests: list[Request], realtime: bool = True) -> dict:
        """Serve the requests (arrival times relative to the start)."""
        torch = self.torch
        order = sorted(requests, key=lambda r: r.arrival)
        pending: list[Request] = []
        nxt = 0
        t0 = time.perf_counter()
        inflight = 0
        while nxt < len(order) or pending or inflight:
            now = time.perf_counter() - t0
            while nxt < len(order) and (order[nxt].arrival <= now or not realtime):
                pending.append(order[nxt])
                nxt += 1
            if pending:
                before = len(pending)
                pending = self._admit(pending, now)
                inflight += before - len(pending)
                if pending and inflight == 0 and not self.slots_busy():
                    raise RuntimeError("admission impossible: a batch and its outputs do not fit "
                                       f"in the device memory budget ({self._free_bytes()} bytes free)")
            busy = [s for s in self.slots if s.lanes or s.ev is not None]
            for s in busy:
                # a batch whose last steps are still running is left alone, so a
                # slow batch never holds up the others
                if s.ev is not None and not s.ev.query():
                    continue
                if s.ev is not None:
                    mask = s.batch.poll()            # its stream is idle: returns at once
                    s.ev = None
                    if mask:
                        done_now = time.perf_counter() - t0
                        n_before = len(s.lanes)
                        self._finish(s, mask, done_now, t0)
                        inflight -= n_before - len(s.lanes)
                if s.lanes:
                    s.batch.step(self.steps_per_poll)
                    s.ev = torch.cuda.Event()
                    s.ev.record(s.batch.stream)
            if not busy and not pending and nxt < len(order) and realtime:
                wait = order[nxt].arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.01))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        return summarize(requests, wall)

    def slots_busy(self) -> bool:
        return any(s.lanes for s in self.slots)

    def close(self):
        for s in self.slots:
            s.batch.close()
        self.slots = []


def plan_lanes(wanted: int, ws_bytes: int, lane_bytes: int, free_bytes: int,
               others_running: bool) -> int:
    """Pure memory admission of one traversal (host logic, testable without
    a GPU): the lanes (queries) to start now out of `wanted`, given the
    workspace the launch would allocate first and the bytes each lane's
    output needs.  All of them when they fit; when they do not and other
    traversals are running, 0 (wait: those return memory when they finish);
    when nothing else runs, as many as fit, at least 1 -- and MemoryError if
    not even one lane fits."""
    if wanted <= 0:
        return 0
    if ws_bytes + wanted * lane_bytes <= free_bytes:
        return wanted
    if others_running:
        return 0
    fit = (free_bytes - ws_bytes) // lane_bytes if lane_bytes > 0 else wanted
    if fit < 1:
        raise MemoryError(f"a traversal needs {ws_bytes + lane_bytes} bytes of device memory, "
                          f"{free_bytes} are free")
    return int(min(wanted, fit))


def batch_threshold(t_single_ms: float, t_batch_ms: dict, max_ms: float | None = None):
    """Batch sizes worth serving from measured times (t_batch_ms: lanes ->
    time of one traversal of that many lanes): (smallest n from which
    sharing one traversal costs less than n single-source traversals, i.e.
    time / n < t_single; the most lanes whose traversal stays within max_ms,
    the latency a batch may add -- read off the measured sizes, at least the
    smallest winning one).  (65, 64) -- never batch -- when no measured size
    wins within max_ms.  Host logic, testable without a GPU."""
    wins = [n for n, t in sorted(t_batch_ms.items())
            if n >= 2 and t < n * t_single_ms and (max_ms is None or t <= max_ms)]
    if not wins:
        return 65, 64
    # from the smallest winning size on, assume larger batches win too; the
    # lane cap is the largest measured size within the latency bound
    ok = [n for n, t in sorted(t_batch_ms.items()) if max_ms is None or t <= max_ms]
    return wins[0], max(max(ok), wins[0])


def plan_job(pending: dict, sssp_multi_min: int = 24, lanes: int = 64, busy=(), bfs_multi_min: int = 2,
             thresholds: dict | None = None):
    """Pure policy of the traversal-boundary server (host logic, testable
    without a GPU).  pending: (graph, kind) -> requests in arrival order;
    busy: graphs with a traversal in flight (a graph's workspace serves one
    traversal at a time).  The key whose oldest request arrived first is
    served next: BFS requests (up to `lanes`) share one multi-source traversal
    when there are two or more, SSSP requests when at least `sssp_multi_min`
    wait (a batched SSSP lane costs less than a single-source traversal only
    in a full batch); `thresholds` ((graph, kind) -> (smallest, largest
    batch)) overrides both per graph; otherwise the oldest request runs alone.  Returns
    (key, requests, multi) or None when nothing can start."""
    keys = [k for k, v in pending.items() if v and k[0] not in busy]
    if not keys:
        return None
    key = min(keys, key=lambda k: (pending[k][0].arrival, pending[k][0].rid))
    waiting = pending[key]
    thresh = bfs_multi_min if key[1] == "bfs" else sssp_multi_min
    if thresholds and key in thresholds:
        thresh, lanes = thresholds[key]
    if len(waiting) >= thresh:
        return key, waiting[:lanes], True
    return key, waiting[:1], False


class TraversalServer:
    """Continuous batching at traversal boundaries: requests that arrive while
    a traversal runs join the next one of their graph and kind, which the
    persistent multi-source kernels run (64 lanes, one launch).  Compared with
    joining at level boundaries (``Server``) a request may wait for the
    traversal in flight, but every level costs one grid barrier instead of a
    host round trip and several launches.  Graph handles are independent:
    each has its own workspace, stream and one traversal in flight, so
    traversals of different graphs (or of replica handles of one graph) run
    side by side, each on a share of the persistent grid while other work
    waits (a small graph's levels are as fast on a third of the SMs), on the
    whole grid when it runs alone.  A traversal starts only when its device
    memory fits (``plan_lanes``: the handle's multi-source workspace on its
    first use, plus per lane the output and the reduction's scratch).  Each
    query's result is its single-source result (tests check alone vs. in the
    mix)."""

    def __init__(self, graphs: dict, degrees: dict, sssp_multi_min: int = 24,
                 keep_results: bool = False, replicas: dict | None = None,
                 share_big: int = 2, share_small: int = 4, reserve_bytes: int = 1 << 30,
                 budget_bytes: int | None = None, calibrate: bool = False, sssp_share: int = 0,
                 exclusive_ms: float | None = None, max_batch_ms: float | None = None,
                 full_grid_ms: float | None = None):
        """replicas: graph name -> extra loaded handles of the same graph
        (each with its own workspace), so that several traversals of one
        graph can be in flight.  budget_bytes caps the device memory the
        server's traversals may take (default: what is free, less
        reserve_bytes).  calibrate: time one single-source and one 8- and
        64-lane traversal of each graph and kind at start-up and batch a kind
        only from the size where sharing a traversal wins (batch_threshold);
        otherwise BFS batches from 2 waiting requests and SSSP from
        sssp_multi_min.  sssp_share > 0: an SSSP traversal that shares the
        GPU runs on 1/sssp_share of the grid instead of its graph's share.
        exclusive_ms (needs calibrate): a kind whose calibrated single-source
        time is at least this long runs alone on the whole grid -- it starts
        when nothing else runs and nothing starts beside it -- as in the
        one-at-a-time baseline, so sharing never stretches the longest
        queries, which set the tail latency; shorter kinds batch and share.
        max_batch_ms (with calibrate): a batch's traversal may take at most
        this long (the latency batching may add to its queries).
        full_grid_ms (with calibrate): kinds whose single-source time is at
        least this long start on the whole grid at once, beside whatever runs
        (their blocks take SMs as they free up); the rest use shares."""
        import torch

        from . import grx
        self.torch, self.grx = torch, grx
        self.degrees = degrees
        self.sssp_multi_min = sssp_multi_min
        self.keep = keep_results
        self.handles = {name: [g] + list((replicas or {}).get(name, [])) for name, g in graphs.items()}
        self.streams = {(name, i): torch.cuda.Stream() for name, hs in self.handles.items()
                        for i in range(len(hs))}
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        full = props.multi_processor_count * 3
        # grid share while other traversals run: 1/share_small of the
        # persistent grid, 1/share_big for the largest graphs (their levels
        # scale with the SMs); 1 = the whole grid
        big = max(g.ne for g in graphs.values())
        self.share = {name: max(1, full // (share_big if g.ne * 4 >= big else share_small))
                      for name, g in graphs.items()}
        self.full = full
        self.sssp_share = max(1, full // sssp_share) if sssp_share > 0 else 0
        self.t_single = {}
        self.max_batch_ms = max_batch_ms
        self.thresholds = self._calibrate(graphs) if calibrate else None
        self.exclusive = {k for k, t in self.t_single.items()
                          if exclusive_ms is not None and t >= exclusive_ms}
        self.full_grid = {k for k, t in self.t_single.items()
                          if full_grid_ms is not None and t >= full_grid_ms}
        self.reserve = reserve_bytes
        self.budget = budget_bytes
        self.used = 0                                 # bytes taken under budget_bytes
        self.admission_waits = 0                      # traversals that waited for memory
        self.shrunk = 0                               # traversals started with fewer lanes

    def _calibrate(self, graphs: dict) -> dict:
        """(graph, kind) -> (smallest, largest) batch worth a shared traversal."""
        from . import inputs
        grx, torch = self.grx, self.torch
        out = {}

        def ms(fn):
            fn()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            return a.elapsed_time(b)
        for name, g in graphs.items():
            deg = self.degrees[name].cpu().numpy()
            ro = np.concatenate([[0], np.cumsum(deg.astype(np.int64))])
            srcs = [int(x) for x in inputs.pick_sources(ro, 64, seed=99)]
            for kind in ("bfs", "sssp"):
                if kind == "sssp" and not g.weighted:
                    continue
                one = grx.bfs if kind == "bfs" else grx.sssp
                many = grx.bfs_multi if kind == "bfs" else grx.sssp_multi
                t1 = statistics.median(ms(lambda s=s: one(g, s)) for s in srcs[:3])
                self.t_single[(name, kind)] = t1
                tb = {n: ms(lambda n=n: many(g, srcs[:n])) for n in (4, 8, 16, 32, 64)}
                out[(name, kind)] = batch_threshold(t1, tb, self.max_batch_ms)
        torch.cuda.synchronize()
        return out

    def _free_bytes(self) -> int:
        if self.budget is not None:
            return self.budget - self.used
        torch = self.torch
        free, _ = torch.cuda.mem_get_info()
        cached = torch.cuda.memory_reserved() - torch.cuda.memory_allocated()
        return free + cached - self.reserve

    def _lane_bytes(self, name: str) -> int:
        # output (4 bytes per vertex), reached flags (1) and the masked degree
        # the edge count reduces (4), per lane
        return 9 * self.handles[name][0].nv + 64

    def _launch(self, slot, key, reqs, multi, grid_blocks):
        grx, torch = self.grx, self.torch
        g = self.handles[key[0]][slot[1]]
        st = self.streams[slot]
        o = grx.opts(grid_blocks=grid_blocks)
        with torch.cuda.stream(st):
            srcs = [r.src for r in reqs]
            if key[1] == "bfs":
                out = grx.bfs_multi(g, srcs, opts=o, stream=st) if multi else \
                    grx.bfs(g, srcs[0], opts=o, stream=st).view(1, -1)
                reached = out >= 0
            else:
                out = grx.sssp_multi(g, srcs, opts=o, stream=st) if multi else \
                    grx.sssp(g, srcs[0], opts=o, stream=st).view(1, -1)
                reached = out != -1                  # UINT32_MAX bits read as int32 -1
            edges = torch.where(reached, self.degrees[key[0]], 0).sum(dim=1, dtype=torch.int64)
            del reached
            ev = torch.cuda.Event()
            ev.record(st)
        return out, edges, ev

    def run(self, requests: list[Request], realtime: bool = True) -> dict:
        torch = self.torch
        self.admission_waits = 0
        self.shrunk = 0
        order = sorted(requests, key=lambda r: r.arrival)
        pending: dict = {}
        nxt = 0
        jobs: dict = {}                               # (graph, replica) -> (requests, out, edges, event, bytes)
        job_keys: dict = {}                           # (graph, replica) -> (graph, kind) of its traversal
        t0 = time.perf_counter()
        while nxt < len(order) or jobs or any(pending.values()):
            now = time.perf_counter() - t0
            while nxt < len(order) and (order[nxt].arrival <= now or not realtime):
                r = order[nxt]
                pending.setdefault((r.graph, r.kind), []).append(r)
                nxt += 1
            for slot in list(jobs):
                reqs, out, edges, ev, nbytes = jobs[slot]
                if not ev.query():
                    continue
                self.used -= nbytes
                job_keys.pop(slot, None)
                done = time.perf_counter() - t0
                e = edges.cpu().tolist()
                # copies are made on the job's stream: its output memory goes back to
                # that stream's pool and is reused by the stream's next job
                with torch.cuda.stream(self.streams[slot]):
                    for i, r in enumerate(reqs):
                        r.done = done
                        r.edges = int(e[i])
                        if self.keep:
                            r.result = out[i].clone()
                del jobs[slot]
            while True:
                if any(k in self.exclusive for k in job_keys.values()):
                    break                             # an exclusive traversal runs alone
                busy = {name for name, hs in self.handles.items()
                        if all((name, i) in jobs for i in range(len(hs)))}
                plan = plan_job(pending, self.sssp_multi_min, busy=busy, thresholds=self.thresholds)
                if plan is None:
                    break
                key, reqs, multi = plan
                if key in self.exclusive and jobs:
                    break                             # waits until the GPU is free
                slot = next((key[0], i) for i in range(len(self.handles[key[0]])) if (key[0], i) not in jobs)
                g = self.handles[key[0]][slot[1]]
                ws = self.grx.multi_footprint(g, KINDS[key[1]]) if multi else 0
                lanes = plan_lanes(len(reqs), ws, self._lane_bytes(key[0]), self._free_bytes(),
                                   others_running=bool(jobs))
                if lanes == 0:                        # waits for memory from running traversals
                    self.admission_waits += 1
                    break
                if lanes < len(reqs):
                    self.shrunk += 1
                    reqs = reqs[:lanes]
                    multi = multi and lanes > 1
                    ws = ws if multi else 0
                pending[key] = pending[key][len(reqs):]
                others = bool(jobs) or any(v for k, v in pending.items() if v and k != key)
                for r in reqs:
                    r.admitted = now
                nbytes = len(reqs) * self._lane_bytes(key[0])
                self.used += ws + nbytes               # the workspace stays with the handle
                share = self.share[key[0]]
                if key[1] == "sssp" and self.sssp_share:
                    share = max(share, self.sssp_share)
                if key in self.exclusive or key in self.full_grid:
                    others = False                    # the whole grid
                out, edges, ev = self._launch(slot, key, reqs, multi, share if others else 0)
                jobs[slot] = (reqs, out, edges, ev, nbytes)
                job_keys[slot] = key
            if not jobs and nxt < len(order) and realtime:
                wait = order[nxt].arrival - (time.perf_counter() - t0)
                if wait > 2e-4:
                    time.sleep(min(wait - 1e-4, 0.01))
        torch.cuda.synchronize()
        return dict(summarize(requests, time.perf_counter() - t0), admission_waits=self.admission_waits,
                    shrunk=self.shrunk)


def summarize(requests: list[Request], wall: float) -> dict:
    lat = np.array([r.done - r.arrival for r in requests if r.done >= 0])
    edges = sum(r.edges for r in requests)
    first = min(r.arrival for r in requests)
    last = max(r.done for r in requests)
    span = max(last - first, 1e-9)
    return {"queries": len(requests), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "gteps": edges / span / 1e9, "span_s": span, "wall_s": wall}


def run_one_at_a_time(graphs: dict, degrees: dict, requests: list[Request],
                      realtime: bool = True, keep_results: bool = False) -> dict:
    """Baseline: FIFO, one single-source traversal at a time, one stream."""
    import torch

    from . import grx
    order = sorted(requests, key=lambda r: r.arrival)
    t0 = time.perf_counter()
    for r in order:
        if realtime:
            wait = r.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        g = graphs[r.graph]
        r.admitted = time.perf_counter() - t0
        out = grx.bfs(g, r.src) if r.kind == "bfs" else grx.sssp(g, r.src)
        reached = out >= 0 if r.kind == "bfs" else out != -1
        r.edges = int((degrees[r.graph] * reached).sum().item())
        r.done = time.perf_counter() - t0
        if keep_results:
            r.result = out
    torch.cuda.synchronize()
    return summarize(requests, time.perf_counter() - t0)
