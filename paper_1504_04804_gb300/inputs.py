"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 7).

This module generates graphs, edge weights and source vertices.  It holds none
of the traversal arithmetic: it is the one module that both the CPU oracle's
tests and the CUDA path take their inputs from.

* R-MAT (Sec. 7: "a GPU-based R-MAT generator faithful to GTgraph",
  {A,B,C,D} = {0.57,0.19,0.19,0.05}): ``ef * 2**scale`` undirected edges are
  drawn; each picks one quadrant per bit level, most significant bit first.
  No noise and no vertex relabelling.
* Grid: a ``w x h`` 4-neighbour lattice with every undirected edge deleted
  independently with probability ``p_del`` (stand-in for the road networks the
  paper calls overhead-bound, Sec. 5.2 and 7).
* Every graph is made undirected, self-loops and duplicates removed (Sec. 7),
  and stored as a CSR with rows sorted ascending.
* Weights: integer, symmetric per undirected edge, uniform in ``[1, wmax]``.
* Sources: distinct non-isolated vertices by seeded rejection sampling.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast Splittable
Pseudorandom Number Generators", OOPSLA 2014), used counter-style: draw ``n``
of stream ``seed`` is ``mix64(seed + (n + 1) * 0x9E3779B97F4A7C15)``.  The CUDA
library carries a twin of the edge and weight generators for large scales;
the tests check the two bit-for-bit.
"""
from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction

import numpy as np

GOLDEN_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB

RMAT_ABCD = ("0.57", "0.19", "0.19", "0.05")


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(_M1)
        z ^= z >> np.uint64(27)
        z *= np.uint64(_M2)
        z ^= z >> np.uint64(31)
    return z


def draw(seed: int, counters: np.ndarray) -> np.ndarray:
    """Counter-based SplitMix64: element ``n`` of the stream seeded with ``seed``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * np.uint64(GOLDEN_GAMMA)
    return mix64(state)


def rmat_thresholds(abcd=RMAT_ABCD):
    """Integer thresholds on the top 53 bits of a draw: r < t0 picks quadrant A,
    r < t1 picks B, r < t2 picks C, else D.  Exact (rational) so every twin agrees."""
    a, b, c, d = (Fraction(x) for x in abcd)
    if a + b + c + d != 1:
        raise ValueError("R-MAT probabilities must sum to 1")
    s = 1 << 53
    return (int(a * s), int((a + b) * s), int((a + b + c) * s))


def rmat_edges(scale: int, edge_factor: int, seed: int, abcd=RMAT_ABCD,
               chunk: int = 1 << 22):
    """Directed R-MAT edge list (u, v) as int32 arrays, before symmetrisation.

    Edge ``i`` uses draws ``i*scale + l`` for bit levels ``l = 0..scale-1``;
    level ``l`` sets bit ``scale-1-l`` of u (rows) and v (columns)."""
    if not (1 <= scale <= 30):
        raise ValueError("scale must be in [1, 30]")
    m = edge_factor << scale
    t0, t1, t2 = (np.uint64(t) for t in rmat_thresholds(abcd))
    us = np.empty(m, dtype=np.int32)
    vs = np.empty(m, dtype=np.int32)
    for lo in range(0, m, chunk):
        hi = min(m, lo + chunk)
        i = np.arange(lo, hi, dtype=np.uint64)
        u = np.zeros(hi - lo, dtype=np.uint64)
        v = np.zeros(hi - lo, dtype=np.uint64)
        base = i * np.uint64(scale)
        for level in range(scale):
            r = draw(seed, base + np.uint64(level)) >> np.uint64(11)
            bu = (r >= t1).astype(np.uint64)                    # C or D: lower half
            bv = ((r >= t0) & (r < t1)) | (r >= t2)              # B or D: right half
            shift = np.uint64(scale - 1 - level)
            u |= bu << shift
            v |= bv.astype(np.uint64) << shift
        us[lo:hi] = u.astype(np.int32)
        vs[lo:hi] = v.astype(np.int32)
    return us, vs


def grid_edges(width: int, height: int, p_del: float, seed: int):
    """Undirected 4-neighbour lattice edges (u, v) with each edge kept with
    probability 1 - p_del.  Vertex (x, y) has id y*width + x.  Horizontal edge
    (x,y)-(x+1,y) has edge id y*(width-1)+x; vertical edge (x,y)-(x,y+1) has id
    height*(width-1) + y*width + x.  An edge is deleted when the top 53 bits of
    draw(seed, edge id) fall below p_del * 2**53."""
    t = np.uint64(int(Fraction(str(p_del)) * (1 << 53)))
    xs, ys = np.meshgrid(np.arange(width - 1, dtype=np.int64),
                         np.arange(height, dtype=np.int64))
    h_id = (ys * (width - 1) + xs).ravel()
    h_u = (ys * width + xs).ravel()
    h_v = h_u + 1
    xs, ys = np.meshgrid(np.arange(width, dtype=np.int64),
                         np.arange(height - 1, dtype=np.int64))
    v_id = (height * (width - 1) + ys * width + xs).ravel()
    v_u = (ys * width + xs).ravel()
    v_v = v_u + width
    eid = np.concatenate([h_id, v_id]).astype(np.uint64)
    u = np.concatenate([h_u, v_u])
    v = np.concatenate([h_v, v_v])
    keep = (draw(seed, eid) >> np.uint64(11)) >= t
    return u[keep].astype(np.int32), v[keep].astype(np.int32)


def build_csr(nv: int, u: np.ndarray, v: np.ndarray):
    """Symmetrise, drop self-loops and duplicate edges, and return
    (row_offsets int64[nv+1], col_indices int32[ne]) with rows sorted."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    keys = np.concatenate([u * nv + v, v * nv + u])
    keys = np.unique(keys)
    rows = keys // nv
    col = (keys % nv).astype(np.int32)
    counts = np.bincount(rows, minlength=nv)
    ro = np.zeros(nv + 1, dtype=np.int64)
    np.cumsum(counts, out=ro[1:])
    return ro, col


def edge_weights(row_offsets: np.ndarray, col_indices: np.ndarray, wmax: int,
                 seed: int) -> np.ndarray:
    """uint32 weight per CSR entry, uniform in [1, wmax] and equal for (u,v) and
    (v,u): 1 + draw(seed, min(u,v)*nv + max(u,v)) mod wmax."""
    ro = np.asarray(row_offsets, dtype=np.int64)
    nv = ro.shape[0] - 1
    rows = np.repeat(np.arange(nv, dtype=np.int64), np.diff(ro))
    col = np.asarray(col_indices, dtype=np.int64)
    lo = np.minimum(rows, col).astype(np.uint64)
    hi = np.maximum(rows, col).astype(np.uint64)
    r = draw(seed, lo * np.uint64(nv) + hi)
    return (np.uint64(1) + r % np.uint64(wmax)).astype(np.uint32)


def pick_sources(row_offsets: np.ndarray, count: int, seed: int) -> np.ndarray:
    """``count`` distinct non-isolated vertices: candidate k is
    draw(seed, k) mod nv, accepted if its degree is > 0 and not yet taken."""
    ro = np.asarray(row_offsets, dtype=np.int64)
    nv = ro.shape[0] - 1
    deg = np.diff(ro)
    n_ok = int(np.count_nonzero(deg))
    if count > n_ok:
        raise ValueError("not enough non-isolated vertices")
    out, seen, k = [], set(), 0
    while len(out) < count:
        batch = draw(seed, np.arange(k, k + 1024, dtype=np.uint64)) % np.uint64(nv)
        for c in batch.astype(np.int64):
            if deg[c] > 0 and c not in seen:
                seen.add(int(c))
                out.append(int(c))
                if len(out) == count:
                    break
        k += 1024
    return np.asarray(out, dtype=np.int32)


@dataclass
class Graph:
    """A host-side CSR graph with optional symmetric weights."""
    name: str
    row_offsets: np.ndarray      # int64 [nv+1]
    col_indices: np.ndarray      # int32 [ne]
    weights: np.ndarray | None = None

    @property
    def nv(self) -> int:
        return self.row_offsets.shape[0] - 1

    @property
    def ne(self) -> int:
        return int(self.row_offsets[-1])


def rmat_graph(scale: int, edge_factor: int = 16, seed: int | None = None,
               wmax: int | None = None, weight_seed: int | None = None) -> Graph:
    """R-MAT graph of the paper's kind (Sec. 7), optionally weighted."""
    seed = scale if seed is None else seed
    u, v = rmat_edges(scale, edge_factor, seed)
    ro, col = build_csr(1 << scale, u, v)
    w = None
    if wmax is not None:
        w = edge_weights(ro, col, wmax, 100 + seed if weight_seed is None else weight_seed)
    return Graph(f"rmat_s{scale}_ef{edge_factor}", ro, col, w)


def grid_graph(width: int, height: int, p_del: float = 0.1, seed: int | None = None,
               wmax: int | None = None, weight_seed: int | None = None) -> Graph:
    seed = width if seed is None else seed
    u, v = grid_edges(width, height, p_del, seed)
    ro, col = build_csr(width * height, u, v)
    w = None
    if wmax is not None:
        w = edge_weights(ro, col, wmax, 100 + seed if weight_seed is None else weight_seed)
    return Graph(f"grid_{width}x{height}", ro, col, w)


def csr_from_edges(nv: int, edges, name: str = "edges", weights=None) -> Graph:
    """Small helper for tests: an undirected CSR from a list of (u, v) pairs."""
    if len(edges):
        e = np.asarray(edges, dtype=np.int64)
        ro, col = build_csr(nv, e[:, 0], e[:, 1])
    else:
        ro, col = np.zeros(nv + 1, dtype=np.int64), np.zeros(0, dtype=np.int32)
    return Graph(name, ro, col, weights)


def reached_edges(row_offsets: np.ndarray, reached_mask: np.ndarray) -> int:
    """TEPS numerator: the sum of degrees over the vertices a traversal reached
    (the directed CSR edges inside the source's component)."""
    deg = np.diff(np.asarray(row_offsets, dtype=np.int64))
    return int(deg[np.asarray(reached_mask, dtype=bool)].sum())
