// Multi-source BFS: up to 64 sources share one traversal and one edge stream.
//
// Every vertex carries 64-bit lane masks: seen[v] (lanes that have labelled
// v) and cur_L[v] (lanes whose level-L frontier holds v).  Lane b's result
// equals a single-source BFS from srcs[b] (Algorithm 1); the lanes only share
// the reading of the graph.  Levels are direction-optimised on lane counts
// (Sec. 6.1 with FV = the frontier's edge count and BV = (unseen
// vertex-lane pairs) * V / (seen pairs)).
//
//  * Push level (sparse frontier): the frontier queue's edges are cut into
//    equal warp tiles (the degree prefix is stored with every queue slot).
//    For edge (u, v) the lanes cur[u] & ~seen[v] are OR-ed into next[v]; the
//    first warp to touch v lists it (large levels instead mark v in a
//    touched bitmap with reductions only, which warps owning 32-word chunks
//    scan).  A finalize phase turns each touched vertex's next mask into its
//    new lanes, labels them (scattered depth writes: few), and appends the
//    vertex to the next queue.
//  * Pull level (dense frontier): static tiles of equal edge count over the
//    non-isolated vertices (their edge prefix is the CSR offsets).  A block
//    stages a tile's rows, drops the rows whose lanes are all seen, gathers
//    cur[u] over the remaining rows' edges into a per-row OR in shared
//    memory, and finishes the rows that lie inside the tile; a row that
//    crosses tiles ORs its partials into a global accumulator and is
//    finished by a fix-up phase.
//  * Depths found by pull levels are not written per level: the level's new
//    lane masks go to one of MS_HSLOTS history slots, and a flush pass
//    writes them lane-major with coalesced stores (and, at the end, -1 for
//    every pair never reached, so the output needs no initial fill).
//  * cur rotates through three buffers: level L reads cur[L%3] and writes
//    cur[(L+1)%3], only for vertices with new lanes; nothing is cleared.  A
//    stale entry holds lanes that reached the vertex at depth L-3 or less,
//    so every neighbour already has them and they cannot label anything: a
//    pull ANDs the gathered lanes with the row's missing lanes, and a push
//    reads cur only for queue entries, which the previous level wrote.  The
//    queue of a push after a pull comes from the pull's history slot.
//  * A pull tile whose rows have every lane seen stays so: it is flagged and
//    skipped by later pull levels.
//  * One cooperative persistent kernel; levels and their phases are
//    separated by the bounded flag barrier.
#include <cstring>

#include "grx_internal.cuh"

namespace {

constexpr int MS_BLOCK = 256;
constexpr int MS_WARPS = MS_BLOCK / 32;
constexpr int MS_ITEMS = 8;
constexpr int MS_WTILE = 32 * MS_ITEMS;             // push: edges per warp tile
constexpr int MS_PITEMS = 7;
constexpr int MS_PTILE = MS_BLOCK * MS_PITEMS;      // pull: edges per block tile
constexpr int MS_HSLOTS = 6;                        // history slots of pull levels
#ifndef GRX_MS_MIN_BLOCKS
#define GRX_MS_MIN_BLOCKS 3                         // resident blocks per SM (register cap)
#endif

enum { DIR_PUSH = 0, DIR_PULL = 1 };
enum { MOP_COMPACT, MOP_EXPAND, MOP_FINAL, MOP_FLUSH, MOP_PULL, MOP_FIXUP };

template <typename OffT>
struct MsArgs {
    int32_t nv;
    int64_t ne;
    const OffT *ro;
    const int32_t *col;
    const int32_t *active;
    const uint32_t *aoff;
    const int2 *tiles;                // pull tiles: (first active row, rows)
    int64_t ntiles;
    int n;
    unsigned long long lanes;         // active lane mask
    int32_t src[64];
    unsigned long long *seen;
    unsigned long long *next;         // push: lane OR per touched vertex; pull: cross-tile OR
    unsigned long long *cur[3];
    unsigned long long *hist[MS_HSLOTS];
    int32_t *fix;                     // per pull tile: the crossing row it finishes (-1: none)
    uint8_t *sat;                     // per pull tile: every row has all lanes seen
    int32_t *Q[3];
    uint32_t *E[3];
    OffT *R[3];
    int32_t *touched;
    uint32_t *tbits;                  // bitmap push: touched vertices, [ceil(nv/32)]
    int64_t words;
    uint32_t bmp_min_T;               // push levels with at least this many edges use tbits
    int32_t *depth;                   // [n][nv]
    TravCtl *ctl;
    unsigned int *bar_flags;
    DevStats *stats;
    int mode;
    float alpha, beta;
    unsigned long long timeout_ns;
};

struct MsState {
    int L;
    uint8_t dir, switched, back, done, phase;
    uint8_t qin;        // Q_L exists as a queue
    uint8_t compact;    // push level whose queue is first built from cur_L
    uint8_t hslots;     // history slots holding pull levels' masks
    uint8_t flush;      // this pull level starts with a flush (slots full)
    uint8_t bmp;        // push level that marks touched vertices in a bitmap
    int32_t slot_depth[MS_HSLOTS];
    uint32_t q, T;      // |Q_L| and its edge count
    unsigned long long seen_pairs;    // (vertex, lane) pairs labelled so far
};

template <typename OffT>
union MsWarpSmem {
    struct {
        uint32_t qe[MS_WTILE + 2];
        OffT rs[MS_WTILE + 1];
        unsigned long long cm[MS_WTILE + 1];
    };
    uint16_t list[32 * 32];           // bitmap finalize: set bits of a 32-word chunk
};

struct MsPullSmem {
    uint32_t qe[MS_PTILE + 2];
    int32_t vid[MS_PTILE + 1];
    unsigned long long miss[MS_PTILE + 1];
    unsigned long long acc[MS_PTILE + 1];
};

template <typename OffT>
union MsSmem {
    MsWarpSmem<OffT> w[MS_WARPS];
    MsPullSmem p;
};

template <typename T>
__device__ __forceinline__ T pk3(T a, T b, T c, int i) { return i == 0 ? a : (i == 1 ? b : c); }

__device__ __forceinline__ int ms_phases(const MsState &s) {
    return s.dir == DIR_PUSH ? 2 + s.compact : 2 + s.flush;
}

__device__ __forceinline__ int ms_op(const MsState &s) {
    if (s.dir == DIR_PUSH) {
        const int p = (int)s.phase - (int)s.compact;
        return p < 0 ? MOP_COMPACT : (p == 0 ? MOP_EXPAND : MOP_FINAL);
    }
    const int p = (int)s.phase - (int)s.flush;
    return p < 0 ? MOP_FLUSH : (p == 0 ? MOP_PULL : MOP_FIXUP);
}

template <typename OffT>
__device__ __forceinline__ void ms_set_kind(const MsArgs<OffT> &a, MsState &s) {
    s.compact = s.dir == DIR_PUSH && !s.qin;
    s.flush = s.dir == DIR_PULL && s.hslots >= MS_HSLOTS;
    s.bmp = s.dir == DIR_PUSH && s.T >= a.bmp_min_T;
}

// Label the new lanes of v at depth d in the lane-major depth output.
__device__ __forceinline__ void write_depths(int32_t *depth, int32_t nv, int32_t v,
                                             unsigned long long nw, int32_t d) {
    while (nw) {
        const int b = __ffsll((long long)nw) - 1;
        nw &= nw - 1;
        depth[(int64_t)b * nv + v] = d;
    }
}

template <typename OffT>
__device__ MsState ms_next_state(const MsArgs<OffT> &a, const MsState &st, bool stats) {
    MsState ns = st;
    if ((int)st.phase + 1 < ms_phases(st)) {
        ns.phase = st.phase + 1;
        return ns;
    }
    ns.L = st.L + 1;
    ns.phase = 0;
    const unsigned long long pk = ld_relaxed_u64(&a.ctl->qpack[(st.L + 1) & 3]);
    ns.q = (uint32_t)(pk >> 32);
    ns.T = (uint32_t)pk;
    ns.qin = st.dir == DIR_PUSH;
    if (st.dir == DIR_PULL) {
        const int h = st.flush ? 0 : st.hslots;
        ns.slot_depth[h] = st.L + 1;
        ns.hslots = (uint8_t)(h + 1);
    }
    const unsigned long long found = ld_relaxed_u64(&a.ctl->pairs[(st.L + 1) & 3]);
    ns.seen_pairs = st.seen_pairs + found;
    if (stats && blockIdx.x == 0 && st.L < GRX_MAX_LEVELS_STATS) a.stats->discovered[st.L] = found;
    if (ns.q == 0) {
        ns.done = 1;
        return ns;
    }
    if (a.mode == GRX_DIR_PUSH) {
        ns.dir = DIR_PUSH;
    } else if (a.mode == GRX_DIR_PULL) {
        ns.dir = DIR_PULL;
    } else {
        const double V = (double)a.nv;
        const double total = (double)a.n * V;
        const double FV = (double)ns.T;
        const double BV = (total - (double)ns.seen_pairs) * V / (double)ns.seen_pairs;
        if (st.dir == DIR_PUSH && !st.switched && FV > BV * (double)a.alpha) {
            ns.dir = DIR_PULL;
            ns.switched = 1;
        } else if (st.dir == DIR_PULL && FV < BV * (double)a.beta) {
            ns.dir = DIR_PUSH;
            ns.back = 1;
        }
    }
    ms_set_kind(a, ns);
    return ns;
}

// Phase 0: masks empty (history slots, the OR buffer and the touched bitmap
// are kept zero between traversals; after one that did not finish they are
// cleared here).
template <typename OffT>
__device__ void ms_init_fill(const MsArgs<OffT> &a, bool dirty) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = tid; v < a.nv; v += stride) {
        a.seen[v] = 0ull;
        a.cur[0][v] = 0ull;
        a.cur[1][v] = 0ull;
        a.cur[2][v] = 0ull;
        if (dirty) {
            a.next[v] = 0ull;
            for (int s = 0; s < MS_HSLOTS; ++s) a.hist[s][v] = 0ull;
        }
    }
    if (dirty)
        for (int64_t w = tid; w < a.words; w += stride) a.tbits[w] = 0u;
    for (int64_t t = tid; t < a.ntiles; t += stride) a.sat[t] = 0;
}

// Phase 1 (one thread): seed the lanes (depth 0), the first frontier
// (distinct sources with at least one edge) and the counters.
template <typename OffT>
__device__ void ms_seed(const MsArgs<OffT> &a) {
    uint32_t cnt = 0, edges = 0;
    for (int b = 0; b < a.n; ++b) {
        const int32_t v = a.src[b];
        const unsigned long long bit = 1ull << b;
        if (a.seen[v] == 0ull) {
            const OffT rb = a.ro[v];
            const uint32_t deg = (uint32_t)(a.ro[v + 1] - rb);
            if (deg) {
                a.Q[0][cnt] = v;
                a.E[0][cnt] = edges;
                a.R[0][cnt] = rb;
                ++cnt;
                edges += deg;
            }
        }
        a.seen[v] |= bit;
        a.cur[0][v] |= bit;
        a.depth[(int64_t)b * a.nv + v] = 0;
    }
    a.ctl->qpack[0] = ((unsigned long long)cnt << 32) | edges;
    for (int i = 1; i < 4; ++i) a.ctl->qpack[i] = 0ull;
    for (int i = 0; i < 4; ++i) a.ctl->pairs[i] = 0ull;
    a.ctl->ucount[1] = 0u;
    a.ctl->cpack = 0ull;
    a.ctl->ms_grid = gridDim.x;
    a.ctl->ms_done = 0u;
}

// Push, phase 1: lanes of each frontier edge's source go to next[v] of the
// target where not yet seen; the first toucher lists v (or, on large levels,
// marks it in the touched bitmap).
template <typename OffT, bool STATS>
__device__ void ms_push_expand(const MsArgs<OffT> &a, const MsState &st, MsWarpSmem<OffT> &w) {
    const int L = st.L;
    const unsigned int lane = threadIdx.x & 31;
    const int32_t *Qv = pk3(a.Q[0], a.Q[1], a.Q[2], L % 3);
    const uint32_t *Qe = pk3(a.E[0], a.E[1], a.E[2], L % 3);
    const OffT *Qr = pk3(a.R[0], a.R[1], a.R[2], L % 3);
    const unsigned long long *cin = pk3(a.cur[0], a.cur[1], a.cur[2], L % 3);
    unsigned int *tctr = &a.ctl->ucount[(L + 1) & 3];
    const int64_t q = st.q;
    const uint64_t T = st.T;
    const uint64_t ntiles = (T + MS_WTILE - 1) / MS_WTILE;
    const uint64_t nwarps = (uint64_t)gridDim.x * MS_WARPS;
    const uint64_t gw = (uint64_t)blockIdx.x * MS_WARPS + (threadIdx.x >> 5);
    const uint64_t per = (ntiles + nwarps - 1) / nwarps;
    const uint64_t tb0 = gw * per;
    const uint64_t tb1 = min(ntiles, tb0 + per);
    if (tb0 >= tb1) return;
    int64_t i0 = warp_upper_index_cg(Qe, q, (uint32_t)(tb0 * MS_WTILE));
    for (uint64_t tile = tb0; tile < tb1; ++tile) {
        const uint64_t e0 = tile * MS_WTILE;
        const uint32_t e1 = (uint32_t)min(T, e0 + MS_WTILE);
        int n = 0;
        for (;;) {
            const int64_t idx = i0 + n + lane;
            uint32_t qe = 0xffffffffu;
            if (idx < q) qe = __ldcg(Qe + idx);
            const bool in = idx < q && qe < e1;
            if (n + (int)lane <= MS_WTILE + 1) w.qe[n + lane] = qe;
            if (in && n + (int)lane <= MS_WTILE) {
                w.rs[n + lane] = __ldcg(Qr + idx);
                w.cm[n + lane] = __ldcg(cin + __ldcg(Qv + idx)) & a.lanes;
            }
            const int cnt = __popc(__ballot_sync(GRX_FULL_MASK, in));
            n += cnt;
            if (cnt < 32) break;
            if (n > MS_WTILE) {
                if (lane == 0) grx_set_status(a.ctl, GRX_EINVAL);
                n = MS_WTILE;
                break;
            }
        }
        __syncwarp();
        const uint32_t next_start = w.qe[n];
        const uint64_t t0 = e0 + (uint64_t)lane * MS_ITEMS;
        int32_t v[MS_ITEMS];
        unsigned long long m[MS_ITEMS];
#pragma unroll
        for (int k = 0; k < MS_ITEMS; ++k) {
            v[k] = 0;
            m[k] = 0ull;
        }
        if (t0 < e1) {
            int j = upper_index_smem(w.qe, n, (uint32_t)t0);
#pragma unroll
            for (int k = 0; k < MS_ITEMS; ++k) {
                const uint32_t e = (uint32_t)t0 + k;
                if (e < e1) {
                    while (w.qe[j + 1] <= e) ++j;
                    v[k] = __ldg(a.col + w.rs[j] + (OffT)(e - w.qe[j]));
                    m[k] = w.cm[j];
                }
            }
        }
        unsigned long long sv[MS_ITEMS];
#pragma unroll
        for (int k = 0; k < MS_ITEMS; ++k) sv[k] = m[k] ? __ldcg(a.seen + v[k]) : ~0ull;
        if (st.bmp) {
            // reductions only: the touched bitmap lists the targets
#pragma unroll
            for (int k = 0; k < MS_ITEMS; ++k) {
                const unsigned long long mk = m[k] & ~sv[k];
                if (mk) {
                    atomicOr(a.next + v[k], mk);
                    atomicOr(a.tbits + (v[k] >> 5), 1u << (v[k] & 31));
                }
            }
        } else {
            uint32_t tmask = 0;
#pragma unroll
            for (int k = 0; k < MS_ITEMS; ++k) {
                const unsigned long long mk = m[k] & ~sv[k];
                if (mk && atomicOr(a.next + v[k], mk) == 0ull) tmask |= 1u << k;
            }
            warp_append_list_items<MS_ITEMS>(v, tmask, a.touched, tctr);
        }
        i0 = (next_start == e1) ? i0 + n : i0 + n - 1;
        __syncwarp();
    }
}

// A touched vertex v (or -1): its next mask becomes its new lanes (labelled
// here) and, with edges, a slot of the next frontier.  All 32 lanes call.
template <typename OffT>
__device__ __forceinline__ void ms_touched(const MsArgs<OffT> &a, int L, int32_t vv,
                                           unsigned long long *cout, int32_t *Qv_out,
                                           uint32_t *Qe_out, OffT *Qr_out, unsigned long long *ctr,
                                           unsigned long long &found) {
    int32_t v[1] = {vv < 0 ? 0 : vv};
    uint32_t deg[1] = {0};
    OffT rb[1] = {0};
    uint32_t app = 0;
    if (vv >= 0) {
        const unsigned long long nx = __ldcg(a.next + vv);
        a.next[vv] = 0ull;
        const unsigned long long sv = __ldcg(a.seen + vv);
        const unsigned long long nw = nx & ~sv & a.lanes;
        if (nw) {
            a.seen[vv] = sv | nw;
            cout[vv] = nw;
            write_depths(a.depth, a.nv, vv, nw, L + 1);
            found += (unsigned long long)__popcll(nw);
            rb[0] = __ldg(a.ro + vv);
            deg[0] = (uint32_t)(__ldg(a.ro + vv + 1) - rb[0]);
            if (deg[0]) app = 1;
        }
    }
    warp_append_items<1, OffT>(v, deg, rb, app, Qv_out, Qe_out, Qr_out, ctr);
}

// Push, phase 2: the touched vertices (from the list, or from the bitmap by
// warps that own 32-word chunks of it, clearing it) become the next frontier.
template <typename OffT>
__device__ void ms_push_finalize(const MsArgs<OffT> &a, const MsState &st, uint16_t *list) {
    const int L = st.L;
    unsigned long long *cout = pk3(a.cur[0], a.cur[1], a.cur[2], (L + 1) % 3);
    int32_t *Qv_out = pk3(a.Q[0], a.Q[1], a.Q[2], (L + 1) % 3);
    uint32_t *Qe_out = pk3(a.E[0], a.E[1], a.E[2], (L + 1) % 3);
    OffT *Qr_out = pk3(a.R[0], a.R[1], a.R[2], (L + 1) % 3);
    unsigned long long *ctr = &a.ctl->qpack[(L + 1) & 3];
    unsigned long long found = 0;
    if (st.bmp) {
        const unsigned int lane = threadIdx.x & 31;
        const int64_t nsc = (a.words + 31) / 32;
        const int64_t nwarps = (int64_t)gridDim.x * MS_WARPS;
        for (int64_t sc = (int64_t)blockIdx.x * MS_WARPS + (threadIdx.x >> 5); sc < nsc; sc += nwarps) {
            const int64_t wd = sc * 32 + lane;
            const uint32_t bits = wd < a.words ? __ldcg(a.tbits + wd) : 0u;
            if (bits) a.tbits[wd] = 0u;
            const int n = warp_compact_bits(bits, list);
            for (int base = 0; base < n; base += 32) {
                const int i = base + (int)lane;
                ms_touched<OffT>(a, L, i < n ? (int32_t)(sc * 1024 + list[i]) : -1, cout, Qv_out, Qe_out,
                                 Qr_out, ctr, found);
            }
            __syncwarp();
        }
    } else {
        const int64_t count = ld_relaxed_u32(&a.ctl->ucount[(L + 1) & 3]);
        const int64_t span = (count + 31) & ~(int64_t)31;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < span;
             i += (int64_t)gridDim.x * blockDim.x)
            ms_touched<OffT>(a, L, i < count ? __ldcg(a.touched + i) : -1, cout, Qv_out, Qe_out, Qr_out,
                             ctr, found);
    }
    found = warp_sum(found);
    if ((threadIdx.x & 31) == 0 && found) atomicAdd(&a.ctl->pairs[(L + 1) & 3], found);
}

// Push after a pull level: Q_L (vertex, edge prefix, row start) from the
// vertices that got new lanes in level L-1 -- exactly the nonzero entries of
// that level's history slot -- through the compaction counter.
template <typename OffT>
__device__ void ms_compact(const MsArgs<OffT> &a, const MsState &st) {
    const int L = st.L;
    const unsigned long long *cin = a.hist[st.hslots - 1];
    int32_t *Qv = pk3(a.Q[0], a.Q[1], a.Q[2], L % 3);
    uint32_t *Qe = pk3(a.E[0], a.E[1], a.E[2], L % 3);
    OffT *Qr = pk3(a.R[0], a.R[1], a.R[2], L % 3);
    const int64_t span = ((int64_t)a.nv + 31) & ~(int64_t)31;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < span;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v[1] = {(int32_t)i};
        uint32_t deg[1] = {0};
        OffT rb[1] = {0};
        uint32_t app = 0;
        if (i < a.nv && __ldcg(cin + i) != 0ull) {
            rb[0] = __ldg(a.ro + i);
            deg[0] = (uint32_t)(__ldg(a.ro + i + 1) - rb[0]);
            app = deg[0] ? 1u : 0u;
        }
        warp_append_items<1, OffT>(v, deg, rb, app, Qv, Qe, Qr, &a.ctl->cpack);
    }
}

// Per-thread counters of the next frontier found by a pull level.
struct MsCounts {
    unsigned long long q, T, pairs, gathered, rows;
};

// A pull-level row v gets its new lanes nw: seen, the history slot and the
// frontier counters (its depth is written by the next flush).
__device__ __forceinline__ void ms_pull_finish(unsigned long long *seen, unsigned long long *hs,
                                               int32_t v, unsigned long long old_seen,
                                               unsigned long long nw, uint32_t deg, MsCounts &c) {
    seen[v] = old_seen | nw;
    hs[v] = nw;
    c.q += 1;
    c.T += deg;
    c.pairs += (unsigned long long)__popcll(nw);
}

// Pull, phase 1: one block per static tile of the active list's edges.
// ORs each item's lane mask into its row's shared accumulator.  A thread's
// items are consecutive positions with non-decreasing rows, and a warp's
// threads hold consecutive runs of positions, so a row's items within a warp
// sit in consecutive lanes.  A row strictly inside one lane's items is stored
// by that lane alone; rows at lane boundaries are OR-ed across the warp by a
// segmented shuffle scan and added once per warp by the lane where they end
// (a hub row filling a tile costs one shared atomic per warp, not one per
// thread).  All 32 lanes call; valid = the lane's item count (0..MS_PITEMS).
__device__ __forceinline__ void or_runs(unsigned long long *acc, const int (&row)[MS_PITEMS],
                                        const unsigned long long (&g)[MS_PITEMS], int valid) {
    const unsigned int lane = threadIdx.x & 31;
    int fk = -1, lk = -1;          // rows of the lane's first run (when it ends inside the lane) and last run
    unsigned long long fs = 0ull, ls = 0ull;
    if (valid > 0) {
        int cj = row[0];
        unsigned long long part = 0ull;
        bool first = true;
#pragma unroll
        for (int k = 0; k < MS_PITEMS; ++k) {
            if (k < valid) {
                if (row[k] != cj) {
                    if (first) {
                        fk = cj;
                        fs = part;
                        first = false;
                    } else if (part) {
                        acc[cj] = part;           // a row inside this lane's items
                    }
                    part = 0ull;
                    cj = row[k];
                }
                part |= g[k];
            }
        }
        lk = cj;
        ls = part;
    }
    const int pk = __shfl_up_sync(GRX_FULL_MASK, lk, 1);
    const bool prev_same = lane > 0 && pk == lk && lk >= 0;
    unsigned long long m = ls;
    int head = (fk >= 0 || !prev_same) ? 1 : 0;
    // segmented inclusive OR-scan of the last runs (Hillis-Steele with head flags)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long m2 = __shfl_up_sync(GRX_FULL_MASK, m, o);
        const int h2 = __shfl_up_sync(GRX_FULL_MASK, head, o);
        if (lane >= (unsigned)o && !head) {
            m |= m2;
            head |= h2;
        }
    }
    const unsigned long long pm = __shfl_up_sync(GRX_FULL_MASK, m, 1);
    if (fk >= 0) {
        const unsigned long long x = fs | ((lane > 0 && pk == fk) ? pm : 0ull);
        if (x) atomicOr(&acc[fk], x);
    }
    const int nfk = __shfl_down_sync(GRX_FULL_MASK, fk, 1);
    const int nlk = __shfl_down_sync(GRX_FULL_MASK, lk, 1);
    const bool next_cont = lane < 31 && ((nfk >= 0 && nfk == lk) || (nfk < 0 && nlk == lk));
    if (lk >= 0 && !next_cont && m) atomicOr(&acc[lk], m);
}

template <typename OffT, bool STATS>
__device__ void ms_pull(const MsArgs<OffT> &a, const MsState &st, MsPullSmem &p, MsCounts &c) {
    const int L = st.L;
    const unsigned long long *cin = pk3(a.cur[0], a.cur[1], a.cur[2], L % 3);
    unsigned long long *cout = pk3(a.cur[0], a.cur[1], a.cur[2], (L + 1) % 3);
    unsigned long long *hs = a.hist[st.flush ? 0 : st.hslots];
    __shared__ int s_open;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        if (__ldcg(a.sat + tile)) continue;                  // uniform in the block
        const uint64_t e0 = (uint64_t)tile * MS_PTILE;
        const uint64_t e1 = min((uint64_t)a.ne, e0 + MS_PTILE);
        const int len = (int)(e1 - e0);
        const int2 tr = __ldg(a.tiles + tile);
        const int64_t i0 = tr.x;
        const int n = tr.y;
        for (int j = threadIdx.x; j <= n; j += MS_BLOCK) {   // n+1 prefixes: qe[n] = end of last row
            p.qe[j] = __ldg(a.aoff + i0 + j);
            if (j < n) {
                const int32_t v = __ldg(a.active + i0 + j);
                p.vid[j] = v;
                p.miss[j] = a.lanes & ~__ldcg(a.seen + v);
                p.acc[j] = 0ull;
            }
        }
        if (threadIdx.x == 0) {
            a.fix[tile] = -1;
            s_open = 0;
            if (STATS) c.rows += (unsigned long long)n;
        }
        __syncthreads();
        // a run of MS_PITEMS consecutive edges per thread: rows first, then
        // every column and every gather in flight together; rows with every
        // lane seen gather nothing
        const int t0 = threadIdx.x * MS_PITEMS;
        int rj[MS_PITEMS];
        unsigned long long gv[MS_PITEMS];
#pragma unroll
        for (int k = 0; k < MS_PITEMS; ++k) {
            rj[k] = 0;
            gv[k] = 0ull;
        }
        if (t0 < len) {
            int j = upper_index_smem(p.qe, n, (uint32_t)(e0 + t0));
#pragma unroll
            for (int k = 0; k < MS_PITEMS; ++k) {
                const uint32_t e = (uint32_t)(e0 + t0 + k);
                if (t0 + k < len)
                    while (p.qe[j + 1] <= e) ++j;
                rj[k] = j;
            }
            int32_t u[MS_PITEMS];
#pragma unroll
            for (int k = 0; k < MS_PITEMS; ++k)
                u[k] = (t0 + k < len && p.miss[rj[k]]) ? __ldg(a.col + e0 + t0 + k) : -1;
#pragma unroll
            for (int k = 0; k < MS_PITEMS; ++k) gv[k] = u[k] >= 0 ? __ldca(cin + u[k]) : 0ull;
            if (STATS) {
#pragma unroll
                for (int k = 0; k < MS_PITEMS; ++k) c.gathered += u[k] >= 0 ? 1ull : 0ull;
            }
        }
        or_runs(p.acc, rj, gv, t0 < len ? min(MS_PITEMS, len - t0) : 0);
        __syncthreads();
        int open = 0;
        for (int j = threadIdx.x; j < n; j += MS_BLOCK) {
            const int32_t v = p.vid[j];
            const uint32_t start = p.qe[j], end = p.qe[j + 1];
            const unsigned long long nw = p.acc[j] & p.miss[j];
            if (p.miss[j] & ~nw) open = 1;                    // lanes still missing after this level
            if (start >= e0 && end <= e1) {
                if (nw) {
                    cout[v] = nw;
                    ms_pull_finish(a.seen, hs, v, a.lanes & ~p.miss[j], nw, end - start, c);
                }
            } else {
                if (nw) atomicOr(a.next + v, nw);
                if (end <= e1) a.fix[tile] = v;               // this tile holds the row's last edge
            }
        }
        if (open) s_open = 1;
        __syncthreads();
        // a crossing row's lanes from other tiles are not known here: the flag
        // may stay clear one level longer than needed, never the other way
        if (threadIdx.x == 0 && !s_open) a.sat[tile] = 1;
    }
}

// Pull, phase 2: rows that cross tiles, finished by the tile holding their
// last edge.
template <typename OffT>
__device__ void ms_pull_fixup(const MsArgs<OffT> &a, const MsState &st, MsCounts &c) {
    const int L = st.L;
    unsigned long long *cout = pk3(a.cur[0], a.cur[1], a.cur[2], (L + 1) % 3);
    unsigned long long *hs = a.hist[st.flush ? 0 : st.hslots];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.ntiles;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = __ldcg(a.fix + t);
        if (v < 0) continue;
        const unsigned long long acc = __ldcg(a.next + v);
        if (acc) a.next[v] = 0ull;
        const unsigned long long sv = __ldcg(a.seen + v);
        const unsigned long long nw = acc & a.lanes & ~sv;
        if (nw) {
            cout[v] = nw;
            ms_pull_finish(a.seen, hs, v, sv, nw, (uint32_t)(__ldg(a.ro + v + 1) - __ldg(a.ro + v)), c);
        }
    }
}

// Depths of the pull levels held in the first nslots history slots, written
// lane-major (for each lane, consecutive threads write consecutive vertices);
// the slots are cleared.  The final flush also writes -1 for every pair that
// was never reached.  Masks are split into 32-bit halves so the per-lane
// tests are single-word operations.
template <typename OffT>
__device__ void ms_flush(const MsArgs<OffT> &a, int nslots, const int32_t *slot_depth, bool final) {
    int32_t sd[MS_HSLOTS];
#pragma unroll
    for (int s = 0; s < MS_HSLOTS; ++s) sd[s] = s < nslots ? slot_depth[s] : 0;
    const int nlo = min(a.n, 32);
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < a.nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        uint32_t hl[MS_HSLOTS], hh[MS_HSLOTS];
        unsigned long long any = 0ull;
#pragma unroll
        for (int s = 0; s < MS_HSLOTS; ++s) {
            const unsigned long long h = s < nslots ? __ldcg(a.hist[s] + v) : 0ull;
            if (h) a.hist[s][v] = 0ull;
            hl[s] = (uint32_t)h;
            hh[s] = (uint32_t)(h >> 32);
            any |= h;
        }
        const unsigned long long unseen = final ? (a.lanes & ~__ldcg(a.seen + v)) : 0ull;
        if (!(any | unseen)) continue;
        int32_t *out = a.depth + v;
        if (!any && unseen == a.lanes) {             // reached by no lane
            for (int b = 0; b < a.n; ++b) out[(int64_t)b * a.nv] = -1;
            continue;
        }
        const uint32_t ul = (uint32_t)unseen, uh = (uint32_t)(unseen >> 32);
        for (int b = 0; b < nlo; ++b) {
            int d = (ul >> b & 1u) ? -1 : -2;
#pragma unroll
            for (int s = 0; s < MS_HSLOTS; ++s) d = (hl[s] >> b & 1u) ? sd[s] : d;
            if (d != -2) out[(int64_t)b * a.nv] = d;
        }
        for (int b = 32; b < a.n; ++b) {
            int d = (uh >> (b - 32) & 1u) ? -1 : -2;
#pragma unroll
            for (int s = 0; s < MS_HSLOTS; ++s) d = (hh[s] >> (b - 32) & 1u) ? sd[s] : d;
            if (d != -2) out[(int64_t)b * a.nv] = d;
        }
    }
}

template <typename OffT, bool STATS>
__global__ void __launch_bounds__(MS_BLOCK, GRX_MS_MIN_BLOCKS) k_msbfs_persistent(MsArgs<OffT> a) {
    __shared__ MsState s_st;
    __shared__ int s_dirty;
    __shared__ MsSmem<OffT> sm;
    FlagBarrier bar{a.bar_flags, &a.ctl->bar_release, a.ctl, a.timeout_ns, 0u};
    if (threadIdx.x == 0) {
        // the previous traversal left the history slots and the OR buffer
        // zero only if every one of its blocks finished its final pass
        const unsigned int g = ld_relaxed_u32(&a.ctl->ms_grid);
        s_dirty = !(g > 0 && ld_relaxed_u32(&a.ctl->ms_done) == g);
    }
    __syncthreads();
    ms_init_fill(a, s_dirty != 0);
    if (!flag_barrier(bar)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ms_seed(a);
    if (!flag_barrier(bar)) return;
    if (threadIdx.x == 0) {
        MsState s;
        memset(&s, 0, sizeof s);
        const unsigned long long pk = ld_relaxed_u64(&a.ctl->qpack[0]);
        s.dir = a.mode == GRX_DIR_PULL ? DIR_PULL : DIR_PUSH;
        s.switched = a.mode == GRX_DIR_PULL;
        s.q = (uint32_t)(pk >> 32);
        s.T = (uint32_t)pk;
        s.qin = 1;
        s.seen_pairs = (unsigned long long)a.n;
        s.done = s.q == 0;
        ms_set_kind(a, s);
        s_st = s;
    }
    __syncthreads();
    for (;;) {
        const MsState st = s_st;
        if (st.done) break;
        const int L = st.L;
        const int op = ms_op(st);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if ((int)st.phase + 1 == ms_phases(st)) a.ctl->cpack = 0ull;   // used by first phases only
            if (st.phase == 0) {
                a.ctl->qpack[(L + 2) & 3] = 0ull;
                a.ctl->ucount[(L + 2) & 3] = 0u;
                a.ctl->pairs[(L + 2) & 3] = 0ull;
                if (STATS && L < GRX_MAX_LEVELS_STATS) {
                    a.stats->level_t0[L] = grx_globaltimer();
                    a.stats->dir[L] = st.dir;
                    a.stats->frontier[L] = st.q;
                    a.stats->levels = L + 1;
                    if (st.dir == DIR_PUSH) {
                        a.stats->edges_examined[L] = st.T;
                        a.stats->vertices_scanned[L] = st.q;
                    }
                }
            }
        }
        if (op == MOP_COMPACT) {
            ms_compact<OffT>(a, st);
        } else if (op == MOP_EXPAND) {
            ms_push_expand<OffT, STATS>(a, st, sm.w[threadIdx.x >> 5]);
        } else if (op == MOP_FINAL) {
            ms_push_finalize<OffT>(a, st, sm.w[threadIdx.x >> 5].list);
        } else if (op == MOP_FLUSH) {
            ms_flush<OffT>(a, MS_HSLOTS, st.slot_depth, false);
        } else {
            MsCounts c = {0ull, 0ull, 0ull, 0ull, 0ull};
            if (op == MOP_PULL) ms_pull<OffT, STATS>(a, st, sm.p, c);
            else ms_pull_fixup<OffT>(a, st, c);
            c.q = warp_sum(c.q);
            c.T = warp_sum(c.T);
            c.pairs = warp_sum(c.pairs);
            if (STATS) {
                c.gathered = warp_sum(c.gathered);
                c.rows = warp_sum(c.rows);
            }
            if ((threadIdx.x & 31) == 0) {
                if (c.q) atomicAdd(&a.ctl->qpack[(L + 1) & 3], (c.q << 32) | c.T);
                if (c.pairs) atomicAdd(&a.ctl->pairs[(L + 1) & 3], c.pairs);
                if (STATS && c.gathered && L < GRX_MAX_LEVELS_STATS)
                    atomicAdd(&a.stats->edges_examined[L], c.gathered);
                if (STATS && c.rows && L < GRX_MAX_LEVELS_STATS)
                    atomicAdd(&a.stats->vertices_scanned[L], c.rows);   // rows of the tiles not skipped
            }
        }
        if (!flag_barrier(bar)) return;
        if (threadIdx.x == 0) s_st = ms_next_state(a, st, STATS);
        __syncthreads();
    }
    // depths of the pull levels still in the history slots, -1 for the rest
    ms_flush<OffT>(a, s_st.hslots, s_st.slot_depth, true);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&a.ctl->ms_done, 1u);
        if (blockIdx.x == 0) {
            a.ctl->levels_run = s_st.L;
            if (STATS && s_st.L <= GRX_MAX_LEVELS_STATS) a.stats->level_t0[s_st.L] = grx_globaltimer();
        }
    }
}

template <typename OffT, bool STATS>
grx_status ms_launch_typed(grx_graph *g, const int32_t *srcs, int n, int32_t *depth,
                           const grx_opts *o, cudaStream_t s) {
    MsArgs<OffT> a;
    a.nv = g->nv;
    a.ne = g->ne;
    a.ro = (const OffT *)g->ro;
    a.col = g->col;
    a.active = g->active;
    a.aoff = g->aoff;
    a.ntiles = (g->ne + MS_PTILE - 1) / MS_PTILE;
    a.tiles = nullptr;
    if (a.ntiles > 0) {
        grx_status st = grx_edge_tiles(g, MS_PTILE, s, &a.tiles);
        if (st != GRX_OK) return st;
    }
    if (!g->ms_fix) {
        g->ms_sat = (uint8_t *)grx_alloc(g, (size_t)(a.ntiles > 0 ? a.ntiles : 1), s);
        g->ms_fix = g->ms_sat ? (int32_t *)grx_alloc(g, (size_t)(a.ntiles > 0 ? a.ntiles : 1) * 4, s) : nullptr;
        for (int i = 0; i < MS_HSLOTS && g->ms_fix; ++i) {
            g->ms_hist[i] = (unsigned long long *)grx_alloc(g, (size_t)g->nv * 8, s);
            if (!g->ms_hist[i]) return grx_fail(GRX_ENOMEM, "bfs_multi: history slot allocation failed");
        }
        if (!g->ms_fix) return grx_fail(GRX_ENOMEM, "bfs_multi: workspace allocation failed");
    }
    a.fix = g->ms_fix;
    a.sat = g->ms_sat;
    for (int i = 0; i < MS_HSLOTS; ++i) a.hist[i] = g->ms_hist[i];
    a.n = n;
    a.lanes = n == 64 ? ~0ull : ((1ull << n) - 1ull);
    for (int i = 0; i < 64; ++i) a.src[i] = i < n ? srcs[i] : 0;
    a.seen = g->ms_seen;
    a.next = g->ms_next;
    for (int i = 0; i < 3; ++i) {
        a.cur[i] = g->ms_cur[i];
        a.Q[i] = g->qv[i];
        a.E[i] = g->qe[i];
        a.R[i] = (OffT *)g->qr[i];
    }
    a.touched = g->ulist[0];
    if (!g->ms_tbits) {
        g->ms_tbits = (uint32_t *)grx_alloc(g, (size_t)g->words * 4 + 16, s);
        if (!g->ms_tbits) return grx_fail(GRX_ENOMEM, "bfs_multi: touched bitmap allocation failed");
        GRX_CUDA(cudaMemsetAsync(g->ms_tbits, 0, (size_t)g->words * 4 + 16, s));
    }
    a.tbits = g->ms_tbits;
    a.words = g->words;
    {   // bitmap push when a level's edges reach push_bitmap * nv (0 = 1/8, < 0 = never)
        const double pb = o->push_bitmap == 0.f ? 0.125 : (double)o->push_bitmap;
        const double t = pb * (double)g->nv;
        a.bmp_min_T = pb < 0 ? 0xffffffffu : (t < 1.0 ? 1u : (t > 4294967295.0 ? 0xffffffffu : (uint32_t)t));
    }
    a.depth = depth;
    a.ctl = g->ctl;
    a.bar_flags = g->bar_flags;
    a.stats = g->stats;
    a.mode = o->direction;
    a.alpha = o->alpha;
    a.beta = o->beta;
    a.timeout_ns = grx_timeout_ns(o);
    static int per_sm = -1;
    if (per_sm < 0) {
        GRX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_msbfs_persistent<OffT, STATS>,
                                                               MS_BLOCK, 0));
        if (per_sm < 1) return grx_fail(GRX_ECUDA, "bfs_multi: persistent kernel does not fit on an SM");
    }
    int max_grid = per_sm * g->ctx->num_sms;
    if (max_grid > GRX_MAX_GRID) max_grid = GRX_MAX_GRID;
    int blocks = o->grid_blocks > 0 && o->grid_blocks < max_grid ? o->grid_blocks : max_grid;
    GRX_CUDA(cudaMemsetAsync(g->bar_flags, 0, sizeof(unsigned int) * (size_t)blocks, s));
    GRX_CUDA(cudaMemsetAsync(&g->ctl->bar_release, 0, sizeof(unsigned int), s));
    if (o->collect_stats) GRX_CUDA(cudaMemsetAsync(g->stats, 0, sizeof(DevStats), s));
    void *args[] = {(void *)&a};
    if (o->ev_begin) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_begin, s));
    GRX_CUDA(cudaLaunchCooperativeKernel((const void *)k_msbfs_persistent<OffT, STATS>, dim3(blocks),
                                         dim3(MS_BLOCK), args, 0, s));
    if (o->ev_end) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_end, s));
    return GRX_OK;
}

}  // namespace

size_t grx_msbfs_new_bytes(const grx_graph *g) {
    size_t b = 0;
    const int64_t ntiles = (g->ne + MS_PTILE - 1) / MS_PTILE;
    const size_t nt = (size_t)(ntiles > 0 ? ntiles : 1);
    bool have_tiles = false;
    for (int i = 0; i < (int)(sizeof g->etiles / sizeof g->etiles[0]); ++i)
        if (g->etiles[i] && g->etile_size[i] == MS_PTILE) have_tiles = true;
    if (ntiles > 0 && !have_tiles) b += nt * sizeof(int2);
    if (!g->ms_fix) b += nt + nt * 4 + (size_t)MS_HSLOTS * (size_t)g->nv * 8;
    if (!g->ms_tbits) b += (size_t)g->words * 4 + 16;
    return b;
}

grx_status grx_msbfs_launch(grx_graph *g, const int32_t *srcs, int n, int32_t *depth,
                            const grx_opts *o, cudaStream_t s) {
    if (g->off64)
        return o->collect_stats ? ms_launch_typed<int64_t, true>(g, srcs, n, depth, o, s)
                                : ms_launch_typed<int64_t, false>(g, srcs, n, depth, o, s);
    return o->collect_stats ? ms_launch_typed<int32_t, true>(g, srcs, n, depth, o, s)
                            : ms_launch_typed<int32_t, false>(g, srcs, n, depth, o, s);
}
