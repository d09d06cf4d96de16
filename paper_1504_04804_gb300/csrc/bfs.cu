// BFS and direction-optimising BFS (Algorithms 1 and 2, Sec. 6.1).
//
// Design (one GPU, GB300):
//  * The whole traversal, including the initialisation of the outputs and
//    bitmaps, is one cooperative persistent kernel.  Levels (and the phases
//    of a level) are separated by a flag-based grid barrier with bounded
//    waits, so no host round trip or launch happens per level (the
//    per-iteration overhead l of Sec. 5.2).  A host-stepped variant (one
//    launch per phase) and a CUDA-graph variant exist for comparison.
//  * Work inside a phase is warp-independent: no block-wide barrier, so a
//    warp waiting on memory never holds up its neighbours.
//  * Frontiers: the queue Q_L (vertex, row start, exclusive prefix of the
//    frontier's degrees) feeds push levels; the bitmap F_L feeds pull levels.
//    Three of each rotate (slot L % 3).
//  * Push with a small frontier (queue push): advance and filter are fused
//    (Sec. 6.3).  The frontier's edges are cut into equal warp tiles (the
//    degree prefix needs no scan pass); each lane takes PUSH_ITEMS edges of
//    the tile, item k at position k*32 + lane, so each of the warp's column
//    loads reads one contiguous run, and keeps their loads, bitmap probes and
//    atomics in flight together.  The visited bitmap is the filter (test, then
//    atomicOr; the winner labels the vertex and appends it with one
//    warp-aggregated atomic).
//  * Push with a large frontier (bitmap push, 2 phases): the same tiles mark
//    every unvisited target in visited and F_{L+1} with fire-and-forget
//    atomic ORs (no returned value on the path); then warps that own 32-word
//    chunks of F_{L+1} label the marked vertices and append them to Q_{L+1}
//    in vertex order.  Per-edge atomics with a return value and the
//    contended append counter leave the hot loop.
//  * Pull (bottom-up, Sec. 6.1): warps own 32-word chunks of the bitmaps.
//    The unvisited non-isolated vertices of a chunk are compacted in shared
//    memory; each lane takes PULL_PER_LANE of them and probes their first
//    PULL_LIGHT neighbours against F_L at once; the lists with no hit yet
//    are consumed together in load-balanced warp steps, each list leaving at
//    its first step with a hit (edge skipping).  The chunk's owner writes its
//    visited and F_{L+1} words whole: no atomics on labels, bitmaps or
//    queues; only one counter update per warp per level.
//  * Bitmap words that are read-only in a phase (F_L during a pull) or only
//    filter (visited during a push: a stale 0 costs one redundant atomic,
//    never a wrong label) are read through L1: the words of high-degree
//    vertices are probed by most edges of a large level.  Bits written before
//    the last grid barrier are always seen (acquire at the barrier).
//  * A push level after pull levels first compacts F_L into Q_L (a phase).
//  * Direction switch (Sec. 6.1): FV = |Q|*E/V, BV = |U|*V/|P|; push->pull
//    once when FV > BV*alpha, pull->push when FV < BV*beta.  With
//    exact_fv = 1, FV is the frontier's exact edge count, which the level's
//    counter provides.  Every block evaluates the rule identically.
#include <cstdio>
#include <cstring>

#include "grx_internal.cuh"

namespace {

#ifndef GRX_PUSH_ITEMS
#define GRX_PUSH_ITEMS 8
#endif
#ifndef GRX_PUSH_DEDUP
#define GRX_PUSH_DEDUP 1
#endif

constexpr int BFS_BLOCK = 256;
#ifndef GRX_BFS_MIN_BLOCKS
#define GRX_BFS_MIN_BLOCKS 3                        // resident blocks per SM (register cap)
#endif
constexpr int WARPS = BFS_BLOCK / 32;
constexpr int PUSH_ITEMS = GRX_PUSH_ITEMS;
constexpr int WTILE = 32 * PUSH_ITEMS;              // edges per warp tile
constexpr int PULL_LIGHT = 2;                       // neighbours probed per vertex first
#ifndef GRX_PULL_PER_LANE
#define GRX_PULL_PER_LANE 4
#endif
constexpr int PULL_PER_LANE = GRX_PULL_PER_LANE;    // candidates per lane per round
constexpr int PULL_WCH = 32 * PULL_PER_LANE;        // candidates per warp round
constexpr int PULL_HITEMS = PUSH_ITEMS;             // heavy-phase edges per lane per step
constexpr int PULL_HSTEP = 32 * PULL_HITEMS;        // heavy-phase edges per warp step
constexpr int SC_VERTS = 32 * 32;                   // vertices of a 32-word chunk
static_assert(WTILE == 256 && PULL_HSTEP == 256, "warp_tile_rows8 covers 256-position tiles");

enum { DIR_PUSH = 0, DIR_PULL = 1 };
enum { OP_QPUSH, OP_BMARK, OP_BFINAL, OP_COMPACT, OP_PULL, OP_PULL_LIST };

struct LevelState {
    int L;              // level being expanded (frontier = vertices at depth L)
    uint8_t dir;
    uint8_t switched;   // push->pull has happened
    uint8_t back;       // pull->push has happened (final)
    uint8_t done;
    uint8_t fwrite;     // this level leaves bits in F_{L+1}
    uint8_t fprev;      // F_L may hold bits
    uint8_t fclear;     // F_{L-1} may hold bits: this level zeroes it
    uint8_t qin;        // Q_L exists as a queue
    uint8_t qprev_ok;   // Q_{L-1} exists as a queue
    uint8_t bmp;        // push by bitmap marking + finalize phase
    uint8_t compact;    // push whose frontier is first compacted F_L -> Q_L
    uint8_t phase;      // phase of the level being run
    uint8_t uin;        // U_L (candidates left unfound by a pull level L-1) exists
    uint8_t lmode;      // pull over the list U_L instead of a sweep of all chunks
    uint8_t uwrite;     // this pull level writes U_{L+1}
    uint32_t seq;       // phases run so far in this traversal (chunk-counter ring index)
    uint32_t ucnt;      // |U_L|
    uint32_t q, T;      // |Q_L| and its edge count
    uint32_t nprev;     // |Q_{L-1}|
    unsigned long long vcount;   // visited vertices including Q_L
};

template <typename OffT>
struct BfsArgs {
    int32_t nv;
    int64_t ne;
    int64_t words;
    const OffT *ro;
    const int32_t *col;
    const uint32_t *nz;
    uint32_t *visited;
    uint32_t *F[3];
    int32_t *Q[3];
    uint32_t *E[3];
    OffT *R[3];
    int32_t *depth;
    int32_t *parent;
    TravCtl *ctl;
    unsigned int *bar_flags;
    DevStats *stats;
    int mode;
    int exact_fv;
    float alpha, beta;
    int32_t *U[2];                // candidate lists left by pull levels, ping-pong by level
    const int2 *first2;           // first two neighbours of each row, or NULL (read the CSR)
    uint32_t bmp_min_T;           // push levels with at least this many edges mark a bitmap
    uint32_t ulist_max;           // a pull level works on U_L when |U_L| <= ulist_max
    unsigned long long timeout_ns;
    int32_t src;
};

template <typename OffT>
struct PushWarpSmem {
    uint32_t qe[WTILE + 2];
    int32_t u[WTILE + 1];
    OffT rs[WTILE + 1];
    alignas(16) uint16_t rid[WTILE];   // row of each tile position
};

template <typename OffT>
struct PullWarpSmem {
    uint16_t list[SC_VERTS];       // compacted candidates of the chunk (offsets)
    OffT hb[PULL_WCH];             // heavy lists: next edge
    uint32_t hl[PULL_WCH];         // heavy lists: edges left
    uint32_t hofs[PULL_WCH + 1];   // heavy lists: prefix of the unresolved lengths
    alignas(16) uint16_t hrid[PULL_HSTEP];   // heavy step: list of each position
    int32_t hpar[PULL_WCH];        // heavy lists: parent found (-1: none yet)
    uint16_t hv[PULL_WCH];         // heavy lists: the candidate (offset in its chunk)
    uint32_t fb[32];               // found bits of the chunk's words
};

template <typename OffT>
union WarpSmem {
    PushWarpSmem<OffT> p;
    PullWarpSmem<OffT> l;
};

// Each warp's shared memory, in the block's dynamic shared memory (WARPS
// entries; more than the 48 KB a block may declare statically with 64-bit
// offsets, so the kernels opt in to the larger size before their first launch).
template <typename OffT>
constexpr size_t bfs_smem_bytes() { return WARPS * sizeof(WarpSmem<OffT>); }

template <typename OffT>
__device__ __forceinline__ WarpSmem<OffT> &warp_smem() {
    extern __shared__ __align__(16) unsigned char bfs_dsmem[];
    return reinterpret_cast<WarpSmem<OffT> *>(bfs_dsmem)[threadIdx.x >> 5];
}

__device__ __forceinline__ int level_phases(const LevelState &s) {
    return s.dir == DIR_PULL ? 1 : 1 + s.compact + s.bmp;
}

__device__ __forceinline__ int level_op(const LevelState &s) {
    if (s.dir == DIR_PULL) return s.lmode ? OP_PULL_LIST : OP_PULL;
    const int p = (int)s.phase - (int)s.compact;
    if (p < 0) return OP_COMPACT;
    if (p == 0) return s.bmp ? OP_BMARK : OP_QPUSH;
    return OP_BFINAL;
}

template <typename OffT>
__device__ __forceinline__ void set_kind(const BfsArgs<OffT> &a, LevelState &s) {
    s.compact = s.dir == DIR_PUSH && !s.qin;
    s.bmp = s.dir == DIR_PUSH && s.T >= a.bmp_min_T;
    s.lmode = s.dir == DIR_PULL && s.uin && s.ucnt <= a.ulist_max;
    s.uwrite = s.dir == DIR_PULL;
    // a queue push feeds F_{L+1} only while a pull may still follow
    s.fwrite = s.dir == DIR_PULL || s.bmp || (a.mode == GRX_DIR_AUTO && !s.back);
}

template <typename OffT>
__device__ LevelState initial_state(const BfsArgs<OffT> &a) {
    LevelState s;
    memset(&s, 0, sizeof s);
    s.L = 0;
    s.dir = a.mode == GRX_DIR_PULL ? DIR_PULL : DIR_PUSH;
    s.switched = a.mode == GRX_DIR_PULL;
    s.fprev = 1;                 // F_0 = {src}
    s.qin = 1;                   // Q_0 = {src}
    const uint32_t deg = (uint32_t)(__ldg(a.ro + a.src + 1) - __ldg(a.ro + a.src));
    s.q = deg > 0 ? 1u : 0u;
    s.T = deg;
    s.vcount = 1;
    set_kind(a, s);
    if (s.q == 0) s.done = 1;
    return s;
}

// State of the next phase: the same level's next phase, or level L+1 from the
// counters level L left.
template <typename OffT>
__device__ LevelState next_state(const BfsArgs<OffT> &a, const LevelState &st, bool stats) {
    LevelState ns = st;
    ns.seq = st.seq + 1;
    if ((int)st.phase + 1 < level_phases(st)) {
        ns.phase = st.phase + 1;
        return ns;
    }
    ns.L = st.L + 1;
    ns.phase = 0;
    const unsigned long long pk = ld_relaxed_u64(&a.ctl->qpack[(st.L + 1) & 3]);
    ns.q = (uint32_t)(pk >> 32);
    ns.T = (uint32_t)pk;
    ns.nprev = st.q;
    ns.vcount = st.vcount + ns.q;
    ns.fclear = st.fprev;
    ns.fprev = st.fwrite;
    ns.qprev_ok = st.qin || st.compact;
    ns.qin = st.dir == DIR_PUSH || st.lmode;     // a list pull appends what it finds
    ns.uin = st.uwrite;
    ns.ucnt = st.uwrite ? ld_relaxed_u32(&a.ctl->ucount[(st.L + 1) & 3]) : 0u;
    if (stats && blockIdx.x == 0 && st.L < GRX_MAX_LEVELS_STATS) a.stats->discovered[st.L] = ns.q;
    if (ns.q == 0) {
        ns.done = 1;
        return ns;
    }
    if (a.mode == GRX_DIR_PUSH) {
        ns.dir = DIR_PUSH;
    } else if (a.mode == GRX_DIR_PULL) {
        ns.dir = DIR_PULL;
    } else {
        // Sec. 6.1: FV = |Q|*E/V (or the exact frontier edge count), BV = |U|*V/|P|
        const double V = (double)a.nv, E = (double)a.ne;
        const double FV = a.exact_fv ? (double)ns.T : (double)ns.q * E / V;
        const double BV = (double)(a.nv - (long long)ns.vcount) * V / (double)ns.vcount;
        if (st.dir == DIR_PUSH && !st.switched && FV > BV * (double)a.alpha) {
            ns.dir = DIR_PULL;
            ns.switched = 1;
        } else if (st.dir == DIR_PULL && FV < BV * (double)a.beta) {
            ns.dir = DIR_PUSH;
            ns.back = 1;
        }
    }
    set_kind(a, ns);
    return ns;
}

// Loads warp tile `tile` of the frontier's edge sequence: the frontier
// elements that start before the tile's end go to shared memory (i0 = the
// element holding the tile's first edge), then every lane takes PUSH_ITEMS
// edges of the tile, item k at position k*32 + lane (a warp's column loads
// are contiguous): destination v[k], source u[k] (when WANT_U), valid bits.
// Returns the element holding the next tile's first edge.
template <typename OffT, bool WANT_U>
__device__ __forceinline__ int64_t push_tile(const BfsArgs<OffT> &a, const int32_t *Qv,
                                             const uint32_t *Qe, const OffT *Qr, int64_t q,
                                             uint64_t T, uint64_t tile, int64_t i0,
                                             PushWarpSmem<OffT> &w, int32_t (&v)[PUSH_ITEMS],
                                             int32_t (&u)[PUSH_ITEMS], uint32_t &valid) {
    const unsigned int lane = threadIdx.x & 31;
    const uint64_t e0 = tile * WTILE;
    const uint32_t e1 = (uint32_t)min(T, e0 + WTILE);
    // frontier elements starting before e1, 32 per round; w.qe[n] ends up
    // holding the start of the first element past the tile
    int n = 0;
    for (;;) {
        const int64_t idx = i0 + n + lane;
        uint32_t qe = 0xffffffffu;
        if (idx < q) qe = __ldcg(Qe + idx);
        const bool in = idx < q && qe < e1;
        if (n + (int)lane <= WTILE + 1) w.qe[n + lane] = qe;
        if (in && n + (int)lane <= WTILE) {
            if (WANT_U) w.u[n + lane] = __ldcg(Qv + idx);
            w.rs[n + lane] = __ldcg(Qr + idx);
        }
        const int cnt = __popc(__ballot_sync(GRX_FULL_MASK, in));
        n += cnt;
        if (cnt < 32) break;
        if (n > WTILE) {              // only possible with a malformed graph
            if (lane == 0) grx_set_status(a.ctl, GRX_EINVAL);
            n = WTILE;
            break;
        }
    }
    __syncwarp();
    const uint32_t next_start = w.qe[n];
    int row[PUSH_ITEMS];
    warp_tile_rows8_strided(w.rid, w.qe, (uint32_t)e0, n, row);
    valid = 0;
#pragma unroll
    for (int k = 0; k < PUSH_ITEMS; ++k) {
        const uint32_t e = (uint32_t)e0 + (uint32_t)k * 32 + lane;
        const int j = row[k];
        const bool ok = e < e1;
        v[k] = ok ? __ldg(a.col + w.rs[j] + (OffT)(e - w.qe[j])) : 0;
        u[k] = (WANT_U && ok) ? w.u[j] : 0;
        valid |= (ok ? 1u : 0u) << k;
    }
    __syncwarp();
    // the element holding e1 starts the next tile
    return (next_start == e1) ? i0 + n : i0 + n - 1;
}

// Next 32-word chunk of a word-owning sweep for the calling warp: chunks are
// handed out in increasing order from the phase's counter, so warps that
// meet cheap chunks take more of them and all finish together.
__device__ __forceinline__ int64_t grab_chunk(unsigned int *ctr) {
    unsigned int c = 0;
    if ((threadIdx.x & 31) == 0) c = atomicAdd(ctr, 1u);
    return (int64_t)__shfl_sync(GRX_FULL_MASK, c, 0);
}

// Lanes aiming at the same vertex: only the lowest one keeps its bit.
__device__ __forceinline__ uint32_t dedup_items(const int32_t (&v)[PUSH_ITEMS], uint32_t cand) {
#if GRX_PUSH_DEDUP
    uint32_t out = 0;
#pragma unroll
    for (int k = 0; k < PUSH_ITEMS; ++k) {
        const bool c = cand >> k & 1u;
        const unsigned int same = __match_any_sync(GRX_FULL_MASK, c ? v[k] : -1 - (int)(threadIdx.x & 31));
        if (c && (same & lanemask_lt()) == 0) out |= 1u << k;
    }
    return out;
#else
    return cand;
#endif
}

// Queue push: claim with atomicOr on visited, label, append to Q_{L+1}.
template <typename OffT, bool PARENT>
__device__ void push_queue(const BfsArgs<OffT> &a, const LevelState &st, PushWarpSmem<OffT> &w) {
    const int L = st.L;
    const int32_t *Qv = pick3(a.Q[0], a.Q[1], a.Q[2], L % 3);
    const uint32_t *Qe = pick3(a.E[0], a.E[1], a.E[2], L % 3);
    const OffT *Qr = pick3(a.R[0], a.R[1], a.R[2], L % 3);
    int32_t *Qv_out = pick3(a.Q[0], a.Q[1], a.Q[2], (L + 1) % 3);
    uint32_t *Qe_out = pick3(a.E[0], a.E[1], a.E[2], (L + 1) % 3);
    OffT *Qr_out = pick3(a.R[0], a.R[1], a.R[2], (L + 1) % 3);
    uint32_t *Fout = pick3(a.F[0], a.F[1], a.F[2], (L + 1) % 3);
    unsigned long long *ctr = &a.ctl->qpack[(L + 1) & 3];
    const int64_t q = st.q;
    const uint64_t T = st.T;
    const uint64_t ntiles = (T + WTILE - 1) / WTILE;
    const uint64_t nwarps = (uint64_t)gridDim.x * WARPS;
    const uint64_t gw = (uint64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    // each warp owns a contiguous range of tiles: one search for its first element
    const uint64_t per = (ntiles + nwarps - 1) / nwarps;
    const uint64_t tb0 = gw * per;
    const uint64_t tb1 = min(ntiles, tb0 + per);
    if (tb0 >= tb1) return;
    int64_t i0 = warp_upper_index_cg(Qe, q, (uint32_t)(tb0 * WTILE));
    for (uint64_t tile = tb0; tile < tb1; ++tile) {
        int32_t v[PUSH_ITEMS], par[PUSH_ITEMS];
        uint32_t valid;
        i0 = push_tile<OffT, PARENT>(a, Qv, Qe, Qr, q, T, tile, i0, w, v, par, valid);
        uint32_t wv[PUSH_ITEMS];
#pragma unroll
        for (int k = 0; k < PUSH_ITEMS; ++k)   // a filter: the atomic's old value decides
            wv[k] = (valid >> k & 1u) ? __ldca(a.visited + (v[k] >> 5)) : 0xffffffffu;
        uint32_t cand = 0;
#pragma unroll
        for (int k = 0; k < PUSH_ITEMS; ++k)
            if (!((wv[k] >> (v[k] & 31)) & 1u)) cand |= 1u << k;
        cand = dedup_items(v, cand);
        uint32_t old[PUSH_ITEMS];
#pragma unroll
        for (int k = 0; k < PUSH_ITEMS; ++k)
            old[k] = (cand >> k & 1u) ? atomicOr(a.visited + (v[k] >> 5), 1u << (v[k] & 31)) : 0xffffffffu;
        uint32_t disc = 0;
#pragma unroll
        for (int k = 0; k < PUSH_ITEMS; ++k)
            if (!((old[k] >> (v[k] & 31)) & 1u)) disc |= 1u << k;
        uint32_t deg[PUSH_ITEMS];
        OffT rb[PUSH_ITEMS], re[PUSH_ITEMS];
#pragma unroll
        for (int k = 0; k < PUSH_ITEMS; ++k) {
            rb[k] = 0;
            re[k] = 0;
            if (disc >> k & 1u) {
                rb[k] = __ldg(a.ro + v[k]);
                re[k] = __ldg(a.ro + v[k] + 1);
            }
        }
        uint32_t app = 0;
#pragma unroll
        for (int k = 0; k < PUSH_ITEMS; ++k) {
            deg[k] = (uint32_t)(re[k] - rb[k]);
            if (disc >> k & 1u) {
                a.depth[v[k]] = L + 1;
                if (PARENT) a.parent[v[k]] = par[k];
                if (deg[k]) {
                    app |= 1u << k;
                    if (st.fwrite) atomicOr(Fout + (v[k] >> 5), 1u << (v[k] & 31));
                }
            }
        }
        warp_append_items<PUSH_ITEMS, OffT>(v, deg, rb, app, Qv_out, Qe_out, Qr_out, ctr);
        __syncwarp();
    }
}

// Bitmap push, phase 1: every target whose visited bit is clear gets its bit
// in visited and in F_{L+1} (reductions: no value returned).  The visited
// probe is a filter: a stale clear bit only repeats a reduction, and bits of
// earlier levels are always seen (they were written before the level's
// barrier), so F_{L+1} ends up holding exactly the vertices first reached in
// this level.  One probe per edge is the cost that matters: each is a random
// cache line.  With PARENT, a marking lane stores its source as the parent:
// every writer is a valid parent, one of them remains.
template <typename OffT, bool PARENT>
__device__ void push_mark(const BfsArgs<OffT> &a, const LevelState &st, PushWarpSmem<OffT> &w) {
    const int L = st.L;
    const int32_t *Qv = pick3(a.Q[0], a.Q[1], a.Q[2], L % 3);
    const uint32_t *Qe = pick3(a.E[0], a.E[1], a.E[2], L % 3);
    const OffT *Qr = pick3(a.R[0], a.R[1], a.R[2], L % 3);
    uint32_t *Fout = pick3(a.F[0], a.F[1], a.F[2], (L + 1) % 3);
    const int64_t q = st.q;
    const uint64_t T = st.T;
    const uint64_t ntiles = (T + WTILE - 1) / WTILE;
    const uint64_t nwarps = (uint64_t)gridDim.x * WARPS;
    const uint64_t gw = (uint64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    const uint64_t per = (ntiles + nwarps - 1) / nwarps;
    const uint64_t tb0 = gw * per;
    const uint64_t tb1 = min(ntiles, tb0 + per);
    if (tb0 >= tb1) return;
    int64_t i0 = warp_upper_index_cg(Qe, q, (uint32_t)(tb0 * WTILE));
    for (uint64_t tile = tb0; tile < tb1; ++tile) {
        int32_t v[PUSH_ITEMS], par[PUSH_ITEMS];
        uint32_t valid;
        i0 = push_tile<OffT, PARENT>(a, Qv, Qe, Qr, q, T, tile, i0, w, v, par, valid);
        uint32_t wv[PUSH_ITEMS];
#pragma unroll
        for (int k = 0; k < PUSH_ITEMS; ++k)
            wv[k] = (valid >> k & 1u) ? __ldca(a.visited + (v[k] >> 5)) : 0xffffffffu;
#pragma unroll
        for (int k = 0; k < PUSH_ITEMS; ++k) {
            if (!((wv[k] >> (v[k] & 31)) & 1u)) {
                const uint32_t bit = 1u << (v[k] & 31);
                if (PARENT) a.parent[v[k]] = par[k];
                atomicOr(a.visited + (v[k] >> 5), bit);     // results unused: reductions
                atomicOr(Fout + (v[k] >> 5), bit);
            }
        }
    }
}

// Word-owning pass from a frontier bitmap to a frontier queue.  FINAL (bitmap
// push, phase 2): B = F_{L+1} (already in visited); its vertices are
// labelled L+1 and appended to Q_{L+1} (counter of level L).  Otherwise (compaction
// before a push level): B = F_L, appended to Q_L through the compaction
// counter.  Vertices without edges are labelled but not queued.
template <typename OffT, bool FINAL>
__device__ void bitmap_to_queue(const BfsArgs<OffT> &a, const LevelState &st, PullWarpSmem<OffT> &w) {
    const int L = st.L;
    const int ring = FINAL ? (L + 1) % 3 : L % 3;
    uint32_t *B = pick3(a.F[0], a.F[1], a.F[2], ring);
    int32_t *Qv = pick3(a.Q[0], a.Q[1], a.Q[2], ring);
    uint32_t *Qe = pick3(a.E[0], a.E[1], a.E[2], ring);
    OffT *Qr = pick3(a.R[0], a.R[1], a.R[2], ring);
    unsigned long long *ctr = FINAL ? &a.ctl->qpack[(L + 1) & 3] : &a.ctl->cpack;
    const unsigned int lane = threadIdx.x & 31;
    const int64_t nsc = (a.words + 31) / 32;
    unsigned int *wq = &a.ctl->wq[st.seq & 3];
    // first chunk: the warp's own index; later ones from the phase's counter
    // (offset by the warp count).  The next chunk is requested at the start
    // of the body and read at its end, so the counter's round trip overlaps
    // this chunk's work.
    const unsigned int nwarps = gridDim.x * WARPS;
    int64_t sc = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    while (sc < nsc) {
        unsigned int nn = 0;
        if (lane == 0) nn = nwarps + atomicAdd(wq, 1u);
        const int64_t wd = sc * 32 + lane;
        const uint32_t bits = wd < a.words ? __ldcg(B + wd) : 0u;
        if (FINAL && bits) {
            // a frontier bitmap holds vertices with edges only (as the queue does)
            const uint32_t nzw = __ldg(a.nz + wd);
            if (bits & ~nzw) B[wd] = bits & nzw;
        }
        const int n = warp_compact_bits(bits, w.list);
        for (int base = 0; base < n; base += PULL_WCH) {
            int32_t v[PULL_PER_LANE];
            OffT rb[PULL_PER_LANE], re[PULL_PER_LANE];
            uint32_t deg[PULL_PER_LANE];
            uint32_t app = 0;
#pragma unroll
            for (int k = 0; k < PULL_PER_LANE; ++k) {
                const int i = base + k * 32 + (int)lane;
                v[k] = i < n ? (int32_t)(sc * SC_VERTS + w.list[i]) : -1;
                rb[k] = 0;
                re[k] = 0;
                if (v[k] >= 0) {
                    rb[k] = __ldg(a.ro + v[k]);
                    re[k] = __ldg(a.ro + v[k] + 1);
                }
            }
#pragma unroll
            for (int k = 0; k < PULL_PER_LANE; ++k) {
                deg[k] = (uint32_t)(re[k] - rb[k]);
                if (v[k] >= 0) {
                    if (FINAL) a.depth[v[k]] = L + 1;
                    if (deg[k]) app |= 1u << k;
                }
            }
            warp_append_items<PULL_PER_LANE, OffT>(v, deg, rb, app, Qv, Qe, Qr, ctr);
        }
        __syncwarp();
        sc = (int64_t)__shfl_sync(GRX_FULL_MASK, nn, 0);
    }
}

// Row start, degree and first two neighbours of the candidates a lane takes
// in the round starting at list entry `base` (entries base + k*32 + lane;
// vertex = origin + list[i]).
template <typename OffT>
__device__ __forceinline__ void load_candidates(const BfsArgs<OffT> &a, int64_t origin, const uint16_t *list,
                                                int base, int n, int32_t (&v)[PULL_PER_LANE],
                                                OffT (&b)[PULL_PER_LANE], uint32_t (&deg)[PULL_PER_LANE],
                                                int2 (&f2)[PULL_PER_LANE]) {
    const unsigned int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < PULL_PER_LANE; ++k) {
        const int i = base + k * 32 + (int)lane;
        v[k] = i < n ? (int32_t)(origin + list[i]) : -1;
        OffT e = 0;
        b[k] = 0;
        f2[k] = make_int2(-1, -1);
        if (v[k] >= 0) {
            b[k] = __ldg(a.ro + v[k]);
            e = __ldg(a.ro + v[k] + 1);
            if (a.first2) f2[k] = __ldg(a.first2 + v[k]);
        }
        deg[k] = (uint32_t)(e - b[k]);
    }
}

// Light phase of a pull round over up to PULL_WCH candidates of a warp (lane
// holds candidates k*32 + lane): v (-1 = empty slot), row start b, degree
// deg, first two neighbours f2.  The first PULL_LIGHT neighbours of every
// candidate are probed against F_L, all in flight at once.  par[k] = the
// parent found (-1: none); bit k of the result = candidate k still needs its
// remaining neighbours (heavy).  F_L is read-only during the level, so its
// probes may be served by L1 (hot words of high-degree vertices are then not
// refetched from L2 by every warp).
template <typename OffT, bool STATS>
__device__ __forceinline__ uint32_t pull_light(const BfsArgs<OffT> &a, const uint32_t *Fin,
                                               const int32_t (&v)[PULL_PER_LANE], const OffT (&b)[PULL_PER_LANE],
                                               const uint32_t (&deg)[PULL_PER_LANE],
                                               const int2 (&f2)[PULL_PER_LANE], int32_t (&par)[PULL_PER_LANE],
                                               unsigned long long &scanned_e, unsigned long long &scanned_v) {
    static_assert(PULL_LIGHT == 2, "the light phase probes the two neighbours of first2");
    int32_t u0[PULL_PER_LANE], u1[PULL_PER_LANE];
#pragma unroll
    for (int k = 0; k < PULL_PER_LANE; ++k) {
        if (a.first2) {          // loaded by the caller beside the row offsets
            u0[k] = f2[k].x;
            u1[k] = f2[k].y;
        } else {
            u0[k] = deg[k] > 0 ? __ldg(a.col + b[k]) : -1;
            u1[k] = deg[k] > 1 ? __ldg(a.col + b[k] + 1) : -1;
        }
    }
    uint32_t f0[PULL_PER_LANE], f1[PULL_PER_LANE];
#pragma unroll
    for (int k = 0; k < PULL_PER_LANE; ++k) {
        f0[k] = u0[k] >= 0 ? __ldca(Fin + (u0[k] >> 5)) : 0u;
        f1[k] = u1[k] >= 0 ? __ldca(Fin + (u1[k] >> 5)) : 0u;
    }
    uint32_t heavy = 0;
#pragma unroll
    for (int k = 0; k < PULL_PER_LANE; ++k) {
        par[k] = -1;
        if (u0[k] >= 0 && ((f0[k] >> (u0[k] & 31)) & 1u)) par[k] = u0[k];
        else if (u1[k] >= 0 && ((f1[k] >> (u1[k] & 31)) & 1u)) par[k] = u1[k];
        if (STATS && v[k] >= 0) {
            scanned_v += 1;
            scanned_e += (unsigned long long)min((uint32_t)PULL_LIGHT, deg[k]);
        }
        if (v[k] >= 0 && par[k] < 0 && deg[k] > PULL_LIGHT) heavy |= 1u << k;
    }
    return heavy;
}

// Appends the heavy candidates (bit k of `heavy`) to the warp's pending heavy
// lists after the nh already there: next edge, edges left, no parent yet, the
// vertex's offset in its 1,024-vertex chunk.  hpos[k] = entry of candidate k.  Returns the new
// count (warp-uniform; at most PULL_WCH, which the caller guarantees).
template <typename OffT>
__device__ __forceinline__ int heavy_add(PullWarpSmem<OffT> &w, int nh, uint32_t heavy,
                                         const int32_t (&v)[PULL_PER_LANE], const OffT (&b)[PULL_PER_LANE],
                                         const uint32_t (&deg)[PULL_PER_LANE], int (&hpos)[PULL_PER_LANE]) {
#pragma unroll
    for (int k = 0; k < PULL_PER_LANE; ++k) {
        const unsigned int m = __ballot_sync(GRX_FULL_MASK, heavy >> k & 1u);
        hpos[k] = nh + __popc(m & lanemask_lt());
        if (heavy >> k & 1u) {
            w.hb[hpos[k]] = b[k] + PULL_LIGHT;
            w.hl[hpos[k]] = deg[k] - PULL_LIGHT;
            w.hpar[hpos[k]] = -1;
            w.hv[hpos[k]] = (uint16_t)(v[k] & (SC_VERTS - 1));
        }
        nh += __popc(m);
    }
    __syncwarp();
    return nh;
}

// Heavy phase over the warp's nh pending lists: they are concatenated and
// consumed front to back in load-balanced steps of PULL_HSTEP edges shared by
// the whole warp; a list leaves once any of its edges hits the frontier (any
// frontier neighbour is a valid parent: edge skipping).  On return w.hpar[h]
// holds each list's parent (-1: none).
template <typename OffT, bool STATS>
__device__ __forceinline__ void heavy_run(const BfsArgs<OffT> &a, const uint32_t *Fin, PullWarpSmem<OffT> &w,
                                          int nh, unsigned long long &scanned_e) {
    const unsigned int lane = threadIdx.x & 31;
    while (nh > 0) {
        // exclusive prefix of the unresolved lengths; lane owns entries lane*PULL_PER_LANE + r
        uint32_t ln[PULL_PER_LANE], lsum = 0;
#pragma unroll
        for (int r = 0; r < PULL_PER_LANE; ++r) {
            const int h = (int)lane * PULL_PER_LANE + r;
            ln[r] = (h < nh && w.hpar[h] < 0) ? w.hl[h] : 0u;
            lsum += ln[r];
        }
        uint32_t x = lsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(GRX_FULL_MASK, x, o);
            if (lane >= (unsigned)o) x += y;
        }
        const uint32_t total = __shfl_sync(GRX_FULL_MASK, x, 31);
        if (total == 0) break;
        uint32_t off = x - lsum;
#pragma unroll
        for (int r = 0; r < PULL_PER_LANE; ++r) {
            const int h = (int)lane * PULL_PER_LANE + r;
            if (h < nh) w.hofs[h] = off;
            off += ln[r];
        }
        if (lane == 0) w.hofs[nh] = total;
        __syncwarp();
        const uint32_t steplen = min(total, (uint32_t)PULL_HSTEP);
        int hrow[PULL_HITEMS];
        warp_tile_rows8_strided(w.hrid, w.hofs, 0u, nh, hrow);   // item k at position k*32 + lane
        int32_t uu[PULL_HITEMS];
#pragma unroll
        for (int k = 0; k < PULL_HITEMS; ++k) {
            const uint32_t j = (uint32_t)k * 32 + lane;
            const int h = hrow[k];
            uu[k] = j < steplen ? __ldg(a.col + w.hb[h] + (OffT)(j - w.hofs[h])) : -1;
        }
#pragma unroll
        for (int k = 0; k < PULL_HITEMS; ++k) {
            if (uu[k] >= 0 && ((__ldca(Fin + (uu[k] >> 5)) >> (uu[k] & 31)) & 1u))
                w.hpar[hrow[k]] = uu[k];          // any hit is a valid parent
        }
        if (STATS) {
#pragma unroll
            for (int k = 0; k < PULL_HITEMS; ++k) scanned_e += (uint32_t)k * 32 + lane < steplen ? 1ull : 0ull;
        }
        __syncwarp();
        // the step consumed the first steplen edges of the concatenation
#pragma unroll
        for (int r = 0; r < PULL_PER_LANE; ++r) {
            const int h = (int)lane * PULL_PER_LANE + r;
            if (ln[r] > 0 && w.hpar[h] < 0) {
                const uint32_t o = w.hofs[h];
                const uint32_t used = steplen > o ? min(ln[r], steplen - o) : 0u;
                w.hb[h] += (OffT)used;
                w.hl[h] = ln[r] - used;
            }
        }
        __syncwarp();
    }
}

// Appends the vertices of bit set `bits` (lane holds word wd = word index of
// its 32 vertices) to list[] with one counter update per warp; order within
// the warp's batch is the vertex order.  Uses w.list as staging.
template <typename OffT>
__device__ __forceinline__ void warp_append_bits(uint32_t bits, int64_t sc, PullWarpSmem<OffT> &w,
                                                 int32_t *list, unsigned int *ctr) {
    const unsigned int lane = threadIdx.x & 31;
    const int n = warp_compact_bits(bits, w.list);
    if (n == 0) return;
    unsigned int base = 0;
    if (lane == 0) base = atomicAdd(ctr, (unsigned)n);
    base = __shfl_sync(GRX_FULL_MASK, base, 0);
    for (int i = (int)lane; i < n; i += 32) list[base + i] = (int32_t)(sc * SC_VERTS + w.list[i]);
    __syncwarp();
}

// Pull level over all vertices (sweep): the owner of each 32-word chunk finds
// a frontier parent for the chunk's unvisited non-isolated vertices and
// writes the chunk's visited and F_{L+1} words (and, with fclear, zeroes its
// F_{L-1} words).  Chunks come from the phase's counter.  Candidates are
// compacted in shared memory and probed PULL_WCH per round (pull_light); the
// lists still unresolved after their first neighbours wait in the warp's
// pending heavy lists, which are scanned together (heavy_run) when the next
// round could overflow them and at the end of the chunk, so a chunk usually
// takes one heavy scan instead of one per round.  Found vertices are labelled
// and their bits collect in the chunk's masks.  The candidates left unfound
// form the list U_{L+1} (in chunk order), which a following pull level may
// work on instead of sweeping again.
template <typename OffT, bool PARENT, bool STATS>
__device__ void pull_level(const BfsArgs<OffT> &a, const LevelState &st, PullWarpSmem<OffT> &w,
                           unsigned long long &scanned_e, unsigned long long &scanned_v) {
    const int L = st.L;
    const unsigned int lane = threadIdx.x & 31;
    const uint32_t *Fin = pick3(a.F[0], a.F[1], a.F[2], L % 3);
    uint32_t *Fout = pick3(a.F[0], a.F[1], a.F[2], (L + 1) % 3);
    uint32_t *Fold = pick3(a.F[0], a.F[1], a.F[2], (L + 2) % 3);
    int32_t *Unext = a.U[(L + 1) & 1];
    unsigned int *uctr = &a.ctl->ucount[(L + 1) & 3];
    const int64_t nsc = (a.words + 31) / 32;
    unsigned int *wq = &a.ctl->wq[st.seq & 3];
    uint32_t nfound = 0;
    uint32_t nedges = 0;
    // first chunk: the warp's own index; later ones from the phase's counter
    // (offset by the warp count).  The next chunk is requested at the start
    // of the body and read at its end, so the counter's round trip overlaps
    // this chunk's work.
    const unsigned int nwarps = gridDim.x * WARPS;
    int64_t sc = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    while (sc < nsc) {
        unsigned int nn = 0;
        if (lane == 0) nn = nwarps + atomicAdd(wq, 1u);
        const int64_t wd = sc * 32 + lane;
        const bool own = wd < a.words;
        const uint32_t vis = own ? __ldcg(a.visited + wd) : 0xffffffffu;
        const uint32_t cand = own ? (__ldg(a.nz + wd) & ~vis) : 0u;
        if (own && st.fclear) Fold[wd] = 0u;
        w.fb[lane] = 0u;
        const int n = warp_compact_bits(cand, w.list);
        const int64_t origin = sc * SC_VERTS;
        int32_t vn[PULL_PER_LANE];
        OffT bn[PULL_PER_LANE];
        uint32_t dn[PULL_PER_LANE];
        int2 fn[PULL_PER_LANE];
        load_candidates(a, origin, w.list, 0, n, vn, bn, dn, fn);
        // the chunk's pending heavy lists: scanned, then their found vertices
        // labelled like the light ones
        int nh = 0;
        auto flush_heavy = [&]() {
            heavy_run<OffT, STATS>(a, Fin, w, nh, scanned_e);
            for (int h = (int)lane; h < nh; h += 32) {
                const int32_t p = w.hpar[h];
                if (p >= 0) {
                    const int32_t u = (int32_t)(origin + w.hv[h]);
                    a.depth[u] = L + 1;
                    if (PARENT) a.parent[u] = p;
                    atomicOr(&w.fb[(u >> 5) & 31], 1u << (u & 31));
                    nfound += 1;
                    nedges += (uint32_t)(__ldg(a.ro + u + 1) - __ldg(a.ro + u));
                }
            }
            __syncwarp();
            nh = 0;
        };
        // one flush site: before a round whose heavy lists could overflow the
        // pending ones, and after the last round
        for (int base = 0;; base += PULL_WCH) {
            const bool more = base < n;
            int32_t v[PULL_PER_LANE];
            OffT b[PULL_PER_LANE];
            uint32_t deg[PULL_PER_LANE];
            int2 f2[PULL_PER_LANE];
#pragma unroll
            for (int k = 0; k < PULL_PER_LANE; ++k) {
                v[k] = vn[k];
                b[k] = bn[k];
                deg[k] = dn[k];
                f2[k] = fn[k];
            }
            int32_t par[PULL_PER_LANE];
            uint32_t heavy = 0;
            int nnew = 0;
            if (more) {
                heavy = pull_light<OffT, STATS>(a, Fin, v, b, deg, f2, par, scanned_e, scanned_v);
                nnew = (int)warp_sum((uint32_t)__popc(heavy));
            }
            if (!more || nh + nnew > PULL_WCH) flush_heavy();
            if (!more) break;
            // the next round's loads go out and travel while this round is labelled
            load_candidates(a, origin, w.list, base + PULL_WCH, n, vn, bn, dn, fn);
            // label the found vertices; their bits go to the chunk's word masks
#pragma unroll
            for (int k = 0; k < PULL_PER_LANE; ++k) {
                if (par[k] >= 0) {
                    a.depth[v[k]] = L + 1;
                    if (PARENT) a.parent[v[k]] = par[k];
                    atomicOr(&w.fb[(v[k] >> 5) & 31], 1u << (v[k] & 31));
                    nfound += 1;
                    nedges += deg[k];
                }
            }
            int hpos[PULL_PER_LANE];
            nh = heavy_add(w, nh, heavy, v, b, deg, hpos);
        }
        const uint32_t fb = w.fb[lane];
        if (own) {
            if (fb) a.visited[wd] = vis | fb;
            Fout[wd] = fb;               // whole word: F_{L+1} needs no clearing first
        }
        __syncwarp();
        if (st.uwrite) warp_append_bits(cand & ~fb, sc, w, Unext, uctr);
        sc = (int64_t)__shfl_sync(GRX_FULL_MASK, nn, 0);
    }
    // one counter update per warp: (found << 32 | their edges)
    const unsigned long long cnt = warp_sum((unsigned long long)nfound);
    const unsigned long long edg = warp_sum((unsigned long long)nedges);
    if (lane == 0 && cnt) atomicAdd(&a.ctl->qpack[(L + 1) & 3], (cnt << 32) | edg);
}

// Pull level over the list U_L of the candidates the previous pull level
// left unfound (every one unvisited and non-isolated): slices of PULL_WCH
// list entries per warp, light probes then the heavy lists of the slice.  Found vertices are labelled,
// their bits set in visited and F_{L+1} (reductions: a word is shared with
// other warps' vertices), and they are appended to Q_{L+1} with their degrees
// and row starts, so a push level that follows needs no compaction.  The
// unfound ones form U_{L+1}.
template <typename OffT, bool PARENT, bool STATS>
__device__ void pull_list(const BfsArgs<OffT> &a, const LevelState &st, PullWarpSmem<OffT> &w,
                          unsigned long long &scanned_e, unsigned long long &scanned_v) {
    const int L = st.L;
    const unsigned int lane = threadIdx.x & 31;
    const uint32_t *Fin = pick3(a.F[0], a.F[1], a.F[2], L % 3);
    uint32_t *Fout = pick3(a.F[0], a.F[1], a.F[2], (L + 1) % 3);
    int32_t *Qv_out = pick3(a.Q[0], a.Q[1], a.Q[2], (L + 1) % 3);
    uint32_t *Qe_out = pick3(a.E[0], a.E[1], a.E[2], (L + 1) % 3);
    OffT *Qr_out = pick3(a.R[0], a.R[1], a.R[2], (L + 1) % 3);
    unsigned long long *qctr = &a.ctl->qpack[(L + 1) & 3];
    const int32_t *U = a.U[L & 1];
    int32_t *Unext = a.U[(L + 1) & 1];
    unsigned int *uctr = &a.ctl->ucount[(L + 1) & 3];
    const int64_t n = st.ucnt;
    const int64_t nsl = (n + PULL_WCH - 1) / PULL_WCH;
    unsigned int *wq = &a.ctl->wq[st.seq & 3];
    const unsigned int nwarps = gridDim.x * WARPS;
    int64_t sl = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    for (; sl < nsl; sl = nwarps + grab_chunk(wq)) {
        const int64_t base = sl * PULL_WCH;
        int32_t v[PULL_PER_LANE];
        OffT b[PULL_PER_LANE];
        uint32_t deg[PULL_PER_LANE];
        int2 f2[PULL_PER_LANE];
#pragma unroll
        for (int k = 0; k < PULL_PER_LANE; ++k) {
            const int64_t i = base + k * 32 + (int)lane;
            v[k] = i < n ? __ldcg(U + i) : -1;
        }
#pragma unroll
        for (int k = 0; k < PULL_PER_LANE; ++k) {
            OffT e = 0;
            b[k] = 0;
            f2[k] = make_int2(-1, -1);
            if (v[k] >= 0) {
                b[k] = __ldg(a.ro + v[k]);
                e = __ldg(a.ro + v[k] + 1);
                if (a.first2) f2[k] = __ldg(a.first2 + v[k]);
            }
            deg[k] = (uint32_t)(e - b[k]);
        }
        int32_t par[PULL_PER_LANE];
        const uint32_t heavy = pull_light<OffT, STATS>(a, Fin, v, b, deg, f2, par, scanned_e, scanned_v);
        int hpos[PULL_PER_LANE];
        const int nh = heavy_add(w, 0, heavy, v, b, deg, hpos);
        heavy_run<OffT, STATS>(a, Fin, w, nh, scanned_e);
#pragma unroll
        for (int k = 0; k < PULL_PER_LANE; ++k)
            if (heavy >> k & 1u) par[k] = w.hpar[hpos[k]];
        __syncwarp();
        uint32_t app = 0, left = 0;
#pragma unroll
        for (int k = 0; k < PULL_PER_LANE; ++k) {
            if (v[k] < 0) continue;
            if (par[k] >= 0) {
                const uint32_t bit = 1u << (v[k] & 31);
                a.depth[v[k]] = L + 1;
                if (PARENT) a.parent[v[k]] = par[k];
                atomicOr(a.visited + (v[k] >> 5), bit);
                atomicOr(Fout + (v[k] >> 5), bit);
                app |= 1u << k;
            } else {
                left |= 1u << k;
            }
        }
        warp_append_items<PULL_PER_LANE, OffT>(v, deg, b, app, Qv_out, Qe_out, Qr_out, qctr);
        if (st.uwrite) warp_append_list_items<PULL_PER_LANE>(v, left, Unext, uctr);
        __syncwarp();
    }
}

template <typename OffT, bool PARENT, bool STATS>
__device__ void run_phase(const BfsArgs<OffT> &a, const LevelState &st, WarpSmem<OffT> &w) {
    const int L = st.L;
    const int op = level_op(st);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // the compaction counter is only used by a first phase; zero it in a last one
        if ((int)st.phase + 1 == level_phases(st)) a.ctl->cpack = 0ull;
        // chunk counter of the phase after next (phase seq + 2 runs after two barriers)
        a.ctl->wq[(st.seq + 2) & 3] = 0u;
        if (st.phase == 0) a.ctl->ucount[(L + 2) & 3] = 0u;
        if (st.phase == 0) {
            a.ctl->qpack[(L + 2) & 3] = 0ull;
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
    if (st.phase == 0 && st.fclear && (st.dir == DIR_PUSH || st.lmode)) {
        // zero F_{L-1} (sweeping pull levels do it in their word loop)
        uint32_t *Fp = pick3(a.F[0], a.F[1], a.F[2], (L + 2) % 3);
        if (st.qprev_ok && (int64_t)st.nprev * 8 < a.words) {
            // F_{L-1} only holds bits of Q_{L-1}'s vertices: zero their words
            // (scattered stores; a queue of more than words/8 entries costs
            // more than zeroing every word with coalesced stores)
            const int32_t *Qp = pick3(a.Q[0], a.Q[1], a.Q[2], (L + 2) % 3);
            for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)st.nprev;
                 i += (int64_t)gridDim.x * blockDim.x)
                Fp[__ldcg(Qp + i) >> 5] = 0u;
        } else {
            for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.words;
                 i += (int64_t)gridDim.x * blockDim.x)
                Fp[i] = 0u;
        }
    }
    switch (op) {
    case OP_QPUSH: push_queue<OffT, PARENT>(a, st, w.p); break;
    case OP_BMARK: push_mark<OffT, PARENT>(a, st, w.p); break;
    case OP_BFINAL: bitmap_to_queue<OffT, true>(a, st, w.l); break;
    case OP_COMPACT: bitmap_to_queue<OffT, false>(a, st, w.l); break;
    default: {
        unsigned long long scanned_e = 0, scanned_v = 0;
        if (op == OP_PULL_LIST) pull_list<OffT, PARENT, STATS>(a, st, w.l, scanned_e, scanned_v);
        else pull_level<OffT, PARENT, STATS>(a, st, w.l, scanned_e, scanned_v);
        if (STATS) {
            scanned_e = warp_sum(scanned_e);
            scanned_v = warp_sum(scanned_v);
            if ((threadIdx.x & 31) == 0 && L < GRX_MAX_LEVELS_STATS) {
                if (scanned_e) atomicAdd(&a.stats->edges_examined[L], scanned_e);
                if (scanned_v) atomicAdd(&a.stats->vertices_scanned[L], scanned_v);
            }
        }
    }
    }
}

// Phase 0 of a traversal: depth = -1 (0 at src), parent = -1 (src at src),
// visited = {src}, F_0 = {src}, the other frontier bitmaps empty, the
// counters and the first frontier slot.  Every word is written by exactly one
// thread, so clearing and seeding need no barrier between them.
template <typename OffT, bool PARENT>
__device__ void init_phase(const BfsArgs<OffT> &a, const LevelState &st0) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int32_t src = a.src;
    for (int64_t v = tid; v < a.nv; v += stride) {
        a.depth[v] = v == src ? 0 : -1;
        if (PARENT) a.parent[v] = v == src ? src : -1;
    }
    const int64_t sw = src >> 5;
    const uint32_t sb = 1u << (src & 31);
    for (int64_t w = tid; w < a.words; w += stride) {
        a.visited[w] = w == sw ? sb : 0u;
        a.F[0][w] = w == sw ? sb : 0u;
        a.F[1][w] = 0u;
        a.F[2][w] = 0u;
    }
    if (tid == 0) {
        a.Q[0][0] = src;
        a.E[0][0] = 0;
        a.R[0][0] = __ldg(a.ro + src);
        a.ctl->qpack[0] = st0.q ? ((1ull << 32) | st0.T) : 0ull;
        for (int i = 1; i < 4; ++i) a.ctl->qpack[i] = 0ull;
        a.ctl->cpack = 0ull;
        for (int i = 0; i < 4; ++i) a.ctl->wq[i] = 0u;
        for (int i = 0; i < 4; ++i) a.ctl->ucount[i] = 0u;
    }
}

template <typename OffT, bool PARENT, bool STATS>
__global__ void __launch_bounds__(BFS_BLOCK, GRX_BFS_MIN_BLOCKS) k_bfs_persistent(BfsArgs<OffT> a) {
    __shared__ LevelState s_st;
    WarpSmem<OffT> &w = warp_smem<OffT>();
    FlagBarrier bar{a.bar_flags, &a.ctl->bar_release, a.ctl, a.timeout_ns, 0u};
    if (threadIdx.x == 0) s_st = initial_state(a);
    __syncthreads();
    init_phase<OffT, PARENT>(a, s_st);
    if (!flag_barrier(bar)) return;
    for (;;) {
        const LevelState st = s_st;
        if (st.done) break;
        run_phase<OffT, PARENT, STATS>(a, st, w);
        if (!flag_barrier(bar)) return;
        if (threadIdx.x == 0) s_st = next_state(a, st, STATS);
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->levels_run = s_st.L;
        if (STATS && s_st.L <= GRX_MAX_LEVELS_STATS) a.stats->level_t0[s_st.L] = grx_globaltimer();
    }
}

// Host-stepped variant: launch 0 initialises, launch i >= 1 runs phase i-1.
// The state of a phase is derived at the start of its launch from the state
// the previous launch stored and the counters it left, so no block ever
// waits on another.
template <typename OffT, bool PARENT, bool STATS>
__global__ void __launch_bounds__(BFS_BLOCK) k_bfs_step(BfsArgs<OffT> a, int launch) {
    __shared__ LevelState s_st;
    static_assert(sizeof(LevelState) <= sizeof(long long) * 8, "state must fit hstate");
    if (launch == 0) {
        if (threadIdx.x == 0) s_st = initial_state(a);
        __syncthreads();
        init_phase<OffT, PARENT>(a, s_st);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            LevelState st = s_st;
            memcpy((void *)a.ctl->hstate[0], &st, sizeof st);
        }
        return;
    }
    if (threadIdx.x == 0) {
        LevelState prev;
        memcpy(&prev, (const void *)a.ctl->hstate[(launch - 1) & 1], sizeof prev);
        s_st = (launch == 1 || prev.done) ? prev : next_state(a, prev, STATS);
    }
    __syncthreads();
    const LevelState st = s_st;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        memcpy((void *)a.ctl->hstate[launch & 1], &st, sizeof st);
        if (st.done) a.ctl->levels_run = st.L;
    }
    if (st.done) return;
    run_phase<OffT, PARENT, STATS>(a, st, warp_smem<OffT>());
}

// CUDA-graph variant: the body of a device-evaluated WHILE node is one phase
// kernel followed by a one-thread tick that derives the next phase's state
// and sets the loop condition.  The arguments live in device memory so one
// instantiated graph serves every call on the graph.
template <typename OffT, bool PARENT>
__global__ void __launch_bounds__(BFS_BLOCK) k_bfs_glevel(const BfsArgs<OffT> *ap) {
    __shared__ LevelState s_st;
    const BfsArgs<OffT> &a = *ap;
    if (threadIdx.x == 0) memcpy(&s_st, (const void *)a.ctl->hstate[0], sizeof(LevelState));
    __syncthreads();
    const LevelState st = s_st;
    if (st.done) return;
    run_phase<OffT, PARENT, false>(a, st, warp_smem<OffT>());
}

template <typename OffT>
__global__ void k_bfs_gtick(const BfsArgs<OffT> *ap, cudaGraphConditionalHandle h) {
    const BfsArgs<OffT> &a = *ap;
    LevelState st;
    memcpy(&st, (const void *)a.ctl->hstate[0], sizeof st);
    const LevelState ns = st.done ? st : next_state(a, st, false);
    memcpy((void *)a.ctl->hstate[0], &ns, sizeof ns);
    if (ns.done) a.ctl->levels_run = ns.L;
    cudaGraphSetConditional(h, ns.done ? 0u : 1u);
}

// Opt every kernel of an instantiation in to its dynamic shared memory size
// (once per process).
template <typename OffT, bool PARENT, bool STATS>
grx_status prepare_kernels() {
    static bool done = false;
    if (done) return GRX_OK;
    const int bytes = (int)bfs_smem_bytes<OffT>();
    GRX_CUDA(cudaFuncSetAttribute((const void *)k_bfs_persistent<OffT, PARENT, STATS>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    GRX_CUDA(cudaFuncSetAttribute((const void *)k_bfs_step<OffT, PARENT, STATS>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    GRX_CUDA(cudaFuncSetAttribute((const void *)k_bfs_step<OffT, PARENT, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    GRX_CUDA(cudaFuncSetAttribute((const void *)k_bfs_glevel<OffT, PARENT>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done = true;
    return GRX_OK;
}

template <typename OffT>
BfsArgs<OffT> make_args(grx_graph *g, int32_t src, int32_t *depth, int32_t *parent,
                        const grx_opts *o) {
    BfsArgs<OffT> a;
    a.nv = g->nv;
    a.ne = g->ne;
    a.words = g->words;
    a.ro = (const OffT *)g->ro;
    a.col = g->col;
    a.nz = g->nz_bits;
    a.visited = g->visited;
    for (int i = 0; i < 3; ++i) {
        a.F[i] = g->fbits[i];
        a.Q[i] = g->qv[i];
        a.E[i] = g->qe[i];
        a.R[i] = (OffT *)g->qr[i];
    }
    a.depth = depth;
    a.parent = parent;
    a.ctl = g->ctl;
    a.bar_flags = g->bar_flags;
    a.stats = g->stats;
    a.mode = o->direction;
    a.exact_fv = o->exact_fv;
    a.alpha = o->alpha;
    a.beta = o->beta;
    // bitmap push when a level's edges reach push_bitmap * nv (0 = 1/8, < 0 = never)
    const double pb = o->push_bitmap == 0.f ? 0.125 : (double)o->push_bitmap;
    if (pb < 0) {
        a.bmp_min_T = 0xffffffffu;
    } else {
        const double t = pb * (double)g->nv;
        a.bmp_min_T = t < 1.0 ? 1u : (t > 4294967295.0 ? 0xffffffffu : (uint32_t)t);
    }
    a.U[0] = g->ulist[0];
    a.U[1] = g->ulist[1];
    a.first2 = g->first2;
    a.ulist_max = (uint32_t)(g->nv / 64 > 0 ? g->nv / 64 : 1);
    a.timeout_ns = grx_timeout_ns(o);
    a.src = src;
    return a;
}

// Build (once per graph and parent flag) the instantiated CUDA graph of the
// level loop: WHILE(cond) { level kernel -> tick kernel }.
template <typename OffT, bool PARENT>
grx_status graph_exec(grx_graph *g, cudaGraphExec_t *out) {
    cudaGraphExec_t &slot = g->bfs_gexec[PARENT ? 1 : 0];
    if (slot) {
        *out = slot;
        return GRX_OK;
    }
    if (!g->bfs_gargs) {
        g->bfs_gargs = grx_alloc(g, sizeof(BfsArgs<int64_t>), (cudaStream_t)g->last_stream);
        if (!g->bfs_gargs) return grx_fail(GRX_ENOMEM, "bfs: graph-mode argument block allocation failed");
    }
    const BfsArgs<OffT> *ap = (const BfsArgs<OffT> *)g->bfs_gargs;
    cudaGraph_t graph = nullptr;
    GRX_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode, n1, n2;
    if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp);
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaKernelNodeParams k1 = {};
        void *a1[] = {(void *)&ap};
        k1.func = (void *)k_bfs_glevel<OffT, PARENT>;
        k1.gridDim = dim3(g->ctx->num_sms * 3);
        k1.blockDim = dim3(BFS_BLOCK);
        k1.sharedMemBytes = (unsigned int)bfs_smem_bytes<OffT>();
        k1.kernelParams = a1;
        e = cudaGraphAddKernelNode(&n1, body, nullptr, 0, &k1);
        cudaKernelNodeParams k2 = {};
        void *a2[] = {(void *)&ap, (void *)&h};
        k2.func = (void *)k_bfs_gtick<OffT>;
        k2.gridDim = dim3(1);
        k2.blockDim = dim3(1);
        k2.kernelParams = a2;
        if (e == cudaSuccess) e = cudaGraphAddKernelNode(&n2, body, &n1, 1, &k2);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&slot, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        slot = nullptr;
        return grx_cuda_fail(e, "bfs: building the level-loop CUDA graph");
    }
    *out = slot;
    return GRX_OK;
}

template <typename OffT, bool PARENT, bool STATS>
grx_status launch_typed(grx_graph *g, int32_t src, int32_t *depth, int32_t *parent,
                        const grx_opts *o, cudaStream_t s) {
    BfsArgs<OffT> a = make_args<OffT>(g, src, depth, parent, o);
    grx_status pst = prepare_kernels<OffT, PARENT, STATS>();
    if (pst != GRX_OK) return pst;
    const size_t smem = bfs_smem_bytes<OffT>();
    if (o->loop == GRX_LOOP_GRAPH) {
        if (STATS) return grx_fail(GRX_EINVAL, "bfs: collect_stats needs the persistent or host loop");
        cudaGraphExec_t ex = nullptr;
        grx_status st = graph_exec<OffT, PARENT>(g, &ex);
        if (st != GRX_OK) return st;
        // arguments of this call (copied before the call returns), then the
        // initialisation launch and the level loop
        GRX_CUDA(cudaMemcpyAsync(g->bfs_gargs, &a, sizeof a, cudaMemcpyHostToDevice, s));
        if (o->ev_begin) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_begin, s));
        k_bfs_step<OffT, PARENT, false><<<g->ctx->num_sms * 3, BFS_BLOCK, smem, s>>>(a, 0);
        GRX_CUDA(cudaGetLastError());
        GRX_CUDA(cudaGraphLaunch(ex, s));
        if (o->ev_end) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_end, s));
        return GRX_OK;
    }
    if (o->loop == GRX_LOOP_HOST) {
        int blocks = o->grid_blocks > 0 ? o->grid_blocks : g->ctx->num_sms * 4;
        // Poll the done flag every 16 launches; a traversal has at most nv
        // levels of at most 3 phases each.
        long long st_host[8];
        if (o->ev_begin) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_begin, s));
        const long long max_launch = 3ll * ((long long)g->nv + 1) + 1;
        for (long long launch = 0; launch <= max_launch; ++launch) {
            k_bfs_step<OffT, PARENT, STATS><<<blocks, BFS_BLOCK, smem, s>>>(a, (int)launch);
            if ((launch & 15) == 15) {
                GRX_CUDA(cudaMemcpyAsync(st_host, (const void *)g->ctl->hstate[launch & 1],
                                         sizeof st_host, cudaMemcpyDeviceToHost, s));
                GRX_CUDA(cudaStreamSynchronize(s));
                LevelState ls;
                memcpy(&ls, st_host, sizeof ls);
                if (ls.done) break;
            }
        }
        if (o->ev_end) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_end, s));
        GRX_CUDA(cudaGetLastError());
        return GRX_OK;
    }
    static int max_blocks_per_sm = -1;
    if (max_blocks_per_sm < 0) {
        GRX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &max_blocks_per_sm, k_bfs_persistent<OffT, PARENT, STATS>, BFS_BLOCK, smem));
        if (max_blocks_per_sm < 1)
            return grx_fail(GRX_ECUDA, "bfs: persistent kernel does not fit on an SM");
    }
    int max_grid = max_blocks_per_sm * g->ctx->num_sms;
    if (max_grid > GRX_MAX_GRID) max_grid = GRX_MAX_GRID;
    int blocks = o->grid_blocks > 0 && o->grid_blocks < max_grid ? o->grid_blocks : max_grid;
    GRX_CUDA(cudaMemsetAsync(g->bar_flags, 0, sizeof(unsigned int) * (size_t)blocks, s));
    GRX_CUDA(cudaMemsetAsync(&g->ctl->bar_release, 0, sizeof(unsigned int), s));
    void *args[] = {(void *)&a};
    if (o->ev_begin) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_begin, s));
    GRX_CUDA(cudaLaunchCooperativeKernel((const void *)k_bfs_persistent<OffT, PARENT, STATS>,
                                         dim3(blocks), dim3(BFS_BLOCK), args, smem, s));
    if (o->ev_end) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_end, s));
    return GRX_OK;
}

template <typename OffT>
grx_status launch_off(grx_graph *g, int32_t src, int32_t *depth, int32_t *parent,
                      const grx_opts *o, cudaStream_t s) {
    const bool stats = o->collect_stats != 0;
    if (parent) {
        return stats ? launch_typed<OffT, true, true>(g, src, depth, parent, o, s)
                     : launch_typed<OffT, true, false>(g, src, depth, parent, o, s);
    }
    return stats ? launch_typed<OffT, false, true>(g, src, depth, parent, o, s)
                 : launch_typed<OffT, false, false>(g, src, depth, parent, o, s);
}

}  // namespace

grx_status grx_bfs_launch(grx_graph *g, int32_t src, int32_t *depth, int32_t *parent,
                          const grx_opts *o, cudaStream_t s) {
    if (o->collect_stats) GRX_CUDA(cudaMemsetAsync(g->stats, 0, sizeof(DevStats), s));
    return g->off64 ? launch_off<int64_t>(g, src, depth, parent, o, s)
                    : launch_off<int32_t>(g, src, depth, parent, o, s);
}
