// BFS and direction-optimising BFS (Algorithms 1 and 2, Sec. 6.1).
//
// Design (one GPU, GB300):
//  * The whole traversal, including the initialisation of the outputs and
//    bitmaps, is one cooperative persistent kernel.  Levels are separated by a
//    flag-based grid barrier with bounded waits, so no host round trip or
//    launch happens per level (the per-iteration overhead l of Sec. 5.2).  A
//    host-stepped variant (one launch per level) exists for comparison.
//  * Work inside a level is warp-independent: no block-wide barrier, so a
//    warp waiting on memory never holds up its neighbours.
//  * Push (top-down): advance and filter are fused (Sec. 6.3).  A frontier
//    slot holds the vertex, its row start and the exclusive prefix of the
//    frontier's degrees; all three come from the append that discovered the
//    vertex (one warp-aggregated atomic), so the next level cuts the
//    frontier's edges into equal warp tiles with no scan pass and reads a
//    tile's rows in one round trip.  Each warp owns a contiguous range of
//    tiles; each lane takes a run of PUSH_ITEMS consecutive edges and keeps
//    their loads, bitmap probes and atomics in flight together.  The visited
//    bitmap is the filter (test, then atomicOr; lanes of a warp that aim at
//    the same vertex send one atomic; the winner labels the vertex).
//  * Pull (bottom-up, Sec. 6.1): each lane takes PULL_PER_LANE unvisited
//    vertices and probes their first PULL_LIGHT neighbours against the
//    frontier bitmap at once; the vertices with longer lists and no hit yet
//    are scanned by groups of PULL_GROUP lanes, PULL_GROUP neighbours per step,
//    stopping at the first hit (edge skipping).  No atomics on labels.  The
//    unvisited set is split into newly discovered vertices (appended, with
//    degree and row start, to the next frontier, so pull->push costs nothing)
//    and the still-unvisited list.
//  * Direction switch (Sec. 6.1): FV = |Q|*E/V, BV = |U|*V/|P|; push->pull
//    once when FV > BV*alpha, pull->push when FV < BV*beta.  With
//    exact_fv = 1, FV is the frontier's exact edge count, which the append
//    atomic already provides.  Every block evaluates the rule identically.
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
constexpr int WARPS = BFS_BLOCK / 32;
constexpr int PUSH_ITEMS = GRX_PUSH_ITEMS;
constexpr int WTILE = 32 * PUSH_ITEMS;              // edges per warp tile
constexpr int PULL_LIGHT = 2;                       // neighbours probed per vertex first
constexpr int PULL_PER_LANE = 4;
constexpr int PULL_WCH = 32 * PULL_PER_LANE;        // candidates per warp chunk
constexpr int PULL_GROUP = 8;                       // lanes per long list

enum { DIR_PUSH = 0, DIR_PULL = 1 };

struct LevelState {
    int L;            // level being expanded (frontier = vertices at depth L)
    int dir;
    int switched;     // push->pull has happened
    int back;         // pull->push has happened (final)
    int first_pull;   // pull level without an unvisited list yet: scan the bitmaps
    int fwrite;       // this level sets F_{L+1} bits for discovered vertices
    int fprev;        // F_L holds the frontier's bits
    int fclear;       // this level clears F_{L-1} (word by word from Q_{L-1})
    int done;
    uint32_t q, T;    // |Q_L| and its edge count
    uint32_t qprev;   // |Q_{L-1}|
    uint32_t ucount;  // unvisited-list length (non-first pull levels)
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
    int32_t *U[2];
    int32_t *depth;
    int32_t *parent;
    TravCtl *ctl;
    unsigned int *bar_flags;
    DevStats *stats;
    int mode;
    int exact_fv;
    float alpha, beta;
    unsigned long long timeout_ns;
    int32_t src;
};

template <typename OffT>
struct PushWarpSmem {
    uint32_t qe[WTILE + 2];
    int32_t u[WTILE + 1];
    OffT rs[WTILE + 1];
};

template <typename OffT>
struct PullWarpSmem {
    int32_t slot[PULL_WCH];
    OffT hb[PULL_WCH];
    OffT he[PULL_WCH];
    int32_t hpar[PULL_WCH];
};

template <typename OffT>
union WarpSmem {
    PushWarpSmem<OffT> p;
    PullWarpSmem<OffT> l;
};

template <typename OffT>
__device__ LevelState initial_state(const BfsArgs<OffT> &a) {
    LevelState s;
    s.L = 0;
    s.dir = a.mode == GRX_DIR_PULL ? DIR_PULL : DIR_PUSH;
    s.switched = a.mode == GRX_DIR_PULL;
    s.back = 0;
    s.first_pull = a.mode == GRX_DIR_PULL;
    s.fwrite = a.mode != GRX_DIR_PUSH;
    s.fprev = a.mode != GRX_DIR_PUSH;
    s.fclear = 0;
    s.done = 0;
    uint32_t deg = (uint32_t)(__ldg(a.ro + a.src + 1) - __ldg(a.ro + a.src));
    s.q = deg > 0 ? 1u : 0u;
    s.T = deg;
    s.qprev = 0;
    s.ucount = 0;
    s.vcount = 1;
    if (s.q == 0) s.done = 1;
    return s;
}

// State of level L+1 from the state of level L and the counters level L left.
template <typename OffT>
__device__ LevelState next_state(const BfsArgs<OffT> &a, const LevelState &st, bool stats) {
    LevelState ns = st;
    ns.L = st.L + 1;
    unsigned long long pk = ld_relaxed_u64(&a.ctl->qpack[(st.L + 1) & 3]);
    ns.q = (uint32_t)(pk >> 32);
    ns.T = (uint32_t)pk;
    ns.qprev = st.q;
    ns.ucount = ld_relaxed_u32(&a.ctl->ucount[(st.L + 1) & 3]);
    ns.vcount = st.vcount + ns.q;
    ns.fclear = st.fprev;
    ns.fprev = st.fwrite;
    if (stats && blockIdx.x == 0 && st.L < GRX_MAX_LEVELS_STATS) a.stats->discovered[st.L] = ns.q;
    if (ns.q == 0) {
        ns.done = 1;
        return ns;
    }
    ns.first_pull = 0;
    if (a.mode == GRX_DIR_PUSH) {
        ns.dir = DIR_PUSH;
        ns.fwrite = 0;
    } else if (a.mode == GRX_DIR_PULL) {
        ns.dir = DIR_PULL;
        ns.fwrite = 1;
    } else {
        // Sec. 6.1: FV = |Q|*E/V (or the exact frontier edge count), BV = |U|*V/|P|
        double V = (double)a.nv, E = (double)a.ne;
        double FV = a.exact_fv ? (double)ns.T : (double)ns.q * E / V;
        double BV = (double)(a.nv - (long long)ns.vcount) * V / (double)ns.vcount;
        if (st.dir == DIR_PUSH && !st.switched && FV > BV * (double)a.alpha) {
            ns.dir = DIR_PULL;
            ns.switched = 1;
            ns.first_pull = 1;
        } else if (st.dir == DIR_PULL && FV < BV * (double)a.beta) {
            ns.dir = DIR_PUSH;
            ns.back = 1;
        }
        ns.fwrite = !ns.back;
    }
    return ns;
}

template <typename OffT, bool PARENT, bool STATS>
__device__ void push_level(const BfsArgs<OffT> &a, const LevelState &st, PushWarpSmem<OffT> &w) {
    const int L = st.L;
    const unsigned int lane = threadIdx.x & 31;
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
                w.u[n + lane] = __ldcg(Qv + idx);
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
        // a run of PUSH_ITEMS consecutive edges per lane
        const uint64_t t0 = e0 + (uint64_t)lane * PUSH_ITEMS;
        int32_t v[PUSH_ITEMS];
        int32_t par[PUSH_ITEMS];
        uint32_t valid = 0;
#pragma unroll
        for (int k = 0; k < PUSH_ITEMS; ++k) {
            v[k] = 0;
            par[k] = 0;
        }
        if (t0 < e1) {
            int j = upper_index_smem(w.qe, n, (uint32_t)t0);
#pragma unroll
            for (int k = 0; k < PUSH_ITEMS; ++k) {
                const uint32_t e = (uint32_t)t0 + k;
                if (e < e1) {
                    while (w.qe[j + 1] <= e) ++j;
                    v[k] = __ldg(a.col + w.rs[j] + (OffT)(e - w.qe[j]));
                    if (PARENT) par[k] = w.u[j];
                    valid |= 1u << k;
                }
            }
        }
        uint32_t wv[PUSH_ITEMS];
#pragma unroll
        for (int k = 0; k < PUSH_ITEMS; ++k)
            wv[k] = (valid >> k & 1u) ? __ldcg(a.visited + (v[k] >> 5)) : 0xffffffffu;
        uint32_t cand = 0;
#pragma unroll
        for (int k = 0; k < PUSH_ITEMS; ++k) {
            const bool c = !((wv[k] >> (v[k] & 31)) & 1u);
#if GRX_PUSH_DEDUP
            // lanes aiming at the same vertex: only the lowest one tries to claim it
            const unsigned int same = __match_any_sync(GRX_FULL_MASK, c ? v[k] : -1 - (int)lane);
            if (c && (same & lanemask_lt()) == 0) cand |= 1u << k;
#else
            if (c) cand |= 1u << k;
#endif
        }
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
        // the element holding e1 starts the next tile
        i0 = (next_start == e1) ? i0 + n : i0 + n - 1;
        __syncwarp();
    }
}

template <typename OffT, bool PARENT, bool STATS>
__device__ void pull_level(const BfsArgs<OffT> &a, const LevelState &st, PullWarpSmem<OffT> &w,
                           unsigned long long &scanned_e, unsigned long long &scanned_v) {
    const int L = st.L;
    const unsigned int lane = threadIdx.x & 31;
    const uint32_t *Fin = pick3(a.F[0], a.F[1], a.F[2], L % 3);
    uint32_t *Fout = pick3(a.F[0], a.F[1], a.F[2], (L + 1) % 3);
    int32_t *Qv_out = pick3(a.Q[0], a.Q[1], a.Q[2], (L + 1) % 3);
    uint32_t *Qe_out = pick3(a.E[0], a.E[1], a.E[2], (L + 1) % 3);
    OffT *Qr_out = pick3(a.R[0], a.R[1], a.R[2], (L + 1) % 3);
    unsigned long long *ctr = &a.ctl->qpack[(L + 1) & 3];
    const int32_t *Uin = (L & 1) ? a.U[1] : a.U[0];
    int32_t *Uout = (L & 1) ? a.U[0] : a.U[1];
    unsigned int *uctr = &a.ctl->ucount[(L + 1) & 3];
    const bool first = st.first_pull != 0;
    const int64_t nchunks = first ? (a.words + PULL_PER_LANE - 1) / PULL_PER_LANE
                                  : ((int64_t)st.ucount + PULL_WCH - 1) / PULL_WCH;
    const int64_t nwarps = (int64_t)gridDim.x * WARPS;
    const int64_t gw = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    for (int64_t c = gw; c < nchunks; c += nwarps) {
        // 1. candidates: lane takes vertex k*32+lane of the chunk
        int32_t v[PULL_PER_LANE];
        if (first) {
            uint32_t any = 0;
#pragma unroll
            for (int k = 0; k < PULL_PER_LANE; ++k) {
                const int64_t wd = c * PULL_PER_LANE + k;
                const uint32_t bits = wd < a.words ? (__ldg(a.nz + wd) & ~__ldcg(a.visited + wd)) : 0u;
                any |= bits;
                v[k] = ((bits >> lane) & 1u) ? (int32_t)(wd * 32 + lane) : -1;
            }
            if (any == 0) continue;                  // same words in every lane
        } else {
#pragma unroll
            for (int k = 0; k < PULL_PER_LANE; ++k) {
                const int64_t i = c * PULL_WCH + k * 32 + lane;
                v[k] = i < (int64_t)st.ucount ? __ldcg(Uin + i) : -1;
            }
        }
        // 2. light phase: the first PULL_LIGHT neighbours of every candidate, all in flight
        OffT b[PULL_PER_LANE], e[PULL_PER_LANE];
#pragma unroll
        for (int k = 0; k < PULL_PER_LANE; ++k) {
            b[k] = 0;
            e[k] = 0;
            if (v[k] >= 0) {
                b[k] = __ldg(a.ro + v[k]);
                e[k] = __ldg(a.ro + v[k] + 1);
            }
        }
        int32_t u0[PULL_PER_LANE], u1[PULL_PER_LANE];
#pragma unroll
        for (int k = 0; k < PULL_PER_LANE; ++k) {
            u0[k] = b[k] < e[k] ? __ldg(a.col + b[k]) : -1;
            u1[k] = b[k] + 1 < e[k] ? __ldg(a.col + b[k] + 1) : -1;
        }
        uint32_t f0[PULL_PER_LANE], f1[PULL_PER_LANE];
#pragma unroll
        for (int k = 0; k < PULL_PER_LANE; ++k) {
            f0[k] = u0[k] >= 0 ? __ldcg(Fin + (u0[k] >> 5)) : 0u;
            f1[k] = u1[k] >= 0 ? __ldcg(Fin + (u1[k] >> 5)) : 0u;
        }
        int32_t par[PULL_PER_LANE];
        uint32_t heavy = 0;
#pragma unroll
        for (int k = 0; k < PULL_PER_LANE; ++k) {
            par[k] = -1;
            if (u0[k] >= 0 && ((f0[k] >> (u0[k] & 31)) & 1u)) par[k] = u0[k];
            else if (u1[k] >= 0 && ((f1[k] >> (u1[k] & 31)) & 1u)) par[k] = u1[k];
            if (STATS && v[k] >= 0) {
                scanned_v += 1;
                scanned_e += (unsigned long long)min((OffT)PULL_LIGHT, e[k] - b[k]);
            }
            if (v[k] >= 0 && par[k] < 0 && e[k] - b[k] > PULL_LIGHT) heavy |= 1u << k;
        }
        // 3. heavy phase: the warp's longer lists, PULL_GROUP lanes each
        int nh = 0;
        int hpos[PULL_PER_LANE];
#pragma unroll
        for (int k = 0; k < PULL_PER_LANE; ++k) {
            const unsigned int m = __ballot_sync(GRX_FULL_MASK, heavy >> k & 1u);
            hpos[k] = nh + __popc(m & lanemask_lt());
            if (heavy >> k & 1u) {
                w.hb[hpos[k]] = b[k] + PULL_LIGHT;
                w.he[hpos[k]] = e[k];
            }
            nh += __popc(m);
        }
        __syncwarp();
        const int grp = (int)(lane / PULL_GROUP), gl = (int)(lane % PULL_GROUP);
        for (int h0 = 0; h0 < nh; h0 += 32 / PULL_GROUP) {
            const int h = h0 + grp;
            OffT hb = 0, he = 0;
            if (h < nh) {
                hb = w.hb[h];
                he = w.he[h];
            }
            int32_t found = -1;
            bool done = h >= nh;
            while (__any_sync(GRX_FULL_MASK, !done)) {
                int32_t uu = -1;
                bool hit = false;
                if (!done && hb + gl < he) {
                    uu = __ldg(a.col + hb + gl);
                    hit = (__ldcg(Fin + (uu >> 5)) >> (uu & 31)) & 1u;
                }
                const unsigned int gm = (__ballot_sync(GRX_FULL_MASK, hit) >> (grp * PULL_GROUP)) &
                                        ((1u << PULL_GROUP) - 1u);
                const int32_t first_hit =
                    __shfl_sync(GRX_FULL_MASK, uu, grp * PULL_GROUP + (gm ? __ffs(gm) - 1 : 0));
                if (!done) {
                    if (STATS && gl == 0)
                        scanned_e += (unsigned long long)(gm ? __ffs(gm) : min((OffT)PULL_GROUP, he - hb));
                    if (gm) {
                        found = first_hit;
                        done = true;
                    } else {
                        hb += PULL_GROUP;
                        done = hb >= he;
                    }
                }
            }
            if (h < nh && gl == 0) w.hpar[h] = found;
        }
        __syncwarp();
        // 4. label the found vertices; append found / still-unvisited
        uint32_t fmask = 0, smask = 0;
        uint32_t deg[PULL_PER_LANE];
#pragma unroll
        for (int k = 0; k < PULL_PER_LANE; ++k) {
            if (heavy >> k & 1u) par[k] = w.hpar[hpos[k]];
            deg[k] = (uint32_t)(e[k] - b[k]);
            const bool fnd = v[k] >= 0 && par[k] >= 0;
            if (fnd) {
                a.depth[v[k]] = L + 1;
                if (PARENT) a.parent[v[k]] = par[k];
                fmask |= 1u << k;
            } else if (v[k] >= 0) {
                smask |= 1u << k;
            }
            if (first) {
                // slot k of every lane lies in the same bitmap word: one atomic per word
                const uint32_t bits = __reduce_or_sync(GRX_FULL_MASK, fnd ? 1u << lane : 0u);
                if (lane == 0 && bits) {
                    const int64_t wd = c * PULL_PER_LANE + k;
                    atomicOr(a.visited + wd, bits);
                    if (st.fwrite) atomicOr(Fout + wd, bits);
                }
            } else if (fnd) {
                const uint32_t bit = 1u << (v[k] & 31);
                atomicOr(a.visited + (v[k] >> 5), bit);
                if (st.fwrite) atomicOr(Fout + (v[k] >> 5), bit);
            }
        }
        warp_append_items<PULL_PER_LANE, OffT>(v, deg, b, fmask, Qv_out, Qe_out, Qr_out, ctr);
        warp_append_list_items<PULL_PER_LANE>(v, smask, Uout, uctr);
        __syncwarp();
    }
}

template <typename OffT, bool PARENT, bool STATS>
__device__ void run_level(const BfsArgs<OffT> &a, const LevelState &st, WarpSmem<OffT> &w) {
    const int L = st.L;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->qpack[(L + 2) & 3] = 0ull;
        a.ctl->ucount[(L + 2) & 3] = 0u;
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
    if (st.fclear) {
        // F_{L-1} only holds bits of Q_{L-1}'s vertices: zero their words.
        const int32_t *Qp = pick3(a.Q[0], a.Q[1], a.Q[2], (L + 2) % 3);
        uint32_t *Fp = pick3(a.F[0], a.F[1], a.F[2], (L + 2) % 3);
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)st.qprev;
             i += (int64_t)gridDim.x * blockDim.x)
            Fp[__ldcg(Qp + i) >> 5] = 0u;
    }
    if (st.dir == DIR_PUSH) {
        push_level<OffT, PARENT, STATS>(a, st, w.p);
    } else {
        unsigned long long scanned_e = 0, scanned_v = 0;
        pull_level<OffT, PARENT, STATS>(a, st, w.l, scanned_e, scanned_v);
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

// Phase 0 of a traversal: depth = -1 (0 at src), parent = -1 (src at src),
// visited = {src}, frontier bitmaps = {src} / empty, the frontier counters
// and the first frontier slot.  Every word is written by exactly one thread,
// so clearing and seeding need no barrier between them.
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
    const bool use_f = a.mode != GRX_DIR_PUSH;
    for (int64_t w = tid; w < a.words; w += stride) {
        a.visited[w] = w == sw ? sb : 0u;
        if (use_f) {
            a.F[0][w] = (w == sw && st0.q) ? sb : 0u;
            a.F[1][w] = 0u;
            a.F[2][w] = 0u;
        }
    }
    if (tid == 0) {
        a.Q[0][0] = src;
        a.E[0][0] = 0;
        a.R[0][0] = __ldg(a.ro + src);
        a.ctl->qpack[0] = st0.q ? ((1ull << 32) | st0.T) : 0ull;
        for (int i = 1; i < 4; ++i) a.ctl->qpack[i] = 0ull;
        for (int i = 0; i < 4; ++i) a.ctl->ucount[i] = 0u;
    }
}

template <typename OffT, bool PARENT, bool STATS>
__global__ void __launch_bounds__(BFS_BLOCK, 3) k_bfs_persistent(BfsArgs<OffT> a) {
    __shared__ LevelState s_st;
    __shared__ WarpSmem<OffT> wsm[WARPS];
    WarpSmem<OffT> &w = wsm[threadIdx.x >> 5];
    FlagBarrier bar{a.bar_flags, &a.ctl->bar_release, a.ctl, a.timeout_ns, 0u};
    if (threadIdx.x == 0) s_st = initial_state(a);
    __syncthreads();
    init_phase<OffT, PARENT>(a, s_st);
    if (!flag_barrier(bar)) return;
    for (;;) {
        const LevelState st = s_st;
        if (st.done) break;
        run_level<OffT, PARENT, STATS>(a, st, w);
        if (!flag_barrier(bar)) return;
        if (threadIdx.x == 0) s_st = next_state(a, st, STATS);
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->levels_run = s_st.L;
        if (STATS && s_st.L <= GRX_MAX_LEVELS_STATS) a.stats->level_t0[s_st.L] = grx_globaltimer();
    }
}

// Host-stepped variant: launch 0 initialises, launch i >= 1 runs level i-1.
// The state of a level is derived at the start of its launch from the state
// the previous launch stored and the counters it left, so no block ever
// waits on another.
template <typename OffT, bool PARENT, bool STATS>
__global__ void __launch_bounds__(BFS_BLOCK) k_bfs_step(BfsArgs<OffT> a, int launch) {
    __shared__ LevelState s_st;
    __shared__ WarpSmem<OffT> wsm[WARPS];
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
    run_level<OffT, PARENT, STATS>(a, st, wsm[threadIdx.x >> 5]);
}

// CUDA-graph variant: the body of a device-evaluated WHILE node is one level
// kernel followed by a one-thread tick that derives the next level's state
// and sets the loop condition.  The arguments live in device memory so one
// instantiated graph serves every call on the graph.
template <typename OffT, bool PARENT>
__global__ void __launch_bounds__(BFS_BLOCK) k_bfs_glevel(const BfsArgs<OffT> *ap) {
    __shared__ LevelState s_st;
    __shared__ WarpSmem<OffT> wsm[WARPS];
    const BfsArgs<OffT> &a = *ap;
    if (threadIdx.x == 0) memcpy(&s_st, (const void *)a.ctl->hstate[0], sizeof(LevelState));
    __syncthreads();
    const LevelState st = s_st;
    if (st.done) return;
    run_level<OffT, PARENT, false>(a, st, wsm[threadIdx.x >> 5]);
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
    a.U[0] = g->ulist[0];
    a.U[1] = g->ulist[1];
    a.depth = depth;
    a.parent = parent;
    a.ctl = g->ctl;
    a.bar_flags = g->bar_flags;
    a.stats = g->stats;
    a.mode = o->direction;
    a.exact_fv = o->exact_fv;
    a.alpha = o->alpha;
    a.beta = o->beta;
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
    if (o->loop == GRX_LOOP_GRAPH) {
        if (STATS) return grx_fail(GRX_EINVAL, "bfs: collect_stats needs the persistent or host loop");
        cudaGraphExec_t ex = nullptr;
        grx_status st = graph_exec<OffT, PARENT>(g, &ex);
        if (st != GRX_OK) return st;
        // arguments of this call (copied before the call returns), then the
        // initialisation launch and the level loop
        GRX_CUDA(cudaMemcpyAsync(g->bfs_gargs, &a, sizeof a, cudaMemcpyHostToDevice, s));
        if (o->ev_begin) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_begin, s));
        k_bfs_step<OffT, PARENT, false><<<g->ctx->num_sms * 3, BFS_BLOCK, 0, s>>>(a, 0);
        GRX_CUDA(cudaGetLastError());
        GRX_CUDA(cudaGraphLaunch(ex, s));
        if (o->ev_end) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_end, s));
        return GRX_OK;
    }
    if (o->loop == GRX_LOOP_HOST) {
        int blocks = o->grid_blocks > 0 ? o->grid_blocks : g->ctx->num_sms * 4;
        // Poll the done flag every 16 launches; a traversal has at most nv levels.
        long long st_host[8];
        if (o->ev_begin) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_begin, s));
        for (int launch = 0; launch <= g->nv + 1; ++launch) {
            k_bfs_step<OffT, PARENT, STATS><<<blocks, BFS_BLOCK, 0, s>>>(a, launch);
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
            &max_blocks_per_sm, k_bfs_persistent<OffT, PARENT, STATS>, BFS_BLOCK, 0));
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
                                         dim3(blocks), dim3(BFS_BLOCK), args, 0, s));
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
