// Batched betweenness centrality: up to 64 sources share one forward and one
// backward sweep (the lane scheme of the 64-lane multi-source BFS applied to
// Table 1's BC; per lane the result is Brandes' dependency of that source,
// and bc_out is their sum).
//
// Per vertex v: seen[v] / next[v] (64-bit lane masks), hist[k][v] = lanes in
// which v sits at depth k (kept for every level, BCM_MAX_LEVELS at most),
// and vertex-major float64 rows sig[v][64] (path counts) and acc[v][64]
// (successor sums, then coefficients (1 + delta) / sigma), so one edge's
// lanes are one coalesced row.
//
//  * Forward level k: equal warp tiles over the list of vertices with
//    hist[k] != 0; an edge (u, w) is a shortest-path edge for the lanes
//    m = hist[k][u] & ~seen[w]: next[w] |= m and w's bit goes into a touched
//    bitmap (reductions), and the warp adds sig[u][b] to sig[w][b] for every
//    lane b of m (float64 reductions, one row per edge).  A second phase, by
//    owners of 32-word chunks of the bitmap, moves next into seen and
//    hist[k + 1] and lists the touched vertices (vertex order).
//  * Backward, from the deepest level D up to 1: level k is finished (per
//    lane b of hist[k][v]: delta = sig * acc is added to bc[v], acc becomes
//    1 / sig + acc) while the list of level k - 1 is rebuilt from hist; then
//    level k's vertices w push acc[w][b] (their coefficients) into acc[v][b]
//    along edges with b in hist[k][w] & hist[k - 1][v] (float64 reductions).
// Every value is per lane and every lane's phases are ordered by the grid
// barrier, so no lane reads another's partial values.  One persistent
// cooperative kernel; every wait bounded.
#include "grx_internal.cuh"

namespace {

constexpr int BCM_BLOCK = 128;
constexpr int BCM_WARPS = BCM_BLOCK / 32;
constexpr int BCM_ITEMS = 8;
constexpr int BCM_WTILE = 32 * BCM_ITEMS;
static_assert(BCM_WTILE == 256, "warp_tile_rows8 covers 256-position tiles");

template <typename OffT>
struct BcmArgs {
    int32_t nv;
    int64_t words;
    const OffT *ro;
    const int32_t *col;
    unsigned long long *seen, *next;     // [nv] lane masks
    unsigned long long *hist;            // [GRX_BCM_MAX_LEVELS][nv]
    uint32_t *touched;                   // [words]
    double *sig, *acc;                   // [nv][64]
    double *bc;
    int32_t *Q[2];
    uint32_t *E[2];
    OffT *R[2];
    TravCtl *ctl;
    unsigned int *bar_flags;
    DevStats *stats;                     // NULL, or per-phase statistics
    unsigned long long timeout_ns;
};

enum { MOP_EXPAND, MOP_FINAL, MOP_FIN_BUILD, MOP_PUSH };

struct BcmState {
    int op;
    int k;                     // level
    int cur;                   // list buffer of level k (EXPAND/FINAL/FIN_BUILD) or k + 1 (PUSH)
    int done;
    int phase;
    uint32_t q, T;             // list in Q[cur]
    uint32_t q2, T2;           // PUSH: level k's list in Q[cur ^ 1]
};

struct DagEntry {
    int32_t dst, src;
    unsigned long long m;
};

template <typename OffT>
struct BcmWarpSmem {
    uint32_t qe[BCM_WTILE + 2];
    OffT rs[BCM_WTILE + 1];
    int32_t u[BCM_WTILE + 1];
    unsigned long long f[BCM_WTILE + 1];
    alignas(16) uint16_t rid[BCM_WTILE];
    union {
        DagEntry dag[BCM_WTILE];        // edge phases: the tile's shortest-path edges
        uint16_t list[32 * 32];         // finalize: compacted bits of a 32-word chunk
    };
};

__device__ __forceinline__ unsigned long long *hist_level(const BcmArgs<int32_t> &a, int k) {
    return a.hist + (size_t)k * (size_t)a.nv;
}
__device__ __forceinline__ unsigned long long *hist_level(const BcmArgs<int64_t> &a, int k) {
    return a.hist + (size_t)k * (size_t)a.nv;
}

// The warp adds src[b] into dst[b] for the lanes b of each listed edge,
// BCM_DAG_BATCH edges at a time: their loads are all in flight before the
// reductions go out.
constexpr int BCM_DAG_BATCH = 8;
__device__ __forceinline__ void dag_rows(const DagEntry *dag, int cnt, double *base_dst, const double *base_src) {
    const unsigned int lane = threadIdx.x & 31;
    for (int i = 0; i < cnt; i += BCM_DAG_BATCH) {
        double x0[BCM_DAG_BATCH], x1[BCM_DAG_BATCH];
        unsigned long long mm[BCM_DAG_BATCH];
        int32_t dd[BCM_DAG_BATCH];
#pragma unroll
        for (int j = 0; j < BCM_DAG_BATCH; ++j) {
            mm[j] = 0ull;
            dd[j] = 0;
            x0[j] = 0.0;
            x1[j] = 0.0;
            if (i + j < cnt) {
                const DagEntry e = dag[i + j];
                mm[j] = e.m;
                dd[j] = e.dst;
                const double *src = base_src + (size_t)e.src * 64;
                if ((e.m >> lane) & 1ull) x0[j] = __ldcg(src + lane);
                if ((e.m >> (lane + 32)) & 1ull) x1[j] = __ldcg(src + lane + 32);
            }
        }
#pragma unroll
        for (int j = 0; j < BCM_DAG_BATCH; ++j) {
            double *dst = base_dst + (size_t)dd[j] * 64;
            if ((mm[j] >> lane) & 1ull) atomicAdd(dst + lane, x0[j]);                 // reductions
            if ((mm[j] >> (lane + 32)) & 1ull) atomicAdd(dst + lane + 32, x1[j]);
        }
    }
}

// One level's edges in equal warp tiles.  FWD: shortest-path lanes are the
// source's hist[k] lanes not yet seen at the target; BACK: the source's
// hist[k + 1] lanes in which the target sits at depth k.
template <typename OffT, bool FWD>
__device__ void level_edges(const BcmArgs<OffT> &a, const BcmState &st, BcmWarpSmem<OffT> &w,
                            unsigned long long &lane_edges) {
    const unsigned int lane = threadIdx.x & 31;
    const int ksrc = FWD ? st.k : st.k + 1;
    const unsigned long long *hsrc = hist_level(a, ksrc);
    const unsigned long long *hdst = FWD ? nullptr : hist_level(a, st.k);
    const int32_t *Qv = a.Q[st.cur];
    const uint32_t *Qe = a.E[st.cur];
    const OffT *Qr = a.R[st.cur];
    const int64_t q = st.q;
    const uint64_t T = st.T;
    const uint64_t ntiles = (T + BCM_WTILE - 1) / BCM_WTILE;
    const uint64_t nwarps = (uint64_t)gridDim.x * BCM_WARPS;
    const uint64_t gw = (uint64_t)blockIdx.x * BCM_WARPS + (threadIdx.x >> 5);
    const uint64_t per = (ntiles + nwarps - 1) / nwarps;
    const uint64_t tb0 = gw * per;
    const uint64_t tb1 = min(ntiles, tb0 + per);
    if (tb0 >= tb1) return;
    int64_t i0 = warp_upper_index_cg(Qe, q, (uint32_t)(tb0 * BCM_WTILE));
    for (uint64_t tile = tb0; tile < tb1; ++tile) {
        const uint64_t e0 = tile * BCM_WTILE;
        const uint32_t e1 = (uint32_t)min(T, e0 + BCM_WTILE);
        int n = 0;
        for (;;) {
            const int64_t idx = i0 + n + lane;
            uint32_t qe = 0xffffffffu;
            if (idx < q) qe = __ldcg(Qe + idx);
            const bool in = idx < q && qe < e1;
            if (n + (int)lane <= BCM_WTILE + 1) w.qe[n + lane] = qe;
            if (in && n + (int)lane <= BCM_WTILE) {
                const int32_t u = __ldcg(Qv + idx);
                w.rs[n + lane] = __ldcg(Qr + idx);
                w.u[n + lane] = u;
                w.f[n + lane] = __ldcg(hsrc + u);
            }
            const int cnt = __popc(__ballot_sync(GRX_FULL_MASK, in));
            n += cnt;
            if (cnt < 32) break;
            if (n > BCM_WTILE) {                 // only possible with a malformed graph
                if (lane == 0) grx_set_status(a.ctl, GRX_EINVAL);
                n = BCM_WTILE;
                break;
            }
        }
        __syncwarp();
        const uint32_t next_start = w.qe[n];
        int row[BCM_ITEMS];
        warp_tile_rows8(w.rid, w.qe, (uint32_t)e0, n, row);
        const uint32_t t0 = (uint32_t)e0 + lane * BCM_ITEMS;
        int32_t v[BCM_ITEMS];
        int32_t us[BCM_ITEMS];
        unsigned long long fs[BCM_ITEMS];
#pragma unroll
        for (int k = 0; k < BCM_ITEMS; ++k) {
            const uint32_t e = t0 + k;
            const int j = row[k];
            const bool ok = e < e1;
            const OffT idx = ok ? w.rs[j] + (OffT)(e - w.qe[j]) : (OffT)0;
            v[k] = ok ? __ldg(a.col + idx) : -1;
            us[k] = ok ? w.u[j] : 0;
            fs[k] = ok ? w.f[j] : 0ull;
        }
        unsigned long long m[BCM_ITEMS];
#pragma unroll
        for (int k = 0; k < BCM_ITEMS; ++k) {
            m[k] = 0ull;
            if (v[k] >= 0) m[k] = FWD ? fs[k] & ~__ldcg(a.seen + v[k]) : fs[k] & __ldcg(hdst + v[k]);
        }
        if (FWD) {
#pragma unroll
            for (int k = 0; k < BCM_ITEMS; ++k) {
                if (m[k]) {
                    atomicOr(a.next + v[k], m[k]);                                 // reductions
                    atomicOr(a.touched + (v[k] >> 5), 1u << (v[k] & 31));
                }
            }
        }
        // list the tile's shortest-path edges, then update their lanes' rows
        __syncwarp();
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < BCM_ITEMS; ++k) {
            const unsigned int bal = __ballot_sync(GRX_FULL_MASK, m[k] != 0ull);
            if (m[k]) {
                const int pos = cnt + __popc(bal & lanemask_lt());
                // forward: sig[target] += sig[source]; backward: acc[target] += acc[source]
                w.dag[pos] = DagEntry{v[k], us[k], m[k]};
                if (a.stats) lane_edges += (unsigned long long)__popcll(m[k]);
            }
            cnt += __popc(bal);
        }
        __syncwarp();
        if (FWD) dag_rows(w.dag, cnt, a.sig, a.sig);
        else dag_rows(w.dag, cnt, a.acc, a.acc);
        i0 = (next_start == e1) ? i0 + n : i0 + n - 1;
        __syncwarp();
    }
}

// Forward, second phase of level k: touched vertices take their new lanes.
template <typename OffT>
__device__ void forward_final(const BcmArgs<OffT> &a, const BcmState &st, uint16_t *list) {
    const int k1 = st.k + 1;
    const bool fits = k1 < GRX_BCM_MAX_LEVELS;
    unsigned long long *h1 = hist_level(a, fits ? k1 : 0);
    int32_t *Qv = a.Q[st.cur ^ 1];
    uint32_t *Qe = a.E[st.cur ^ 1];
    OffT *Qr = a.R[st.cur ^ 1];
    unsigned long long *ctr = &a.ctl->qpack[k1 & 3];
    const unsigned int lane = threadIdx.x & 31;
    const int64_t nsc = (a.words + 31) / 32;
    const int64_t nwarps = (int64_t)gridDim.x * BCM_WARPS;
    for (int64_t sc = (int64_t)blockIdx.x * BCM_WARPS + (threadIdx.x >> 5); sc < nsc; sc += nwarps) {
        const int64_t wd = sc * 32 + lane;
        uint32_t bits = wd < a.words ? __ldcg(a.touched + wd) : 0u;
        if (bits) {
            a.touched[wd] = 0u;
            if (!fits) {
                grx_set_status(a.ctl, GRX_ERANGE);               // deeper than the level masks
                bits = 0u;
            }
        }
        const int n = warp_compact_bits(bits, list);
        for (int base = 0; base < n; base += 32) {
            const int i = base + (int)lane;
            int32_t v[1] = {0};
            uint32_t deg[1] = {0};
            OffT rb[1] = {0};
            uint32_t app = 0;
            if (i < n) {
                v[0] = (int32_t)(sc * 1024 + list[i]);
                const unsigned long long nx = __ldcg(a.next + v[0]);
                a.next[v[0]] = 0ull;
                a.seen[v[0]] = __ldcg(a.seen + v[0]) | nx;
                h1[v[0]] = nx;
                rb[0] = __ldg(a.ro + v[0]);
                deg[0] = (uint32_t)(__ldg(a.ro + v[0] + 1) - rb[0]);
                if (deg[0]) app = 1;
            }
            warp_append_items<1, OffT>(v, deg, rb, app, Qv, Qe, Qr, ctr);
        }
        __syncwarp();
    }
}

// Backward, level k: its vertices finish (one warp per vertex, two lanes of
// the 64 per thread); the list of level k - 1 is rebuilt from hist.
template <typename OffT>
__device__ void finish_and_build(const BcmArgs<OffT> &a, const BcmState &st) {
    const unsigned int lane = threadIdx.x & 31;
    const int64_t gwarp = (int64_t)blockIdx.x * BCM_WARPS + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * BCM_WARPS;
    const unsigned long long *hk = hist_level(a, st.k);
    const int32_t *Qv = a.Q[st.cur];
    constexpr int VB = 4;                                // vertices per warp pass, loads in flight together
    for (int64_t i0 = gwarp * VB; i0 < (int64_t)st.q; i0 += nwarps * VB) {
        int32_t v[VB];
        unsigned long long hv[VB];
#pragma unroll
        for (int j = 0; j < VB; ++j) v[j] = i0 + j < (int64_t)st.q ? __ldcg(Qv + i0 + j) : -1;
#pragma unroll
        for (int j = 0; j < VB; ++j) hv[j] = v[j] >= 0 ? __ldcg(hk + v[j]) : 0ull;
        double s[VB][2], sg[VB][2];
#pragma unroll
        for (int j = 0; j < VB; ++j) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int b = (int)lane + 32 * h;
                s[j][h] = 0.0;
                sg[j][h] = 1.0;
                if ((hv[j] >> b) & 1ull) {
                    const size_t ix = (size_t)v[j] * 64 + b;
                    s[j][h] = __ldcg(a.acc + ix);
                    sg[j][h] = __ldcg(a.sig + ix);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < VB; ++j) {
            double part = 0.0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int b = (int)lane + 32 * h;
                if ((hv[j] >> b) & 1ull) {
                    part += sg[j][h] * s[j][h];
                    a.acc[(size_t)v[j] * 64 + b] = 1.0 / sg[j][h] + s[j][h];
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(GRX_FULL_MASK, part, o);
            if (lane == 0 && part != 0.0) a.bc[v[j]] += part;   // v is in this level's list once
        }
    }
    if (st.k <= 1) return;                               // level 0 holds the sources: not needed
    const unsigned long long *hp = hist_level(a, st.k - 1);
    int32_t *Qo = a.Q[st.cur ^ 1];
    uint32_t *Eo = a.E[st.cur ^ 1];
    OffT *Ro = a.R[st.cur ^ 1];
    unsigned long long *ctr = &a.ctl->qpack[(st.k - 1) & 3];
    for (int64_t base = gwarp * 32; base < a.nv; base += nwarps * 32) {
        const int64_t vv = base + lane;
        int32_t v[1] = {(int32_t)vv};
        uint32_t deg[1] = {0};
        OffT rb[1] = {0};
        uint32_t app = 0;
        if (vv < a.nv && __ldcg(hp + vv) != 0ull) {
            rb[0] = __ldg(a.ro + vv);
            deg[0] = (uint32_t)(__ldg(a.ro + vv + 1) - rb[0]);
            if (deg[0]) app = 1;
        }
        warp_append_items<1, OffT>(v, deg, rb, app, Qo, Eo, Ro, ctr);
    }
}

template <typename OffT>
__device__ BcmState bcm_next(const BcmArgs<OffT> &a, const BcmState &st) {
    BcmState ns = st;
    ns.phase = st.phase + 1;
    if (st.op == MOP_EXPAND) {
        ns.op = MOP_FINAL;
        return ns;
    }
    if (st.op == MOP_FINAL) {
        const unsigned long long pk = ld_relaxed_u64(&a.ctl->qpack[(st.k + 1) & 3]);
        const uint32_t q = (uint32_t)(pk >> 32);
        if (q > 0) {
            ns.op = MOP_EXPAND;
            ns.k = st.k + 1;
            ns.cur = st.cur ^ 1;
            ns.q = q;
            ns.T = (uint32_t)pk;
        } else {
            ns.op = MOP_FIN_BUILD;                           // level k is the deepest
            ns.done = st.k == 0;
        }
        return ns;
    }
    if (st.op == MOP_FIN_BUILD) {
        if (st.k <= 1) {
            ns.done = 1;
            return ns;
        }
        const unsigned long long pk = ld_relaxed_u64(&a.ctl->qpack[(st.k - 1) & 3]);
        ns.op = MOP_PUSH;                                    // level k's vertices push into level k - 1
        ns.k = st.k - 1;
        ns.q2 = (uint32_t)(pk >> 32);
        ns.T2 = (uint32_t)pk;
        return ns;
    }
    // after PUSH into level k: finish level k, whose list is in Q[cur ^ 1]
    ns.op = MOP_FIN_BUILD;
    ns.cur = st.cur ^ 1;
    ns.q = st.q2;
    ns.T = st.T2;
    return ns;
}

template <typename OffT>
__global__ void __launch_bounds__(BCM_BLOCK) k_bcm_persistent(BcmArgs<OffT> a) {
    __shared__ BcmState s_st;
    __shared__ BcmWarpSmem<OffT> wsm[BCM_WARPS];
    BcmWarpSmem<OffT> &w = wsm[threadIdx.x >> 5];
    FlagBarrier bar{a.bar_flags, &a.ctl->bar_release, a.ctl, a.timeout_ns, 0u};
    if (threadIdx.x == 0) {
        BcmState s;
        memset(&s, 0, sizeof s);
        const unsigned long long pk = ld_relaxed_u64(&a.ctl->qpack[0]);
        s.op = MOP_EXPAND;
        s.q = (uint32_t)(pk >> 32);
        s.T = (uint32_t)pk;
        s.done = s.q == 0;
        s_st = s;
    }
    __syncthreads();
    for (;;) {
        const BcmState st = s_st;
        if (st.done) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            // list counters: level j's list uses qpack[j & 3]; a counter is
            // zeroed a full phase after its last reader
            if (st.op == MOP_EXPAND) a.ctl->qpack[(st.k + 2) & 3] = 0ull;
            if (st.op == MOP_FINAL) a.ctl->qpack[(st.k + 3) & 3] = 0ull;
            if (st.op == MOP_PUSH) a.ctl->qpack[(st.k + 3) & 3] = 0ull;
            if (a.stats && st.phase < GRX_MAX_LEVELS_STATS) {
                a.stats->level_t0[st.phase] = grx_globaltimer();
                a.stats->dir[st.phase] = st.op >= MOP_FIN_BUILD;
                a.stats->frontier[st.phase] = st.q;
                a.stats->edges_examined[st.phase] = (st.op == MOP_EXPAND || st.op == MOP_PUSH) ? st.T : 0;
                a.stats->levels = st.phase + 1;
            }
        }
        unsigned long long lane_edges = 0;
        if (st.op == MOP_EXPAND) {
            // hist[k + 1] is written by the next phase for touched vertices only
            if (st.k + 1 < GRX_BCM_MAX_LEVELS) {
                unsigned long long *h1 = hist_level(a, st.k + 1);
                for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < a.nv;
                     v += (int64_t)gridDim.x * blockDim.x)
                    h1[v] = 0ull;
            }
            level_edges<OffT, true>(a, st, w, lane_edges);
        } else if (st.op == MOP_FINAL) {
            forward_final<OffT>(a, st, w.list);
        } else if (st.op == MOP_FIN_BUILD) {
            finish_and_build<OffT>(a, st);
        } else {
            level_edges<OffT, false>(a, st, w, lane_edges);
        }
        if (a.stats) {
            lane_edges = warp_sum(lane_edges);
            if ((threadIdx.x & 31) == 0 && lane_edges && st.phase < GRX_MAX_LEVELS_STATS)
                atomicAdd(&a.stats->vertices_scanned[st.phase], lane_edges);
        }
        if (!flag_barrier(bar)) return;
        if (threadIdx.x == 0) s_st = bcm_next(a, st);
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->levels_run = s_st.k + 1;
        if (a.stats && s_st.phase <= GRX_MAX_LEVELS_STATS) a.stats->level_t0[s_st.phase] = grx_globaltimer();
    }
}

// Sources: lanes of the same vertex share its list entry.
template <typename OffT>
__global__ void k_bcm_init(const int32_t *srcs, int n, const OffT *ro, unsigned long long *seen,
                           unsigned long long *hist0, double *sig, int32_t *Q, uint32_t *E, OffT *R,
                           TravCtl *ctl) {
    uint32_t q = 0, T = 0;
    for (int i = 0; i < 4; ++i) ctl->qpack[i] = 0ull;
    for (int i = 0; i < n; ++i) {
        const int32_t s = srcs[i];
        const uint32_t deg = (uint32_t)(ro[s + 1] - ro[s]);
        if (hist0[s] == 0ull && deg > 0) {
            Q[q] = s;
            E[q] = T;
            R[q] = ro[s];
            ++q;
            T += deg;
        }
        hist0[s] |= 1ull << i;
        seen[s] |= 1ull << i;
        sig[(size_t)s * 64 + i] = 1.0;
    }
    ctl->qpack[0] = ((unsigned long long)q << 32) | T;
}

template <typename OffT>
grx_status launch_typed(grx_graph *g, const int32_t *srcs_host, int n, double *bc_out, const grx_opts *o,
                        cudaStream_t s) {
    BcmArgs<OffT> a;
    a.nv = g->nv;
    a.words = g->words;
    a.ro = (const OffT *)g->ro;
    a.col = g->col;
    a.seen = g->bcm_seen;
    a.next = g->bcm_next;
    a.hist = g->bcm_hist;
    a.touched = g->fbits[2];
    a.sig = g->bcm_sig;
    a.acc = g->bcm_acc;
    a.bc = bc_out;
    for (int i = 0; i < 2; ++i) {
        a.Q[i] = g->qv[i];
        a.E[i] = g->qe[i];
        a.R[i] = (OffT *)g->qr[i];
    }
    a.ctl = g->ctl;
    a.bar_flags = g->bar_flags;
    a.stats = o->collect_stats ? g->stats : nullptr;
    a.timeout_ns = grx_timeout_ns(o);
    const size_t nv = (size_t)g->nv;
    GRX_CUDA(cudaMemcpyAsync(g->bcm_srcs, srcs_host, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s));
    GRX_CUDA(cudaMemsetAsync(bc_out, 0, nv * 8, s));
    GRX_CUDA(cudaMemsetAsync(a.seen, 0, nv * 8, s));
    GRX_CUDA(cudaMemsetAsync(a.next, 0, nv * 8, s));
    GRX_CUDA(cudaMemsetAsync(a.hist, 0, nv * 8, s));                 // level 0; deeper levels by the kernel
    GRX_CUDA(cudaMemsetAsync(a.touched, 0, (size_t)g->words * 4, s));
    GRX_CUDA(cudaMemsetAsync(a.sig, 0, nv * 64 * 8, s));
    GRX_CUDA(cudaMemsetAsync(a.acc, 0, nv * 64 * 8, s));
    if (o->collect_stats) GRX_CUDA(cudaMemsetAsync(g->stats, 0, sizeof(DevStats), s));
    k_bcm_init<OffT><<<1, 1, 0, s>>>(g->bcm_srcs, n, a.ro, a.seen, a.hist, a.sig, a.Q[0], a.E[0], a.R[0], g->ctl);
    GRX_CUDA(cudaGetLastError());
    static int per_sm = -1;
    if (per_sm < 0) {
        GRX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bcm_persistent<OffT>, BCM_BLOCK, 0));
        if (per_sm < 1) return grx_fail(GRX_ECUDA, "bc_multi: persistent kernel does not fit on an SM");
    }
    int max_grid = per_sm * g->ctx->num_sms;
    if (max_grid > GRX_MAX_GRID) max_grid = GRX_MAX_GRID;
    const int blocks = o->grid_blocks > 0 && o->grid_blocks < max_grid ? o->grid_blocks : max_grid;
    GRX_CUDA(cudaMemsetAsync(g->bar_flags, 0, sizeof(unsigned int) * (size_t)blocks, s));
    GRX_CUDA(cudaMemsetAsync(&g->ctl->bar_release, 0, sizeof(unsigned int), s));
    void *args[] = {(void *)&a};
    if (o->ev_begin) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_begin, s));
    GRX_CUDA(cudaLaunchCooperativeKernel((const void *)k_bcm_persistent<OffT>, dim3(blocks), dim3(BCM_BLOCK),
                                         args, 0, s));
    if (o->ev_end) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_end, s));
    return GRX_OK;
}

}  // namespace

grx_status grx_bcm_launch(grx_graph *g, const int32_t *srcs, int n, double *bc_out, const grx_opts *o,
                          cudaStream_t s) {
    return g->off64 ? launch_typed<int64_t>(g, srcs, n, bc_out, o, s)
                    : launch_typed<int32_t>(g, srcs, n, bc_out, o, s);
}
