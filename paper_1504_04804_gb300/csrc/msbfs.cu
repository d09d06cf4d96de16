// Multi-source BFS: up to 64 sources share one traversal and one edge stream.
//
// Every vertex carries 64-bit lane masks: seen[v] (lanes that have labelled
// v), next[v] (lanes reaching v in the level being expanded) and cur[v] (lanes
// whose frontier holds v).  Lane b's result equals a single-source BFS from
// srcs[b] (Algorithm 1); the lanes only share the reading of the graph.
//
//  * Push level: the frontier (vertices with a non-empty cur mask) is cut into
//    equal warp tiles of edges using the degree prefix stored with every
//    frontier slot (as in single-source BFS).  For edge (u, v) the lanes
//    m = cur[u] & ~seen[v] are OR-ed into next[v]; the first warp to touch
//    v lists it.  A finalize phase turns each touched vertex's next mask into
//    its new lanes, labels them and appends the vertex, with degree and row
//    start, to the next frontier.
//  * Pull level: every vertex still missing some active lane ORs the cur
//    masks of its neighbours, stopping as soon as all missing lanes are found
//    (edge skipping, Sec. 6.1), and labels the found lanes itself (no atomics
//    on labels).
//  * Direction (Sec. 6.1 on lane popcounts): FV = the frontier's edge count,
//    BV = (unseen vertex-lane pairs) * V / (seen pairs); push->pull once when
//    FV > BV*alpha, pull->push when FV < BV*beta.
//  * cur rotates through three arrays: level L reads cur[L%3], writes
//    cur[(L+1)%3] and clears the entries of Q_{L-1} in cur[(L+2)%3], so no
//    clear ever races with a read or a write.
//  * One cooperative persistent kernel, levels separated by the bounded flag
//    barrier.
#include <cstring>

#include "grx_internal.cuh"

namespace {

constexpr int MS_BLOCK = 256;
constexpr int MS_WARPS = MS_BLOCK / 32;
constexpr int MS_ITEMS = 8;
constexpr int MS_WTILE = 32 * MS_ITEMS;

enum { DIR_PUSH = 0, DIR_PULL = 1 };

template <typename OffT>
struct MsArgs {
    int32_t nv;
    int64_t ne;
    const OffT *ro;
    const int32_t *col;
    int n;
    unsigned long long lanes;         // active lane mask
    int32_t src[64];
    unsigned long long *seen;
    unsigned long long *next;
    unsigned long long *cur[3];
    int32_t *Q[3];
    uint32_t *E[3];
    OffT *R[3];
    int32_t *touched;
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
    int dir;
    int switched;
    int back;
    int done;
    uint32_t q, T, qprev;
    unsigned long long seen_pairs;    // (vertex, lane) pairs labelled so far
};

template <typename OffT>
struct MsWarpSmem {
    uint32_t qe[MS_WTILE + 2];
    OffT rs[MS_WTILE + 1];
    unsigned long long cm[MS_WTILE + 1];
};

template <typename T>
__device__ __forceinline__ T pk3(T a, T b, T c, int i) { return i == 0 ? a : (i == 1 ? b : c); }

// Label the new lanes of v at level L+1 in the lane-major depth output.
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
    ns.L = st.L + 1;
    const unsigned long long pk = ld_relaxed_u64(&a.ctl->qpack[(st.L + 1) & 3]);
    ns.q = (uint32_t)(pk >> 32);
    ns.T = (uint32_t)pk;
    ns.qprev = st.q;
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
    return ns;
}

}  // namespace

namespace {

// Phase 0: depth = -1 except 0 at each lane's source; all masks empty.
template <typename OffT>
__device__ void ms_init_fill(const MsArgs<OffT> &a) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int b = 0; b < a.n; ++b) {
        int32_t *d = a.depth + (int64_t)b * a.nv;
        const int32_t s = a.src[b];
        for (int64_t v = tid; v < a.nv; v += stride) d[v] = v == s ? 0 : -1;
    }
    for (int64_t v = tid; v < a.nv; v += stride) {
        a.seen[v] = 0ull;
        a.next[v] = 0ull;
        a.cur[0][v] = 0ull;
        a.cur[1][v] = 0ull;
        a.cur[2][v] = 0ull;
    }
}

// Phase 1 (one thread): seed the lanes and the first frontier (distinct
// sources with at least one edge).
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
    }
    a.ctl->qpack[0] = ((unsigned long long)cnt << 32) | edges;
    for (int i = 1; i < 4; ++i) a.ctl->qpack[i] = 0ull;
    for (int i = 0; i < 4; ++i) {
        a.ctl->ucount[i] = 0u;
        a.ctl->pairs[i] = 0ull;
    }
}

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
        uint32_t tmask = 0;
#pragma unroll
        for (int k = 0; k < MS_ITEMS; ++k) {
            const unsigned long long mk = m[k] & ~sv[k];
            if (mk && atomicOr(a.next + v[k], mk) == 0ull) tmask |= 1u << k;
        }
        warp_append_list_items<MS_ITEMS>(v, tmask, a.touched, tctr);
        i0 = (next_start == e1) ? i0 + n : i0 + n - 1;
        __syncwarp();
    }
}

// Turn the touched vertices' next masks into new lanes and the next frontier.
template <typename OffT>
__device__ void ms_push_finalize(const MsArgs<OffT> &a, const MsState &st) {
    const int L = st.L;
    unsigned long long *cout = pk3(a.cur[0], a.cur[1], a.cur[2], (L + 1) % 3);
    int32_t *Qv_out = pk3(a.Q[0], a.Q[1], a.Q[2], (L + 1) % 3);
    uint32_t *Qe_out = pk3(a.E[0], a.E[1], a.E[2], (L + 1) % 3);
    OffT *Qr_out = pk3(a.R[0], a.R[1], a.R[2], (L + 1) % 3);
    unsigned long long *ctr = &a.ctl->qpack[(L + 1) & 3];
    const int64_t count = ld_relaxed_u32(&a.ctl->ucount[(L + 1) & 3]);
    const int64_t span = (count + 31) & ~(int64_t)31;
    unsigned long long found = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < span;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v[1] = {0};
        uint32_t deg[1] = {0};
        OffT rb[1] = {0};
        uint32_t app = 0;
        if (i < count) {
            v[0] = __ldcg(a.touched + i);
            const unsigned long long nx = __ldcg(a.next + v[0]);
            a.next[v[0]] = 0ull;
            const unsigned long long sv = __ldcg(a.seen + v[0]);
            const unsigned long long nw = nx & ~sv & a.lanes;
            if (nw) {
                a.seen[v[0]] = sv | nw;
                cout[v[0]] = nw;
                write_depths(a.depth, a.nv, v[0], nw, L + 1);
                found += (unsigned long long)__popcll(nw);
                rb[0] = __ldg(a.ro + v[0]);
                deg[0] = (uint32_t)(__ldg(a.ro + v[0] + 1) - rb[0]);
                if (deg[0]) app = 1;
            }
        }
        warp_append_items<1, OffT>(v, deg, rb, app, Qv_out, Qe_out, Qr_out, ctr);
    }
    found = warp_sum(found);
    if ((threadIdx.x & 31) == 0 && found) atomicAdd(&a.ctl->pairs[(L + 1) & 3], found);
}

// Pull: each vertex missing some active lane ORs its neighbours' cur masks,
// stopping once every missing lane is found.
template <typename OffT, bool STATS>
__device__ void ms_pull(const MsArgs<OffT> &a, const MsState &st, unsigned long long &scanned) {
    const int L = st.L;
    const unsigned long long *cin = pk3(a.cur[0], a.cur[1], a.cur[2], L % 3);
    unsigned long long *cout = pk3(a.cur[0], a.cur[1], a.cur[2], (L + 1) % 3);
    int32_t *Qv_out = pk3(a.Q[0], a.Q[1], a.Q[2], (L + 1) % 3);
    uint32_t *Qe_out = pk3(a.E[0], a.E[1], a.E[2], (L + 1) % 3);
    OffT *Qr_out = pk3(a.R[0], a.R[1], a.R[2], (L + 1) % 3);
    unsigned long long *ctr = &a.ctl->qpack[(L + 1) & 3];
    const int64_t span = ((int64_t)a.nv + 31) & ~(int64_t)31;
    unsigned long long found = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < span;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v[1] = {(int32_t)i};
        uint32_t deg[1] = {0};
        OffT rb[1] = {0};
        uint32_t app = 0;
        if (i < a.nv) {
            const unsigned long long sv = __ldcg(a.seen + i);
            const unsigned long long miss = a.lanes & ~sv;
            if (miss) {
                const OffT b = __ldg(a.ro + i), e = __ldg(a.ro + i + 1);
                unsigned long long acc = 0ull;
                OffT k = b;
                for (; k < e && acc != miss; ++k) acc |= __ldcg(cin + __ldg(a.col + k)) & miss;
                if (STATS) scanned += (unsigned long long)(k - b);
                if (acc) {
                    a.seen[i] = sv | acc;
                    cout[i] = acc;
                    write_depths(a.depth, a.nv, (int32_t)i, acc, L + 1);
                    found += (unsigned long long)__popcll(acc);
                    rb[0] = b;
                    deg[0] = (uint32_t)(e - b);
                    app = 1;
                }
            }
        }
        warp_append_items<1, OffT>(v, deg, rb, app, Qv_out, Qe_out, Qr_out, ctr);
    }
    found = warp_sum(found);
    if ((threadIdx.x & 31) == 0 && found) atomicAdd(&a.ctl->pairs[(L + 1) & 3], found);
}

}  // namespace

namespace {

template <typename OffT, bool STATS>
__global__ void __launch_bounds__(MS_BLOCK, 2) k_msbfs_persistent(MsArgs<OffT> a) {
    __shared__ MsState s_st;
    __shared__ MsWarpSmem<OffT> wsm[MS_WARPS];
    MsWarpSmem<OffT> &w = wsm[threadIdx.x >> 5];
    FlagBarrier bar{a.bar_flags, &a.ctl->bar_release, a.ctl, a.timeout_ns, 0u};
    ms_init_fill(a);
    if (!flag_barrier(bar)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ms_seed(a);
    if (!flag_barrier(bar)) return;
    if (threadIdx.x == 0) {
        MsState s;
        const unsigned long long pk = ld_relaxed_u64(&a.ctl->qpack[0]);
        s.L = 0;
        s.dir = a.mode == GRX_DIR_PULL ? DIR_PULL : DIR_PUSH;
        s.switched = a.mode == GRX_DIR_PULL;
        s.back = 0;
        s.q = (uint32_t)(pk >> 32);
        s.T = (uint32_t)pk;
        s.qprev = 0;
        s.seen_pairs = (unsigned long long)a.n;
        s.done = s.q == 0;
        s_st = s;
    }
    __syncthreads();
    for (;;) {
        const MsState st = s_st;
        if (st.done) break;
        const int L = st.L;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
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
        {   // the lanes of Q_{L-1} leave cur[(L+2)%3]
            const int32_t *Qp = pk3(a.Q[0], a.Q[1], a.Q[2], (L + 2) % 3);
            unsigned long long *cp = pk3(a.cur[0], a.cur[1], a.cur[2], (L + 2) % 3);
            for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)st.qprev;
                 i += (int64_t)gridDim.x * blockDim.x)
                cp[__ldcg(Qp + i)] = 0ull;
        }
        if (st.dir == DIR_PUSH) {
            ms_push_expand<OffT, STATS>(a, st, w);
            if (!flag_barrier(bar)) return;
            ms_push_finalize<OffT>(a, st);
        } else {
            unsigned long long scanned = 0;
            ms_pull<OffT, STATS>(a, st, scanned);
            if (STATS) {
                scanned = warp_sum(scanned);
                if ((threadIdx.x & 31) == 0 && scanned && L < GRX_MAX_LEVELS_STATS)
                    atomicAdd(&a.stats->edges_examined[L], scanned);
            }
        }
        if (!flag_barrier(bar)) return;
        if (threadIdx.x == 0) s_st = ms_next_state(a, st, STATS);
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->levels_run = s_st.L;
        if (STATS && s_st.L <= GRX_MAX_LEVELS_STATS) a.stats->level_t0[s_st.L] = grx_globaltimer();
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

grx_status grx_msbfs_launch(grx_graph *g, const int32_t *srcs, int n, int32_t *depth,
                            const grx_opts *o, cudaStream_t s) {
    if (g->off64)
        return o->collect_stats ? ms_launch_typed<int64_t, true>(g, srcs, n, depth, o, s)
                                : ms_launch_typed<int64_t, false>(g, srcs, n, depth, o, s);
    return o->collect_stats ? ms_launch_typed<int32_t, true>(g, srcs, n, depth, o, s)
                            : ms_launch_typed<int32_t, false>(g, srcs, n, depth, o, s);
}
