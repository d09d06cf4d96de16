// SSSP (Table 1): frontier label-correcting relaxation.  Each round advances
// the vertices whose distance improved in the previous round: for every edge
// (u, v, w) it proposes dist[u] + w with an atomic min -- the min combiner the
// paper uses for SSSP labels (Sec. 3) -- and v joins the next frontier once.
// Rounds repeat until no distance improves; the result is the exact
// shortest-path distance.
//
// Same persistent, load-balanced structure as the push step of BFS: a frontier
// queue slot carries the vertex, its row start and the exclusive prefix of the
// frontier's degrees, so the frontier's edges are cut into equal warp tiles
// (each warp a contiguous range, rows by a branch-free scatter + max-scan) and
// each lane keeps 8 edges' loads in flight, item k at tile position
// k*32 + lane so the warp's column and weight loads are contiguous runs.  Two
// kinds of rounds:
//  * small rounds: an improving lane claims v with the atomic min's old value,
//    a per-vertex round stamp keeps v once, and v is appended with one
//    warp-aggregated atomic;
//  * rounds with at least push_bitmap * V edges: the atomic min is a
//    reduction (no value returned) and v's bit is OR-ed into a changed bitmap;
//    a second phase, by warps owning 32-word chunks of the bitmap, appends the
//    changed vertices in vertex order and clears the bitmap.  A lane reduces
//    only when its proposal beats the current distance read from L2, so every
//    marked vertex did improve in the round and every improvement is marked.
// Near-far bands (Davidson et al.'s near-far split, opt-in with delta > 0):
// an improved vertex joins the next frontier only if its distance is below
// the threshold, else it waits once in a far pile (a bitmap keeps it unique).
// When the frontier runs dry, the threshold moves to the pile's smallest
// distance + delta and the pile's vertices below it form the next frontier;
// entries below the old threshold were relaxed since and are dropped.  High-
// diameter weighted graphs then relax far fewer edges more than once.
// Rounds and phases are separated by the bounded grid barrier.
#include "grx_internal.cuh"

namespace {

constexpr int SS_BLOCK = 256;
#ifndef GRX_SS_MIN_BLOCKS
#define GRX_SS_MIN_BLOCKS 3                         // resident blocks per SM (register cap)
#endif
constexpr int SS_WARPS = SS_BLOCK / 32;
constexpr int SS_ITEMS = 8;
constexpr int SS_WTILE = 32 * SS_ITEMS;
constexpr int SS_RPL = 4;                    // finalize: vertices per lane per round

template <typename OffT>
struct SsspArgs {
    int32_t nv;
    int64_t words;
    const OffT *ro;
    const int32_t *col;
    const uint32_t *w;
    uint32_t *dist;
    int32_t *stamp;
    uint32_t *cbits;                         // changed bitmap of reduction rounds
    uint32_t *fbits;                         // near-far: far pile membership
    int32_t *far[2];                         // near-far: far piles (ping-pong)
    uint32_t delta;                          // near-far band width (0 = no bands)
    int32_t *Q[3];
    uint32_t *E[3];
    OffT *R[3];
    TravCtl *ctl;
    unsigned int *bar_flags;
    DevStats *stats;
    uint32_t bmp_min_T;
    unsigned long long timeout_ns;
    int32_t src;
};

enum { SOP_RELAX, SOP_FINAL, SOP_FARMIN, SOP_FARSPLIT };

struct SsState {
    int L;
    int op;
    int bmp;
    int done;
    int fsel;                                // current far pile
    uint32_t q, T;
    uint32_t thr;                            // near-far threshold (UINT32_MAX: no bands)
    uint32_t oldthr;                         // threshold before the last advance
    uint32_t nfar;                           // current far pile length
};

template <typename OffT>
union SsWarpSmem {
    struct {
        uint32_t qe[SS_WTILE + 2];
        int32_t u[SS_WTILE + 1];
        OffT rs[SS_WTILE + 1];
        uint32_t du[SS_WTILE + 1];
        alignas(16) uint16_t rid[SS_WTILE];
    };
    uint16_t list[32 * 32];
};

template <typename OffT>
__device__ __forceinline__ void ss_set_kind(const SsspArgs<OffT> &a, SsState &s) {
    s.bmp = s.T >= a.bmp_min_T;
}

// v improved to a distance at or above the threshold: into the far pile once.
template <typename OffT>
__device__ __forceinline__ void far_push(const SsspArgs<OffT> &a, const SsState &st, int32_t v) {
    const uint32_t bit = 1u << (v & 31);
    if (!(atomicOr(a.fbits + (v >> 5), bit) & bit)) {
        const unsigned int pos = atomicAdd(&a.ctl->farcnt[st.fsel], 1u);
        a.far[st.fsel][pos] = v;
    }
}

// Phase 0 of round L: relax the edges of Q_L.
template <typename OffT, bool BMP>
__device__ void relax_round(const SsspArgs<OffT> &a, const SsState &st, SsWarpSmem<OffT> &w) {
    const int L = st.L;
    const unsigned int lane = threadIdx.x & 31;
    const int32_t *Qv = pick3(a.Q[0], a.Q[1], a.Q[2], L % 3);
    const uint32_t *Qe = pick3(a.E[0], a.E[1], a.E[2], L % 3);
    const OffT *Qr = pick3(a.R[0], a.R[1], a.R[2], L % 3);
    int32_t *Qv_out = pick3(a.Q[0], a.Q[1], a.Q[2], (L + 1) % 3);
    uint32_t *Qe_out = pick3(a.E[0], a.E[1], a.E[2], (L + 1) % 3);
    OffT *Qr_out = pick3(a.R[0], a.R[1], a.R[2], (L + 1) % 3);
    unsigned long long *ctr = &a.ctl->qpack[(L + 1) & 3];
    const int64_t q = st.q;
    const uint64_t T = st.T;
    const uint64_t ntiles = (T + SS_WTILE - 1) / SS_WTILE;
    const uint64_t nwarps = (uint64_t)gridDim.x * SS_WARPS;
    const uint64_t gw = (uint64_t)blockIdx.x * SS_WARPS + (threadIdx.x >> 5);
    const uint64_t per = (ntiles + nwarps - 1) / nwarps;
    const uint64_t tb0 = gw * per;
    const uint64_t tb1 = min(ntiles, tb0 + per);
    if (tb0 >= tb1) return;
    int64_t i0 = warp_upper_index_cg(Qe, q, (uint32_t)(tb0 * SS_WTILE));
    for (uint64_t tile = tb0; tile < tb1; ++tile) {
        const uint64_t e0 = tile * SS_WTILE;
        const uint32_t e1 = (uint32_t)min(T, e0 + SS_WTILE);
        // frontier elements starting before e1, 32 per round
        int n = 0;
        for (;;) {
            const int64_t idx = i0 + n + lane;
            uint32_t qe = 0xffffffffu;
            if (idx < q) qe = __ldcg(Qe + idx);
            const bool in = idx < q && qe < e1;
            if (n + (int)lane <= SS_WTILE + 1) w.qe[n + lane] = qe;
            if (in && n + (int)lane <= SS_WTILE) {
                const int32_t u = __ldcg(Qv + idx);
                w.u[n + lane] = u;
                w.rs[n + lane] = __ldcg(Qr + idx);
                w.du[n + lane] = __ldcg(a.dist + u);
            }
            const int cnt = __popc(__ballot_sync(GRX_FULL_MASK, in));
            n += cnt;
            if (cnt < 32) break;
            if (n > SS_WTILE) {              // only possible with a malformed graph
                if (lane == 0) grx_set_status(a.ctl, GRX_EINVAL);
                n = SS_WTILE;
                break;
            }
        }
        __syncwarp();
        const uint32_t next_start = w.qe[n];
        int row[SS_ITEMS];
        warp_tile_rows8_strided(w.rid, w.qe, (uint32_t)e0, n, row);   // item k at position k*32 + lane
        int32_t v[SS_ITEMS];
        uint32_t wt[SS_ITEMS], du[SS_ITEMS];
#pragma unroll
        for (int k = 0; k < SS_ITEMS; ++k) {
            const uint32_t e = (uint32_t)e0 + (uint32_t)k * 32 + lane;
            const int j = row[k];
            const bool ok = e < e1;
            const OffT idx = ok ? w.rs[j] + (OffT)(e - w.qe[j]) : (OffT)0;
            v[k] = ok ? __ldg(a.col + idx) : -1;
            wt[k] = ok ? __ldg(a.w + idx) : 0u;
            du[k] = ok ? w.du[j] : 0xffffffffu;
        }
        __syncwarp();
        uint32_t nd[SS_ITEMS], cur[SS_ITEMS];
#pragma unroll
        for (int k = 0; k < SS_ITEMS; ++k) {
            nd[k] = 0xffffffffu;
            if (v[k] >= 0 && du[k] != 0xffffffffu) {
                const uint64_t s64 = (uint64_t)du[k] + wt[k];
                if (s64 >= 0xffffffffull) grx_set_status(a.ctl, GRX_ERANGE);
                else nd[k] = (uint32_t)s64;
            }
            cur[k] = nd[k] != 0xffffffffu ? __ldcg(a.dist + v[k]) : 0u;
        }
        if (BMP) {
#pragma unroll
            for (int k = 0; k < SS_ITEMS; ++k) {
                if (nd[k] < cur[k]) {
                    atomicMin(a.dist + v[k], nd[k]);                     // results unused: reductions
                    atomicOr(a.cbits + (v[k] >> 5), 1u << (v[k] & 31));
                }
            }
        } else {
            uint32_t improved = 0;
#pragma unroll
            for (int k = 0; k < SS_ITEMS; ++k) {
                if (nd[k] < cur[k]) {
                    const uint32_t old = atomicMin(a.dist + v[k], nd[k]);
                    if (nd[k] < old) improved |= 1u << k;
                }
            }
            uint32_t queued = 0;
#pragma unroll
            for (int k = 0; k < SS_ITEMS; ++k) {
                if (!(improved >> k & 1u)) continue;
                if (nd[k] >= st.thr) far_push(a, st, v[k]);
                else if (atomicExch(a.stamp + v[k], L + 1) != L + 1) queued |= 1u << k;
            }
            uint32_t deg[SS_ITEMS];
            OffT rb[SS_ITEMS];
            uint32_t app = 0;
#pragma unroll
            for (int k = 0; k < SS_ITEMS; ++k) {
                rb[k] = 0;
                deg[k] = 0;
                if (queued >> k & 1u) {
                    rb[k] = __ldg(a.ro + v[k]);
                    deg[k] = (uint32_t)(__ldg(a.ro + v[k] + 1) - rb[k]);
                    if (deg[k]) app |= 1u << k;
                }
            }
            warp_append_items<SS_ITEMS, OffT>(v, deg, rb, app, Qv_out, Qe_out, Qr_out, ctr);
        }
        i0 = (next_start == e1) ? i0 + n : i0 + n - 1;
        __syncwarp();
    }
}

// Phase 1 of a reduction round: the changed bitmap's vertices (with edges)
// become Q_{L+1} in vertex order; the bitmap is cleared.
template <typename OffT>
__device__ void changed_to_queue(const SsspArgs<OffT> &a, const SsState &st, uint16_t *list) {
    const int L = st.L;
    int32_t *Qv_out = pick3(a.Q[0], a.Q[1], a.Q[2], (L + 1) % 3);
    uint32_t *Qe_out = pick3(a.E[0], a.E[1], a.E[2], (L + 1) % 3);
    OffT *Qr_out = pick3(a.R[0], a.R[1], a.R[2], (L + 1) % 3);
    unsigned long long *ctr = &a.ctl->qpack[(L + 1) & 3];
    const unsigned int lane = threadIdx.x & 31;
    const int64_t nsc = (a.words + 31) / 32;
    const int64_t nwarps = (int64_t)gridDim.x * SS_WARPS;
    for (int64_t sc = (int64_t)blockIdx.x * SS_WARPS + (threadIdx.x >> 5); sc < nsc; sc += nwarps) {
        const int64_t wd = sc * 32 + lane;
        const uint32_t bits = wd < a.words ? __ldcg(a.cbits + wd) : 0u;
        if (bits) a.cbits[wd] = 0u;
        const int n = warp_compact_bits(bits, list);
        for (int base = 0; base < n; base += 32 * SS_RPL) {
            int32_t v[SS_RPL];
            uint32_t deg[SS_RPL];
            OffT rb[SS_RPL];
            uint32_t app = 0;
#pragma unroll
            for (int k = 0; k < SS_RPL; ++k) {
                const int i = base + k * 32 + (int)lane;
                v[k] = i < n ? (int32_t)(sc * 1024 + list[i]) : 0;
                rb[k] = 0;
                deg[k] = 0;
                if (i < n && __ldcg(a.dist + v[k]) >= st.thr) {
                    far_push(a, st, v[k]);
                } else if (i < n) {
                    rb[k] = __ldg(a.ro + v[k]);
                    deg[k] = (uint32_t)(__ldg(a.ro + v[k] + 1) - rb[k]);
                    if (deg[k]) app |= 1u << k;
                }
            }
            warp_append_items<SS_RPL, OffT>(v, deg, rb, app, Qv_out, Qe_out, Qr_out, ctr);
        }
        __syncwarp();
    }
}

// Band advance, phase 1: the smallest distance in the far pile.  The minimum
// of pile f goes to farmin[f]; farmin[f ^ 1], read by every block after the
// previous advance's barrier, is reset here for the next advance.
template <typename OffT>
__device__ void far_min(const SsspArgs<OffT> &a, const SsState &st) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->farcnt[st.fsel ^ 1] = 0u;
        a.ctl->farmin[st.fsel ^ 1] = 0xffffffffu;
    }
    const int32_t *F = a.far[st.fsel];
    uint32_t m = 0xffffffffu;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)st.nfar;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t d = __ldcg(a.dist + __ldcg(F + i));
        if (d >= st.thr) m = min(m, d);          // below the threshold: relaxed since, stale
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(GRX_FULL_MASK, m, o));
    if ((threadIdx.x & 31) == 0 && m != 0xffffffffu) atomicMin(&a.ctl->farmin[st.fsel], m);
}

// Band advance, phase 2 (threshold already raised): far vertices below the
// new threshold form Q_L, the others move to the other pile, stale ones drop.
template <typename OffT>
__device__ void far_split(const SsspArgs<OffT> &a, const SsState &st) {
    const int L = st.L;
    int32_t *Qv = pick3(a.Q[0], a.Q[1], a.Q[2], L % 3);
    uint32_t *Qe = pick3(a.E[0], a.E[1], a.E[2], L % 3);
    OffT *Qr = pick3(a.R[0], a.R[1], a.R[2], L % 3);
    const int32_t *F = a.far[st.fsel];
    int32_t *G = a.far[st.fsel ^ 1];
    const int64_t span = ((int64_t)st.nfar + 31) & ~(int64_t)31;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < span;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v[1] = {0};
        uint32_t deg[1] = {0};
        OffT rb[1] = {0};
        uint32_t app = 0;
        if (i < (int64_t)st.nfar) {
            v[0] = __ldcg(F + i);
            const uint32_t d = __ldcg(a.dist + v[0]);
            if (d >= st.thr) {                                   // still far
                const unsigned int pos = atomicAdd(&a.ctl->farcnt[st.fsel ^ 1], 1u);
                G[pos] = v[0];
            } else {
                atomicAnd(a.fbits + (v[0] >> 5), ~(1u << (v[0] & 31)));
                if (d >= st.oldthr) {                            // first reached the band now
                    rb[0] = __ldg(a.ro + v[0]);
                    deg[0] = (uint32_t)(__ldg(a.ro + v[0] + 1) - rb[0]);
                    if (deg[0]) app = 1;
                }
            }
        }
        warp_append_items<1, OffT>(v, deg, rb, app, Qv, Qe, Qr, &a.ctl->qpack[L & 3]);
    }
}

// State of the next phase.
template <typename OffT>
__device__ SsState ss_next(const SsspArgs<OffT> &a, const SsState &st, bool stats) {
    SsState ns = st;
    if (st.op == SOP_RELAX && st.bmp) {
        ns.op = SOP_FINAL;
        return ns;
    }
    if (st.op == SOP_FARMIN) {
        const uint32_t m = ld_relaxed_u32(&a.ctl->farmin[st.fsel]);
        ns.op = SOP_FARSPLIT;
        ns.oldthr = st.thr;
        ns.thr = m == 0xffffffffu ? st.thr
                                  : (m > 0xffffffffu - a.delta ? 0xffffffffu : m + a.delta);
        if (m == 0xffffffffu) ns.thr = 0xffffffffu;              // every entry stale: one last split
        return ns;
    }
    uint32_t q, T;
    int L;
    if (st.op == SOP_FARSPLIT) {                                 // Q_L came from the far pile
        L = st.L;
        ns.fsel = st.fsel ^ 1;
        ns.nfar = ld_relaxed_u32(&a.ctl->farcnt[ns.fsel]);
    } else {                                                     // end of round st.L
        L = st.L + 1;
        ns.nfar = ld_relaxed_u32(&a.ctl->farcnt[st.fsel]);
    }
    const unsigned long long pk = ld_relaxed_u64(&a.ctl->qpack[L & 3]);
    q = (uint32_t)(pk >> 32);
    T = (uint32_t)pk;
    if (stats && blockIdx.x == 0 && st.op != SOP_FARSPLIT && st.L < GRX_MAX_LEVELS_STATS)
        a.stats->discovered[st.L] = q;
    ns.L = L;
    ns.q = q;
    ns.T = T;
    if (q > 0) {
        ns.op = SOP_RELAX;
        ss_set_kind(a, ns);
    } else if (a.delta && ns.nfar > 0) {
        ns.op = SOP_FARMIN;
        ns.bmp = 0;
    } else {
        ns.done = 1;
    }
    return ns;
}

template <typename OffT, bool STATS>
__global__ void __launch_bounds__(SS_BLOCK, GRX_SS_MIN_BLOCKS) k_sssp_persistent(SsspArgs<OffT> a) {
    __shared__ SsState s_st;
    __shared__ SsWarpSmem<OffT> wsm[SS_WARPS];
    SsWarpSmem<OffT> &w = wsm[threadIdx.x >> 5];
    FlagBarrier bar{a.bar_flags, &a.ctl->bar_release, a.ctl, a.timeout_ns, 0u};
    if (threadIdx.x == 0) {
        SsState s;
        memset(&s, 0, sizeof s);
        const uint32_t deg = (uint32_t)(a.ro[a.src + 1] - a.ro[a.src]);
        s.op = SOP_RELAX;
        s.q = deg ? 1u : 0u;
        s.T = deg;
        s.done = deg == 0;
        s.thr = a.delta ? a.delta : 0xffffffffu;
        ss_set_kind(a, s);
        s_st = s;
    }
    __syncthreads();
    for (;;) {
        const SsState st = s_st;
        if (st.done) break;
        const int L = st.L;
        if (st.op == SOP_RELAX && blockIdx.x == 0 && threadIdx.x == 0) {
            a.ctl->qpack[(L + 2) & 3] = 0ull;
            if (STATS && L < GRX_MAX_LEVELS_STATS) {
                a.stats->level_t0[L] = grx_globaltimer();
                a.stats->dir[L] = 0;
                a.stats->frontier[L] = st.q;
                a.stats->edges_examined[L] = st.T;
                a.stats->vertices_scanned[L] = st.q;
                a.stats->levels = L + 1;
            }
        }
        if (st.op == SOP_FINAL) changed_to_queue<OffT>(a, st, w.list);
        else if (st.op == SOP_FARMIN) far_min<OffT>(a, st);
        else if (st.op == SOP_FARSPLIT) far_split<OffT>(a, st);
        else if (st.bmp) relax_round<OffT, true>(a, st, w);
        else relax_round<OffT, false>(a, st, w);
        if (!flag_barrier(bar)) return;
        if (threadIdx.x == 0) s_st = ss_next(a, st, STATS);
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->levels_run = s_st.L;
        if (STATS && s_st.L <= GRX_MAX_LEVELS_STATS) a.stats->level_t0[s_st.L] = grx_globaltimer();
    }
}

template <typename OffT>
__global__ void k_sssp_init(int32_t src, const OffT *ro, uint32_t *dist, int32_t *Q0, uint32_t *E0, OffT *R0,
                            TravCtl *ctl, DevStats *stats, int stats_on) {
    const OffT b = ro[src];
    const uint32_t deg = (uint32_t)(ro[src + 1] - b);
    dist[src] = 0;
    Q0[0] = src;
    E0[0] = 0;
    R0[0] = b;
    ctl->qpack[0] = deg ? ((1ull << 32) | deg) : 0ull;
    for (int i = 1; i < 4; ++i) ctl->qpack[i] = 0ull;
    ctl->farcnt[0] = 0u;
    ctl->farcnt[1] = 0u;
    ctl->farmin[0] = 0xffffffffu;
    ctl->farmin[1] = 0xffffffffu;
    if (stats_on) stats->levels = 0;
}

template <typename OffT, bool STATS>
grx_status launch_typed(grx_graph *g, int32_t src, uint32_t *dist, const grx_opts *o,
                        cudaStream_t s) {
    SsspArgs<OffT> a;
    a.nv = g->nv;
    a.words = g->words;
    a.ro = (const OffT *)g->ro;
    a.col = g->col;
    a.w = g->w;
    a.dist = dist;
    a.stamp = g->stamp;
    a.cbits = g->fbits[0];
    a.fbits = g->fbits[1];
    a.far[0] = g->ulist[0];
    a.far[1] = g->ulist[1];
    a.delta = o->sssp_delta;
    for (int i = 0; i < 3; ++i) {
        a.Q[i] = g->qv[i];
        a.E[i] = g->qe[i];
        a.R[i] = (OffT *)g->qr[i];
    }
    a.ctl = g->ctl;
    a.bar_flags = g->bar_flags;
    a.stats = g->stats;
    a.timeout_ns = grx_timeout_ns(o);
    a.src = src;
    {   // reduction rounds when a round's edges reach push_bitmap * nv (0 = 1/8, < 0 = never)
        const double pb = o->push_bitmap == 0.f ? 0.125 : (double)o->push_bitmap;
        const double t = pb * (double)g->nv;
        a.bmp_min_T = pb < 0 ? 0xffffffffu : (t < 1.0 ? 1u : (t > 4294967295.0 ? 0xffffffffu : (uint32_t)t));
    }
    k_sssp_init<OffT><<<1, 1, 0, s>>>(src, a.ro, dist, g->qv[0], g->qe[0], a.R[0], g->ctl, g->stats,
                                      o->collect_stats);
    GRX_CUDA(cudaGetLastError());
    static int per_sm = -1;
    if (per_sm < 0) {
        GRX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sssp_persistent<OffT, STATS>,
                                                               SS_BLOCK, 0));
        if (per_sm < 1) return grx_fail(GRX_ECUDA, "sssp: persistent kernel does not fit on an SM");
    }
    int max_grid = per_sm * g->ctx->num_sms;
    if (max_grid > GRX_MAX_GRID) max_grid = GRX_MAX_GRID;
    int blocks = o->grid_blocks > 0 && o->grid_blocks < max_grid ? o->grid_blocks : max_grid;
    GRX_CUDA(cudaMemsetAsync(g->bar_flags, 0, sizeof(unsigned int) * (size_t)blocks, s));
    GRX_CUDA(cudaMemsetAsync(&g->ctl->bar_release, 0, sizeof(unsigned int), s));
    void *args[] = {(void *)&a};
    if (o->ev_begin) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_begin, s));
    GRX_CUDA(cudaLaunchCooperativeKernel((const void *)k_sssp_persistent<OffT, STATS>, dim3(blocks),
                                         dim3(SS_BLOCK), args, 0, s));
    if (o->ev_end) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_end, s));
    return GRX_OK;
}

}  // namespace

grx_status grx_sssp_launch(grx_graph *g, int32_t src, uint32_t *dist, const grx_opts *o,
                           cudaStream_t s) {
    const size_t nv = (size_t)g->nv;
    GRX_CUDA(cudaMemsetAsync(dist, 0xff, nv * 4, s));
    GRX_CUDA(cudaMemsetAsync(g->stamp, 0, nv * 4, s));
    GRX_CUDA(cudaMemsetAsync(g->fbits[0], 0, (size_t)g->words * 4, s));
    if (o->sssp_delta) GRX_CUDA(cudaMemsetAsync(g->fbits[1], 0, (size_t)g->words * 4, s));
    if (o->collect_stats) GRX_CUDA(cudaMemsetAsync(g->stats, 0, sizeof(DevStats), s));
    if (g->off64)
        return o->collect_stats ? launch_typed<int64_t, true>(g, src, dist, o, s)
                                : launch_typed<int64_t, false>(g, src, dist, o, s);
    return o->collect_stats ? launch_typed<int32_t, true>(g, src, dist, o, s)
                            : launch_typed<int32_t, false>(g, src, dist, o, s);
}
