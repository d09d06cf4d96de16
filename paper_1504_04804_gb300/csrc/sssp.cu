// SSSP (Table 1): frontier label-correcting relaxation.  Each round advances
// the vertices whose distance improved in the previous round: for every edge
// (u, v, w) it proposes dist[u] + w with atomicMin -- the min combiner the
// paper uses for SSSP labels (Sec. 3) -- and queues v at most once per round
// (a per-vertex round stamp is the filter).  Rounds repeat until no distance
// improves; the result is the exact shortest-path distance.
//
// Same persistent, load-balanced structure as the push step of BFS: the
// frontier's edges are cut into equal tiles using the degree prefix that the
// append atomic produced, each thread keeps a run of SS_ITEMS edges' loads and
// atomics in flight, and rounds are separated by a bounded grid barrier.
#include "grx_internal.cuh"

namespace {

constexpr int SS_BLOCK = 256;
constexpr int SS_ITEMS = 8;
constexpr int SS_TILE = SS_BLOCK * SS_ITEMS;

template <typename OffT>
struct SsspArgs {
    int32_t nv;
    const OffT *ro;
    const int32_t *col;
    const uint32_t *w;
    uint32_t *dist;
    int32_t *stamp;
    int32_t *Q[3];
    uint32_t *E[3];
    TravCtl *ctl;
    unsigned int *bar_flags;
    DevStats *stats;
    unsigned long long timeout_ns;
    int32_t src;
};

template <typename OffT>
struct SsspSmem {
    uint32_t qe[SS_TILE + 1];
    int32_t u[SS_TILE + 1];
    OffT rs[SS_TILE + 1];
    uint32_t du[SS_TILE + 1];
    int64_t i0;
    int n;
    uint32_t q, T;
    int done;
};

template <typename OffT, bool STATS>
__device__ void relax_round(const SsspArgs<OffT> &a, int L, uint32_t q, uint64_t T,
                            SsspSmem<OffT> &sm) {
    const int32_t *Qv = pick3(a.Q[0], a.Q[1], a.Q[2], L % 3);
    const uint32_t *Qe = pick3(a.E[0], a.E[1], a.E[2], L % 3);
    int32_t *Qv_out = pick3(a.Q[0], a.Q[1], a.Q[2], (L + 1) % 3);
    uint32_t *Qe_out = pick3(a.E[0], a.E[1], a.E[2], (L + 1) % 3);
    unsigned long long *ctr = &a.ctl->qpack[(L + 1) & 3];
    const uint64_t ntiles = (T + SS_TILE - 1) / SS_TILE;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t e0 = tile * SS_TILE;
        const uint64_t e1 = min(T, e0 + SS_TILE);
        if (threadIdx.x == 0) {
            int64_t i0 = upper_index_cg(Qe, q, (uint32_t)e0);
            int64_t i1 = upper_index_cg(Qe, q, (uint32_t)(e1 - 1));
            int n = (int)(i1 - i0 + 1);
            if (n > SS_TILE + 1) {
                grx_set_status(a.ctl, GRX_EINVAL);
                n = SS_TILE + 1;
            }
            sm.i0 = i0;
            sm.n = n;
        }
        __syncthreads();
        const int64_t i0 = sm.i0;
        const int n = sm.n;
        for (int j = threadIdx.x; j < n; j += SS_BLOCK) {
            int32_t u = __ldcg(Qv + i0 + j);
            sm.qe[j] = __ldcg(Qe + i0 + j);
            sm.u[j] = u;
            sm.rs[j] = __ldg(a.ro + u);
            sm.du[j] = __ldcg(a.dist + u);
        }
        __syncthreads();
        // a run of SS_ITEMS consecutive edges per thread, all loads in flight together
        const uint64_t t0 = e0 + (uint64_t)threadIdx.x * SS_ITEMS;
        int32_t v[SS_ITEMS];
        uint32_t nd[SS_ITEMS];
        uint32_t valid = 0;
#pragma unroll
        for (int k = 0; k < SS_ITEMS; ++k) {
            v[k] = 0;
            nd[k] = 0xffffffffu;
        }
        if (t0 < e1) {
            int j = upper_index_smem(sm.qe, n, (uint32_t)t0);
            uint32_t wt[SS_ITEMS];
            uint32_t du[SS_ITEMS];
#pragma unroll
            for (int k = 0; k < SS_ITEMS; ++k) {
                const uint64_t e = t0 + k;
                wt[k] = 0;
                du[k] = 0xffffffffu;
                if (e < e1) {
                    while (j + 1 < n && sm.qe[j + 1] <= (uint32_t)e) ++j;
                    const OffT idx = sm.rs[j] + (OffT)((uint32_t)e - sm.qe[j]);
                    v[k] = __ldg(a.col + idx);
                    wt[k] = __ldg(a.w + idx);
                    du[k] = sm.du[j];
                    valid |= 1u << k;
                }
            }
#pragma unroll
            for (int k = 0; k < SS_ITEMS; ++k) {
                if (valid >> k & 1u) {
                    const uint64_t s64 = (uint64_t)du[k] + wt[k];
                    if (s64 >= 0xffffffffull) {
                        grx_set_status(a.ctl, GRX_ERANGE);
                        valid &= ~(1u << k);
                    } else {
                        nd[k] = (uint32_t)s64;
                    }
                }
            }
        }
        uint32_t cur[SS_ITEMS];
#pragma unroll
        for (int k = 0; k < SS_ITEMS; ++k) cur[k] = (valid >> k & 1u) ? __ldcg(a.dist + v[k]) : 0u;
        uint32_t improved = 0;
#pragma unroll
        for (int k = 0; k < SS_ITEMS; ++k) {
            if ((valid >> k & 1u) && nd[k] < cur[k]) {
                const uint32_t old = atomicMin(a.dist + v[k], nd[k]);
                if (nd[k] < old) improved |= 1u << k;
            }
        }
        uint32_t queued = 0;
#pragma unroll
        for (int k = 0; k < SS_ITEMS; ++k)
            if ((improved >> k & 1u) && atomicExch(a.stamp + v[k], L + 1) != L + 1) queued |= 1u << k;
        uint32_t deg[SS_ITEMS];
        OffT rb[SS_ITEMS], re[SS_ITEMS];
#pragma unroll
        for (int k = 0; k < SS_ITEMS; ++k) {
            rb[k] = 0;
            re[k] = 0;
            if (queued >> k & 1u) {
                rb[k] = __ldg(a.ro + v[k]);
                re[k] = __ldg(a.ro + v[k] + 1);
            }
        }
        uint32_t app = 0;
#pragma unroll
        for (int k = 0; k < SS_ITEMS; ++k) {
            deg[k] = (uint32_t)(re[k] - rb[k]);
            if ((queued >> k & 1u) && deg[k]) app |= 1u << k;
        }
        warp_append_items<SS_ITEMS, OffT>(v, deg, rb, app, Qv_out, Qe_out, (OffT *)nullptr, ctr);
        __syncthreads();
    }
    if (STATS && blockIdx.x == 0 && threadIdx.x == 0 && L < GRX_MAX_LEVELS_STATS) {
        a.stats->dir[L] = 0;
        a.stats->frontier[L] = q;
        a.stats->edges_examined[L] = T;
        a.stats->vertices_scanned[L] = q;
        a.stats->levels = L + 1;
    }
}

template <typename OffT, bool STATS>
__global__ void __launch_bounds__(SS_BLOCK) k_sssp_persistent(SsspArgs<OffT> a) {
    __shared__ SsspSmem<OffT> sm;
    FlagBarrier bar{a.bar_flags, &a.ctl->bar_release, a.ctl, a.timeout_ns, 0u};
    if (threadIdx.x == 0) {
        uint32_t deg = (uint32_t)(a.ro[a.src + 1] - a.ro[a.src]);
        sm.q = deg ? 1u : 0u;
        sm.T = deg;
        sm.done = deg == 0;
    }
    __syncthreads();
    int L = 0;
    for (;; ++L) {
        const uint32_t q = sm.q;
        const uint32_t T = sm.T;
        if (sm.done) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.ctl->qpack[(L + 2) & 3] = 0ull;
            if (STATS && L < GRX_MAX_LEVELS_STATS) a.stats->level_t0[L] = grx_globaltimer();
        }
        relax_round<OffT, STATS>(a, L, q, T, sm);
        if (!flag_barrier(bar)) return;
        if (threadIdx.x == 0) {
            unsigned long long pk = ld_relaxed_u64(&a.ctl->qpack[(L + 1) & 3]);
            sm.q = (uint32_t)(pk >> 32);
            sm.T = (uint32_t)pk;
            sm.done = sm.q == 0;
            if (STATS && blockIdx.x == 0 && L < GRX_MAX_LEVELS_STATS) a.stats->discovered[L] = sm.q;
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->levels_run = L;
        if (STATS && L <= GRX_MAX_LEVELS_STATS) a.stats->level_t0[L] = grx_globaltimer();
    }
}

__global__ void k_sssp_init(int32_t src, const void *ro, int off64, uint32_t *dist, int32_t *Q0,
                            uint32_t *E0, TravCtl *ctl, DevStats *stats, int stats_on) {
    int64_t b = off64 ? ((const int64_t *)ro)[src] : ((const int32_t *)ro)[src];
    int64_t e = off64 ? ((const int64_t *)ro)[src + 1] : ((const int32_t *)ro)[src + 1];
    uint32_t deg = (uint32_t)(e - b);
    dist[src] = 0;
    Q0[0] = src;
    E0[0] = 0;
    ctl->qpack[0] = deg ? ((1ull << 32) | deg) : 0ull;
    for (int i = 1; i < 4; ++i) ctl->qpack[i] = 0ull;
    ctl->bar_count = 0u;
    if (stats_on) stats->levels = 0;
}

template <typename OffT, bool STATS>
grx_status launch_typed(grx_graph *g, int32_t src, uint32_t *dist, const grx_opts *o,
                        cudaStream_t s) {
    SsspArgs<OffT> a;
    a.nv = g->nv;
    a.ro = (const OffT *)g->ro;
    a.col = g->col;
    a.w = g->w;
    a.dist = dist;
    a.stamp = g->stamp;
    for (int i = 0; i < 3; ++i) {
        a.Q[i] = g->qv[i];
        a.E[i] = g->qe[i];
    }
    a.ctl = g->ctl;
    a.bar_flags = g->bar_flags;
    a.stats = g->stats;
    a.timeout_ns = grx_timeout_ns(o);
    a.src = src;
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
    if (o->collect_stats) GRX_CUDA(cudaMemsetAsync(g->stats, 0, sizeof(DevStats), s));
    k_sssp_init<<<1, 1, 0, s>>>(src, g->ro, g->off64, dist, g->qv[0], g->qe[0], g->ctl, g->stats,
                                o->collect_stats);
    GRX_CUDA(cudaGetLastError());
    if (g->off64)
        return o->collect_stats ? launch_typed<int64_t, true>(g, src, dist, o, s)
                                : launch_typed<int64_t, false>(g, src, dist, o, s);
    return o->collect_stats ? launch_typed<int32_t, true>(g, src, dist, o, s)
                            : launch_typed<int32_t, false>(g, src, dist, o, s);
}
