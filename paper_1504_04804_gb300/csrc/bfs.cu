// BFS and direction-optimising BFS (Algorithms 1 and 2, Sec. 6.1).
//
// Design (one GPU, GB300):
//  * The whole traversal is one cooperative persistent kernel; levels are
//    separated by a bounded grid barrier, so no host round trip or launch
//    happens per level (the per-iteration overhead l of Sec. 5.2).  A
//    host-stepped variant (one launch per level) exists for comparison.
//  * Push (top-down) advance+filter are fused (Sec. 6.3): each frontier slot
//    carries the exclusive prefix of its vertices' degrees, produced by the
//    same warp-aggregated atomic that appends the vertex, so the next level
//    splits the frontier's edges into equal tiles with no separate scan.  A
//    tile's threads find their source vertex by binary search in shared
//    memory; the visited bitmap is the filter (test, then atomicOr).
//  * Pull (bottom-up): one thread per unvisited vertex scans its neighbours
//    in order and stops at the first one in the frontier bitmap (edge
//    skipping); no atomics on labels.  The unvisited list is split into the
//    newly discovered vertices (appended to the next push-ready frontier,
//    so pull->push costs nothing, Sec. 6.1) and the still-unvisited list.
//  * Direction switch (Sec. 6.1): FV = |Q|*E/V, BV = |U|*V/|P|; push->pull
//    once when FV > BV*alpha, pull->push when FV < BV*beta.  Every block
//    evaluates it identically from the device counters after the barrier.
#include <cstdio>

#include "grx_internal.cuh"

namespace {

constexpr int BFS_BLOCK = 256;
constexpr int PUSH_ITEMS = 8;
constexpr int PUSH_TILE = BFS_BLOCK * PUSH_ITEMS;   // edges per tile

enum { DIR_PUSH = 0, DIR_PULL = 1 };

struct LevelState {
    int L;            // level being expanded (frontier = vertices at depth L)
    int dir;
    int switched;     // push->pull has happened
    int back;         // pull->push has happened (final)
    int first_pull;   // pull level without an unvisited list yet: scan all vertices
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
    const OffT *ro;
    const int32_t *col;
    const uint32_t *nz;
    uint32_t *visited;
    uint32_t *F[3];
    int32_t *Q[3];
    uint32_t *E[3];
    int32_t *U[2];
    int32_t *depth;
    int32_t *parent;
    TravCtl *ctl;
    DevStats *stats;
    int mode;
    float alpha, beta;
    unsigned long long timeout_ns;
    int32_t src;
};

template <typename OffT>
struct PushSmem {
    uint32_t qe[PUSH_TILE + 1];
    int32_t u[PUSH_TILE + 1];
    OffT rs[PUSH_TILE + 1];
    int64_t i0;
    int n;
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
    uint32_t deg = (uint32_t)(a.ro[a.src + 1] - a.ro[a.src]);
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
        // Sec. 6.1 estimates: FV = |Q|*E/V, BV = |U|*V/|P|, P = visited incl. Q
        double V = (double)a.nv, E = (double)a.ne;
        double FV = (double)ns.q * E / V;
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
__device__ void push_level(const BfsArgs<OffT> &a, const LevelState &st, PushSmem<OffT> &sm) {
    const int L = st.L;
    const int32_t *Qv = pick3(a.Q[0], a.Q[1], a.Q[2], L % 3);
    const uint32_t *Qe = pick3(a.E[0], a.E[1], a.E[2], L % 3);
    int32_t *Qv_out = pick3(a.Q[0], a.Q[1], a.Q[2], (L + 1) % 3);
    uint32_t *Qe_out = pick3(a.E[0], a.E[1], a.E[2], (L + 1) % 3);
    uint32_t *Fout = pick3(a.F[0], a.F[1], a.F[2], (L + 1) % 3);
    unsigned long long *ctr = &a.ctl->qpack[(L + 1) & 3];
    const uint32_t q = st.q;
    const uint64_t T = st.T;
    const uint64_t ntiles = (T + PUSH_TILE - 1) / PUSH_TILE;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t e0 = tile * PUSH_TILE;
        const uint64_t e1 = min(T, e0 + PUSH_TILE);
        if (threadIdx.x == 0) {
            int64_t i0 = upper_index_cg(Qe, q, (uint32_t)e0);
            int64_t i1 = upper_index_cg(Qe, q, (uint32_t)(e1 - 1));
            int n = (int)(i1 - i0 + 1);
            if (n > PUSH_TILE + 1) {      // only possible with a malformed graph
                grx_set_status(a.ctl, GRX_EINVAL);
                n = PUSH_TILE + 1;
            }
            sm.i0 = i0;
            sm.n = n;
        }
        __syncthreads();
        const int64_t i0 = sm.i0;
        const int n = sm.n;
        for (int j = threadIdx.x; j < n; j += BFS_BLOCK) {
            int32_t u = __ldcg(Qv + i0 + j);
            sm.qe[j] = __ldcg(Qe + i0 + j);
            sm.u[j] = u;
            sm.rs[j] = __ldg(a.ro + u);
        }
        __syncthreads();
#pragma unroll 2
        for (int k = 0; k < PUSH_ITEMS; ++k) {
            const uint64_t e = e0 + (uint64_t)(k * BFS_BLOCK + threadIdx.x);
            bool disc = false;
            int32_t v = 0;
            uint32_t deg = 0;
            if (e < e1) {
                int j = upper_index_smem(sm.qe, n, (uint32_t)e);
                int32_t u = sm.u[j];
                v = __ldg(a.col + sm.rs[j] + (OffT)((uint32_t)e - sm.qe[j]));
                const uint32_t bit = 1u << (v & 31);
                uint32_t *wp = a.visited + (v >> 5);
                if (!(__ldcg(wp) & bit)) {
                    uint32_t old = atomicOr(wp, bit);
                    if (!(old & bit)) {
                        disc = true;
                        a.depth[v] = L + 1;
                        if (PARENT) a.parent[v] = u;
                        deg = (uint32_t)(__ldg(a.ro + v + 1) - __ldg(a.ro + v));
                        if (st.fwrite && deg) atomicOr(Fout + (v >> 5), bit);
                    }
                }
            }
            warp_append_frontier(disc && deg > 0, v, deg, Qv_out, Qe_out, ctr);
        }
        __syncthreads();
    }
    if (STATS && blockIdx.x == 0 && threadIdx.x == 0 && L < GRX_MAX_LEVELS_STATS) {
        a.stats->edges_examined[L] = T;
        a.stats->vertices_scanned[L] = q;
    }
}

template <typename OffT, bool PARENT, bool STATS>
__device__ void pull_level(const BfsArgs<OffT> &a, const LevelState &st) {
    const int L = st.L;
    const uint32_t *Fin = pick3(a.F[0], a.F[1], a.F[2], L % 3);
    uint32_t *Fout = pick3(a.F[0], a.F[1], a.F[2], (L + 1) % 3);
    int32_t *Qv_out = pick3(a.Q[0], a.Q[1], a.Q[2], (L + 1) % 3);
    uint32_t *Qe_out = pick3(a.E[0], a.E[1], a.E[2], (L + 1) % 3);
    unsigned long long *ctr = &a.ctl->qpack[(L + 1) & 3];
    const int32_t *Uin = (L & 1) ? a.U[1] : a.U[0];
    int32_t *Uout = (L & 1) ? a.U[0] : a.U[1];
    unsigned int *uctr = &a.ctl->ucount[(L + 1) & 3];
    const bool first = st.first_pull != 0;
    const int64_t count = first ? (int64_t)a.nv : (int64_t)st.ucount;
    const int64_t span = (count + 31) & ~(int64_t)31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long scanned_e = 0, scanned_v = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < span; i += stride) {
        int32_t v = -1;
        if (i < count) {
            if (first) {
                uint32_t w = __ldg(a.nz + (i >> 5)) & ~__ldcg(a.visited + (i >> 5));
                if ((w >> (i & 31)) & 1u) v = (int32_t)i;
            } else {
                v = __ldcg(Uin + i);
            }
        }
        bool found = false, still = false;
        uint32_t deg = 0;
        if (v >= 0) {
            const OffT b = __ldg(a.ro + v), e = __ldg(a.ro + v + 1);
            int32_t par = -1;
            OffT k = b;
            for (; k < e; ++k) {
                int32_t u = __ldg(a.col + k);
                if ((__ldcg(Fin + (u >> 5)) >> (u & 31)) & 1u) {
                    par = u;
                    break;
                }
            }
            if (STATS) {
                scanned_v += 1;
                scanned_e += (unsigned long long)((k < e ? k + 1 : e) - b);
            }
            if (par >= 0) {
                found = true;
                a.depth[v] = L + 1;
                if (PARENT) a.parent[v] = par;
                const uint32_t bit = 1u << (v & 31);
                atomicOr(a.visited + (v >> 5), bit);
                deg = (uint32_t)(e - b);
                if (st.fwrite) atomicOr(Fout + (v >> 5), bit);
            } else {
                still = true;
            }
        }
        warp_append_frontier(found, v, deg, Qv_out, Qe_out, ctr);
        warp_append_list(still, v, Uout, uctr);
    }
    if (STATS) {
        scanned_e = warp_sum(scanned_e);
        scanned_v = warp_sum(scanned_v);
        if (lane_id() == 0 && L < GRX_MAX_LEVELS_STATS) {
            if (scanned_e) atomicAdd(&a.stats->edges_examined[L], scanned_e);
            if (scanned_v) atomicAdd(&a.stats->vertices_scanned[L], scanned_v);
        }
    }
}

template <typename OffT, bool PARENT, bool STATS>
__device__ void run_level(const BfsArgs<OffT> &a, const LevelState &st, PushSmem<OffT> &sm) {
    const int L = st.L;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->qpack[(L + 2) & 3] = 0ull;
        a.ctl->ucount[(L + 2) & 3] = 0u;
        if (STATS && L < GRX_MAX_LEVELS_STATS) {
            a.stats->dir[L] = st.dir;
            a.stats->frontier[L] = st.q;
            a.stats->levels = L + 1;
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
    if (st.dir == DIR_PUSH) push_level<OffT, PARENT, STATS>(a, st, sm);
    else pull_level<OffT, PARENT, STATS>(a, st);
}

template <typename OffT, bool PARENT, bool STATS>
__global__ void __launch_bounds__(BFS_BLOCK) k_bfs_persistent(BfsArgs<OffT> a) {
    __shared__ LevelState s_st;
    __shared__ PushSmem<OffT> sm;
    if (threadIdx.x == 0) s_st = initial_state(a);
    __syncthreads();
    for (;;) {
        const LevelState st = s_st;
        if (st.done) break;
        run_level<OffT, PARENT, STATS>(a, st, sm);
        if (!grid_barrier(a.ctl, a.timeout_ns)) break;
        if (threadIdx.x == 0) s_st = next_state(a, st, STATS);
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->levels_run = s_st.L;
}

// Host-stepped variant: launch i runs level i.  The state of level i is
// derived at the start of launch i from the state launch i-1 stored and the
// counters it left, so no block ever waits on another.
template <typename OffT, bool PARENT, bool STATS>
__global__ void __launch_bounds__(BFS_BLOCK) k_bfs_step(BfsArgs<OffT> a, int launch) {
    __shared__ LevelState s_st;
    __shared__ PushSmem<OffT> sm;
    static_assert(sizeof(LevelState) <= sizeof(long long) * 8, "state must fit hstate");
    if (threadIdx.x == 0) {
        LevelState st;
        if (launch == 0) {
            st = initial_state(a);
        } else {
            LevelState prev;
            memcpy(&prev, (const void *)a.ctl->hstate[(launch - 1) & 1], sizeof prev);
            st = prev.done ? prev : next_state(a, prev, STATS);
        }
        s_st = st;
    }
    __syncthreads();
    const LevelState st = s_st;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        memcpy((void *)a.ctl->hstate[launch & 1], &st, sizeof st);
        if (st.done) a.ctl->levels_run = st.L;
    }
    if (st.done) return;
    run_level<OffT, PARENT, STATS>(a, st, sm);
}

__global__ void k_bfs_init(int32_t src, const void *ro, int off64, int32_t *depth, int32_t *parent,
                           uint32_t *visited, uint32_t *F0, int32_t *Q0, uint32_t *E0,
                           TravCtl *ctl, DevStats *stats, int stats_on) {
    int64_t b = off64 ? ((const int64_t *)ro)[src] : ((const int32_t *)ro)[src];
    int64_t e = off64 ? ((const int64_t *)ro)[src + 1] : ((const int32_t *)ro)[src + 1];
    uint32_t deg = (uint32_t)(e - b);
    depth[src] = 0;
    if (parent) parent[src] = src;
    visited[src >> 5] = 1u << (src & 31);
    if (F0 && deg) F0[src >> 5] = 1u << (src & 31);
    Q0[0] = src;
    E0[0] = 0;
    ctl->qpack[0] = deg ? ((1ull << 32) | deg) : 0ull;
    for (int i = 1; i < 4; ++i) ctl->qpack[i] = 0ull;
    for (int i = 0; i < 4; ++i) ctl->ucount[i] = 0u;
    ctl->bar_count = 0u;
    ctl->levels_run = 0;
    if (stats_on) stats->levels = 0;
}

template <typename OffT>
BfsArgs<OffT> make_args(grx_graph *g, int32_t src, int32_t *depth, int32_t *parent,
                        const grx_opts *o) {
    BfsArgs<OffT> a;
    a.nv = g->nv;
    a.ne = g->ne;
    a.ro = (const OffT *)g->ro;
    a.col = g->col;
    a.nz = g->nz_bits;
    a.visited = g->visited;
    for (int i = 0; i < 3; ++i) {
        a.F[i] = g->fbits[i];
        a.Q[i] = g->qv[i];
        a.E[i] = g->qe[i];
    }
    a.U[0] = g->ulist[0];
    a.U[1] = g->ulist[1];
    a.depth = depth;
    a.parent = parent;
    a.ctl = g->ctl;
    a.stats = g->stats;
    a.mode = o->direction;
    a.alpha = o->alpha;
    a.beta = o->beta;
    a.timeout_ns = grx_timeout_ns(o);
    a.src = src;
    return a;
}

template <typename OffT, bool PARENT, bool STATS>
grx_status launch_typed(grx_graph *g, int32_t src, int32_t *depth, int32_t *parent,
                        const grx_opts *o, cudaStream_t s) {
    BfsArgs<OffT> a = make_args<OffT>(g, src, depth, parent, o);
    if (o->loop == GRX_LOOP_HOST) {
        int blocks = o->grid_blocks > 0 ? o->grid_blocks : g->ctx->num_sms * 4;
        // Poll the done flag every 16 launches; a traversal has at most nv levels.
        long long st_host[8];
        if (o->ev_begin) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_begin, s));
        for (int launch = 0; launch <= g->nv; ++launch) {
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
    int blocks = o->grid_blocks > 0 && o->grid_blocks < max_grid ? o->grid_blocks : max_grid;
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
    const size_t nv = (size_t)g->nv;
    const size_t wb = (size_t)g->words * 4;
    GRX_CUDA(cudaMemsetAsync(depth, 0xff, nv * 4, s));
    if (parent) GRX_CUDA(cudaMemsetAsync(parent, 0xff, nv * 4, s));
    GRX_CUDA(cudaMemsetAsync(g->visited, 0, wb, s));
    const bool use_f = o->direction != GRX_DIR_PUSH;
    if (use_f)
        for (int i = 0; i < 3; ++i) GRX_CUDA(cudaMemsetAsync(g->fbits[i], 0, wb, s));
    if (o->collect_stats) GRX_CUDA(cudaMemsetAsync(g->stats, 0, sizeof(DevStats), s));
    k_bfs_init<<<1, 1, 0, s>>>(src, g->ro, g->off64, depth, parent, g->visited,
                               use_f ? g->fbits[0] : nullptr, g->qv[0], g->qe[0], g->ctl,
                               g->stats, o->collect_stats);
    GRX_CUDA(cudaGetLastError());
    return g->off64 ? launch_off<int64_t>(g, src, depth, parent, o, s)
                    : launch_off<int32_t>(g, src, depth, parent, o, s);
}
