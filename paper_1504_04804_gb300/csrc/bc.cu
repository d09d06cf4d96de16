// Betweenness centrality (Table 1): Brandes' dependencies summed over the
// given sources, with the forward-and-backward level scheme of McLaughlin
// and Bader's GPU BC (Sec. 2) that Table 1 describes (W = 2|E|, S ~ D/2).
// For a source s: sigma[v] = number of shortest s-v paths, and
// delta[v] = sum over successors w (neighbours one level deeper) of
// sigma[v] / sigma[w] * (1 + delta[w]); bc[v] += delta[v] for v != s.
//
//  * Forward: a push BFS from s that keeps every level, in level order, in
//    one list (vertex, exclusive edge prefix within its level, row start).
//    An edge (u, w) out of level d claims an unreached w for level d + 1
//    with a compare-and-swap on its depth and, whenever w sits at depth
//    d + 1, adds sigma[u] to sigma[w] (float64 reduction).  A vertex's
//    predecessors are few where it matters: hubs are reached early, from
//    small levels.
//  * Backward, level k from the deepest one up, one phase per level: every
//    vertex v of level k sums coef[w] = (1 + delta[w]) / sigma[w] over its
//    neighbours w at depth k + 1 (a pull: no atomic per edge, so a hub with
//    a million successors costs no contention).  With acc[v] that sum,
//    delta[v] = sigma[v] * acc[v]; v adds it to bc[v] and leaves
//    coef[v] = 1 / sigma[v] + acc[v] for level k - 1.  The sums are per row
//    of the level's equal warp tiles (shared-memory partials); a row that
//    crosses tiles adds its partials to acc[v] and a per-vertex edge count,
//    and the tile that completes the count finishes v (fence, then read).
//    The deepest level has no successors: coef = 1 / sigma, delta = 0.
// One persistent cooperative kernel; levels separated by the bounded grid
// barrier.  Float64 throughout: path counts are exact integers below 2^53,
// and sums differ from a sequential order only in the last bits.
#include "grx_internal.cuh"

namespace {

constexpr int BC_BLOCK = 256;
constexpr int BC_WARPS = BC_BLOCK / 32;
constexpr int BC_ITEMS = 8;
constexpr int BC_WTILE = 32 * BC_ITEMS;
static_assert(BC_WTILE == 256, "warp_tile_rows8 covers 256-position tiles");

template <typename OffT>
struct BcArgs {
    const OffT *ro;
    const int32_t *col;
    int32_t *depth;
    double *sigma;
    double *acc;               // backward: row sums, then coef of finished vertices
    unsigned int *cnt;         // backward: edges summed so far of rows crossing tiles (left at 0)
    double *bc;
    int32_t *Q;                // every level's vertices, level after level
    uint32_t *E;               // exclusive edge prefix within the vertex's level
    OffT *R;                   // row start
    uint32_t *lstart;          // per level: index of its first vertex in Q
    uint32_t *ledges;          // per level: its edges
    TravCtl *ctl;
    unsigned int *bar_flags;
    unsigned long long timeout_ns;
    int32_t src;
};

struct BcState {
    int d;                     // level being processed
    int back;                  // 0 forward, 1 backward
    int deepest;               // backward: d is the deepest level
    int done;
    int levels;                // levels of the traversal (known once the forward pass ends)
    uint32_t start, q, T;      // level d: first list index, vertices, edges
};

template <typename OffT>
struct BcWarpSmem {
    uint32_t qe[BC_WTILE + 2];
    OffT rs[BC_WTILE + 1];
    double val[BC_WTILE + 1];  // forward: sigma of the element; backward: its row's partial sum
    alignas(16) uint16_t rid[BC_WTILE];
};

// Stages the level elements that start before e1 (from index i0) into shared
// memory; returns their count.  Forward also stages sigma of each element.
template <typename OffT, bool BACK>
__device__ __forceinline__ int stage_elements(const BcArgs<OffT> &a, const int32_t *Qv, const uint32_t *Qe,
                                              const OffT *Qr, int64_t q, int64_t i0, uint32_t e1,
                                              BcWarpSmem<OffT> &w) {
    const unsigned int lane = threadIdx.x & 31;
    int n = 0;
    for (;;) {
        const int64_t idx = i0 + n + lane;
        uint32_t qe = 0xffffffffu;
        if (idx < q) qe = __ldcg(Qe + idx);
        const bool in = idx < q && qe < e1;
        if (n + (int)lane <= BC_WTILE + 1) w.qe[n + lane] = qe;
        if (in && n + (int)lane <= BC_WTILE) {
            w.rs[n + lane] = __ldcg(Qr + idx);
            w.val[n + lane] = BACK ? 0.0 : __ldcg(a.sigma + __ldcg(Qv + idx));
        }
        const int cnt = __popc(__ballot_sync(GRX_FULL_MASK, in));
        n += cnt;
        if (cnt < 32) break;
        if (n > BC_WTILE) {                  // only possible with a malformed graph
            if (lane == 0) grx_set_status(a.ctl, GRX_EINVAL);
            n = BC_WTILE;
            break;
        }
    }
    __syncwarp();
    return n;
}

// Finishes v of level k >= 1 from its successor sum s.
template <typename OffT>
__device__ __forceinline__ void finish_vertex(const BcArgs<OffT> &a, int32_t v, double s) {
    const double sg = __ldcg(a.sigma + v);
    const double dv = sg * s;
    if (dv != 0.0) a.bc[v] += dv;            // v occurs once per source: plain update
    a.acc[v] = 1.0 / sg + s;
}

// Forward step of level d: claims level d + 1 and adds path counts.
template <typename OffT>
__device__ void forward_level(const BcArgs<OffT> &a, const BcState &st, BcWarpSmem<OffT> &w) {
    const int d = st.d;
    const unsigned int lane = threadIdx.x & 31;
    const int32_t *Qv = a.Q + st.start;
    const uint32_t *Qe = a.E + st.start;
    const OffT *Qr = a.R + st.start;
    int32_t *Qv_out = a.Q + st.start + st.q;          // level d + 1 follows level d
    uint32_t *Qe_out = a.E + st.start + st.q;
    OffT *Qr_out = a.R + st.start + st.q;
    unsigned long long *ctr = &a.ctl->qpack[(d + 1) & 3];
    const uint64_t T = st.T;
    const uint64_t ntiles = (T + BC_WTILE - 1) / BC_WTILE;
    const uint64_t nwarps = (uint64_t)gridDim.x * BC_WARPS;
    const uint64_t gw = (uint64_t)blockIdx.x * BC_WARPS + (threadIdx.x >> 5);
    const uint64_t per = (ntiles + nwarps - 1) / nwarps;
    const uint64_t tb0 = gw * per;
    const uint64_t tb1 = min(ntiles, tb0 + per);
    if (tb0 >= tb1) return;
    int64_t i0 = warp_upper_index_cg(Qe, st.q, (uint32_t)(tb0 * BC_WTILE));
    for (uint64_t tile = tb0; tile < tb1; ++tile) {
        const uint64_t e0 = tile * BC_WTILE;
        const uint32_t e1 = (uint32_t)min(T, e0 + BC_WTILE);
        const int n = stage_elements<OffT, false>(a, Qv, Qe, Qr, st.q, i0, e1, w);
        const uint32_t next_start = w.qe[n];
        int row[BC_ITEMS];
        warp_tile_rows8(w.rid, w.qe, (uint32_t)e0, n, row);
        const uint32_t t0 = (uint32_t)e0 + lane * BC_ITEMS;
        int32_t v[BC_ITEMS];
        double su[BC_ITEMS];
#pragma unroll
        for (int k = 0; k < BC_ITEMS; ++k) {
            const uint32_t e = t0 + k;
            const int j = row[k];
            const bool ok = e < e1;
            const OffT idx = ok ? w.rs[j] + (OffT)(e - w.qe[j]) : (OffT)0;
            v[k] = ok ? __ldg(a.col + idx) : -1;
            su[k] = ok ? w.val[j] : 0.0;
        }
        __syncwarp();
        int dv[BC_ITEMS];
#pragma unroll
        for (int k = 0; k < BC_ITEMS; ++k) dv[k] = v[k] >= 0 ? __ldcg(a.depth + v[k]) : -2;
        uint32_t claimed = 0;
#pragma unroll
        for (int k = 0; k < BC_ITEMS; ++k) {
            if (dv[k] == -1) {
                const int old = atomicCAS(a.depth + v[k], -1, d + 1);
                if (old == -1) claimed |= 1u << k;
                dv[k] = old == -1 ? d + 1 : old;
            }
        }
#pragma unroll
        for (int k = 0; k < BC_ITEMS; ++k)
            if (dv[k] == d + 1) atomicAdd(a.sigma + v[k], su[k]);       // result unused: reduction
        uint32_t deg[BC_ITEMS];
        OffT rb[BC_ITEMS];
        uint32_t app = 0;
#pragma unroll
        for (int k = 0; k < BC_ITEMS; ++k) {
            rb[k] = 0;
            deg[k] = 0;
            if (claimed >> k & 1u) {
                rb[k] = __ldg(a.ro + v[k]);
                deg[k] = (uint32_t)(__ldg(a.ro + v[k] + 1) - rb[k]);
                if (deg[k]) app |= 1u << k;
            }
        }
        warp_append_items<BC_ITEMS, OffT>(v, deg, rb, app, Qv_out, Qe_out, Qr_out, ctr);
        i0 = (next_start == e1) ? i0 + n : i0 + n - 1;
        __syncwarp();
    }
}

// Backward step of level k >= 1 (not the deepest): pull of the successors'
// coefficients, per-row sums, vertices finished.
template <typename OffT>
__device__ void backward_level(const BcArgs<OffT> &a, const BcState &st, BcWarpSmem<OffT> &w) {
    const int k1 = st.d + 1;
    const unsigned int lane = threadIdx.x & 31;
    const int32_t *Qv = a.Q + st.start;
    const uint32_t *Qe = a.E + st.start;
    const OffT *Qr = a.R + st.start;
    const uint64_t T = st.T;
    const uint64_t ntiles = (T + BC_WTILE - 1) / BC_WTILE;
    const uint64_t nwarps = (uint64_t)gridDim.x * BC_WARPS;
    const uint64_t gw = (uint64_t)blockIdx.x * BC_WARPS + (threadIdx.x >> 5);
    const uint64_t per = (ntiles + nwarps - 1) / nwarps;
    const uint64_t tb0 = gw * per;
    const uint64_t tb1 = min(ntiles, tb0 + per);
    if (tb0 >= tb1) return;
    int64_t i0 = warp_upper_index_cg(Qe, st.q, (uint32_t)(tb0 * BC_WTILE));
    for (uint64_t tile = tb0; tile < tb1; ++tile) {
        const uint64_t e0 = tile * BC_WTILE;
        const uint32_t e1 = (uint32_t)min(T, e0 + BC_WTILE);
        const int n = stage_elements<OffT, true>(a, Qv, Qe, Qr, st.q, i0, e1, w);
        const uint32_t next_start = w.qe[n];
        int row[BC_ITEMS];
        warp_tile_rows8(w.rid, w.qe, (uint32_t)e0, n, row);
        const uint32_t t0 = (uint32_t)e0 + lane * BC_ITEMS;
        int32_t u[BC_ITEMS];
#pragma unroll
        for (int k = 0; k < BC_ITEMS; ++k) {
            const uint32_t e = t0 + k;
            const int j = row[k];
            const OffT idx = e < e1 ? w.rs[j] + (OffT)(e - w.qe[j]) : (OffT)0;
            u[k] = e < e1 ? __ldg(a.col + idx) : -1;
        }
        int du[BC_ITEMS];
#pragma unroll
        for (int k = 0; k < BC_ITEMS; ++k) du[k] = u[k] >= 0 ? __ldcg(a.depth + u[k]) : -2;
        double c[BC_ITEMS];
#pragma unroll
        for (int k = 0; k < BC_ITEMS; ++k) c[k] = du[k] == k1 ? __ldcg(a.acc + u[k]) : 0.0;
        // runs of equal rows within the lane, added into the rows' shared partials
        {
            int cj = row[0];
            double part = 0.0;
#pragma unroll
            for (int k = 0; k < BC_ITEMS; ++k) {
                if (t0 + k < e1) {
                    if (row[k] != cj) {
                        if (part != 0.0) atomicAdd(&w.val[cj], part);
                        part = 0.0;
                        cj = row[k];
                    }
                    part += c[k];
                }
            }
            if (part != 0.0) atomicAdd(&w.val[cj], part);
        }
        __syncwarp();
        // rows inside the tile finish here; rows crossing it go through acc and cnt
        for (int j = (int)lane; j < n; j += 32) {
            const uint32_t rb = w.qe[j];
            const uint32_t re = i0 + j + 1 < (int64_t)st.q ? w.qe[j + 1] : (uint32_t)T;   // row end
            const uint32_t lo = rb > (uint32_t)e0 ? rb : (uint32_t)e0;
            const uint32_t hi = re < e1 ? re : e1;
            if (hi <= lo) continue;                          // empty row
            const int32_t v = __ldcg(Qv + i0 + j);
            const double s = w.val[j];
            if (rb >= (uint32_t)e0 && re <= e1) {
                finish_vertex(a, v, s);
            } else {
                const uint32_t len = re - rb;
                if (s != 0.0) atomicAdd(a.acc + v, s);
                __threadfence();
                const unsigned int before = atomicAdd(a.cnt + v, hi - lo);
                if (before + (hi - lo) == len) {             // every tile of the row has added
                    __threadfence();
                    a.cnt[v] = 0u;
                    finish_vertex(a, v, __ldcg(a.acc + v));
                }
            }
        }
        i0 = (next_start == e1) ? i0 + n : i0 + n - 1;
        __syncwarp();
    }
}

// Deepest level: no successors.
template <typename OffT>
__device__ void deepest_level(const BcArgs<OffT> &a, const BcState &st) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)st.q;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = __ldcg(a.Q + st.start + i);
        a.acc[v] = 1.0 / __ldcg(a.sigma + v);
    }
}

template <typename OffT>
__device__ BcState bc_next(const BcArgs<OffT> &a, const BcState &st) {
    BcState ns = st;
    ns.deepest = 0;
    if (!st.back) {
        const unsigned long long pk = ld_relaxed_u64(&a.ctl->qpack[(st.d + 1) & 3]);
        const uint32_t q = (uint32_t)(pk >> 32);
        if (q > 0) {
            ns.d = st.d + 1;
            ns.start = st.start + st.q;
            ns.q = q;
            ns.T = (uint32_t)pk;
        } else {
            ns.levels = st.d + 1;
            ns.back = 1;                                     // level d is the deepest
            ns.deepest = 1;
            ns.done = st.d == 0;                             // only the source: nothing to add
        }
        return ns;
    }
    if (st.d == 1) {
        ns.done = 1;
        return ns;
    }
    ns.d = st.d - 1;
    ns.start = ld_relaxed_u32(a.lstart + ns.d);
    ns.q = st.start - ns.start;
    ns.T = ld_relaxed_u32(a.ledges + ns.d);
    return ns;
}

template <typename OffT>
__global__ void __launch_bounds__(BC_BLOCK) k_bc_persistent(BcArgs<OffT> a) {
    __shared__ BcState s_st;
    __shared__ BcWarpSmem<OffT> wsm[BC_WARPS];
    BcWarpSmem<OffT> &w = wsm[threadIdx.x >> 5];
    FlagBarrier bar{a.bar_flags, &a.ctl->bar_release, a.ctl, a.timeout_ns, 0u};
    if (threadIdx.x == 0) {
        BcState s;
        memset(&s, 0, sizeof s);
        const uint32_t deg = (uint32_t)(a.ro[a.src + 1] - a.ro[a.src]);
        s.q = 1;
        s.T = deg;
        s.done = deg == 0;
        s.levels = 1;
        s_st = s;
    }
    __syncthreads();
    for (;;) {
        const BcState st = s_st;
        if (st.done) break;
        if (!st.back) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                a.ctl->qpack[(st.d + 2) & 3] = 0ull;
                a.lstart[st.d] = st.start;
                a.ledges[st.d] = st.T;
            }
            forward_level<OffT>(a, st, w);
        } else if (st.deepest) {
            deepest_level<OffT>(a, st);
        } else {
            backward_level<OffT>(a, st, w);
        }
        if (!flag_barrier(bar)) return;
        if (threadIdx.x == 0) s_st = bc_next(a, st);
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->levels_run = s_st.levels;
}

template <typename OffT>
__global__ void k_bc_init(int32_t src, const OffT *ro, int32_t *depth, double *sigma, int32_t *Q, uint32_t *E,
                          OffT *R, TravCtl *ctl) {
    depth[src] = 0;
    sigma[src] = 1.0;
    Q[0] = src;
    E[0] = 0;
    R[0] = ro[src];
    for (int i = 0; i < 4; ++i) ctl->qpack[i] = 0ull;
}

template <typename OffT>
grx_status launch_typed(grx_graph *g, const int32_t *srcs, int n, double *bc_out, const grx_opts *o,
                        cudaStream_t s) {
    BcArgs<OffT> a;
    a.ro = (const OffT *)g->ro;
    a.col = g->col;
    a.depth = g->stamp;
    a.sigma = g->bc_sigma;
    a.acc = g->bc_acc;
    a.cnt = reinterpret_cast<unsigned int *>(g->ulist[0]);
    a.bc = bc_out;
    a.Q = g->qv[0];
    a.E = g->qe[0];
    a.R = (OffT *)g->qr[0];
    a.lstart = g->qe[1];
    a.ledges = g->qe[2];
    a.ctl = g->ctl;
    a.bar_flags = g->bar_flags;
    a.timeout_ns = grx_timeout_ns(o);
    static int per_sm = -1;
    if (per_sm < 0) {
        GRX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bc_persistent<OffT>, BC_BLOCK, 0));
        if (per_sm < 1) return grx_fail(GRX_ECUDA, "bc: persistent kernel does not fit on an SM");
    }
    int max_grid = per_sm * g->ctx->num_sms;
    if (max_grid > GRX_MAX_GRID) max_grid = GRX_MAX_GRID;
    const int blocks = o->grid_blocks > 0 && o->grid_blocks < max_grid ? o->grid_blocks : max_grid;
    const size_t nv = (size_t)g->nv;
    GRX_CUDA(cudaMemsetAsync(bc_out, 0, nv * 8, s));
    GRX_CUDA(cudaMemsetAsync(a.cnt, 0, nv * 4, s));
    if (o->ev_begin) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_begin, s));
    for (int i = 0; i < n; ++i) {
        a.src = srcs[i];
        GRX_CUDA(cudaMemsetAsync(a.depth, 0xff, nv * 4, s));
        GRX_CUDA(cudaMemsetAsync(a.sigma, 0, nv * 8, s));
        GRX_CUDA(cudaMemsetAsync(a.acc, 0, nv * 8, s));
        k_bc_init<OffT><<<1, 1, 0, s>>>(a.src, a.ro, a.depth, a.sigma, a.Q, a.E, a.R, g->ctl);
        GRX_CUDA(cudaGetLastError());
        GRX_CUDA(cudaMemsetAsync(g->bar_flags, 0, sizeof(unsigned int) * (size_t)blocks, s));
        GRX_CUDA(cudaMemsetAsync(&g->ctl->bar_release, 0, sizeof(unsigned int), s));
        void *args[] = {(void *)&a};
        GRX_CUDA(cudaLaunchCooperativeKernel((const void *)k_bc_persistent<OffT>, dim3(blocks), dim3(BC_BLOCK),
                                             args, 0, s));
    }
    if (o->ev_end) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_end, s));
    return GRX_OK;
}

}  // namespace

grx_status grx_bc_launch(grx_graph *g, const int32_t *srcs, int n, double *bc_out, double *sigma_out,
                         const grx_opts *o, cudaStream_t s) {
    grx_status st = g->off64 ? launch_typed<int64_t>(g, srcs, n, bc_out, o, s)
                             : launch_typed<int32_t>(g, srcs, n, bc_out, o, s);
    if (st != GRX_OK) return st;
    if (sigma_out) GRX_CUDA(cudaMemcpyAsync(sigma_out, g->bc_sigma, (size_t)g->nv * 8, cudaMemcpyDeviceToDevice, s));
    return GRX_OK;
}
