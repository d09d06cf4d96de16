// BFS over graphs with 64-bit vertex ids (Sec. 6.2 and Sec. 7: graphs too
// large for 32-bit ids take 64-bit ids, at about half the throughput).
//
// A separate, simpler traversal than bfs.cu's, 64-bit throughout: vertex ids,
// row offsets, frontier sizes and edge counts are int64, so nothing here
// limits a graph to 2^31 vertices or 2^32 edges.  The same direction-
// optimising rule (Sec. 6.1) picks push or pull per level; one cooperative
// persistent kernel runs every level, phases separated by the bounded flag
// barrier.
//  * Push: a warp per frontier vertex walks the first LONG edges of its row
//    (visited test, then atomicOr; the winner labels the vertex and appends
//    it to the next queue).  A row longer than that leaves its remainder on a
//    long-row list whose append counter packs (rows << 40 | LONG-edge chunks),
//    so row bases come out in position order; a second phase hands the
//    chunks to warps from a counter, so a hub's edges spread over the grid.
//  * Pull: warps own 32-word chunks of the bitmaps (chunks from a counter);
//    each candidate (unvisited, with edges) scans its row until a neighbour
//    is in the frontier (edge skipping); the owner writes its visited and
//    next-frontier words whole.
//  * A push level after pull levels first turns the frontier bitmap into a
//    queue (a compaction phase).
// Frontier bitmaps rotate through three slots; each level zeroes the slot of
// level L-1, which is the slot level L+1 fills.
#include "grx_internal.cuh"

namespace {

constexpr int B64_BLOCK = 256;
constexpr int B64_WARPS = B64_BLOCK / 32;
constexpr int64_t LONG = 1024;                 // row edges a push warp takes at once
constexpr int CHUNK_VERTS = 1024;              // vertices of a 32-word chunk
constexpr int LR_SHIFT = 40;                   // long-row counter: rows << 40 | chunks

enum { D_PUSH = 0, D_PULL = 1 };

struct B64Args {
    int64_t nv, ne, words;
    const int64_t *ro;
    const int64_t *col;
    const uint32_t *nz;
    uint32_t *vis;
    uint32_t *F[3];
    int64_t *Q[2];
    int64_t *lu, *ls;                          // long rows: vertex, next edge
    unsigned long long *lb;                    // long rows: first chunk
    int32_t *depth;
    int64_t *parent;
    TravCtl *ctl;
    unsigned int *bar_flags;
    int mode, exact_fv;
    float alpha, beta;
    unsigned long long timeout_ns;
    int64_t src;
};

// Level-L counters (rings of 4): frontier size, frontier edges, long rows,
// compaction appends; a phase's chunk counter rotates with the phase number.
__device__ __forceinline__ unsigned long long *cnt_q(const B64Args &a, int64_t L) { return &a.ctl->qpack[L & 3]; }
__device__ __forceinline__ unsigned long long *cnt_e(const B64Args &a, int64_t L) { return &a.ctl->pairs[L & 3]; }
__device__ __forceinline__ unsigned long long *cnt_lr(const B64Args &a, int64_t L) {
    return reinterpret_cast<unsigned long long *>(&a.ctl->hstate[0][L & 3]);
}
__device__ __forceinline__ unsigned long long *cnt_cq(const B64Args &a, int64_t L) {
    return reinterpret_cast<unsigned long long *>(&a.ctl->hstate[1][L & 3]);
}

struct B64State {
    int64_t L;
    uint64_t q, T, vcount;
    uint32_t seq;                               // phases run (chunk-counter ring)
    uint8_t dir, switched, back, done, qin;
};

__device__ __forceinline__ int64_t rdeg(const B64Args &a, int64_t v) { return __ldg(a.ro + v + 1) - __ldg(a.ro + v); }

// Next level's state from the counters level st.L left (Sec. 6.1 rule).
__device__ B64State b64_next(const B64Args &a, const B64State &st) {
    B64State ns = st;
    ns.L = st.L + 1;
    ns.q = ld_relaxed_u64(cnt_q(a, ns.L));
    ns.T = ld_relaxed_u64(cnt_e(a, ns.L));
    ns.vcount = st.vcount + ns.q;
    ns.qin = st.dir == D_PUSH;
    if (ns.q == 0) {
        ns.done = 1;
        return ns;
    }
    if (a.mode == GRX_DIR_PUSH) {
        ns.dir = D_PUSH;
    } else if (a.mode == GRX_DIR_PULL) {
        ns.dir = D_PULL;
    } else {
        const double V = (double)a.nv, E = (double)a.ne;
        const double FV = a.exact_fv ? (double)ns.T : (double)ns.q * E / V;
        const double BV = (double)(a.nv - (int64_t)ns.vcount) * V / (double)ns.vcount;
        if (st.dir == D_PUSH && !st.switched && FV > BV * (double)a.alpha) {
            ns.dir = D_PULL;
            ns.switched = 1;
        } else if (st.dir == D_PULL && FV < BV * (double)a.beta) {
            ns.dir = D_PUSH;
            ns.back = 1;
        }
    }
    return ns;
}

// A push warp's edges [e0, e1) of row u (lane-strided): visited test, claim,
// label, append.  Appends and edge totals are aggregated per warp step.
__device__ __forceinline__ void push_edges(const B64Args &a, int64_t L, int64_t u, int64_t e0, int64_t e1,
                                           uint32_t *Fout, int64_t *Qout) {
    const unsigned int lane = threadIdx.x & 31;
    for (int64_t base = e0; base < e1; base += 32) {
        const int64_t e = base + lane;
        bool won = false;
        int64_t v = -1;
        if (e < e1) {
            v = __ldg(a.col + e);
            const uint32_t bit = 1u << (v & 31);
            if (!(__ldca(a.vis + (v >> 5)) & bit)) {
                const uint32_t old = atomicOr(a.vis + (v >> 5), bit);
                won = !(old & bit);
            }
        }
        const unsigned int m = __ballot_sync(GRX_FULL_MASK, won);
        if (!m) continue;
        unsigned long long dg = 0;
        if (won) {
            a.depth[v] = (int32_t)(L + 1);
            if (a.parent) a.parent[v] = u;
            atomicOr(Fout + (v >> 5), 1u << (v & 31));
            dg = (unsigned long long)rdeg(a, v);
        }
        dg = warp_sum(dg);
        unsigned long long pos = 0;
        if (lane == 0) {
            pos = atomicAdd(cnt_q(a, L + 1), (unsigned long long)__popc(m));
            atomicAdd(cnt_e(a, L + 1), dg);
        }
        pos = __shfl_sync(GRX_FULL_MASK, pos, 0);
        if (won) Qout[pos + __popc(m & lanemask_lt())] = v;
    }
}

__global__ void __launch_bounds__(B64_BLOCK) k_bfs64(B64Args a) {
    __shared__ B64State s_st;
    __shared__ uint16_t s_list[B64_WARPS][CHUNK_VERTS];
    __shared__ uint32_t s_fb[B64_WARPS][32];
    const unsigned int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t gwarp = (int64_t)blockIdx.x * B64_WARPS + wi;
    const int64_t nwarps = (int64_t)gridDim.x * B64_WARPS;
    FlagBarrier bar{a.bar_flags, &a.ctl->bar_release, a.ctl, a.timeout_ns, 0u};

    // init: depth -1 (0 at src), parent -1 (src at src), visited = F0 = {src}
    for (int64_t v = tid; v < a.nv; v += stride) {
        a.depth[v] = v == a.src ? 0 : -1;
        if (a.parent) a.parent[v] = v == a.src ? a.src : -1;
    }
    const int64_t sw = a.src >> 5;
    const uint32_t sb = 1u << (a.src & 31);
    for (int64_t w = tid; w < a.words; w += stride) {
        a.vis[w] = w == sw ? sb : 0u;
        a.F[0][w] = w == sw ? sb : 0u;
        a.F[1][w] = 0u;
        a.F[2][w] = 0u;
    }
    if (tid == 0) {
        a.Q[0][0] = a.src;
        for (int i = 0; i < 4; ++i) {
            a.ctl->qpack[i] = 0ull;
            a.ctl->pairs[i] = 0ull;
            a.ctl->hstate[0][i] = 0;
            a.ctl->hstate[1][i] = 0;
            a.ctl->wq[i] = 0u;
        }
    }
    if (threadIdx.x == 0) {
        B64State st;
        st.L = 0;
        st.vcount = 1;
        st.seq = 0;
        const int64_t d = rdeg(a, a.src);
        st.q = d > 0 ? 1 : 0;
        st.T = (uint64_t)d;
        st.dir = a.mode == GRX_DIR_PULL ? D_PULL : D_PUSH;
        st.switched = a.mode == GRX_DIR_PULL;
        st.back = 0;
        st.done = st.q == 0;
        st.qin = 1;
        s_st = st;
    }
    if (!flag_barrier(bar)) return;

    for (;;) {
        B64State st = s_st;
        if (st.done) break;
        const int64_t L = st.L;
        uint32_t *Fin = a.F[L % 3];
        uint32_t *Fout = a.F[(L + 1) % 3];
        uint32_t *Fold = a.F[(L + 2) % 3];
        // counters of level L+2
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.ctl->qpack[(L + 2) & 3] = 0ull;
            a.ctl->pairs[(L + 2) & 3] = 0ull;
            a.ctl->hstate[0][(L + 2) & 3] = 0;
            a.ctl->hstate[1][(L + 2) & 3] = 0;
        }
        // every phase begins by zeroing the chunk counter of the phase after
        // next (phase seq + 2 runs after two barriers)
        auto phase_begin = [&](uint32_t seq) {
            if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->wq[(seq + 2) & 3] = 0u;
        };
        // F_{L-1} is not needed any more; level L+1 fills this slot
        if (L >= 1)
            for (int64_t w = tid; w < a.words; w += stride) Fold[w] = 0u;
        const int64_t nsc = (a.words + 31) / 32;
        if (st.dir == D_PULL) {
            phase_begin(st.seq);
            unsigned int *wq = &a.ctl->wq[st.seq & 3];
            unsigned long long found = 0, fedges = 0;
            for (int64_t sc = gwarp; sc < nsc; sc = nwarps + (int64_t)__shfl_sync(GRX_FULL_MASK,
                                                                        lane == 0 ? atomicAdd(wq, 1u) : 0u, 0)) {
                const int64_t wd = sc * 32 + lane;
                const bool own = wd < a.words;
                const uint32_t vw = own ? __ldcg(a.vis + wd) : 0xffffffffu;
                const uint32_t cand = own ? (__ldg(a.nz + wd) & ~vw) : 0u;
                s_fb[wi][lane] = 0u;
                const int n = warp_compact_bits(cand, s_list[wi]);
                for (int i = (int)lane; i < n; i += 32) {
                    const int64_t v = sc * CHUNK_VERTS + s_list[wi][i];
                    const int64_t rb = __ldg(a.ro + v), re = __ldg(a.ro + v + 1);
                    for (int64_t e = rb; e < re; ++e) {
                        const int64_t u = __ldg(a.col + e);
                        if ((__ldca(Fin + (u >> 5)) >> (u & 31)) & 1u) {
                            a.depth[v] = (int32_t)(L + 1);
                            if (a.parent) a.parent[v] = u;
                            atomicOr(&s_fb[wi][(v >> 5) & 31], 1u << (v & 31));
                            found += 1;
                            fedges += (unsigned long long)(re - rb);
                            break;
                        }
                    }
                }
                __syncwarp();
                if (own) {
                    const uint32_t fb = s_fb[wi][lane];
                    if (fb) a.vis[wd] = vw | fb;
                    Fout[wd] = fb;
                }
                __syncwarp();
            }
            found = warp_sum(found);
            fedges = warp_sum(fedges);
            if (lane == 0 && found) {
                atomicAdd(cnt_q(a, L + 1), found);
                atomicAdd(cnt_e(a, L + 1), fedges);
            }
            if (!flag_barrier(bar)) return;
            st.seq += 1;
        } else {
            int64_t *Qin = a.Q[L & 1];
            int64_t *Qout = a.Q[(L + 1) & 1];
            uint64_t q = st.q;
            if (!st.qin) {
                // the frontier bitmap F_L becomes the queue Q_L
                phase_begin(st.seq);
                unsigned int *wq = &a.ctl->wq[st.seq & 3];
                for (int64_t sc = gwarp; sc < nsc; sc = nwarps + (int64_t)__shfl_sync(GRX_FULL_MASK,
                                                                            lane == 0 ? atomicAdd(wq, 1u) : 0u, 0)) {
                    const int64_t wd = sc * 32 + lane;
                    const uint32_t bits = wd < a.words ? __ldcg(Fin + wd) : 0u;
                    const int n = warp_compact_bits(bits, s_list[wi]);
                    unsigned long long base = 0;
                    if (lane == 0 && n) base = atomicAdd(cnt_cq(a, L), (unsigned long long)n);
                    base = __shfl_sync(GRX_FULL_MASK, base, 0);
                    for (int i = (int)lane; i < n; i += 32) Qin[base + i] = sc * CHUNK_VERTS + s_list[wi][i];
                    __syncwarp();
                }
                if (!flag_barrier(bar)) return;
                st.seq += 1;
                q = ld_relaxed_u64(cnt_cq(a, L));
            }
            // phase A: a warp per frontier vertex, first LONG edges of its row
            phase_begin(st.seq);
            for (int64_t i = gwarp; i < (int64_t)q; i += nwarps) {
                const int64_t u = __ldcg(Qin + i);
                const int64_t rb = __ldg(a.ro + u), re = __ldg(a.ro + u + 1);
                const int64_t e1 = re - rb > LONG ? rb + LONG : re;
                if (lane == 0 && re > e1) {
                    const unsigned long long chunks = (unsigned long long)((re - e1 + LONG - 1) / LONG);
                    const unsigned long long old = atomicAdd(cnt_lr(a, L), (1ull << LR_SHIFT) | chunks);
                    const unsigned long long pos = old >> LR_SHIFT;
                    if (pos >= (1ull << (64 - LR_SHIFT)) - 1 || pos >= (unsigned long long)a.nv) {
                        grx_set_status(a.ctl, GRX_ERANGE);
                    } else {
                        a.lu[pos] = u;
                        a.ls[pos] = e1;
                        a.lb[pos] = old & ((1ull << LR_SHIFT) - 1);
                    }
                }
                push_edges(a, L, u, rb, e1, Fout, Qout);
            }
            if (!flag_barrier(bar)) return;
            st.seq += 1;
            // phase B: the long rows' remaining edges, LONG per chunk, chunks from a counter
            phase_begin(st.seq);
            const unsigned long long lr = ld_relaxed_u64(cnt_lr(a, L));
            const int64_t nl = (int64_t)(lr >> LR_SHIFT);
            const int64_t nch = (int64_t)(lr & ((1ull << LR_SHIFT) - 1));
            if (nl > 0) {
                unsigned int *wq = &a.ctl->wq[st.seq & 3];
                for (int64_t c = gwarp; c < nch; c = nwarps + (int64_t)__shfl_sync(GRX_FULL_MASK,
                                                                          lane == 0 ? atomicAdd(wq, 1u) : 0u, 0)) {
                    // the long row holding chunk c: largest j with lb[j] <= c
                    int64_t lo = 0, hi = nl;
                    while (hi - lo > 1) {
                        const int64_t mid = (lo + hi) >> 1;
                        if ((int64_t)__ldcg(a.lb + mid) <= c) lo = mid; else hi = mid;
                    }
                    const int64_t u = __ldcg(a.lu + lo);
                    const int64_t e0 = __ldcg(a.ls + lo) + (c - (int64_t)__ldcg(a.lb + lo)) * LONG;
                    const int64_t re = __ldg(a.ro + u + 1);
                    push_edges(a, L, u, e0, e0 + LONG < re ? e0 + LONG : re, Fout, Qout);
                }
            }
            if (!flag_barrier(bar)) return;
            st.seq += 1;
        }
        if (threadIdx.x == 0) {
            B64State ns = b64_next(a, st);
            s_st = ns;
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->levels_run = (int)s_st.L;
}

__global__ void k_nz64(const int64_t *ro, int64_t nv, uint32_t *bits, int64_t words) {
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words;
         w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = 0;
        for (int k = 0; k < 32; ++k) {
            const int64_t v = w * 32 + k;
            if (v < nv && ro[v + 1] > ro[v]) b |= 1u << k;
        }
        bits[w] = b;
    }
}

// Offsets monotone from 0 to ne, columns in range, rows sorted without
// self-loops or duplicates, every edge present in both rows.
__global__ void k_validate64(const int64_t *ro, const int64_t *col, int64_t nv, int64_t ne,
                             unsigned long long *bad) {
    unsigned long long local = 0;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (tid == 0 && (ro[0] != 0 || ro[nv] != ne)) ++local;
    for (int64_t v = tid; v < nv; v += stride) {
        const int64_t b = ro[v], e = ro[v + 1];
        if (e < b || b < 0 || e > ne) { ++local; continue; }
        for (int64_t i = b; i < e; ++i) {
            const int64_t u = col[i];
            if (u < 0 || u >= nv) { ++local; continue; }
            if (u == v) ++local;
            if (i > b && col[i - 1] >= u) ++local;
            int64_t lo = ro[u], hi = ro[u + 1];
            if (hi < lo || lo < 0 || hi > ne) { ++local; continue; }
            bool found = false;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                const int64_t c = col[mid];
                if (c == v) { found = true; break; }
                if (c < v) lo = mid + 1; else hi = mid;
            }
            if (!found) ++local;
        }
    }
    if (local) atomicAdd(bad, local);
}

grx_status ensure_ws64(grx_graph *g, cudaStream_t s) {
    if (g->ws64_ready) return GRX_OK;
    const size_t nv = (size_t)g->nv64, wb = (size_t)g->words * 4;
    g->visited = (uint32_t *)grx_alloc(g, wb, s);
    for (int i = 0; i < 3; ++i) g->fbits[i] = (uint32_t *)grx_alloc(g, wb, s);
    for (int i = 0; i < 2; ++i) g->q64[i] = (int64_t *)grx_alloc(g, nv * 8, s);
    for (int i = 0; i < 3; ++i) g->lr64[i] = (int64_t *)grx_alloc(g, nv * 8, s);
    g->ctl = (TravCtl *)grx_alloc(g, sizeof(TravCtl), s);
    g->bar_flags = (unsigned int *)grx_alloc(g, sizeof(unsigned int) * GRX_MAX_GRID, s);
    bool ok = g->visited && g->ctl && g->bar_flags;
    for (int i = 0; i < 3; ++i) ok = ok && g->fbits[i] && g->lr64[i];
    for (int i = 0; i < 2; ++i) ok = ok && g->q64[i];
    if (!ok) return grx_fail(GRX_ENOMEM, "bfs64: workspace allocation failed (nv=%lld)", (long long)g->nv64);
    GRX_CUDA(cudaMemsetAsync(g->ctl, 0, sizeof(TravCtl), s));
    g->ws64_ready = 1;
    return GRX_OK;
}

}  // namespace

extern "C" grx_status graph_load_csr64(grx_ctx *ctx, int64_t nv, int64_t ne, const int64_t *row_offsets,
                                       const int64_t *col_indices, int flags, void *stream, grx_graph **out) {
    if (!ctx || !out) return grx_fail(GRX_EINVAL, "graph_load_csr64: ctx/out is NULL");
    *out = nullptr;
    if (nv < 1 || ne < 0) return grx_fail(GRX_EINVAL, "graph_load_csr64: nv must be >= 1, ne >= 0");
    if (nv >= (1ll << 42)) return grx_fail(GRX_ERANGE, "graph_load_csr64: nv >= 2^42");
    if (!row_offsets || (ne > 0 && !col_indices))
        return grx_fail(GRX_EINVAL, "graph_load_csr64: NULL row_offsets or col_indices");
    cudaStream_t s = (cudaStream_t)stream;
    const bool dev_in = (flags & GRX_DEVICE_PTRS) != 0;
    const cudaMemcpyKind kind = dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (!dev_in && (row_offsets[0] != 0 || row_offsets[nv] != ne))
        return grx_fail(GRX_EINVAL, "graph_load_csr64: row_offsets[0] must be 0 and row_offsets[nv] must equal ne");
    grx_graph *g = (grx_graph *)calloc(1, sizeof(grx_graph));
    if (!g) return grx_fail(GRX_ENOMEM, "graph_load_csr64: host allocation failed");
    g->ctx = ctx;
    g->vid64 = 1;
    g->nv64 = nv;
    g->nv = nv < (1ll << 31) ? (int32_t)nv : -1;
    g->ne = ne;
    g->off64 = 1;
    g->last_stream = stream;
    g->words = ((nv + 31) / 32 + 31) / 32 * 32;
    grx_status st = GRX_OK;
    g->ro = grx_alloc(g, (size_t)(nv + 1) * 8, s);
    g->col64 = (int64_t *)grx_alloc(g, (size_t)(ne > 0 ? ne : 1) * 8, s);
    g->nz_bits = (uint32_t *)grx_alloc(g, (size_t)g->words * 4, s);
    if (!g->ro || !g->col64 || !g->nz_bits) {
        st = grx_fail(GRX_ENOMEM, "graph_load_csr64: device allocation failed");
    } else {
        cudaError_t e = cudaMemcpyAsync(g->ro, row_offsets, (size_t)(nv + 1) * 8, kind, s);
        if (e == cudaSuccess && ne > 0) e = cudaMemcpyAsync(g->col64, col_indices, (size_t)ne * 8, kind, s);
        if (e != cudaSuccess) st = grx_cuda_fail(e, "graph_load_csr64: copy");
    }
    if (st == GRX_OK) {
        const int64_t blocks = (g->words + 255) / 256 < 65536 ? (g->words + 255) / 256 : 65536;
        k_nz64<<<(unsigned)blocks, 256, 0, s>>>((const int64_t *)g->ro, nv, g->nz_bits, g->words);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = grx_cuda_fail(e, "graph_load_csr64: non-isolated bitmap");
    }
    if (st == GRX_OK && (flags & GRX_VALIDATE)) {
        unsigned long long *bad = (unsigned long long *)grx_ctx_alloc(ctx, 8, s);
        if (!bad) {
            st = grx_fail(GRX_ENOMEM, "graph_load_csr64: validation buffer");
        } else {
            unsigned long long h = 0;
            cudaError_t e = cudaMemsetAsync(bad, 0, 8, s);
            const int64_t blocks = (nv + 255) / 256 < 65536 ? (nv + 255) / 256 : 65536;
            if (e == cudaSuccess)
                k_validate64<<<(unsigned)blocks, 256, 0, s>>>((const int64_t *)g->ro, g->col64, nv, ne, bad);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpyAsync(&h, bad, 8, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            grx_ctx_free(ctx, bad, 8, s);
            if (e != cudaSuccess) st = grx_cuda_fail(e, "graph_load_csr64: validation");
            else if (h) st = grx_fail(GRX_EINVAL, "graph_load_csr64: %llu CSR violations (offsets, range, "
                                                  "order, self-loops, symmetry)", h);
        }
    }
    if (st != GRX_OK) {
        for (int i = 0; i < g->nallocs; ++i) grx_ctx_free(ctx, g->allocs[i].p, g->allocs[i].n, s);
        free(g);
        return st;
    }
    *out = g;
    return GRX_OK;
}

extern "C" grx_status bfs64(grx_graph *g, int64_t src, int32_t *depth_out, int64_t *parent_out,
                            const grx_opts *opts, void *stream) {
    if (!g) return grx_fail(GRX_EINVAL, "bfs64: NULL graph");
    if (!g->vid64) return grx_fail(GRX_EINVAL, "bfs64: the graph has 32-bit vertex ids (use bfs)");
    if (src < 0 || src >= g->nv64) return grx_fail(GRX_EINVAL, "bfs64: source %lld out of range", (long long)src);
    if (!depth_out) return grx_fail(GRX_EINVAL, "bfs64: depth_out is NULL");
    grx_opts o;
    grx_resolve_opts(opts, &o);
    if (o.direction < GRX_DIR_AUTO || o.direction > GRX_DIR_PULL)
        return grx_fail(GRX_EINVAL, "bfs64: bad direction %d", o.direction);
    if (o.collect_stats || o.loop != GRX_LOOP_PERSISTENT)
        return grx_fail(GRX_EINVAL, "bfs64: only the persistent loop, without per-level counters");
    cudaStream_t s = (cudaStream_t)stream;
    g->last_stream = stream;
    grx_status st = ensure_ws64(g, s);
    if (st != GRX_OK) return st;
    B64Args a;
    a.nv = g->nv64;
    a.ne = g->ne;
    a.words = g->words;
    a.ro = (const int64_t *)g->ro;
    a.col = g->col64;
    a.nz = g->nz_bits;
    a.vis = g->visited;
    for (int i = 0; i < 3; ++i) a.F[i] = g->fbits[i];
    for (int i = 0; i < 2; ++i) a.Q[i] = g->q64[i];
    a.lu = g->lr64[0];
    a.ls = g->lr64[1];
    a.lb = (unsigned long long *)g->lr64[2];
    a.depth = depth_out;
    a.parent = parent_out;
    a.ctl = g->ctl;
    a.bar_flags = g->bar_flags;
    a.mode = o.direction;
    a.exact_fv = o.exact_fv;
    a.alpha = o.alpha;
    a.beta = o.beta;
    a.timeout_ns = grx_timeout_ns(&o);
    a.src = src;
    static int per_sm = -1;
    if (per_sm < 0) {
        GRX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bfs64, B64_BLOCK, 0));
        if (per_sm < 1) return grx_fail(GRX_ECUDA, "bfs64: kernel does not fit on an SM");
    }
    int max_grid = per_sm * g->ctx->num_sms;
    if (max_grid > GRX_MAX_GRID) max_grid = GRX_MAX_GRID;
    const int blocks = o.grid_blocks > 0 && o.grid_blocks < max_grid ? o.grid_blocks : max_grid;
    GRX_CUDA(cudaMemsetAsync(g->bar_flags, 0, sizeof(unsigned int) * (size_t)blocks, s));
    GRX_CUDA(cudaMemsetAsync(&g->ctl->bar_release, 0, sizeof(unsigned int), s));
    void *args[] = {(void *)&a};
    if (o.ev_begin) GRX_CUDA(cudaEventRecord((cudaEvent_t)o.ev_begin, s));
    GRX_CUDA(cudaLaunchCooperativeKernel((const void *)k_bfs64, dim3(blocks), dim3(B64_BLOCK), args, 0, s));
    if (o.ev_end) GRX_CUDA(cudaEventRecord((cudaEvent_t)o.ev_end, s));
    return GRX_OK;
}
