// Batched SSSP: up to 64 sources share one edge stream (Table 1 SSSP, the
// min combiner of Sec. 3, per lane).
//
//  * Distances live vertex-major inside the library, D[v][lane] (64 uint32
//    per vertex), so a warp relaxes one edge (u, v, w) for 32 lanes at once
//    with coalesced 128-byte reads of D[u][*] and D[v][*]; lanes that improve
//    use atomicMin on their own word.  The output is transposed to the
//    caller's lane-major layout at the end.
//  * A vertex's "changed" mask lists the lanes whose distance improved in the
//    last round; only those lanes relax its edges.  A warp stages a tile's 64
//    edges in shared memory (coalesced) and relaxes 8 of them at a time, all
//    their distance loads in flight.  Improved lanes are OR-ed into next[v]
//    (one atomic per warp and edge); the first toucher lists v -- or, in
//    rounds with at least push_bitmap * V edges, the min and the OR are
//    reductions and v is marked in a touched bitmap -- and a finalize phase
//    moves next into the frontier's masks.
//  * Frontier slots carry the degree prefix and row start (equal warp tiles of
//    edges, as in BFS); the changed masks rotate through three arrays like the
//    multi-source BFS lane masks.  One cooperative persistent kernel, rounds
//    separated by the bounded flag barrier, until no distance improves.
#include "grx_internal.cuh"

namespace {

constexpr int MP_BLOCK = 256;
constexpr int MP_WARPS = MP_BLOCK / 32;
constexpr int MP_WTILE = 64;                 // edges per warp tile
constexpr int MP_UNROLL = 8;                 // edges relaxed together by a warp

template <typename OffT>
struct MpArgs {
    int32_t nv;
    const OffT *ro;
    const int32_t *col;
    const uint32_t *w;
    int n;
    unsigned long long lanes;
    int32_t src[64];
    uint32_t *D;                             // [nv][64]
    unsigned long long *next;
    unsigned long long *cur[3];
    int32_t *Q[3];
    uint32_t *E[3];
    OffT *R[3];
    int32_t *touched;
    uint32_t *tbits;                         // touched bitmap of large rounds
    int64_t words;
    uint32_t bmp_min_T;
    TravCtl *ctl;
    unsigned int *bar_flags;
    DevStats *stats;
    unsigned long long timeout_ns;
};

template <typename OffT>
struct MpWarpSmem {
    uint32_t qe[MP_WTILE + 2];
    int32_t u[MP_WTILE + 1];
    OffT rs[MP_WTILE + 1];
    unsigned long long cm[MP_WTILE + 1];
    int32_t ev[MP_WTILE];                    // the tile's edges: target, weight, row
    uint32_t ew[MP_WTILE];
    int32_t er[MP_WTILE];
};

template <typename T>
__device__ __forceinline__ T pk3(T a, T b, T c, int i) { return i == 0 ? a : (i == 1 ? b : c); }

template <typename OffT>
__device__ void mp_init_fill(const MpArgs<OffT> &a) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // only the batch's lanes (rounded up to a 32-byte sector) are ever read
    const int nl = (a.n + 7) & ~7;
    const int64_t total = (int64_t)a.nv * nl;
    for (int64_t i = tid; i < total; i += stride) a.D[(i / nl) * 64 + (i % nl)] = 0xffffffffu;
    for (int64_t v = tid; v < a.nv; v += stride) {
        a.next[v] = 0ull;
        a.cur[0][v] = 0ull;
        a.cur[1][v] = 0ull;
        a.cur[2][v] = 0ull;
    }
    for (int64_t w = tid; w < a.words; w += stride) a.tbits[w] = 0u;
}

template <typename OffT>
__device__ void mp_seed(const MpArgs<OffT> &a) {
    uint32_t cnt = 0, edges = 0;
    for (int b = 0; b < a.n; ++b) {
        const int32_t v = a.src[b];
        a.D[(int64_t)v * 64 + b] = 0u;
        if (a.cur[0][v] == 0ull) {
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
        a.cur[0][v] |= 1ull << b;
    }
    a.ctl->qpack[0] = ((unsigned long long)cnt << 32) | edges;
    for (int i = 1; i < 4; ++i) a.ctl->qpack[i] = 0ull;
    for (int i = 0; i < 4; ++i) a.ctl->ucount[i] = 0u;
}

}  // namespace

namespace {

// Relaxes a staged tile of `len` edges for every lane of the batch: one edge
// at a time across the warp, thread = lane b (and b + 32 with two halves).
// Improved lanes go to next[v] (and the touched bitmap in reduction rounds,
// or the tile's touched list tbuf / nt otherwise).
template <typename OffT>
__device__ __forceinline__ void relax_lanes(const MpArgs<OffT> &a, MpWarpSmem<OffT> &w, int len, bool bmp,
                                            int32_t *tbuf, int &nt, int halves) {
    const unsigned int lane = threadIdx.x & 31;
        for (int eb = 0; eb < len; eb += MP_UNROLL) {
        int32_t vv[MP_UNROLL], uu[MP_UNROLL];
        uint32_t ww[MP_UNROLL];
        unsigned long long mm[MP_UNROLL];
#pragma unroll
        for (int k = 0; k < MP_UNROLL; ++k) {
            const bool ok = eb + k < len;
            const int j = ok ? w.er[eb + k] : 0;
            vv[k] = ok ? w.ev[eb + k] : 0;
            ww[k] = ok ? w.ew[eb + k] : 0u;
            uu[k] = ok ? w.u[j] : 0;
            mm[k] = ok ? w.cm[j] : 0ull;
        }
        unsigned long long imp[MP_UNROLL];
#pragma unroll
        for (int k = 0; k < MP_UNROLL; ++k) imp[k] = 0ull;
        for (int h = 0; h < halves; ++h) {
            const int b = (int)lane + 32 * h;
            uint32_t du[MP_UNROLL], dv[MP_UNROLL];
#pragma unroll
            for (int k = 0; k < MP_UNROLL; ++k) {
                const bool act = (mm[k] >> b) & 1ull;
                du[k] = act ? __ldcg(a.D + (int64_t)uu[k] * 64 + b) : 0xffffffffu;
                dv[k] = act ? __ldcg(a.D + (int64_t)vv[k] * 64 + b) : 0u;
            }
#pragma unroll
            for (int k = 0; k < MP_UNROLL; ++k) {
                bool improved = false;
                if (du[k] != 0xffffffffu) {
                    const uint64_t nd = (uint64_t)du[k] + ww[k];
                    if (nd >= 0xffffffffull) {
                        grx_set_status(a.ctl, GRX_ERANGE);
                    } else if ((uint32_t)nd < dv[k]) {
                        if (bmp) {
                            // a reduction: the lane improves in this round,
                            // by this proposal or a smaller one
                            atomicMin(a.D + (int64_t)vv[k] * 64 + b, (uint32_t)nd);
                            improved = true;
                        } else {
                            const uint32_t old = atomicMin(a.D + (int64_t)vv[k] * 64 + b, (uint32_t)nd);
                            improved = (uint32_t)nd < old;
                        }
                    }
                }
                imp[k] |= (unsigned long long)__ballot_sync(GRX_FULL_MASK, improved) << (32 * h);
            }
        }
        if (bmp) {
#pragma unroll
            for (int k = 0; k < MP_UNROLL; ++k) {
                if (lane == (unsigned)k && imp[k]) {
                    atomicOr(a.next + vv[k], imp[k]);                // results unused: reductions
                    atomicOr(a.tbits + (vv[k] >> 5), 1u << (vv[k] & 31));
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < MP_UNROLL; ++k) {
                bool first = false;
                if (lane == (unsigned)k && imp[k]) first = atomicOr(a.next + vv[k], imp[k]) == 0ull;
                const unsigned int fm = __ballot_sync(GRX_FULL_MASK, first);
                if (first) tbuf[nt + __popc(fm & lanemask_lt())] = vv[k];
                nt += __popc(fm);
            }
        }
    }
}

// The same for batches of at most G lanes (G = 8 or 16): the warp splits into
// 32 / G groups and each group relaxes its own edge, thread = lane b of its
// group's edge, so one warp instruction serves 32 / G edges.
template <typename OffT, int G>
__device__ __forceinline__ void relax_groups(const MpArgs<OffT> &a, MpWarpSmem<OffT> &w, int len, bool bmp,
                                             int32_t *tbuf, int &nt) {
    static_assert(G == 8 || G == 16, "lane groups of 8 or 16");
    constexpr int EPW = 32 / G;                   // edges per warp instruction
    const unsigned int lane = threadIdx.x & 31;
    const int gi = (int)lane / G;                 // the thread's edge within a step
    const int b = (int)lane % G;                  // its SSSP lane
    const unsigned int gmask = (1u << G) - 1u;
    for (int eb = 0; eb < len; eb += MP_UNROLL * EPW) {
        int32_t vv[MP_UNROLL], uu[MP_UNROLL];
        uint32_t ww[MP_UNROLL];
        bool act[MP_UNROLL];
#pragma unroll
        for (int k = 0; k < MP_UNROLL; ++k) {
            const int e = eb + k * EPW + gi;
            const bool ok = e < len;
            const int j = ok ? w.er[e] : 0;
            vv[k] = ok ? w.ev[e] : 0;
            ww[k] = ok ? w.ew[e] : 0u;
            uu[k] = ok ? w.u[j] : 0;
            act[k] = ok && ((w.cm[j] >> b) & 1ull);
        }
        uint32_t du[MP_UNROLL], dv[MP_UNROLL];
#pragma unroll
        for (int k = 0; k < MP_UNROLL; ++k) {
            du[k] = act[k] ? __ldcg(a.D + (int64_t)uu[k] * 64 + b) : 0xffffffffu;
            dv[k] = act[k] ? __ldcg(a.D + (int64_t)vv[k] * 64 + b) : 0u;
        }
#pragma unroll
        for (int k = 0; k < MP_UNROLL; ++k) {
            bool improved = false;
            if (du[k] != 0xffffffffu) {
                const uint64_t nd = (uint64_t)du[k] + ww[k];
                if (nd >= 0xffffffffull) {
                    grx_set_status(a.ctl, GRX_ERANGE);
                } else if ((uint32_t)nd < dv[k]) {
                    if (bmp) {
                        atomicMin(a.D + (int64_t)vv[k] * 64 + b, (uint32_t)nd);
                        improved = true;
                    } else {
                        const uint32_t old = atomicMin(a.D + (int64_t)vv[k] * 64 + b, (uint32_t)nd);
                        improved = (uint32_t)nd < old;
                    }
                }
            }
            // the group's improved lanes; its first thread publishes them
            const unsigned int imp = (__ballot_sync(GRX_FULL_MASK, improved) >> (gi * G)) & gmask;
            bool first = false;
            if (b == 0 && imp) {
                if (bmp) {
                    atomicOr(a.next + vv[k], (unsigned long long)imp);        // results unused: reductions
                    atomicOr(a.tbits + (vv[k] >> 5), 1u << (vv[k] & 31));
                } else {
                    first = atomicOr(a.next + vv[k], (unsigned long long)imp) == 0ull;
                }
            }
            if (!bmp) {
                const unsigned int fm = __ballot_sync(GRX_FULL_MASK, first);
                if (first) tbuf[nt + __popc(fm & lanemask_lt())] = vv[k];
                nt += __popc(fm);
            }
        }
    }
}

template <typename OffT>
__device__ void mp_expand(const MpArgs<OffT> &a, int L, uint32_t q, uint64_t T, MpWarpSmem<OffT> &w,
                          int32_t *tbuf, bool bmp) {
    const unsigned int lane = threadIdx.x & 31;
    const int32_t *Qv = pk3(a.Q[0], a.Q[1], a.Q[2], L % 3);
    const uint32_t *Qe = pk3(a.E[0], a.E[1], a.E[2], L % 3);
    const OffT *Qr = pk3(a.R[0], a.R[1], a.R[2], L % 3);
    const unsigned long long *cin = pk3(a.cur[0], a.cur[1], a.cur[2], L % 3);
    unsigned int *tctr = &a.ctl->ucount[(L + 1) & 3];
    const uint64_t ntiles = (T + MP_WTILE - 1) / MP_WTILE;
    const uint64_t nwarps = (uint64_t)gridDim.x * MP_WARPS;
    const uint64_t gw = (uint64_t)blockIdx.x * MP_WARPS + (threadIdx.x >> 5);
    const uint64_t per = (ntiles + nwarps - 1) / nwarps;
    const uint64_t tb0 = gw * per;
    const uint64_t tb1 = min(ntiles, tb0 + per);
    if (tb0 >= tb1) return;
    const int halves = a.n > 32 ? 2 : 1;
    int64_t i0 = warp_upper_index_cg(Qe, (int64_t)q, (uint32_t)(tb0 * MP_WTILE));
    for (uint64_t tile = tb0; tile < tb1; ++tile) {
        const uint64_t e0 = tile * MP_WTILE;
        const uint32_t e1 = (uint32_t)min(T, e0 + MP_WTILE);
        int n = 0;
        for (;;) {
            const int64_t idx = i0 + n + lane;
            uint32_t qe = 0xffffffffu;
            if (idx < (int64_t)q) qe = __ldcg(Qe + idx);
            const bool in = idx < (int64_t)q && qe < e1;
            if (n + (int)lane <= MP_WTILE + 1) w.qe[n + lane] = qe;
            if (in && n + (int)lane <= MP_WTILE) {
                const int32_t u = __ldcg(Qv + idx);
                w.u[n + lane] = u;
                w.rs[n + lane] = __ldcg(Qr + idx);
                w.cm[n + lane] = __ldcg(cin + u) & a.lanes;
            }
            const int cnt = __popc(__ballot_sync(GRX_FULL_MASK, in));
            n += cnt;
            if (cnt < 32) break;
            if (n > MP_WTILE) {
                if (lane == 0) grx_set_status(a.ctl, GRX_EINVAL);
                n = MP_WTILE;
                break;
            }
        }
        __syncwarp();
        const uint32_t next_start = w.qe[n];
        // the tile's edges, two per lane, coalesced: target, weight, row
#pragma unroll
        for (int h = 0; h < MP_WTILE / 32; ++h) {
            const uint32_t e = (uint32_t)e0 + lane + 32 * h;
            if (e < e1) {
                const int j = upper_index_smem(w.qe, n, e);
                const OffT idx = w.rs[j] + (OffT)(e - w.qe[j]);
                w.ev[lane + 32 * h] = __ldg(a.col + idx);
                w.ew[lane + 32 * h] = __ldg(a.w + idx);
                w.er[lane + 32 * h] = j;
            }
        }
        __syncwarp();
        const int len = (int)(e1 - (uint32_t)e0);
        int nt = 0;                                   // touched vertices of this tile (list rounds)
        if (a.n <= 8) relax_groups<OffT, 8>(a, w, len, bmp, tbuf, nt);
        else if (a.n <= 16) relax_groups<OffT, 16>(a, w, len, bmp, tbuf, nt);
        else relax_lanes<OffT>(a, w, len, bmp, tbuf, nt, halves);
        __syncwarp();
        // one append of the tile's touched vertices
        unsigned int base = 0;
        if (lane == 0 && nt) base = atomicAdd(tctr, (unsigned)nt);
        base = __shfl_sync(GRX_FULL_MASK, base, 0);
        for (int t = (int)lane; t < nt; t += 32) a.touched[base + t] = tbuf[t];
        i0 = (next_start == e1) ? i0 + n : i0 + n - 1;
        __syncwarp();
    }
}

// A touched vertex (or -1): its improved lanes become its changed mask in
// the next frontier.  All 32 lanes of the warp call.
template <typename OffT>
__device__ __forceinline__ void mp_touched(const MpArgs<OffT> &a, int32_t vv, unsigned long long *cout,
                                           int32_t *Qv_out, uint32_t *Qe_out, OffT *Qr_out,
                                           unsigned long long *ctr) {
    int32_t v[1] = {vv < 0 ? 0 : vv};
    uint32_t deg[1] = {0};
    OffT rb[1] = {0};
    uint32_t app = 0;
    if (vv >= 0) {
        const unsigned long long nx = __ldcg(a.next + vv);
        a.next[vv] = 0ull;
        cout[vv] = nx & a.lanes;
        rb[0] = __ldg(a.ro + vv);
        deg[0] = (uint32_t)(__ldg(a.ro + vv + 1) - rb[0]);
        if (deg[0]) app = 1;
    }
    warp_append_items<1, OffT>(v, deg, rb, app, Qv_out, Qe_out, Qr_out, ctr);
}

// Round phase 2: touched vertices (list, or the bitmap by warps owning 32-word
// chunks, which clear it) become the next frontier.
template <typename OffT>
__device__ void mp_finalize(const MpArgs<OffT> &a, int L, bool bmp, uint16_t *list) {
    unsigned long long *cout = pk3(a.cur[0], a.cur[1], a.cur[2], (L + 1) % 3);
    int32_t *Qv_out = pk3(a.Q[0], a.Q[1], a.Q[2], (L + 1) % 3);
    uint32_t *Qe_out = pk3(a.E[0], a.E[1], a.E[2], (L + 1) % 3);
    OffT *Qr_out = pk3(a.R[0], a.R[1], a.R[2], (L + 1) % 3);
    unsigned long long *ctr = &a.ctl->qpack[(L + 1) & 3];
    if (bmp) {
        const unsigned int lane = threadIdx.x & 31;
        const int64_t nsc = (a.words + 31) / 32;
        const int64_t nwarps = (int64_t)gridDim.x * MP_WARPS;
        for (int64_t sc = (int64_t)blockIdx.x * MP_WARPS + (threadIdx.x >> 5); sc < nsc; sc += nwarps) {
            const int64_t wd = sc * 32 + lane;
            const uint32_t bits = wd < a.words ? __ldcg(a.tbits + wd) : 0u;
            if (bits) a.tbits[wd] = 0u;
            const int n = warp_compact_bits(bits, list);
            for (int base = 0; base < n; base += 32) {
                const int i = base + (int)lane;
                mp_touched<OffT>(a, i < n ? (int32_t)(sc * 1024 + list[i]) : -1, cout, Qv_out, Qe_out, Qr_out,
                                 ctr);
            }
            __syncwarp();
        }
        return;
    }
    const int64_t count = ld_relaxed_u32(&a.ctl->ucount[(L + 1) & 3]);
    const int64_t span = (count + 31) & ~(int64_t)31;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < span;
         i += (int64_t)gridDim.x * blockDim.x)
        mp_touched<OffT>(a, i < count ? __ldcg(a.touched + i) : -1, cout, Qv_out, Qe_out, Qr_out, ctr);
}

}  // namespace

namespace {

template <typename OffT>
__global__ void __launch_bounds__(MP_BLOCK, 3) k_mssp_persistent(MpArgs<OffT> a) {
    __shared__ MpWarpSmem<OffT> wsm[MP_WARPS];
    __shared__ int32_t tbufs[MP_WARPS][MP_WTILE];
    __shared__ uint16_t lists[MP_WARPS][32 * 32];
    __shared__ uint32_t s_q, s_T;
    __shared__ int s_done;
    const int wi = threadIdx.x >> 5;
    FlagBarrier bar{a.bar_flags, &a.ctl->bar_release, a.ctl, a.timeout_ns, 0u};
    mp_init_fill(a);
    if (!flag_barrier(bar)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) mp_seed(a);
    if (!flag_barrier(bar)) return;
    uint32_t qprev = 0;
    for (int L = 0;; ++L) {
        if (threadIdx.x == 0) {
            const unsigned long long pk = ld_relaxed_u64(&a.ctl->qpack[L & 3]);
            s_q = (uint32_t)(pk >> 32);
            s_T = (uint32_t)pk;
            s_done = s_q == 0;
        }
        __syncthreads();
        const uint32_t q = s_q, T = s_T;
        if (s_done) {
            if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->levels_run = L;
            break;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.ctl->qpack[(L + 2) & 3] = 0ull;
            a.ctl->ucount[(L + 2) & 3] = 0u;
        }
        {   // Q_{L-1}'s masks leave cur[(L+2)%3]
            const int32_t *Qp = pk3(a.Q[0], a.Q[1], a.Q[2], (L + 2) % 3);
            unsigned long long *cp = pk3(a.cur[0], a.cur[1], a.cur[2], (L + 2) % 3);
            for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)qprev;
                 i += (int64_t)gridDim.x * blockDim.x)
                cp[__ldcg(Qp + i)] = 0ull;
        }
        const bool bmp = T >= a.bmp_min_T;
        mp_expand(a, L, q, T, wsm[wi], tbufs[wi], bmp);
        if (!flag_barrier(bar)) return;
        mp_finalize(a, L, bmp, lists[wi]);
        if (!flag_barrier(bar)) return;
        qprev = q;
    }
}

// D[v][b] (vertex-major, 64 lanes) -> out[b][v] for b < n, through a shared tile.
__global__ void k_mssp_transpose(const uint32_t *__restrict__ D, int32_t nv, int n,
                                 uint32_t *__restrict__ out) {
    __shared__ uint32_t tile[32][65];
    const int64_t v0 = (int64_t)blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t v = v0 + r;
        for (int b = threadIdx.x; b < 64; b += 32)
            tile[r][b] = v < nv ? D[v * 64 + b] : 0u;
    }
    __syncthreads();
    for (int b = threadIdx.y; b < n; b += blockDim.y) {
        const int64_t v = v0 + threadIdx.x;
        if (v < nv) out[(int64_t)b * nv + v] = tile[threadIdx.x][b];
    }
}

template <typename OffT>
grx_status mp_launch_typed(grx_graph *g, const int32_t *srcs, int n, uint32_t *dist,
                           const grx_opts *o, cudaStream_t s) {
    MpArgs<OffT> a;
    a.nv = g->nv;
    a.ro = (const OffT *)g->ro;
    a.col = g->col;
    a.w = g->w;
    a.n = n;
    a.lanes = n == 64 ? ~0ull : ((1ull << n) - 1ull);
    for (int i = 0; i < 64; ++i) a.src[i] = i < n ? srcs[i] : 0;
    a.D = g->ms_dist;
    a.next = g->ms_next;
    for (int i = 0; i < 3; ++i) {
        a.cur[i] = g->ms_cur[i];
        a.Q[i] = g->qv[i];
        a.E[i] = g->qe[i];
        a.R[i] = (OffT *)g->qr[i];
    }
    a.touched = g->ulist[0];
    a.tbits = g->ms_tbits;
    a.words = g->words;
    {   // reduction rounds when a round's edges reach push_bitmap * nv (0 = 1/8, < 0 = never)
        const double pb = o->push_bitmap == 0.f ? 0.125 : (double)o->push_bitmap;
        const double t = pb * (double)g->nv;
        a.bmp_min_T = pb < 0 ? 0xffffffffu : (t < 1.0 ? 1u : (t > 4294967295.0 ? 0xffffffffu : (uint32_t)t));
    }
    a.ctl = g->ctl;
    a.bar_flags = g->bar_flags;
    a.stats = g->stats;
    a.timeout_ns = grx_timeout_ns(o);
    static int per_sm = -1;
    if (per_sm < 0) {
        GRX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mssp_persistent<OffT>, MP_BLOCK, 0));
        if (per_sm < 1) return grx_fail(GRX_ECUDA, "sssp_multi: persistent kernel does not fit on an SM");
    }
    int max_grid = per_sm * g->ctx->num_sms;
    if (max_grid > GRX_MAX_GRID) max_grid = GRX_MAX_GRID;
    int blocks = o->grid_blocks > 0 && o->grid_blocks < max_grid ? o->grid_blocks : max_grid;
    GRX_CUDA(cudaMemsetAsync(g->bar_flags, 0, sizeof(unsigned int) * (size_t)blocks, s));
    GRX_CUDA(cudaMemsetAsync(&g->ctl->bar_release, 0, sizeof(unsigned int), s));
    void *args[] = {(void *)&a};
    if (o->ev_begin) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_begin, s));
    GRX_CUDA(cudaLaunchCooperativeKernel((const void *)k_mssp_persistent<OffT>, dim3(blocks),
                                         dim3(MP_BLOCK), args, 0, s));
    const unsigned tblocks = (unsigned)(((int64_t)g->nv + 31) / 32);
    k_mssp_transpose<<<tblocks, dim3(32, 8), 0, s>>>(g->ms_dist, g->nv, n, dist);
    if (o->ev_end) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_end, s));
    GRX_CUDA(cudaGetLastError());
    return GRX_OK;
}

}  // namespace

size_t grx_mssp_new_bytes(const grx_graph *g) {
    size_t b = 0;
    if (!g->ms_dist) b += (size_t)g->nv * 64 * sizeof(uint32_t);
    if (!g->ms_tbits) b += (size_t)g->words * 4 + 16;
    return b;
}

grx_status grx_mssp_launch(grx_graph *g, const int32_t *srcs, int n, uint32_t *dist,
                           const grx_opts *o, cudaStream_t s) {
    if (!g->ms_dist) {
        g->ms_dist = (uint32_t *)grx_alloc(g, (size_t)g->nv * 64 * sizeof(uint32_t), s);
        if (!g->ms_dist) return grx_fail(GRX_ENOMEM, "sssp_multi: distance workspace allocation failed");
    }
    if (!g->ms_tbits) {
        g->ms_tbits = (uint32_t *)grx_alloc(g, (size_t)g->words * 4 + 16, s);
        if (!g->ms_tbits) return grx_fail(GRX_ENOMEM, "sssp_multi: touched bitmap allocation failed");
        GRX_CUDA(cudaMemsetAsync(g->ms_tbits, 0, (size_t)g->words * 4 + 16, s));
    }
    return g->off64 ? mp_launch_typed<int64_t>(g, srcs, n, dist, o, s)
                    : mp_launch_typed<int32_t>(g, srcs, n, dist, o, s);
}
