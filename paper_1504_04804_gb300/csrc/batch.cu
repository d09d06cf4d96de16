// Continuous batching: a resident 64-lane traversal of one graph that queries
// join and leave between level steps.
//
// A batch keeps the multi-source lane masks (BFS: seen / next / cur; SSSP:
// vertex-major distances D[v][64] with "changed" masks) and a frontier.  The
// host runs it level by level (grx_batch_step); between steps a new query is
// admitted into a free lane: its bit is cleared everywhere, its output is
// reset, its source joins the current frontier and the lane records its
// start level, so a vertex found at level L+1 gets depth L+1-start.  A lane
// retires when no frontier vertex carries its bit; grx_batch_poll reports it
// and the lane is free again.  Each lane's result is the single-source result
// (Algorithm 1 / Table 1 SSSP) whatever the other lanes do, because lanes
// only share the reading of the graph.
//
// Every kernel here is an ordinary launch with a grid-stride or tile loop that
// reads the level's state from device memory; nothing waits on another block.
#include <cstdlib>
#include <cstring>

#include "grx_internal.cuh"

struct BatchCtl {
    unsigned long long qpack[4];      // frontier ring (count << 32 | edges), slot = level & 3
    unsigned int ucount[4];           // touched-list ring
    int L;                            // level whose frontier is the next step's input
    int dir;                          // unused (directions are per lane)
    uint32_t qprev;                   // |Q_{L-1}|
    int status;
    unsigned long long active;        // admitted, not yet retired lanes
    unsigned long long alive;         // lanes present in the frontier being built
    unsigned long long retired;       // lanes retired since the last poll
    int32_t start[64];                // level at which each lane joined
    void *out[64];                    // per-lane result (int32 depth or uint32 distance)
    unsigned long long push_lanes;    // lanes expanded top-down this level
    unsigned long long pull_lanes;    // lanes searched bottom-up this level (BFS)
    unsigned long long lane_T[2][64]; // per-lane frontier edge count, by level parity
    int bmp;                          // this level marks touched vertices in a bitmap
};

struct grx_batch {
    grx_graph *g;
    int kind;
    cudaStream_t s;
    unsigned long long *seen, *next, *cur[3];
    uint32_t *D;
    int32_t *Q[3];
    uint32_t *E[3];
    void *R[3];
    int32_t *touched;
    uint32_t *tbits;                  // touched bitmap of large levels
    BatchCtl *ctl;
    unsigned long long busy;          // host view of occupied lanes
    void *out_host[64];
    struct { void *p; size_t n; } allocs[24];
    int nallocs;
    int blocks;
};

namespace {

constexpr int BT_BLOCK = 256;
constexpr int BT_WARPS = BT_BLOCK / 32;
constexpr int BT_ITEMS = 8;
constexpr int BT_WTILE = 32 * BT_ITEMS;
constexpr int BTX_BLOCK = 128;                      // expansion kernel (shared memory per warp)
constexpr int BTX_WARPS = BTX_BLOCK / 32;
static_assert(BT_WTILE == 256, "warp_tile_rows8 covers 256-position tiles");
constexpr double BT_PULL_FRACTION = 1.0 / 32.0;   // a lane pulls when its frontier edges > E/32

template <typename T>
__device__ __forceinline__ T pk3(T a, T b, T c, int i) { return i == 0 ? a : (i == 1 ? b : c); }

template <typename OffT>
struct BatchArgs {
    int32_t nv;
    int64_t ne;
    const OffT *ro;
    const int32_t *col;
    const uint32_t *w;
    int kind;
    unsigned long long *seen, *next, *cur[3];
    uint32_t *D;
    int32_t *Q[3];
    uint32_t *E[3];
    OffT *R[3];
    int32_t *touched;
    uint32_t *tbits;
    int64_t words;
    BatchCtl *ctl;
};

template <typename OffT>
struct BtWarpSmem {
    uint32_t qe[BT_WTILE + 2];
    int32_t u[BT_WTILE + 1];
    OffT rs[BT_WTILE + 1];
    unsigned long long cm[BT_WTILE + 1];
    alignas(16) uint16_t rid[BT_WTILE];
};

// Level begin (one thread): a direction per lane (Sec. 6.1 applied lane by
// lane: a lane whose own frontier holds many edges is searched bottom-up),
// reset the ring slots.
template <typename OffT>
__global__ void k_bt_begin(BatchArgs<OffT> a) {
    BatchCtl *c = a.ctl;
    const int L = c->L;
    unsigned long long pull = 0ull;
    for (int b = 0; b < 64; ++b) {
        if (a.kind == GRX_KIND_BFS && ((c->active >> b) & 1ull) &&
            (double)c->lane_T[L & 1][b] > BT_PULL_FRACTION * (double)a.ne)
            pull |= 1ull << b;
        c->lane_T[(L + 1) & 1][b] = 0ull;
    }
    c->pull_lanes = pull;
    c->push_lanes = c->active & ~pull;
    // large levels: reductions plus a touched bitmap instead of claiming atomics
    c->bmp = (uint32_t)c->qpack[L & 3] >= (uint32_t)(a.nv / 8);
    c->qpack[(L + 1) & 3] = 0ull;
    c->qpack[(L + 2) & 3] = 0ull;
    c->ucount[(L + 1) & 3] = 0u;
    c->alive = 0ull;
}

// The lanes of Q_{L-1} leave cur[(L+2)%3].
template <typename OffT>
__device__ void bt_clear_prev(const BatchArgs<OffT> &a, int L, uint32_t qprev) {
    const int32_t *Qp = pk3(a.Q[0], a.Q[1], a.Q[2], (L + 2) % 3);
    unsigned long long *cp = pk3(a.cur[0], a.cur[1], a.cur[2], (L + 2) % 3);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)qprev;
         i += (int64_t)gridDim.x * blockDim.x)
        cp[Qp[i]] = 0ull;
}

}  // namespace

namespace {

// Load the frontier elements of one warp tile (elements starting before e1)
// into shared memory; returns the element count, w.qe[n] = next start.
template <typename OffT>
__device__ __forceinline__ int bt_load_tile(const BatchArgs<OffT> &a, const int32_t *Qv,
                                            const uint32_t *Qe, const OffT *Qr,
                                            const unsigned long long *cin, unsigned long long lanes,
                                            int64_t q, int64_t i0, uint32_t e1, int wtile,
                                            BtWarpSmem<OffT> &w) {
    const unsigned int lane = threadIdx.x & 31;
    int n = 0;
    for (;;) {
        const int64_t idx = i0 + n + lane;
        uint32_t qe = 0xffffffffu;
        if (idx < q) qe = Qe[idx];
        const bool in = idx < q && qe < e1;
        if (n + (int)lane <= wtile + 1) w.qe[n + lane] = qe;
        if (in && n + (int)lane <= wtile) {
            const int32_t u = Qv[idx];
            w.u[n + lane] = u;
            w.rs[n + lane] = Qr[idx];
            w.cm[n + lane] = cin[u] & lanes;
        }
        const int cnt = __popc(__ballot_sync(GRX_FULL_MASK, in));
        n += cnt;
        if (cnt < 32) break;
        if (n > wtile) {
            n = wtile;
            break;
        }
    }
    __syncwarp();
    return n;
}

template <typename OffT>
__global__ void __launch_bounds__(BTX_BLOCK) k_bt_expand(BatchArgs<OffT> a) {
    __shared__ BtWarpSmem<OffT> wsm[BTX_WARPS];
    BatchCtl *c = a.ctl;
    const int L = c->L;
    bt_clear_prev(a, L, c->qprev);
    if (c->push_lanes == 0ull) return;
    BtWarpSmem<OffT> &w = wsm[threadIdx.x >> 5];
    const unsigned int lane = threadIdx.x & 31;
    const unsigned long long lanes = c->push_lanes;
    const bool bmp = c->bmp != 0;
    const int32_t *Qv = pk3(a.Q[0], a.Q[1], a.Q[2], L % 3);
    const uint32_t *Qe = pk3(a.E[0], a.E[1], a.E[2], L % 3);
    const OffT *Qr = pk3(a.R[0], a.R[1], a.R[2], L % 3);
    const unsigned long long *cin = pk3(a.cur[0], a.cur[1], a.cur[2], L % 3);
    unsigned int *tctr = &c->ucount[(L + 1) & 3];
    const unsigned long long pk = c->qpack[L & 3];
    const int64_t q = (int64_t)(pk >> 32);
    const uint64_t T = (uint32_t)pk;
    const bool sssp = a.kind == GRX_KIND_SSSP;
    const int wtile = BT_WTILE;
    const uint64_t ntiles = (T + wtile - 1) / wtile;
    const uint64_t nwarps = (uint64_t)gridDim.x * BTX_WARPS;
    const uint64_t gw = (uint64_t)blockIdx.x * BTX_WARPS + (threadIdx.x >> 5);
    const uint64_t per = (ntiles + nwarps - 1) / nwarps;
    const uint64_t tb0 = gw * per, tb1 = min(ntiles, tb0 + per);
    if (tb0 >= tb1) return;
    int64_t i0 = 0;
    {   // first element of the warp's first tile: 32-ary search
        int64_t lo = 0, hi = q;
        const uint32_t key = (uint32_t)(tb0 * wtile);
        while (hi - lo > 1) {
            const int64_t step = (hi - lo + 31) / 32;
            const int64_t idx = lo + (int64_t)lane * step;
            const unsigned int m = __ballot_sync(GRX_FULL_MASK, idx < hi && Qe[idx] <= key);
            lo += (int64_t)(31 - __clz(m)) * step;
            hi = min(hi, lo + step);
        }
        i0 = lo;
    }
    for (uint64_t tile = tb0; tile < tb1; ++tile) {
        const uint64_t e0 = tile * wtile;
        const uint32_t e1 = (uint32_t)min(T, e0 + wtile);
        const int n = bt_load_tile(a, Qv, Qe, Qr, cin, lanes, q, i0, e1, wtile, w);
        const uint32_t next_start = w.qe[n];
        int row[BT_ITEMS];
        warp_tile_rows8(w.rid, w.qe, (uint32_t)e0, n, row);
        // each lane a run of BT_ITEMS edges; per edge the lanes to OR into
        // next[v]: BFS m & ~seen[v]; SSSP the lanes of m whose relaxation
        // improves D[v][lane] (cost per edge = popcount of m)
        const uint32_t t0 = (uint32_t)e0 + lane * BT_ITEMS;
        int32_t v[BT_ITEMS], uu[BT_ITEMS];
        uint32_t ww[BT_ITEMS];
        unsigned long long m[BT_ITEMS];
#pragma unroll
        for (int k = 0; k < BT_ITEMS; ++k) {
            const uint32_t e = t0 + k;
            const int j = row[k];
            const bool ok = e < e1;
            const OffT idx = ok ? w.rs[j] + (OffT)(e - w.qe[j]) : (OffT)0;
            v[k] = ok ? __ldg(a.col + idx) : 0;
            m[k] = ok ? w.cm[j] : 0ull;
            ww[k] = (ok && sssp) ? __ldg(a.w + idx) : 0u;
            uu[k] = (ok && sssp) ? w.u[j] : 0;
        }
        __syncwarp();
        unsigned long long mk[BT_ITEMS];
#pragma unroll
        for (int k = 0; k < BT_ITEMS; ++k) {
            mk[k] = 0ull;
            if (m[k] && !sssp) {
                mk[k] = m[k] & ~__ldg(a.seen + v[k]);
            } else if (m[k]) {
                unsigned long long bits = m[k];
                while (bits) {
                    const int bl = __ffsll((long long)bits) - 1;
                    bits &= bits - 1;
                    const uint64_t nd = (uint64_t)__ldcg(a.D + (int64_t)uu[k] * 64 + bl) + ww[k];
                    if (nd >= 0xffffffffull) {
                        atomicCAS(&c->status, 0, GRX_ERANGE);
                    } else if ((uint32_t)nd < __ldcg(a.D + (int64_t)v[k] * 64 + bl)) {
                        if (bmp) {
                            // a reduction: the lane did improve in this level,
                            // by this proposal or a smaller one
                            atomicMin(a.D + (int64_t)v[k] * 64 + bl, (uint32_t)nd);
                            mk[k] |= 1ull << bl;
                        } else if ((uint32_t)nd < atomicMin(a.D + (int64_t)v[k] * 64 + bl, (uint32_t)nd)) {
                            mk[k] |= 1ull << bl;
                        }
                    }
                }
            }
        }
        if (bmp) {
#pragma unroll
            for (int k = 0; k < BT_ITEMS; ++k) {
                if (mk[k]) {
                    atomicOr(a.next + v[k], mk[k]);                   // results unused: reductions
                    atomicOr(a.tbits + (v[k] >> 5), 1u << (v[k] & 31));
                }
            }
        } else {
            uint32_t tm = 0;
#pragma unroll
            for (int k = 0; k < BT_ITEMS; ++k)
                if (mk[k] && atomicOr(a.next + v[k], mk[k]) == 0ull) tm |= 1u << k;
            warp_append_list_items<BT_ITEMS>(v, tm, a.touched, tctr);
        }
        i0 = (next_start == e1) ? i0 + n : i0 + n - 1;
        __syncwarp();
    }
}

}  // namespace

namespace {

__device__ __forceinline__ void bt_label(BatchCtl *c, int32_t v, unsigned long long nw, int L) {
    while (nw) {
        const int b = __ffsll((long long)nw) - 1;
        nw &= nw - 1;
        ((int32_t *)c->out[b])[v] = L + 1 - c->start[b];
    }
}

// Per-block per-lane frontier edge counts, flushed to lane_T of level L+1.
struct LaneT {
    unsigned long long t[64];
};

__device__ __forceinline__ void lane_t_add(LaneT &s, unsigned long long lanes, uint32_t deg) {
    while (lanes) {
        const int b = __ffsll((long long)lanes) - 1;
        lanes &= lanes - 1;
        atomicAdd(&s.t[b], (unsigned long long)deg);
    }
}

__device__ __forceinline__ void lane_t_flush(LaneT &s, BatchCtl *c, int L) {
    __syncthreads();
    if (threadIdx.x < 64 && s.t[threadIdx.x]) atomicAdd(&c->lane_T[(L + 1) & 1][threadIdx.x], s.t[threadIdx.x]);
}

// One touched vertex (or -1): its next mask becomes its new push lanes (BFS:
// not yet seen; labelled here), it joins the next frontier (once), and its
// lanes stay alive.  All 32 lanes of the warp call.
template <typename OffT>
__device__ __forceinline__ void bt_finish_vertex(const BatchArgs<OffT> &a, BatchCtl *c, int L,
                                                 unsigned long long lanes, bool bfsk, int32_t vv,
                                                 unsigned long long *cout, int32_t *Qv_out,
                                                 uint32_t *Qe_out, OffT *Qr_out, LaneT &sT,
                                                 unsigned long long &alive) {
    int32_t v[1] = {vv < 0 ? 0 : vv};
    uint32_t deg[1] = {0};
    OffT rb[1] = {0};
    uint32_t app = 0;
    if (vv >= 0) {
        const unsigned long long nx = a.next[vv];
        a.next[vv] = 0ull;
        unsigned long long nw = nx & lanes;
        if (bfsk) {
            const unsigned long long sv = a.seen[vv];
            nw &= ~sv;
            if (nw) {
                a.seen[vv] = sv | nw;
                bt_label(c, vv, nw, L);
            }
        }
        if (nw) {
            const unsigned long long before = cout[vv];
            cout[vv] = before | nw;
            rb[0] = a.ro[vv];
            deg[0] = (uint32_t)(a.ro[vv + 1] - rb[0]);
            if (deg[0]) {
                alive |= nw;
                lane_t_add(sT, nw, deg[0]);
                if (before == 0ull) app = 1;
            }
        }
    }
    warp_append_items<1, OffT>(v, deg, rb, app, Qv_out, Qe_out, Qr_out, &c->qpack[(L + 1) & 3]);
}

// Touched vertices -> their new push lanes, the next frontier, the alive mask.
// Runs after the pull kernel: a vertex the pull already put in the frontier
// only gains lanes (no second append).  Large levels read the touched bitmap
// (warps own 32-word chunks and clear them), small ones the touched list.
template <typename OffT>
__global__ void __launch_bounds__(BT_BLOCK) k_bt_finalize(BatchArgs<OffT> a) {
    __shared__ LaneT sT;
    __shared__ uint16_t lists[BT_WARPS][32 * 32];
    BatchCtl *c = a.ctl;
    const int L = c->L;
    if (threadIdx.x < 64) sT.t[threadIdx.x] = 0ull;
    __syncthreads();
    const unsigned long long lanes = c->push_lanes;
    const bool bfsk = a.kind == GRX_KIND_BFS;
    unsigned long long *cout = pk3(a.cur[0], a.cur[1], a.cur[2], (L + 1) % 3);
    int32_t *Qv_out = pk3(a.Q[0], a.Q[1], a.Q[2], (L + 1) % 3);
    uint32_t *Qe_out = pk3(a.E[0], a.E[1], a.E[2], (L + 1) % 3);
    OffT *Qr_out = pk3(a.R[0], a.R[1], a.R[2], (L + 1) % 3);
    unsigned long long alive = 0ull;
    if (c->bmp) {
        uint16_t *list = lists[threadIdx.x >> 5];
        const unsigned int lane = threadIdx.x & 31;
        const int64_t nsc = (a.words + 31) / 32;
        const int64_t nwarps = (int64_t)gridDim.x * BT_WARPS;
        for (int64_t sc = (int64_t)blockIdx.x * BT_WARPS + (threadIdx.x >> 5); sc < nsc; sc += nwarps) {
            const int64_t wd = sc * 32 + lane;
            const uint32_t bits = wd < a.words ? a.tbits[wd] : 0u;
            if (bits) a.tbits[wd] = 0u;
            const int n = warp_compact_bits(bits, list);
            for (int base = 0; base < n; base += 32) {
                const int i = base + (int)lane;
                bt_finish_vertex<OffT>(a, c, L, lanes, bfsk, i < n ? (int32_t)(sc * 1024 + list[i]) : -1, cout,
                                       Qv_out, Qe_out, Qr_out, sT, alive);
            }
            __syncwarp();
        }
    } else {
        const int64_t count = c->ucount[(L + 1) & 3];
        const int64_t span = (count + 31) & ~(int64_t)31;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < span;
             i += (int64_t)gridDim.x * blockDim.x)
            bt_finish_vertex<OffT>(a, c, L, lanes, bfsk, i < count ? a.touched[i] : -1, cout, Qv_out, Qe_out,
                                   Qr_out, sT, alive);
    }
    for (int o = 16; o > 0; o >>= 1) alive |= __shfl_xor_sync(GRX_FULL_MASK, alive, o);
    if ((threadIdx.x & 31) == 0 && alive) atomicOr(&c->alive, alive);
    lane_t_flush(sT, c, L);
}

// BFS pull for the pull lanes: each vertex missing one of them ORs its
// neighbours' cur masks, stopping once all its missing pull lanes are found.
template <typename OffT>
__global__ void __launch_bounds__(BT_BLOCK) k_bt_pull(BatchArgs<OffT> a) {
    __shared__ LaneT sT;
    BatchCtl *c = a.ctl;
    const unsigned long long lanes = c->pull_lanes;
    if (lanes == 0ull) return;
    const int L = c->L;
    if (threadIdx.x < 64) sT.t[threadIdx.x] = 0ull;
    __syncthreads();
    const unsigned long long *cin = pk3(a.cur[0], a.cur[1], a.cur[2], L % 3);
    unsigned long long *cout = pk3(a.cur[0], a.cur[1], a.cur[2], (L + 1) % 3);
    int32_t *Qv_out = pk3(a.Q[0], a.Q[1], a.Q[2], (L + 1) % 3);
    uint32_t *Qe_out = pk3(a.E[0], a.E[1], a.E[2], (L + 1) % 3);
    OffT *Qr_out = pk3(a.R[0], a.R[1], a.R[2], (L + 1) % 3);
    const int64_t span = ((int64_t)a.nv + 31) & ~(int64_t)31;
    unsigned long long alive = 0ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < span;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v[1] = {(int32_t)i};
        uint32_t deg[1] = {0};
        OffT rb[1] = {0};
        uint32_t app = 0;
        if (i < a.nv) {
            const unsigned long long sv = a.seen[i];
            const unsigned long long miss = lanes & ~sv;
            if (miss) {
                const OffT b = a.ro[i], e = a.ro[i + 1];
                unsigned long long acc = 0ull;
                for (OffT k = b; k < e && acc != miss; ++k) acc |= cin[a.col[k]] & miss;
                if (acc) {
                    a.seen[i] = sv | acc;
                    cout[i] = acc;
                    bt_label(c, (int32_t)i, acc, L);
                    rb[0] = b;
                    deg[0] = (uint32_t)(e - b);
                    app = 1;
                    alive |= acc;
                    lane_t_add(sT, acc, deg[0]);
                }
            }
        }
        warp_append_items<1, OffT>(v, deg, rb, app, Qv_out, Qe_out, Qr_out, &c->qpack[(L + 1) & 3]);
    }
    for (int o = 16; o > 0; o >>= 1) alive |= __shfl_xor_sync(GRX_FULL_MASK, alive, o);
    if ((threadIdx.x & 31) == 0 && alive) atomicOr(&c->alive, alive);
    lane_t_flush(sT, c, L);
}

// Level end (one thread): lanes absent from the new frontier retire.
__global__ void k_bt_end(BatchCtl *c) {
    const int L = c->L;
    const unsigned long long done = c->active & ~c->alive;
    c->retired |= done;
    c->active &= ~done;
    c->qprev = (uint32_t)(c->qpack[L & 3] >> 32);
    c->L = L + 1;
}

// Admit a query into `lane`: clear the lane everywhere, reset its output, put
// its source into the current frontier.
template <typename OffT>
__global__ void k_bt_admit(BatchArgs<OffT> a, int lane, int32_t src, void *out) {
    BatchCtl *c = a.ctl;
    const int L = c->L;
    const unsigned long long bit = 1ull << lane;
    const bool bfsk = a.kind == GRX_KIND_BFS;
    unsigned long long *cin = pk3(a.cur[0], a.cur[1], a.cur[2], L % 3);
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < a.nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        for (int i = 0; i < 3; ++i) a.cur[i][v] &= ~bit;
        if (bfsk) {
            a.seen[v] &= ~bit;
            ((int32_t *)out)[v] = v == src ? 0 : -1;
        } else {
            a.D[v * 64 + lane] = v == src ? 0u : 0xffffffffu;
        }
        if (v == src) {
            if (bfsk) a.seen[v] |= bit;
            const unsigned long long rest = cin[v];          // other lanes already at src
            cin[v] = rest | bit;
            const OffT rb = a.ro[v];
            const uint32_t deg = (uint32_t)(a.ro[v + 1] - rb);
            if (rest == 0ull && deg) {
                const unsigned long long old =
                    atomicAdd(&c->qpack[L & 3], (1ull << 32) | (unsigned long long)deg);
                const uint32_t pos = (uint32_t)(old >> 32);
                pk3(a.Q[0], a.Q[1], a.Q[2], L % 3)[pos] = v;
                pk3(a.E[0], a.E[1], a.E[2], L % 3)[pos] = (uint32_t)old;
                pk3(a.R[0], a.R[1], a.R[2], L % 3)[pos] = rb;
            }
            c->start[lane] = L;
            c->out[lane] = out;
            c->lane_T[L & 1][lane] = deg;
            c->active |= bit;
        }
    }
}

// SSSP result of a retired lane: its column of D.
__global__ void k_bt_extract(const uint32_t *D, int32_t nv, int lane, uint32_t *out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x)
        out[v] = D[v * 64 + lane];
}

}  // namespace

// ---------------------------------------------------------------------------
// host API
// ---------------------------------------------------------------------------
namespace {

size_t batch_bytes(const grx_graph *g, int kind) {
    const size_t nv = (size_t)g->nv;
    size_t b = nv * 8 * 4;                                     // next + 3 cur masks
    if (kind == GRX_KIND_BFS) b += nv * 8;                     // seen
    else b += nv * 64 * 4;                                     // D[v][64]
    b += 3 * nv * (4 + 4 + (g->off64 ? 8 : 4));                // frontier ring
    b += nv * 4 + sizeof(BatchCtl);                            // touched list, control
    b += ((nv + 31) / 32) * 4 + 16;                             // touched bitmap
    return b;
}

void *batch_alloc(grx_batch *b, size_t n) {
    void *p = grx_ctx_alloc(b->g->ctx, n, b->s);
    if (p && b->nallocs < (int)(sizeof b->allocs / sizeof b->allocs[0])) b->allocs[b->nallocs++] = {p, n};
    else if (p) { grx_ctx_free(b->g->ctx, p, n, b->s); p = nullptr; }
    return p;
}

void batch_release(grx_batch *b) {
    cudaStreamSynchronize(b->s);
    for (int i = b->nallocs - 1; i >= 0; --i) grx_ctx_free(b->g->ctx, b->allocs[i].p, b->allocs[i].n, b->s);
    free(b);
}

template <typename OffT>
BatchArgs<OffT> batch_args(grx_batch *b) {
    BatchArgs<OffT> a;
    a.nv = b->g->nv;
    a.ne = b->g->ne;
    a.ro = (const OffT *)b->g->ro;
    a.col = b->g->col;
    a.w = b->g->w;
    a.kind = b->kind;
    a.seen = b->seen;
    a.next = b->next;
    for (int i = 0; i < 3; ++i) {
        a.cur[i] = b->cur[i];
        a.Q[i] = b->Q[i];
        a.E[i] = b->E[i];
        a.R[i] = (OffT *)b->R[i];
    }
    a.D = b->D;
    a.touched = b->touched;
    a.tbits = b->tbits;
    a.words = b->g->words;
    a.ctl = b->ctl;
    return a;
}

template <typename OffT>
grx_status batch_step_typed(grx_batch *b, int steps) {
    BatchArgs<OffT> a = batch_args<OffT>(b);
    for (int i = 0; i < steps; ++i) {
        k_bt_begin<OffT><<<1, 1, 0, b->s>>>(a);
        k_bt_expand<OffT><<<b->blocks * (BT_BLOCK / BTX_BLOCK), BTX_BLOCK, 0, b->s>>>(a);
        if (b->kind == GRX_KIND_BFS) k_bt_pull<OffT><<<b->blocks, BT_BLOCK, 0, b->s>>>(a);
        k_bt_finalize<OffT><<<b->blocks, BT_BLOCK, 0, b->s>>>(a);
        k_bt_end<<<1, 1, 0, b->s>>>(b->ctl);
    }
    GRX_CUDA(cudaGetLastError());
    return GRX_OK;
}

}  // namespace

extern "C" grx_status grx_batch_footprint(const grx_graph *g, int kind, size_t *bytes_out) {
    if (!g || !bytes_out) return grx_fail(GRX_EINVAL, "grx_batch_footprint: NULL argument");
    if (g->vid64) return grx_fail(GRX_EINVAL, "grx_batch_footprint: 64-bit vertex ids are served by bfs64 only");
    if (kind != GRX_KIND_BFS && kind != GRX_KIND_SSSP)
        return grx_fail(GRX_EINVAL, "grx_batch_footprint: bad kind %d", kind);
    *bytes_out = batch_bytes(g, kind);
    return GRX_OK;
}

extern "C" grx_status grx_batch_open(grx_graph *g, int kind, void *stream, grx_batch **out) {
    if (!g || !out) return grx_fail(GRX_EINVAL, "grx_batch_open: NULL argument");
    *out = nullptr;
    if (g->vid64) return grx_fail(GRX_EINVAL, "grx_batch_open: 64-bit vertex ids are served by bfs64 only");
    if (kind != GRX_KIND_BFS && kind != GRX_KIND_SSSP)
        return grx_fail(GRX_EINVAL, "grx_batch_open: bad kind %d", kind);
    if (kind == GRX_KIND_SSSP && !g->w) return grx_fail(GRX_EINVAL, "grx_batch_open: SSSP needs weights");
    grx_batch *b = (grx_batch *)calloc(1, sizeof(grx_batch));
    if (!b) return grx_fail(GRX_ENOMEM, "grx_batch_open: host allocation failed");
    b->g = g;
    b->kind = kind;
    b->s = (cudaStream_t)stream;
    b->blocks = g->ctx->num_sms * 4;
    const size_t nv = (size_t)g->nv;
    bool ok = true;
    b->next = (unsigned long long *)batch_alloc(b, nv * 8);
    for (int i = 0; i < 3; ++i) {
        b->cur[i] = (unsigned long long *)batch_alloc(b, nv * 8);
        b->Q[i] = (int32_t *)batch_alloc(b, nv * 4);
        b->E[i] = (uint32_t *)batch_alloc(b, nv * 4);
        b->R[i] = batch_alloc(b, nv * (g->off64 ? 8 : 4));
        ok = ok && b->cur[i] && b->Q[i] && b->E[i] && b->R[i];
    }
    if (kind == GRX_KIND_BFS) b->seen = (unsigned long long *)batch_alloc(b, nv * 8);
    else b->D = (uint32_t *)batch_alloc(b, nv * 64 * 4);
    b->touched = (int32_t *)batch_alloc(b, nv * 4);
    b->tbits = (uint32_t *)batch_alloc(b, ((nv + 31) / 32) * 4 + 16);
    b->ctl = (BatchCtl *)batch_alloc(b, sizeof(BatchCtl));
    ok = ok && b->next && b->touched && b->tbits && b->ctl && (kind == GRX_KIND_BFS ? b->seen != nullptr : b->D != nullptr);
    if (!ok) {
        batch_release(b);
        return grx_fail(GRX_ENOMEM, "grx_batch_open: device allocation of %zu bytes failed",
                        batch_bytes(g, kind));
    }
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMemsetAsync(b->cur[i], 0, nv * 8, b->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->next, 0, nv * 8, b->s);
    if (e == cudaSuccess && b->seen) e = cudaMemsetAsync(b->seen, 0, nv * 8, b->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ctl, 0, sizeof(BatchCtl), b->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->tbits, 0, ((nv + 31) / 32) * 4 + 16, b->s);
    if (e != cudaSuccess) {
        batch_release(b);
        return grx_cuda_fail(e, "grx_batch_open: initialisation");
    }
    *out = b;
    return GRX_OK;
}

extern "C" grx_status grx_batch_close(grx_batch *b) {
    if (b) batch_release(b);
    return GRX_OK;
}

extern "C" grx_status grx_batch_admit(grx_batch *b, int32_t src, void *out_dev, int *lane_out) {
    if (!b || !out_dev) return grx_fail(GRX_EINVAL, "grx_batch_admit: NULL argument");
    if (src < 0 || src >= b->g->nv) return grx_fail(GRX_EINVAL, "grx_batch_admit: source %d out of range", src);
    if (b->busy == ~0ull) return grx_fail(GRX_EBUSY, "grx_batch_admit: all 64 lanes are busy");
    const int lane = __builtin_ctzll(~b->busy);
    const int blocks = b->blocks;
    if (b->g->off64) k_bt_admit<int64_t><<<blocks, BT_BLOCK, 0, b->s>>>(batch_args<int64_t>(b), lane, src, out_dev);
    else k_bt_admit<int32_t><<<blocks, BT_BLOCK, 0, b->s>>>(batch_args<int32_t>(b), lane, src, out_dev);
    GRX_CUDA(cudaGetLastError());
    b->busy |= 1ull << lane;
    b->out_host[lane] = out_dev;
    if (lane_out) *lane_out = lane;
    return GRX_OK;
}

extern "C" grx_status grx_batch_step(grx_batch *b, int steps) {
    if (!b || steps < 0) return grx_fail(GRX_EINVAL, "grx_batch_step: bad argument");
    return b->g->off64 ? batch_step_typed<int64_t>(b, steps) : batch_step_typed<int32_t>(b, steps);
}

extern "C" grx_status grx_batch_poll(grx_batch *b, uint64_t *retired_mask_out) {
    if (!b || !retired_mask_out) return grx_fail(GRX_EINVAL, "grx_batch_poll: NULL argument");
    unsigned long long r = 0;
    int st = 0;
    GRX_CUDA(cudaMemcpyAsync(&r, &b->ctl->retired, 8, cudaMemcpyDeviceToHost, b->s));
    GRX_CUDA(cudaMemcpyAsync(&st, &b->ctl->status, 4, cudaMemcpyDeviceToHost, b->s));
    GRX_CUDA(cudaStreamSynchronize(b->s));
    if (r) {
        GRX_CUDA(cudaMemsetAsync(&b->ctl->retired, 0, 8, b->s));
        if (b->kind == GRX_KIND_SSSP) {
            for (int lane = 0; lane < 64; ++lane)
                if (r >> lane & 1ull)
                    k_bt_extract<<<b->blocks, BT_BLOCK, 0, b->s>>>(b->D, b->g->nv, lane,
                                                                  (uint32_t *)b->out_host[lane]);
            GRX_CUDA(cudaGetLastError());
        }
        GRX_CUDA(cudaStreamSynchronize(b->s));
        b->busy &= ~r;
    }
    *retired_mask_out = r;
    if (st) {
        GRX_CUDA(cudaMemsetAsync(&b->ctl->status, 0, 4, b->s));
        return grx_fail((grx_status)st, "grx_batch_poll: device-side status %d", st);
    }
    return GRX_OK;
}
