// Betweenness centrality (Table 1): Brandes' dependencies summed over the
// given sources, with the forward-and-backward level scheme of McLaughlin
// and Bader's GPU BC (Sec. 2) that Table 1 describes (W = 2|E|, S ~ D/2).
// For a source s: sigma[v] = number of shortest s-v paths, and
// delta[v] = sum over successors w (neighbours one level deeper) of
// sigma[v] / sigma[w] * (1 + delta[w]); bc[v] += delta[v] for v != s.
//
//  * Level codes.  The neighbours of a vertex at depth d sit at depth d - 1,
//    d or d + 1 (or are unreached), so every test the passes make is decided
//    by depth mod 3: each vertex keeps a 2-bit code, depth mod 3 once
//    reached, 3 before.  At 16 vertices per word the codes of 67M vertices
//    take 16.8 MB and stay in L2, where a 4-byte depth probe per edge would
//    pay a DRAM sector.
//  * Forward: a push BFS from s that keeps every level, in level order, in
//    one list (vertex, exclusive edge prefix within its level, row start).
//    An edge (u, w) out of level d whose w is unreached (or claimed for
//    d + 1) is a shortest-path edge: sigma[u] is added to sigma[w] (float64
//    reduction).  Small levels claim w by clearing its code bits (atomic AND;
//    the lane that saw 3 appends w).  Levels with at least push_bitmap * V
//    edges only OR w's bit into a next-level bitmap (no returned atomics);
//    a second phase, by warps owning 32-word chunks of it, writes the new
//    codes, appends the vertices in vertex order and clears the bitmap.
//  * Backward, level k from the deepest one up, one phase per level: every
//    vertex v of level k sums coef[w] = (1 + delta[w]) / sigma[w] over its
//    neighbours w at depth k + 1 (a pull: no atomic per edge, so a hub with
//    a million successors costs no contention).  With acc[v] that sum,
//    delta[v] = sigma[v] * acc[v]; v adds it to bc[v] and leaves
//    coef[v] = 1 / sigma[v] + acc[v] for level k - 1.  The sums are per row
//    of the level's equal warp tiles (a segmented scan across the lanes'
//    runs); a row that crosses tiles adds its partials to acc[v] (float64
//    reductions), the tile holding its last edge lists v, and a short phase
//    after the barrier finishes the listed vertices.  The deepest level has
//    no successors: coef = 1 / sigma, delta = 0.
// One persistent cooperative kernel; phases separated by the bounded grid
// barrier.  Float64 throughout: path counts are exact integers below 2^53,
// and sums differ from a sequential order only in the last bits.
#include "grx_internal.cuh"

namespace {

constexpr int BC_BLOCK = 256;
constexpr int BC_WARPS = BC_BLOCK / 32;
constexpr int BC_ITEMS = 8;
constexpr int BC_WTILE = 32 * BC_ITEMS;
constexpr int BC_RPL = 4;                  // finalize: vertices per lane per round
static_assert(BC_WTILE == 256, "warp_tile_rows8 covers 256-position tiles");

template <typename OffT>
struct BcArgs {
    int64_t words;             // 32-vertex words of the bitmap
    const OffT *ro;
    const int32_t *col;
    uint32_t *code;            // 2-bit level codes, 16 vertices per word (3 = unreached)
    uint32_t *F;               // next-level bitmap of bitmap levels
    double *sigma;
    double *acc;               // backward: row sums, then coef of finished vertices
    int32_t *fix;              // backward: vertices whose rows crossed tiles
    double *bc;
    int32_t *Q;                // every level's vertices, level after level
    uint32_t *E;               // exclusive edge prefix within the vertex's level
    OffT *R;                   // row start
    uint32_t *lstart;          // per level: index of its first vertex in Q
    uint32_t *ledges;          // per level: its edges
    TravCtl *ctl;
    unsigned int *bar_flags;
    DevStats *stats;           // NULL, or per-phase statistics
    uint32_t bmp_min_T;        // forward levels with at least this many edges use the bitmap
    unsigned long long timeout_ns;
    int32_t src;
};

enum { BOP_FWD, BOP_FWD_BMP, BOP_FWD_FINAL, BOP_DEEPEST, BOP_BACK, BOP_BACK_FIX };

struct BcState {
    int d;                     // level being processed
    int op;
    int done;
    int levels;                // levels of the traversal (known once the forward pass ends)
    int phase;                 // phases run so far
    uint32_t start, q, T;      // level d: first list index, vertices, edges
    uint32_t fq;               // fix-up phase: listed vertices
};

template <typename OffT>
union BcWarpSmem {
    struct {
        uint32_t qe[BC_WTILE + 2];
        OffT rs[BC_WTILE + 1];
        double val[BC_WTILE + 1];   // forward: sigma of the element; backward: its row's tile sum
        alignas(16) uint16_t rid[BC_WTILE];
    };
    uint16_t list[32 * 32];         // finalize: compacted bits of a 32-word chunk
};

__device__ __forceinline__ uint32_t level_code(const uint32_t *code, int32_t v) {
    return (__ldcg(code + (v >> 4)) >> ((v & 15) * 2)) & 3u;
}

// Bit i of the 16-bit x moved to bit 2i.
__device__ __forceinline__ uint32_t spread16(uint32_t x) {
    x &= 0xffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

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
            if (!BACK) w.val[n + lane] = __ldcg(a.sigma + __ldcg(Qv + idx));
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

// Warp-tile range [tb0, tb1) of this warp over a level with T edges; false if empty.
__device__ __forceinline__ bool warp_tiles(uint64_t T, uint64_t &tb0, uint64_t &tb1) {
    const uint64_t ntiles = (T + BC_WTILE - 1) / BC_WTILE;
    const uint64_t nwarps = (uint64_t)gridDim.x * BC_WARPS;
    const uint64_t gw = (uint64_t)blockIdx.x * BC_WARPS + (threadIdx.x >> 5);
    const uint64_t per = (ntiles + nwarps - 1) / nwarps;
    tb0 = gw * per;
    tb1 = min(ntiles, tb0 + per);
    return tb0 < tb1;
}

// Forward step of level d: shortest-path edges add sigma; unreached vertices
// are claimed for level d + 1 (claim mode) or marked in F (bitmap mode).
template <typename OffT, bool BMP>
__device__ void forward_level(const BcArgs<OffT> &a, const BcState &st, BcWarpSmem<OffT> &w) {
    const int d = st.d;
    const uint32_t cn = (uint32_t)((d + 1) % 3);
    const unsigned int lane = threadIdx.x & 31;
    const int32_t *Qv = a.Q + st.start;
    const uint32_t *Qe = a.E + st.start;
    const OffT *Qr = a.R + st.start;
    int32_t *Qv_out = a.Q + st.start + st.q;          // level d + 1 follows level d
    uint32_t *Qe_out = a.E + st.start + st.q;
    OffT *Qr_out = a.R + st.start + st.q;
    unsigned long long *ctr = &a.ctl->qpack[(d + 1) & 3];
    const uint64_t T = st.T;
    uint64_t tb0, tb1;
    if (!warp_tiles(T, tb0, tb1)) return;
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
        uint32_t c[BC_ITEMS];
#pragma unroll
        for (int k = 0; k < BC_ITEMS; ++k) c[k] = v[k] >= 0 ? level_code(a.code, v[k]) : 0xffu;
        if (BMP) {
#pragma unroll
            for (int k = 0; k < BC_ITEMS; ++k) {
                if (c[k] == 3u) {                                // codes do not change in this phase
                    atomicAdd(a.sigma + v[k], su[k]);           // results unused: reductions
                    atomicOr(a.F + (v[k] >> 5), 1u << (v[k] & 31));
                }
            }
        } else {
            uint32_t claimed = 0, dag = 0;
#pragma unroll
            for (int k = 0; k < BC_ITEMS; ++k) {
                if (c[k] == 3u) {
                    const uint32_t sh = (uint32_t)(v[k] & 15) * 2u;
                    const uint32_t old = atomicAnd(a.code + (v[k] >> 4), ~((3u ^ cn) << sh));
                    if (((old >> sh) & 3u) == 3u) claimed |= 1u << k;
                    dag |= 1u << k;
                } else if (c[k] == cn) {
                    dag |= 1u << k;
                }
            }
#pragma unroll
            for (int k = 0; k < BC_ITEMS; ++k)
                if (dag >> k & 1u) atomicAdd(a.sigma + v[k], su[k]);
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
        }
        i0 = (next_start == e1) ? i0 + n : i0 + n - 1;
        __syncwarp();
    }
}

// Second phase of a bitmap level: the owner of each 32-word chunk of F writes
// its vertices' codes (d + 1 mod 3), appends them (with edges) to level d + 1
// in vertex order and clears the chunk.
template <typename OffT>
__device__ void forward_final(const BcArgs<OffT> &a, const BcState &st, uint16_t *list) {
    const int d = st.d;
    const uint32_t cpat = (uint32_t)((d + 1) % 3) * 0x55555555u;
    int32_t *Qv_out = a.Q + st.start + st.q;
    uint32_t *Qe_out = a.E + st.start + st.q;
    OffT *Qr_out = a.R + st.start + st.q;
    unsigned long long *ctr = &a.ctl->qpack[(d + 1) & 3];
    const unsigned int lane = threadIdx.x & 31;
    const int64_t nsc = (a.words + 31) / 32;
    const int64_t nwarps = (int64_t)gridDim.x * BC_WARPS;
    for (int64_t sc = (int64_t)blockIdx.x * BC_WARPS + (threadIdx.x >> 5); sc < nsc; sc += nwarps) {
        const int64_t wd = sc * 32 + lane;
        const uint32_t bits = wd < a.words ? __ldcg(a.F + wd) : 0u;
        if (bits) {
            a.F[wd] = 0u;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t half = (bits >> (16 * h)) & 0xffffu;
                if (half) {
                    uint32_t m = spread16(half);
                    m |= m << 1;
                    uint32_t *cw = a.code + wd * 2 + h;
                    *cw = (__ldcg(cw) & ~m) | (cpat & m);
                }
            }
        }
        const int n = warp_compact_bits(bits, list);
        for (int base = 0; base < n; base += 32 * BC_RPL) {
            int32_t v[BC_RPL];
            uint32_t deg[BC_RPL];
            OffT rb[BC_RPL];
            uint32_t app = 0;
#pragma unroll
            for (int k = 0; k < BC_RPL; ++k) {
                const int i = base + k * 32 + (int)lane;
                v[k] = i < n ? (int32_t)(sc * 1024 + list[i]) : 0;
                rb[k] = 0;
                deg[k] = 0;
                if (i < n) {
                    rb[k] = __ldg(a.ro + v[k]);
                    deg[k] = (uint32_t)(__ldg(a.ro + v[k] + 1) - rb[k]);
                    if (deg[k]) app |= 1u << k;
                }
            }
            warp_append_items<BC_RPL, OffT>(v, deg, rb, app, Qv_out, Qe_out, Qr_out, ctr);
        }
        __syncwarp();
    }
}

// Backward step of level k >= 1 (not the deepest): pull of the successors'
// coefficients, per-row sums, vertices finished.
template <typename OffT>
__device__ void backward_level(const BcArgs<OffT> &a, const BcState &st, BcWarpSmem<OffT> &w) {
    const uint32_t ck = (uint32_t)((st.d + 1) % 3);             // successors' code
    const unsigned int lane = threadIdx.x & 31;
    const int32_t *Qv = a.Q + st.start;
    const uint32_t *Qe = a.E + st.start;
    const OffT *Qr = a.R + st.start;
    const uint64_t T = st.T;
    uint64_t tb0, tb1;
    if (!warp_tiles(T, tb0, tb1)) return;
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
        uint32_t cu[BC_ITEMS];
#pragma unroll
        for (int k = 0; k < BC_ITEMS; ++k) cu[k] = u[k] >= 0 ? level_code(a.code, u[k]) : 0xffu;
        double c[BC_ITEMS];
#pragma unroll
        for (int k = 0; k < BC_ITEMS; ++k) c[k] = cu[k] == ck ? __ldcg(a.acc + u[k]) : 0.0;
        // Runs of equal rows in the lane.  Runs between the lane's first and
        // last one are whole rows of the tile; the first (hr, hs) and last
        // (tr, ts) may continue in the neighbouring lanes.
        int hr = -1, tr = -1;
        double hs = 0.0, ts = 0.0;
        {
            int cur = -1;
            double part = 0.0;
#pragma unroll
            for (int k = 0; k < BC_ITEMS; ++k) {
                if (t0 + k < e1) {
                    if (row[k] != cur) {
                        if (cur >= 0) {
                            if (hr < 0) {
                                hr = cur;
                                hs = part;
                            } else {
                                w.val[cur] = part;
                            }
                        }
                        cur = row[k];
                        part = 0.0;
                    }
                    part += c[k];
                }
            }
            if (cur >= 0) {
                if (hr < 0) {
                    hr = cur;
                    hs = part;
                }
                tr = cur;
                ts = part;
            }
        }
        // Segmented inclusive scan of the lanes' last runs: a lane continues
        // the previous lane's segment when its items all belong to that row.
        const int prev_tr = __shfl_up_sync(GRX_FULL_MASK, tr, 1);
        const bool single = hr == tr;
        int f = (lane > 0 && single && tr >= 0 && prev_tr == tr) ? 0 : 1;
        double sv = ts;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double pv = __shfl_up_sync(GRX_FULL_MASK, sv, o);
            const int pf = __shfl_up_sync(GRX_FULL_MASK, f, o);
            if (lane >= (unsigned)o) {
                if (!f) sv += pv;
                f |= pf;
            }
        }
        const double prev_sv = __shfl_up_sync(GRX_FULL_MASK, sv, 1);
        const int next_hr = __shfl_down_sync(GRX_FULL_MASK, hr, 1);
        if (!single && hr >= 0) w.val[hr] = (lane > 0 && prev_tr == hr ? prev_sv : 0.0) + hs;
        if (tr >= 0 && (lane == 31 || next_hr != tr)) w.val[tr] = sv;
        __syncwarp();
        // rows inside the tile finish here; rows crossing it add to acc, and
        // the tile with the row's last edge lists the vertex for the fix-up
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
                if (s != 0.0) atomicAdd(a.acc + v, s);       // result unused: reduction
                if (re <= e1) a.fix[atomicAdd(&a.ctl->bcfix[st.d % 3], 1u)] = v;
            }
        }
        i0 = (next_start == e1) ? i0 + n : i0 + n - 1;
        __syncwarp();
    }
}

// After a backward level: the vertices whose rows crossed tiles.
template <typename OffT>
__device__ void backward_fix(const BcArgs<OffT> &a, const BcState &st) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)st.q;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = __ldcg(a.fix + i);
        finish_vertex(a, v, __ldcg(a.acc + v));
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
__device__ __forceinline__ int forward_op(const BcArgs<OffT> &a, uint32_t T) {
    return T >= a.bmp_min_T ? BOP_FWD_BMP : BOP_FWD;
}

template <typename OffT>
__device__ BcState bc_next(const BcArgs<OffT> &a, const BcState &st) {
    BcState ns = st;
    ns.phase = st.phase + 1;
    if (st.op == BOP_FWD_BMP) {
        ns.op = BOP_FWD_FINAL;
        return ns;
    }
    if (st.op == BOP_FWD || st.op == BOP_FWD_FINAL) {           // end of forward level d
        const unsigned long long pk = ld_relaxed_u64(&a.ctl->qpack[(st.d + 1) & 3]);
        const uint32_t q = (uint32_t)(pk >> 32);
        if (q > 0) {
            ns.d = st.d + 1;
            ns.start = st.start + st.q;
            ns.q = q;
            ns.T = (uint32_t)pk;
            ns.op = forward_op(a, ns.T);
        } else {
            ns.levels = st.d + 1;
            ns.op = BOP_DEEPEST;                                // level d is the deepest
            ns.done = st.d == 0;                                // only the source: nothing to add
        }
        return ns;
    }
    if (st.op == BOP_BACK) {                                    // rows that crossed tiles?
        const uint32_t nfix = ld_relaxed_u32(&a.ctl->bcfix[st.d % 3]);
        if (nfix > 0) {
            ns.op = BOP_BACK_FIX;
            ns.fq = nfix;
            return ns;
        }
    }
    if (st.d == 1) {                                            // level 0 is the source
        ns.done = 1;
        return ns;
    }
    ns.op = BOP_BACK;
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
        s.op = forward_op(a, deg);
        s.done = deg == 0;
        s.levels = 1;
        s_st = s;
    }
    __syncthreads();
    for (;;) {
        const BcState st = s_st;
        if (st.done) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (st.op == BOP_FWD || st.op == BOP_FWD_BMP) {
                a.ctl->qpack[(st.d + 2) & 3] = 0ull;
                a.lstart[st.d] = st.start;
                a.ledges[st.d] = st.T;
            }
            // the fix-up counter of level d - 1 was last read two barriers ago
            if (st.op == BOP_BACK) a.ctl->bcfix[(st.d + 2) % 3] = 0u;
            if (a.stats && st.phase < GRX_MAX_LEVELS_STATS) {
                // phases in order: forward levels (dir 0), then backward levels (dir 1)
                a.stats->level_t0[st.phase] = grx_globaltimer();
                a.stats->dir[st.phase] = st.op >= BOP_DEEPEST;
                a.stats->frontier[st.phase] = st.op == BOP_BACK_FIX ? st.fq : st.q;
                a.stats->edges_examined[st.phase] = (st.op == BOP_FWD_FINAL || st.op == BOP_BACK_FIX) ? 0 : st.T;
                a.stats->levels = st.phase + 1;
            }
        }
        switch (st.op) {
            case BOP_FWD: forward_level<OffT, false>(a, st, w); break;
            case BOP_FWD_BMP: forward_level<OffT, true>(a, st, w); break;
            case BOP_FWD_FINAL: forward_final<OffT>(a, st, w.list); break;
            case BOP_DEEPEST: deepest_level<OffT>(a, st); break;
            case BOP_BACK_FIX: {
                BcState fs = st;
                fs.q = st.fq;
                backward_fix<OffT>(a, fs);
                break;
            }
            default: backward_level<OffT>(a, st, w); break;
        }
        if (!flag_barrier(bar)) return;
        if (threadIdx.x == 0) s_st = bc_next(a, st);
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->levels_run = s_st.levels;
        if (a.stats && s_st.phase <= GRX_MAX_LEVELS_STATS) a.stats->level_t0[s_st.phase] = grx_globaltimer();
    }
}

template <typename OffT>
__global__ void k_bc_init(int32_t src, const OffT *ro, uint32_t *code, double *sigma, int32_t *Q, uint32_t *E,
                          OffT *R, TravCtl *ctl) {
    code[src >> 4] &= ~(3u << ((src & 15) * 2));               // level 0
    sigma[src] = 1.0;
    Q[0] = src;
    E[0] = 0;
    R[0] = ro[src];
    for (int i = 0; i < 4; ++i) ctl->qpack[i] = 0ull;
    for (int i = 0; i < 3; ++i) ctl->bcfix[i] = 0u;
}

template <typename OffT>
grx_status launch_typed(grx_graph *g, const int32_t *srcs, int n, double *bc_out, const grx_opts *o,
                        cudaStream_t s) {
    BcArgs<OffT> a;
    a.words = g->words;
    a.ro = (const OffT *)g->ro;
    a.col = g->col;
    a.code = g->bc_code;
    a.F = g->fbits[1];
    a.sigma = g->bc_sigma;
    a.acc = g->bc_acc;
    a.fix = g->ulist[0];
    a.bc = bc_out;
    a.Q = g->qv[0];
    a.E = g->qe[0];
    a.R = (OffT *)g->qr[0];
    a.lstart = g->qe[1];
    a.ledges = g->qe[2];
    a.ctl = g->ctl;
    a.bar_flags = g->bar_flags;
    a.stats = o->collect_stats ? g->stats : nullptr;
    a.timeout_ns = grx_timeout_ns(o);
    {   // bitmap forward levels from push_bitmap * nv edges (0 = 1/8, < 0 = never)
        const double pb = o->push_bitmap == 0.f ? 0.125 : (double)o->push_bitmap;
        const double t = pb * (double)g->nv;
        a.bmp_min_T = pb < 0 ? 0xffffffffu : (t < 1.0 ? 1u : (t > 4294967295.0 ? 0xffffffffu : (uint32_t)t));
    }
    if (o->collect_stats) GRX_CUDA(cudaMemsetAsync(g->stats, 0, sizeof(DevStats), s));
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
    if (o->ev_begin) GRX_CUDA(cudaEventRecord((cudaEvent_t)o->ev_begin, s));
    for (int i = 0; i < n; ++i) {
        a.src = srcs[i];
        GRX_CUDA(cudaMemsetAsync(a.code, 0xff, (size_t)g->words * 8, s));
        GRX_CUDA(cudaMemsetAsync(a.F, 0, (size_t)g->words * 4, s));
        GRX_CUDA(cudaMemsetAsync(a.sigma, 0, nv * 8, s));
        GRX_CUDA(cudaMemsetAsync(a.acc, 0, nv * 8, s));
        k_bc_init<OffT><<<1, 1, 0, s>>>(a.src, a.ro, a.code, a.sigma, a.Q, a.E, a.R, g->ctl);
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
