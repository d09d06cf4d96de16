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
//    edges only add the path counts (no claim, no returned atomics): after
//    the barrier the unreached vertices with a nonzero count are exactly the
//    new level, and warps owning 32-word chunks of the vertices find them,
//    write their codes and append them in vertex order.
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
//  * Direction per level (the paper's direction-optimising idea, Sec. 6.1,
//    carried over to both sweeps, by edge counts the level lists provide):
//    a forward level whose frontier has more than four times the edges of
//    all still-unreached vertices together is a pull instead -- every unreached non-isolated
//    vertex sums sigma over its neighbours at depth d (all of them: no early
//    exit, sigma needs every parent) and joins level d + 1 if that sum is
//    nonzero; a backward level whose rows hold more edges than the level
//    below it is a push instead -- each vertex w of level k + 1 adds coef[w]
//    into acc[v] of its neighbours at depth k (float64 reductions), and a
//    second phase finishes level k's vertices.
// One persistent cooperative kernel; phases separated by the bounded grid
// barrier.  Float64 throughout: path counts are exact integers below 2^53,
// and sums differ from a sequential order only in the last bits.
#include "grx_internal.cuh"

namespace {

#ifndef GRX_BC_MIN_BLOCKS
#define GRX_BC_MIN_BLOCKS 3                 // resident blocks per SM (register cap)
#endif
constexpr int BC_BLOCK = 256;
constexpr int BC_WARPS = BC_BLOCK / 32;
constexpr int BC_ITEMS = 8;
constexpr int BC_WTILE = 32 * BC_ITEMS;
constexpr int BC_RPL = 4;                  // finalize: vertices per lane per round
// A forward pull reads every edge of every unreached vertex (no early exit)
// with a row per lane; measured on GB300 one pulled edge costs about four
// pushed ones, so a level is pulled when the unreached vertices' edges times
// this ratio are fewer than the frontier's.
constexpr unsigned long long BC_PULL_RATIO = 4;
static_assert(BC_WTILE == 256, "warp_tile_rows8 covers 256-position tiles");

template <typename OffT>
struct BcArgs {
    int64_t words;             // 32-vertex words of the bitmap
    int64_t ne;                // edges of the graph
    int mode;                  // 0 edge-count rule, 1 forward push / backward pull only, 2 the other way only
    const uint32_t *nz;        // non-isolated bitmap
    const OffT *ro;
    const int32_t *col;
    uint32_t *code;            // 2-bit level codes, 16 vertices per word (3 = unreached)
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

enum { BOP_FWD, BOP_FWD_BMP, BOP_FWD_FINAL, BOP_FWD_PULL, BOP_DEEPEST, BOP_BACK, BOP_BACK_FIX,
       BOP_BACK_PUSH, BOP_BACK_FIN };

struct BcState {
    int d;                     // level being processed
    int op;
    int done;
    int levels;                // levels of the traversal (known once the forward pass ends)
    int phase;                 // phases run so far
    uint32_t start, q, T;      // level d: first list index, vertices, edges
    uint32_t fq;               // fix-up phase: listed vertices
    uint32_t ps, pq, pT;       // backward: level d + 1's list slice and edges
    unsigned long long seenE;  // forward: edges of the levels up to d
};

template <typename OffT>
union BcWarpSmem {
    struct {
        uint32_t qe[BC_WTILE + 2];
        OffT rs[BC_WTILE + 1];
        double val[BC_WTILE + 1];   // forward: sigma of the element; backward: its row's tile sum
        alignas(16) uint16_t rid[BC_WTILE];
    };
    struct {
        uint16_t list[32 * 32];     // finalize / pull: compacted bits of a 32-word chunk
        uint32_t fb[32];            // pull: bits of the chunk's vertices that joined level d + 1
    };
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

// Even bits of x's 2-bit fields that equal 3 (unreached), packed into 16 bits.
__device__ __forceinline__ uint32_t unreached16(uint32_t x) {
    x = x & (x >> 1) & 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0f0f0f0fu;
    x = (x | (x >> 4)) & 0x00ff00ffu;
    x = (x | (x >> 8)) & 0x0000ffffu;
    return x;
}

// Stages the level elements that start before e1 (from index i0) into shared
// memory; returns their count, with sigma or acc of each element if asked.
enum { STAGE_SIGMA, STAGE_NONE, STAGE_ACC };

template <typename OffT, int WHAT>
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
            if (WHAT == STAGE_SIGMA) w.val[n + lane] = __ldcg(a.sigma + __ldcg(Qv + idx));
            if (WHAT == STAGE_ACC) w.val[n + lane] = __ldcg(a.acc + __ldcg(Qv + idx));
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
        const int n = stage_elements<OffT, STAGE_SIGMA>(a, Qv, Qe, Qr, st.q, i0, e1, w);
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
                if (c[k] == 3u) atomicAdd(a.sigma + v[k], su[k]);   // codes fixed in this phase; reduction
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

// Second phase of a bitmap level: per 32-word chunk of vertices, the
// unreached ones whose path count became nonzero form level d + 1; the owner
// writes their codes (d + 1 mod 3) and appends them (with edges) in vertex
// order.  The warp reads the chunk's path counts word by word (coalesced).
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
        uint32_t cand = 0u;
        if (wd < a.words)
            cand = (unreached16(__ldcg(a.code + 2 * wd)) | (unreached16(__ldcg(a.code + 2 * wd + 1)) << 16)) &
                   __ldg(a.nz + wd);
        uint32_t bits = 0u;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
            const uint32_t cj = __shfl_sync(GRX_FULL_MASK, cand, j);
            const bool hit = ((cj >> lane) & 1u) && __ldcg(a.sigma + ((sc * 32 + j) * 32 + lane)) != 0.0;
            const uint32_t b = __ballot_sync(GRX_FULL_MASK, hit);
            if ((int)lane == j) bits = b;
        }
        if (bits) {
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
        const int n = stage_elements<OffT, STAGE_NONE>(a, Qv, Qe, Qr, st.q, i0, e1, w);
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


// Forward pull of level d: the owner of each 32-word chunk sums, for every
// unreached non-isolated vertex of the chunk, sigma over its neighbours at
// depth d; a vertex with such a neighbour joins level d + 1 (sigma, code,
// appended in vertex order).  Rows longer than 32 edges are summed by the
// whole warp.
template <typename OffT>
__device__ void forward_pull(const BcArgs<OffT> &a, const BcState &st, BcWarpSmem<OffT> &w) {
    const int d = st.d;
    const uint32_t cd = (uint32_t)(d % 3);
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
        uint32_t cand = 0u;
        if (wd < a.words)
            cand = (unreached16(__ldcg(a.code + 2 * wd)) | (unreached16(__ldcg(a.code + 2 * wd + 1)) << 16)) &
                   __ldg(a.nz + wd);
        w.fb[lane] = 0u;
        const int n = warp_compact_bits(cand, w.list);
        for (int base = 0; base < n; base += 32) {
            const int i = base + (int)lane;
            const int32_t v = i < n ? (int32_t)(sc * 1024 + w.list[i]) : -1;
            OffT rb = 0;
            uint32_t deg = 0;
            if (v >= 0) {
                rb = __ldg(a.ro + v);
                deg = (uint32_t)(__ldg(a.ro + v + 1) - rb);
            }
            double s = 0.0;
            const bool longrow = deg > 32u;
            if (!longrow) {
                for (uint32_t k = 0; k < deg; k += 4) {
                    int32_t u[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) u[j] = k + j < deg ? __ldg(a.col + rb + (OffT)(k + j)) : -1;
                    uint32_t cu[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) cu[j] = u[j] >= 0 ? level_code(a.code, u[j]) : 0xffu;
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (cu[j] == cd) s += __ldcg(a.sigma + u[j]);
                }
            }
            unsigned int lm = __ballot_sync(GRX_FULL_MASK, longrow);
            while (lm) {
                const int owner = __ffs(lm) - 1;
                lm &= lm - 1;
                const OffT lrb = __shfl_sync(GRX_FULL_MASK, rb, owner);
                const uint32_t ldeg = __shfl_sync(GRX_FULL_MASK, deg, owner);
                double ls = 0.0;
                for (uint32_t k = lane; k < ldeg; k += 32) {
                    const int32_t u = __ldg(a.col + lrb + (OffT)k);
                    if (level_code(a.code, u) == cd) ls += __ldcg(a.sigma + u);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) ls += __shfl_xor_sync(GRX_FULL_MASK, ls, o);
                if ((int)lane == owner) s = ls;
            }
            if (s > 0.0) {
                a.sigma[v] = s;
                atomicOr(&w.fb[(v >> 5) & 31], 1u << (v & 31));
            }
        }
        __syncwarp();
        const uint32_t bits = w.fb[lane];
        if (bits) {
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
        const int m = warp_compact_bits(bits, w.list);
        for (int base = 0; base < m; base += 32 * BC_RPL) {
            int32_t v[BC_RPL];
            uint32_t deg[BC_RPL];
            OffT rb[BC_RPL];
            uint32_t app = 0;
#pragma unroll
            for (int k = 0; k < BC_RPL; ++k) {
                const int i = base + k * 32 + (int)lane;
                v[k] = i < m ? (int32_t)(sc * 1024 + w.list[i]) : 0;
                rb[k] = 0;
                deg[k] = 0;
                if (i < m) {
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

// Backward push into level d: every vertex w of level d + 1 adds coef[w]
// into acc[v] of its neighbours at depth d (float64 reductions).
template <typename OffT>
__device__ void backward_push(const BcArgs<OffT> &a, const BcState &st, BcWarpSmem<OffT> &w) {
    const uint32_t cd = (uint32_t)(st.d % 3);
    const unsigned int lane = threadIdx.x & 31;
    const int32_t *Qv = a.Q + st.ps;
    const uint32_t *Qe = a.E + st.ps;
    const OffT *Qr = a.R + st.ps;
    const uint64_t T = st.pT;
    uint64_t tb0, tb1;
    if (!warp_tiles(T, tb0, tb1)) return;
    int64_t i0 = warp_upper_index_cg(Qe, st.pq, (uint32_t)(tb0 * BC_WTILE));
    for (uint64_t tile = tb0; tile < tb1; ++tile) {
        const uint64_t e0 = tile * BC_WTILE;
        const uint32_t e1 = (uint32_t)min(T, e0 + BC_WTILE);
        const int n = stage_elements<OffT, STAGE_ACC>(a, Qv, Qe, Qr, st.pq, i0, e1, w);
        const uint32_t next_start = w.qe[n];
        int row[BC_ITEMS];
        warp_tile_rows8(w.rid, w.qe, (uint32_t)e0, n, row);
        const uint32_t t0 = (uint32_t)e0 + lane * BC_ITEMS;
        int32_t v[BC_ITEMS];
        double x[BC_ITEMS];
#pragma unroll
        for (int k = 0; k < BC_ITEMS; ++k) {
            const uint32_t e = t0 + k;
            const int j = row[k];
            const bool ok = e < e1;
            const OffT idx = ok ? w.rs[j] + (OffT)(e - w.qe[j]) : (OffT)0;
            v[k] = ok ? __ldg(a.col + idx) : -1;
            x[k] = ok ? w.val[j] : 0.0;
        }
        __syncwarp();
        uint32_t cv[BC_ITEMS];
#pragma unroll
        for (int k = 0; k < BC_ITEMS; ++k) cv[k] = v[k] >= 0 ? level_code(a.code, v[k]) : 0xffu;
#pragma unroll
        for (int k = 0; k < BC_ITEMS; ++k)
            if (cv[k] == cd) atomicAdd(a.acc + v[k], x[k]);              // result unused: reduction
        i0 = (next_start == e1) ? i0 + n : i0 + n - 1;
        __syncwarp();
    }
}

// After a backward push: every vertex of level d finishes from acc.
template <typename OffT>
__device__ void backward_fin(const BcArgs<OffT> &a, const BcState &st) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)st.q;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = __ldcg(a.Q + st.start + i);
        finish_vertex(a, v, __ldcg(a.acc + v));
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

// Kind of forward level d with T frontier edges; seenE = edges of the levels
// up to d.  Pull when the still-unreached vertices have fewer edges.
template <typename OffT>
__device__ __forceinline__ int forward_op(const BcArgs<OffT> &a, int d, uint32_t T, unsigned long long seenE) {
    const unsigned long long left = (unsigned long long)a.ne > seenE ? (unsigned long long)a.ne - seenE : 0ull;
    if (d > 0 && (a.mode == 2 || (a.mode == 0 && left * BC_PULL_RATIO < (unsigned long long)T)))
        return BOP_FWD_PULL;
    return T >= a.bmp_min_T ? BOP_FWD_BMP : BOP_FWD;
}

// Backward level d (>= 1) after level d + 1 = (start, q, T) of st: its state.
template <typename OffT>
__device__ __forceinline__ BcState backward_state(const BcArgs<OffT> &a, const BcState &st, BcState ns) {
    ns.d = st.d - 1;
    ns.ps = st.start;
    ns.pq = st.q;
    ns.pT = st.T;
    ns.start = ld_relaxed_u32(a.lstart + ns.d);
    ns.q = st.start - ns.start;
    ns.T = ld_relaxed_u32(a.ledges + ns.d);
    ns.op = (a.mode == 2 || (a.mode == 0 && ns.pT < ns.T)) ? BOP_BACK_PUSH : BOP_BACK;
    return ns;
}

template <typename OffT>
__device__ BcState bc_next(const BcArgs<OffT> &a, const BcState &st) {
    BcState ns = st;
    ns.phase = st.phase + 1;
    if (st.op == BOP_FWD_BMP) {
        ns.op = BOP_FWD_FINAL;
        return ns;
    }
    if (st.op == BOP_FWD || st.op == BOP_FWD_FINAL || st.op == BOP_FWD_PULL) {   // end of forward level d
        const unsigned long long pk = ld_relaxed_u64(&a.ctl->qpack[(st.d + 1) & 3]);
        const uint32_t q = (uint32_t)(pk >> 32);
        if (q > 0) {
            ns.d = st.d + 1;
            ns.start = st.start + st.q;
            ns.q = q;
            ns.T = (uint32_t)pk;
            ns.seenE = st.seenE + ns.T;
            ns.op = forward_op(a, ns.d, ns.T, ns.seenE);
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
    if (st.op == BOP_BACK_PUSH) {
        ns.op = BOP_BACK_FIN;
        return ns;
    }
    if (st.d == 1) {                                            // level 0 is the source
        ns.done = 1;
        return ns;
    }
    return backward_state(a, st, ns);
}

template <typename OffT>
__global__ void __launch_bounds__(BC_BLOCK, GRX_BC_MIN_BLOCKS) k_bc_persistent(BcArgs<OffT> a) {
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
        s.seenE = deg;
        s.op = forward_op(a, 0, deg, s.seenE);
        s.done = deg == 0;
        s.levels = 1;
        s_st = s;
    }
    __syncthreads();
    for (;;) {
        const BcState st = s_st;
        if (st.done) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (st.op == BOP_FWD || st.op == BOP_FWD_BMP || st.op == BOP_FWD_PULL) {
                a.ctl->qpack[(st.d + 2) & 3] = 0ull;
                a.lstart[st.d] = st.start;
                a.ledges[st.d] = st.T;
            }
            // the fix-up counter of level d - 1 was last read at least two barriers ago
            if (st.op == BOP_BACK || st.op == BOP_BACK_PUSH) a.ctl->bcfix[(st.d + 2) % 3] = 0u;
            if (a.stats && st.phase < GRX_MAX_LEVELS_STATS) {
                // phases in order: forward levels (dir 0), then backward levels (dir 1)
                a.stats->level_t0[st.phase] = grx_globaltimer();
                a.stats->dir[st.phase] = st.op >= BOP_DEEPEST;
                a.stats->frontier[st.phase] = st.op == BOP_BACK_FIX ? st.fq : st.q;
                // edges the phase reads: a forward pull reads the unreached vertices' rows,
                // a backward push the rows of level d + 1
                a.stats->edges_examined[st.phase] =
                    st.op == BOP_BACK_PUSH ? st.pT
                    : st.op == BOP_FWD_PULL ? ((unsigned long long)a.ne > st.seenE ? a.ne - st.seenE : 0)
                    : (st.op == BOP_FWD_FINAL || st.op == BOP_BACK_FIX || st.op == BOP_BACK_FIN) ? 0 : st.T;
                a.stats->vertices_scanned[st.phase] = st.op;    // the phase's kind
                a.stats->levels = st.phase + 1;
            }
        }
        switch (st.op) {
            case BOP_FWD: forward_level<OffT, false>(a, st, w); break;
            case BOP_FWD_BMP: forward_level<OffT, true>(a, st, w); break;
            case BOP_FWD_FINAL: forward_final<OffT>(a, st, w.list); break;
            case BOP_FWD_PULL: forward_pull<OffT>(a, st, w); break;
            case BOP_BACK_PUSH: backward_push<OffT>(a, st, w); break;
            case BOP_BACK_FIN: backward_fin<OffT>(a, st); break;
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
    a.ne = g->ne;
    a.mode = o->direction;
    a.nz = g->nz_bits;
    a.ro = (const OffT *)g->ro;
    a.col = g->col;
    a.code = g->bc_code;
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
