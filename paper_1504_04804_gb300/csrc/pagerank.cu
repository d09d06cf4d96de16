// PageRank (Algorithm 3) in the normalised mode with dangling compensation
// (Sec. 7).  Pull formulation, atomic-free on the rank array:
//
//   c_i[u]   = r_i[u] / deg(u)                       (non-isolated u)
//   r_{i+1}[v] = base_i + d * sum_{u in N(v)} c_i[u],  base_i = (1-d)/N + d*D_i/N
//
// On a symmetric graph a zero-degree vertex has no in-edges either, so every
// isolated vertex holds the same rank; D_i = n_isolated * r_i[isolated] and
// base_i follow from a scalar recurrence the host evaluates in double.
//
// One launch per iteration over equal tiles of the edge array (the active
// list of non-isolated vertices has the CSR offsets as its edge prefix, so a
// tile holds at most TILE+1 rows; the first row and row count of every tile
// are computed once per graph and cached).  Each thread loads a contiguous
// run of PR_ITEMS edges' c[col[e]] (all loads in flight before any use),
// finds their rows by a scatter + max-scan in shared memory, and adds one
// partial per run of equal rows to the row's shared accumulator.  Rows inside the tile are finished there;
// rows that cross a tile boundary add their partial to a global accumulator
// and are finished by a small fix-up launch.  Accumulation is FP32.
#include <vector>

#include "grx_internal.cuh"

namespace {

constexpr int PR_BLOCK = 256;
constexpr int PR_ITEMS = 9;                  // odd: conflict-free strided smem reads
constexpr int PR_TILE = PR_BLOCK * PR_ITEMS;

struct PrSmem {
    union alignas(16) {
        float acc[PR_TILE + 2];
        int32_t colt[PR_TILE];         // the tile's columns, staged before the gathers
    };
    uint32_t qe[PR_TILE + 2];
    int32_t u[PR_TILE + 2];
    uint16_t rid[PR_TILE];
    int wmax[PR_BLOCK / 32];
};

// Row of each of a thread's PR_ITEMS consecutive tile positions, with no
// per-item search: positions start at row 0; every row j > 0 writes j at its
// first position (starts[j] - origin, strictly increasing for rows with
// edges); an inclusive max-scan over positions (per thread, then across the
// block's threads) gives each position its row.  All threads call.
__device__ __forceinline__ void block_tile_rows(uint16_t *rid, int *wmax, const uint32_t *starts,
                                                uint32_t origin, int n, int len, int (&row)[PR_ITEMS]) {
    const int t0 = threadIdx.x * PR_ITEMS;
#pragma unroll
    for (int k = 0; k < PR_ITEMS; ++k) rid[t0 + k] = 0;
    __syncthreads();
    for (int j = 1 + threadIdx.x; j < n; j += PR_BLOCK) {
        const uint32_t p = starts[j] - origin;
        if (p < (uint32_t)len) rid[p] = (uint16_t)j;
    }
    __syncthreads();
    int m = 0;
#pragma unroll
    for (int k = 0; k < PR_ITEMS; ++k) {
        m = max(m, (int)rid[t0 + k]);
        row[k] = m;
    }
    const unsigned int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(GRX_FULL_MASK, x, o);
        if (lane >= (unsigned)o) x = max(x, y);
    }
    if (lane == 31) wmax[wid] = x;
    __syncthreads();
    int carry = __shfl_up_sync(GRX_FULL_MASK, x, 1);
    if (lane == 0) carry = 0;
    for (unsigned int w = 0; w < wid; ++w) carry = max(carry, wmax[w]);
#pragma unroll
    for (int k = 0; k < PR_ITEMS; ++k) row[k] = max(row[k], carry);
}

// Adds each item's value to its row's shared accumulator.  A thread's items
// are consecutive positions and its rows non-decreasing, and a warp's threads
// hold consecutive runs of positions, so a row's items within a warp sit in
// consecutive lanes.  A row whose items all fall strictly inside one lane's
// items (neither its first nor its last run) has that lane as its only writer:
// a plain store.  Rows at lane boundaries are summed across the warp by a
// segmented shuffle scan and added once per warp by the lane where they end
// (a hub row filling a whole tile costs one shared atomic per warp instead of
// one per thread).
__device__ __forceinline__ void add_runs(float *acc, const int (&row)[PR_ITEMS], const float (&g)[PR_ITEMS],
                                         int valid) {
    const unsigned int lane = threadIdx.x & 31;
    int fk = -1, lk = -1;          // rows of the lane's first run (when it ends inside the lane) and last run
    float fs = 0.f, ls = 0.f;
    if (valid > 0) {
        int cj = row[0];
        float part = 0.f;
        bool first = true;
#pragma unroll
        for (int k = 0; k < PR_ITEMS; ++k) {
            if (k < valid) {
                if (row[k] != cj) {
                    if (first) {
                        fk = cj;
                        fs = part;
                        first = false;
                    } else {
                        acc[cj] = part;           // a row inside this lane's items
                    }
                    part = 0.f;
                    cj = row[k];
                }
                part += g[k];
            }
        }
        lk = cj;
        ls = part;
    }
    // The last run continues the previous lane's last run when the lane has a
    // single run of the same row; otherwise it starts a segment.
    const int pk = __shfl_up_sync(GRX_FULL_MASK, lk, 1);
    const bool prev_same = lane > 0 && pk == lk && lk >= 0;
    float sum = ls;
    int head = (fk >= 0 || !prev_same) ? 1 : 0;
    // segmented inclusive scan of the last runs (Hillis-Steele with head flags)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float s2 = __shfl_up_sync(GRX_FULL_MASK, sum, o);
        const int h2 = __shfl_up_sync(GRX_FULL_MASK, head, o);
        if (lane >= (unsigned)o && !head) {
            sum += s2;
            head |= h2;
        }
    }
    // the previous lane's scanned last run, for this lane's first run
    const float ps = __shfl_up_sync(GRX_FULL_MASK, sum, 1);
    if (fk >= 0) atomicAdd(&acc[fk], fs + ((lane > 0 && pk == fk) ? ps : 0.f));
    // a last run whose row the next lane does not continue ends here
    const int nfk = __shfl_down_sync(GRX_FULL_MASK, fk, 1);
    const int nlk = __shfl_down_sync(GRX_FULL_MASK, lk, 1);
    const bool next_cont = lane < 31 && ((nfk >= 0 && nfk == lk) || (nfk < 0 && nlk == lk));
    if (lk >= 0 && !next_cont) atomicAdd(&acc[lk], sum);
}

__global__ void __launch_bounds__(PR_BLOCK) k_pr_iter(
    const int32_t *__restrict__ col, const int32_t *__restrict__ active,
    const uint32_t *__restrict__ aoff, const int2 *__restrict__ tiles, int64_t ne,
    const float *__restrict__ c_in, float *__restrict__ c_out, float *__restrict__ s_acc,
    int32_t *__restrict__ fix, float *__restrict__ rank, float base, float d) {
    __shared__ PrSmem sm;
    const uint64_t tile = blockIdx.x;
    const uint64_t e0 = tile * PR_TILE;
    const uint64_t e1 = min((uint64_t)ne, e0 + PR_TILE);
    const int len = (int)(e1 - e0);
    const int t0 = threadIdx.x * PR_ITEMS;
    // The tile's columns arrive in shared memory by coalesced 16-byte loads
    // (a tile starts on a 16-byte boundary when the column array does:
    // PR_TILE * 4 is a multiple of 16; the last tile's tail past its last
    // full vector, or a column array an outside allocator left unaligned, is
    // read word by word), then each thread takes its PR_ITEMS consecutive
    // columns from there (odd stride: conflict-free) and issues all its
    // gathers at once.
    {
        const int nvec = ((uintptr_t)col & 15u) == 0 ? len >> 2 : 0;
        const int4 *src = reinterpret_cast<const int4 *>(col + e0);
        int4 *dst = reinterpret_cast<int4 *>(sm.colt);
        for (int i = threadIdx.x; i < nvec; i += PR_BLOCK) dst[i] = __ldg(src + i);
        for (int i = (nvec << 2) + threadIdx.x; i < len; i += PR_BLOCK) sm.colt[i] = __ldg(col + e0 + i);
    }
    const int2 tr = __ldg(tiles + tile);
    __syncthreads();
    int32_t u[PR_ITEMS];
#pragma unroll
    for (int k = 0; k < PR_ITEMS; ++k) u[k] = t0 + k < len ? sm.colt[t0 + k] : -1;
    float g[PR_ITEMS];
#pragma unroll
    for (int k = 0; k < PR_ITEMS; ++k) g[k] = u[k] >= 0 ? __ldg(c_in + u[k]) : 0.f;
    __syncthreads();                   // colt is reused as the row accumulators below
    const int64_t i0 = tr.x;
    const int n = tr.y;
    if (threadIdx.x == 0) fix[tile] = -1;
    for (int j = threadIdx.x; j <= n; j += PR_BLOCK) {   // n+1 prefixes: qe[n] = end of last row
        sm.qe[j] = __ldg(aoff + i0 + j);
        if (j < n) sm.u[j] = __ldg(active + i0 + j);
        sm.acc[j] = 0.f;
    }
    __syncthreads();
    int row[PR_ITEMS];
    block_tile_rows(sm.rid, sm.wmax, sm.qe, (uint32_t)e0, n, len, row);
    add_runs(sm.acc, row, g, len - t0);
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += PR_BLOCK) {
        const int32_t v = sm.u[j];
        const uint32_t start = sm.qe[j], end = sm.qe[j + 1];
        if (start >= e0 && end <= e1) {
            const float r = base + d * sm.acc[j];
            c_out[v] = r / (float)(end - start);
            if (rank) rank[v] = r;
        } else {
            atomicAdd(s_acc + v, sm.acc[j]);
            if (end <= e1) fix[tile] = v;   // this tile holds the row's last edge
        }
    }
}

__global__ void k_pr_fixup(const int32_t *__restrict__ fix, int64_t ntiles, const void *ro, int off64,
                           float *__restrict__ s_acc, float *__restrict__ c_out,
                           float *__restrict__ rank, float base, float d) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntiles;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = fix[t];
        if (v < 0) continue;
        const int64_t deg = off64 ? ((const int64_t *)ro)[v + 1] - ((const int64_t *)ro)[v]
                                  : (int64_t)(((const int32_t *)ro)[v + 1] - ((const int32_t *)ro)[v]);
        const float r = base + d * s_acc[v];
        s_acc[v] = 0.f;
        c_out[v] = r / (float)deg;
        if (rank) rank[v] = r;
    }
}

__global__ void k_pr_init(const int32_t *__restrict__ active, const uint32_t *__restrict__ aoff,
                          int64_t n_active, float r0, float *__restrict__ c0) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_active;
         i += (int64_t)gridDim.x * blockDim.x)
        c0[active[i]] = r0 / (float)(aoff[i + 1] - aoff[i]);
}

// Rank of every isolated vertex (or of all vertices when iters == 0).
__global__ void k_pr_fill(const uint32_t *__restrict__ nz, int32_t nv, float value, int all,
                          float *__restrict__ rank) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x)
        if (all || !((nz[v >> 5] >> (v & 31)) & 1u)) rank[v] = value;
}

// ---------------------------------------------------------------------------
// Column-blocked gathers.  When the contribution array c is larger than L2,
// every gather c[col[e]] is a DRAM sector.  The columns are then cut into K
// blocks of 2^shift vertices; since every row is sorted, its neighbours in
// block k form one contiguous segment of the row.  Iteration pass k visits
// the segments of block k only (in row order, in equal edge tiles), so its
// gathers hit a 4*2^shift-byte slice of c that stays in L2; the per-row sums
// of the K passes meet in an FP32 accumulator (reductions), and a finishing
// pass turns them into ranks.  Segments: (row vertex, first edge) plus the
// per-block edge prefix, built once per graph and block width.
// ---------------------------------------------------------------------------
constexpr int PRB_BUILD = 256;

// First position in col[lo, hi) whose value is >= key (sorted row).
__device__ __forceinline__ uint32_t row_lower_bound(const int32_t *col, uint32_t lo, uint32_t hi,
                                                    int64_t key) {
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if ((int64_t)__ldg(col + mid) < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Per build block and column block: number of non-empty segments and their edges.
__global__ void __launch_bounds__(PRB_BUILD) k_prb_count(const int32_t *__restrict__ col,
                                                         const uint32_t *__restrict__ aoff,
                                                         int64_t n_active, int shift, int K,
                                                         uint32_t *cnt, uint32_t *es) {
    extern __shared__ uint32_t sh[];                 // [2K]
    for (int k = threadIdx.x; k < 2 * K; k += blockDim.x) sh[k] = 0u;
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)PRB_BUILD + threadIdx.x;
    if (i < n_active) {
        const uint32_t e0 = __ldg(aoff + i), e1 = __ldg(aoff + i + 1);
        uint32_t lo = e0;
        for (int k = 0; k < K && lo < e1; ++k) {
            const uint32_t hi = k + 1 < K ? row_lower_bound(col, lo, e1, (int64_t)(k + 1) << shift) : e1;
            if (hi > lo) {
                atomicAdd(&sh[k], 1u);
                atomicAdd(&sh[K + k], hi - lo);
            }
            lo = hi;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        cnt[(int64_t)k * gridDim.x + blockIdx.x] = sh[k];
        es[(int64_t)k * gridDim.x + blockIdx.x] = sh[K + k];
    }
}

// Writes the segments in (column block, row) order.  cpre/epre: per (k, build
// block) exclusive prefixes of counts and edges within block k; kbase[k]: first
// segment of block k.  Segment j of block k has its edge prefix at pre[j + k].
__global__ void __launch_bounds__(PRB_BUILD) k_prb_fill(const int32_t *__restrict__ col,
                                                        const int32_t *__restrict__ active,
                                                        const uint32_t *__restrict__ aoff,
                                                        int64_t n_active, int shift, int K,
                                                        const uint32_t *cpre, const uint32_t *epre,
                                                        const int64_t *kbase, int32_t *seg_v,
                                                        uint32_t *seg_start, uint32_t *pre) {
    const int64_t i = blockIdx.x * (int64_t)PRB_BUILD + threadIdx.x;
    const bool ok = i < n_active;
    const uint32_t e0 = ok ? __ldg(aoff + i) : 0u, e1 = ok ? __ldg(aoff + i + 1) : 0u;
    const int32_t v = ok ? __ldg(active + i) : 0;
    uint32_t lo = e0;
    for (int k = 0; k < K; ++k) {                    // uniform loop: block scans inside
        uint32_t hi = lo;
        if (ok && lo < e1) hi = k + 1 < K ? row_lower_bound(col, lo, e1, (int64_t)(k + 1) << shift) : e1;
        const uint32_t len = hi - lo;
        uint32_t rc, re, rz, tc, te, tz;
        block_scan3<PRB_BUILD>(len ? 1u : 0u, len, 0u, rc, re, rz, tc, te, tz);
        if (len) {
            const int64_t pos = kbase[k] + cpre[(int64_t)k * gridDim.x + blockIdx.x] + rc;
            seg_v[pos] = v;
            seg_start[pos] = lo;
            pre[pos + k] = epre[(int64_t)k * gridDim.x + blockIdx.x] + re;
        }
        lo = hi;
    }
}

__global__ void k_prb_sentinels(const int64_t *kbase, const uint32_t *kedges, int K, uint32_t *pre) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x)
        pre[kbase[k + 1] + k] = kedges[k];
}

// Tile t of block k: first segment and segment count (searching the prefix).
__global__ void k_prb_tiles(const uint32_t *pre, const int64_t *kbase, const uint32_t *kedges,
                            const int64_t *tbase, int K, int2 *tiles) {
    const int64_t total = tbase[K];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int k = 0;
        while (tbase[k + 1] <= t) ++k;
        const uint32_t *pk = pre + kbase[k] + k;
        const int64_t nseg = kbase[k + 1] - kbase[k];
        const uint64_t e0 = (uint64_t)(t - tbase[k]) * PR_TILE;
        const uint64_t e1 = min((uint64_t)kedges[k], e0 + PR_TILE);
        const int64_t j0 = upper_index(pk, nseg, (uint32_t)e0);
        const int64_t j1 = upper_index(pk, nseg, (uint32_t)(e1 - 1));
        tiles[t] = make_int2((int)j0, (int)min(j1 - j0 + 1, (int64_t)PR_TILE + 1));
    }
}

struct PrbSmem {
    uint32_t qe[PR_TILE + 2];
    uint32_t st[PR_TILE + 1];
    int32_t vv[PR_TILE + 1];
    float acc[PR_TILE + 1];
    uint16_t rid[PR_TILE];
    int wmax[PR_BLOCK / 32];
};

// Pass k of an iteration: per tile of block k's segment edges, sum
// c_in[col[e]] per segment (rows by scatter + max-scan, then all of a
// thread's loads in flight), then add each segment's sum to its row's
// accumulator.
__global__ void __launch_bounds__(PR_BLOCK) k_prb_pass(const int32_t *__restrict__ col,
                                                       const int32_t *__restrict__ seg_v,
                                                       const uint32_t *__restrict__ seg_start,
                                                       const uint32_t *__restrict__ pre, uint32_t E_k,
                                                       const int2 *__restrict__ tiles,
                                                       const float *__restrict__ c_in,
                                                       float *__restrict__ acc_g) {
    __shared__ PrbSmem sm;
    const uint64_t e0 = (uint64_t)blockIdx.x * PR_TILE;
    const uint64_t e1 = min((uint64_t)E_k, e0 + PR_TILE);
    const int len = (int)(e1 - e0);
    const int2 tr = __ldg(tiles + blockIdx.x);
    const int64_t j0 = tr.x;
    const int n = tr.y;
    for (int j = threadIdx.x; j <= n; j += PR_BLOCK) {
        sm.qe[j] = __ldg(pre + j0 + j);
        if (j < n) {
            sm.st[j] = __ldg(seg_start + j0 + j);
            sm.vv[j] = __ldg(seg_v + j0 + j);
            sm.acc[j] = 0.f;
        }
    }
    __syncthreads();
    int row[PR_ITEMS];
    block_tile_rows(sm.rid, sm.wmax, sm.qe, (uint32_t)e0, n, len, row);
    const int t0 = threadIdx.x * PR_ITEMS;
    int32_t u[PR_ITEMS];
#pragma unroll
    for (int k = 0; k < PR_ITEMS; ++k) {
        const uint32_t e = (uint32_t)(e0 + t0 + k);
        u[k] = t0 + k < len ? __ldg(col + sm.st[row[k]] + (e - sm.qe[row[k]])) : -1;
    }
    float g[PR_ITEMS];
#pragma unroll
    for (int k = 0; k < PR_ITEMS; ++k) g[k] = u[k] >= 0 ? __ldg(c_in + u[k]) : 0.f;
    add_runs(sm.acc, row, g, len - t0);
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += PR_BLOCK)
        if (sm.acc[j] != 0.f) atomicAdd(acc_g + sm.vv[j], sm.acc[j]);
}

// Ranks of the non-isolated vertices from the accumulated sums; clears them.
__global__ void k_prb_finish(const int32_t *__restrict__ active, const uint32_t *__restrict__ aoff,
                             int64_t n_active, float *__restrict__ acc_g, float *__restrict__ c_out,
                             float *__restrict__ rank, float base, float d) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_active;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = active[i];
        const float r = base + d * acc_g[v];
        acc_g[v] = 0.f;
        c_out[v] = r / (float)(aoff[i + 1] - aoff[i]);
        if (rank) rank[v] = r;
    }
}

// Builds the column-blocked segments of g for blocks of 2^shift vertices.
grx_status prb_build(grx_graph *g, int shift, cudaStream_t s) {
    const int64_t B = 1ll << shift;
    const int K = (int)((g->nv + B - 1) / B);
    const int64_t nb = (g->n_active + PRB_BUILD - 1) / PRB_BUILD;
    g->prb_K = 0;
    if (K < 2 || K > GRX_PRB_MAX_K || nb == 0) return GRX_OK;
    const size_t nkb = (size_t)K * (size_t)nb;
    uint32_t *cnt = (uint32_t *)grx_ctx_alloc(g->ctx, nkb * 4, s);
    uint32_t *es = (uint32_t *)grx_ctx_alloc(g->ctx, nkb * 4, s);
    int64_t *dk = (int64_t *)grx_ctx_alloc(g->ctx, (size_t)(3 * K + 3) * 8, s);
    if (!cnt || !es || !dk) return grx_fail(GRX_ENOMEM, "pagerank: column-block build allocation failed");
    k_prb_count<<<(unsigned)nb, PRB_BUILD, (size_t)2 * K * 4, s>>>(g->col, g->aoff, g->n_active, shift, K,
                                                                  cnt, es);
    std::vector<uint32_t> hc(nkb), he(nkb);
    GRX_CUDA(cudaMemcpyAsync(hc.data(), cnt, nkb * 4, cudaMemcpyDeviceToHost, s));
    GRX_CUDA(cudaMemcpyAsync(he.data(), es, nkb * 4, cudaMemcpyDeviceToHost, s));
    GRX_CUDA(cudaStreamSynchronize(s));
    int64_t kbase[GRX_PRB_MAX_K + 1], tbase[GRX_PRB_MAX_K + 1];
    uint32_t kedges[GRX_PRB_MAX_K];
    kbase[0] = 0;
    tbase[0] = 0;
    for (int k = 0; k < K; ++k) {
        uint64_t c = 0, e = 0;
        for (int64_t b = 0; b < nb; ++b) {
            const size_t x = (size_t)k * nb + b;
            const uint32_t cc = hc[x], ee = he[x];
            hc[x] = (uint32_t)c;
            he[x] = (uint32_t)e;
            c += cc;
            e += ee;
        }
        kbase[k + 1] = kbase[k] + (int64_t)c;
        kedges[k] = (uint32_t)e;
        tbase[k + 1] = tbase[k] + (int64_t)((e + PR_TILE - 1) / PR_TILE);
    }
    const int64_t nseg = kbase[K];
    int32_t *seg_v = (int32_t *)grx_alloc(g, (size_t)nseg * 4 + 16, s);
    uint32_t *seg_start = (uint32_t *)grx_alloc(g, (size_t)nseg * 4 + 16, s);
    uint32_t *pre = (uint32_t *)grx_alloc(g, (size_t)(nseg + K) * 4 + 16, s);
    int2 *tiles = (int2 *)grx_alloc(g, (size_t)tbase[K] * 8 + 16, s);
    if (!seg_v || !seg_start || !pre || !tiles)
        return grx_fail(GRX_ENOMEM, "pagerank: column-block segment allocation failed");
    std::vector<int64_t> hk((size_t)(3 * K + 3));
    for (int k = 0; k <= K; ++k) {
        hk[(size_t)k] = kbase[k];
        hk[(size_t)(K + 1 + k)] = tbase[k];
    }
    for (int k = 0; k < K; ++k) hk[(size_t)(2 * K + 2 + k)] = kedges[k];
    GRX_CUDA(cudaMemcpyAsync(cnt, hc.data(), nkb * 4, cudaMemcpyHostToDevice, s));
    GRX_CUDA(cudaMemcpyAsync(es, he.data(), nkb * 4, cudaMemcpyHostToDevice, s));
    GRX_CUDA(cudaMemcpyAsync(dk, hk.data(), hk.size() * 8, cudaMemcpyHostToDevice, s));
    // kedges as uint32 for the kernels, packed after the int64 tables
    uint32_t *dke = (uint32_t *)(dk + 2 * K + 2);
    std::vector<uint32_t> hke(kedges, kedges + K);
    GRX_CUDA(cudaMemcpyAsync(dke, hke.data(), (size_t)K * 4, cudaMemcpyHostToDevice, s));
    k_prb_fill<<<(unsigned)nb, PRB_BUILD, 0, s>>>(g->col, g->active, g->aoff, g->n_active, shift, K, cnt, es,
                                                  dk, seg_v, seg_start, pre);
    k_prb_sentinels<<<1, 256, 0, s>>>(dk, dke, K, pre);
    if (tbase[K] > 0) {
        const int64_t blocks = (tbase[K] + 255) / 256 < 65536 ? (tbase[K] + 255) / 256 : 65536;
        k_prb_tiles<<<(unsigned)blocks, 256, 0, s>>>(pre, dk, dke, dk + K + 1, K, tiles);
    }
    GRX_CUDA(cudaGetLastError());
    GRX_CUDA(cudaStreamSynchronize(s));    // host tables above are locals
    grx_ctx_free(g->ctx, cnt, nkb * 4, s);
    grx_ctx_free(g->ctx, es, nkb * 4, s);
    grx_ctx_free(g->ctx, dk, (size_t)(3 * K + 3) * 8, s);
    g->prb_seg_v = seg_v;
    g->prb_seg_start = seg_start;
    g->prb_pre = pre;
    g->prb_tiles = tiles;
    for (int k = 0; k <= K; ++k) {
        g->prb_kbase[k] = kbase[k];
        g->prb_tbase[k] = tbase[k];
    }
    for (int k = 0; k < K; ++k) g->prb_kedges[k] = kedges[k];
    g->prb_K = K;
    g->prb_shift = shift;
    return GRX_OK;
}

}  // namespace

grx_status grx_pr_launch(grx_graph *g, float damping, int iters, float *rank, cudaStream_t s) {
    const int64_t ntiles = (g->ne + PR_TILE - 1) / PR_TILE;
    if (!g->pr_c[0]) {
        g->pr_c[0] = (float *)grx_alloc(g, (size_t)g->nv * 4, s);
        g->pr_c[1] = (float *)grx_alloc(g, (size_t)g->nv * 4, s);
        g->pr_s = (float *)grx_alloc(g, (size_t)g->nv * 4, s);
        g->pr_fix = (int32_t *)grx_alloc(g, (size_t)(ntiles > 0 ? ntiles : 1) * 4, s);
        if (!g->pr_c[0] || !g->pr_c[1] || !g->pr_s || !g->pr_fix)
            return grx_fail(GRX_ENOMEM, "pagerank: workspace allocation failed");
        GRX_CUDA(cudaMemsetAsync(g->pr_s, 0, (size_t)g->nv * 4, s));
    }
    // column blocks only when asked for: on GB300 at R-MAT scale 26 the
    // unblocked gathers (22.5 ms per iteration) beat 2^21..2^25-vertex
    // blocks (32..38 ms), the extra segment reads and reductions costing
    // more than the DRAM sectors the L2-resident slices save
    const int want = g->pr_shift_req > 0 ? g->pr_shift_req : -1;
    bool blocked = false;
    if (want > 0 && g->ne > 0 && ((int64_t)g->nv >> want) >= 1) {
        if (!(g->prb_K >= 2 && g->prb_shift == want)) {
            grx_status st = prb_build(g, want, s);
            if (st != GRX_OK) return st;
        }
        blocked = g->prb_K >= 2 && g->prb_shift == want;
    }
    const double N = (double)g->nv;
    const double d = (double)damping;
    const int64_t n_iso = (int64_t)g->nv - g->n_active;
    const int fill_blocks = (int)((g->nv + 255) / 256 < 8192 ? (g->nv + 255) / 256 : 8192);
    if (iters == 0) {
        k_pr_fill<<<fill_blocks, 256, 0, s>>>(g->nz_bits, g->nv, (float)(1.0 / N), 1, rank);
        GRX_CUDA(cudaGetLastError());
        return GRX_OK;
    }
    // Scalar recurrence of the isolated vertices' rank (all equal).
    std::vector<float> base((size_t)iters);
    double riso = 1.0 / N;
    for (int i = 0; i < iters; ++i) {
        const double D = (double)n_iso * riso;
        const double b = (1.0 - d) / N + d * D / N;
        base[(size_t)i] = (float)b;
        riso = b;
    }
    const int init_blocks = (int)((g->n_active + 255) / 256 < 8192 ? (g->n_active + 255) / 256 : 8192);
    if (g->n_active > 0)
        k_pr_init<<<init_blocks > 0 ? init_blocks : 1, 256, 0, s>>>(g->active, g->aoff, g->n_active,
                                                                  (float)(1.0 / N), g->pr_c[0]);
    const int fix_blocks = (int)((ntiles + 255) / 256 > 0 ? (ntiles + 255) / 256 : 1);
    const int2 *tiles = nullptr;
    if (ntiles > 0 && !blocked) {
        grx_status st = grx_edge_tiles(g, PR_TILE, s, &tiles);
        if (st != GRX_OK) return st;
    }
    for (int i = 0; i < iters && ntiles > 0; ++i) {
        const float *c_in = g->pr_c[i & 1];
        float *c_out = g->pr_c[(i + 1) & 1];
        float *r_out = i == iters - 1 ? rank : nullptr;
        if (blocked) {
            for (int k = 0; k < g->prb_K; ++k) {
                const int64_t nt = g->prb_tbase[k + 1] - g->prb_tbase[k];
                if (nt == 0) continue;
                const int64_t kb = g->prb_kbase[k];
                k_prb_pass<<<(unsigned)nt, PR_BLOCK, 0, s>>>(g->col, g->prb_seg_v + kb, g->prb_seg_start + kb,
                                                            g->prb_pre + kb + k, g->prb_kedges[k],
                                                            g->prb_tiles + g->prb_tbase[k], c_in, g->pr_s);
            }
            k_prb_finish<<<init_blocks > 0 ? init_blocks : 1, 256, 0, s>>>(
                g->active, g->aoff, g->n_active, g->pr_s, c_out, r_out, base[(size_t)i], damping);
        } else {
            k_pr_iter<<<(unsigned)ntiles, PR_BLOCK, 0, s>>>(g->col, g->active, g->aoff, tiles, g->ne, c_in,
                                                           c_out, g->pr_s, g->pr_fix, r_out,
                                                           base[(size_t)i], damping);
            k_pr_fixup<<<fix_blocks, 256, 0, s>>>(g->pr_fix, ntiles, g->ro, g->off64, g->pr_s, c_out, r_out,
                                                  base[(size_t)i], damping);
        }
    }
    k_pr_fill<<<fill_blocks, 256, 0, s>>>(g->nz_bits, g->nv, (float)riso, 0, rank);
    GRX_CUDA(cudaGetLastError());
    return GRX_OK;
}
