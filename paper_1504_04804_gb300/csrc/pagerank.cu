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
// are computed once per graph and cached).  A tile stages c[col[e]] for its edges in shared memory;
// each thread sums a contiguous run of edges per row and adds its partial to
// the row's shared accumulator.  Rows inside the tile are finished there;
// rows that cross a tile boundary add their partial to a global accumulator
// and are finished by a small fix-up launch.  Accumulation is FP32.
#include <vector>

#include "grx_internal.cuh"

namespace {

constexpr int PR_BLOCK = 256;
constexpr int PR_ITEMS = 9;                  // odd: conflict-free strided smem reads
constexpr int PR_TILE = PR_BLOCK * PR_ITEMS;

struct PrSmem {
    float val[PR_TILE];
    float acc[PR_TILE + 2];
    uint32_t qe[PR_TILE + 2];
    int32_t u[PR_TILE + 2];
};

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
    const int2 tr = __ldg(tiles + tile);
    const int64_t i0 = tr.x;
    const int n = tr.y;
    if (threadIdx.x == 0) fix[tile] = -1;
    for (int j = threadIdx.x; j <= n; j += PR_BLOCK) {   // n+1 prefixes: qe[n] = end of last row
        sm.qe[j] = __ldg(aoff + i0 + j);
        if (j < n) sm.u[j] = __ldg(active + i0 + j);
        sm.acc[j] = 0.f;
    }
    for (int k = threadIdx.x; k < len; k += PR_BLOCK) sm.val[k] = __ldg(c_in + __ldg(col + e0 + k));
    __syncthreads();
    // contiguous run of PR_ITEMS edges per thread
    const int t0 = threadIdx.x * PR_ITEMS;
    if (t0 < len) {
        int j = upper_index_smem(sm.qe, n, (uint32_t)(e0 + t0));
        uint32_t next_start = sm.qe[j + 1];
        float part = 0.f;
        const int t1 = min(len, t0 + PR_ITEMS);
        for (int k = t0; k < t1; ++k) {
            const uint32_t e = (uint32_t)(e0 + k);
            while (e >= next_start) {
                atomicAdd(&sm.acc[j], part);
                part = 0.f;
                ++j;
                next_start = sm.qe[j + 1];
            }
            part += sm.val[k];
        }
        atomicAdd(&sm.acc[j], part);
    }
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
    if (ntiles > 0) {
        grx_status st = grx_edge_tiles(g, PR_TILE, s, &tiles);
        if (st != GRX_OK) return st;
    }
    for (int i = 0; i < iters && ntiles > 0; ++i) {
        const float *c_in = g->pr_c[i & 1];
        float *c_out = g->pr_c[(i + 1) & 1];
        float *r_out = i == iters - 1 ? rank : nullptr;
        k_pr_iter<<<(unsigned)ntiles, PR_BLOCK, 0, s>>>(g->col, g->active, g->aoff, tiles,
                                                       g->ne, c_in, c_out, g->pr_s, g->pr_fix, r_out,
                                                       base[(size_t)i], damping);
        k_pr_fixup<<<fix_blocks, 256, 0, s>>>(g->pr_fix, ntiles, g->ro, g->off64, g->pr_s, c_out, r_out,
                                              base[(size_t)i], damping);
    }
    k_pr_fill<<<fill_blocks, 256, 0, s>>>(g->nz_bits, g->nv, (float)riso, 0, rank);
    GRX_CUDA(cudaGetLastError());
    return GRX_OK;
}
