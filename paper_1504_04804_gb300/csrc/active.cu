// The active list: non-isolated vertices in increasing id order with their row
// starts.  Because isolated rows hold no edges, the active list's edge
// prefix equals the CSR offsets, so "every vertex's edges" frontiers (CC
// hooking, PageRank gathers) reuse the load-balanced tile machinery with a
// bounded number of rows per tile.
#include <cstdlib>
#include <vector>

#include "grx_internal.cuh"

namespace {

constexpr int ACT_BLOCK = 256;
constexpr int ACT_WORDS_PER_THREAD = 4;
constexpr int ACT_WORDS_PER_BLOCK = ACT_BLOCK * ACT_WORDS_PER_THREAD;

__global__ void k_block_popcounts(const uint32_t *bits, int64_t words, uint32_t *bsum) {
    int64_t w0 = (int64_t)blockIdx.x * ACT_WORDS_PER_BLOCK + threadIdx.x * ACT_WORDS_PER_THREAD;
    uint32_t c = 0;
    for (int k = 0; k < ACT_WORDS_PER_THREAD; ++k)
        if (w0 + k < words) c += __popc(bits[w0 + k]);
    c = warp_sum(c);
    __shared__ uint32_t ws[ACT_BLOCK / 32];
    if (lane_id() == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < ACT_BLOCK / 32; ++i) t += ws[i];
        bsum[blockIdx.x] = t;
    }
}

template <typename OffT>
__global__ void k_fill_active(const uint32_t *bits, int64_t words, const uint32_t *bprefix,
                              const OffT *ro, int32_t *active, uint32_t *aoff) {
    int64_t w0 = (int64_t)blockIdx.x * ACT_WORDS_PER_BLOCK + threadIdx.x * ACT_WORDS_PER_THREAD;
    uint32_t wb[ACT_WORDS_PER_THREAD];
    uint32_t c = 0;
    for (int k = 0; k < ACT_WORDS_PER_THREAD; ++k) {
        wb[k] = w0 + k < words ? bits[w0 + k] : 0u;
        c += __popc(wb[k]);
    }
    // block-wide exclusive scan of the per-thread counts
    uint32_t x = c;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(GRX_FULL_MASK, x, o);
        if (lane_id() >= (unsigned)o) x += y;
    }
    __shared__ uint32_t ws[ACT_BLOCK / 32];
    if (lane_id() == 31) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    uint32_t warp_base = 0;
    for (int i = 0; i < (int)(threadIdx.x >> 5); ++i) warp_base += ws[i];
    uint32_t pos = bprefix[blockIdx.x] + warp_base + x - c;
    for (int k = 0; k < ACT_WORDS_PER_THREAD; ++k) {
        uint32_t b = wb[k];
        while (b) {
            int bit = __ffs(b) - 1;
            b &= b - 1;
            int32_t v = (int32_t)((w0 + k) * 32 + bit);
            active[pos] = v;
            aoff[pos] = (uint32_t)ro[v];
            ++pos;
        }
    }
}

// Row range of every all-edges tile: tile t covers edges [t*tile, (t+1)*tile)
// and active rows [i0, i0 + n).  One thread per tile.
__global__ void k_edge_tiles(const uint32_t *aoff, int64_t n_active, int64_t ne, int tile,
                             int64_t ntiles, int2 *out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntiles;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t e0 = (uint64_t)t * tile;
        const uint64_t e1 = min((uint64_t)ne, e0 + tile);
        const int64_t i0 = upper_index(aoff, n_active, (uint32_t)e0);
        const int64_t i1 = upper_index(aoff, n_active, (uint32_t)(e1 - 1));
        out[t] = make_int2((int)i0, (int)min(i1 - i0 + 1, (int64_t)tile + 1));
    }
}

}  // namespace

grx_status grx_edge_tiles(grx_graph *g, int tile, cudaStream_t s, const int2 **out) {
    const int nslots = (int)(sizeof g->etiles / sizeof g->etiles[0]);
    int slot = -1;
    for (int i = 0; i < nslots; ++i) {
        if (g->etiles[i] && g->etile_size[i] == tile) {
            *out = g->etiles[i];
            return GRX_OK;
        }
        if (!g->etiles[i] && slot < 0) slot = i;
    }
    if (slot < 0) return grx_fail(GRX_EINVAL, "edge tiles: too many tile sizes requested");
    const int64_t ntiles = (g->ne + tile - 1) / tile;
    int2 *p = (int2 *)grx_alloc(g, (size_t)(ntiles > 0 ? ntiles : 1) * sizeof(int2), s);
    if (!p) return grx_fail(GRX_ENOMEM, "edge tiles: allocation failed");
    if (ntiles > 0) {
        int64_t blocks = (ntiles + 255) / 256;
        if (blocks > 65536) blocks = 65536;
        k_edge_tiles<<<(unsigned)blocks, 256, 0, s>>>(g->aoff, g->n_active, g->ne, tile, ntiles, p);
        GRX_CUDA(cudaGetLastError());
    }
    g->etiles[slot] = p;
    g->etile_size[slot] = tile;
    *out = p;
    return GRX_OK;
}

grx_status grx_build_active(grx_graph *g, cudaStream_t s) {
    const int64_t nblocks = (g->words + ACT_WORDS_PER_BLOCK - 1) / ACT_WORDS_PER_BLOCK;
    uint32_t *bsum = (uint32_t *)grx_ctx_alloc(g->ctx, (size_t)nblocks * 4, s);
    if (!bsum) return grx_fail(GRX_ENOMEM, "active list: allocation failed");
    k_block_popcounts<<<(unsigned)nblocks, ACT_BLOCK, 0, s>>>(g->nz_bits, g->words, bsum);
    std::vector<uint32_t> h((size_t)nblocks);
    cudaError_t e = cudaMemcpyAsync(h.data(), bsum, (size_t)nblocks * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        grx_ctx_free(g->ctx, bsum, (size_t)nblocks * 4, s);
        return grx_cuda_fail(e, "active list: block counts");
    }
    uint64_t total = 0;
    for (int64_t i = 0; i < nblocks; ++i) {
        uint32_t c = h[(size_t)i];
        h[(size_t)i] = (uint32_t)total;
        total += c;
    }
    g->n_active = (int64_t)total;
    g->active = (int32_t *)grx_alloc(g, (size_t)total * 4 + 16, s);
    g->aoff = (uint32_t *)grx_alloc(g, (size_t)(total + 1) * 4 + 16, s);
    if (!g->active || !g->aoff) {
        grx_ctx_free(g->ctx, bsum, (size_t)nblocks * 4, s);
        return grx_fail(GRX_ENOMEM, "active list: allocation failed");
    }
    e = cudaMemcpyAsync(bsum, h.data(), (size_t)nblocks * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        grx_ctx_free(g->ctx, bsum, (size_t)nblocks * 4, s);
        return grx_cuda_fail(e, "active list: prefix upload");
    }
    if (g->off64)
        k_fill_active<<<(unsigned)nblocks, ACT_BLOCK, 0, s>>>(g->nz_bits, g->words, bsum,
                                                               (const int64_t *)g->ro, g->active, g->aoff);
    else
        k_fill_active<<<(unsigned)nblocks, ACT_BLOCK, 0, s>>>(g->nz_bits, g->words, bsum,
                                                               (const int32_t *)g->ro, g->active, g->aoff);
    uint32_t ne32 = (uint32_t)g->ne;
    e = cudaMemcpyAsync(g->aoff + total, &ne32, 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // ne32 and h are stack/heap locals
    grx_ctx_free(g->ctx, bsum, (size_t)nblocks * 4, s);
    if (e != cudaSuccess) return grx_cuda_fail(e, "active list: fill");
    return GRX_OK;
}

// ---------------------------------------------------------------------------
// First two neighbours of every row, side by side: the probe a pull step makes
// first for each candidate (its first neighbours in row order) becomes one
// coalesced 8-byte load per candidate instead of a row-offset load followed by
// a scattered column load.  -1 marks a missing neighbour.
// ---------------------------------------------------------------------------
namespace {

template <typename OffT>
__global__ void k_first2(const OffT *ro, const int32_t *col, int64_t nv, int2 *first2) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        const OffT b = ro[v], e = ro[v + 1];
        first2[v] = make_int2(e > b ? col[b] : -1, e > b + 1 ? col[b + 1] : -1);
    }
}

}  // namespace

grx_status grx_build_first2(grx_graph *g, cudaStream_t s) {
    const int64_t nv = g->nv;
    const int blocks = (int)((nv + 255) / 256 < 65536 ? (nv + 255) / 256 : 65536);
    if (g->off64)
        k_first2<int64_t><<<blocks, 256, 0, s>>>((const int64_t *)g->ro, g->col, nv, g->first2);
    else
        k_first2<int32_t><<<blocks, 256, 0, s>>>((const int32_t *)g->ro, g->col, nv, g->first2);
    GRX_CUDA(cudaGetLastError());
    return GRX_OK;
}
