// Device twins of the seeded input generators (R-MAT edges, symmetric edge
// weights).  They reproduce the host generators of the inputs module bit for
// bit: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used counter-style,
// draw n of stream s = mix64(s + (n + 1) * 0x9E3779B97F4A7C15).
#include "grx_internal.cuh"

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t draw(uint64_t seed, uint64_t n) {
    return mix64(seed + (n + 1) * 0x9E3779B97F4A7C15ull);
}

__global__ void k_rmat(int scale, int64_t m, uint64_t seed, uint64_t t0, uint64_t t1, uint64_t t2,
                       int32_t *u_out, int32_t *v_out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t u = 0, v = 0;
        const uint64_t base = (uint64_t)i * (uint64_t)scale;
        for (int l = 0; l < scale; ++l) {
            const uint64_t r = draw(seed, base + l) >> 11;
            const uint32_t bu = r >= t1;                       // quadrant C or D
            const uint32_t bv = (r >= t0 && r < t1) || r >= t2;  // quadrant B or D
            u |= bu << (scale - 1 - l);
            v |= bv << (scale - 1 - l);
        }
        u_out[i] = (int32_t)u;
        v_out[i] = (int32_t)v;
    }
}

__global__ void k_weights(int64_t nv, int64_t ne, const int64_t *ro, const int32_t *col,
                          uint32_t wmax, uint64_t seed, uint32_t *w) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nv;
         r += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t e = ro[r]; e < ro[r + 1]; ++e) {
            const uint64_t c = (uint64_t)col[e];
            const uint64_t lo = (uint64_t)r < c ? (uint64_t)r : c;
            const uint64_t hi = (uint64_t)r < c ? c : (uint64_t)r;
            w[e] = (uint32_t)(1 + draw(seed, lo * (uint64_t)nv + hi) % wmax);
        }
    }
}

// Grid lattice: horizontal edge (x,y)-(x+1,y) has id y*(w-1)+x, vertical edge
// (x,y)-(x,y+1) has id h*(w-1) + y*w + x; the edge is deleted when the top 53
// bits of draw(seed, id) are below t_del.  Writes (u, v) for every potential
// edge and keep[id] = 1 for the kept ones.
__global__ void k_grid(int64_t w, int64_t h, uint64_t seed, uint64_t t_del, int32_t *u_out,
                       int32_t *v_out, uint8_t *keep) {
    const int64_t nh = h * (w - 1), total = nh + (h - 1) * w;
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        int64_t a, b;
        if (id < nh) {
            const int64_t y = id / (w - 1), x = id - y * (w - 1);
            a = y * w + x;
            b = a + 1;
        } else {
            const int64_t r = id - nh, y = r / w, x = r - y * w;
            a = y * w + x;
            b = a + w;
        }
        u_out[id] = (int32_t)a;
        v_out[id] = (int32_t)b;
        keep[id] = (draw(seed, (uint64_t)id) >> 11) >= t_del ? 1 : 0;
    }
}

}  // namespace

extern "C" grx_status grx_grid_edges(int64_t width, int64_t height, uint64_t seed, uint64_t t_del,
                                     int32_t *u_out, int32_t *v_out, uint8_t *keep_out, void *stream) {
    if (width < 1 || height < 1 || width * height >= (1ll << 31) || !u_out || !v_out || !keep_out)
        return grx_fail(GRX_EINVAL, "grx_grid_edges: bad argument");
    const int64_t total = height * (width - 1) + (height - 1) * width;
    if (total == 0) return GRX_OK;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    k_grid<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(width, height, seed, t_del, u_out, v_out,
                                                              keep_out);
    GRX_CUDA(cudaGetLastError());
    return GRX_OK;
}

extern "C" grx_status grx_rmat_edges(int scale, int64_t m, uint64_t seed, uint64_t t0, uint64_t t1,
                                     uint64_t t2, int32_t *u_out, int32_t *v_out, void *stream) {
    if (scale < 1 || scale > 30) return grx_fail(GRX_EINVAL, "grx_rmat_edges: scale must be in 1..30");
    if (m < 0 || !u_out || !v_out) return grx_fail(GRX_EINVAL, "grx_rmat_edges: bad output");
    if (!(t0 <= t1 && t1 <= t2 && t2 <= (1ull << 53)))
        return grx_fail(GRX_EINVAL, "grx_rmat_edges: thresholds must be ordered and <= 2^53");
    if (m == 0) return GRX_OK;
    int64_t blocks = (m + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    k_rmat<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(scale, m, seed, t0, t1, t2, u_out, v_out);
    GRX_CUDA(cudaGetLastError());
    return GRX_OK;
}

extern "C" grx_status grx_edge_weights(int64_t nv, int64_t ne, const int64_t *row_offsets,
                                       const int32_t *col_indices, uint32_t wmax, uint64_t seed,
                                       uint32_t *w_out, void *stream) {
    if (nv < 1 || ne < 0 || !row_offsets || (ne && (!col_indices || !w_out)) || wmax < 1)
        return grx_fail(GRX_EINVAL, "grx_edge_weights: bad argument");
    if (ne == 0) return GRX_OK;
    int64_t blocks = (nv + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    k_weights<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(nv, ne, row_offsets, col_indices, wmax,
                                                                 seed, w_out);
    GRX_CUDA(cudaGetLastError());
    return GRX_OK;
}
