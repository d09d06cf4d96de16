// C ABI of libgrx: contexts, graph loading and validation, workspace, and the
// entry points declared in include/grx.h.  The traversal kernels live in
// bfs.cu, sssp.cu, cc.cu, pagerank.cu and msbfs.cu.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "grx_internal.cuh"

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char t_err[512];

grx_status grx_fail(grx_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof t_err, fmt, ap);
    va_end(ap);
    return st;
}

grx_status grx_cuda_fail(cudaError_t e, const char *what) {
    return grx_fail(e == cudaErrorMemoryAllocation ? GRX_ENOMEM : GRX_ECUDA, "%s: %s (%d)",
                    what, cudaGetErrorString(e), (int)e);
}

extern "C" const char *grx_last_error(void) { return t_err; }

// ---------------------------------------------------------------------------
// allocation
// ---------------------------------------------------------------------------
void *grx_ctx_alloc(grx_ctx *c, size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    if (c->has_alloc) return c->alloc.alloc(bytes, (void *)s, c->alloc.user);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void grx_ctx_free(grx_ctx *c, void *p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    if (bytes == 0) bytes = 16;
    if (c->has_alloc) c->alloc.free(p, bytes, (void *)s, c->alloc.user);
    else cudaFreeAsync(p, s);
}

void *grx_alloc(grx_graph *g, size_t bytes, cudaStream_t s) {
    if (g->nallocs >= (int)(sizeof g->allocs / sizeof g->allocs[0])) return nullptr;
    void *p = grx_ctx_alloc(g->ctx, bytes, s);
    if (p) g->allocs[g->nallocs++] = {p, bytes};
    return p;
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" grx_status grx_ctx_create(const grx_allocator *allocator, grx_ctx **out) {
    if (!out) return grx_fail(GRX_EINVAL, "grx_ctx_create: out is NULL");
    *out = nullptr;
    if (allocator && (!allocator->alloc || !allocator->free))
        return grx_fail(GRX_EINVAL, "grx_ctx_create: allocator needs alloc and free");
    int dev = 0;
    GRX_CUDA(cudaGetDevice(&dev));
    int sms = 0;
    GRX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    grx_ctx *c = (grx_ctx *)calloc(1, sizeof(grx_ctx));
    if (!c) return grx_fail(GRX_ENOMEM, "grx_ctx_create: host allocation failed");
    if (allocator) {
        c->alloc = *allocator;
        c->has_alloc = 1;
    }
    c->device = dev;
    c->num_sms = sms;
    *out = c;
    return GRX_OK;
}

extern "C" grx_status grx_ctx_destroy(grx_ctx *ctx) {
    free(ctx);
    return GRX_OK;
}

// ---------------------------------------------------------------------------
// options
// ---------------------------------------------------------------------------
extern "C" void grx_opts_default(grx_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->direction = GRX_DIR_AUTO;
    o->alpha = 0.01f;
    o->beta = 0.1f;
    o->loop = GRX_LOOP_PERSISTENT;
    o->grid_blocks = 0;
    o->block_threads = 0;
    o->timeout_s = 5.0;
    o->collect_stats = 0;
}

void grx_resolve_opts(const grx_opts *in, grx_opts *out) {
    if (in) *out = *in;
    else grx_opts_default(out);
    if (!(out->timeout_s > 0)) out->timeout_s = 5.0;
}

unsigned long long grx_timeout_ns(const grx_opts *o) {
    double ns = o->timeout_s * 1e9;
    if (ns > 3.6e12) ns = 3.6e12;
    if (ns < 1e3) ns = 1e3;
    return (unsigned long long)ns;
}

// ---------------------------------------------------------------------------
// graph loading
// ---------------------------------------------------------------------------
__global__ void k_offsets_64_to_32(const int64_t *in, int32_t *out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)in[i];
}

__global__ void k_offsets_32_to_64(const int32_t *in, int64_t *out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int64_t)in[i];
}

// Bitmap of vertices with at least one edge.  One thread per 32-vertex word.
template <typename OffT>
__global__ void k_nonzero_bits(const OffT *ro, int32_t nv, uint32_t *bits, int64_t words) {
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words;
         w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = 0;
        int64_t v0 = w * 32;
        for (int k = 0; k < 32; ++k) {
            int64_t v = v0 + k;
            if (v < nv && ro[v + 1] > ro[v]) b |= 1u << k;
        }
        bits[w] = b;
    }
}

// Validation of a CSR on the device: offsets monotone with ro[0] == 0 and
// ro[nv] == ne; columns in range; rows strictly increasing (sorted, no
// duplicates); no self-loops; every edge (u,v) has its reverse (v,u) with the
// same weight.  Counts violations into *bad.
template <typename OffT>
__global__ void k_validate(const OffT *ro, const int32_t *col, const uint32_t *w, int32_t nv,
                           int64_t ne, unsigned long long *bad) {
    unsigned long long local = 0;
    int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (tid == 0 && (ro[0] != 0 || (int64_t)ro[nv] != ne)) ++local;
    for (int64_t v = tid; v < nv; v += stride) {
        int64_t b = ro[v], e = ro[v + 1];
        if (e < b || b < 0 || e > ne) { ++local; continue; }
        for (int64_t i = b; i < e; ++i) {
            int32_t u = col[i];
            if (u < 0 || u >= nv) { ++local; continue; }
            if (u == v) ++local;
            if (i > b && col[i - 1] >= u) ++local;
            // reverse edge by binary search in row u
            int64_t lo = ro[u], hi = ro[u + 1];
            if (hi < lo || lo < 0 || hi > ne) { ++local; continue; }
            bool found = false;
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                int32_t c = col[mid];
                if (c == v) { found = true; lo = mid; break; }
                if (c < v) lo = mid + 1; else hi = mid;
            }
            if (!found) ++local;
            else if (w && w[lo] != w[i]) ++local;
        }
    }
    if (local) atomicAdd(bad, local);
}

extern "C" grx_status graph_load_csr(grx_ctx *ctx, int64_t nv, int64_t ne, const void *row_offsets,
                                     int offsets_are_64bit, const int32_t *col_indices,
                                     const uint32_t *weights, int flags, void *stream,
                                     grx_graph **out) {
    if (!ctx || !out) return grx_fail(GRX_EINVAL, "graph_load_csr: ctx/out is NULL");
    *out = nullptr;
    if (nv < 1 || ne < 0) return grx_fail(GRX_EINVAL, "graph_load_csr: nv must be >= 1, ne >= 0");
    if (nv >= (1ll << 31)) return grx_fail(GRX_ERANGE, "graph_load_csr: nv >= 2^31");
    if (ne >= (1ll << 32)) return grx_fail(GRX_ERANGE, "graph_load_csr: ne >= 2^32");
    if (!row_offsets || (ne > 0 && !col_indices))
        return grx_fail(GRX_EINVAL, "graph_load_csr: NULL row_offsets or col_indices");
    cudaStream_t s = (cudaStream_t)stream;
    const bool dev_in = (flags & GRX_DEVICE_PTRS) != 0;
    const cudaMemcpyKind kind = dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;

    if (!dev_in) {  // cheap host-side checks of the offsets' ends
        int64_t first = offsets_are_64bit ? ((const int64_t *)row_offsets)[0]
                                          : ((const int32_t *)row_offsets)[0];
        int64_t last = offsets_are_64bit ? ((const int64_t *)row_offsets)[nv]
                                         : ((const int32_t *)row_offsets)[nv];
        if (first != 0 || last != ne)
            return grx_fail(GRX_EINVAL, "graph_load_csr: row_offsets[0] must be 0 and "
                                        "row_offsets[nv] must equal ne");
    }

    grx_graph *g = (grx_graph *)calloc(1, sizeof(grx_graph));
    if (!g) return grx_fail(GRX_ENOMEM, "graph_load_csr: host allocation failed");
    g->ctx = ctx;
    g->nv = (int32_t)nv;
    g->ne = ne;
    g->off64 = ne >= (1ll << 31) || (flags & GRX_OFFSETS64) != 0;
    g->last_stream = stream;
    g->words = ((nv + 31) / 32 + 31) / 32 * 32;
    grx_status st = GRX_OK;
    const size_t ro_bytes = (size_t)(nv + 1) * (g->off64 ? 8 : 4);

#define LOAD_FAIL(code, ...)              \
    do {                                  \
        st = grx_fail(code, __VA_ARGS__); \
        goto fail;                        \
    } while (0)

    g->ro = grx_alloc(g, ro_bytes, s);
    g->col = (int32_t *)grx_alloc(g, (size_t)ne * 4, s);
    g->nz_bits = (uint32_t *)grx_alloc(g, (size_t)g->words * 4, s);
    if (weights) g->w = (uint32_t *)grx_alloc(g, (size_t)ne * 4, s);
    if (!g->ro || !g->col || !g->nz_bits || (weights && !g->w))
        LOAD_FAIL(GRX_ENOMEM, "graph_load_csr: device allocation of %zu bytes failed",
                  ro_bytes + (size_t)ne * 8);
    {
        const bool in64 = offsets_are_64bit != 0;
        if (in64 == (bool)g->off64) {
            if (cudaMemcpyAsync(g->ro, row_offsets, ro_bytes, kind, s) != cudaSuccess)
                LOAD_FAIL(GRX_ECUDA, "graph_load_csr: copy of row_offsets failed");
        } else {
            // stage the caller's offsets on the device, then convert
            size_t in_bytes = (size_t)(nv + 1) * (in64 ? 8 : 4);
            void *tmp = grx_ctx_alloc(ctx, in_bytes, s);
            if (!tmp) LOAD_FAIL(GRX_ENOMEM, "graph_load_csr: staging allocation failed");
            if (cudaMemcpyAsync(tmp, row_offsets, in_bytes, kind, s) != cudaSuccess) {
                grx_ctx_free(ctx, tmp, in_bytes, s);
                LOAD_FAIL(GRX_ECUDA, "graph_load_csr: copy of row_offsets failed");
            }
            int blocks = (int)((nv + 1 + 255) / 256);
            if (blocks > 4096) blocks = 4096;
            if (in64) k_offsets_64_to_32<<<blocks, 256, 0, s>>>((const int64_t *)tmp, (int32_t *)g->ro, nv + 1);
            else k_offsets_32_to_64<<<blocks, 256, 0, s>>>((const int32_t *)tmp, (int64_t *)g->ro, nv + 1);
            grx_ctx_free(ctx, tmp, in_bytes, s);
        }
        if (ne > 0 && cudaMemcpyAsync(g->col, col_indices, (size_t)ne * 4, kind, s) != cudaSuccess)
            LOAD_FAIL(GRX_ECUDA, "graph_load_csr: copy of col_indices failed");
        if (weights && ne > 0 &&
            cudaMemcpyAsync(g->w, weights, (size_t)ne * 4, kind, s) != cudaSuccess)
            LOAD_FAIL(GRX_ECUDA, "graph_load_csr: copy of weights failed");
        cudaMemsetAsync(g->nz_bits, 0, (size_t)g->words * 4, s);
        int blocks = (int)((g->words + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        if (g->off64) k_nonzero_bits<<<blocks, 256, 0, s>>>((const int64_t *)g->ro, g->nv, g->nz_bits, g->words);
        else k_nonzero_bits<<<blocks, 256, 0, s>>>((const int32_t *)g->ro, g->nv, g->nz_bits, g->words);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) LOAD_FAIL(GRX_ECUDA, "graph_load_csr: %s", cudaGetErrorString(e));
    }
    if (flags & GRX_VALIDATE) {
        unsigned long long *bad = (unsigned long long *)grx_ctx_alloc(ctx, 8, s);
        if (!bad) LOAD_FAIL(GRX_ENOMEM, "graph_load_csr: validation allocation failed");
        cudaMemsetAsync(bad, 0, 8, s);
        int blocks = ctx->num_sms * 8;
        if (g->off64) k_validate<<<blocks, 256, 0, s>>>((const int64_t *)g->ro, g->col, g->w, g->nv, ne, bad);
        else k_validate<<<blocks, 256, 0, s>>>((const int32_t *)g->ro, g->col, g->w, g->nv, ne, bad);
        unsigned long long h_bad = 0;
        cudaError_t e = cudaMemcpyAsync(&h_bad, bad, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        grx_ctx_free(ctx, bad, 8, s);
        if (e != cudaSuccess) LOAD_FAIL(GRX_ECUDA, "graph_load_csr: validation: %s", cudaGetErrorString(e));
        if (h_bad) LOAD_FAIL(GRX_EINVAL, "graph_load_csr: %llu CSR violations (offsets, column "
                             "range, sorting, self-loops or symmetry)", h_bad);
    }
    if ((st = grx_build_active(g, s)) != GRX_OK) goto fail;
    *out = g;
    return GRX_OK;
fail:
    for (int i = 0; i < g->nallocs; ++i) grx_ctx_free(ctx, g->allocs[i].p, g->allocs[i].n, s);
    free(g);
    return st;
#undef LOAD_FAIL
}

extern "C" grx_status graph_free(grx_graph *g) {
    if (!g) return GRX_OK;
    cudaStream_t s = (cudaStream_t)g->last_stream;
    for (int i = 0; i < 2; ++i)
        if (g->bfs_gexec[i]) {
            cudaStreamSynchronize(s);
            cudaGraphExecDestroy(g->bfs_gexec[i]);
        }
    for (int i = g->nallocs - 1; i >= 0; --i) grx_ctx_free(g->ctx, g->allocs[i].p, g->allocs[i].n, s);
    free(g);
    return GRX_OK;
}

extern "C" grx_status grx_graph_info(const grx_graph *g, int64_t *nv, int64_t *ne) {
    if (!g) return grx_fail(GRX_EINVAL, "grx_graph_info: NULL graph");
    if (nv) *nv = g->vid64 ? g->nv64 : g->nv;
    if (ne) *ne = g->ne;
    return GRX_OK;
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
grx_status grx_ensure_workspace(grx_graph *g, cudaStream_t s) {
    if (g->ws_ready) return GRX_OK;
    const size_t nv = (size_t)g->nv;
    const size_t wb = (size_t)g->words * 4;
    g->visited = (uint32_t *)grx_alloc(g, wb, s);
    for (int i = 0; i < 3; ++i) {
        g->fbits[i] = (uint32_t *)grx_alloc(g, wb, s);
        g->qv[i] = (int32_t *)grx_alloc(g, nv * 4, s);
        g->qe[i] = (uint32_t *)grx_alloc(g, nv * 4, s);
        g->qr[i] = grx_alloc(g, nv * (g->off64 ? 8 : 4), s);
    }
    for (int i = 0; i < 2; ++i) g->ulist[i] = (int32_t *)grx_alloc(g, nv * 4, s);
    g->first2 = (int2 *)grx_alloc(g, nv * sizeof(int2), s);
    g->ctl = (TravCtl *)grx_alloc(g, sizeof(TravCtl), s);
    g->bar_flags = (unsigned int *)grx_alloc(g, sizeof(unsigned int) * GRX_MAX_GRID, s);
    g->stats = (DevStats *)grx_alloc(g, sizeof(DevStats), s);
    g->stamp = (int32_t *)grx_alloc(g, nv * 4, s);
    bool ok = g->visited && g->ctl && g->bar_flags && g->stats && g->stamp && g->first2;
    for (int i = 0; i < 3; ++i) ok = ok && g->fbits[i] && g->qv[i] && g->qe[i] && g->qr[i];
    for (int i = 0; i < 2; ++i) ok = ok && g->ulist[i];
    if (!ok) return grx_fail(GRX_ENOMEM, "traversal workspace allocation failed (nv=%d)", g->nv);
    GRX_CUDA(cudaMemsetAsync(g->ctl, 0, sizeof(TravCtl), s));
    GRX_CUDA(cudaMemsetAsync(g->stats, 0, sizeof(DevStats), s));
    grx_status st = grx_build_first2(g, s);
    if (st != GRX_OK) return st;
    g->ws_ready = 1;
    return GRX_OK;
}

grx_status grx_ensure_ms_workspace(grx_graph *g, cudaStream_t s) {
    grx_status st = grx_ensure_workspace(g, s);
    if (st != GRX_OK) return st;
    if (g->ms_ready) return GRX_OK;
    const size_t b = (size_t)g->nv * 8;
    for (int i = 0; i < 3; ++i) g->ms_cur[i] = (unsigned long long *)grx_alloc(g, b, s);
    g->ms_next = (unsigned long long *)grx_alloc(g, b, s);
    g->ms_seen = (unsigned long long *)grx_alloc(g, b, s);
    if (!g->ms_cur[0] || !g->ms_cur[1] || !g->ms_cur[2] || !g->ms_next || !g->ms_seen)
        return grx_fail(GRX_ENOMEM, "multi-source workspace allocation failed (nv=%d)", g->nv);
    g->ms_ready = 1;
    return GRX_OK;
}

// Bytes grx_ensure_workspace / grx_ensure_ms_workspace would allocate now.
static size_t workspace_new_bytes(const grx_graph *g, bool multi) {
    const size_t nv = (size_t)g->nv, wb = (size_t)g->words * 4;
    size_t b = 0;
    if (!g->ws_ready)
        b += wb + 3 * (wb + nv * 8 + nv * (g->off64 ? 8 : 4)) + 2 * nv * 4 + nv * sizeof(int2) +
             sizeof(TravCtl) + sizeof(unsigned int) * GRX_MAX_GRID + sizeof(DevStats) + nv * 4;
    if (multi && !g->ms_ready) b += 5 * nv * 8;
    return b;
}

extern "C" grx_status grx_multi_footprint(const grx_graph *g, int kind, size_t *bytes_out) {
    if (!g || !bytes_out) return grx_fail(GRX_EINVAL, "grx_multi_footprint: NULL argument");
    if (g->vid64) return grx_fail(GRX_EINVAL, "grx_multi_footprint: 64-bit vertex ids are served by bfs64 only");
    if (kind != GRX_KIND_BFS && kind != GRX_KIND_SSSP)
        return grx_fail(GRX_EINVAL, "grx_multi_footprint: bad kind %d", kind);
    *bytes_out = workspace_new_bytes(g, true) +
                 (kind == GRX_KIND_BFS ? grx_msbfs_new_bytes(g) : grx_mssp_new_bytes(g));
    return GRX_OK;
}

extern "C" grx_status grx_graph_status(grx_graph *g, void *stream) {
    if (!g) return grx_fail(GRX_EINVAL, "grx_graph_status: NULL graph");
    cudaStream_t s = (cudaStream_t)stream;
    GRX_CUDA(cudaStreamSynchronize(s));
    if (!g->ws_ready && !g->ws64_ready) return GRX_OK;
    int st = 0;
    GRX_CUDA(cudaMemcpy(&st, &g->ctl->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        GRX_CUDA(cudaMemset(&g->ctl->status, 0, sizeof(int)));
        return grx_fail((grx_status)st, "device-side status %d from the last traversal", st);
    }
    return GRX_OK;
}

extern "C" grx_status grx_last_stats(grx_graph *g, void *stream, grx_trav_stats *out) {
    if (!g || !out) return grx_fail(GRX_EINVAL, "grx_last_stats: NULL argument");
    if (!g->ws_ready) return grx_fail(GRX_EINVAL, "grx_last_stats: no traversal has run");
    GRX_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    DevStats *h = (DevStats *)malloc(sizeof(DevStats));
    if (!h) return grx_fail(GRX_ENOMEM, "grx_last_stats: host allocation failed");
    cudaError_t e = cudaMemcpy(h, g->stats, sizeof(DevStats), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        free(h);
        return grx_cuda_fail(e, "grx_last_stats copy");
    }
    out->levels = h->levels;
    int n = h->levels < GRX_MAX_LEVELS_STATS ? h->levels : GRX_MAX_LEVELS_STATS;
    for (int i = 0; i < GRX_MAX_LEVELS_STATS; ++i) {
        bool in = i < n;
        out->dir[i] = in ? h->dir[i] : 0;
        out->frontier[i] = in ? (int64_t)h->frontier[i] : 0;
        out->edges_examined[i] = in ? (int64_t)h->edges_examined[i] : 0;
        out->vertices_scanned[i] = in ? (int64_t)h->vertices_scanned[i] : 0;
        out->discovered[i] = in ? (int64_t)h->discovered[i] : 0;
        out->level_ns[i] = in && h->level_t0[i + 1] >= h->level_t0[i]
                               ? (int64_t)(h->level_t0[i + 1] - h->level_t0[i]) : 0;
    }
    free(h);
    return GRX_OK;
}

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------
static grx_status check_graph(grx_graph *g, const char *who) {
    if (!g) return grx_fail(GRX_EINVAL, "%s: NULL graph", who);
    if (g->vid64)
        return grx_fail(GRX_EINVAL, "%s: the graph has 64-bit vertex ids (graph_load_csr64); bfs64 "
                                    "traverses it", who);
    return GRX_OK;
}

extern "C" grx_status bfs(grx_graph *g, int32_t src, int32_t *depth_out, int32_t *parent_out,
                          const grx_opts *opts, void *stream) {
    grx_status st = check_graph(g, "bfs");
    if (st) return st;
    if (src < 0 || src >= g->nv) return grx_fail(GRX_EINVAL, "bfs: source %d out of range", src);
    if (!depth_out) return grx_fail(GRX_EINVAL, "bfs: depth_out is NULL");
    grx_opts o;
    grx_resolve_opts(opts, &o);
    if (o.direction < GRX_DIR_AUTO || o.direction > GRX_DIR_PULL)
        return grx_fail(GRX_EINVAL, "bfs: bad direction %d", o.direction);
    g->last_stream = stream;
    if ((st = grx_ensure_workspace(g, (cudaStream_t)stream))) return st;
    return grx_bfs_launch(g, src, depth_out, parent_out, &o, (cudaStream_t)stream);
}

extern "C" grx_status sssp(grx_graph *g, int32_t src, uint32_t *dist_out, const grx_opts *opts,
                           void *stream) {
    grx_status st = check_graph(g, "sssp");
    if (st) return st;
    if (!g->w) return grx_fail(GRX_EINVAL, "sssp: graph has no weights");
    if (src < 0 || src >= g->nv) return grx_fail(GRX_EINVAL, "sssp: source %d out of range", src);
    if (!dist_out) return grx_fail(GRX_EINVAL, "sssp: dist_out is NULL");
    grx_opts o;
    grx_resolve_opts(opts, &o);
    g->last_stream = stream;
    if ((st = grx_ensure_workspace(g, (cudaStream_t)stream))) return st;
    return grx_sssp_launch(g, src, dist_out, &o, (cudaStream_t)stream);
}

extern "C" grx_status cc(grx_graph *g, int32_t *label_out, void *stream) {
    grx_status st = check_graph(g, "cc");
    if (st) return st;
    if (!label_out) return grx_fail(GRX_EINVAL, "cc: label_out is NULL");
    grx_opts o;
    grx_resolve_opts(nullptr, &o);
    g->last_stream = stream;
    if ((st = grx_ensure_workspace(g, (cudaStream_t)stream))) return st;
    return grx_cc_launch(g, label_out, &o, (cudaStream_t)stream);
}

extern "C" grx_status bc(grx_graph *g, const int32_t *srcs_host, int n, double *bc_out, double *sigma_out,
                         const grx_opts *opts, void *stream) {
    grx_status st = check_graph(g, "bc");
    if (st) return st;
    if (!srcs_host || n < 1) return grx_fail(GRX_EINVAL, "bc: need at least one source");
    for (int i = 0; i < n; ++i)
        if (srcs_host[i] < 0 || srcs_host[i] >= g->nv)
            return grx_fail(GRX_EINVAL, "bc: source %d (index %d) out of range", srcs_host[i], i);
    if (!bc_out) return grx_fail(GRX_EINVAL, "bc: bc_out is NULL");
    grx_opts o;
    grx_resolve_opts(opts, &o);
    if (o.direction < GRX_DIR_AUTO || o.direction > GRX_DIR_PULL)
        return grx_fail(GRX_EINVAL, "bc: bad direction %d", o.direction);
    g->last_stream = stream;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = grx_ensure_workspace(g, s))) return st;
    if (!g->bc_sigma) {
        g->bc_sigma = (double *)grx_alloc(g, (size_t)g->nv * 8, s);
        g->bc_acc = (double *)grx_alloc(g, (size_t)g->nv * 8, s);
        g->bc_code = (uint32_t *)grx_alloc(g, (size_t)g->words * 8, s);
        if (!g->bc_sigma || !g->bc_acc || !g->bc_code)
            return grx_fail(GRX_ENOMEM, "bc: workspace allocation failed (nv=%d)", g->nv);
    }
    return grx_bc_launch(g, srcs_host, n, bc_out, sigma_out, &o, s);
}

extern "C" grx_status pagerank(grx_graph *g, float damping, int iters, float *rank_out,
                               void *stream) {
    grx_status st = check_graph(g, "pagerank");
    if (st) return st;
    if (!rank_out) return grx_fail(GRX_EINVAL, "pagerank: rank_out is NULL");
    if (iters < 0) return grx_fail(GRX_EINVAL, "pagerank: iters must be >= 0");
    if (!(damping >= 0.f && damping <= 1.f))
        return grx_fail(GRX_EINVAL, "pagerank: damping must be in [0, 1]");
    g->last_stream = stream;
    if ((st = grx_ensure_workspace(g, (cudaStream_t)stream))) return st;
    return grx_pr_launch(g, damping, iters, rank_out, (cudaStream_t)stream);
}

extern "C" grx_status grx_pagerank_block(grx_graph *g, int shift) {
    grx_status st = check_graph(g, "grx_pagerank_block");
    if (st) return st;
    if (shift > 0 && (shift > 31 || (((int64_t)g->nv + (1ll << shift) - 1) >> shift) > GRX_PRB_MAX_K))
        return grx_fail(GRX_EINVAL, "grx_pagerank_block: 2^%d-vertex blocks give more than %d blocks", shift,
                        GRX_PRB_MAX_K);
    g->pr_shift_req = shift;
    return GRX_OK;
}


static grx_status check_sources(grx_graph *g, const int32_t *srcs, int n, const char *who) {
    if (!srcs) return grx_fail(GRX_EINVAL, "%s: srcs is NULL", who);
    if (n < 1 || n > 64) return grx_fail(GRX_EINVAL, "%s: n must be in 1..64 (got %d)", who, n);
    for (int i = 0; i < n; ++i)
        if (srcs[i] < 0 || srcs[i] >= g->nv)
            return grx_fail(GRX_EINVAL, "%s: source %d (lane %d) out of range", who, srcs[i], i);
    return GRX_OK;
}

extern "C" grx_status bc_multi(grx_graph *g, const int32_t *srcs_host, int n, double *bc_out,
                               const grx_opts *opts, void *stream) {
    grx_status st = check_graph(g, "bc_multi");
    if (st) return st;
    if ((st = check_sources(g, srcs_host, n, "bc_multi"))) return st;
    if (!bc_out) return grx_fail(GRX_EINVAL, "bc_multi: bc_out is NULL");
    grx_opts o;
    grx_resolve_opts(opts, &o);
    g->last_stream = stream;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = grx_ensure_workspace(g, s))) return st;
    if (!g->bcm_sig) {
        const size_t nv = (size_t)g->nv;
        g->bcm_seen = (unsigned long long *)grx_alloc(g, nv * 8, s);
        g->bcm_next = (unsigned long long *)grx_alloc(g, nv * 8, s);
        g->bcm_hist = (unsigned long long *)grx_alloc(g, nv * 8 * GRX_BCM_MAX_LEVELS, s);
        g->bcm_sig = (double *)grx_alloc(g, nv * 64 * 8, s);
        g->bcm_acc = (double *)grx_alloc(g, nv * 64 * 8, s);
        g->bcm_srcs = (int32_t *)grx_alloc(g, 64 * 4, s);
        if (!g->bcm_seen || !g->bcm_next || !g->bcm_hist || !g->bcm_sig || !g->bcm_acc || !g->bcm_srcs)
            return grx_fail(GRX_ENOMEM, "bc_multi: workspace allocation failed (nv=%d)", g->nv);
    }
    return grx_bcm_launch(g, srcs_host, n, bc_out, &o, s);
}

extern "C" grx_status bfs_multi(grx_graph *g, const int32_t *srcs_host, int n, int32_t *depth_out,
                                const grx_opts *opts, void *stream) {
    grx_status st = check_graph(g, "bfs_multi");
    if (st) return st;
    if ((st = check_sources(g, srcs_host, n, "bfs_multi"))) return st;
    if (!depth_out) return grx_fail(GRX_EINVAL, "bfs_multi: depth_out is NULL");
    grx_opts o;
    grx_resolve_opts(opts, &o);
    if (o.direction < GRX_DIR_AUTO || o.direction > GRX_DIR_PULL)
        return grx_fail(GRX_EINVAL, "bfs_multi: bad direction %d", o.direction);
    g->last_stream = stream;
    if ((st = grx_ensure_ms_workspace(g, (cudaStream_t)stream))) return st;
    return grx_msbfs_launch(g, srcs_host, n, depth_out, &o, (cudaStream_t)stream);
}

extern "C" grx_status sssp_multi(grx_graph *g, const int32_t *srcs_host, int n, uint32_t *dist_out,
                                 const grx_opts *opts, void *stream) {
    grx_status st = check_graph(g, "sssp_multi");
    if (st) return st;
    if (!g->w) return grx_fail(GRX_EINVAL, "sssp_multi: graph has no weights");
    if ((st = check_sources(g, srcs_host, n, "sssp_multi"))) return st;
    if (!dist_out) return grx_fail(GRX_EINVAL, "sssp_multi: dist_out is NULL");
    grx_opts o;
    grx_resolve_opts(opts, &o);
    g->last_stream = stream;
    if ((st = grx_ensure_ms_workspace(g, (cudaStream_t)stream))) return st;
    return grx_mssp_launch(g, srcs_host, n, dist_out, &o, (cudaStream_t)stream);
}
