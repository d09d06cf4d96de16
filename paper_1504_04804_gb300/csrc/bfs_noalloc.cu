// bfs_noalloc: the BFS entry point for callers that cannot allocate device
// memory.
//
// Some programs that embed this library must not call cudaMalloc or any
// allocating routine: a host framework that owns every byte of the GPU through
// its own pool and forbids outside allocations, a latency-critical loop where
// cudaMalloc/cudaFree would implicitly synchronise the device, or a request
// path that may not fail with out-of-memory half-way.  bfs_noalloc serves
// them: the caller passes the CSR arrays and the output arrays (all device
// memory it owns), and every piece of traversal scratch -- frontier queues,
// bitmaps, candidate lists, the control block -- lives in one file-scope
// __device__ array of fixed size, reserved when the library is loaded and held
// by every GPU that loads it until the process exits.
//
// Shared-state rules: every call uses the same array, and the array keeps the
// previous call's contents; each call clears what must start at zero.  Two
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on the array and corrupt each other's results: order them.
#include <mutex>

#include "grx_internal.cuh"

namespace {

constexpr int64_t kMaxNv = GRX_NOALLOC_MAX_NV;
constexpr int64_t kWords = ((kMaxNv + 31) / 32 + 31) / 32 * 32;
constexpr int kMaxDevices = 64;

struct NoallocScratch {
    TravCtl ctl;
    unsigned int bar_flags[GRX_MAX_GRID];
    uint32_t visited[kWords];
    uint32_t fbits[3][kWords];
    uint32_t nz[kWords];
    int32_t qv[3][kMaxNv];
    uint32_t qe[3][kMaxNv];
    int32_t qr[3][kMaxNv];
    int32_t ulist[2][kMaxNv];
};
static_assert(sizeof(NoallocScratch) == GRX_NOALLOC_SCRATCH_BYTES,
              "grx.h states the size of the fixed scratch array");

// Bitmap of vertices with at least one edge (int32 offsets).
__global__ void k_noalloc_nz(const int32_t *ro, int32_t nv, uint32_t *bits, int64_t words) {
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words;
         w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = 0;
        for (int k = 0; k < 32; ++k) {
            int64_t v = w * 32 + k;
            if (v < nv && ro[v + 1] > ro[v]) b |= 1u << k;
        }
        bits[w] = b;
    }
}

}  // namespace

// The scratch array itself.  Host code may not use this symbol as an address:
// the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

namespace {

std::mutex g_setup_mu;
NoallocScratch *g_scratch_addr[kMaxDevices];   // device address per device ordinal
int g_num_sms[kMaxDevices];

// Once per device, with that device current: look up the array's device
// address and the SM count.  Neither call allocates.
grx_status setup_device(int dev, NoallocScratch **out, int *sms) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return grx_cuda_fail(e, "bfs_noalloc: cudaGetSymbolAddress");
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return grx_cuda_fail(e, "bfs_noalloc: SM count");
        g_num_sms[dev] = n;
        g_scratch_addr[dev] = (NoallocScratch *)p;
    }
    *out = g_scratch_addr[dev];
    *sms = g_num_sms[dev];
    return GRX_OK;
}

}  // namespace

extern "C" grx_status bfs_noalloc(int64_t nv, int64_t ne, const int32_t *row_offsets,
                                  const int32_t *col_indices, int32_t src, int32_t *depth_out,
                                  int32_t *parent_out, int32_t *status_out, const grx_opts *opts,
                                  void *stream) {
    if (nv < 1 || nv > kMaxNv)
        return grx_fail(GRX_ERANGE, "bfs_noalloc: nv = %lld is outside 1..%lld (the fixed scratch "
                        "holds at most %lld vertices)", (long long)nv, (long long)kMaxNv,
                        (long long)kMaxNv);
    if (ne < 0 || ne >= (1ll << 31))
        return grx_fail(GRX_ERANGE, "bfs_noalloc: ne must be in 0..2^31-1 (int32 offsets)");
    if (!row_offsets || (ne > 0 && !col_indices) || !depth_out)
        return grx_fail(GRX_EINVAL, "bfs_noalloc: NULL row_offsets, col_indices or depth_out");
    if (src < 0 || src >= nv) return grx_fail(GRX_EINVAL, "bfs_noalloc: source %d out of range", src);
    grx_opts o;
    grx_resolve_opts(opts, &o);
    if (o.collect_stats) return grx_fail(GRX_EINVAL, "bfs_noalloc: collect_stats is not supported");
    // The CUDA-graph level loop instantiates a graph and keeps its arguments
    // in device memory of their own: both would be allocations.
    if (o.loop == GRX_LOOP_GRAPH)
        return grx_fail(GRX_EINVAL, "bfs_noalloc: GRX_LOOP_GRAPH allocates; use the persistent or host loop");
    if (o.loop != GRX_LOOP_PERSISTENT && o.loop != GRX_LOOP_HOST)
        return grx_fail(GRX_EINVAL, "bfs_noalloc: bad loop %d", o.loop);
    if (o.direction < GRX_DIR_AUTO || o.direction > GRX_DIR_PULL)
        return grx_fail(GRX_EINVAL, "bfs_noalloc: bad direction %d", o.direction);
    int dev = 0;
    GRX_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return grx_fail(GRX_ERANGE, "bfs_noalloc: device ordinal %d", dev);
    NoallocScratch *sc = nullptr;
    int sms = 0;
    grx_status st = setup_device(dev, &sc, &sms);
    if (st != GRX_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    // Everything that must start at zero: the control block (counters,
    // barrier, status).  The traversal launcher clears the bitmaps and
    // initialises depth / parent itself.
    GRX_CUDA(cudaMemsetAsync(&sc->ctl, 0, sizeof(TravCtl), s));
    const int64_t words = ((nv + 31) / 32 + 31) / 32 * 32;
    int blocks = (int)((words + 255) / 256);
    k_noalloc_nz<<<blocks, 256, 0, s>>>(row_offsets, (int32_t)nv, sc->nz, words);
    GRX_CUDA(cudaGetLastError());

    // A graph and context view over the caller's arrays and the scratch; the
    // traversal launcher only reads these fields and allocates nothing.
    grx_ctx ctx{};
    ctx.device = dev;
    ctx.num_sms = sms;
    grx_graph g{};
    g.ctx = &ctx;
    g.nv = (int32_t)nv;
    g.ne = ne;
    g.off64 = 0;
    g.ro = (void *)row_offsets;
    g.col = (int32_t *)col_indices;
    g.nz_bits = sc->nz;
    g.words = words;
    g.visited = sc->visited;
    for (int i = 0; i < 3; ++i) {
        g.fbits[i] = sc->fbits[i];
        g.qv[i] = sc->qv[i];
        g.qe[i] = sc->qe[i];
        g.qr[i] = sc->qr[i];
    }
    g.ulist[0] = sc->ulist[0];
    g.ulist[1] = sc->ulist[1];
    g.ctl = &sc->ctl;
    g.bar_flags = sc->bar_flags;
    g.ws_ready = 1;
    st = grx_bfs_launch(&g, src, depth_out, parent_out, &o, s);
    if (st != GRX_OK) return st;
    if (status_out)
        GRX_CUDA(cudaMemcpyAsync(status_out, &sc->ctl.status, sizeof(int32_t),
                                 cudaMemcpyDeviceToDevice, s));
    return GRX_OK;
}
