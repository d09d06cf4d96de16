// Connected components (Table 1; Soman et al.'s GPU CC): rounds of hooking
// over every edge followed by pointer jumping, until a round hooks nothing.
//
//  * label[v] starts at v.  Hooking: for an undirected edge (u, v) with u < v,
//    find both roots; if they differ, atomicMin the larger root's parent to
//    the smaller root.  Parents only ever decrease and point to a smaller id
//    in the same component, so the forest stays acyclic and the final root of
//    a component is its minimum vertex id -- the canonical label.
//  * Jumping: every vertex follows parents to its root and stores it, so the
//    next round's finds are one step.
//  * The edge loop uses the active list (non-isolated vertices), whose edge
//    prefix is the CSR offsets: tiles of equal edge count (first row and row
//    count of each tile cached per graph), row of each edge by binary search
//    in shared memory, coalesced column reads.
//  * One persistent cooperative kernel; hook and jump phases are separated by
//    bounded grid barriers.  Isolated vertices keep label = own id.
#include "grx_internal.cuh"

namespace {

constexpr int CC_BLOCK = 256;
constexpr int CC_ITEMS = 8;
constexpr int CC_TILE = CC_BLOCK * CC_ITEMS;

struct CcArgs {
    int32_t nv;
    int64_t ne;
    const int32_t *col;
    const int32_t *active;
    const uint32_t *aoff;
    const int2 *tiles;
    int32_t *label;
    TravCtl *ctl;
    unsigned int *bar_flags;
    unsigned long long timeout_ns;
};

struct CcSmem {
    uint32_t qe[CC_TILE + 1];
    int32_t u[CC_TILE + 1];
    int changed;
};

__device__ __forceinline__ int32_t find_root(int32_t *label, int32_t x) {
    int32_t p = __ldcg(label + x);
    while (p != x) {
        x = p;
        p = __ldcg(label + x);
    }
    return x;
}

__device__ void hook_phase(const CcArgs &a, int round, CcSmem &sm) {
    const uint64_t T = (uint64_t)a.ne;
    const uint64_t ntiles = (T + CC_TILE - 1) / CC_TILE;
    int changed = 0;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t e0 = tile * CC_TILE;
        const uint64_t e1 = min(T, e0 + CC_TILE);
        const int2 tr = __ldg(a.tiles + tile);
        const int64_t i0 = tr.x;
        const int n = tr.y;
        for (int j = threadIdx.x; j < n; j += CC_BLOCK) {
            sm.qe[j] = __ldg(a.aoff + i0 + j);
            sm.u[j] = __ldg(a.active + i0 + j);
        }
        __syncthreads();
        for (int k = 0; k < CC_ITEMS; ++k) {
            const uint64_t e = e0 + (uint64_t)(k * CC_BLOCK + threadIdx.x);
            if (e >= e1) break;
            const int32_t v = __ldg(a.col + e);
            const int32_t u = sm.u[upper_index_smem(sm.qe, n, (uint32_t)e)];
            if (u >= v) continue;                 // each undirected edge once
            int32_t ru = find_root(a.label, u);
            int32_t rv = find_root(a.label, v);
            if (ru != rv) {
                int32_t hi = ru > rv ? ru : rv, lo = ru ^ rv ^ hi;
                atomicMin(a.label + hi, lo);
                changed = 1;
            }
        }
        __syncthreads();
    }
    changed = __syncthreads_or(changed);
    if (changed && threadIdx.x == 0) atomicOr(&a.ctl->cc_changed[round & 3], 1u);
}

__device__ void jump_phase(const CcArgs &a) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < a.nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t p = __ldcg(a.label + v);
        if (p == v) continue;
        int32_t r = find_root(a.label, p);
        if (r != p) a.label[v] = r;
    }
}

__global__ void __launch_bounds__(CC_BLOCK) k_cc_persistent(CcArgs a) {
    __shared__ CcSmem sm;
    FlagBarrier bar{a.bar_flags, &a.ctl->bar_release, a.ctl, a.timeout_ns, 0u};
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < a.nv;
         v += (int64_t)gridDim.x * blockDim.x)
        a.label[v] = (int32_t)v;
    if (blockIdx.x == 0 && threadIdx.x < 4) a.ctl->cc_changed[threadIdx.x] = 0u;
    if (!flag_barrier(bar)) return;
    for (int round = 0;; ++round) {
        if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->cc_changed[(round + 2) & 3] = 0u;
        hook_phase(a, round, sm);
        if (!flag_barrier(bar)) return;
        if (threadIdx.x == 0) sm.changed = ld_relaxed_u32(&a.ctl->cc_changed[round & 3]) != 0;
        __syncthreads();
        if (!sm.changed) {
            if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->levels_run = round + 1;
            return;
        }
        jump_phase(a);
        if (!flag_barrier(bar)) return;
    }
}

}  // namespace

grx_status grx_cc_launch(grx_graph *g, int32_t *label, const grx_opts *o, cudaStream_t s) {
    CcArgs a;
    a.nv = g->nv;
    a.ne = g->ne;
    a.col = g->col;
    a.active = g->active;
    a.aoff = g->aoff;
    a.tiles = nullptr;
    if (g->ne > 0) {
        grx_status st = grx_edge_tiles(g, CC_TILE, s, &a.tiles);
        if (st != GRX_OK) return st;
    }
    a.label = label;
    a.ctl = g->ctl;
    a.bar_flags = g->bar_flags;
    a.timeout_ns = grx_timeout_ns(o);
    static int per_sm = -1;
    if (per_sm < 0) {
        GRX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cc_persistent, CC_BLOCK, 0));
        if (per_sm < 1) return grx_fail(GRX_ECUDA, "cc: persistent kernel does not fit on an SM");
    }
    int max_grid = per_sm * g->ctx->num_sms;
    if (max_grid > GRX_MAX_GRID) max_grid = GRX_MAX_GRID;
    int blocks = o->grid_blocks > 0 && o->grid_blocks < max_grid ? o->grid_blocks : max_grid;
    GRX_CUDA(cudaMemsetAsync(g->bar_flags, 0, sizeof(unsigned int) * (size_t)blocks, s));
    GRX_CUDA(cudaMemsetAsync(&g->ctl->bar_release, 0, sizeof(unsigned int), s));
    void *args[] = {(void *)&a};
    GRX_CUDA(cudaLaunchCooperativeKernel((const void *)k_cc_persistent, dim3(blocks), dim3(CC_BLOCK),
                                         args, 0, s));
    return GRX_OK;
}
