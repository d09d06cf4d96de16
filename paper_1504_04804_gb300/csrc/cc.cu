// Connected components (Table 1; Soman et al.'s GPU CC): hooking of trees
// along edges with pointer jumping, labels = the minimum vertex id of each
// component.
//
//  * label[v] starts at v.  Hooking an edge (u, v) joins the trees of u and
//    v: the larger root is hooked under the smaller one with a compare and
//    swap that succeeds only while the larger one is still a root (else the
//    hook retries from the new roots).  Parents only ever decrease and point
//    to a smaller id in the same component, so the forest stays acyclic and
//    the final root of a component is its minimum vertex id -- the canonical
//    label.
//  * Pointer jumping (compression) makes every vertex point at its root.
//  * Most edges need no hooking at all (the sampling refinement of hooking
//    of Sutton et al., Afforest, IPDPS 2018): after hooking every vertex to
//    its first two neighbours and compressing, the largest component is found
//    from a sample of vertices; only the vertices outside it hook the rest of
//    their edges.  An edge between the largest component and another one is
//    still hooked, from its endpoint outside (the graph is symmetric).
//  * One persistent cooperative kernel; phases separated by bounded grid
//    barriers.  Isolated vertices keep label = own id.
#include "grx_internal.cuh"

namespace {

constexpr int CC_BLOCK = 256;
constexpr int CC_SAMPLES = 1024;              // vertices sampled for the largest component

struct CcArgs {
    int32_t nv;
    const int32_t *col;
    const int2 *first2;                       // first two neighbours of every row (-1 = none)
    const int32_t *active;
    const uint32_t *aoff;
    int64_t n_active;
    int32_t *label;
    TravCtl *ctl;
    DevStats *stats;
    unsigned int *bar_flags;
    unsigned long long timeout_ns;
};

__device__ __forceinline__ int32_t find_root(int32_t *label, int32_t x) {
    int32_t p = __ldcg(label + x);
    while (p != x) {
        x = p;
        p = __ldcg(label + x);
    }
    return x;
}

// Joins the trees of u and v: the larger root goes under the smaller one.
// Every failed attempt means some parent decreased, so the loop ends; the cap
// only guards against a corrupted label array (then the status is set).
__device__ __forceinline__ void hook(int32_t *label, int32_t u, int32_t v, TravCtl *ctl) {
    // The first parents may come from L1 (a hub's label is read by most of its
    // neighbours' hooks): a stale parent is still an ancestor, and the
    // compare-and-swap below reads the larger root's parent fresh before it
    // writes, so a stale start only costs a retry.
    int32_t p1 = __ldca(label + u), p2 = __ldca(label + v);
    for (int tries = 0; p1 != p2; ++tries) {
        if (tries > (1 << 24)) {
            grx_set_status(ctl, GRX_ETIMEOUT);
            return;
        }
        const int32_t hi = p1 > p2 ? p1 : p2, lo = p1 ^ p2 ^ hi;
        const int32_t ph = __ldcg(label + hi);
        if (ph == lo) return;                                   // already joined
        if (ph == hi && atomicCAS(label + hi, hi, lo) == hi) return;
        p1 = __ldcg(label + __ldcg(label + hi));                // hi moved on: retry from there
        p2 = __ldcg(label + lo);
    }
}

// Root of x during a compress phase: no hooking runs, so roots cannot change
// and every parent a write replaces is replaced by the root itself; a stale
// parent is still an ancestor.  Reads may therefore be served by L1 (the
// grid barrier's acquire drops what earlier phases left there), which keeps
// the labels of the few large components' roots, read at the end of most
// chains, out of a single L2 slice.
__device__ __forceinline__ int32_t find_root_ca(const int32_t *label, int32_t x) {
    int32_t p = __ldca(label + x);
    while (p != x) {
        x = p;
        p = __ldca(label + x);
    }
    return x;
}

// Every vertex points at its root.
__device__ void compress(const CcArgs &a) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < a.nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = __ldcg(a.label + v);
        if (p == v) continue;
        const int32_t r = find_root_ca(a.label, p);
        if (r != p) a.label[v] = r;
    }
}

// Hooks every non-isolated vertex to its k-th neighbour (k = 0 or 1), read
// from the pair array of first neighbours: 8 bytes per vertex in vertex
// order instead of a row start and a scattered column sector.
__device__ void hook_kth(const CcArgs &a, uint32_t k) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n_active;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = __ldg(a.active + i);
        const int2 f = __ldg(a.first2 + v);
        const int32_t u = k == 0 ? f.x : f.y;
        if (u >= 0) hook(a.label, v, u, a.ctl);
    }
}

// Block 0: the most frequent root among CC_SAMPLES vertices spread over the
// active list (ties go to the smaller root).
__device__ void find_giant(const CcArgs &a) {
    __shared__ int32_t roots[CC_SAMPLES];
    __shared__ unsigned long long best;
    if (threadIdx.x == 0) best = 0ull;
    for (int s = threadIdx.x; s < CC_SAMPLES; s += blockDim.x) {
        // Knuth's multiplicative hash of s spreads the samples
        const uint64_t h = ((uint64_t)s * 2654435761ull) % (uint64_t)(a.n_active > 0 ? a.n_active : 1);
        roots[s] = a.n_active > 0 ? __ldcg(a.label + __ldg(a.active + h)) : 0;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < CC_SAMPLES; s += blockDim.x) {
        int c = 0;
        for (int t = 0; t < CC_SAMPLES; ++t) c += roots[t] == roots[s];
        atomicMax(&best, ((unsigned long long)c << 32) | (unsigned)(0x7fffffff - roots[s]));
    }
    __syncthreads();
    if (threadIdx.x == 0) a.ctl->cc_giant = 0x7fffffff - (int32_t)(best & 0xffffffffull);
}

// Vertices outside the largest component hook their remaining edges.
__device__ void hook_rest(const CcArgs &a, int32_t giant, unsigned long long &linked) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n_active;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = __ldg(a.active + i);
        // Membership in the largest component through L1: a stale view only
        // shows an earlier ancestor chain, and trees only merge, so a vertex
        // seen under the giant root is in its component (its edges to other
        // components are hooked from their side); a stale view that misses
        // the root only costs this vertex's own hooks.
        if (find_root_ca(a.label, v) == giant) continue;
        const uint32_t b = __ldg(a.aoff + i), e = __ldg(a.aoff + i + 1);
        for (uint32_t k = b + 2; k < e; ++k) hook(a.label, v, __ldg(a.col + k), a.ctl);
        linked += e > b + 2 ? e - b - 2 : 0u;
    }
}

__global__ void __launch_bounds__(CC_BLOCK) k_cc_persistent(CcArgs a) {
    FlagBarrier bar{a.bar_flags, &a.ctl->bar_release, a.ctl, a.timeout_ns, 0u};
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < a.nv;
         v += (int64_t)gridDim.x * blockDim.x)
        a.label[v] = (int32_t)v;
    if (!flag_barrier(bar)) return;
    for (uint32_t k = 0; k < 2; ++k) {
        hook_kth(a, k);
        if (!flag_barrier(bar)) return;
        compress(a);
        if (!flag_barrier(bar)) return;
    }
    if (blockIdx.x == 0) find_giant(a);
    if (!flag_barrier(bar)) return;
    const int32_t giant = ld_relaxed_u32((const unsigned int *)&a.ctl->cc_giant);
    unsigned long long linked = 0;
    hook_rest(a, giant, linked);
    if (!flag_barrier(bar)) return;
    compress(a);
    linked = warp_sum(linked);
    if ((threadIdx.x & 31) == 0 && linked) atomicAdd(&a.stats->edges_examined[0], linked);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->levels_run = 1;
        a.stats->levels = 1;
    }
}

}  // namespace

grx_status grx_cc_launch(grx_graph *g, int32_t *label, const grx_opts *o, cudaStream_t s) {
    CcArgs a;
    a.nv = g->nv;
    a.col = g->col;
    a.first2 = g->first2;
    a.active = g->active;
    a.aoff = g->aoff;
    a.n_active = g->n_active;
    a.label = label;
    a.ctl = g->ctl;
    a.stats = g->stats;
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
    GRX_CUDA(cudaMemsetAsync(&g->stats->levels, 0, sizeof(int32_t), s));
    GRX_CUDA(cudaMemsetAsync(&g->stats->edges_examined[0], 0, sizeof(unsigned long long), s));
    void *args[] = {(void *)&a};
    GRX_CUDA(cudaLaunchCooperativeKernel((const void *)k_cc_persistent, dim3(blocks), dim3(CC_BLOCK),
                                         args, 0, s));
    return GRX_OK;
}
