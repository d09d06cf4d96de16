// Internal declarations shared by the libgrx translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "grx.h"

#define GRX_FULL_MASK 0xffffffffu

// ---------------------------------------------------------------------------
// Host-side objects
// ---------------------------------------------------------------------------
struct grx_ctx {
    grx_allocator alloc;
    int has_alloc;
    int device;
    int num_sms;
};

// Device control block of a graph's traversals.  Barrier words live on their
// own 128-byte lines so spinning blocks do not contend with counter updates.
struct alignas(128) TravCtl {
    // frontier ring: packed (count << 32 | edges) per slot; slot = level & 3
    unsigned long long qpack[4];
    unsigned int ucount[4];          // unvisited-list lengths, same ring
    unsigned int disc[4];            // vertices discovered per level, same ring
    int status;                      // first device-side error (0 = ok)
    int levels_run;                  // levels completed by the last traversal
    unsigned long long cpack;        // BFS bitmap->queue compaction counter (count << 32 | edges)
    unsigned int ms_grid;            // multi-source BFS: grid of the last traversal
    unsigned int ms_done;            // ... blocks that completed its final pass
    int cc_giant;                    // CC: root of the sampled largest component
    unsigned int farcnt[2];          // SSSP near-far: far pile lengths (ping-pong)
    unsigned int farmin[2];          // SSSP near-far: smallest distance in the far pile (by pile)
    unsigned int bcfix[3];           // BC backward: rows finished after the barrier, by level mod 3
    unsigned int wq[4];              // BFS: chunk counters of the word-owning sweeps, ring by phase
    unsigned int pad0[2];
    unsigned int bar_count;          // grid barrier arrivals
    unsigned int pad1[31];
    unsigned int bar_gen;            // grid barrier generation
    unsigned int pad2[31];
    // host-stepped mode: per-launch state, double buffered
    long long hstate[2][8];
    // PageRank dangling-mass accumulators (ring of 3)
    double pr_dangling[3];
    unsigned int flags;              // misc device flags (e.g. CC "changed")
    unsigned int cc_changed[4];
    unsigned int pad3[26];
    unsigned int bar_release;        // flag-barrier release word (own line)
    unsigned int pad4[31];
    unsigned long long pairs[4];     // multi-source: (vertex, lane) pairs discovered, ring
};

// Maximum grid of the persistent kernels (size of the barrier flag array).
#define GRX_MAX_GRID 4096
// PageRank column blocks: at most this many.
#define GRX_PRB_MAX_K 256

struct DevStats {                    // device mirror of grx_trav_stats
    int32_t levels;
    int32_t dir[GRX_MAX_LEVELS_STATS];
    unsigned long long frontier[GRX_MAX_LEVELS_STATS];
    unsigned long long edges_examined[GRX_MAX_LEVELS_STATS];
    unsigned long long vertices_scanned[GRX_MAX_LEVELS_STATS];
    unsigned long long discovered[GRX_MAX_LEVELS_STATS];
    unsigned long long level_t0[GRX_MAX_LEVELS_STATS + 1];   // globaltimer at level start
};

struct grx_graph {
    grx_ctx *ctx;
    int32_t nv;
    int64_t ne;
    int off64;                       // row offsets stored as int64
    void *ro;                        // int32 or int64 [nv+1]
    int32_t *col;                    // [ne]
    uint32_t *w;                     // [ne] or NULL
    uint32_t *nz_bits;               // non-isolated vertex bitmap [words]
    int64_t words;                   // (nv + 31) / 32 rounded up to 32
    // non-isolated vertices in increasing id order and their row starts:
    // active[i] = v, aoff[i] = ro[v], aoff[n_active] = ne.  With isolated
    // rows dropped, edge e of this list is CSR edge e.
    int32_t *active;
    uint32_t *aoff;
    int64_t n_active;
    // static row ranges of all-edges tiles (CC hooking, PageRank, multi-source
    // pull), per tile size
    int2 *etiles[4];
    int etile_size[4];
    void *last_stream;
    // ---- traversal workspace (allocated on first use) ----
    int ws_ready;
    uint32_t *visited;               // [words]
    uint32_t *fbits[3];              // frontier bitmaps [words] each
    int32_t *qv[3];                  // frontier vertices [nv] each
    uint32_t *qe[3];                 // exclusive edge prefix per frontier slot
    void *qr[3];                     // row start (OffT) per frontier slot
    int32_t *ulist[2];               // unvisited lists [nv] each
    int2 *first2;                    // [nv] first two neighbours of each row (-1 = none)
    TravCtl *ctl;
    unsigned int *bar_flags;         // [GRX_MAX_GRID] per-block arrival flags
    DevStats *stats;
    // SSSP
    int32_t *stamp;                  // [nv] round in which v was last queued
    // PageRank
    float *pr_c[2];                  // contribution r/deg ping-pong
    float *pr_s;                     // cross-tile partial sums
    int32_t *pr_fix;                 // per-tile row needing a fix-up
    int64_t pr_fix_len;
    // PageRank column blocks (segments of rows per block of 2^prb_shift columns)
    int pr_shift_req;                // requested block width (0 = automatic, < 0 = never)
    int prb_K, prb_shift;            // built blocks (prb_K < 2: none)
    int32_t *prb_seg_v;              // segment's row vertex
    uint32_t *prb_seg_start;         // segment's first edge
    uint32_t *prb_pre;               // per block: exclusive edge prefix (+ sentinel)
    int2 *prb_tiles;                 // per block: equal edge tiles (first segment, count)
    int64_t prb_kbase[GRX_PRB_MAX_K + 1];
    int64_t prb_tbase[GRX_PRB_MAX_K + 1];
    uint32_t prb_kedges[GRX_PRB_MAX_K];
    // multi-source
    unsigned long long *ms_cur[3], *ms_next, *ms_seen;   // [nv] each
    unsigned long long *ms_hist[6];  // multi-source BFS: pull levels' new lanes, [nv] each
    int32_t *ms_fix;                 // multi-source BFS: per pull tile, the crossing row it finishes
    uint32_t *ms_tbits;              // multi-source BFS: touched bitmap of bitmap push levels
    uint8_t *ms_sat;                 // multi-source BFS: per pull tile, all lanes seen
    uint32_t *ms_dist;               // batched SSSP, vertex-major [nv][64]
    int ms_ready;
    // betweenness centrality (allocated on first use)
    double *bc_sigma, *bc_acc;       // [nv] each: path counts; successor sums / coefficients
    uint32_t *bc_code;               // [2 * words]: 2-bit level codes
    // batched betweenness centrality (allocated on first use)
    unsigned long long *bcm_seen, *bcm_next;   // [nv] lane masks
    unsigned long long *bcm_hist;    // [GRX_BCM_MAX_LEVELS][nv] lanes at each depth
    double *bcm_sig, *bcm_acc;       // [nv][64]
    int32_t *bcm_srcs;               // [64] device copy of the sources
    // CUDA-graph level loop of bfs (GRX_LOOP_GRAPH), per parent flag
    cudaGraphExec_t bfs_gexec[2];
    void *bfs_gargs;                 // device copy of the call's arguments
    // 64-bit vertex ids (graph_load_csr64): columns, frontier queues and
    // long-row lists of bfs64; nv64 is the vertex count (nv is -1 past 2^31)
    int vid64;
    int64_t nv64;
    int64_t *col64;
    int64_t *q64[2];
    int64_t *lr64[3];
    int ws64_ready;
    // bookkeeping for frees
    struct Alloc { void *p; size_t n; } allocs[96];
    int nallocs;
};

// Allocation through the context allocator (or cudaMallocAsync).
void *grx_alloc(grx_graph *g, size_t bytes, cudaStream_t s);
void *grx_ctx_alloc(grx_ctx *c, size_t bytes, cudaStream_t s);
void grx_ctx_free(grx_ctx *c, void *p, size_t bytes, cudaStream_t s);
grx_status grx_ensure_workspace(grx_graph *g, cudaStream_t s);
grx_status grx_ensure_ms_workspace(grx_graph *g, cudaStream_t s);

// Error helpers (thread-local message).
grx_status grx_fail(grx_status st, const char *fmt, ...);
grx_status grx_cuda_fail(cudaError_t e, const char *what);
#define GRX_CUDA(call)                                                         \
    do {                                                                       \
        cudaError_t _e = (call);                                               \
        if (_e != cudaSuccess) return grx_cuda_fail(_e, #call);                \
    } while (0)

// Builds g->active / g->aoff / g->n_active (synchronises s once).
grx_status grx_build_active(grx_graph *g, cudaStream_t s);
// Fills g->first2 (allocated by the caller) from the CSR.
grx_status grx_build_first2(grx_graph *g, cudaStream_t s);
// Cached (first active row, row count) of every tile of `tile` consecutive
// edges over the whole edge array.
grx_status grx_edge_tiles(grx_graph *g, int tile, cudaStream_t s, const int2 **out);

grx_status grx_msbfs_launch(grx_graph *g, const int32_t *srcs, int n, int32_t *depth,
                            const grx_opts *o, cudaStream_t s);
// Device bytes the next multi-source BFS / batched SSSP launch allocates for
// its own workspace on g (0 once allocated; shared pieces counted by both).
size_t grx_msbfs_new_bytes(const grx_graph *g);
size_t grx_mssp_new_bytes(const grx_graph *g);
grx_status grx_mssp_launch(grx_graph *g, const int32_t *srcs, int n, uint32_t *dist,
                           const grx_opts *o, cudaStream_t s);

// Options resolution.
void grx_resolve_opts(const grx_opts *in, grx_opts *out);
unsigned long long grx_timeout_ns(const grx_opts *o);

// Kernel launchers (one per translation unit).
grx_status grx_bfs_launch(grx_graph *g, int32_t src, int32_t *depth, int32_t *parent,
                          const grx_opts *o, cudaStream_t s);
grx_status grx_sssp_launch(grx_graph *g, int32_t src, uint32_t *dist, const grx_opts *o,
                           cudaStream_t s);
grx_status grx_cc_launch(grx_graph *g, int32_t *label, const grx_opts *o, cudaStream_t s);
grx_status grx_bc_launch(grx_graph *g, const int32_t *srcs, int n, double *bc_out, double *sigma_out,
                         const grx_opts *o, cudaStream_t s);
grx_status grx_bcm_launch(grx_graph *g, const int32_t *srcs, int n, double *bc_out, const grx_opts *o,
                          cudaStream_t s);
grx_status grx_pr_launch(grx_graph *g, float damping, int iters, float *rank,
                         cudaStream_t s);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

__device__ __forceinline__ unsigned long long grx_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Record the first device-side error; later ones are dropped.
__device__ __forceinline__ void grx_set_status(TravCtl *ctl, int st) {
    atomicCAS(&ctl->status, 0, st);
}

// Grid-wide barrier for cooperative launches.  Every wait is bounded by
// `timeout_ns` of global time: a block that gives up records GRX_ETIMEOUT and
// returns false, and the caller leaves its loop.  Memory written before the
// barrier by any block is visible after it (release by the last arriver,
// acquire by the waiters).
__device__ __forceinline__ bool grid_barrier(TravCtl *ctl, unsigned long long timeout_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned int gen = ld_acquire_u32(&ctl->bar_gen);
        __threadfence();
        unsigned int arrived = atomicAdd(&ctl->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            st_release_u32(&ctl->bar_gen, gen + 1);
        } else {
            unsigned long long t0 = grx_globaltimer();
            while (ld_acquire_u32(&ctl->bar_gen) == gen) {
                if (grx_globaltimer() - t0 > timeout_ns) {
                    grx_set_status(ctl, GRX_ETIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Flag-based grid barrier: block b (> 0) publishes its arrival in flags[b];
// block 0's threads gather all flags in parallel, then release everyone with
// one word.  No contended atomic.  `gen` counts barriers within a launch
// (flags and release word are zeroed before the launch, gen starts at 0).
// Every wait is bounded by timeout_ns; a block that gives up records
// GRX_ETIMEOUT and returns false.
struct FlagBarrier {
    unsigned int *flags;
    unsigned int *release;
    TravCtl *ctl;
    unsigned long long timeout_ns;
    unsigned int gen;
};

__device__ __forceinline__ bool flag_barrier(FlagBarrier &b) {
    __shared__ int s_ok;
    const unsigned int gen = ++b.gen;
    __syncthreads();
    if (blockIdx.x == 0) {
        int ok = 1;
        for (unsigned int i = threadIdx.x + 1; i < gridDim.x && ok; i += blockDim.x) {
            if (ld_acquire_u32(b.flags + i) == gen) continue;
            const unsigned long long t0 = grx_globaltimer();
            while (ld_acquire_u32(b.flags + i) != gen) {
                if (grx_globaltimer() - t0 > b.timeout_ns) { ok = 0; break; }
                __nanosleep(32);
            }
        }
        ok = __syncthreads_and(ok);
        if (threadIdx.x == 0) {
            if (ok) {
                __threadfence();
                st_release_u32(b.release, gen);
            } else {
                grx_set_status(b.ctl, GRX_ETIMEOUT);
            }
            s_ok = ok;
        }
    } else if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        st_release_u32(b.flags + blockIdx.x, gen);
        if (ld_acquire_u32(b.release) != gen) {
            const unsigned long long t0 = grx_globaltimer();
            while (ld_acquire_u32(b.release) != gen) {
                if (grx_globaltimer() - t0 > b.timeout_ns) {
                    grx_set_status(b.ctl, GRX_ETIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Warp-aggregated append of up to N items per lane (bit k of mask = item k
// present) to a frontier whose counter packs (count << 32 | edge total).  One
// atomic per warp; the edge prefix stays monotone in position order.  Must be
// called by all 32 lanes.
template <int N, typename OffT>
__device__ __forceinline__ void warp_append_items(const int32_t (&v)[N], const uint32_t (&deg)[N],
                                                  const OffT (&rs)[N], uint32_t mask, int32_t *qv,
                                                  uint32_t *qe, OffT *qr, unsigned long long *ctr) {
    uint32_t cnt = __popc(mask), dsum = 0;
#pragma unroll
    for (int k = 0; k < N; ++k)
        if (mask >> k & 1u) dsum += deg[k];
    const unsigned int lane = threadIdx.x & 31;
    uint32_t c = cnt, s = dsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t c2 = __shfl_up_sync(0xffffffffu, c, o);
        uint32_t s2 = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= (unsigned)o) { c += c2; s += s2; }
    }
    const uint32_t tc = __shfl_sync(0xffffffffu, c, 31);
    if (tc == 0) return;
    const uint32_t ts = __shfl_sync(0xffffffffu, s, 31);
    unsigned long long base = 0;
    if (lane == 31) base = atomicAdd(ctr, ((unsigned long long)tc << 32) | (unsigned long long)ts);
    base = __shfl_sync(0xffffffffu, base, 31);
    uint32_t pos = (uint32_t)(base >> 32) + c - cnt;
    uint32_t eo = (uint32_t)base + s - dsum;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        if (mask >> k & 1u) {
            qv[pos] = v[k];
            qe[pos] = eo;
            if (qr) qr[pos] = rs[k];
            ++pos;
            eo += deg[k];
        }
    }
}

// Warp-aggregated append of up to N list items per lane with a 32-bit counter.
template <int N>
__device__ __forceinline__ void warp_append_list_items(const int32_t (&v)[N], uint32_t mask,
                                                       int32_t *list, unsigned int *ctr) {
    const unsigned int lane = threadIdx.x & 31;
    const uint32_t cnt = __popc(mask);
    uint32_t c = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t c2 = __shfl_up_sync(0xffffffffu, c, o);
        if (lane >= (unsigned)o) c += c2;
    }
    const uint32_t tc = __shfl_sync(0xffffffffu, c, 31);
    if (tc == 0) return;
    unsigned int base = 0;
    if (lane == 31) base = atomicAdd(ctr, tc);
    base = __shfl_sync(0xffffffffu, base, 31);
    uint32_t pos = base + c - cnt;
#pragma unroll
    for (int k = 0; k < N; ++k)
        if (mask >> k & 1u) list[pos++] = v[k];
}

__device__ __forceinline__ unsigned int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ unsigned int lanemask_lt() {
    unsigned int m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Warp-aggregated append of (v, deg) to a frontier whose counter packs
// (count << 32 | edge total).  One atomic per warp; positions and edge
// prefixes come from the same atomic, so the prefix array stays monotone in
// position order.  Must be called by all 32 lanes.
__device__ __forceinline__ void warp_append_frontier(bool flag, int32_t v, uint32_t deg,
                                                     int32_t *qv, uint32_t *qe,
                                                     unsigned long long *ctr) {
    unsigned int mask = __ballot_sync(GRX_FULL_MASK, flag);
    if (mask == 0) return;
    unsigned int lane = lane_id();
    uint32_t x = flag ? deg : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(GRX_FULL_MASK, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    uint32_t total = __shfl_sync(GRX_FULL_MASK, x, 31);
    unsigned long long base = 0;
    if (lane == 0)
        base = atomicAdd(ctr, ((unsigned long long)__popc(mask) << 32) | (unsigned long long)total);
    base = __shfl_sync(GRX_FULL_MASK, base, 0);
    if (flag) {
        uint32_t pos = (uint32_t)(base >> 32) + __popc(mask & lanemask_lt());
        qv[pos] = v;
        qe[pos] = (uint32_t)base + (x - deg);
    }
}

// Warp-aggregated append of v to a plain list with a 32-bit counter.
__device__ __forceinline__ void warp_append_list(bool flag, int32_t v, int32_t *list,
                                                 unsigned int *ctr) {
    unsigned int mask = __ballot_sync(GRX_FULL_MASK, flag);
    if (mask == 0) return;
    unsigned int base = 0;
    if (lane_id() == 0) base = atomicAdd(ctr, (unsigned)__popc(mask));
    base = __shfl_sync(GRX_FULL_MASK, base, 0);
    if (flag) list[base + __popc(mask & lanemask_lt())] = v;
}

// Largest i in [0, n) with a[i] <= key (a ascending, a[0] <= key).
template <typename T, typename K>
__device__ __forceinline__ int64_t upper_index(const T *a, int64_t n, K key) {
    int64_t lo = 0, hi = n;             // invariant: a[lo] <= key, answer in [lo, hi)
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if ((K)a[mid] <= key) lo = mid; else hi = mid;
    }
    return lo;
}

template <typename T>
__device__ __forceinline__ T pick3(T a, T b, T c, int i) { return i == 0 ? a : (i == 1 ? b : c); }

// Largest i in [0, n) with a[i] <= key, reading through L2 (a was written by
// other blocks earlier in the same kernel).  Requires a[0] <= key.
__device__ __forceinline__ int64_t upper_index_cg(const uint32_t *a, int64_t n, uint32_t key) {
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldcg(a + mid) <= key) lo = mid; else hi = mid;
    }
    return lo;
}

// Same search in shared memory.
__device__ __forceinline__ int upper_index_smem(const uint32_t *a, int n, uint32_t key) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (a[mid] <= key) lo = mid; else hi = mid;
    }
    return lo;
}

// Largest i in [0, n) with a[i] <= key (a ascending, a[0] <= key), found by
// one full warp with a 32-ary search: each round probes 32 points at once, so
// the dependent round trips are log32(n).  All 32 lanes get the result.
__device__ __forceinline__ int64_t warp_upper_index_cg(const uint32_t *a, int64_t n, uint32_t key) {
    const unsigned int lane = threadIdx.x & 31;
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t idx = lo + (int64_t)lane * step;
        const bool ok = idx < hi && __ldcg(a + idx) <= key;
        const unsigned int m = __ballot_sync(0xffffffffu, ok);
        const int last = 31 - __clz(m);
        lo = lo + (int64_t)last * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// Block-wide exclusive scan of three counters (blockDim.x == NT, a multiple
// of 32).  Returns the exclusive prefixes and, in every thread, the totals.
template <int NT>
__device__ __forceinline__ void block_scan3(uint32_t a, uint32_t b, uint32_t c, uint32_t &ea,
                                            uint32_t &eb, uint32_t &ec, uint32_t &ta, uint32_t &tb,
                                            uint32_t &tc) {
    __shared__ uint32_t ws[3][NT / 32];
    const unsigned int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = a, y = b, z = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t x2 = __shfl_up_sync(0xffffffffu, x, o);
        uint32_t y2 = __shfl_up_sync(0xffffffffu, y, o);
        uint32_t z2 = __shfl_up_sync(0xffffffffu, z, o);
        if (lane >= (unsigned)o) { x += x2; y += y2; z += z2; }
    }
    if (lane == 31) { ws[0][wid] = x; ws[1][wid] = y; ws[2][wid] = z; }
    __syncthreads();
    uint32_t px = 0, py = 0, pz = 0, sx = 0, sy = 0, sz = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
        const uint32_t wx = ws[0][w], wy = ws[1][w], wz = ws[2][w];
        if ((unsigned)w < wid) { px += wx; py += wy; pz += wz; }
        sx += wx; sy += wy; sz += wz;
    }
    ea = px + x - a; eb = py + y - b; ec = pz + z - c;
    ta = sx; tb = sy; tc = sz;
    __syncthreads();
}

// Compacts the set bits of a 32-word bitmap chunk (lane i holds word i) into
// list[] as chunk offsets (word * 32 + bit) in increasing order.  Returns the
// count in every lane.
__device__ __forceinline__ int warp_compact_bits(uint32_t bits, uint16_t *list) {
    const unsigned int lane = threadIdx.x & 31;
    const int c = __popc(bits);
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(GRX_FULL_MASK, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    const int total = __shfl_sync(GRX_FULL_MASK, x, 31);
    int pos = x - c;
    while (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1;
        list[pos++] = (uint16_t)(lane * 32 + b);
    }
    __syncwarp();
    return total;
}

// Row of every position of a warp tile, without per-item searches or loops
// (branches are the scarce resource of a hot tile loop): positions start at
// row 0; each non-empty row j > 0 that starts inside the tile writes j at its
// start; an inclusive max-scan over the positions then gives every position
// its row.  rid (16-byte aligned) holds 256 entries, 8 consecutive ones per lane;
// starts[0..n] are the rows' first positions (non-decreasing, starts[n] =
// end of row n-1).  On return row[k] is the row of position
// lane*8 + k (meaningful where the position lies inside a row).
__device__ __forceinline__ void warp_tile_rows8(uint16_t *rid, const uint32_t *starts, uint32_t origin,
                                                int n, int (&row)[8]) {
    const unsigned int lane = threadIdx.x & 31;
    reinterpret_cast<uint4 *>(rid)[lane] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
    for (int j = 1 + (int)lane; j < n; j += 32) {
        const uint32_t p = starts[j] - origin;
        if (p < 256u && starts[j + 1] > starts[j]) rid[p] = (uint16_t)j;
    }
    __syncwarp();
    const uint4 q4 = reinterpret_cast<const uint4 *>(rid)[lane];
    const uint32_t pk[4] = {q4.x, q4.y, q4.z, q4.w};
    int m = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        m = max(m, (int)((pk[k >> 1] >> ((k & 1) * 16)) & 0xffffu));
        row[k] = m;
    }
    int x = m;                                   // inclusive max-scan of the lanes' maxima
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(GRX_FULL_MASK, x, o);
        if (lane >= (unsigned)o) x = max(x, y);
    }
    int carry = __shfl_up_sync(GRX_FULL_MASK, x, 1);
    if (lane == 0) carry = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) row[k] = max(row[k], carry);
    __syncwarp();
}

// Rows of the positions k*32 + lane of a 256-position warp tile (inputs as
// warp_tile_rows8).  With this assignment item k of the 32 lanes covers 32
// consecutive positions, so a warp's column loads for item k read one
// contiguous 128-byte run (and the sorted targets of a row sit side by side
// across the lanes) instead of 32 runs 32 bytes apart.  rid ends up holding
// the row of every position.
__device__ __forceinline__ void warp_tile_rows8_strided(uint16_t *rid, const uint32_t *starts, uint32_t origin,
                                                        int n, int (&row)[8]) {
    warp_tile_rows8(rid, starts, origin, n, row);     // rows of positions lane*8 + k
    const unsigned int lane = threadIdx.x & 31;
    reinterpret_cast<uint4 *>(rid)[lane] =
        make_uint4((uint32_t)row[0] | (uint32_t)row[1] << 16, (uint32_t)row[2] | (uint32_t)row[3] << 16,
                   (uint32_t)row[4] | (uint32_t)row[5] << 16, (uint32_t)row[6] | (uint32_t)row[7] << 16);
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 8; ++k) row[k] = rid[k * 32 + lane];
    __syncwarp();
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(GRX_FULL_MASK, x, o);
    return x;
}

#endif  // __CUDACC__
