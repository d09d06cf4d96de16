/*
 * grx.h -- C ABI of libgrx, a single-GPU (GB300, sm_103a) implementation of the
 * frontier-traversal hot path of "Multi-GPU Graph Analytics" (Pan, Wang, Wu,
 * Yang, Owens; arXiv 1504.04804): advance/filter over a CSR graph, the
 * direction-optimising (push/pull) traversal of Sec. 6.1, and the BFS, SSSP,
 * connected-components and PageRank primitives of Sec. 4 (Table 1,
 * Algorithms 1-3), plus 64-source batched traversal.
 *
 * Conventions for every call:
 *  - All calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL = the legacy default stream).  Nothing synchronises the host unless
 *    the call says so.  Device-side failures (a bounded wait that ran out, a
 *    distance that overflowed) are recorded in the graph's status word and
 *    returned by grx_graph_status().
 *  - Output arrays are caller-owned DEVICE buffers of the documented size.
 *    Input arrays are copied; the graph owns its copies.
 *  - Errors are returned as grx_status codes; nothing throws across the ABI.
 *    grx_last_error() gives a message for the calling thread's last failure.
 *  - Vertex ids are int32 (nv < 2^31, else GRX_ERANGE).  The CSR must be
 *    symmetric (every undirected edge stored in both rows, Sec. 7), without
 *    self-loops or duplicate edges, rows sorted ascending.  The pull step,
 *    CC and PageRank rely on symmetry; GRX_VALIDATE checks it on the device.
 *  - One grx_ctx per host thread; a ctx and its graphs are not thread-safe.
 *    Calls on the same graph must be issued on one stream (or ordered by the
 *    caller), because a graph's traversal workspace is shared by its calls.
 */
#ifndef GRX_H
#define GRX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GRX_OK = 0,
    GRX_EINVAL = -1,    /* bad argument or malformed graph */
    GRX_ENOMEM = -2,    /* the allocator returned NULL */
    GRX_ECUDA = -3,     /* a CUDA runtime call failed */
    GRX_ETIMEOUT = -4,  /* a device-side bounded wait gave up */
    GRX_ERANGE = -5,    /* a size or value exceeds the supported range */
    GRX_EBUSY = -6      /* no free lane / slot */
} grx_status;

typedef struct grx_ctx grx_ctx;
typedef struct grx_graph grx_graph;
typedef struct grx_batch grx_batch;

/* Device-memory allocator.  alloc must return a device pointer usable on
 * `stream` (or NULL on failure); free receives the same pointer and size.
 * The library keeps no pointer past the matching free. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} grx_allocator;

/* Create a context bound to the current CUDA device.  allocator == NULL
 * selects cudaMallocAsync/cudaFreeAsync.  The allocator struct is copied. */
grx_status grx_ctx_create(const grx_allocator *allocator, grx_ctx **out);
grx_status grx_ctx_destroy(grx_ctx *ctx);

/* Message for the calling thread's most recent failed call ("" if none). */
const char *grx_last_error(void);

/* flags for graph_load_csr */
#define GRX_HOST_PTRS   0x0   /* inputs are host pointers */
#define GRX_DEVICE_PTRS 0x1   /* inputs are device pointers */
#define GRX_VALIDATE    0x2   /* check offsets, column range, sortedness, no
                                 self-loops, symmetry and weight symmetry on
                                 the device (synchronises `stream`) */
#define GRX_OFFSETS64   0x4   /* store 64-bit row offsets even when ne < 2^31 */

/* graph_load_csr -- Sec. 7 inputs: an undirected graph with self-loops and
 * duplicate edges removed, stored as CSR (the paper's Csr, Appendix A).
 *   nv, ne           vertex count (< 2^31) and directed edge count (< 2^32)
 *   row_offsets      nv+1 entries, int32 (offsets_are_64bit = 0) or int64
 *   col_indices      ne int32 vertex ids
 *   weights          ne uint32 SSSP weights (Sec. 7), or NULL
 *   flags            GRX_HOST_PTRS | GRX_DEVICE_PTRS, optionally GRX_VALIDATE
 * The library copies the arrays into memory from the ctx allocator and owns
 * them until graph_free.  Offsets are stored as int32 when ne < 2^31 (unless
 * GRX_OFFSETS64), else
 * int64.  Returns GRX_EINVAL for malformed input (with GRX_VALIDATE), and
 * GRX_ERANGE for nv >= 2^31 or ne >= 2^32. */
grx_status graph_load_csr(grx_ctx *ctx, int64_t nv, int64_t ne,
                          const void *row_offsets, int offsets_are_64bit,
                          const int32_t *col_indices, const uint32_t *weights,
                          int flags, void *stream, grx_graph **out);

/* Free the graph's device memory (enqueued on the stream of the last call). */
grx_status graph_free(grx_graph *g);

/* Vertex and edge counts of a loaded graph. */
grx_status grx_graph_info(const grx_graph *g, int64_t *nv, int64_t *ne);

/* Synchronise `stream` and return (then clear) the device-side status word of
 * the graph's traversals since the last call: GRX_OK, GRX_ETIMEOUT (a bounded
 * wait ran out; outputs are not valid) or GRX_ERANGE (an SSSP distance did not
 * fit below UINT32_MAX). */
grx_status grx_graph_status(grx_graph *g, void *stream);

/* ---- traversal options ------------------------------------------------- */
#define GRX_DIR_AUTO 0   /* Sec. 6.1 push/pull switch with alpha (do_a), beta (do_b) */
#define GRX_DIR_PUSH 1   /* top-down only (Algorithm 1) */
#define GRX_DIR_PULL 2   /* bottom-up from the first level (for testing) */

#define GRX_LOOP_PERSISTENT 0  /* one cooperative kernel runs every level */
#define GRX_LOOP_HOST       1  /* one launch per level, host polls every 16 */
#define GRX_LOOP_GRAPH      2  /* levels captured in a CUDA graph with a
                                  device-evaluated WHILE condition node */

typedef struct {
    int direction;        /* GRX_DIR_* (BFS and multi-source BFS) */
    float alpha;          /* push->pull when FV > BV * alpha (paper: do_a) */
    float beta;           /* pull->push when FV < BV * beta  (paper: do_b) */
    int loop;             /* GRX_LOOP_* */
    int grid_blocks;      /* persistent grid size; 0 = SMs x occupancy */
    int block_threads;    /* 0 = library default */
    double timeout_s;     /* bound on every device-side wait; <= 0 = 5 s */
    int collect_stats;    /* record per-level counters for grx_last_stats */
    int exact_fv;         /* 1: FV is the frontier's exact edge count (known
                             for free from the append counter) instead of
                             the paper's |Q|*E/V estimate */
    void *ev_begin;       /* optional cudaEvent_t recorded on `stream` just  */
    void *ev_end;         /* before / after the traversal kernel(s) (timing) */
    float push_bitmap;    /* BFS and multi-source BFS push levels with at
                             least push_bitmap * nv frontier edges mark their
                             targets in a bitmap and build the next frontier
                             in a second pass (no per-edge atomic with a
                             return value); 0 = 1/8, < 0 = never.  Results do
                             not depend on it. */
    unsigned int sssp_delta; /* SSSP near-far band width (Davidson et al.'s
                             near-far priority split of the frontier): a
                             round relaxes only vertices closer than the
                             current threshold, the others wait in a far pile
                             until the threshold advances to the pile's
                             smallest distance + delta.  0 = no bands (plain
                             label-correcting rounds).  Results do not depend
                             on it. */
} grx_opts;

/* Library defaults: AUTO direction, alpha 0.01, beta 0.1 (Sec. 6.1's values
 * for social graphs), persistent loop, full-occupancy grid, 5 s timeout. */
void grx_opts_default(grx_opts *o);

/* bfs -- Algorithm 1 (BFS) and, with direction AUTO, Algorithm 2 (DOBFS,
 * Sec. 6.1).  depth_out: device int32[nv], hop distance from src, -1 if
 * unreached.  parent_out: NULL or device int32[nv]; parent_out[src] = src,
 * -1 if unreached, else a neighbour one level closer (any valid one).
 * opts NULL = defaults.  Invalid src -> GRX_EINVAL. */
grx_status bfs(grx_graph *g, int32_t src, int32_t *depth_out, int32_t *parent_out,
               const grx_opts *opts, void *stream);

/* bfs_multi -- up to 64 BFS sources in one traversal that shares the edge
 * stream: every vertex carries 64-bit frontier / seen lane masks and lane b
 * starts at srcs_host[b] (host array).  depth_out: device int32[n][nv]
 * (lane-major), lane b equal to bfs(srcs_host[b]).  n in 1..64; duplicate
 * sources allowed.  opts->direction, alpha, beta act on lane popcounts. */
grx_status bfs_multi(grx_graph *g, const int32_t *srcs_host, int n, int32_t *depth_out,
                     const grx_opts *opts, void *stream);

/* sssp -- Table 1 SSSP: frontier label-correcting relaxation with atomicMin
 * (the paper's min combiner, Sec. 3) until no distance improves.
 * dist_out: device uint32[nv], UINT32_MAX if unreached.  Needs weights
 * (else GRX_EINVAL).  A distance >= UINT32_MAX sets GRX_ERANGE status. */
grx_status sssp(grx_graph *g, int32_t src, uint32_t *dist_out,
                const grx_opts *opts, void *stream);

/* sssp_multi -- up to 64 SSSP sources sharing one edge stream (per lane the
 * result of sssp()).  dist_out: device uint32[n][nv] (lane-major),
 * UINT32_MAX if unreached.  Needs weights.  Uses 256 bytes of workspace per
 * vertex (distances are kept vertex-major inside the library). */
grx_status sssp_multi(grx_graph *g, const int32_t *srcs_host, int n, uint32_t *dist_out,
                      const grx_opts *opts, void *stream);

/* bc -- Table 1 BC: Brandes' dependencies of each source, by a forward
 * shortest-path-counting BFS and a backward pass over the same levels
 * (McLaughlin and Bader's scheme, Sec. 2).  For source s,
 *   delta_s(v) = sum over t != s, v of sigma_st(v) / sigma_st
 * (sigma_st = number of shortest s-t paths, sigma_st(v) = those through v).
 * bc_out: device float64[nv], overwritten with the sum of delta_s over the n
 * sources in srcs_host (host array, n >= 1, duplicates allowed); the source
 * itself gets nothing from its own traversal, unreached vertices nothing.
 * Ordered pairs: summed over every source of an undirected graph each
 * unordered pair counts twice.  sigma_out: NULL or device float64[nv], the
 * shortest-path counts sigma_{s,v} of the last source (0 if unreached).
 * The graph must be symmetric (undirected, as every graph of Sec. 7).
 * Float64 arithmetic; reductions arrive in any order, so values match a
 * sequential float64 sum to rounding.  Forward levels with at least
 * opts->push_bitmap * nv edges only add path counts and find the next level
 * afterwards from the nonzero counts, instead of claiming vertices one by
 * one (results do not depend on it).  opts->direction: GRX_DIR_AUTO picks
 * per level by edge counts -- a forward level is a pull over the unreached
 * vertices when they have less than a quarter of the frontier's edges, a
 * backward level pushes from the level below when that one has fewer edges;
 * GRX_DIR_PUSH keeps forward push / backward pull, GRX_DIR_PULL the other
 * way round (after the source level).  Uses about 16 bytes of workspace per
 * vertex.  With opts->collect_stats, grx_last_stats describes the last
 * source's phases: forward levels (dir 0) then backward levels (dir 1),
 * frontier = the level's vertices, edges_examined = the edges the phase
 * reads (a forward pull: the unreached vertices' rows; a backward push: the
 * rows of the level below), vertices_scanned = the phase's kind.
 * Bad source, n < 1, bad direction or NULL output -> GRX_EINVAL. */
grx_status bc(grx_graph *g, const int32_t *srcs_host, int n, double *bc_out, double *sigma_out,
              const grx_opts *opts, void *stream);

/* bc_multi -- the same sum as bc() for up to 64 sources (n in 1..64,
 * duplicates allowed), computed in one forward and one backward sweep shared
 * by all sources: per vertex 64-bit lane masks and a 64-lane float64 row of
 * path counts and of successor sums (every lane is one source's Brandes
 * traversal).  bc_out: device float64[nv], overwritten.  Needs about
 * 1,040 + 8 * GRX_BCM_MAX_LEVELS bytes of workspace per vertex (allocated on
 * first use).  Graphs deeper than GRX_BCM_MAX_LEVELS - 1 levels set
 * GRX_ERANGE status (reported by grx_graph_status; use bc() there).  The
 * graph must be symmetric.  With opts->collect_stats, grx_last_stats lists
 * the phases (dir 0 forward, 1 backward), vertices_scanned = the
 * (edge, lane) pairs on shortest paths the phase updated.  n outside 1..64,
 * a bad source or NULL output -> GRX_EINVAL. */
#define GRX_BCM_MAX_LEVELS 16
grx_status bc_multi(grx_graph *g, const int32_t *srcs_host, int n, double *bc_out, const grx_opts *opts,
                    void *stream);

/* cc -- Table 1 CC (Soman et al.'s hooking + pointer jumping).  label_out:
 * device int32[nv], the minimum vertex id of the vertex's component. */
grx_status cc(grx_graph *g, int32_t *label_out, void *stream);

/* pagerank -- Algorithm 3 in the normalised mode with dangling compensation
 * (Sec. 7): r0 = 1/N, then `iters` updates
 *   r'[v] = (1-d)/N + d * (sum_{u in N(v)} r[u]/deg(u) + D/N),
 *   D = sum of r over zero-degree vertices.
 * rank_out: device float[nv].  FP32 arithmetic. */
grx_status pagerank(grx_graph *g, float damping, int iters, float *rank_out, void *stream);

/* grx_pagerank_block -- column-block width of pagerank's gathers.  When the
 * contribution array (4*nv bytes) outgrows L2, each iteration runs one pass
 * per block of 2^shift columns over the row segments that fall in it, so the
 * gathers of a pass hit a slice that stays in L2.  shift <= 0 = no blocks
 * (the default: measured faster on GB300 up to R-MAT scale 26), else 2^shift
 * vertices (must give at most 256 blocks: GRX_EINVAL otherwise).
 * The segment tables (12 bytes per segment) are built on the next pagerank
 * call.  Results agree within the FP32 tolerance either way. */
grx_status grx_pagerank_block(grx_graph *g, int shift);

/* ---- 64-bit vertex ids (graphs past 2^31 vertices) --------------------------
 * Sec. 6.2 / Sec. 7: graphs too large for 32-bit vertex ids use 64-bit ids,
 * at about half the throughput (Table 5).  graph_load_csr64 keeps every id,
 * offset and count 64-bit, for any graph size (a small graph loaded this way
 * exercises the same path); bfs64 traverses such a graph.  The other
 * primitives refuse these graphs with GRX_EINVAL.
 *
 * graph_load_csr64 -- as graph_load_csr, with int64 row_offsets[nv+1] and
 *   int64 col_indices[ne]; nv < 2^42; no weights.  flags: GRX_HOST_PTRS or
 *   GRX_DEVICE_PTRS, optionally GRX_VALIDATE (offsets, column range, sorted
 *   rows, no self-loops, symmetry; synchronises `stream`).  The library
 *   copies the arrays.  grx_graph_info reports nv; graph_free frees it. */
grx_status graph_load_csr64(grx_ctx *ctx, int64_t nv, int64_t ne, const int64_t *row_offsets,
                            const int64_t *col_indices, int flags, void *stream, grx_graph **out);

/* bfs64 -- Algorithm 1 / 2 (direction-optimising with opts->direction AUTO,
 * the Sec. 6.1 rule with alpha / beta / exact_fv) on a graph_load_csr64
 * graph.  depth_out: device int32[nv], hop distance, -1 if unreached.
 * parent_out: NULL or device int64[nv] (src at src, -1 unreached, else a
 * neighbour one level closer).  Persistent loop only, no collect_stats
 * (GRX_EINVAL otherwise); a graph with 32-bit ids -> GRX_EINVAL (use bfs).
 * A push level with more than 2^24 rows of over 1,024 edges sets GRX_ERANGE
 * status.  Uses about 40 bytes of workspace per vertex (first use). */
grx_status bfs64(grx_graph *g, int64_t src, int32_t *depth_out, int64_t *parent_out,
                 const grx_opts *opts, void *stream);

/* ---- allocation-free BFS ---------------------------------------------------
 * bfs_noalloc -- the same traversal as bfs(), for callers that cannot allocate
 * device memory (a host framework that owns the GPU's memory pool and forbids
 * outside allocations, a latency-critical loop where cudaMalloc/cudaFree would
 * synchronise the device, a request path that must not fail with
 * out-of-memory).  The paper has no counterpart: this is a deployment variant.
 *
 * It allocates nothing.  The caller passes device arrays it owns:
 *   row_offsets  int32[nv+1], col_indices int32[ne]: a symmetric CSR as for
 *                graph_load_csr (not copied; must stay valid until the work
 *                on `stream` completes)
 *   depth_out    int32[nv] (as bfs), parent_out int32[nv] or NULL (as bfs)
 *   status_out   int32[1] or NULL: receives the device-side status of this
 *                call (0, or GRX_ETIMEOUT if a bounded wait ran out)
 * All traversal scratch lives in one fixed __device__ array sized for
 * GRX_NOALLOC_MAX_NV vertices (GRX_NOALLOC_SCRATCH_BYTES, about 23.4 MB),
 * which every GPU that loads the library holds until the process exits.  nv
 * above that limit returns GRX_ERANGE; ne must be below 2^31.  opts as for
 * bfs, except that collect_stats must be 0 and loop must be
 * GRX_LOOP_PERSISTENT or GRX_LOOP_HOST: GRX_LOOP_GRAPH (which instantiates a
 * CUDA graph and allocates its argument block) returns GRX_EINVAL.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any CUDA
 * stream capture.  Every call shares the array and clears what it needs;
 * calls whose GPU work overlaps race on it, so order them (one stream). */
#define GRX_NOALLOC_MAX_NV (1 << 19)
#define GRX_NOALLOC_SCRATCH_BYTES 23413632
grx_status bfs_noalloc(int64_t nv, int64_t ne, const int32_t *row_offsets,
                       const int32_t *col_indices, int32_t src, int32_t *depth_out,
                       int32_t *parent_out, int32_t *status_out, const grx_opts *opts,
                       void *stream);

/* ---- per-traversal counters (instrumented runs, collect_stats = 1) ------ */
#define GRX_MAX_LEVELS_STATS 16384
typedef struct {
    int32_t levels;            /* levels run (frontier non-empty) */
    int32_t dir[GRX_MAX_LEVELS_STATS];          /* 0 push, 1 pull */
    int64_t frontier[GRX_MAX_LEVELS_STATS];     /* |Q| entering the level */
    int64_t edges_examined[GRX_MAX_LEVELS_STATS];
    int64_t vertices_scanned[GRX_MAX_LEVELS_STATS]; /* pull: |U| scanned */
    int64_t discovered[GRX_MAX_LEVELS_STATS];   /* vertices labelled */
    int64_t level_ns[GRX_MAX_LEVELS_STATS];     /* device time of the level */
} grx_trav_stats;

/* Synchronise `stream` and copy the counters of the graph's last traversal
 * that ran with collect_stats = 1.  After cc (which always counts), only
 * `levels` is set: the number of hooking rounds.  For multi-source BFS pull
 * levels, vertices_scanned counts the rows of the edge tiles not skipped. */
grx_status grx_last_stats(grx_graph *g, void *stream, grx_trav_stats *out);

/* ---- seeded input generation (device twins of the host generators) ------ */
/* R-MAT edges (Sec. 7): edge i draws SplitMix64 values i*scale + l of stream
 * `seed` for bit levels l; a draw's top 53 bits r pick quadrant A if r < t0,
 * B if r < t1, C if r < t2, else D.  u_out, v_out: device int32[m]. */
grx_status grx_rmat_edges(int scale, int64_t m, uint64_t seed, uint64_t t0, uint64_t t1,
                          uint64_t t2, int32_t *u_out, int32_t *v_out, void *stream);

/* Grid lattice (stand-in for road networks, Sec. 7): width x height vertices,
 * vertex (x,y) = y*width + x.  Horizontal edge (x,y)-(x+1,y) has id
 * y*(width-1)+x, vertical edge (x,y)-(x,y+1) has id height*(width-1) +
 * y*width + x; the edge is deleted when the top 53 bits of draw(seed, id) are
 * below t_del.  Writes u_out, v_out (device int32) and keep_out (device uint8,
 * 1 = kept) for every one of the height*(width-1)+(height-1)*width ids. */
grx_status grx_grid_edges(int64_t width, int64_t height, uint64_t seed, uint64_t t_del,
                          int32_t *u_out, int32_t *v_out, uint8_t *keep_out, void *stream);

/* Symmetric weights: w[e] = 1 + draw(seed, min(u,v)*nv + max(u,v)) mod wmax
 * for CSR edge e = (u, v).  row_offsets int64 device [nv+1]. */
grx_status grx_edge_weights(int64_t nv, int64_t ne, const int64_t *row_offsets,
                            const int32_t *col_indices, uint32_t wmax, uint64_t seed,
                            uint32_t *w_out, void *stream);

/* ---- continuous batching (the serving loop's device side) ---------------
 * A batch is a resident 64-lane traversal of one graph (spec serving
 * pattern; the paper's API runs one source at a time, Appendix A).  Queries
 * join a free lane between level steps and leave when their own frontier is
 * empty; each lane's result equals the single-source bfs()/sssp() result.
 * All calls are ordered on the batch's stream. */
#define GRX_KIND_BFS 0
#define GRX_KIND_SSSP 1

/* Open a batch of `kind` on g; its workspace (grx_batch_footprint bytes) comes
 * from the ctx allocator.  SSSP needs weights. */
grx_status grx_batch_open(grx_graph *g, int kind, void *stream, grx_batch **out);
/* Synchronise the batch's stream and free it. */
grx_status grx_batch_close(grx_batch *b);
/* Admit a query from src into a free lane (GRX_EBUSY if all 64 are busy); it
 * joins at the next level step.  out_dev: caller-owned device int32[nv] (BFS
 * depth, -1 unreached) or uint32[nv] (SSSP distance, UINT32_MAX unreached)
 * that must stay valid until the lane is reported retired. */
grx_status grx_batch_admit(grx_batch *b, int32_t src, void *out_dev, int *lane_out);
/* Enqueue `steps` level steps.  Does not wait. */
grx_status grx_batch_step(grx_batch *b, int steps);
/* Synchronise the stream; report (bit b = lane b) and free the lanes that
 * finished since the last poll; their outputs are complete on return. */
grx_status grx_batch_poll(grx_batch *b, uint64_t *retired_mask_out);
/* Device bytes a batch of `kind` on g needs (for admission by free memory). */
grx_status grx_batch_footprint(const grx_graph *g, int kind, size_t *bytes_out);

/* Device bytes the next bfs_multi (kind GRX_KIND_BFS) or sssp_multi
 * (GRX_KIND_SSSP) call on g will allocate from the ctx allocator for its
 * workspace -- 0 once a previous call allocated it; the caller's output
 * array is not included.  For admission by free memory (the north-star
 * serving loop; the paper sizes its buffers "just enough", Sec. 6.2).
 * NULL argument or bad kind -> GRX_EINVAL. */
grx_status grx_multi_footprint(const grx_graph *g, int kind, size_t *bytes_out);

#ifdef __cplusplus
}
#endif
#endif /* GRX_H */
