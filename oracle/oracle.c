/*
 * Plain CPU oracle for the frontier-traversal primitives of "Multi-GPU Graph
 * Analytics" (Pan, Wang, Wu, Yang, Owens; arXiv 1504.04804).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header, table or helper with the CUDA library and includes nothing
 * from it; the library never calls it.
 *
 * Graph convention for every routine: a CSR adjacency with nv vertices,
 * row_offsets[nv+1] (int64, non-decreasing, row_offsets[0]==0) and
 * col_indices[row_offsets[nv]] (int32 vertex ids).  The graphs the paper
 * measures are undirected (Sec. 7: "converted to undirected", self-loops and
 * duplicates removed), so the CSR lists every undirected edge in both rows.
 *
 * Every routine returns 0 on success and a negative number on bad input; none
 * allocates more than O(nv + ne) host memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_ERANGE (-5)

/* ------------------------------------------------------------------------ */
/* BFS.  Algorithm 1 (Sec. 4) advances the frontier one hop per iteration    */
/* and stops when the frontier is empty; the label it leaves on a vertex is  */
/* its hop distance from the source.  The plain definition of that result is */
/* the textbook FIFO-queue BFS below.  Unreached vertices keep label -1.     */
/* ------------------------------------------------------------------------ */
int oracle_bfs(int64_t nv, const int64_t *row_offsets, const int32_t *col_indices,
               int32_t src, int32_t *depth)
{
    if (nv < 0 || !row_offsets || !depth || (nv > 0 && !col_indices && row_offsets[nv] > 0))
        return OR_EINVAL;
    if (src < 0 || (int64_t)src >= nv) return OR_EINVAL;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    if (!queue) return OR_ENOMEM;
    for (int64_t v = 0; v < nv; ++v) depth[v] = -1;
    int64_t head = 0, tail = 0;
    depth[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
            int32_t v = col_indices[e];
            if (depth[v] < 0) {
                depth[v] = depth[u] + 1;
                queue[tail++] = v;
            }
        }
    }
    free(queue);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* SSSP.  Table 1 (Sec. 4) lists SSSP with min-combination of labels         */
/* (Sec. 3: the combiner keeps the smaller distance); Sec. 7 draws integer   */
/* edge weights.  The exact result is the shortest-path distance, defined    */
/* here by Dijkstra's algorithm with a binary min-heap (lazy deletion).      */
/* Distances are accumulated in uint64; a finite distance that does not fit  */
/* below UINT32_MAX is reported as OR_ERANGE.  Unreached = UINT32_MAX.       */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t d; int32_t v; } heap_item;

static void heap_push(heap_item *h, int64_t *n, heap_item it)
{
    int64_t i = (*n)++;
    h[i] = it;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].d <= h[i].d) break;
        heap_item t = h[p]; h[p] = h[i]; h[i] = t;
        i = p;
    }
}

static heap_item heap_pop(heap_item *h, int64_t *n)
{
    heap_item top = h[0];
    h[0] = h[--(*n)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *n && h[l].d < h[m].d) m = l;
        if (r < *n && h[r].d < h[m].d) m = r;
        if (m == i) break;
        heap_item t = h[m]; h[m] = h[i]; h[i] = t;
        i = m;
    }
    return top;
}

int oracle_sssp(int64_t nv, const int64_t *row_offsets, const int32_t *col_indices,
                const uint32_t *weights, int32_t src, uint32_t *dist)
{
    if (nv < 0 || !row_offsets || !dist || !weights) return OR_EINVAL;
    if (src < 0 || (int64_t)src >= nv) return OR_EINVAL;
    int64_t ne = row_offsets[nv];
    uint64_t *d = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nv > 0 ? nv : 1));
    unsigned char *done = (unsigned char *)calloc((size_t)(nv > 0 ? nv : 1), 1);
    /* every push corresponds to one improving edge relaxation or the source */
    heap_item *heap = (heap_item *)malloc(sizeof(heap_item) * (size_t)(ne + 1));
    if (!d || !done || !heap) { free(d); free(done); free(heap); return OR_ENOMEM; }
    const uint64_t INF = UINT64_MAX;
    for (int64_t v = 0; v < nv; ++v) d[v] = INF;
    int64_t n = 0;
    d[src] = 0;
    heap_push(heap, &n, (heap_item){0, src});
    while (n > 0) {
        heap_item it = heap_pop(heap, &n);
        int32_t u = it.v;
        if (done[u]) continue;
        done[u] = 1;
        for (int64_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
            int32_t v = col_indices[e];
            uint64_t nd = d[u] + (uint64_t)weights[e];
            if (nd < d[v]) {
                d[v] = nd;
                heap_push(heap, &n, (heap_item){nd, v});
            }
        }
    }
    int rc = OR_OK;
    for (int64_t v = 0; v < nv; ++v) {
        if (d[v] == INF) dist[v] = UINT32_MAX;
        else if (d[v] >= (uint64_t)UINT32_MAX) { dist[v] = UINT32_MAX; rc = OR_ERANGE; }
        else dist[v] = (uint32_t)d[v];
    }
    free(d); free(done); free(heap);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Connected components.  The paper runs Soman et al.'s hooking and pointer  */
/* jumping (Sec. 2, Table 1).  The result it computes is the partition into  */
/* connected components; the canonical label chosen for each component is    */
/* its minimum vertex id.  Defined here with a union-find forest: find uses  */
/* path halving, union links the larger root below the smaller one, so every */
/* root is the minimum id of its tree.                                       */
/* ------------------------------------------------------------------------ */
static int32_t uf_find(int32_t *parent, int32_t x)
{
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

int oracle_cc(int64_t nv, const int64_t *row_offsets, const int32_t *col_indices,
              int32_t *label)
{
    if (nv < 0 || !row_offsets || !label) return OR_EINVAL;
    for (int64_t v = 0; v < nv; ++v) label[v] = (int32_t)v;
    for (int64_t u = 0; u < nv; ++u) {
        for (int64_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
            int32_t ru = uf_find(label, (int32_t)u);
            int32_t rv = uf_find(label, col_indices[e]);
            if (ru == rv) continue;
            if (ru < rv) label[rv] = ru; else label[ru] = rv;
        }
    }
    for (int64_t v = 0; v < nv; ++v) label[v] = uf_find(label, (int32_t)v);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* PageRank.  Algorithm 3 (Sec. 4): each iteration accumulates every         */
/* vertex's rank share into its neighbours, then updates the ranks.  The     */
/* normalised mode with compensation (Sec. 7, correctness check) spreads the */
/* rank of zero-out-degree vertices evenly over all vertices, so the ranks   */
/* sum to 1.  Written as the power iteration, starting from r = 1/N:         */
/*     D     = sum of r[u] over u with deg(u) == 0                           */
/*     r'[v] = (1-d)/N + d * ( sum over edges u->v of r[u]/deg(u) + D/N )    */
/* run for exactly `iters` updates, in double precision, pushing each        */
/* vertex's share along its out-edges.                                       */
/* ------------------------------------------------------------------------ */
int oracle_pagerank(int64_t nv, const int64_t *row_offsets, const int32_t *col_indices,
                    double damping, int iters, double *rank)
{
    if (nv <= 0 || !row_offsets || !rank || iters < 0) return OR_EINVAL;
    double *acc = (double *)malloc(sizeof(double) * (size_t)nv);
    if (!acc) return OR_ENOMEM;
    const double N = (double)nv;
    for (int64_t v = 0; v < nv; ++v) rank[v] = 1.0 / N;
    for (int it = 0; it < iters; ++it) {
        double dangling = 0.0;
        for (int64_t v = 0; v < nv; ++v) acc[v] = 0.0;
        for (int64_t u = 0; u < nv; ++u) {
            int64_t deg = row_offsets[u + 1] - row_offsets[u];
            if (deg == 0) { dangling += rank[u]; continue; }
            double share = rank[u] / (double)deg;
            for (int64_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e)
                acc[col_indices[e]] += share;
        }
        for (int64_t v = 0; v < nv; ++v)
            rank[v] = (1.0 - damping) / N + damping * (acc[v] + dangling / N);
    }
    free(acc);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Betweenness centrality.  Table 1 (Sec. 4) lists BC as a forward traversal */
/* plus a backward pass over the same levels (W = 2|E|, S ~ D/2), the GPU    */
/* scheme of McLaughlin and Bader (Sec. 2), which computes Brandes'          */
/* dependencies.  For a source s on the undirected graph:                    */
/*   sigma[v]  = number of shortest s-v paths (sigma[s] = 1);                */
/*   delta[v]  = sum over t != s, v of sigma_st(v) / sigma_st, obtained by   */
/*               delta[v] = sum over neighbours w one level deeper of        */
/*                          sigma[v] / sigma[w] * (1 + delta[w]),            */
/*               processing vertices in non-increasing distance from s.      */
/* bc[v] is the sum of delta over the given sources (the source itself gets  */
/* nothing from its own traversal); ordered pairs, so the all-sources sum on */
/* an undirected graph counts each unordered pair twice.  Everything is      */
/* float64.  sigma_last (optional) receives sigma of the last source, 0 for  */
/* unreached vertices.                                                       */
/* ------------------------------------------------------------------------ */
int oracle_bc(int64_t nv, const int64_t *row_offsets, const int32_t *col_indices,
              const int32_t *srcs, int64_t n_srcs, double *bc, double *sigma_last)
{
    if (nv <= 0 || !row_offsets || !bc || n_srcs < 0 || (n_srcs > 0 && !srcs)) return OR_EINVAL;
    for (int64_t i = 0; i < n_srcs; ++i)
        if (srcs[i] < 0 || (int64_t)srcs[i] >= nv) return OR_EINVAL;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    double *sigma = (double *)malloc(sizeof(double) * (size_t)nv);
    double *delta = (double *)malloc(sizeof(double) * (size_t)nv);
    if (!order || !dist || !sigma || !delta) {
        free(order); free(dist); free(sigma); free(delta);
        return OR_ENOMEM;
    }
    for (int64_t v = 0; v < nv; ++v) bc[v] = 0.0;
    for (int64_t i = 0; i < n_srcs; ++i) {
        const int32_t s = srcs[i];
        for (int64_t v = 0; v < nv; ++v) {
            dist[v] = -1;
            sigma[v] = 0.0;
            delta[v] = 0.0;
        }
        /* forward: BFS in FIFO order; order[] lists vertices by distance */
        int64_t head = 0, tail = 0;
        dist[s] = 0;
        sigma[s] = 1.0;
        order[tail++] = s;
        while (head < tail) {
            const int32_t u = order[head++];
            for (int64_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
                const int32_t w = col_indices[e];
                if (dist[w] < 0) {
                    dist[w] = dist[u] + 1;
                    order[tail++] = w;
                }
                if (dist[w] == dist[u] + 1) sigma[w] += sigma[u];
            }
        }
        /* backward: vertices in reverse BFS order, each one's delta complete
           before any neighbour one level closer to s reads it */
        for (int64_t k = tail - 1; k >= 0; --k) {
            const int32_t v = order[k];
            double sum = 0.0;
            for (int64_t e = row_offsets[v]; e < row_offsets[v + 1]; ++e) {
                const int32_t w = col_indices[e];
                if (dist[w] == dist[v] + 1) sum += sigma[v] / sigma[w] * (1.0 + delta[w]);
            }
            delta[v] = sum;
            if (v != s) bc[v] += delta[v];
        }
        if (sigma_last && i == n_srcs - 1)
            for (int64_t v = 0; v < nv; ++v) sigma_last[v] = sigma[v];
    }
    free(order); free(dist); free(sigma); free(delta);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Invariant checkers.  These hold at any size, so they let a full-size run  */
/* be checked where only sampled sources can be re-solved exactly.  Each     */
/* returns the number of violations found (0 = valid), or a negative error.  */
/* ------------------------------------------------------------------------ */

/* BFS depths: depth[src]==0 and no other vertex has depth 0; on every edge
 * (u,v) either both ends are unreached or both reached with
 * |depth[u]-depth[v]| <= 1; every reached v != src has a neighbour at
 * depth[v]-1.  Together these fix the depths uniquely: following
 * predecessors from any reached vertex descends one level per step and can
 * only end at the one depth-0 vertex, the source, so depth[v] is the length
 * of a path from src (>= the hop distance); and the +-1 rule along a
 * shortest path bounds it by the hop distance.  If parent != NULL,
 * parent[v] must be a neighbour of v at depth[v]-1 for reached v != src,
 * parent[src]==src, and -1 for unreached v. */
int64_t oracle_check_bfs(int64_t nv, const int64_t *row_offsets, const int32_t *col_indices,
                         int32_t src, const int32_t *depth, const int32_t *parent)
{
    if (nv <= 0 || src < 0 || (int64_t)src >= nv) return OR_EINVAL;
    int64_t bad = 0;
    if (depth[src] != 0) ++bad;
    for (int64_t v = 0; v < nv; ++v) {
        int32_t dv = depth[v];
        if (dv < -1) { ++bad; continue; }
        if (dv == 0 && v != src) ++bad;          /* a second root */
        int has_pred = 0, parent_ok = 0;
        for (int64_t e = row_offsets[v]; e < row_offsets[v + 1]; ++e) {
            int32_t u = col_indices[e];
            int32_t du = depth[u];
            if ((dv < 0) != (du < 0)) { ++bad; continue; }
            if (dv >= 0) {
                int32_t diff = dv - du;
                if (diff > 1 || diff < -1) ++bad;
                if (du == dv - 1) has_pred = 1;
                if (parent && parent[v] == u && du == dv - 1) parent_ok = 1;
            }
        }
        if (dv > 0 && !has_pred) ++bad;
        if (parent) {
            if (v == src) { if (parent[v] != src) ++bad; }
            else if (dv < 0) { if (parent[v] != -1) ++bad; }
            else if (!parent_ok) ++bad;
        }
    }
    return bad;
}

/* SSSP distances: dist[src]==0; dist[v] <= dist[u] + w(u,v) on every edge
 * (triangle inequality, in uint64); an unreached vertex has no reached
 * neighbour; and every reached vertex is reachable from src along tight
 * edges (dist[v] == dist[u] + w(u,v)), found by a FIFO sweep from src over
 * tight edges.  The sweep makes each dist[v] the length of a real path
 * (>= the shortest distance) and the triangle inequality along a shortest
 * path bounds it from above, so the distances are the shortest ones.  A
 * local "has a tight edge" test would not do: with zero weights a component
 * away from src could carry distance 0 throughout. */
int64_t oracle_check_sssp(int64_t nv, const int64_t *row_offsets, const int32_t *col_indices,
                          const uint32_t *weights, int32_t src, const uint32_t *dist)
{
    if (nv <= 0 || src < 0 || (int64_t)src >= nv) return OR_EINVAL;
    int64_t bad = 0;
    if (dist[src] != 0) ++bad;
    for (int64_t v = 0; v < nv; ++v) {
        for (int64_t e = row_offsets[v]; e < row_offsets[v + 1]; ++e) {
            int32_t u = col_indices[e];
            /* edge (v,u) with weight w: the undirected weight is the same both ways */
            if (dist[u] == UINT32_MAX) { if (dist[v] != UINT32_MAX) ++bad; continue; }
            uint64_t via = (uint64_t)dist[u] + weights[e];
            if (dist[v] == UINT32_MAX || (uint64_t)dist[v] > via) ++bad;
        }
    }
    if (dist[src] != 0) return bad;
    /* tight-edge reachability from src */
    uint8_t *seen = (uint8_t *)calloc((size_t)nv, 1);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    if (!seen || !queue) { free(seen); free(queue); return OR_ENOMEM; }
    int64_t head = 0, tail = 0;
    seen[src] = 1;
    queue[tail++] = src;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
            int32_t v = col_indices[e];
            if (!seen[v] && dist[v] != UINT32_MAX &&
                (uint64_t)dist[v] == (uint64_t)dist[u] + weights[e]) {
                seen[v] = 1;
                queue[tail++] = v;
            }
        }
    }
    for (int64_t v = 0; v < nv; ++v)
        if (dist[v] != UINT32_MAX && !seen[v]) ++bad;
    free(seen);
    free(queue);
    return bad;
}

/* CC labels: label[v] must be the smallest vertex id of v's connected
 * component.  The components are found here by FIFO sweeps (a method other
 * than the union-find of oracle_cc): vertices are taken in increasing id
 * order, and each one not yet swept starts a sweep of its whole component, so
 * it is that component's minimum; every vertex the sweep reaches must carry
 * it as its label.  This rejects wrong representatives and merged or split
 * components alike. */
int64_t oracle_check_cc(int64_t nv, const int64_t *row_offsets, const int32_t *col_indices,
                        const int32_t *label)
{
    if (nv <= 0) return OR_EINVAL;
    uint8_t *seen = (uint8_t *)calloc((size_t)nv, 1);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    if (!seen || !queue) { free(seen); free(queue); return OR_ENOMEM; }
    int64_t bad = 0;
    for (int64_t r = 0; r < nv; ++r) {
        if (seen[r]) continue;
        int64_t head = 0, tail = 0;
        seen[r] = 1;
        queue[tail++] = (int32_t)r;
        while (head < tail) {
            int32_t u = queue[head++];
            if ((int64_t)label[u] != r) ++bad;
            for (int64_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
                int32_t v = col_indices[e];
                if (!seen[v]) { seen[v] = 1; queue[tail++] = v; }
            }
        }
    }
    free(seen);
    free(queue);
    return bad;
}
