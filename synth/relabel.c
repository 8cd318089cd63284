/*
 * relabel.c -- breadth-first locality relabelling of a symmetric CSR, the
 * input preparation the R-MAT workloads prescribe ("degree-sorted + BFS
 * locality reorder").  Input generation only: no arithmetic of the layout
 * method lives here.
 *
 * Rule (the same labels as the library's snap_graph_reorder, written here
 * independently so that the oracle's inputs never pass through the library):
 *   - searches start from the vertex of highest degree not reached yet, ties
 *     broken by smaller id;
 *   - a search is first-in first-out; a vertex taken from the queue appends its
 *     unreached neighbours in the order its row lists them (ascending id);
 *   - new label = position in the visiting order; isolated vertices, reached
 *     by no search but their own, end up last (degree 0 sorts last).
 * Output: perm[old] = new, and the relabelled CSR with every row sorted
 * ascending.
 *
 * Build: compiled with rmat_native.c into one shared library by
 * synth/graphs.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Returns 0, -1 on allocation failure, -2 on a malformed CSR. */
int synth_bfs_relabel(const int64_t *row_ptr, const int32_t *col_idx, int32_t n,
                      int32_t *perm, int64_t *row_ptr_out, int32_t *col_idx_out)
{
    if (n < 1 || row_ptr[0] != 0)
        return -2;
    int64_t dmax = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t d = row_ptr[v + 1] - row_ptr[v];
        if (d < 0)
            return -2;
        if (d > dmax)
            dmax = d;
    }
    int64_t *bucket = (int64_t *)calloc((size_t)dmax + 2, sizeof(int64_t));
    int32_t *seeds = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!bucket || !seeds || !queue) {
        free(bucket);
        free(seeds);
        free(queue);
        return -1;
    }
    /* counting sort by degree, descending; ids ascending within a degree */
    for (int32_t v = 0; v < n; ++v)
        bucket[dmax - (row_ptr[v + 1] - row_ptr[v]) + 1]++;
    for (int64_t d = 1; d <= dmax + 1; ++d)
        bucket[d] += bucket[d - 1];
    for (int32_t v = 0; v < n; ++v)
        seeds[bucket[dmax - (row_ptr[v + 1] - row_ptr[v])]++] = v;
    free(bucket);

    for (int32_t v = 0; v < n; ++v)
        perm[v] = -1;
    int32_t tail = 0;
    for (int32_t q = 0; q < n; ++q) {
        int32_t s = seeds[q];
        if (perm[s] >= 0)
            continue;
        int32_t head = tail;
        perm[s] = tail;
        queue[tail++] = s;
        while (head < tail) {
            int32_t u = queue[head++];
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                int32_t w = col_idx[e];
                if (w < 0 || w >= n) {
                    free(seeds);
                    free(queue);
                    return -2;
                }
                if (perm[w] < 0) {
                    perm[w] = tail;
                    queue[tail++] = w;
                }
            }
        }
    }
    free(seeds);

    /* queue[new] = old; new row u takes old row queue[u], relabelled and sorted */
    row_ptr_out[0] = 0;
    for (int32_t u = 0; u < n; ++u) {
        int32_t old = queue[u];
        row_ptr_out[u + 1] = row_ptr_out[u] + (row_ptr[old + 1] - row_ptr[old]);
    }
    for (int32_t u = 0; u < n; ++u) {
        int32_t old = queue[u];
        int32_t *dst = col_idx_out + row_ptr_out[u];
        int64_t len = row_ptr[old + 1] - row_ptr[old];
        for (int64_t q = 0; q < len; ++q)
            dst[q] = perm[col_idx[row_ptr[old] + q]];
        qsort(dst, (size_t)len, sizeof(int32_t), cmp_i32);
    }
    free(queue);
    return 0;
}
