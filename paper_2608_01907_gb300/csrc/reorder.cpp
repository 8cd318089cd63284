// reorder.cpp -- snap_graph_reorder: breadth-first locality relabelling of a
// symmetric CSR (host code).
//
// Vertices are relabelled in breadth-first order; each search starts from
// the highest-degree vertex not yet reached (ties: smaller id), and a popped
// vertex enqueues its unvisited neighbours in ascending id order.  Vertices
// near each other in the graph thus get nearby labels, so the partners of a
// source bundle share cache lines.  Isolated vertices come last.
//
// The relabelled CSR is filled by scattering each new row u into the rows of
// its neighbours in increasing u: because the graph is symmetric, row v then
// receives exactly v's neighbours, already in ascending order, in O(nnz).
// Row counts are checked against the input; full symmetry is checked by
// snap_layout_create, not here.
#include <stdint.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/snap_layout.h"

namespace snap {
// Records the message returned by snap_last_error (defined in capi.cu).
snap_status reorder_fail(snap_status st, const char *msg);
}

extern "C" snap_status snap_graph_reorder(const int64_t *row_ptr, const int32_t *col_idx, int32_t n,
                                          int32_t *perm_out, int64_t *row_ptr_out, int32_t *col_idx_out) {
    if (!row_ptr || !perm_out || !row_ptr_out) return snap::reorder_fail(SNAP_ERR_INVALID_ARG, "NULL argument");
    if (n < 1) return snap::reorder_fail(SNAP_ERR_INVALID_ARG, "n must be >= 1");
    if (row_ptr[0] != 0) return snap::reorder_fail(SNAP_ERR_INVALID_ARG, "row_ptr[0] must be 0");
    for (int32_t i = 0; i < n; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return snap::reorder_fail(SNAP_ERR_INVALID_ARG, "row_ptr decreases");
    const int64_t nnz = row_ptr[n];
    if (nnz >= ((int64_t)1 << 40)) return snap::reorder_fail(SNAP_ERR_INVALID_ARG, "nnz exceeds 2^40-1");
    if (nnz > 0 && (!col_idx || !col_idx_out)) return snap::reorder_fail(SNAP_ERR_INVALID_ARG, "NULL col_idx");
    for (int64_t e = 0; e < nnz; ++e)
        if (col_idx[e] < 0 || col_idx[e] >= n)
            return snap::reorder_fail(SNAP_ERR_INVALID_ARG, "column outside [0, n)");
    try {
        std::vector<int32_t> by_degree((size_t)n);
        std::iota(by_degree.begin(), by_degree.end(), 0);
        std::stable_sort(by_degree.begin(), by_degree.end(), [&](int32_t a, int32_t b) {
            return row_ptr[a + 1] - row_ptr[a] > row_ptr[b + 1] - row_ptr[b];
        });
        std::vector<int32_t> order;   // new -> old
        order.reserve((size_t)n);
        std::vector<int32_t> new_of_old((size_t)n, -1);
        for (int32_t seed : by_degree) {
            if (new_of_old[(size_t)seed] >= 0) continue;
            size_t head = order.size();
            new_of_old[(size_t)seed] = (int32_t)order.size();
            order.push_back(seed);
            while (head < order.size()) {
                const int32_t u = order[head++];
                for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                    const int32_t v = col_idx[e];
                    if (new_of_old[(size_t)v] < 0) {
                        new_of_old[(size_t)v] = (int32_t)order.size();
                        order.push_back(v);
                    }
                }
            }
        }
        row_ptr_out[0] = 0;
        for (int32_t u = 0; u < n; ++u) {
            const int32_t old = order[(size_t)u];
            row_ptr_out[u + 1] = row_ptr_out[u] + (row_ptr[old + 1] - row_ptr[old]);
        }
        std::vector<int64_t> cursor(row_ptr_out, row_ptr_out + n);
        for (int32_t u = 0; u < n; ++u) {
            const int32_t old = order[(size_t)u];
            for (int64_t e = row_ptr[old]; e < row_ptr[old + 1]; ++e) {
                const int32_t v = new_of_old[(size_t)col_idx[e]];
                if (cursor[(size_t)v] >= row_ptr_out[v + 1])
                    return snap::reorder_fail(SNAP_ERR_INVALID_ARG, "the CSR is not symmetric");
                col_idx_out[cursor[(size_t)v]++] = u;
            }
        }
        for (int32_t v = 0; v < n; ++v)
            if (cursor[(size_t)v] != row_ptr_out[v + 1])
                return snap::reorder_fail(SNAP_ERR_INVALID_ARG, "the CSR is not symmetric");
        for (int32_t old = 0; old < n; ++old) perm_out[old] = new_of_old[(size_t)old];
    } catch (const std::bad_alloc &) {
        return snap::reorder_fail(SNAP_ERR_OUT_OF_MEMORY, "host allocation failed in snap_graph_reorder");
    }
    return SNAP_OK;
}
