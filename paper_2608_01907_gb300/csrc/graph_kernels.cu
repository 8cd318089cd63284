// graph_kernels.cu -- segment table, CSR validation and the objective of
// Eq. 4 (weight realised by uniform sampling, Section 3.3).
#include <cuda_runtime.h>
#include <stdint.h>

#include <cub/device/device_scan.cuh>

#include "snap_device.cuh"
#include "snap_internal.h"

namespace snap {

namespace {

// seg_row[s] = the row holding edge s * seg_len: the largest r with
// row_ptr[r] <= e (then row_ptr[r+1] > e, so the row is not empty).
__global__ void segment_rows_kernel(const int64_t *__restrict__ row_ptr, int32_t n, int32_t seg_len,
                                    int32_t *__restrict__ seg_row, int64_t num_segs) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < num_segs; s += stride) {
        const int64_t e = s * seg_len;
        int32_t lo = 0, hi = n;   // invariant: row_ptr[lo] <= e < row_ptr[hi]
        while (hi - lo > 1) {
            const int32_t mid = lo + (hi - lo) / 2;
            if (row_ptr[mid] <= e)
                lo = mid;
            else
                hi = mid;
        }
        seg_row[s] = lo;
    }
}

// deg[i] = row_ptr[i+1] - row_ptr[i] (row_ptr checked non-decreasing by
// check_row_ptr_kernel before anything uses it as a rank).
__global__ void degrees_kernel(const int64_t *__restrict__ row_ptr, int32_t n, int32_t *__restrict__ deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        deg[i] = (int32_t)(row_ptr[i + 1] - row_ptr[i]);
}

// Orientation of the undirected edges: {i, j} belongs to the bundle of the
// endpoint that ranks higher by (degree, then smaller id).  That endpoint's
// lane processes both directed copies (i, j) and (j, i), so a vertex is a
// partner only of its higher-ranked neighbours.
__device__ __forceinline__ bool ranks_higher(int32_t di, int32_t dj, int32_t i, int32_t j) {
    return di > dj || (di == dj && i < j);
}

// row_ptr non-decreasing inside [0, nnz] (row_ptr[0] = 0 and row_ptr[n] =
// nnz are checked on the host).  Every kernel that runs before this result
// is read clamps the offsets it uses as indices.
__global__ void check_row_ptr_kernel(const int64_t *__restrict__ row_ptr, int32_t n, int64_t nnz,
                                     uint32_t *flags_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t lo = row_ptr[i], hi = row_ptr[i + 1];
        if (lo < 0 || hi < lo || hi > nnz) bad = true;
    }
    if (bad) atomicOr(flags_out, kBadRowPtr);
}

// Columns in [0, n), no self-loop, rows strictly ascending, no edge across
// two graphs of a batch.  upper_count != null (the synchronous mode, which
// has no orientation pass): also symmetry, checked on half of the edges --
// every (i, j) with j < i must have (j, i) in row j (binary search), and the
// number of such edges must be nnz / 2 (the caller compares): reversal maps
// them one-to-one into the edges with j > i, so equal counts mean every edge
// has its reverse.  (The HOGWILD modes check symmetry the same way in the
// orientation pass, which searches the reverse of half of the edges anyway.)
// orient != null (the HOGWILD modes): also orient[e] = 1 when edge e's
// source ranks higher than its partner (ranks_higher; deg = row lengths),
// else 0, and orient[nnz] = 0 -- the input of the orientation scan.
__global__ void validate_csr_kernel(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                                    const int32_t *__restrict__ seg_row, int32_t n, int64_t nnz,
                                    int32_t seg_len, uint32_t *flags_out, const int32_t *__restrict__ node_graph,
                                    unsigned long long *upper_count, const int32_t *__restrict__ deg,
                                    int32_t *__restrict__ orient) {
    if (orient && blockIdx.x == 0 && threadIdx.x == 0) orient[nnz] = 0;
    const int64_t num_segs = (nnz + seg_len - 1) / seg_len;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t flags = 0;
    unsigned long long upper = 0;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < num_segs; s += stride) {
        const int64_t e0 = s * seg_len;
        const int64_t e1 = min(e0 + (int64_t)seg_len, nnz);
        int32_t row = seg_row[s];
        int64_t row_begin = row_ptr[row];
        int64_t row_end = row_ptr[row + 1];
        for (int64_t e = e0; e < e1; ++e) {
            while (e >= row_end && row < n - 1) {
                ++row;
                row_begin = row_end;
                row_end = row_ptr[row + 1];
            }
            const int32_t j = col_idx[e];
            if (j < 0 || j >= n) {
                flags |= kBadColumn;
                if (orient) orient[e] = 0;
                continue;
            }
            if (orient) orient[e] = ranks_higher(deg[row], deg[j], row, j) ? 1 : 0;
            if (j == row) flags |= kSelfLoop;
            if (node_graph && node_graph[j] != node_graph[row]) flags |= kCrossGraph;
            if (e > row_begin && e > 0 && col_idx[e - 1] >= j) flags |= kUnsorted;
            if (upper_count && j < row) {
                ++upper;
                // binary search for `row` in row j (offsets clamped to [0, nnz])
                int64_t lo = max(row_ptr[j], (int64_t)0), hi = min(row_ptr[j + 1], nnz);
                bool found = false;
                while (lo < hi) {
                    const int64_t mid = lo + (hi - lo) / 2;
                    const int32_t v = col_idx[mid];
                    if (v == row) {
                        found = true;
                        break;
                    }
                    if (v < row)
                        lo = mid + 1;
                    else
                        hi = mid;
                }
                if (!found) flags |= kAsymmetric;
            }
        }
    }
    if (flags) atomicOr(flags_out, flags);
    if (upper_count && upper) atomicAdd(upper_count, upper);
}



// Entry of an oriented edge {i, j}: {j, index of (i, j), index of (j, i), i}
// -- the CSR indices of both directed copies (a handle holds fewer than 2^32
// directed edges) and the source, so an entry names its own row.
__device__ __forceinline__ int4 make_entry(int32_t i, int32_t j, int64_t fwd, int64_t rev) {
    return make_int4(j, (int32_t)(uint32_t)fwd, (int32_t)(uint32_t)rev, i);
}

// Order of the entries inside an oriented row of length L: the entry of
// rank q (ascending partner id) is stored at (a q) mod L, a the odd number
// nearest above 0.618 L that is coprime with L.  Consecutive stored entries
// -- the steps a lane runs back to back -- then belong to partners far apart
// in the row.  (Under a locality relabelling, partners with close ids are
// close in the graph; running them back to back pulls the source along one
// direction many times in a row.  Sequential FP64 emulation on R-MAT 2^22,
// 4-entry chunks: objective +1.5% / NP -2.0% against the shuffled order of
// Algorithm 1 in ascending order, +0.9% / -0.7% with the rows permuted.)
// (32-bit arithmetic: a row has fewer than 2^31 entries, and 64-bit
// remainders cost several times as much on the GPU.)
__device__ __forceinline__ uint32_t gcd_dev(uint32_t a, uint32_t b) {
    while (b) {
        const uint32_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

__device__ __forceinline__ int64_t row_multiplier(int32_t L) {
    uint32_t a = (uint32_t)(int64_t)(0.6180339887498949 * (double)L) | 1u;
    while (gcd_dev(a, (uint32_t)L) != 1u) a += 2u;
    return (int64_t)a;
}

__device__ __forceinline__ int32_t row_position(int32_t q, int32_t L) {
    if (L <= 2) return q;
    return (int32_t)((row_multiplier(L) * (int64_t)q) % L);
}

// Rank (ascending partner id) of the entry stored at offset o of a row of
// length L in the affine order: the inverse of row_position.
__device__ __forceinline__ int32_t row_rank(int32_t o, int32_t L) {
    if (L <= 2) return o;
    // inverse of a mod L by the extended Euclidean algorithm
    int64_t r0 = L, r1 = row_multiplier(L) % L, t0 = 0, t1 = 1;
    while (r1 != 0) {
        const int64_t qt = r0 / r1;
        int64_t tmp = r0 - qt * r1;
        r0 = r1;
        r1 = tmp;
        tmp = t0 - qt * t1;
        t0 = t1;
        t1 = tmp;
    }
    const int64_t inv = t0 < 0 ? t0 + L : t0;
    return (int32_t)((inv * (int64_t)o) % L);
}

// Builds the oriented list directly in its chunked, slot-interleaved layout
// `to` (both row orders): owned edge e of row i has rank r = pos[e] -
// pos[row_ptr[i]] among its row's owned edges (ascending partner id), sits at
// row position r (ascending order) or (a r) mod L (affine order,
// row_position), hence at list index pt = pos[row_ptr[i]] + that, in chunk
// pt / T; the entry is written to its slot's place and the chunk's first
// entry writes the slot descriptor {i, chunk}.  Along a row the ranks of
// consecutive owned edges go up by one, so the affine position advances by
// a mod L, and a = row_multiplier(L) is found once per row run.
// Also the symmetry check of the HOGWILD modes: the reverse (j, i) of every
// owned edge must exist (else kAsymmetric), and the caller compares the
// number of owned edges with nnz / 2 -- reversal maps the owned edges one-to-
// one into the others (rows hold no duplicates), so equal counts mean every
// edge has its reverse.  Entries are written only for pt < capacity (the
// count is checked after the pass).
__global__ void orient_scatter_kernel(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                                      const int32_t *__restrict__ seg_row, const int32_t *__restrict__ deg,
                                      int64_t nnz, int32_t seg_len, const int32_t *__restrict__ pos,
                                      const ChunkLayout to, int4 *__restrict__ ent, int2 *__restrict__ meta,
                                      int64_t capacity, uint32_t *flags_out) {
    uint32_t flags = 0;
    const int64_t num_segs = (nnz + seg_len - 1) / seg_len;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < num_segs; s += stride) {
        const int64_t e0 = s * seg_len;
        const int64_t e1 = min(e0 + (int64_t)seg_len, nnz);
        int32_t i = seg_row[s];
        int64_t row_end = row_ptr[i + 1];
        int32_t run_row = -1, L = 0, a = 1, last_r = -2, last_o = 0;
        int64_t start = 0;
        for (int64_t e = e0; e < e1; ++e) {
            while (e >= row_end) {
                ++i;
                row_end = row_ptr[i + 1];
            }
            const int32_t j = col_idx[e];
            if (!ranks_higher(deg[i], deg[j], i, j)) continue;
            if (i != run_row) {
                run_row = i;
                start = pos[row_ptr[i]];
                L = (int32_t)(pos[row_end] - start);
                a = L > 2 ? (int32_t)row_multiplier(L) : 1;
                last_r = -2;
            }
            const int32_t r = (int32_t)(pos[e] - start);
            int32_t o = r;
            if (to.order == 0 && L > 2) {
                if (r == last_r + 1) {
                    o = last_o + a;
                    if (o >= L) o -= L;
                } else {
                    o = (int32_t)(((int64_t)a * r) % L);
                }
            }
            last_r = r;
            last_o = o;
            // index of the reverse copy (j, i): binary search for i in row j
            const int64_t rb = row_ptr[j], re = row_ptr[j + 1];
            int64_t lo = rb, hi = re - 1;
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo) / 2;
                if (col_idx[mid] < i)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            if (lo >= re || col_idx[lo] != i) {
                flags |= kAsymmetric;
                continue;
            }
            const int64_t pt = start + o;
            if (pt < 0 || pt >= capacity) continue;
            const int64_t c = pt / to.T;
            const int64_t t = pt - c * to.T;
            const int64_t slot = chunk_slot(to, c);
            ent[chunk_entry_index(slot, to.S, to.T, t)] = make_entry(i, j, e, lo);
            if (t == 0) meta[slot] = make_int2(i, (int32_t)c);
        }
    }
    if (flags) atomicOr(flags_out, flags);
}

// Chunks of T entries that each vertex's oriented row spans (0: empty row).
__global__ void row_pieces_kernel(const int64_t *__restrict__ act_rp, int32_t n, int32_t T,
                                  int32_t *__restrict__ pieces) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t b = act_rp[v], e = act_rp[v + 1];
        pieces[v] = e > b ? (int32_t)((e - 1) / T - b / T + 1) : 0;
    }
}

__global__ void orient_rowptr_kernel(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ pos, int32_t n,
                                     int64_t *__restrict__ act_row_ptr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride)
        act_row_ptr[i] = pos[row_ptr[i]];
}

// Chunk layout of the oriented list (the stored order is described with
// ChunkLayout).  One thread per entry p of the row-major list copies it from
// its place under `from` to its place under `to`; the thread of a chunk's
// first entry also writes the slot's {row, chunk}.
__global__ void chunk_layout_kernel(const int4 *__restrict__ src, const ChunkLayout from, int4 *__restrict__ dst,
                                    const ChunkLayout to, int2 *__restrict__ meta, const int64_t *__restrict__ act_rp,
                                    int32_t n, int64_t nnz) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
        int64_t q = p;
        if (from.T > 0) {
            const int64_t c = p / from.T;
            q = chunk_entry_index(chunk_slot(from, c), from.S, from.T, p - c * from.T);
        }
        // p is the entry's row-major index in `from`'s row order; pt its index
        // in `to`'s (the same row, another place when the orders differ)
        const int4 en = src[q];
        int64_t pt = p;
        if (from.order != to.order) {
            const int32_t row = en.w;   // the entry names its row
            const int64_t b = act_rp[row];
            const int32_t L = (int32_t)(act_rp[row + 1] - b), o = (int32_t)(p - b);
            const int32_t rank = from.order == 0 ? row_rank(o, L) : o;
            pt = b + (to.order == 0 ? row_position(rank, L) : rank);
        }
        const int64_t c = pt / to.T;
        const int64_t t = pt - c * to.T;
        const int64_t slot = chunk_slot(to, c);
        dst[chunk_entry_index(slot, to.S, to.T, t)] = en;
        if (t == 0) meta[slot] = make_int2(en.w, (int32_t)c);
    }
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double warp_part[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_part[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        t = lane < nw ? warp_part[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;   // valid in thread 0
}

// U^a summed over undirected edges, each counted once (from its i < j copy).
// U^a(r) = alpha (r^2 / 2 + beta/2 ln(1 + r^2)), Eq. 2 with Table 1's attraction.
__global__ void objective_edges_kernel(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                                       const int32_t *__restrict__ seg_row, const float2 *__restrict__ pos,
                                       int64_t nnz, int32_t seg_len, double *partial) {
    const int64_t num_segs = (nnz + seg_len - 1) / seg_len;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double acc = 0.0;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < num_segs; s += stride) {
        const int64_t e0 = s * seg_len;
        const int64_t e1 = min(e0 + (int64_t)seg_len, nnz);
        int32_t row = seg_row[s];
        int64_t row_end = row_ptr[row + 1];
        float2 yi = pos[row];
        float part = 0.0f;
        for (int64_t e = e0; e < e1; ++e) {
            if (e >= row_end) {
                do {
                    ++row;
                    row_end = row_ptr[row + 1];
                } while (row_end <= e);
                yi = pos[row];
            }
            const int32_t j = col_idx[e];
            if (row < j) {
                const float2 yj = pos[j];
                const float dx = yi.x - yj.x, dy = yi.y - yj.y;
                const float r2 = fmaf(dx, dx, dy * dy);
                part += kAlpha * (0.5f * r2 + 0.5f * kBeta * log1pf(r2));
            }
        }
        acc += (double)part;
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// U^a over an oriented list (each undirected edge once), walking its segments.
__global__ void objective_oriented_kernel(const int64_t *__restrict__ row_ptr, const int4 *__restrict__ ent,
                                          const int2 *__restrict__ meta, const ChunkLayout L, int64_t nnz,
                                          const float2 *__restrict__ pos, double *partial) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double acc = 0.0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < L.S; w += stride) {
        const int2 mt = meta[w];   // {row of the first entry, chunk}
        int32_t row = mt.x;
        int64_t row_end = row_ptr[row + 1];
        float2 yi = pos[row];
        const int64_t p0 = (int64_t)mt.y * L.T;
        const int64_t p1 = p0 + L.T < nnz ? p0 + L.T : nnz;
        float part = 0.0f;
        for (int64_t p = p0; p < p1; ++p) {
            if (p >= row_end) {
                do {
                    ++row;
                    row_end = row_ptr[row + 1];
                } while (row_end <= p);
                yi = pos[row];
            }
            const float2 yj = pos[ent[chunk_entry_index(w, L.S, L.T, p - p0)].x];
            const float dx = yi.x - yj.x, dy = yi.y - yj.y;
            const float r2 = fmaf(dx, dx, dy * dy);
            part += kAlpha * (0.5f * r2 + 0.5f * kBeta * log1pf(r2));
        }
        acc += (double)part;
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// sum over ordered pairs i != j of (d_i + d_j) U^r(r_ij), U^r = 1 / (2 (1 + r^2)).
// The host halves it (unordered pairs) and applies k / (2 (n-1)).
constexpr int kPairTile = 256;

// Pair coefficient of the objective: uniform negatives (d_i + d_j); weighted
// negatives c_ij = d_i P(j|i) + d_j P(i|j) = x_i z_j + y_i + x_j z_i + y_j from
// the per-vertex factors {x, y, z} (Section 3.3's derivation with P(s|i)).
__device__ __forceinline__ float pair_coef(float di, float dj, const float4 &wi, const float4 &wj, bool weighted) {
    return weighted ? fmaf(wi.x, wj.z, wi.y) + fmaf(wj.x, wi.z, wj.y) : di + dj;
}

template <bool WT>
__global__ void __launch_bounds__(kPairTile) objective_pairs_exact_kernel(const float2 *__restrict__ pos,
                                                                          const int32_t *__restrict__ deg,
                                                                          const float4 *__restrict__ wt,
                                                                          int32_t n, double *partial) {
    __shared__ float2 tp[kPairTile];
    __shared__ float td[kPairTile];
    __shared__ float4 tw[WT ? kPairTile : 1];
    double acc = 0.0;
    for (int64_t base = (int64_t)blockIdx.x * kPairTile; base < n; base += (int64_t)gridDim.x * kPairTile) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < n;
        const float2 yi = valid ? pos[i] : make_float2(0.f, 0.f);
        const float di = valid ? (float)deg[i] : 0.f;
        const float4 wi = (WT && valid) ? wt[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t jb = 0; jb < n; jb += kPairTile) {
            __syncthreads();
            const int64_t jl = jb + threadIdx.x;
            tp[threadIdx.x] = jl < n ? pos[jl] : make_float2(0.f, 0.f);
            td[threadIdx.x] = jl < n ? (float)deg[jl] : 0.f;
            if (WT) tw[threadIdx.x] = jl < n ? wt[jl] : make_float4(0.f, 0.f, 0.f, 0.f);
            __syncthreads();
            if (valid) {
                const int cnt = (int)min((int64_t)kPairTile, n - jb);
                float part = 0.0f;
                for (int q = 0; q < cnt; ++q) {
                    const float dx = yi.x - tp[q].x, dy = yi.y - tp[q].y;
                    const float r2 = fmaf(dx, dx, dy * dy);
                    const float u = 0.5f * __frcp_rn(1.0f + r2);
                    const float c = pair_coef(di, td[q], wi, tw[WT ? q : 0], WT);
                    part += (jb + q == i) ? 0.0f : c * u;
                }
                acc += (double)part;
            }
        }
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// Batch: per vertex i, the sum over j != i of its graph of w_ij U^r(r_ij),
// w_ij = (d_i + d_j) / (2 (n_g - 1)) for uniform negatives or c_ij / 2 for
// weighted ones; one thread per vertex, the graph's vertices in turn.
__global__ void objective_pairs_batch_kernel(const float2 *__restrict__ pos, const int32_t *__restrict__ deg,
                                             const float4 *__restrict__ wt, const int32_t *__restrict__ node_graph,
                                             const GraphInfo *__restrict__ graphs, int32_t n, double *partial) {
    double acc = 0.0;
    const bool weighted = wt != nullptr;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const GraphInfo gi = graphs[node_graph[i]];
        if (gi.n < 2) continue;
        const float2 yi = pos[i];
        const float di = (float)deg[i];
        const float4 wi = weighted ? wt[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        double sum = 0.0;
        float part = 0.0f;
        int cnt = 0;
        for (int32_t j = gi.node_base; j < gi.node_base + gi.n; ++j) {
            if (j == i) continue;
            const float2 yj = pos[j];
            const float dx = yi.x - yj.x, dy = yi.y - yj.y;
            const float r2 = fmaf(dx, dx, dy * dy);
            const float4 wj = weighted ? wt[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            part += pair_coef(di, (float)deg[j], wi, wj, weighted) * (0.5f * __frcp_rn(1.0f + r2));
            if (++cnt == 256) {
                sum += (double)part;
                part = 0.0f;
                cnt = 0;
            }
        }
        sum += (double)part;
        acc += weighted ? 0.5 * sum : sum / (2.0 * (double)(gi.n - 1));
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// Sampled unordered pairs: p -> Philox(ctr = (p_lo, p_hi, 0xFFFFFFFD, 0), key = seed);
// i = floor(w0 n / 2^32), j = negative(w1) of i.  Returns the sum of coef * U^r.
__global__ void objective_pairs_sampled_kernel(const float2 *__restrict__ pos, const int32_t *__restrict__ deg,
                                               const float4 *__restrict__ wt, int32_t n, int64_t pairs,
                                               uint64_t seed, double *partial) {
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const bool weighted = wt != nullptr;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double acc = 0.0;
    float part = 0.0f;
    int cnt = 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < pairs; p += stride) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)((uint64_t)p >> 32), 0xFFFFFFFDu, 0u), key);
        const int32_t i = (int32_t)__umulhi(w.x, (uint32_t)n);
        const int32_t j = negative_of(w.y, i, (uint32_t)(n - 1));
        const float2 yi = pos[i], yj = pos[j];
        const float dx = yi.x - yj.x, dy = yi.y - yj.y;
        const float r2 = fmaf(dx, dx, dy * dy);
        const float4 wi = weighted ? wt[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 wj = weighted ? wt[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        part += pair_coef((float)deg[i], (float)deg[j], wi, wj, weighted) * (0.5f * __frcp_rn(1.0f + r2));
        if (++cnt == 256) {
            acc += (double)part;
            part = 0.0f;
            cnt = 0;
        }
    }
    acc += (double)part;
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

}  // namespace

cudaError_t launch_segment_rows(const int64_t *row_ptr, int32_t n, int64_t nnz, int32_t seg_len,
                                int32_t *seg_row, int64_t num_segs, cudaStream_t s) {
    if (num_segs <= 0) return cudaSuccess;
    const int block = 256;
    const int64_t want = (num_segs + block - 1) / block;
    const int grid = (int)(want < 65536 ? want : 65536);
    segment_rows_kernel<<<grid, block, 0, s>>>(row_ptr, n, seg_len, seg_row, num_segs);
    (void)nnz;
    return cudaGetLastError();
}

cudaError_t launch_degrees(const int64_t *row_ptr, int32_t n, int32_t *deg, cudaStream_t s) {
    const int block = 256;
    const int64_t want = ((int64_t)n + block - 1) / block;
    const int grid = (int)(want < 65536 ? (want > 0 ? want : 1) : 65536);
    degrees_kernel<<<grid, block, 0, s>>>(row_ptr, n, deg);
    return cudaGetLastError();
}

cudaError_t launch_validate_csr(const int64_t *row_ptr, const int32_t *col_idx, const int32_t *seg_row,
                                int32_t n, int64_t nnz, int32_t seg_len, uint32_t *flags, cudaStream_t s,
                                const int32_t *node_graph, unsigned long long *upper_count, const int32_t *deg,
                                int32_t *orient) {
    const int block = 256;
    {
        const int64_t want = ((int64_t)n + block - 1) / block;
        const int grid = (int)(want < 65536 ? (want > 0 ? want : 1) : 65536);
        check_row_ptr_kernel<<<grid, block, 0, s>>>(row_ptr, n, nnz, flags);
    }
    const int64_t num_segs = (nnz + seg_len - 1) / seg_len;
    if (num_segs <= 0) return cudaGetLastError();
    const int64_t want = (num_segs + block - 1) / block;
    const int grid = (int)(want < 65536 ? want : 65536);
    validate_csr_kernel<<<grid, block, 0, s>>>(row_ptr, col_idx, seg_row, n, nnz, seg_len, flags, node_graph,
                                               upper_count, deg, orient);
    return cudaGetLastError();
}

cudaError_t launch_objective_edges(const int64_t *row_ptr, const int32_t *col_idx, const int32_t *seg_row,
                                   const float2 *pos, int64_t nnz, int32_t seg_len, double *partial, int grid,
                                   cudaStream_t s) {
    objective_edges_kernel<<<grid, 256, 0, s>>>(row_ptr, col_idx, seg_row, pos, nnz, seg_len, partial);
    return cudaGetLastError();
}

static int grid_for(int64_t items, int block) {
    const int64_t want = (items + block - 1) / block;
    return (int)(want < 65536 ? (want > 0 ? want : 1) : 65536);
}


cudaError_t exclusive_scan_i32(void *temp, size_t *temp_bytes, const int32_t *in, int32_t *out, int64_t count,
                               cudaStream_t s) {
    return cub::DeviceScan::ExclusiveSum(temp, *temp_bytes, in, out, count, s);
}

cudaError_t launch_orient_scatter(const int64_t *row_ptr, const int32_t *col_idx, const int32_t *seg_row,
                                  const int32_t *deg, int64_t nnz, int32_t seg_len, const int32_t *pos,
                                  const ChunkLayout &to, int4 *ent, int2 *meta, int64_t capacity, uint32_t *flags,
                                  cudaStream_t s) {
    const int64_t segs = (nnz + seg_len - 1) / seg_len;
    orient_scatter_kernel<<<grid_for(segs, 256), 256, 0, s>>>(row_ptr, col_idx, seg_row, deg, nnz, seg_len, pos,
                                                             to, ent, meta, capacity, flags);
    return cudaGetLastError();
}

cudaError_t launch_row_pieces(const int64_t *act_rp, int32_t n, int32_t T, int32_t *pieces, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    row_pieces_kernel<<<grid_for(n, 256), 256, 0, s>>>(act_rp, n, T, pieces);
    return cudaGetLastError();
}

cudaError_t launch_chunk_layout(const int4 *src, const ChunkLayout &from, int4 *dst, const ChunkLayout &to,
                                int2 *meta, const int64_t *act_rp, int32_t n, int64_t nnz, cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    chunk_layout_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(src, from, dst, to, meta, act_rp, n, nnz);
    return cudaGetLastError();
}

cudaError_t launch_objective_oriented(const int64_t *row_ptr, const int4 *ent, const int2 *meta,
                                      const ChunkLayout &L, int64_t nnz, const float2 *pos, double *partial,
                                      int grid, cudaStream_t s) {
    objective_oriented_kernel<<<grid, 256, 0, s>>>(row_ptr, ent, meta, L, nnz, pos, partial);
    return cudaGetLastError();
}

cudaError_t launch_orient_rowptr(const int64_t *row_ptr, const int32_t *pos, int32_t n, int64_t *act_row_ptr,
                                 cudaStream_t s) {
    orient_rowptr_kernel<<<grid_for((int64_t)n + 1, 256), 256, 0, s>>>(row_ptr, pos, n, act_row_ptr);
    return cudaGetLastError();
}

cudaError_t launch_objective_pairs_exact(const float2 *pos, const int32_t *deg, const float4 *wt, int32_t n,
                                         double *partial, int grid, cudaStream_t s) {
    if (wt)
        objective_pairs_exact_kernel<true><<<grid, kPairTile, 0, s>>>(pos, deg, wt, n, partial);
    else
        objective_pairs_exact_kernel<false><<<grid, kPairTile, 0, s>>>(pos, deg, nullptr, n, partial);
    return cudaGetLastError();
}

cudaError_t launch_objective_pairs_batch(const float2 *pos, const int32_t *deg, const float4 *wt,
                                         const int32_t *node_graph, const GraphInfo *graphs, int32_t n,
                                         double *partial, int grid, cudaStream_t s) {
    objective_pairs_batch_kernel<<<grid, 256, 0, s>>>(pos, deg, wt, node_graph, graphs, n, partial);
    return cudaGetLastError();
}

cudaError_t launch_objective_pairs_sampled(const float2 *pos, const int32_t *deg, const float4 *wt, int32_t n,
                                           int64_t pairs, uint64_t seed, double *partial, int grid,
                                           cudaStream_t s) {
    objective_pairs_sampled_kernel<<<grid, 256, 0, s>>>(pos, deg, wt, n, pairs, seed, partial);
    return cudaGetLastError();
}

}  // namespace snap
