// np_kernels.cu -- neighbourhood preservation on the device (Section 4.1,
// "Metrics": NP with r = 2), for the autotuner's quality gate and the
// library's own quality report.
//
// For a sampled vertex i of a graph with vertices [lo, lo + len):
//   N_G(i) = the vertices within two hops of i, i excluded; k = |N_G(i)|;
//   N_L(i) = the k vertices of the same graph nearest to i in the layout, i
//            excluded, ordered by squared distance and then by smaller id;
//   NP_i   = |N_G(i) & N_L(i)| / |N_G(i) | N_L(i)| (a Jaccard index); vertices
//            with k = 0 are skipped.
// Squared distances are formed in FP64 from the FP32 positions,
// (x_i - x_v)^2 + (y_i - y_v)^2 with every operation rounded on its own, so
// the ranking equals that of an FP64 evaluation of the same positions.
//
// One block per sample.  N_G(i) is a bitmap over the graph; a warp marks each
// neighbour's row (so a hub's row is read by 32 lanes).  The k-th nearest key
// (squared distance, then id) is found by an exact most-significant-digit
// radix select: eight 8-bit passes over the distance bits (non-negative
// doubles order as their bit patterns), then four over the ids of the
// vertices at that distance.
//
// Graphs of up to 2^18 vertices (np_sample_kernel): the bitmap lives in shared
// memory (32 KB) and the select runs over all vertices.  Larger graphs
// (np_sample_large_kernel): the bitmap is a global scratch row of the block's
// own, and the distances are formed twice instead of thirteen times (FP64 is
// slow on this GPU): a first pass histograms the top 12 bits of every key
// (sign and exponent: distances within a factor of two share a bin) and finds
// the bin of the k-th; a second counts the members of N_G below that bin and
// copies the keys inside it to a candidate list, over which the select runs.
// A candidate list longer than its scratch falls back to the select over all
// vertices.
#include <cuda_runtime.h>
#include <stdint.h>

#include "snap_internal.h"

namespace snap {
namespace {

__device__ __forceinline__ uint64_t dist_key(float2 a, float2 b) {
    const double dx = __dsub_rn((double)a.x, (double)b.x);
    const double dy = __dsub_rn((double)a.y, (double)b.y);
    return (uint64_t)__double_as_longlong(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}

// Smallest bin b with hist[0..b] >= rank (1-based); rank becomes the rank
// within bin b.  Thread 0 only.
__device__ __forceinline__ uint32_t pick_bin(const uint32_t *hist, uint32_t bins, uint32_t &rank) {
    uint32_t acc = 0;
    for (uint32_t b = 0; b < bins; ++b) {
        if (acc + hist[b] >= rank) {
            rank -= acc;
            return b;
        }
        acc += hist[b];
    }
    return bins - 1;   // not reached: rank <= candidates
}

// Shared state of one block's select.
struct SelectShared {
    uint32_t hist[256];
    uint32_t rank, k, inter, count, bin;
    unsigned long long prefix;
};

// The rank-th smallest (key, id) among the items each() visits (each thread
// calls f(key, id) for its share): *dstar, *idstar on every thread.
template <typename Each>
__device__ void radix_select(Each each, uint32_t rank, SelectShared &sh, uint64_t &dstar, uint32_t &idstar) {
    if (threadIdx.x == 0) {
        sh.rank = rank;
        sh.prefix = 0ull;
    }
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) sh.hist[b] = 0u;
        __syncthreads();
        const uint64_t prefix = sh.prefix;
        each([&](uint64_t key, uint32_t) {
            if (shift == 56 || (key >> (shift + 8)) == (prefix >> (shift + 8)))
                atomicAdd(&sh.hist[(key >> shift) & 255u], 1u);
        });
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t r = sh.rank;
            const uint32_t b = pick_bin(sh.hist, 256u, r);
            sh.rank = r;
            sh.prefix = prefix | ((uint64_t)b << shift);
        }
        __syncthreads();
    }
    dstar = sh.prefix;
    __syncthreads();   // every thread holds dstar before the prefix is reused
    if (threadIdx.x == 0) sh.prefix = 0ull;
    __syncthreads();
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) sh.hist[b] = 0u;
        __syncthreads();
        const uint32_t prefix = (uint32_t)sh.prefix;
        each([&](uint64_t key, uint32_t id) {
            if (key != dstar) return;
            if (shift == 24 || (id >> (shift + 8)) == (prefix >> (shift + 8)))
                atomicAdd(&sh.hist[(id >> shift) & 255u], 1u);
        });
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t r = sh.rank;
            const uint32_t b = pick_bin(sh.hist, 256u, r);
            sh.rank = r;
            sh.prefix = prefix | ((uint32_t)b << shift);
        }
        __syncthreads();
    }
    idstar = (uint32_t)sh.prefix;
    __syncthreads();
}

__device__ __forceinline__ bool has_bit(const uint32_t *bits, int32_t x) { return (bits[x >> 5] >> (x & 31)) & 1u; }

// N_G(i) as a bitmap over [lo, lo + len) (cleared first), i excluded; returns
// k = |N_G(i)| on every thread.
__device__ uint32_t two_hop_bitmap(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                                   int32_t i, int32_t lo, int32_t len, uint32_t *bits, SelectShared &sh) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int32_t words = (len + 31) >> 5;
    for (int32_t w = threadIdx.x; w < words; w += blockDim.x) bits[w] = 0u;
    if (threadIdx.x == 0) sh.k = 0;
    __syncthreads();
    // neighbours and their neighbours, one warp per neighbour
    const int64_t b0 = row_ptr[i], b1 = row_ptr[i + 1];
    for (int64_t e = b0 + warp; e < b1; e += nwarps) {
        const int32_t u = col_idx[e];
        if (lane == 0) atomicOr(&bits[(u - lo) >> 5], 1u << ((u - lo) & 31));
        const int64_t f1 = row_ptr[u + 1];
        for (int64_t f = row_ptr[u] + lane; f < f1; f += 32) {
            const int32_t v = col_idx[f] - lo;
            atomicOr(&bits[v >> 5], 1u << (v & 31));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) bits[(i - lo) >> 5] &= ~(1u << ((i - lo) & 31));
    __syncthreads();
    uint32_t kl = 0;
    for (int32_t w = threadIdx.x; w < words; w += blockDim.x) kl += __popc(bits[w]);
    atomicAdd(&sh.k, kl);
    __syncthreads();
    const uint32_t k = sh.k;
    __syncthreads();
    return k;
}

// The graph of vertex i: [lo, lo + len).
__device__ __forceinline__ void graph_of(int32_t i, const int32_t *node_graph, const GraphInfo *graphs, int32_t n,
                                         int32_t &lo, int32_t &len) {
    lo = 0;
    len = n;
    if (graphs) {
        const GraphInfo gi = graphs[node_graph[i]];
        lo = gi.node_base;
        len = gi.n;
    }
}

// The select over all vertices of [lo, lo + len) except i, and the count of
// N_G & N_L; NP_i on thread 0.
__device__ double np_over_all(const float2 *__restrict__ pos, const uint32_t *bits, int32_t i, int32_t lo,
                              int32_t len, uint32_t k, SelectShared &sh) {
    const float2 yi = pos[i];
    auto all = [&](auto f) {
        for (int32_t v = lo + threadIdx.x; v < lo + len; v += blockDim.x)
            if (v != i) f(dist_key(yi, pos[v]), (uint32_t)v);
    };
    uint64_t dstar;
    uint32_t idstar;
    radix_select(all, k, sh, dstar, idstar);
    if (threadIdx.x == 0) sh.inter = 0;
    __syncthreads();
    uint32_t inter = 0;
    for (int32_t v = lo + threadIdx.x; v < lo + len; v += blockDim.x) {
        if (v == i || !has_bit(bits, v - lo)) continue;
        const uint64_t key = dist_key(yi, pos[v]);
        if (key < dstar || (key == dstar && (uint32_t)v <= idstar)) ++inter;
    }
    atomicAdd(&sh.inter, inter);
    __syncthreads();
    const uint32_t total = sh.inter;
    __syncthreads();
    return (double)total / (double)(2u * k - total);
}

__global__ void __launch_bounds__(256) np_sample_kernel(const int64_t *__restrict__ row_ptr,
                                                        const int32_t *__restrict__ col_idx,
                                                        const float2 *__restrict__ pos,
                                                        const int32_t *__restrict__ nodes, int32_t count,
                                                        const int32_t *__restrict__ node_graph,
                                                        const GraphInfo *__restrict__ graphs, int32_t n,
                                                        double *__restrict__ out) {
    extern __shared__ uint32_t sbits[];
    __shared__ SelectShared sh;
    for (int32_t q = blockIdx.x; q < count; q += gridDim.x) {
        const int32_t i = nodes[q];
        int32_t lo, len;
        graph_of(i, node_graph, graphs, n, lo, len);
        const uint32_t k = two_hop_bitmap(row_ptr, col_idx, i, lo, len, sbits, sh);
        if (k == 0) {
            if (threadIdx.x == 0) out[q] = -1.0;   // skipped
            continue;
        }
        const double v = np_over_all(pos, sbits, i, lo, len, k, sh);
        if (threadIdx.x == 0) out[q] = v;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) np_sample_large_kernel(const int64_t *__restrict__ row_ptr,
                                                              const int32_t *__restrict__ col_idx,
                                                              const float2 *__restrict__ pos,
                                                              const int32_t *__restrict__ nodes, int32_t count,
                                                              const int32_t *__restrict__ node_graph,
                                                              const GraphInfo *__restrict__ graphs, int32_t n,
                                                              double *__restrict__ out, uint32_t *gbits,
                                                              int64_t gbits_words, uint64_t *ckeys, uint32_t *cids,
                                                              int32_t cap) {
    __shared__ SelectShared sh;
    __shared__ uint32_t top[4096];   // histogram of the keys' top 12 bits
    uint32_t *bits = gbits + (int64_t)blockIdx.x * gbits_words;
    uint64_t *ck = ckeys + (int64_t)blockIdx.x * cap;
    uint32_t *ci = cids + (int64_t)blockIdx.x * cap;
    for (int32_t q = blockIdx.x; q < count; q += gridDim.x) {
        const int32_t i = nodes[q];
        int32_t lo, len;
        graph_of(i, node_graph, graphs, n, lo, len);
        const uint32_t k = two_hop_bitmap(row_ptr, col_idx, i, lo, len, bits, sh);
        if (k == 0) {
            if (threadIdx.x == 0) out[q] = -1.0;   // skipped
            continue;
        }
        const float2 yi = pos[i];
        // pass 1: the bin (top 12 bits) of the k-th key, and its rank inside the bin
        for (int b = threadIdx.x; b < 4096; b += blockDim.x) top[b] = 0u;
        __syncthreads();
        for (int32_t v = lo + threadIdx.x; v < lo + len; v += blockDim.x)
            if (v != i) atomicAdd(&top[dist_key(yi, pos[v]) >> 52], 1u);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t r = k;
            sh.bin = pick_bin(top, 4096u, r);
            sh.rank = r;
            sh.count = 0;
            sh.inter = 0;
        }
        __syncthreads();
        const uint64_t bin = sh.bin;
        const uint32_t rank = sh.rank;
        __syncthreads();
        // pass 2: members of N_G below the bin; the bin's keys to the candidate list
        uint32_t inter = 0;
        for (int32_t v = lo + threadIdx.x; v < lo + len; v += blockDim.x) {
            if (v == i) continue;
            const uint64_t key = dist_key(yi, pos[v]);
            const uint64_t t = key >> 52;
            if (t < bin) {
                if (has_bit(bits, v - lo)) ++inter;
            } else if (t == bin) {
                const uint32_t slot = atomicAdd(&sh.count, 1u);
                if (slot < (uint32_t)cap) {
                    ck[slot] = key;
                    ci[slot] = (uint32_t)v;
                }
            }
        }
        atomicAdd(&sh.inter, inter);
        __syncthreads();
        const uint32_t ncand = sh.count, below = sh.inter;
        __syncthreads();
        double np;
        if (ncand > (uint32_t)cap) {
            np = np_over_all(pos, bits, i, lo, len, k, sh);   // candidate list too long
        } else {
            auto cands = [&](auto f) {
                for (uint32_t t = threadIdx.x; t < ncand; t += blockDim.x) f(ck[t], ci[t]);
            };
            uint64_t dstar;
            uint32_t idstar;
            radix_select(cands, rank, sh, dstar, idstar);
            if (threadIdx.x == 0) sh.inter = 0;
            __syncthreads();
            uint32_t in_bin = 0;
            for (uint32_t t = threadIdx.x; t < ncand; t += blockDim.x) {
                const uint64_t key = ck[t];
                const uint32_t id = ci[t];
                if ((key < dstar || (key == dstar && id <= idstar)) && has_bit(bits, (int32_t)id - lo)) ++in_bin;
            }
            atomicAdd(&sh.inter, in_bin);
            __syncthreads();
            const uint32_t total = below + sh.inter;
            np = (double)total / (double)(2u * k - total);
        }
        if (threadIdx.x == 0) out[q] = np;
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_np_samples(const int64_t *row_ptr, const int32_t *col_idx, const float2 *pos, const int32_t *nodes,
                              int32_t count, const int32_t *node_graph, const GraphInfo *graphs, int32_t n,
                              int32_t max_graph, double *out, int grid, uint32_t *gbits, int64_t gbits_words,
                              cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int g = grid < count ? grid : count;
    if (!gbits) {
        const size_t smem = sizeof(uint32_t) * (size_t)((max_graph + 31) / 32);
        np_sample_kernel<<<g, 256, smem, s>>>(row_ptr, col_idx, pos, nodes, count, node_graph, graphs, n, out);
    } else {
        // the bitmap rows of the grid's blocks, then (8-byte aligned) their candidate keys and ids
        const int64_t cap = kNpCandidates;
        uint64_t *ckeys = reinterpret_cast<uint64_t *>(gbits + (((int64_t)grid * gbits_words + 1) & ~(int64_t)1));
        uint32_t *cids = reinterpret_cast<uint32_t *>(ckeys + (int64_t)grid * cap);
        np_sample_large_kernel<<<g, 256, 0, s>>>(row_ptr, col_idx, pos, nodes, count, node_graph, graphs, n, out,
                                                 gbits, gbits_words, ckeys, cids, (int32_t)cap);
    }
    return cudaGetLastError();
}

}  // namespace snap
