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
// One block per sample.  N_G(i) is a bitmap over the graph: in shared memory
// for graphs of up to 2^18 vertices (32 KB), else in a global scratch row of
// the block's own; a warp marks each neighbour's row (so a hub's row is read
// by 32 lanes).  The k-th nearest key (squared
// distance, then id) is found by an exact most-significant-digit radix
// select: eight 8-bit passes over the distance bits (non-negative doubles
// order as their bit patterns), then four over the ids of the vertices at
// that distance.
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
__device__ __forceinline__ uint32_t pick_bin(const uint32_t *hist, uint32_t &rank) {
    uint32_t acc = 0;
    for (uint32_t b = 0; b < 256; ++b) {
        if (acc + hist[b] >= rank) {
            rank -= acc;
            return b;
        }
        acc += hist[b];
    }
    return 255;   // not reached: rank <= candidates
}

__global__ void __launch_bounds__(256) np_sample_kernel(const int64_t *__restrict__ row_ptr,
                                                        const int32_t *__restrict__ col_idx,
                                                        const float2 *__restrict__ pos,
                                                        const int32_t *__restrict__ nodes, int32_t count,
                                                        const int32_t *__restrict__ node_graph,
                                                        const GraphInfo *__restrict__ graphs, int32_t n,
                                                        double *__restrict__ out, uint32_t *gbits,
                                                        int64_t gbits_words) {
    extern __shared__ uint32_t sbits[];
    uint32_t *bits = gbits ? gbits + (int64_t)blockIdx.x * gbits_words : sbits;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    __shared__ uint32_t hist[256];
    __shared__ uint32_t s_rank, s_k, s_inter;
    __shared__ unsigned long long s_prefix;
    for (int32_t q = blockIdx.x; q < count; q += gridDim.x) {
        const int32_t i = nodes[q];
        int32_t lo = 0, len = n;
        if (graphs) {
            const GraphInfo gi = graphs[node_graph[i]];
            lo = gi.node_base;
            len = gi.n;
        }
        const int32_t words = (len + 31) >> 5;
        for (int32_t w = threadIdx.x; w < words; w += blockDim.x) bits[w] = 0u;
        if (threadIdx.x == 0) {
            s_k = 0;
            s_inter = 0;
        }
        __syncthreads();
        // N_G(i): neighbours and their neighbours, one warp per neighbour
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
        atomicAdd(&s_k, kl);
        __syncthreads();
        const uint32_t k = s_k;
        if (k == 0) {
            if (threadIdx.x == 0) out[q] = -1.0;   // skipped
            __syncthreads();
            continue;
        }
        const float2 yi = pos[i];
        // radix select of the k-th smallest distance key
        if (threadIdx.x == 0) {
            s_rank = k;
            s_prefix = 0ull;
        }
        for (int shift = 56; shift >= 0; shift -= 8) {
            for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0u;
            __syncthreads();
            const uint64_t prefix = s_prefix;
            for (int32_t v = lo + threadIdx.x; v < lo + len; v += blockDim.x) {
                if (v == i) continue;
                const uint64_t key = dist_key(yi, pos[v]);
                if (shift == 56 || (key >> (shift + 8)) == (prefix >> (shift + 8)))
                    atomicAdd(&hist[(key >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t r = s_rank;
                const uint32_t b = pick_bin(hist, r);
                s_rank = r;
                s_prefix = prefix | ((uint64_t)b << shift);
            }
            __syncthreads();
        }
        const uint64_t dstar = s_prefix;
        __syncthreads();   // every thread holds dstar before s_prefix is reused
        // among the vertices at distance dstar, the s_rank-th smallest id
        if (threadIdx.x == 0) s_prefix = 0ull;
        __syncthreads();
        for (int shift = 24; shift >= 0; shift -= 8) {
            for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0u;
            __syncthreads();
            const uint32_t prefix = (uint32_t)s_prefix;
            for (int32_t v = lo + threadIdx.x; v < lo + len; v += blockDim.x) {
                if (v == i || dist_key(yi, pos[v]) != dstar) continue;
                const uint32_t id = (uint32_t)v;
                if (shift == 24 || (id >> (shift + 8)) == (prefix >> (shift + 8)))
                    atomicAdd(&hist[(id >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t r = s_rank;
                const uint32_t b = pick_bin(hist, r);
                s_rank = r;
                s_prefix = prefix | ((uint32_t)b << shift);
            }
            __syncthreads();
        }
        const uint32_t idstar = (uint32_t)s_prefix;
        // |N_G & N_L|: vertices of N_G with key <= (dstar, idstar)
        uint32_t inter = 0;
        for (int32_t v = lo + threadIdx.x; v < lo + len; v += blockDim.x) {
            if (v == i || !((bits[(v - lo) >> 5] >> ((v - lo) & 31)) & 1u)) continue;
            const uint64_t key = dist_key(yi, pos[v]);
            if (key < dstar || (key == dstar && (uint32_t)v <= idstar)) ++inter;
        }
        atomicAdd(&s_inter, inter);
        __syncthreads();
        if (threadIdx.x == 0) out[q] = (double)s_inter / (double)(2u * k - s_inter);
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_np_samples(const int64_t *row_ptr, const int32_t *col_idx, const float2 *pos, const int32_t *nodes,
                              int32_t count, const int32_t *node_graph, const GraphInfo *graphs, int32_t n,
                              int32_t max_graph, double *out, int grid, uint32_t *gbits, int64_t gbits_words,
                              cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const size_t smem = gbits ? 0 : sizeof(uint32_t) * (size_t)((max_graph + 31) / 32);
    np_sample_kernel<<<grid < count ? grid : count, 256, smem, s>>>(row_ptr, col_idx, pos, nodes, count, node_graph,
                                                                   graphs, n, out, gbits, gbits_words);
    return cudaGetLastError();
}

}  // namespace snap
