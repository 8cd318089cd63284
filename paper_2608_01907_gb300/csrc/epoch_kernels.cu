// epoch_kernels.cu -- one epoch of edge-centric negative sampling
// (Algorithm 1, Section 3.3) on sm_103a.
//
// Work decomposition.  The directed edges are the CSR entries, row-major, so
// the out-edges of a source i -- its "bundle" (Section 3.4) -- are contiguous.
// The edge array is cut into fixed segments of seg_len edges; lane w of the
// grid owns segment w and walks it in order, keeping the current source's
// position in registers and switching source at row boundaries (the start
// row of every segment is precomputed in seg_row).  Every lane thus runs
// Algorithm 1 sequentially over a contiguous slice of source bundles, like
// one thread of the paper's bundle scheme; a bundle longer than a segment is
// split over several lanes.  Consecutive lanes own consecutive segments, so a
// warp streams a contiguous run of col_idx.
//
// Per directed edge e = (i, j):
//   y_j, and the k negatives s_m = negative(word m of Philox(e, t)), are
//   gathered (L2-resident positions); the attraction F^a(y_i - y_j) is
//   applied as y_i += eta F, y_j -= eta F; then for each m the repulsion
//   F^r(y_i - y_s) as y_i += eta G, y_s -= eta G, each from the current y_i.
//   A partner drawn twice in one step (s == j, or s_m == s_m') sees its
//   earlier update through registers, as in the sequential algorithm.
#include <cuda_runtime.h>
#include <stdint.h>

#include "snap_device.cuh"
#include "snap_internal.h"

namespace snap {

namespace {

// Applies an update to a partner: plain racy store (HOGWILD) or atomic add.
template <bool RED>
__device__ __forceinline__ void apply_partner(float2 *pos, int32_t idx, float2 newv, float2 delta) {
    if (RED) {
        atomicAdd(pos + idx, delta);
    } else {
        store_pos(pos + idx, newv);
    }
}

template <bool RED>
__device__ __forceinline__ void write_source(const EpochArgs &a, int32_t row, float2 yi, float2 yi0,
                                             uint32_t &flags) {
    if (!finite2(yi)) flags |= kStatusNonFinite;
    if (RED) {
        // A bundle split over L segments merges its L source displacements
        // by their mean, so the source takes one sequential pass's step.
        const int64_t rb = __ldg(a.row_ptr + row);
        const int64_t re = __ldg(a.row_ptr + row + 1);
        const int64_t L = (re - 1) / a.seg_len - rb / a.seg_len + 1;
        const float inv = L > 1 ? 1.0f / (float)L : 1.0f;
        atomicAdd(a.pos + row, make_float2((yi.x - yi0.x) * inv, (yi.y - yi0.y) * inv));
    } else {
        store_pos(a.pos + row, yi);
    }
}

template <bool RED>
__device__ __forceinline__ void hogwild_edge(const EpochArgs &a, int64_t e, int32_t i, int32_t j,
                                             float2 &yi, uint2 key, uint32_t nm1) {
    const float eta = a.eta;
    // first group of up to four negatives is gathered together with y_j
    int32_t s[4];
    float2 ys[4];
    int nm = a.k < 4 ? a.k : 4;
    {
        const uint4 w = edge_words(e, a.epoch, 0u, key);
        s[0] = negative_of(w.x, i, nm1);
        s[1] = negative_of(w.y, i, nm1);
        s[2] = negative_of(w.z, i, nm1);
        s[3] = negative_of(w.w, i, nm1);
    }
#pragma unroll
    for (int m = 0; m < 4; ++m)
        if (m < nm) ys[m] = load_pos(a.pos + s[m]);
    float2 yj = load_pos(a.pos + j);

    // attraction (Table 1), evaluated once from the positions before the step
    const float2 f = attraction_on_i(yi.x - yj.x, yi.y - yj.y);
    const float2 df = make_float2(eta * f.x, eta * f.y);
    yi.x += df.x;
    yi.y += df.y;
    yj.x -= df.x;
    yj.y -= df.y;
    apply_partner<RED>(a.pos, j, yj, make_float2(-df.x, -df.y));

    // repulsion from each negative (Table 1), immediate updates
    for (int g = 0; g * 4 < a.k; ++g) {
        if (g > 0) {
            nm = a.k - 4 * g < 4 ? a.k - 4 * g : 4;
            const uint4 w = edge_words(e, a.epoch, (uint32_t)g, key);
            s[0] = negative_of(w.x, i, nm1);
            s[1] = negative_of(w.y, i, nm1);
            s[2] = negative_of(w.z, i, nm1);
            s[3] = negative_of(w.w, i, nm1);
#pragma unroll
            for (int m = 0; m < 4; ++m)
                if (m < nm) ys[m] = load_pos(a.pos + s[m]);
        }
        float2 upd[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            if (m < nm) {
                float2 v = ys[m];
                if (g == 0 && s[m] == j) v = yj;
#pragma unroll
                for (int p = 0; p < m; ++p)
                    if (s[p] == s[m]) v = upd[p];
                const float2 gr = repulsion_on_i(yi.x - v.x, yi.y - v.y);
                const float2 dg = make_float2(eta * gr.x, eta * gr.y);
                yi.x += dg.x;
                yi.y += dg.y;
                v.x -= dg.x;
                v.y -= dg.y;
                upd[m] = v;
                apply_partner<RED>(a.pos, s[m], v, make_float2(-dg.x, -dg.y));
            }
        }
    }
}

template <bool RED>
__global__ void __launch_bounds__(256) hogwild_epoch_kernel(const EpochArgs a) {
    const int64_t num_segs = (a.nnz + a.seg_len - 1) / a.seg_len;
    const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
    const uint32_t nm1 = (uint32_t)(a.n - 1);
    uint32_t flags = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t seg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; seg < num_segs; seg += stride) {
        const int64_t e0 = seg * a.seg_len;
        const int64_t e1 = min(e0 + (int64_t)a.seg_len, a.nnz);
        int32_t row = __ldg(a.seg_row + seg);
        int64_t row_end = __ldg(a.row_ptr + row + 1);
        float2 yi = load_pos(a.pos + row);
        float2 yi0 = yi;
        for (int64_t eb = e0; eb < e1; eb += 4) {
            const int4 c4 = load_cols4(a.col_idx + eb);
            const int32_t cols[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t e = eb + q;
                if (e < e1) {
                    if (e >= row_end) {
                        write_source<RED>(a, row, yi, yi0, flags);
                        do {
                            ++row;
                            row_end = __ldg(a.row_ptr + row + 1);
                        } while (row_end <= e);
                        yi = load_pos(a.pos + row);
                        yi0 = yi;
                    }
                    hogwild_edge<RED>(a, e, row, cols[q], yi, key, nm1);
                }
            }
        }
        write_source<RED>(a, row, yi, yi0, flags);
    }
    if (flags) atomicOr(a.status, flags);
}

// Synchronous chunk: positions frozen (read-only in this launch), every force
// quantised and summed into disp with integer atomics; the source's terms
// are summed in registers (integer addition, so the total is the same as
// adding them one by one) and flushed once per row run.
__global__ void __launch_bounds__(256) sync_chunk_kernel(const SyncArgs a) {
    const int64_t seg_first = a.e_begin / a.seg_len;
    const int64_t seg_last = (a.e_end + a.seg_len - 1) / a.seg_len;   // exclusive
    const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
    const uint32_t nm1 = (uint32_t)(a.n - 1);
    uint32_t flags = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t seg = seg_first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; seg < seg_last;
         seg += stride) {
        const int64_t e0 = max(seg * a.seg_len, a.e_begin);
        const int64_t e1 = min(seg * a.seg_len + a.seg_len, a.e_end);
        int32_t row = __ldg(a.seg_row + seg);
        int64_t row_end = __ldg(a.row_ptr + row + 1);
        while (row_end <= e0) {
            ++row;
            row_end = __ldg(a.row_ptr + row + 1);
        }
        float2 yi = __ldg(a.pos + row);
        long long accx = 0, accy = 0;
        for (int64_t eb = e0 & ~(int64_t)3; eb < e1; eb += 4) {
            const int4 c4 = load_cols4(a.col_idx + eb);
            const int32_t cols[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t e = eb + q;
                if (e >= e0 && e < e1) {
                    if (e >= row_end) {
                        if (accx | accy) {
                            add_fixed(a.disp + 2 * (int64_t)row, accx);
                            add_fixed(a.disp + 2 * (int64_t)row + 1, accy);
                        }
                        accx = accy = 0;
                        do {
                            ++row;
                            row_end = __ldg(a.row_ptr + row + 1);
                        } while (row_end <= e);
                        yi = __ldg(a.pos + row);
                    }
                    const int32_t i = row;
                    const int32_t j = cols[q];
                    const float2 yj = __ldg(a.pos + j);
                    const float2 f = attraction_on_i(yi.x - yj.x, yi.y - yj.y);
                    const long long fx = to_fixed(f.x, flags), fy = to_fixed(f.y, flags);
                    accx += fx;
                    accy += fy;
                    add_fixed(a.disp + 2 * (int64_t)j, -fx);
                    add_fixed(a.disp + 2 * (int64_t)j + 1, -fy);
                    for (int g = 0; g * 4 < a.k; ++g) {
                        const int nm = a.k - 4 * g < 4 ? a.k - 4 * g : 4;
                        const uint4 w = edge_words(e, a.epoch, (uint32_t)g, key);
                        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
                        int32_t s[4];
                        float2 ys[4];
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            s[m] = negative_of(ws[m], i, nm1);
                            if (m < nm) ys[m] = __ldg(a.pos + s[m]);
                        }
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            if (m < nm) {
                                const float2 gr = repulsion_on_i(yi.x - ys[m].x, yi.y - ys[m].y);
                                const long long gx = to_fixed(gr.x, flags), gy = to_fixed(gr.y, flags);
                                accx += gx;
                                accy += gy;
                                add_fixed(a.disp + 2 * (int64_t)s[m], -gx);
                                add_fixed(a.disp + 2 * (int64_t)s[m] + 1, -gy);
                            }
                        }
                    }
                }
            }
        }
        if (accx | accy) {
            add_fixed(a.disp + 2 * (int64_t)row, accx);
            add_fixed(a.disp + 2 * (int64_t)row + 1, accy);
        }
    }
    if (flags) atomicOr(a.status, flags);
}

// y += eta * D * 2^-32 (optionally clipped to length `limit`), then D = 0.
__global__ void __launch_bounds__(256) sync_apply_kernel(float2 *pos, long long *disp, int32_t n, float eta,
                                                         float limit, uint32_t *status) {
    uint32_t flags = 0;
    const int32_t stride = gridDim.x * blockDim.x;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        longlong2 *dp = reinterpret_cast<longlong2 *>(disp) + i;
        const longlong2 d = *dp;
        float sx = eta * (__ll2float_rn(d.x) * kFixInv);
        float sy = eta * (__ll2float_rn(d.y) * kFixInv);
        if (limit > 0.0f) {
            const float len = sqrtf(sx * sx + sy * sy);
            if (len > limit) {
                const float sc = limit / len;
                sx *= sc;
                sy *= sc;
            }
        }
        float2 p = pos[i];
        p.x += sx;
        p.y += sy;
        if (!finite2(p)) flags |= kStatusNonFinite;
        pos[i] = p;
        *dp = make_longlong2(0, 0);
    }
    if (flags) atomicOr(status, flags);
}

}  // namespace

cudaError_t launch_hogwild_epoch(const EpochArgs &a, int red_mode, int grid, int block, cudaStream_t s) {
    if (red_mode)
        hogwild_epoch_kernel<true><<<grid, block, 0, s>>>(a);
    else
        hogwild_epoch_kernel<false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sync_chunk(const SyncArgs &a, int grid, int block, cudaStream_t s) {
    sync_chunk_kernel<<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sync_apply(float2 *pos, long long *disp, int32_t n, float eta, float limit,
                              uint32_t *status, int grid, int block, cudaStream_t s) {
    sync_apply_kernel<<<grid, block, 0, s>>>(pos, disp, n, eta, limit, status);
    return cudaGetLastError();
}

int hogwild_blocks_per_sm(int red_mode, int block) {
    int nb = 0;
    if (red_mode)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, hogwild_epoch_kernel<true>, block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, hogwild_epoch_kernel<false>, block, 0);
    return nb > 0 ? nb : 1;
}

int sync_blocks_per_sm(int block) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sync_chunk_kernel, block, 0);
    return nb > 0 ? nb : 1;
}

}  // namespace snap
