// epoch_kernels.cu -- one epoch of edge-centric negative sampling
// (Algorithm 1, Section 3.3) on sm_103a.
//
// HOGWILD modes work on oriented bundles (built by capi.cu at create):
// every undirected edge {i, j} is listed once, in the row of its
// higher-ranked endpoint (degree, then smaller id), with the CSR indices of
// both directed copies.  The row-major list is cut into chunks of a few
// entries, stored in a pseudo-random slot order; a warp takes one group of
// 32 slots and the order of the groups is an affine permutation that changes
// every epoch (the shuffle before bundling of Section 3.4).  A lane keeps
// the source y_i of its current row in registers and applies both directed
// steps of every entry.
//
// The synchronous mode walks the full CSR (all directed edges, row-major)
// in fixed segments with positions frozen, accumulating int64 fixed-point
// displacements.
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

// ---------------------------------------------------------------------------
// Oriented bundles.  Every undirected edge {i, j} is listed once, in the row
// of its higher-ranked endpoint i (degree, then smaller id), with the CSR
// indices of both directed copies.  The lane owning that row applies both
// directed steps of Algorithm 1 back to back: (i, j) with the negatives of
// source i (keyed by the index of (i, j)), then (j, i) with the negatives of
// source j (keyed by the index of (j, i)).  Each directed edge is processed
// once per epoch with its own random words, as in Algorithm 1; only the order
// differs.  A vertex is then a partner only of its higher-ranked neighbours
// (at most a few hundred even when the top degree is ~10^5), which removes
// the same-address read-after-write chains that hubs cause when they are the
// partner of every neighbour's bundle.
// ---------------------------------------------------------------------------

// Per-lane view of the graph the current segment belongs to.
struct GraphCtx {
    int32_t base;        // first vertex of the graph
    uint32_t nm1;        // n_g - 1
    int64_t edge_base;   // first directed edge of the graph (random-word index origin)
    uint32_t epoch;      // the graph's epoch
    float eta;
    uint2 key;           // Philox key (the graph's seed)
    bool active;
};

__device__ __forceinline__ int32_t negative_in(const GraphCtx &c, uint32_t w, int32_t src) {
    return c.base + negative_of(w, src - c.base, c.nm1);
}

__device__ __forceinline__ uint4 words_in(const GraphCtx &c, int64_t e, uint32_t g) {
    return edge_words(e - c.edge_base, c.epoch, g, c.key);
}

// Step size of epoch t under a schedule (the same expression as the host's).
__device__ __forceinline__ float schedule_eta(const GraphInfo &gi, int32_t t) {
    if (gi.kind == 1) return (float)gi.eta0;
    double eta = gi.eta0 * (1.0 - (double)t / (double)gi.total_epochs);
    return (float)(eta > gi.eta_min ? eta : gi.eta_min);
}

template <bool MULTI>
__device__ __forceinline__ GraphCtx graph_ctx(const OrientedArgs &a, int32_t row) {
    GraphCtx c;
    if (MULTI) {
        const GraphInfo gi = a.graphs[__ldg(a.node_graph + row)];
        const int32_t t = (int32_t)a.epoch - gi.start_tick;
        c.base = gi.node_base;
        c.nm1 = (uint32_t)(gi.n - 1);
        c.edge_base = gi.edge_base;
        c.epoch = (uint32_t)t;
        c.key = make_uint2((uint32_t)gi.seed, (uint32_t)(gi.seed >> 32));
        c.active = t >= 0 && t < gi.total_epochs;
        c.eta = c.active ? schedule_eta(gi, t) : 0.0f;
    } else {
        c.base = 0;
        c.nm1 = (uint32_t)(a.n - 1);
        c.edge_base = 0;
        c.epoch = a.epoch;
        c.eta = a.eta;
        c.key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
        c.active = true;
    }
    return c;
}

// Negatives of one group (up to 4, already gathered into v[]) for source
// `src` held in ysrc; the vertex `other` is register-resident in yoth.
// s[] and v[] are updated in place (v[m] = the value after its update).
template <bool RED>
__device__ __forceinline__ void negative_group(float2 *pos, float eta, const int32_t (&s)[4], float2 (&v)[4], int nm,
                                               float2 &ysrc, int32_t other, float2 &yoth) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (m < nm) {
            float2 x = v[m];
#pragma unroll
            for (int p = 0; p < m; ++p)
                if (s[p] == s[m]) x = v[p];
            if (s[m] == other) x = yoth;
            const float2 gr = repulsion_on_i(ysrc.x - x.x, ysrc.y - x.y);
            const float2 dg = make_float2(eta * gr.x, eta * gr.y);
            ysrc.x += dg.x;
            ysrc.y += dg.y;
            x.x -= dg.x;
            x.y -= dg.y;
            if (s[m] == other)
                yoth = x;
            else
                apply_partner<RED>(pos, s[m], x, make_float2(-dg.x, -dg.y));
            v[m] = x;
        }
    }
}

// Groups 1, 2, ... of negatives (k > 4): gathered after the earlier stores
// of this lane, so memory already holds this lane's updates.
template <bool RED>
__device__ __forceinline__ void later_negatives(const OrientedArgs &a, const GraphCtx &c, int64_t ekey, int32_t src,
                                                float2 &ysrc, int32_t other, float2 &yoth) {
    for (int g = 1; g * 4 < a.k; ++g) {
        const int nm = a.k - 4 * g < 4 ? a.k - 4 * g : 4;
        const uint4 w = words_in(c, ekey, (uint32_t)g);
        int32_t s[4] = {negative_in(c, w.x, src), negative_in(c, w.y, src), negative_in(c, w.z, src),
                        negative_in(c, w.w, src)};
        float2 v[4];
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (m < nm) v[m] = load_pos(a.pos + s[m]);
        negative_group<RED>(a.pos, c.eta, s, v, nm, ysrc, other, yoth);
    }
}

template <bool RED, int G>
__device__ __forceinline__ void oriented_entry(const OrientedArgs &a, const GraphCtx &c, int32_t i, int32_t j,
                                               int32_t e1, int32_t e2, float2 &yi) {
    const float eta = c.eta;
    int32_t s1[4] = {0, 0, 0, 0}, s2[4] = {0, 0, 0, 0};
    float2 v1[4], v2[4];
    if (G > 0) {
        const uint4 w1 = words_in(c, e1, 0u);
        const uint4 w2 = words_in(c, e2, 0u);
        s1[0] = negative_in(c, w1.x, i);
        s1[1] = negative_in(c, w1.y, i);
        s1[2] = negative_in(c, w1.z, i);
        s1[3] = negative_in(c, w1.w, i);
        s2[0] = negative_in(c, w2.x, j);
        s2[1] = negative_in(c, w2.y, j);
        s2[2] = negative_in(c, w2.z, j);
        s2[3] = negative_in(c, w2.w, j);
    }
    const bool prefetch2 = a.k <= 4;   // group 0 of direction 2 can be gathered up front
    float2 yj = load_pos(a.pos + j);
#pragma unroll
    for (int m = 0; m < G; ++m) v1[m] = load_pos(a.pos + s1[m]);
    if (prefetch2) {
#pragma unroll
        for (int m = 0; m < G; ++m) v2[m] = load_pos(a.pos + s2[m]);
    }
    const float2 yj0 = yj;

    // direction 1: (i, j), source i
    {
        const float2 f = attraction_on_i(yi.x - yj.x, yi.y - yj.y);
        const float2 df = make_float2(eta * f.x, eta * f.y);
        yi.x += df.x;
        yi.y += df.y;
        yj.x -= df.x;
        yj.y -= df.y;
        if (G > 0) negative_group<RED>(a.pos, eta, s1, v1, G, yi, j, yj);
        if (a.k > 4) later_negatives<RED>(a, c, e1, i, yi, j, yj);
    }
    // direction 2: (j, i), source j
    {
        const float2 f = attraction_on_i(yj.x - yi.x, yj.y - yi.y);
        const float2 df = make_float2(eta * f.x, eta * f.y);
        yj.x += df.x;
        yj.y += df.y;
        yi.x -= df.x;
        yi.y -= df.y;
        if (G > 0) {
            if (prefetch2) {
                // a negative of j that direction 1 already moved is taken from registers
#pragma unroll
                for (int m = 0; m < G; ++m)
#pragma unroll
                    for (int q = 0; q < G; ++q)
                        if (s1[q] == s2[m]) v2[m] = v1[q];
            } else {
#pragma unroll
                for (int m = 0; m < G; ++m) v2[m] = load_pos(a.pos + s2[m]);
            }
            negative_group<RED>(a.pos, eta, s2, v2, G, yj, i, yi);
        }
        if (a.k > 4) later_negatives<RED>(a, c, e2, j, yj, i, yi);
    }
    apply_partner<RED>(a.pos, j, yj, make_float2(yj.x - yj0.x, yj.y - yj0.y));
}

// Source write-back at the end of a row's run in a chunk.
// HOGWILD writes the lane's copy with an atomic exchange: the same
// last-writer-wins result as a store, but a source cut into many pieces (a
// hub) is written thousands of times per epoch, and L2 serialises plain
// stores to one address behind the loads of it far more than atomics.
// HOGWILD_RED adds the lane's displacement divided by the expected number of
// pieces of the same row in flight together (pieces x lanes / segments, at
// least 1): pieces that run at different times add up, pieces that start
// from the same position are averaged.
template <bool RED>
__device__ __forceinline__ void write_oriented_source(const OrientedArgs &a, int32_t row, float2 yi, float2 yi0,
                                                      int pieces, uint32_t &flags) {
    if (!finite2(yi)) flags |= kStatusNonFinite;
    if (RED) {
        const float together = (float)pieces * a.inflight_share;
        const float inv = together > 1.0f ? 1.0f / together : 1.0f;
        atomicAdd(a.pos + row, make_float2((yi.x - yi0.x) * inv, (yi.y - yi0.y) * inv));
    } else {
        unsigned long long bits;
        memcpy(&bits, &yi, 8);
        atomicExch(reinterpret_cast<unsigned long long *>(a.pos + row), bits);
    }
}

#ifndef SNAP_ORIENTED_MIN_BLOCKS
#define SNAP_ORIENTED_MIN_BLOCKS 1
#endif

// Slot of lane w: the 32 lanes of a warp take the 32 slots of one slot group
// (one 256-byte read of the slot table, one 512-byte read of entries per
// entry step), and the order of the groups is an affine permutation that changes
// every epoch.  The chunks were placed in slots by a fixed bijection at
// create, so the slots of a group hold unrelated parts of the graph.
__device__ __forceinline__ int64_t slot_of(int64_t w, int64_t groups, int64_t mul, int64_t add) {
    const int64_t g = (int64_t)(((uint64_t)mul * (uint64_t)(w >> 5) + (uint64_t)add) % (uint64_t)groups);
    return (g << 5) | (w & 31);
}

// Pieces of a row in the chunk cut: the chunks its entries fall in.
__device__ __forceinline__ int row_pieces(int64_t row_begin, int64_t row_end, int32_t T) {
    return (int)((uint32_t)(row_end - 1) / (uint32_t)T - (uint32_t)row_begin / (uint32_t)T) + 1;
}

// One chunk: the source y_i of the current row is held in registers and
// written back when the walk leaves the row.
template <bool RED, int G, bool MULTI>
__device__ __forceinline__ void oriented_chunk(const OrientedArgs &a, int64_t slot, uint32_t &flags) {
    const int2 mt = __ldg(a.meta + slot);   // {row of the first entry, chunk}
    int32_t row = mt.x;
    int64_t p = (int64_t)mt.y * a.seg_len;
    const int64_t p1 = p + a.seg_len < a.nnz ? p + a.seg_len : a.nnz;
    int64_t row_begin = RED ? __ldg(a.row_ptr + row) : 0;
    int64_t row_end = __ldg(a.row_ptr + row + 1);
    const int4 *ep = a.ent + chunk_entry_index(slot, a.num_segs, a.seg_len, 0);
    const int64_t step = chunk_group_width(slot, a.num_segs);
    GraphCtx c = graph_ctx<MULTI>(a, row);
    float2 yi = load_pos(a.pos + row);
    float2 yi0 = yi;
    for (; p < p1; ++p, ep += step) {
        if (p >= row_end) {
            if (c.active) write_oriented_source<RED>(a, row, yi, yi0, RED ? row_pieces(row_begin, row_end, a.seg_len) : 1,
                                                     flags);
            do {
                ++row;
                row_begin = row_end;
                row_end = __ldg(a.row_ptr + row + 1);
            } while (row_end <= p);
            if (MULTI) c = graph_ctx<MULTI>(a, row);
            yi = load_pos(a.pos + row);
            yi0 = yi;
        }
        if (!c.active) continue;
        const int4 en = load_entry(ep);   // {j, index of (i, j), index of (j, i), -}
        oriented_entry<RED, G>(a, c, row, en.x, en.y, en.z, yi);
    }
    if (c.active) write_oriented_source<RED>(a, row, yi, yi0, RED ? row_pieces(row_begin, row_end, a.seg_len) : 1,
                                             flags);
}

// In a batch a chunk may cross from one graph into the next; the graph is
// looked up again at every row change.
template <bool RED, int G, bool MULTI>
__global__ void __launch_bounds__(256, SNAP_ORIENTED_MIN_BLOCKS) oriented_epoch_kernel(const OrientedArgs a) {
    uint32_t flags = 0;
    const int64_t groups = (a.num_segs + 31) >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;   // a multiple of 32
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < (groups << 5); w += stride) {
        const int64_t ws = slot_of(w, groups, a.perm_mul, a.perm_add);
        if (ws < a.num_segs) oriented_chunk<RED, G, MULTI>(a, ws, flags);
    }
    if (flags) atomicOr(a.status, flags);
}

// Multi-handle epoch (continuous batching): one launch runs one epoch of
// several independent layouts.  The slots of all jobs form one slot space;
// lane w takes slot_of(w), finds its job by binary search over the jobs'
// slot prefixes, and processes the chunk exactly as the single-graph kernel
// would with that job's arrays, epoch, step and seed.
template <bool RED, int G>
__global__ void __launch_bounds__(256, SNAP_ORIENTED_MIN_BLOCKS) multi_epoch_kernel(const MultiArgs m) {
    uint32_t flags = 0;
    const int64_t groups = (m.total_segs + 31) >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < (groups << 5); w += stride) {
        const int64_t ws = slot_of(w, groups, m.perm_mul, m.perm_add);
        if (ws >= m.total_segs) continue;
        int32_t lo = 0, hi = m.num_jobs - 1;   // last job with seg_prefix <= ws
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) / 2;
            if (__ldg(&m.jobs[mid].seg_prefix) <= ws)
                lo = mid;
            else
                hi = mid - 1;
        }
        const JobDesc &jd = m.jobs[lo];
        OrientedArgs a;
        a.row_ptr = jd.row_ptr;
        a.ent = jd.ent;
        a.meta = jd.meta;
        a.pos = jd.pos;
        a.num_segs = jd.num_segs;
        a.nnz = jd.nnz;
        a.seg_len = jd.seg_len;
        a.n = jd.n;
        a.k = m.k;
        a.epoch = jd.epoch;
        a.seed = jd.seed;
        a.eta = jd.eta;
        a.status = m.status;
        a.node_graph = nullptr;
        a.graphs = nullptr;
        a.inflight_share = m.inflight_share;
        oriented_chunk<RED, G, false>(a, ws - jd.seg_prefix, flags);
    }
    if (flags) atomicOr(m.status, flags);
}

// Synchronous chunk: positions frozen (read-only in this launch), every force
// quantised and summed into disp with integer atomics; the source's terms
// are summed in registers (integer addition, so the total is the same as
// adding them one by one) and flushed once per row run.  In a batch the
// graph (vertex range, random-word origin, epoch) is looked up per row.
template <bool MULTI>
__device__ __forceinline__ GraphCtx sync_ctx(const SyncArgs &a, int32_t row) {
    GraphCtx c;
    if (MULTI) {
        const GraphInfo gi = a.graphs[__ldg(a.node_graph + row)];
        const int32_t t = (int32_t)a.epoch - gi.start_tick;
        c.base = gi.node_base;
        c.nm1 = (uint32_t)(gi.n - 1);
        c.edge_base = gi.edge_base;
        c.epoch = (uint32_t)t;
        c.key = make_uint2((uint32_t)gi.seed, (uint32_t)(gi.seed >> 32));
        c.active = t >= 0 && t < gi.total_epochs;
    } else {
        c.base = 0;
        c.nm1 = (uint32_t)(a.n - 1);
        c.edge_base = 0;
        c.epoch = a.epoch;
        c.key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
        c.active = true;
    }
    c.eta = 0.0f;
    return c;
}

template <bool MULTI>
__global__ void __launch_bounds__(256) sync_chunk_kernel(const SyncArgs a) {
    const int64_t seg_first = a.e_begin / a.seg_len;
    const int64_t seg_last = (a.e_end + a.seg_len - 1) / a.seg_len;   // exclusive
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
        GraphCtx c = sync_ctx<MULTI>(a, row);
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
                        if (MULTI) c = sync_ctx<MULTI>(a, row);
                        yi = __ldg(a.pos + row);
                    }
                    if (!c.active) continue;
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
                        const uint4 w = words_in(c, e, (uint32_t)g);
                        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
                        int32_t s[4];
                        float2 ys[4];
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            s[m] = negative_in(c, ws[m], i);
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
template <bool MULTI>
__global__ void __launch_bounds__(256) sync_apply_kernel(float2 *pos, long long *disp, int32_t n, float eta,
                                                         float limit, uint32_t *status, const int32_t *node_graph,
                                                         const GraphInfo *graphs, int32_t tick, float cap) {
    uint32_t flags = 0;
    const int32_t stride = gridDim.x * blockDim.x;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        longlong2 *dp = reinterpret_cast<longlong2 *>(disp) + i;
        const longlong2 d = *dp;
        float eta_i = eta, limit_i = limit;
        if (MULTI) {
            const GraphInfo gi = graphs[node_graph[i]];
            const int32_t t = tick - gi.start_tick;
            if (t < 0 || t >= gi.total_epochs) {
                *dp = make_longlong2(0, 0);
                continue;
            }
            eta_i = schedule_eta(gi, t);
            limit_i = cap > 0.0f ? (float)((double)cap * (double)eta_i / gi.eta0) : 0.0f;
        }
        float sx = eta_i * (__ll2float_rn(d.x) * kFixInv);
        float sy = eta_i * (__ll2float_rn(d.y) * kFixInv);
        if (limit_i > 0.0f) {
            const float len = sqrtf(sx * sx + sy * sy);
            if (len > limit_i) {
                const float sc = limit_i / len;
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

template <bool RED>
static cudaError_t launch_multi_g(const MultiArgs &a, int grid, int block, cudaStream_t s) {
    switch (a.k < 4 ? a.k : 4) {
        case 0: multi_epoch_kernel<RED, 0><<<grid, block, 0, s>>>(a); break;
        case 1: multi_epoch_kernel<RED, 1><<<grid, block, 0, s>>>(a); break;
        case 2: multi_epoch_kernel<RED, 2><<<grid, block, 0, s>>>(a); break;
        case 3: multi_epoch_kernel<RED, 3><<<grid, block, 0, s>>>(a); break;
        default: multi_epoch_kernel<RED, 4><<<grid, block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_multi_epoch(const MultiArgs &a, int red_mode, int grid, int block, cudaStream_t s) {
    return red_mode ? launch_multi_g<true>(a, grid, block, s) : launch_multi_g<false>(a, grid, block, s);
}

template <bool RED, int G>
static int multi_occupancy(int block) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, multi_epoch_kernel<RED, G>, block, 0);
    return nb > 0 ? nb : 1;
}

int multi_blocks_per_sm(int red_mode, int k, int block) {
    const int g = k < 4 ? k : 4;
    if (red_mode) {
        switch (g) {
            case 0: return multi_occupancy<true, 0>(block);
            case 1: return multi_occupancy<true, 1>(block);
            case 2: return multi_occupancy<true, 2>(block);
            case 3: return multi_occupancy<true, 3>(block);
            default: return multi_occupancy<true, 4>(block);
        }
    }
    switch (g) {
        case 0: return multi_occupancy<false, 0>(block);
        case 1: return multi_occupancy<false, 1>(block);
        case 2: return multi_occupancy<false, 2>(block);
        case 3: return multi_occupancy<false, 3>(block);
        default: return multi_occupancy<false, 4>(block);
    }
}

cudaError_t launch_sync_chunk(const SyncArgs &a, int grid, int block, cudaStream_t s) {
    if (a.graphs)
        sync_chunk_kernel<true><<<grid, block, 0, s>>>(a);
    else
        sync_chunk_kernel<false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sync_apply(float2 *pos, long long *disp, int32_t n, float eta, float limit,
                              uint32_t *status, int grid, int block, cudaStream_t s, const int32_t *node_graph,
                              const GraphInfo *graphs, int32_t tick, float cap) {
    if (graphs)
        sync_apply_kernel<true><<<grid, block, 0, s>>>(pos, disp, n, eta, limit, status, node_graph, graphs, tick, cap);
    else
        sync_apply_kernel<false><<<grid, block, 0, s>>>(pos, disp, n, eta, limit, status, nullptr, nullptr, 0, 0.0f);
    return cudaGetLastError();
}

template <bool RED, bool MULTI>
static cudaError_t launch_oriented_g(const OrientedArgs &a, int grid, int block, cudaStream_t s) {
    switch (a.k < 4 ? a.k : 4) {
        case 0: oriented_epoch_kernel<RED, 0, MULTI><<<grid, block, 0, s>>>(a); break;
        case 1: oriented_epoch_kernel<RED, 1, MULTI><<<grid, block, 0, s>>>(a); break;
        case 2: oriented_epoch_kernel<RED, 2, MULTI><<<grid, block, 0, s>>>(a); break;
        case 3: oriented_epoch_kernel<RED, 3, MULTI><<<grid, block, 0, s>>>(a); break;
        default: oriented_epoch_kernel<RED, 4, MULTI><<<grid, block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_oriented_epoch(const OrientedArgs &a, int red_mode, int grid, int block, cudaStream_t s) {
    const bool multi = a.graphs != nullptr;
    if (red_mode)
        return multi ? launch_oriented_g<true, true>(a, grid, block, s) : launch_oriented_g<true, false>(a, grid, block, s);
    return multi ? launch_oriented_g<false, true>(a, grid, block, s) : launch_oriented_g<false, false>(a, grid, block, s);
}

template <bool RED, int G, bool MULTI>
static int oriented_occupancy(int block) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, oriented_epoch_kernel<RED, G, MULTI>, block, 0);
    return nb > 0 ? nb : 1;
}

template <bool RED, bool MULTI>
static int oriented_occupancy_k(int k, int block) {
    switch (k < 4 ? k : 4) {
        case 0: return oriented_occupancy<RED, 0, MULTI>(block);
        case 1: return oriented_occupancy<RED, 1, MULTI>(block);
        case 2: return oriented_occupancy<RED, 2, MULTI>(block);
        case 3: return oriented_occupancy<RED, 3, MULTI>(block);
        default: return oriented_occupancy<RED, 4, MULTI>(block);
    }
}

int oriented_blocks_per_sm(int red_mode, int k, int block, int multi) {
    if (red_mode) return multi ? oriented_occupancy_k<true, true>(k, block) : oriented_occupancy_k<true, false>(k, block);
    return multi ? oriented_occupancy_k<false, true>(k, block) : oriented_occupancy_k<false, false>(k, block);
}

int sync_blocks_per_sm(int block) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sync_chunk_kernel<false>, block, 0);
    return nb > 0 ? nb : 1;
}

}  // namespace snap
