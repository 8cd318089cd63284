// epoch_device.cuh -- the kernels of one epoch of edge-centric negative
// sampling (Algorithm 1, Section 3.3) on sm_103a.  Included by the
// translation units that instantiate them (epoch_kernels.cu: uniform
// negatives and the synchronous mode; epoch_weighted.cu: weighted negatives;
// epoch_energy.cu: epochs that also report the actual energy).
//
// HOGWILD modes work on oriented bundles (built by capi.cu at create):
// every undirected edge {i, j} is listed once, in the row of its
// higher-ranked endpoint (degree, then smaller id), with the CSR indices of
// both directed copies (a row's entries in a fixed affine order of their
// partners, graph_kernels.cu).  The row-major list is cut into chunks of a
// few entries, stored in a pseudo-random slot order; a warp takes one group of
// 32 slots and the order of the groups is an affine permutation that changes
// every epoch (the shuffle before bundling of Section 3.4).  A lane keeps
// the source y_i of its current row in registers and applies both directed
// steps of every entry.
//
// The synchronous mode walks the full CSR (all directed edges, row-major)
// in fixed segments with positions frozen, accumulating int64 fixed-point
// displacements.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "snap_device.cuh"
#include "snap_internal.h"

namespace snap {

namespace {

// Applies an update to a partner: racy write of the lane's value (HOGWILD)
// or atomic add of the change (HOGWILD_RED).  The HOGWILD write is a 64-bit
// atomic exchange -- the same last-writer-wins result as a store -- because
// L2 serialises plain stores to an address that many lanes write at once far
// more than atomics: vertices of high degree on power-law graphs, hubs drawn
// by weighted negatives (epoch times with plain stores -> exchanges: LFR 260k
// 2.41 -> 0.77 ms, R-MAT 2^20 2.06 -> 1.19 ms, R-MAT 2^22 4.92 -> 4.84 ms;
// degree-weighted negatives on R-MAT 2^22 71 -> 9 ms).
template <bool RED>
__device__ __forceinline__ void apply_partner(float2 *pos, int32_t idx, float2 newv, float2 delta) {
    if (RED)
        add_pos(pos + idx, delta);
    else
        exchange_pos(pos + idx, newv);
}

// Adds the block's sum of v to *dst (one atomic per block).
__device__ __forceinline__ void block_add(double v, double *dst) {
    __shared__ double part[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) part[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0 && v != 0.0) atomicAdd(dst, v);
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
// E: add each pair's U^r at the moment of its update to en.
template <bool RED, bool E>
__device__ __forceinline__ void negative_group(float2 *pos, float eta, const int32_t (&s)[4], float2 (&v)[4], int nm,
                                               float2 &ysrc, int32_t other, float2 &yoth, float &en) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (m < nm) {
            float2 x = v[m];
#pragma unroll
            for (int p = 0; p < m; ++p)
                if (s[p] == s[m]) x = v[p];
            if (s[m] == other) x = yoth;
            if (E) en += repulsion_energy(ysrc.x - x.x, ysrc.y - x.y);
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
template <bool RED, bool W, bool E>
__device__ __forceinline__ void later_negatives(const OrientedArgs &a, const GraphCtx &c, int64_t ekey, int32_t src,
                                                float2 &ysrc, int32_t other, float2 &yoth, WordCursor &wc,
                                                float &en) {
    for (int g = 1; g * 4 < a.k; ++g) {
        const int nm = a.k - 4 * g < 4 ? a.k - 4 * g : 4;
        int32_t s[4];
        if (W) {
#pragma unroll
            for (int m = 0; m < 4; ++m) s[m] = m < nm ? weighted_in(c, wc, a.alias, src) : src;
        } else {
            const uint4 w = words_in(c, ekey, (uint32_t)g);
            s[0] = negative_in(c, w.x, src);
            s[1] = negative_in(c, w.y, src);
            s[2] = negative_in(c, w.z, src);
            s[3] = negative_in(c, w.w, src);
        }
        float2 v[4];
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (m < nm) v[m] = load_pos(a.pos + s[m]);
        negative_group<RED, E>(a.pos, c.eta, s, v, nm, ysrc, other, yoth, en);
    }
}

// The CSR indices of an entry's two directed copies (i, j) and (j, i).
__device__ __forceinline__ void entry_edges(int4 ent, int64_t &e1, int64_t &e2) {
    e1 = (int64_t)(uint32_t)ent.y;
    e2 = (int64_t)(uint32_t)ent.z;
}

template <bool RED, int G, bool W, bool E>
__device__ __forceinline__ void oriented_entry(const OrientedArgs &a, const GraphCtx &c, int32_t i, int32_t j,
                                               int64_t e1, int64_t e2, float2 &yi, float &en) {
    const float eta = c.eta;
    int32_t s1[4] = {0, 0, 0, 0}, s2[4] = {0, 0, 0, 0};
    float2 v1[4], v2[4];
    WordCursor wc1 = cursor_in(c, e1), wc2 = cursor_in(c, e2);
    if (G > 0 && W) {
#pragma unroll
        for (int m = 0; m < G; ++m) s1[m] = weighted_in(c, wc1, a.alias, i);
#pragma unroll
        for (int m = 0; m < G; ++m) s2[m] = weighted_in(c, wc2, a.alias, j);
    } else if (G > 0) {
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
        if (E) en += attraction_energy(yi.x - yj.x, yi.y - yj.y);
        const float2 f = attraction_on_i(yi.x - yj.x, yi.y - yj.y);
        const float2 df = make_float2(eta * f.x, eta * f.y);
        yi.x += df.x;
        yi.y += df.y;
        yj.x -= df.x;
        yj.y -= df.y;
        if (G > 0) negative_group<RED, E>(a.pos, eta, s1, v1, G, yi, j, yj, en);
        if (a.k > 4) later_negatives<RED, W, E>(a, c, e1, i, yi, j, yj, wc1, en);
    }
    // direction 2: (j, i), source j
    {
        if (E) en += attraction_energy(yj.x - yi.x, yj.y - yi.y);
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
            negative_group<RED, E>(a.pos, eta, s2, v2, G, yj, i, yi, en);
        }
        if (a.k > 4) later_negatives<RED, W, E>(a, c, e2, j, yj, i, yi, wc2, en);
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
        add_pos(a.pos + row, make_float2((yi.x - yi0.x) * inv, (yi.y - yi0.y) * inv));
    } else {
        exchange_pos(a.pos + row, yi);
    }
}

#ifndef SNAP_ORIENTED_MIN_BLOCKS
#define SNAP_ORIENTED_MIN_BLOCKS 2
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
// Each entry of the chunk is loaded while the previous one is processed (the
// first together with the slot descriptor).
template <bool RED, int G, bool MULTI, bool W, bool E>
__device__ __forceinline__ void oriented_chunk(const OrientedArgs &a, int64_t slot, uint32_t &flags, float &en) {
    const int4 *ep = a.ent + chunk_entry_index(slot, a.num_segs, a.seg_len, 0);
    const int64_t step = chunk_group_width(slot, a.num_segs);
    int4 ent_next = load_entry(ep);   // every stored chunk has at least one entry
    const int2 mt = __ldg(a.meta + slot);   // {row of the first entry, chunk}
    int32_t row = mt.x;
    int64_t p = (int64_t)mt.y * a.seg_len;
    const int64_t p1 = p + a.seg_len < a.nnz ? p + a.seg_len : a.nnz;
    int64_t row_begin = RED ? __ldg(a.row_ptr + row) : 0;
    int64_t row_end = __ldg(a.row_ptr + row + 1);
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
        const int4 ent = ent_next;   // {j, indices of (i, j) and (j, i), i}
        if (p + 1 < p1) ent_next = load_entry(ep + step);
        if (!c.active) continue;
        int64_t e1, e2;
        entry_edges(ent, e1, e2);
        oriented_entry<RED, G, W, E>(a, c, row, ent.x, e1, e2, yi, en);
    }
    if (c.active) write_oriented_source<RED>(a, row, yi, yi0, RED ? row_pieces(row_begin, row_end, a.seg_len) : 1,
                                             flags);
}

// ---------------------------------------------------------------------------
// Pipelining helpers of the direct walk below: an entry is staged (its
// random words drawn, its k + k + 1 gathers issued) one entry ahead of its
// updates.  Values gathered early for a vertex that the entry in between
// then writes are replaced by what this lane's write leaves in memory
// (forwarding), so one lane alone still applies Algorithm 1's updates in its
// order exactly; across lanes the early gathers are as racy as any.
// ---------------------------------------------------------------------------
struct StagedEntry {
    int32_t j;
    int32_t s1[4], s2[4];   // negatives of (i, j) (source i) and of (j, i) (source j)
    float2 yj, v1[4], v2[4];
    int64_t e1, e2;         // the indices of (i, j) and (j, i) (the words of later negatives)
};

// LATER (k > 4): the first four negatives of each direction are drawn here,
// but only those of (i, j) are gathered; the rest are gathered when they are
// applied (finish_entry), after this lane's earlier updates.
template <int G, bool LATER = false>
__device__ __forceinline__ void stage_entry(const OrientedArgs &a, const GraphCtx &c, int32_t i, int4 ent,
                                            StagedEntry &st) {
    st.j = ent.x;
    int64_t e1, e2;
    entry_edges(ent, e1, e2);
    st.e1 = e1;
    st.e2 = e2;
    if (G > 0) {
        const uint4 w1 = words_in(c, e1, 0u);
        const uint4 w2 = words_in(c, e2, 0u);
        const uint32_t ws1[4] = {w1.x, w1.y, w1.z, w1.w};
        const uint32_t ws2[4] = {w2.x, w2.y, w2.z, w2.w};
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            st.s1[m] = negative_in(c, ws1[m], i);
            st.s2[m] = negative_in(c, ws2[m], st.j);
        }
    }
    st.yj = load_pos(a.pos + st.j);
#pragma unroll
    for (int m = 0; m < G; ++m) st.v1[m] = load_pos(a.pos + st.s1[m]);
    if (!LATER) {
#pragma unroll
        for (int m = 0; m < G; ++m) st.v2[m] = load_pos(a.pos + st.s2[m]);
    }
}

// Bits of the staged next entry (and the next row's source) that vertex x
// matches: 1 = its partner, 2..16 = its first negatives of (i, j), 32 = the
// next row's source.
__device__ __forceinline__ uint32_t staged_match(const StagedEntry &nxt, int32_t row_n, int32_t x) {
    uint32_t b = nxt.j == x ? 1u : 0u;
#pragma unroll
    for (int m = 0; m < 4; ++m)
        if (nxt.s1[m] == x) b |= 2u << m;
    if (row_n == x) b |= 32u;
    return b;
}

// Negatives 4, 5, ... of a directed step (k > 4): gathered in groups of four
// after this lane's earlier updates, applied, and every vertex they write
// that the staged next entry already gathered is marked in `stale`.
template <bool RED, bool E>
__device__ __forceinline__ void later_direct(const OrientedArgs &a, const GraphCtx &c, int64_t ekey, int32_t src,
                                             float2 &ysrc, int32_t other, float2 &yoth, const StagedEntry &nxt,
                                             int32_t row_n, bool track, uint32_t &stale, float &en) {
    for (int g = 1; g * 4 < a.k; ++g) {
        const int nm = a.k - 4 * g < 4 ? a.k - 4 * g : 4;
        const uint4 w = words_in(c, ekey, (uint32_t)g);
        const int32_t s[4] = {negative_in(c, w.x, src), negative_in(c, w.y, src), negative_in(c, w.z, src),
                              negative_in(c, w.w, src)};
        float2 v[4];
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (m < nm) v[m] = load_pos(a.pos + s[m]);
        negative_group<RED, E>(a.pos, c.eta, s, v, nm, ysrc, other, yoth, en);
        if (track) {
#pragma unroll
            for (int m = 0; m < 4; ++m)
                if (m < nm && s[m] != other) stale |= staged_match(nxt, row_n, s[m]);
        }
    }
}

// Both directed steps of a staged entry (the arithmetic of oriented_entry);
// on return st.yj, st.v1 and st.v2 hold the values this lane wrote.  LATER:
// the first negatives of (j, i) are gathered after the whole step (i, j),
// then the later groups of each direction follow it (later_direct).
template <bool RED, int G, bool E, bool LATER = false>
__device__ __forceinline__ void finish_entry(const OrientedArgs &a, const GraphCtx &c, int32_t i, StagedEntry &st,
                                             float2 &yi, float &en, const StagedEntry &nxt, int32_t row_n,
                                             bool track, uint32_t &stale) {
    const float eta = c.eta;
    float2 yj = st.yj;
    const float2 yj0 = yj;
    {
        if (E) en += attraction_energy(yi.x - yj.x, yi.y - yj.y);
        const float2 f = attraction_on_i(yi.x - yj.x, yi.y - yj.y);
        const float2 df = make_float2(eta * f.x, eta * f.y);
        yi.x += df.x;
        yi.y += df.y;
        yj.x -= df.x;
        yj.y -= df.y;
        if (G > 0) negative_group<RED, E>(a.pos, eta, st.s1, st.v1, G, yi, st.j, yj, en);
        if (LATER) later_direct<RED, E>(a, c, st.e1, i, yi, st.j, yj, nxt, row_n, track, stale, en);
    }
    {
        if (E) en += attraction_energy(yj.x - yi.x, yj.y - yi.y);
        const float2 f = attraction_on_i(yj.x - yi.x, yj.y - yi.y);
        const float2 df = make_float2(eta * f.x, eta * f.y);
        yj.x += df.x;
        yj.y += df.y;
        yi.x -= df.x;
        yi.y -= df.y;
        if (G > 0) {
            if (LATER) {
                // gathered now: memory holds every update of the step (i, j)
#pragma unroll
                for (int m = 0; m < G; ++m) st.v2[m] = load_pos(a.pos + st.s2[m]);
            } else {
#pragma unroll
                for (int m = 0; m < G; ++m)
#pragma unroll
                    for (int q = 0; q < G; ++q)
                        if (st.s1[q] == st.s2[m]) st.v2[m] = st.v1[q];
            }
            negative_group<RED, E>(a.pos, eta, st.s2, st.v2, G, yj, i, yi, en);
        }
        if (LATER) later_direct<RED, E>(a, c, st.e2, st.j, yj, i, yi, nxt, row_n, track, stale, en);
    }
    const float2 dj = make_float2(__fsub_rn(yj.x, yj0.x), __fsub_rn(yj.y, yj0.y));
    apply_partner<RED>(a.pos, st.j, yj, dj);
    // what memory holds for j after this lane's write: the exchanged value, or
    // the gathered value plus the added change (rounded twice)
    st.yj = RED ? make_float2(__fadd_rn(yj0.x, dj.x), __fadd_rn(yj0.y, dj.y)) : yj;
}

// The value this lane last wrote for vertex x while finishing entry `done`
// of source i (whose value in memory is now yi_mem), else v.  Later writes
// win: the negatives of (i, j) in order, then those of (j, i), then j's
// final write, then the source.
template <int G>
__device__ __forceinline__ float2 forwarded(int32_t x, float2 v, const StagedEntry &done, int32_t i, float2 yi_mem) {
#pragma unroll
    for (int m = 0; m < G; ++m)
        if (done.s1[m] == x) v = done.v1[m];
#pragma unroll
    for (int m = 0; m < G; ++m)
        if (done.s2[m] == x) v = done.v2[m];
    if (x == done.j) v = done.yj;
    if (x == i) v = yi_mem;
    return v;
}

// LATER: next.v2 is not staged (it is gathered when it is applied).
template <int G, bool LATER = false>
__device__ __forceinline__ void forward_into(StagedEntry &next, const StagedEntry &done, int32_t i, float2 yi_mem) {
    next.yj = forwarded<G>(next.j, next.yj, done, i, yi_mem);
#pragma unroll
    for (int m = 0; m < G; ++m) next.v1[m] = forwarded<G>(next.s1[m], next.v1[m], done, i, yi_mem);
    if (!LATER) {
#pragma unroll
        for (int m = 0; m < G; ++m) next.v2[m] = forwarded<G>(next.s2[m], next.v2[m], done, i, yi_mem);
    }
}

// The value the source write-back leaves in memory for this lane's view
// (HOGWILD_RED adds the scaled displacement; HOGWILD writes yi).
template <bool RED>
__device__ __forceinline__ float2 written_source(const OrientedArgs &a, float2 yi, float2 yi0, int pieces) {
    if (!RED) return yi;
    const float together = (float)pieces * a.inflight_share;
    const float inv = together > 1.0f ? 1.0f / together : 1.0f;
    // the operand write_oriented_source adds, then the addition memory performs
    return make_float2(__fadd_rn(yi0.x, __fmul_rn(__fsub_rn(yi.x, yi0.x), inv)),
                       __fadd_rn(yi0.y, __fmul_rn(__fsub_rn(yi.y, yi0.y), inv)));
}

// ---------------------------------------------------------------------------
// Direct chunk walk (the default with uniform negatives, for single graphs,
// batches and multi-handle epochs).  Every entry names its
// source, so a lane needs no row offsets: the first entry of a chunk gives
// the row, and a change of source in a later entry is a row change (in a
// batch, the graph is looked up then).  The next entry's words are drawn and
// its gathers issued before the current entry's updates, with forwarding of
// the lane's own writes, and the slot loop below also loads the lane's next
// chunk's first entry and slot descriptor before it walks the current one,
// so the stream's latency is hidden too.  HOGWILD_RED reads the row's piece
// count (the chunks the row spans) when the row starts, for the write-back's
// scaling.  SNAP_DIRECT = 0 (build switch) keeps the row-offset walk for
// every case.
// ---------------------------------------------------------------------------
#ifndef SNAP_DIRECT
#define SNAP_DIRECT 1
#endif

template <bool RED, int G, bool MULTI, bool LATER = false>
__device__ __forceinline__ void oriented_chunk_direct(const OrientedArgs &a, const GraphCtx &c0, int64_t slot,
                                                      int4 ent0, int2 mt, uint32_t &flags) {
    const int64_t step = chunk_group_width(slot, a.num_segs);
    const int4 *ep = a.ent + chunk_entry_index(slot, a.num_segs, a.seg_len, 0);
    const int64_t first = (int64_t)mt.y * a.seg_len;
    const int32_t len = (int32_t)(a.nnz - first < (int64_t)a.seg_len ? a.nnz - first : (int64_t)a.seg_len);
    float en = 0.0f;
    int32_t row = ent0.w;
    GraphCtx c = MULTI ? graph_ctx<true>(a, row) : c0;   // a batch: the source's graph
    float2 yi = load_pos(a.pos + row);
    int32_t pieces = RED ? __ldg(a.pieces + row) : 1;
    StagedEntry cur, nxt;
    nxt.j = -1;
    if (c.active) stage_entry<G, LATER>(a, c, row, ent0, cur);
    int4 ent_next = len > 1 ? load_entry(ep + step) : ent0;
    float2 yi0 = yi;
    for (int32_t q = 0; q < len; ++q) {
        const bool more = q + 1 < len;
        int32_t row_n = row, pieces_n = pieces;
        float2 yi_n = yi;
        GraphCtx c_n = c;
        if (more) {
            row_n = ent_next.w;
            if (row_n != row) {
                yi_n = load_pos(a.pos + row_n);
                if (RED) pieces_n = __ldg(a.pieces + row_n);
                if (MULTI) c_n = graph_ctx<true>(a, row_n);
            }
            if (c_n.active) stage_entry<G, LATER>(a, c_n, row_n, ent_next, nxt);
            if (q + 2 < len) ent_next = load_entry(ep + (int64_t)(q + 2) * step);
        }
        uint32_t stale = 0;
        if (c.active)
            finish_entry<RED, G, false, LATER>(a, c, row, cur, yi, en, nxt, row_n != row ? row_n : -1,
                                               more && c_n.active, stale);
        if (!more) break;
        if (row_n != row) {
            if (c.active) {
                write_oriented_source<RED>(a, row, yi, yi0, pieces, flags);
                const float2 mem = written_source<RED>(a, yi, yi0, pieces);
                if (c_n.active) {
                    yi_n = forwarded<G>(row_n, yi_n, cur, row, mem);
                    forward_into<G, LATER>(nxt, cur, row, mem);
                }
            }
            row = row_n;
            c = c_n;
            yi = yi_n;
            yi0 = yi;
            pieces = pieces_n;
        } else if (c.active) {
            forward_into<G, LATER>(nxt, cur, row, yi);
        }
        if (LATER && stale) {
            // written by a later negative after they were gathered: gather again
            if (stale & 1u) nxt.yj = load_pos(a.pos + nxt.j);
#pragma unroll
            for (int m = 0; m < 4; ++m)
                if (stale & (2u << m)) nxt.v1[m] = load_pos(a.pos + nxt.s1[m]);
            if (stale & 32u) yi = yi0 = load_pos(a.pos + row);
        }
        cur = nxt;
    }
    if (c.active) write_oriented_source<RED>(a, row, yi, yi0, pieces, flags);
}

// The lanes' slot loop of the direct walk: the next chunk's first entry and
// descriptor are in flight while the current chunk is walked.
template <bool RED, int G, bool MULTI, bool LATER = false>
__device__ __forceinline__ void direct_slots(const OrientedArgs &a, uint32_t &flags) {
    const int64_t groups = (a.num_segs + 31) >> 5;
    const int64_t limit = groups << 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const GraphCtx c = graph_ctx<false>(a, 0);   // single graph (a batch looks its graph up per row)
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t ws = w < limit ? slot_of(w, groups, a.perm_mul, a.perm_add) : a.num_segs;
    int4 ent0 = make_int4(0, 0, 0, 0);
    int2 mt = make_int2(0, 0);
    if (ws < a.num_segs) {
        ent0 = load_entry(a.ent + chunk_entry_index(ws, a.num_segs, a.seg_len, 0));
        mt = __ldg(a.meta + ws);
    }
    while (w < limit) {
        const int64_t w2 = w + stride;
        const int64_t ws2 = w2 < limit ? slot_of(w2, groups, a.perm_mul, a.perm_add) : a.num_segs;
        int4 ent2 = make_int4(0, 0, 0, 0);
        int2 mt2 = make_int2(0, 0);
        if (ws2 < a.num_segs) {
            ent2 = load_entry(a.ent + chunk_entry_index(ws2, a.num_segs, a.seg_len, 0));
            mt2 = __ldg(a.meta + ws2);
        }
        if (ws < a.num_segs) oriented_chunk_direct<RED, G, MULTI, LATER>(a, c, ws, ent0, mt, flags);
        w = w2;
        ws = ws2;
        ent0 = ent2;
        mt = mt2;
    }
}

// In a batch a chunk may cross from one graph into the next; the graph is
// looked up again at every row change.  E: also sum the actual energy of the
// epoch (half the sum over the directed steps of U^a and over the drawn pairs
// of U^r, each at the moment of its update) into *a.energy.
//
// GW is the kernel's negative width: G = min(GW, 4) negatives per direction
// are drawn and gathered together; GW = 5 is the direct walk for k > 4 (the
// first four staged, later groups of four gathered when applied), kept in
// kernels of its own so that it costs the k <= 4 kernels no registers.
template <int GW>
__host__ __device__ constexpr int group_width() { return GW > 4 ? 4 : GW; }

template <bool RED, int GW, bool MULTI, bool W, bool E>
__global__ void __launch_bounds__(256, SNAP_ORIENTED_MIN_BLOCKS) oriented_epoch_kernel(const OrientedArgs a) {
    constexpr int G = group_width<GW>();
    uint32_t flags = 0;
    double energy = 0.0;
    if (SNAP_DIRECT && !W && !E && (!RED || a.pieces)) {
        direct_slots<RED, G, MULTI, (GW > 4)>(a, flags);
        if (flags) atomicOr(a.status, flags);
        return;
    }
    const int64_t groups = (a.num_segs + 31) >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;   // a multiple of 32
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < (groups << 5); w += stride) {
        const int64_t ws = slot_of(w, groups, a.perm_mul, a.perm_add);
        float en = 0.0f;
        if (ws < a.num_segs) oriented_chunk<RED, G, MULTI, W, E>(a, ws, flags, en);
        if (E) energy += (double)en;
    }
    if (flags) atomicOr(a.status, flags);
    if (E) block_add(0.5 * energy, a.energy);
}

// Multi-handle epoch (continuous batching): one launch runs one epoch of
// several independent layouts.  The slots of all jobs form one slot space;
// lane w takes slot_of(w), finds its job by binary search over the jobs'
// slot prefixes, and processes the chunk exactly as the single-graph kernel
// would with that job's arrays, epoch, step and seed.
// WEIGHTED: some job draws weighted negatives (each job's table is checked
// per chunk); otherwise every job is uniform.  The job lookup holds more
// state than the single-graph kernel: one block per SM keeps it in registers.
#ifndef SNAP_MULTI_MIN_BLOCKS
#define SNAP_MULTI_MIN_BLOCKS 1
#endif
template <bool RED, int GW, bool WEIGHTED>
__global__ void __launch_bounds__(256, SNAP_MULTI_MIN_BLOCKS) multi_epoch_kernel(const MultiArgs m) {
    constexpr int G = group_width<GW>();
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
        a.alias = jd.alias;
        a.energy = nullptr;
        a.pieces = jd.pieces;
        float en = 0.0f;
        const int64_t slot = ws - jd.seg_prefix;
        if (WEIGHTED && G > 0 && a.alias) {
            oriented_chunk<RED, G, false, true, false>(a, slot, flags, en);
        } else if (SNAP_DIRECT && (!RED || a.pieces)) {
            const int4 ent0 = load_entry(a.ent + chunk_entry_index(slot, a.num_segs, a.seg_len, 0));
            const int2 mt = __ldg(a.meta + slot);
            oriented_chunk_direct<RED, G, false, (GW > 4)>(a, graph_ctx<false>(a, 0), slot, ent0, mt, flags);
        } else {
            oriented_chunk<RED, G, false, false, false>(a, slot, flags, en);
        }
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
    double energy = 0.0;   // actual energy (a.energy != null): U^a and U^r at the frozen positions
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
                    const float en = sync_edge_terms(a.pos, a.disp, c, a.alias, row, yi, cols[q], e, a.k,
                                                     a.energy != nullptr, accx, accy, flags);
                    energy += (double)en;
                }
            }
        }
        if (accx | accy) {
            add_fixed(a.disp + 2 * (int64_t)row, accx);
            add_fixed(a.disp + 2 * (int64_t)row + 1, accy);
        }
    }
    if (flags) atomicOr(a.status, flags);
    if (a.energy) block_add(0.5 * energy, a.energy);
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

// Launch and occupancy helpers over the negative width GW: min(k, 4), or 5
// for k > 4 where the kernel takes the direct walk (uniform negatives, no
// energy); the weighted and energy kernels handle k > 4 at width 4.
template <bool W, bool E>
inline int negative_width(int k) {
    return k <= 4 ? k : (!W && !E ? 5 : 4);
}

template <bool RED, bool MULTI, bool W, bool E>
cudaError_t launch_oriented_k(const OrientedArgs &a, int grid, int block, cudaStream_t s) {
    switch (negative_width<W, E>(a.k)) {
        case 0: oriented_epoch_kernel<RED, 0, MULTI, false, E><<<grid, block, 0, s>>>(a); break;
        case 1: oriented_epoch_kernel<RED, 1, MULTI, W, E><<<grid, block, 0, s>>>(a); break;
        case 2: oriented_epoch_kernel<RED, 2, MULTI, W, E><<<grid, block, 0, s>>>(a); break;
        case 3: oriented_epoch_kernel<RED, 3, MULTI, W, E><<<grid, block, 0, s>>>(a); break;
        case 4: oriented_epoch_kernel<RED, 4, MULTI, W, E><<<grid, block, 0, s>>>(a); break;
        default:
            if constexpr (!W && !E) oriented_epoch_kernel<RED, 5, MULTI, false, false><<<grid, block, 0, s>>>(a);
            break;
    }
    return cudaGetLastError();
}

template <typename K>
int occupancy_of(K kernel, int block) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, block, 0);
    return nb > 0 ? nb : 1;
}

template <bool RED, bool MULTI, bool W, bool E>
int oriented_occupancy_k(int k, int block) {
    switch (negative_width<W, E>(k)) {
        case 0: return occupancy_of(oriented_epoch_kernel<RED, 0, MULTI, false, E>, block);
        case 1: return occupancy_of(oriented_epoch_kernel<RED, 1, MULTI, W, E>, block);
        case 2: return occupancy_of(oriented_epoch_kernel<RED, 2, MULTI, W, E>, block);
        case 3: return occupancy_of(oriented_epoch_kernel<RED, 3, MULTI, W, E>, block);
        case 4: return occupancy_of(oriented_epoch_kernel<RED, 4, MULTI, W, E>, block);
        default:
            if constexpr (!W && !E) return occupancy_of(oriented_epoch_kernel<RED, 5, MULTI, false, false>, block);
            return 1;
    }
}

// The multi-handle kernel takes width 5 for k > 4 also when some jobs draw
// weighted negatives (those jobs walk their chunks at width 4).
template <bool RED, bool WEIGHTED>
cudaError_t launch_multi_k(const MultiArgs &a, int grid, int block, cudaStream_t s) {
    switch (negative_width<false, false>(a.k)) {
        case 0: multi_epoch_kernel<RED, 0, false><<<grid, block, 0, s>>>(a); break;
        case 1: multi_epoch_kernel<RED, 1, WEIGHTED><<<grid, block, 0, s>>>(a); break;
        case 2: multi_epoch_kernel<RED, 2, WEIGHTED><<<grid, block, 0, s>>>(a); break;
        case 3: multi_epoch_kernel<RED, 3, WEIGHTED><<<grid, block, 0, s>>>(a); break;
        case 4: multi_epoch_kernel<RED, 4, WEIGHTED><<<grid, block, 0, s>>>(a); break;
        default: multi_epoch_kernel<RED, 5, WEIGHTED><<<grid, block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <bool RED, bool WEIGHTED>
int multi_occupancy_k(int k, int block) {
    switch (negative_width<false, false>(k)) {
        case 0: return occupancy_of(multi_epoch_kernel<RED, 0, false>, block);
        case 1: return occupancy_of(multi_epoch_kernel<RED, 1, WEIGHTED>, block);
        case 2: return occupancy_of(multi_epoch_kernel<RED, 2, WEIGHTED>, block);
        case 3: return occupancy_of(multi_epoch_kernel<RED, 3, WEIGHTED>, block);
        case 4: return occupancy_of(multi_epoch_kernel<RED, 4, WEIGHTED>, block);
        default: return occupancy_of(multi_epoch_kernel<RED, 5, WEIGHTED>, block);
    }
}

}  // namespace
}  // namespace snap
