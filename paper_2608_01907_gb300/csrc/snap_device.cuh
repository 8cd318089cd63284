// snap_device.cuh -- device helpers of the epoch and objective kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "snap_internal.h"

namespace snap {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy
// as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies mixed with the
// other half of the counter and the round key; the key advances by the Weyl
// constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Words 4g..4g+3 of the random stream of directed edge e in epoch t.
__device__ __forceinline__ uint4 edge_words(int64_t e, uint32_t t, uint32_t g, uint2 key) {
    return philox4x32_10(make_uint4((uint32_t)e, (uint32_t)((uint64_t)e >> 32), t, g), key);
}

// Uniform negative from V \ {i} (Algorithm 1): u = floor(w (n-1) / 2^32), s = u + (u >= i).
__device__ __forceinline__ int32_t negative_of(uint32_t w, int32_t i, uint32_t n_minus_1) {
    const uint32_t u = __umulhi(w, n_minus_1);
    return (int32_t)(u + (u >= (uint32_t)i ? 1u : 0u));
}

// The word stream of one directed edge, consumed in order by its negatives
// (word w is component w mod 4 of the Philox block w div 4).
struct WordCursor {
    int64_t e;       // edge index (graph-local)
    uint32_t next;   // next word
    uint32_t blk;    // Philox block held in buf (~0u: none)
    uint4 buf;
};

__device__ __forceinline__ WordCursor word_cursor(int64_t e) {
    WordCursor c;
    c.e = e;
    c.next = 0;
    c.blk = ~0u;
    c.buf = make_uint4(0, 0, 0, 0);
    return c;
}

__device__ __forceinline__ uint32_t take_word(WordCursor &c, uint32_t t, uint2 key) {
    const uint32_t b = c.next >> 2;
    if (b != c.blk) {
        c.buf = edge_words(c.e, t, b, key);
        c.blk = b;
    }
    const uint32_t q = c.next & 3u;
    ++c.next;
    return q == 0 ? c.buf.x : q == 1 ? c.buf.y : q == 2 ? c.buf.z : c.buf.w;
}

// Weighted negative (degree or caller weights) through an alias table of n
// entries {threshold, alias} (graph-local ids): two words per attempt --
// column floor(w0 n / 2^32), kept when w1 < threshold, else its alias; an
// attempt that yields the source is rejected, and after 16 rejections the
// uniform rule takes the next word.  Returns a graph-local id.
__device__ __forceinline__ int32_t weighted_negative(WordCursor &c, uint32_t t, uint2 key, const uint2 *table,
                                                     uint32_t n, int32_t src) {
    for (int attempt = 0; attempt < 16; ++attempt) {
        const uint32_t w0 = take_word(c, t, key);
        const uint32_t w1 = take_word(c, t, key);
        const uint32_t col = __umulhi(w0, n);
        const uint2 en = __ldg(table + col);
        const int32_t s = w1 < en.x ? (int32_t)col : (int32_t)en.y;
        if (s != src) return s;
    }
    return negative_of(take_word(c, t, key), src, n - 1);
}

// Force on i from the attraction of Table 1 (t-FDP): pulls i toward the
// partner, coefficient alpha (1 + beta / (1 + r^2)); d = y_i - y_partner.
__device__ __forceinline__ float2 attraction_on_i(float dx, float dy) {
    const float r2 = fmaf(dx, dx, dy * dy);
    const float q = __frcp_rn(1.0f + r2);
    const float ca = kAlpha * fmaf(kBeta, q, 1.0f);
    return make_float2(-ca * dx, -ca * dy);
}

// Force on i from the repulsion of Table 1 (t-FDP, gamma = 2): pushes i away,
// coefficient (1 + r^2)^-2; d = y_i - y_sample.
__device__ __forceinline__ float2 repulsion_on_i(float dx, float dy) {
    const float r2 = fmaf(dx, dx, dy * dy);
    const float q = __frcp_rn(1.0f + r2);
    const float cr = q * q;
    return make_float2(cr * dx, cr * dy);
}

// Position accesses that must see other SMs' writes: cached in L2 only.
// (Measured on GB300 against these intrinsics, with no gain on the R-MAT
// epoch: an explicit vector red.global.add.v2.f32, L2 evict-last / evict-first
// cache policies on positions and entries.)
__device__ __forceinline__ float2 load_pos(const float2 *p) { return __ldcg(p); }

// Adds d to a position (relaxed, device scope, no return value: a vector
// reduction in L2).
__device__ __forceinline__ void add_pos(float2 *p, float2 d) { atomicAdd(p, d); }

// A position written as one 64-bit atomic exchange (racy, last writer wins).
__device__ __forceinline__ void exchange_pos(float2 *p, float2 v) {
    unsigned long long bits;
    memcpy(&bits, &v, 8);
    atomicExch(reinterpret_cast<unsigned long long *>(p), bits);
}

// The edge stream is read once per epoch: evict-first streaming loads.
__device__ __forceinline__ int4 load_cols4(const int32_t *p) {
    return __ldcs(reinterpret_cast<const int4 *>(p));
}

// One oriented entry {j, index of (i, j), index of (j, i), i}.  Read through
// L1: the 32 lanes of a warp read one 512-byte run of entries per step.
__device__ __forceinline__ int4 load_entry(const int4 *p) { return __ldg(p); }

// int64 fixed point (2^-32) of one force component, clamped to +-2^20.
__device__ __forceinline__ long long to_fixed(float v, uint32_t &flags) {
    if (!(fabsf(v) <= kFixClamp)) {
        if (v != v) {
            flags |= kStatusNonFinite;
            return 0;
        }
        flags |= kStatusClamped;
        v = copysignf(kFixClamp, v);
    }
    return __float2ll_rn(v * kFixScale);
}

__device__ __forceinline__ void add_fixed(long long *dst, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)v);
}

__device__ __forceinline__ bool finite2(float2 v) {
    return isfinite(v.x) && isfinite(v.y);
}


// Energies of Table 1 / Eq. 2 for the actual energy of an epoch (Section
// 3.3): U^a = alpha (r^2/2 + beta/2 ln(1 + r^2)), U^r = 1 / (2 (1 + r^2)).
__device__ __forceinline__ float attraction_energy(float dx, float dy) {
    const float r2 = fmaf(dx, dx, dy * dy);
    return kAlpha * fmaf(0.5f, r2, 0.5f * kBeta * log1pf(r2));
}

__device__ __forceinline__ float repulsion_energy(float dx, float dy) {
    return 0.5f * __frcp_rn(1.0f + fmaf(dx, dx, dy * dy));
}

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

__device__ __forceinline__ WordCursor cursor_in(const GraphCtx &c, int64_t e) { return word_cursor(e - c.edge_base); }

// Next weighted negative of source src (global ids); table = the graph's alias table.
__device__ __forceinline__ int32_t weighted_in(const GraphCtx &c, WordCursor &wc, const uint2 *alias, int32_t src) {
    return c.base + weighted_negative(wc, c.epoch, c.key, alias + c.base, c.nm1 + 1u, src - c.base);
}

// One pair's term in the synchronous mode: the force on the source i from
// the attraction (REP = false) or the repulsion (REP = true) of Table 1 at
// the frozen positions, quantised (to_fixed); the source's share is summed
// into accx / accy, the other vertex's is added to disp.
template <bool REP>
__device__ __forceinline__ void sync_pair_term(long long *disp, float2 yi, int32_t x, float2 yx, long long &accx,
                                               long long &accy, uint32_t &flags) {
    const float2 f = REP ? repulsion_on_i(yi.x - yx.x, yi.y - yx.y) : attraction_on_i(yi.x - yx.x, yi.y - yx.y);
    const long long fx = to_fixed(f.x, flags), fy = to_fixed(f.y, flags);
    accx += fx;
    accy += fy;
    add_fixed(disp + 2 * (int64_t)x, -fx);
    add_fixed(disp + 2 * (int64_t)x + 1, -fy);
}

// All force terms of directed edge e = (i, j) in the synchronous mode, with
// positions frozen (read-only during the launch): the attraction of Table 1
// and the repulsion of each of its k negatives (Algorithm 1's draws, in the
// order they consume the edge's random words), each force quantised to int64
// fixed point (2^-32, to_fixed).  The partner's and the negatives' terms are
// added to disp with integer atomics; the source's are summed into accx /
// accy, which the caller flushes once per row run.  Integer addition makes
// the totals independent of the order of the terms.  Returns the energy of
// the step's pairs at the frozen positions (U^a of (i, j) and U^r of each
// drawn pair) when `energy` is set, else 0.  Shared by the synchronous chunk
// kernel of a handle and by the allocation-free entry point.
__device__ __forceinline__ float sync_edge_terms(const float2 *pos, long long *disp, const GraphCtx &c,
                                                 const uint2 *alias, int32_t i, float2 yi, int32_t j, int64_t e,
                                                 int32_t k, bool energy, long long &accx, long long &accy,
                                                 uint32_t &flags) {
    const float2 yj = __ldg(pos + j);
    float en = 0.0f;
    if (energy) en += attraction_energy(yi.x - yj.x, yi.y - yj.y);
    sync_pair_term<false>(disp, yi, j, yj, accx, accy, flags);
    WordCursor wc = cursor_in(c, e);
    for (int g = 0; g * 4 < k; ++g) {
        const int nm = k - 4 * g < 4 ? k - 4 * g : 4;
        int32_t s[4];
        float2 ys[4];
        if (alias) {
#pragma unroll
            for (int m = 0; m < 4; ++m) s[m] = m < nm ? weighted_in(c, wc, alias, i) : i;
        } else {
            const uint4 w = words_in(c, e, (uint32_t)g);
            s[0] = negative_in(c, w.x, i);
            s[1] = negative_in(c, w.y, i);
            s[2] = negative_in(c, w.z, i);
            s[3] = negative_in(c, w.w, i);
        }
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (m < nm) ys[m] = __ldg(pos + s[m]);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            if (m < nm) {
                if (energy) en += repulsion_energy(yi.x - ys[m].x, yi.y - ys[m].y);
                sync_pair_term<true>(disp, yi, s[m], ys[m], accx, accy, flags);
            }
        }
    }
    return en;
}

}  // namespace snap
