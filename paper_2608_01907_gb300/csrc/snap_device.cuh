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
__device__ __forceinline__ float2 load_pos(const float2 *p) { return __ldcg(p); }
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

// One oriented entry {j, low 32 bits of the indices of (i, j) and (j, i),
// their bits 32..47}.
// Read through L1: the 32 lanes of a warp walk one compact run of entries
// over several iterations, so a line fetched for one lane serves others.
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

}  // namespace snap
