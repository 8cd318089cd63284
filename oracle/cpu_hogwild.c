/*
 * cpu_hogwild.c -- multi-threaded FP32 CPU implementation of the paper's
 * lock-free bundle scheme (Section 3.4), the CPU throughput baseline of the
 * bench.
 *
 * BENCH AND TEST INFRASTRUCTURE ONLY, like the oracle beside it: the product
 * library never calls it and shares no code with it.
 *
 * What it computes: epochs of Algorithm 1 with positions in FP32, run by
 * OpenMP threads without locks.  A bundle is all out-edges (i, j) of one
 * source i (a CSR row); bundles are visited in a caller-given order (the
 * random shuffle that precedes bundling, Section 3.4) and handed to threads
 * dynamically, one whole bundle per thread at a time.  Each edge applies the
 * attraction of Table 1 to i and j, then draws k negatives s uniformly from V
 * without i and applies the repulsion to i and s (alpha = 0.1, beta = 8,
 * gamma = 2, Section 3.1).  Updates are immediate and racy: every position is
 * read and written as one relaxed 64-bit access, so concurrent updates may
 * overwrite one another (the HOGWILD! behaviour the paper accepts).
 *
 * Negative draws follow the same definition as the oracle (written out again
 * here): word w of directed edge e in epoch t is component w mod 4 of
 * Philox4x32-10(counter (e_lo, e_hi, t, w div 4), key (seed_lo, seed_hi))
 * (Salmon et al., SC'11); a uniform negative takes one word,
 * u = floor(w (n-1) / 2^32), s = u + (u >= i).
 *
 * Build: gcc -O3 -fopenmp -fPIC -shared (oracle/__init__.py).
 */
#include <omp.h>
#include <stdint.h>
#include <string.h>

typedef union {
    uint64_t bits;
    float v[2];
} pos2;

static inline pos2 get_pos(float *Y, int32_t i)
{
    pos2 p;
    p.bits = __atomic_load_n((uint64_t *)(Y + 2 * (int64_t)i), __ATOMIC_RELAXED);
    return p;
}

static inline void put_pos(float *Y, int32_t i, pos2 p)
{
    __atomic_store_n((uint64_t *)(Y + 2 * (int64_t)i), p.bits, __ATOMIC_RELAXED);
}

static void philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, uint32_t out[4])
{
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c0 = n0;
        c1 = (uint32_t)p1;
        c2 = n2;
        c3 = (uint32_t)p0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Runs epochs [epoch_begin, epoch_begin + epochs) on Y (n x 2 float32) with
 * `threads` OpenMP threads (<= 0: the OpenMP default).  bundle_order is a
 * permutation of the n rows.  Step size: linear decay eta0 (1 - t/T) floored
 * at eta_min (kind 0) or constant eta0 (kind 1).  Returns the number of
 * threads used. */
int cpu_hogwild_epochs(const int64_t *row_ptr, const int32_t *col_idx, int32_t n, float *Y, int32_t epoch_begin,
                       int32_t epochs, int32_t k, int32_t sched_kind, double eta0, double eta_min,
                       int32_t total_epochs, uint64_t seed, int32_t threads, const int32_t *bundle_order)
{
    if (threads <= 0)
        threads = omp_get_max_threads();
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    const uint32_t nm1 = (uint32_t)(n - 1);
    for (int32_t ep = 0; ep < epochs; ++ep) {
        const int32_t t = epoch_begin + ep;
        double etad = eta0;
        if (sched_kind == 0) {
            etad = eta0 * (1.0 - (double)t / (double)total_epochs);
            if (etad < eta_min)
                etad = eta_min;
        }
        const float eta = (float)etad;
#pragma omp parallel for schedule(dynamic, 16) num_threads(threads)
        for (int32_t q = 0; q < n; ++q) {
            const int32_t i = bundle_order[q];
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                const int32_t j = col_idx[e];
                pos2 yi = get_pos(Y, i), yj = get_pos(Y, j);
                float dx = yi.v[0] - yj.v[0], dy = yi.v[1] - yj.v[1];
                float ca = 0.1f * (1.0f + 8.0f / (1.0f + dx * dx + dy * dy));
                float fx = -ca * dx * eta, fy = -ca * dy * eta;
                yi.v[0] += fx;
                yi.v[1] += fy;
                yj.v[0] -= fx;
                yj.v[1] -= fy;
                put_pos(Y, j, yj);
                put_pos(Y, i, yi);
                uint32_t w[4] = {0, 0, 0, 0};
                for (int32_t m = 0; m < k; ++m) {
                    if ((m & 3) == 0)
                        philox((uint32_t)e, (uint32_t)((uint64_t)e >> 32), (uint32_t)t, (uint32_t)(m >> 2), key0, key1,
                               w);
                    const uint32_t u = (uint32_t)(((uint64_t)w[m & 3] * nm1) >> 32);
                    const int32_t s = (int32_t)(u + (u >= (uint32_t)i ? 1u : 0u));
                    yi = get_pos(Y, i);
                    pos2 ys = get_pos(Y, s);
                    float sx = yi.v[0] - ys.v[0], sy = yi.v[1] - ys.v[1];
                    float qr = 1.0f / (1.0f + sx * sx + sy * sy);
                    float cr = qr * qr * eta;
                    yi.v[0] += cr * sx;
                    yi.v[1] += cr * sy;
                    ys.v[0] -= cr * sx;
                    ys.v[1] -= cr * sy;
                    put_pos(Y, s, ys);
                    put_pos(Y, i, yi);
                }
            }
        }
    }
    return threads;
}
