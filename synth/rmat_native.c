/*
 * rmat_native.c -- seeded R-MAT generator for graphs too large for the numpy
 * generator (billions of edges): the same recursive-matrix model
 * (Chakrabarti, Zhan, Faloutsos, SDM 2004) and the same rules as
 * synth.graphs.rmat_graph, drawn from a counter-based stream so that the
 * result does not depend on the thread count.  Input generation only: no
 * arithmetic of the layout method lives here.
 *
 *   candidate t, level l: a uniform r in [0, 1) from splitmix64 of
 *   (seed, t, l / 2) (two 32-bit halves per call); row bit = r >= a + b,
 *   column bit = (a <= r < a + b) or r >= a + b + c.
 *   Undirected keys (min, max) without self-loops are collected, sorted and
 *   deduplicated; candidates are drawn in rounds until at least num_edges
 *   distinct edges exist; a surplus is removed by keeping the num_edges keys
 *   with the smallest 64-bit hash of (key, seed).
 *   Output: symmetric CSR, rows sorted ascending, no duplicates, no loops.
 *
 * Build: gcc -O3 -fopenmp -fPIC -shared (synth/__init__.py does it on first use).
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

/* Parallel LSD radix sort of n 64-bit keys on the low `bits` bits, 11 bits a pass. */
static int radix_sort(uint64_t *keys, int64_t n, int bits)
{
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    if (!tmp)
        return -1;
    const int R = 11, B = 1 << R;
    int T = omp_get_max_threads();
    int64_t *hist = (int64_t *)malloc(sizeof(int64_t) * (size_t)T * B);
    if (!hist) {
        free(tmp);
        return -1;
    }
    uint64_t *src = keys, *dst = tmp;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += R, ++passes) {
        memset(hist, 0, sizeof(int64_t) * (size_t)T * B);
#pragma omp parallel num_threads(T)
        {
            int t = omp_get_thread_num();
            int64_t lo = n * t / T, hi = n * (t + 1) / T;
            int64_t *h = hist + (size_t)t * B;
            for (int64_t i = lo; i < hi; ++i)
                h[(src[i] >> shift) & (B - 1)]++;
        }
        /* exclusive offsets: digit-major, thread-minor (stable) */
        int64_t run = 0;
        for (int d = 0; d < B; ++d)
            for (int t = 0; t < T; ++t) {
                int64_t c = hist[(size_t)t * B + d];
                hist[(size_t)t * B + d] = run;
                run += c;
            }
#pragma omp parallel num_threads(T)
        {
            int t = omp_get_thread_num();
            int64_t lo = n * t / T, hi = n * (t + 1) / T;
            int64_t *h = hist + (size_t)t * B;
            for (int64_t i = lo; i < hi; ++i)
                dst[h[(src[i] >> shift) & (B - 1)]++] = src[i];
        }
        uint64_t *sw = src;
        src = dst;
        dst = sw;
    }
    if (passes & 1)
        memcpy(keys, src, sizeof(uint64_t) * (size_t)n);
    free(tmp);
    free(hist);
    return 0;
}

static int64_t unique_sorted(uint64_t *k, int64_t n)
{
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        if (m == 0 || k[i] != k[m - 1])
            k[m++] = k[i];
    return m;
}

/* Fills row_ptr (n + 1) and col_idx (2 * num_edges).  Returns 0, -1 (memory)
 * or -2 (bad arguments). */
int rmat_native_generate(int32_t scale, int64_t num_edges, double a, double b, double c, uint64_t seed,
                         int32_t threads, int64_t *row_ptr, int32_t *col_idx)
{
    if (scale < 1 || scale > 30 || num_edges < 0 || a < 0 || b < 0 || c < 0 || a + b + c > 1.0)
        return -2;
    if (threads > 0)
        omp_set_num_threads(threads);
    const int64_t n = (int64_t)1 << scale;
    const uint32_t ta = (uint32_t)(a * 4294967296.0), tab = (uint32_t)((a + b) * 4294967296.0);
    const uint64_t tabc64 = (uint64_t)((a + b + c) * 4294967296.0);
    const uint32_t tabc = tabc64 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)tabc64;
    const int bits = 2 * scale;
    uint64_t *keys = NULL;
    int64_t have = 0, cap = 0;
    int64_t next_t = 0;
    int64_t draw = num_edges + num_edges / 4 + 1024;
    while (have < num_edges) {
        int64_t need = have + draw;
        if (need > cap) {
            uint64_t *nk = (uint64_t *)realloc(keys, sizeof(uint64_t) * (size_t)need);
            if (!nk) {
                free(keys);
                return -1;
            }
            keys = nk;
            cap = need;
        }
        int64_t base = next_t;
        uint64_t *out = keys + have;
        /* one candidate per slot; loops become an impossible key that sorts last */
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < draw; ++q) {
            uint64_t t = (uint64_t)(base + q);
            uint64_t row = 0, col = 0, w = 0;
            for (int l = 0; l < scale; ++l) {
                if ((l & 1) == 0)
                    w = splitmix64(seed * 0xD1B54A32D192ED03ull ^ (t * 64u + (uint64_t)(l >> 1)));
                uint32_t r = (l & 1) ? (uint32_t)(w >> 32) : (uint32_t)w;
                uint64_t rb = r >= tab;
                uint64_t cb = (r >= ta && r < tab) || r >= tabc;
                row = (row << 1) | rb;
                col = (col << 1) | cb;
            }
            uint64_t u = row < col ? row : col, v = row < col ? col : row;
            out[q] = u == v ? ~0ull : (u << scale) | v;
        }
        next_t += draw;
        int64_t tot = have + draw;
        if (radix_sort(keys, tot, bits + 1) != 0) {   /* +1 bit: the loop marker sorts last */
            free(keys);
            return -1;
        }
        int64_t m = unique_sorted(keys, tot);
        while (m > 0 && keys[m - 1] == ~0ull)
            --m;
        int64_t fresh = m - have;
        have = m;
        if (have >= num_edges)
            break;
        double frac = (double)fresh / (double)draw;
        if (frac < 0.05)
            frac = 0.05;
        draw = (int64_t)((double)(num_edges - have) / frac * 1.2) + 1024;
    }
    /* surplus: keep the num_edges keys of smallest hash(key, seed) */
    if (have > num_edges) {
        uint64_t *h = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)have);
        if (!h) {
            free(keys);
            return -1;
        }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < have; ++i)
            h[i] = splitmix64(keys[i] ^ (seed * 0x9E3779B97F4A7C15ull));
        uint64_t *hs = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)have);
        if (!hs) {
            free(h);
            free(keys);
            return -1;
        }
        memcpy(hs, h, sizeof(uint64_t) * (size_t)have);
        if (radix_sort(hs, have, 64) != 0) {
            free(h);
            free(hs);
            free(keys);
            return -1;
        }
        uint64_t thr = hs[num_edges - 1];
        int64_t below = 0;
        for (int64_t i = 0; i < num_edges; ++i)
            below += hs[i] < thr;
        int64_t at_thr = num_edges - below;   /* keys with hash == thr to keep, in key order */
        free(hs);
        int64_t m = 0;
        for (int64_t i = 0; i < have; ++i) {
            if (h[i] < thr || (h[i] == thr && at_thr-- > 0))
                keys[m++] = keys[i];
        }
        free(h);
        have = m;
    }
    /* symmetric CSR: row x = its smaller neighbours (from keys (u, x), ascending u),
     * then its larger ones (keys (x, v), ascending v) */
    const uint64_t mask = ((uint64_t)1 << scale) - 1;
    uint64_t *rev = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(have > 0 ? have : 1));
    int64_t *fdeg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *rdeg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!rev || !fdeg || !rdeg) {
        free(rev);
        free(fdeg);
        free(rdeg);
        free(keys);
        return -1;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < have; ++i) {
        uint64_t u = keys[i] >> scale, v = keys[i] & mask;
        rev[i] = (v << scale) | u;
    }
    if (radix_sort(rev, have, bits) != 0) {
        free(rev);
        free(fdeg);
        free(rdeg);
        free(keys);
        return -1;
    }
    for (int64_t i = 0; i < have; ++i) {
        fdeg[keys[i] >> scale]++;
        rdeg[rev[i] >> scale]++;
    }
    /* row offsets and the first key of each row in keys / rev */
    int64_t *fstart = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t *rstart = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!fstart || !rstart) {
        free(fstart);
        free(rstart);
        free(rev);
        free(fdeg);
        free(rdeg);
        free(keys);
        return -1;
    }
    row_ptr[0] = 0;
    fstart[0] = 0;
    rstart[0] = 0;
    for (int64_t x = 0; x < n; ++x) {
        row_ptr[x + 1] = row_ptr[x] + fdeg[x] + rdeg[x];
        fstart[x + 1] = fstart[x] + fdeg[x];
        rstart[x + 1] = rstart[x] + rdeg[x];
    }
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t x = 0; x < n; ++x) {
        int64_t p = row_ptr[x];
        for (int64_t i = rstart[x]; i < rstart[x + 1]; ++i)
            col_idx[p++] = (int32_t)(rev[i] & mask);
        for (int64_t i = fstart[x]; i < fstart[x + 1]; ++i)
            col_idx[p++] = (int32_t)(keys[i] & mask);
    }
    free(fstart);
    free(rstart);
    free(rev);
    free(fdeg);
    free(rdeg);
    free(keys);
    return 0;
}
