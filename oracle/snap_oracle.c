/*
 * snap_oracle.c -- sequential FP64 CPU oracle for SNAP-tFDP
 * ("Massively Scalable Graph Layouts via Sparse Negative Sampling").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the bench's CPU
 * baseline leg do.  It shares no code, header or constant table with the CUDA
 * path: every definition below is written out again from the paper.
 *
 * What it computes (citations are to the paper):
 *   - t-FDP forces and energies, Table 1 and Eq. 2 (alpha=0.1, beta=8, gamma=2,
 *     Section 3.1).
 *   - The degree-weighted objective, Eq. 4, with the weight the edge-centric
 *     sampler realises, (d_i+d_j)/(2(|V|-1)) (Section 3.3), and the designed
 *     weight of Eq. 5, (d_i+d_j)/(2|V|), for reference.
 *   - Algorithm 1 (edge-centric negative sampling), sequential, immediate
 *     updates, the directed edge list shuffled once before the epoch loop.
 *   - A synchronous (chunked Jacobi) variant: positions frozen within a chunk
 *     of rows, all forces of the chunk summed, then applied.  The paper has no
 *     such mode; it is the deterministic reference for the library's
 *     synchronous mode.
 *   - Neighbourhood preservation NP with r = 2 (Section 4.1, Metrics).
 *   - The cluster metrics of Section 4.1: silhouette index (SI) and clustering
 *     quality CQ = ARI(labels, k-means of the layout).
 *   - Weighted negatives (degree or caller weights, the future work of
 *     Section 6) through an alias table, and the objective whose expected
 *     gradient they follow (Section 3.3's derivation with P(s|i) in place of
 *     1/(|V|-1)).
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As
 *     Easy as 1, 2, 3", SC'11) for the negative draws.
 *
 * Readings of the paper that the code depends on:
 *   - Signs.  Table 1 prints attraction along +e_ij and repulsion along -e_ij
 *     with e_ij = (y_i - y_j)/|y_i - y_j|, and Algorithm 1 adds eta*F to y_i.
 *     Taken literally that pushes neighbours apart.  Section 3.1 states the
 *     physics (adjacent vertices drawn together, all vertices repel) and
 *     Eq. 2 states F = -grad U, so the force ON i is
 *        attraction  -alpha (1 + beta/(1+r^2)) (y_i - y_j)
 *        repulsion   +(1+r^2)^-gamma (y_i - y_s)
 *     and the partner always receives the opposite vector.
 *   - The attractive force of one step is evaluated once, from the positions
 *     before the step, and applied to both endpoints.
 *   - The loop index of the inner negative-sample loop of Algorithm 1 reuses
 *     the name j; it is read as a separate counter m = 0..k-1.
 *   - Negatives are uniform over V \ {i}: only the source is excluded; the
 *     draw may hit j and may repeat.
 *   - The step size decays linearly per epoch (Section 3.3 only says it
 *     follows standard practice and decays; Algorithm 1 updates it once per
 *     epoch): eta_t = max(eta0 * (1 - t/T), eta_min).
 *   - Random words: word w of the stream of directed edge e in epoch t is
 *     component (w mod 4) of Philox4x32-10(counter = (e_lo, e_hi, t, w div 4),
 *     key = (seed_lo, seed_hi)); e is the edge's index in the row-major CSR.
 *     The negatives of edge e = (i, j) consume its words in order.  Uniform
 *     (the paper's sampler) takes one word per negative:
 *     u = floor(word*(n-1)/2^32), s = u + (u >= i).
 *   - Weighted negatives (the paper's future work, Section 6: negatives drawn
 *     in proportion to a node weight -- the degree, or a caller's weight):
 *     Walker's alias method (Vose's construction) over integer weights q_s,
 *     two words per attempt -- column c = floor(w0*n/2^32), s = c if
 *     w1 < prob[c] else alias[c] -- an attempt that yields s = i is rejected
 *     and the next two words are tried; after 16 rejections the uniform rule
 *     above is applied to the next word.
 *
 * Build: plain C11, compiled with -ffp-contract=off so that no multiply-add
 * is fused (the rotation test relies on exact IEEE rounding of each op).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* t-FDP parameters recommended by the t-FDP authors and used by the paper
 * (Section 3.1, "t-FDP Model"). */
static const double ORC_ALPHA = 0.1;
static const double ORC_BETA = 8.0;
/* gamma = 2 is written into the formulas below: (1+r^2)^-2 and
 * U^r = (1+r^2)^(1-gamma) / (2(gamma-1)) = 1 / (2(1+r^2)). */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): a 10-round Feistel-like bijection   */
/* on 4x32-bit counters keyed by 2x32-bit keys.                              */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    /* round multipliers and Weyl key increments of Philox4x32 */
    const uint64_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += weyl0;
            k1 += weyl1;
        }
        uint64_t p0 = mult0 * (uint64_t)x0;
        uint64_t p1 = mult1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Word w of the random stream of directed edge e in epoch t. */
uint32_t oracle_edge_word(uint64_t e, uint32_t t, uint32_t w, uint64_t seed)
{
    uint32_t ctr[4] = {(uint32_t)e, (uint32_t)(e >> 32), t, w / 4u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[w % 4u];
}

/* Uniform draw over every vertex except the source i (the negative sample of
 * Algorithm 1). */
int32_t oracle_uniform_negative(uint32_t word, int32_t i, int32_t n)
{
    uint32_t u = (uint32_t)(((uint64_t)word * (uint64_t)(uint32_t)(n - 1)) >> 32);
    return (int32_t)(u + (u >= (uint32_t)i ? 1u : 0u));
}

/* ------------------------------------------------------------------------ */
/* Weighted negative sampling (Section 6 names non-uniform negatives as      */
/* future work; the weight is the degree for the DEGREE sampler).            */
/* ------------------------------------------------------------------------ */

/* Caller weights (float, >= 0, finite, not all zero) to integers:
 * q_s = llround(w_s / max_w * 2^32), so 0 <= q_s <= 2^32.  Returns 0 or -1. */
int oracle_quantize_weights(const float *w, int32_t n, uint64_t *q)
{
    double wmax = 0.0;
    for (int32_t s = 0; s < n; ++s) {
        double v = (double)w[s];
        if (!(v >= 0.0) || isinf(v))
            return -1;
        if (v > wmax)
            wmax = v;
    }
    if (!(wmax > 0.0))
        return -1;
    for (int32_t s = 0; s < n; ++s)
        q[s] = (uint64_t)llround((double)w[s] / wmax * 4294967296.0);
    return 0;
}

/* floor(a * 2^32 / b) for a < b < 2^63, by binary long division. */
static uint32_t frac32(uint64_t a, uint64_t b)
{
    uint32_t r = 0;
    for (int bit = 0; bit < 32; ++bit) {
        a <<= 1;
        r <<= 1;
        if (a >= b) {
            a -= b;
            r |= 1u;
        }
    }
    return r;
}

/* Alias table of the integer weights q (Walker; Vose's construction in exact
 * integer arithmetic).  In units where every column holds Q = sum q, node s
 * brings n*q_s.  Worklists: `small` (n*q_s < Q) is a first-in-first-out
 * queue and `large` a stack, both filled in increasing s.  Repeatedly the
 * first small node l keeps its own mass in column l and the top large node
 * g fills the rest of column l (alias[l] = g) and loses that much; g moves
 * to the small queue when it falls below Q.  Nodes left over fill their own
 * column.  prob[c] = floor(mass_c * 2^32 / Q) for a column shared with its
 * alias; a full column has prob 0xFFFFFFFF and alias c.
 * Requires n * max q < 2^64 and 0 < Q < 2^63.  Returns 0 or -1. */
int oracle_alias_build(const uint64_t *q, int32_t n, uint32_t *prob, int32_t *alias)
{
    uint64_t Q = 0;
    for (int32_t s = 0; s < n; ++s)
        Q += q[s];
    if (n < 1 || Q == 0)
        return -1;
    uint64_t *mass = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    int32_t *small = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *large = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!mass || !small || !large) {
        free(mass);
        free(small);
        free(large);
        return -1;
    }
    int64_t s_head = 0, s_tail = 0, l_top = 0;
    for (int32_t s = 0; s < n; ++s) {
        mass[s] = (uint64_t)n * q[s];
        if (mass[s] < Q)
            small[s_tail++] = s;
        else
            large[l_top++] = s;
    }
    for (int32_t s = 0; s < n; ++s) {
        prob[s] = 0xFFFFFFFFu;
        alias[s] = s;
    }
    while (s_head < s_tail && l_top > 0) {
        int32_t l = small[s_head++];
        int32_t g = large[l_top - 1];
        prob[l] = frac32(mass[l], Q);
        alias[l] = g;
        mass[g] -= Q - mass[l];
        if (mass[g] < Q) {
            --l_top;
            small[s_tail++] = g;
        }
    }
    /* exact arithmetic conserves n*Q in total: whatever is left is full */
    free(mass);
    free(small);
    free(large);
    return 0;
}

/* Word stream of one directed edge: the negatives consume it in order. */
typedef struct {
    uint64_t e;
    uint32_t t;
    uint64_t seed;
    uint32_t next;
} word_cursor;

static uint32_t take_word(word_cursor *c)
{
    return oracle_edge_word(c->e, c->t, c->next++, c->seed);
}

/* The next negative of source i (uniform when prob == NULL). */
static int32_t draw_negative(word_cursor *c, int32_t i, int32_t n, const uint32_t *prob, const int32_t *alias)
{
    if (prob) {
        for (int attempt = 0; attempt < 16; ++attempt) {
            uint32_t w0 = take_word(c);
            uint32_t w1 = take_word(c);
            int32_t col = (int32_t)(((uint64_t)w0 * (uint64_t)(uint32_t)n) >> 32);
            int32_t s = w1 < prob[col] ? col : alias[col];
            if (s != i)
                return s;
        }
    }
    return oracle_uniform_negative(take_word(c), i, n);
}

/* Negatives m = 0..k-1 of directed edge e in epoch t, and the number of
 * words they consumed (for the tests). */
uint32_t oracle_edge_negatives(uint64_t e, uint32_t t, uint64_t seed, int32_t i, int32_t n, int32_t k,
                               const uint32_t *prob, const int32_t *alias, int32_t *out)
{
    word_cursor c = {e, t, seed, 0u};
    for (int32_t m = 0; m < k; ++m)
        out[m] = draw_negative(&c, i, n, prob, alias);
    return c.next;
}

/* Probability that one negative of source i is s (s != i) under the sampler
 * with weights q (NULL: uniform, 1/(n-1)).  A weighted attempt accepts with
 * probability 1 - rho_i, rho_i = q_i/Q; after 16 rejections the draw is
 * uniform: P(s|i) = (1 - rho_i^16) q_s / (Q - q_i) + rho_i^16 / (n-1).
 * (The alias table realises q_s/Q up to its 2^-32 thresholds.) */
static double negative_prob(const uint64_t *q, uint64_t Q, int32_t n, int32_t i, int32_t s)
{
    if (!q)
        return 1.0 / (double)(n - 1);
    double rho = (double)q[i] / (double)Q;
    double r2 = rho * rho, r4 = r2 * r2, r8 = r4 * r4, r16 = r8 * r8;
    uint64_t rest = Q - q[i];
    double p = rest > 0 ? (1.0 - r16) * (double)q[s] / (double)rest : 0.0;
    return p + r16 / (double)(n - 1);
}

/* Pair coefficient of the objective generalised from Section 3.3:
 * c_ij = d_i P(j|i) + d_j P(i|j); w_ij = c_ij / 2.  Uniform: (d_i+d_j)/(n-1). */
static double pair_coefficient(const int64_t *row_ptr, const uint64_t *q, uint64_t Q, int32_t n, int32_t i,
                               int32_t j)
{
    double di = (double)(row_ptr[i + 1] - row_ptr[i]);
    double dj = (double)(row_ptr[j + 1] - row_ptr[j]);
    return di * negative_prob(q, Q, n, i, j) + dj * negative_prob(q, Q, n, j, i);
}

static uint64_t weight_total(const uint64_t *q, int32_t n)
{
    uint64_t Q = 0;
    if (q)
        for (int32_t s = 0; s < n; ++s)
            Q += q[s];
    return Q;
}

/* Step size of epoch t (the paper: it decays with the epochs and changes once
 * per epoch). */
double oracle_step_size(int32_t kind, double eta0, double eta_min, int32_t total_epochs, int32_t t)
{
    if (kind == 1)
        return eta0;                       /* constant */
    double T = (double)(total_epochs > 0 ? total_epochs : 1);
    double eta = eta0 * (1.0 - (double)t / T);
    return eta > eta_min ? eta : eta_min;  /* linear decay with a floor */
}

/* Force on i for the displacement d = y_i - y_other, and the two energies.
 * out = {Fa_x, Fa_y, Fr_x, Fr_y, Ua, Ur}.                                  */
void oracle_pair_terms(double dx, double dy, double out[6])
{
    double r2 = dx * dx + dy * dy;
    double one_r2 = 1.0 + r2;
    /* Table 1, t-FDP attraction: magnitude alpha (r + beta r / (1+r^2)),
     * pulling i toward the neighbour. */
    double ca = ORC_ALPHA * (1.0 + ORC_BETA / one_r2);
    /* Table 1, t-FDP repulsion: magnitude r / (1+r^2)^gamma, gamma = 2,
     * pushing i away from the sample. */
    double cr = 1.0 / (one_r2 * one_r2);
    out[0] = -ca * dx;
    out[1] = -ca * dy;
    out[2] = cr * dx;
    out[3] = cr * dy;
    /* Eq. 2: the energies whose negative gradients are the forces above. */
    out[4] = ORC_ALPHA * (0.5 * r2 + 0.5 * ORC_BETA * log1p(r2));
    out[5] = 0.5 / one_r2;
}

static void attraction_on_i(double dx, double dy, double *fx, double *fy)
{
    double r2 = dx * dx + dy * dy;
    double ca = ORC_ALPHA * (1.0 + ORC_BETA / (1.0 + r2));
    *fx = -ca * dx;
    *fy = -ca * dy;
}

static void repulsion_on_i(double dx, double dy, double *fx, double *fy)
{
    double r2 = dx * dx + dy * dy;
    double one_r2 = 1.0 + r2;
    double cr = 1.0 / (one_r2 * one_r2);
    *fx = cr * dx;
    *fy = cr * dy;
}

static double energy_attr(double dx, double dy)
{
    double r2 = dx * dx + dy * dy;
    return ORC_ALPHA * (0.5 * r2 + 0.5 * ORC_BETA * log1p(r2));
}

static double energy_rep(double dx, double dy)
{
    double r2 = dx * dx + dy * dy;
    return 0.5 / (1.0 + r2);
}

static int32_t *row_of_edges(const int64_t *row_ptr, int32_t n)
{
    int64_t nnz = row_ptr[n];
    int32_t *src = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    if (!src)
        return NULL;
    for (int32_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            src[e] = i;
    return src;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1, sequential, immediate updates.                              */
/* Y is n x 2 row-major doubles, updated in place.  shuffle = 0 keeps the   */
/* CSR order; given_order (nullable, a permutation of the nnz CSR indices)  */
/* fixes the visiting order instead -- each is one of the orders the        */
/* shuffle of Algorithm 1 can produce.                                      */
/* max_edges_per_epoch < 0 processes every edge; otherwise only that many   */
/* edges of the shuffled order are visited in each epoch (a timing sample). */
/* actual_energy (nullable, one value per epoch): half the sum of U^a over  */
/* the visited directed edges plus U^r over the drawn pairs, each taken at  */
/* the moment of its update (Section 3.3's actual energy).                  */
/* Returns 0, or -1 on allocation failure.                                  */
/* ------------------------------------------------------------------------ */
int oracle_seq(const int64_t *row_ptr, const int32_t *col_idx, int32_t n, double *Y,
               int32_t epoch_begin, int32_t epochs, int32_t k,
               int32_t sched_kind, double eta0, double eta_min, int32_t total_epochs,
               uint64_t seed, int32_t shuffle, uint64_t shuffle_seed, int64_t max_edges_per_epoch,
               double *actual_energy, const int64_t *given_order, const uint32_t *prob, const int32_t *alias)
{
    int64_t nnz = row_ptr[n];
    int32_t *src = row_of_edges(row_ptr, n);
    int64_t *order = (int64_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t));
    if (!src || !order) {
        free(src);
        free(order);
        return -1;
    }
    /* "Randomly shuffle edge list E" -- once, before the epoch loop
     * (Fisher-Yates, driven by its own Philox stream). */
    for (int64_t e = 0; e < nnz; ++e)
        order[e] = given_order ? given_order[e] : e;
    if (given_order)
        shuffle = 0;
    uint32_t skey[2] = {(uint32_t)shuffle_seed, (uint32_t)(shuffle_seed >> 32)};
    for (int64_t p = shuffle ? nnz - 1 : 0; p > 0; --p) {
        uint32_t ctr[4] = {(uint32_t)p, (uint32_t)((uint64_t)p >> 32), 0xFFFFFFFEu, 0u};
        uint32_t w[4];
        oracle_philox4x32_10(ctr, skey, w);
        uint64_t r64 = ((uint64_t)w[0] << 32) | w[1];
        int64_t q = (int64_t)(r64 % (uint64_t)(p + 1));
        int64_t tmp = order[p];
        order[p] = order[q];
        order[q] = tmp;
    }
    int64_t visit = (max_edges_per_epoch >= 0 && max_edges_per_epoch < nnz) ? max_edges_per_epoch : nnz;

    for (int32_t ep = 0; ep < epochs; ++ep) {
        int32_t t = epoch_begin + ep;
        double eta = oracle_step_size(sched_kind, eta0, eta_min, total_epochs, t);
        double energy = 0.0;
        for (int64_t q = 0; q < visit; ++q) {
            int64_t e = order[q];
            int32_t i = src[e];
            int32_t j = col_idx[e];
            double *yi = Y + 2 * (int64_t)i;
            double *yj = Y + 2 * (int64_t)j;
            double dx = yi[0] - yj[0], dy = yi[1] - yj[1];
            double fx, fy;
            if (actual_energy)
                energy += energy_attr(dx, dy);
            attraction_on_i(dx, dy, &fx, &fy);
            yi[0] += eta * fx;
            yi[1] += eta * fy;
            yj[0] -= eta * fx;
            yj[1] -= eta * fy;
            word_cursor cur = {(uint64_t)e, (uint32_t)t, seed, 0u};
            for (int32_t m = 0; m < k; ++m) {
                int32_t s = draw_negative(&cur, i, n, prob, alias);
                double *ys = Y + 2 * (int64_t)s;
                double sx = yi[0] - ys[0], sy = yi[1] - ys[1];
                if (actual_energy)
                    energy += energy_rep(sx, sy);
                repulsion_on_i(sx, sy, &fx, &fy);
                yi[0] += eta * fx;
                yi[1] += eta * fy;
                ys[0] -= eta * fx;
                ys[1] -= eta * fy;
            }
        }
        if (actual_energy)
            actual_energy[ep] = 0.5 * energy;
    }
    free(src);
    free(order);
    return 0;
}

/* Row boundaries of the synchronous chunks: chunk c holds rows
 * [bound[c], bound[c+1]); bound[c] for 0 < c < S is the first row r with
 * row_ptr[r] * S >= c * nnz. */
void oracle_sync_chunk_bounds(const int64_t *row_ptr, int32_t n, int32_t S, int32_t *bound)
{
    int64_t nnz = row_ptr[n];
    bound[0] = 0;
    bound[S] = n;
    int32_t r = 0;
    for (int32_t c = 1; c < S; ++c) {
        while (r < n && row_ptr[r] * (int64_t)S < (int64_t)c * nnz)
            ++r;
        bound[c] = r;
    }
}

/* Sum of all sampled forces of rows [r0, r1) with Y frozen, in CSR order,
 * added into D (n x 2). */
static void chunk_displacement(const int64_t *row_ptr, const int32_t *col_idx, int32_t n,
                               const double *Y, int32_t r0, int32_t r1, int32_t k,
                               uint32_t t, uint64_t seed, const uint32_t *prob, const int32_t *alias, double *D)
{
    for (int32_t i = r0; i < r1; ++i) {
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            double fx, fy;
            attraction_on_i(Y[2 * (int64_t)i] - Y[2 * (int64_t)j],
                            Y[2 * (int64_t)i + 1] - Y[2 * (int64_t)j + 1], &fx, &fy);
            D[2 * (int64_t)i] += fx;
            D[2 * (int64_t)i + 1] += fy;
            D[2 * (int64_t)j] -= fx;
            D[2 * (int64_t)j + 1] -= fy;
            word_cursor cur = {(uint64_t)e, t, seed, 0u};
            for (int32_t m = 0; m < k; ++m) {
                int32_t s = draw_negative(&cur, i, n, prob, alias);
                repulsion_on_i(Y[2 * (int64_t)i] - Y[2 * (int64_t)s],
                               Y[2 * (int64_t)i + 1] - Y[2 * (int64_t)s + 1], &fx, &fy);
                D[2 * (int64_t)i] += fx;
                D[2 * (int64_t)i + 1] += fy;
                D[2 * (int64_t)s] -= fx;
                D[2 * (int64_t)s + 1] -= fy;
            }
        }
    }
}

/* One frozen-position epoch displacement (all rows, one chunk): the sampled
 * estimate whose expectation Section 3.3 derives. */
int oracle_epoch_displacement(const int64_t *row_ptr, const int32_t *col_idx, int32_t n,
                              const double *Y, int32_t t, int32_t k, uint64_t seed,
                              const uint32_t *prob, const int32_t *alias, double *D)
{
    memset(D, 0, sizeof(double) * 2 * (size_t)n);
    chunk_displacement(row_ptr, col_idx, n, Y, 0, n, k, (uint32_t)t, seed, prob, alias, D);
    return 0;
}

/* One chunk step of the synchronous mode: the forces of the edges of rows
 * [r0, r1) and of their negatives, summed from Y frozen at the chunk's start
 * (D is n x 2 scratch), then Y += eta * D, each vertex's step clipped to
 * length `limit` when limit > 0. */
static void sync_chunk_step(const int64_t *row_ptr, const int32_t *col_idx, int32_t n, double *Y,
                            int32_t r0, int32_t r1, int32_t k, uint32_t t, uint64_t seed, double eta,
                            double limit, const uint32_t *prob, const int32_t *alias, double *D)
{
    memset(D, 0, sizeof(double) * 2 * (size_t)n);
    chunk_displacement(row_ptr, col_idx, n, Y, r0, r1, k, t, seed, prob, alias, D);
    for (int32_t i = 0; i < n; ++i) {
        double sx = eta * D[2 * (int64_t)i], sy = eta * D[2 * (int64_t)i + 1];
        if (limit > 0.0) {
            double len = sqrt(sx * sx + sy * sy);
            if (len > limit) {
                sx *= limit / len;
                sy *= limit / len;
            }
        }
        Y[2 * (int64_t)i] += sx;
        Y[2 * (int64_t)i + 1] += sy;
    }
}

/* Synchronous mode: per epoch, S chunks of rows; for each chunk the forces of
 * its edges and negatives are summed from positions frozen at the chunk's
 * start, then Y += eta_t * D.  With cap > 0 each node's step is clipped to
 * length cap * eta_t / eta0.  Returns 0, or -1 on allocation failure. */
int oracle_sync(const int64_t *row_ptr, const int32_t *col_idx, int32_t n, double *Y,
                int32_t epoch_begin, int32_t epochs, int32_t k,
                int32_t sched_kind, double eta0, double eta_min, int32_t total_epochs,
                uint64_t seed, int32_t S, double cap, const uint32_t *prob, const int32_t *alias)
{
    if (S < 1)
        S = 1;
    double *D = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
    int32_t *bound = (int32_t *)malloc(sizeof(int32_t) * (size_t)(S + 1));
    if (!D || !bound) {
        free(D);
        free(bound);
        return -1;
    }
    oracle_sync_chunk_bounds(row_ptr, n, S, bound);
    for (int32_t ep = 0; ep < epochs; ++ep) {
        int32_t t = epoch_begin + ep;
        double eta = oracle_step_size(sched_kind, eta0, eta_min, total_epochs, t);
        double limit = cap > 0.0 ? cap * eta / eta0 : 0.0;
        for (int32_t c = 0; c < S; ++c)
            sync_chunk_step(row_ptr, col_idx, n, Y, bound[c], bound[c + 1], k, (uint32_t)t, seed, eta, limit,
                            prob, alias, D);
    }
    free(D);
    free(bound);
    return 0;
}

/* Chunks [c_begin, c_end) of S of epoch t of the synchronous mode, applied to
 * Y in order: the same steps oracle_sync takes for those chunks, started
 * from whatever Y the caller passes (e.g. another implementation's positions
 * at a chunk boundary).  Returns 0, -1 on allocation failure, -2 on a bad
 * chunk range. */
int oracle_sync_chunks(const int64_t *row_ptr, const int32_t *col_idx, int32_t n, double *Y, int32_t t,
                       int32_t c_begin, int32_t c_end, int32_t S, int32_t k, int32_t sched_kind, double eta0,
                       double eta_min, int32_t total_epochs, uint64_t seed, double cap, const uint32_t *prob,
                       const int32_t *alias)
{
    if (S < 1 || c_begin < 0 || c_end > S || c_begin > c_end)
        return -2;
    double *D = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
    int32_t *bound = (int32_t *)malloc(sizeof(int32_t) * (size_t)(S + 1));
    if (!D || !bound) {
        free(D);
        free(bound);
        return -1;
    }
    oracle_sync_chunk_bounds(row_ptr, n, S, bound);
    double eta = oracle_step_size(sched_kind, eta0, eta_min, total_epochs, t);
    double limit = cap > 0.0 ? cap * eta / eta0 : 0.0;
    for (int32_t c = c_begin; c < c_end; ++c)
        sync_chunk_step(row_ptr, col_idx, n, Y, bound[c], bound[c + 1], k, (uint32_t)t, seed, eta, limit, prob,
                        alias, D);
    free(D);
    free(bound);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Objective (Eq. 4) with the weight realised by uniform edge-centric       */
/* sampling (Section 3.3): w_ij = (d_i+d_j) / (2(n-1)); with weighted       */
/* negatives (q != NULL) w_ij = c_ij / 2 from pair_coefficient.             */
/* out = {attraction, repulsion, total, repulsion with Eq. 5's 2n weight    */
/* (uniform only; 0 otherwise)}.                                            */
/* ------------------------------------------------------------------------ */
int oracle_objective(const int64_t *row_ptr, const int32_t *col_idx, int32_t n,
                     const double *Y, int32_t k, const uint64_t *q, double out[4])
{
    double attr = 0.0;
    for (int32_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            if (i < j)
                attr += energy_attr(Y[2 * (int64_t)i] - Y[2 * (int64_t)j],
                                    Y[2 * (int64_t)i + 1] - Y[2 * (int64_t)j + 1]);
        }
    if (q) {
        uint64_t Q = weight_total(q, n);
        double rep = 0.0;   /* sum over i<j of w_ij U^r */
        for (int32_t i = 0; i < n; ++i)
            for (int32_t j = i + 1; j < n; ++j)
                rep += 0.5 * pair_coefficient(row_ptr, q, Q, n, i, j) *
                       energy_rep(Y[2 * (int64_t)i] - Y[2 * (int64_t)j], Y[2 * (int64_t)i + 1] - Y[2 * (int64_t)j + 1]);
        out[0] = attr;
        out[1] = (double)k * rep;
        out[2] = attr + out[1];
        out[3] = 0.0;
        return 0;
    }
    double rep_num = 0.0;   /* sum over i<j of (d_i + d_j) U^r */
    for (int32_t i = 0; i < n; ++i) {
        double di = (double)(row_ptr[i + 1] - row_ptr[i]);
        for (int32_t j = i + 1; j < n; ++j) {
            double dj = (double)(row_ptr[j + 1] - row_ptr[j]);
            rep_num += (di + dj) * energy_rep(Y[2 * (int64_t)i] - Y[2 * (int64_t)j],
                                              Y[2 * (int64_t)i + 1] - Y[2 * (int64_t)j + 1]);
        }
    }
    double rep = n > 1 ? (double)k * rep_num / (2.0 * (double)(n - 1)) : 0.0;
    out[0] = attr;
    out[1] = rep;
    out[2] = attr + rep;
    out[3] = n > 0 ? (double)k * rep_num / (2.0 * (double)n) : 0.0;
    return 0;
}

/* Unbiased estimate of the same objective for large n: the attraction sum is
 * exact; the pair sum is n(n-1)/2 times the mean over `pairs` uniform
 * unordered pairs drawn from Philox(counter = (p_lo, p_hi, 0xFFFFFFFD, 0),
 * key = seed).  out as in oracle_objective (out[3] left 0). */
int oracle_objective_sampled(const int64_t *row_ptr, const int32_t *col_idx, int32_t n,
                             const double *Y, int32_t k, int64_t pairs, uint64_t seed,
                             const uint64_t *q, double out[4])
{
    uint64_t Q = weight_total(q, n);
    double attr = 0.0;
    for (int32_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            if (i < j)
                attr += energy_attr(Y[2 * (int64_t)i] - Y[2 * (int64_t)j],
                                    Y[2 * (int64_t)i + 1] - Y[2 * (int64_t)j + 1]);
        }
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double acc = 0.0;
    for (int64_t p = 0; p < pairs; ++p) {
        uint32_t ctr[4] = {(uint32_t)p, (uint32_t)((uint64_t)p >> 32), 0xFFFFFFFDu, 0u};
        uint32_t w[4];
        oracle_philox4x32_10(ctr, key, w);
        int32_t i = (int32_t)(((uint64_t)w[0] * (uint64_t)(uint32_t)n) >> 32);
        int32_t j = oracle_uniform_negative(w[1], i, n);
        double di = (double)(row_ptr[i + 1] - row_ptr[i]);
        double dj = (double)(row_ptr[j + 1] - row_ptr[j]);
        double c = q ? pair_coefficient(row_ptr, q, Q, n, i, j) : (di + dj) / (double)(n - 1);
        acc += c * energy_rep(Y[2 * (int64_t)i] - Y[2 * (int64_t)j],
                              Y[2 * (int64_t)i + 1] - Y[2 * (int64_t)j + 1]);
    }
    double npairs = 0.5 * (double)n * (double)(n - 1);
    double rep = pairs > 0 && n > 1 ? (double)k * (acc / (double)pairs) * npairs / 2.0 : 0.0;
    out[0] = attr;
    out[1] = rep;
    out[2] = attr + rep;
    out[3] = 0.0;
    return 0;
}

/* Gradient of the objective above with respect to every y_i (n x 2). */
int oracle_exact_gradient(const int64_t *row_ptr, const int32_t *col_idx, int32_t n,
                          const double *Y, int32_t k, const uint64_t *q, double *G)
{
    memset(G, 0, sizeof(double) * 2 * (size_t)n);
    for (int32_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            double fx, fy;
            attraction_on_i(Y[2 * (int64_t)i] - Y[2 * (int64_t)j],
                            Y[2 * (int64_t)i + 1] - Y[2 * (int64_t)j + 1], &fx, &fy);
            G[2 * (int64_t)i] -= fx;          /* grad = -force */
            G[2 * (int64_t)i + 1] -= fy;
        }
    if (n < 2)
        return 0;
    double norm = (double)k / (2.0 * (double)(n - 1));
    uint64_t Q = weight_total(q, n);
    for (int32_t i = 0; i < n; ++i) {
        double di = (double)(row_ptr[i + 1] - row_ptr[i]);
        for (int32_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            double dj = (double)(row_ptr[j + 1] - row_ptr[j]);
            /* k * w_ij, w_ij = c_ij / 2 */
            double kw = q ? 0.5 * (double)k * pair_coefficient(row_ptr, q, Q, n, i, j) : norm * (di + dj);
            double fx, fy;
            repulsion_on_i(Y[2 * (int64_t)i] - Y[2 * (int64_t)j],
                           Y[2 * (int64_t)i + 1] - Y[2 * (int64_t)j + 1], &fx, &fy);
            G[2 * (int64_t)i] -= kw * fx;
            G[2 * (int64_t)i + 1] -= kw * fy;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Neighbourhood preservation (Section 4.1, Metrics), r = 2:                */
/*   NP = mean_i |N_G(i,2) & N_L(i,k_i)| / |N_G(i,2) | N_L(i,k_i)|,         */
/* N_G(i,2) = nodes within two hops of i (i excluded), k_i = |N_G(i,2)|,    */
/* N_L(i,k_i) = the k_i nodes nearest to y_i in the layout (i excluded),    */
/* ties broken by the smaller node id.  Nodes with k_i = 0 are skipped.     */
/* nodes == NULL evaluates every node, else the `count` listed ones.        */
/* ------------------------------------------------------------------------ */
typedef struct {
    double d2;
    int32_t id;
} np_item;

static int np_less(const np_item *a, const np_item *b)
{
    return a->d2 < b->d2 || (a->d2 == b->d2 && a->id < b->id);
}

/* Rearrange v[0..len) so that its first kth items are the kth smallest. */
static void np_select(np_item *v, int64_t len, int64_t kth)
{
    int64_t lo = 0, hi = len - 1;
    uint64_t state = 0x9E3779B97F4A7C15ull;
    while (lo < hi) {
        state = state * 6364136223846793005ull + 1442695040888963407ull;
        int64_t pidx = lo + (int64_t)((state >> 33) % (uint64_t)(hi - lo + 1));
        np_item pivot = v[pidx];
        int64_t a = lo, b = hi;
        while (a <= b) {
            while (np_less(&v[a], &pivot)) ++a;
            while (np_less(&pivot, &v[b])) --b;
            if (a <= b) {
                np_item tmp = v[a]; v[a] = v[b]; v[b] = tmp;
                ++a; --b;
            }
        }
        if (kth - 1 <= b)
            hi = b;
        else if (kth - 1 >= a)
            lo = a;
        else
            break;
    }
}

double oracle_neighborhood_preservation(const int64_t *row_ptr, const int32_t *col_idx, int32_t n,
                                        const double *Y, const int32_t *nodes, int32_t count)
{
    int32_t *stamp = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    np_item *items = (np_item *)malloc(sizeof(np_item) * (size_t)(n > 0 ? n : 1));
    if (!stamp || !items) {
        free(stamp);
        free(items);
        return -1.0;
    }
    int32_t total = nodes ? count : n;
    double sum = 0.0;
    int32_t used = 0;
    for (int32_t q = 0; q < total; ++q) {
        int32_t i = nodes ? nodes[q] : q;
        int32_t mark = q + 1;
        int64_t ki = 0;
        stamp[i] = mark;   /* exclude i itself */
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            if (stamp[j] != mark) { stamp[j] = mark; ++ki; }
        }
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            for (int64_t f = row_ptr[j]; f < row_ptr[j + 1]; ++f) {
                int32_t l = col_idx[f];
                if (stamp[l] != mark) { stamp[l] = mark; ++ki; }
            }
        }
        if (ki == 0)
            continue;
        int64_t len = 0;
        for (int32_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            double dx = Y[2 * (int64_t)i] - Y[2 * (int64_t)j];
            double dy = Y[2 * (int64_t)i + 1] - Y[2 * (int64_t)j + 1];
            items[len].d2 = dx * dx + dy * dy;
            items[len].id = j;
            ++len;
        }
        np_select(items, len, ki);
        int64_t inter = 0;
        for (int64_t p = 0; p < ki; ++p)
            if (stamp[items[p].id] == mark)
                ++inter;
        sum += (double)inter / (double)(2 * ki - inter);
        ++used;
        /* the stamp value of the next node differs, so no reset is needed */
    }
    free(stamp);
    free(items);
    return used > 0 ? sum / (double)used : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Cluster metrics of Section 4.1 (evaluation only).                        */
/* ------------------------------------------------------------------------ */

/* Silhouette index (Rousseeuw 1987) of the layout under ground-truth labels
 * 0..K-1: s(i) = (b(i) - a(i)) / max(a(i), b(i)), a(i) the mean distance
 * from i to the other members of its cluster, b(i) the smallest mean
 * distance from i to the members of another cluster; s(i) = 0 for a member
 * of a singleton cluster.  Mean over `nodes` (NULL: every vertex), with
 * distances to every vertex.  Returns the mean, or NaN on allocation failure
 * or K < 2. */
double oracle_silhouette(const double *Y, const int32_t *labels, int32_t n, int32_t K,
                         const int32_t *nodes, int32_t count)
{
    if (K < 2)
        return NAN;
    double *sum = (double *)malloc(sizeof(double) * (size_t)K);
    int64_t *size = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    if (!sum || !size) {
        free(sum);
        free(size);
        return NAN;
    }
    for (int32_t v = 0; v < n; ++v)
        size[labels[v]]++;
    int32_t m = nodes ? count : n;
    double total = 0.0;
    for (int32_t q = 0; q < m; ++q) {
        int32_t i = nodes ? nodes[q] : q;
        for (int32_t c = 0; c < K; ++c)
            sum[c] = 0.0;
        for (int32_t v = 0; v < n; ++v) {
            if (v == i)
                continue;
            double dx = Y[2 * (int64_t)i] - Y[2 * (int64_t)v], dy = Y[2 * (int64_t)i + 1] - Y[2 * (int64_t)v + 1];
            sum[labels[v]] += sqrt(dx * dx + dy * dy);
        }
        int32_t own = labels[i];
        if (size[own] < 2)
            continue;   /* s(i) = 0 */
        double a = sum[own] / (double)(size[own] - 1);
        double b = INFINITY;
        for (int32_t c = 0; c < K; ++c)
            if (c != own && size[c] > 0 && sum[c] / (double)size[c] < b)
                b = sum[c] / (double)size[c];
        double mx = a > b ? a : b;
        total += mx > 0.0 ? (b - a) / mx : 0.0;
    }
    free(sum);
    free(size);
    return m > 0 ? total / (double)m : 0.0;
}

/* Adjusted Rand index (Hubert & Arabie 1985) of two labelings with labels in
 * [0, Ka) and [0, Kb): (I - E) / (M - E), I = sum over the contingency table
 * of C(n_ij, 2), E = sum_i C(a_i, 2) sum_j C(b_j, 2) / C(n, 2), M = the mean
 * of the two marginal sums.  1 for identical partitions. */
double oracle_adjusted_rand(const int32_t *la, const int32_t *lb, int32_t n, int32_t Ka, int32_t Kb)
{
    int64_t *tab = (int64_t *)calloc((size_t)Ka * (size_t)Kb, sizeof(int64_t));
    int64_t *ra = (int64_t *)calloc((size_t)Ka, sizeof(int64_t));
    int64_t *rb = (int64_t *)calloc((size_t)Kb, sizeof(int64_t));
    if (!tab || !ra || !rb) {
        free(tab);
        free(ra);
        free(rb);
        return NAN;
    }
    for (int32_t v = 0; v < n; ++v) {
        tab[(size_t)la[v] * (size_t)Kb + (size_t)lb[v]]++;
        ra[la[v]]++;
        rb[lb[v]]++;
    }
    double I = 0.0, A = 0.0, B = 0.0;
    for (size_t t = 0; t < (size_t)Ka * (size_t)Kb; ++t)
        I += 0.5 * (double)tab[t] * (double)(tab[t] - 1);
    for (int32_t i = 0; i < Ka; ++i)
        A += 0.5 * (double)ra[i] * (double)(ra[i] - 1);
    for (int32_t j = 0; j < Kb; ++j)
        B += 0.5 * (double)rb[j] * (double)(rb[j] - 1);
    free(tab);
    free(ra);
    free(rb);
    double pairs = 0.5 * (double)n * (double)(n - 1);
    double E = pairs > 0.0 ? A * B / pairs : 0.0;
    double M = 0.5 * (A + B);
    return M - E != 0.0 ? (I - E) / (M - E) : 1.0;
}

/* k-means of the layout (Lloyd's iterations from a k-means++ start, Arthur &
 * Vassilvitskii 2007; the start's random numbers from Philox with counter
 * (draw, 0, 0xFFFFFFFC, restart) and key seed), `restarts` starts, the
 * partition of least inertia written to out.  Returns that inertia, or -1. */
double oracle_kmeans(const double *Y, int32_t n, int32_t K, int32_t iters, int32_t restarts, uint64_t seed,
                     int32_t *out)
{
    double *C = (double *)malloc(sizeof(double) * 2 * (size_t)K);
    double *d2 = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *acc = (double *)malloc(sizeof(double) * 3 * (size_t)K);
    if (!C || !d2 || !lab || !acc || K < 1 || n < K) {
        free(C);
        free(d2);
        free(lab);
        free(acc);
        return -1.0;
    }
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double best = INFINITY;
    for (int32_t r = 0; r < restarts; ++r) {
        uint32_t draw = 0;
        /* k-means++: first centre uniform, then proportional to squared distance */
        for (int32_t c = 0; c < K; ++c) {
            uint32_t ctr[4] = {draw++, 0u, 0xFFFFFFFCu, (uint32_t)r}, w[4];
            oracle_philox4x32_10(ctr, key, w);
            double u = ((double)w[0] + 4294967296.0 * (double)(w[1] >> 11)) / (4294967296.0 * 2097152.0);
            int32_t pick = 0;
            if (c == 0) {
                pick = (int32_t)(u * (double)n);
                if (pick >= n)
                    pick = n - 1;
            } else {
                double tot = 0.0;
                for (int32_t v = 0; v < n; ++v)
                    tot += d2[v];
                double target = u * tot, run = 0.0;
                pick = n - 1;
                for (int32_t v = 0; v < n; ++v) {
                    run += d2[v];
                    if (run > target) {
                        pick = v;
                        break;
                    }
                }
            }
            C[2 * c] = Y[2 * (int64_t)pick];
            C[2 * c + 1] = Y[2 * (int64_t)pick + 1];
            for (int32_t v = 0; v < n; ++v) {
                double dx = Y[2 * (int64_t)v] - C[2 * c], dy = Y[2 * (int64_t)v + 1] - C[2 * c + 1];
                double dd = dx * dx + dy * dy;
                if (c == 0 || dd < d2[v])
                    d2[v] = dd;
            }
        }
        double inertia = 0.0;
        for (int32_t it = 0; it <= iters; ++it) {
            inertia = 0.0;
            int changed = 0;
            for (int32_t v = 0; v < n; ++v) {
                int32_t bc = 0;
                double bd = INFINITY;
                for (int32_t c = 0; c < K; ++c) {
                    double dx = Y[2 * (int64_t)v] - C[2 * c], dy = Y[2 * (int64_t)v + 1] - C[2 * c + 1];
                    double dd = dx * dx + dy * dy;
                    if (dd < bd) {
                        bd = dd;
                        bc = c;
                    }
                }
                if (it == 0 || lab[v] != bc)
                    changed = 1;
                lab[v] = bc;
                inertia += bd;
            }
            if (!changed || it == iters)
                break;
            for (int32_t c = 0; c < 3 * K; ++c)
                acc[c] = 0.0;
            for (int32_t v = 0; v < n; ++v) {
                acc[3 * lab[v]] += Y[2 * (int64_t)v];
                acc[3 * lab[v] + 1] += Y[2 * (int64_t)v + 1];
                acc[3 * lab[v] + 2] += 1.0;
            }
            for (int32_t c = 0; c < K; ++c)
                if (acc[3 * c + 2] > 0.0) {
                    C[2 * c] = acc[3 * c] / acc[3 * c + 2];
                    C[2 * c + 1] = acc[3 * c + 1] / acc[3 * c + 2];
                }
        }
        if (inertia < best) {
            best = inertia;
            memcpy(out, lab, sizeof(int32_t) * (size_t)n);
        }
    }
    free(C);
    free(d2);
    free(lab);
    free(acc);
    return best;
}
