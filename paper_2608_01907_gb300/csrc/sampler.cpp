// sampler.cpp -- host construction of the weighted-negative tables.
//
// The paper draws negatives uniformly (Algorithm 1) and names non-uniform
// negatives as future work (Section 6).  The library offers two weighted
// samplers: DEGREE (a node is drawn in proportion to its degree) and WEIGHTS
// (in proportion to a caller's non-negative weight).  Both use Walker's alias
// method; the table is built here, exactly, in integer arithmetic, so that it
// is the same on every machine:
//
//   * integer weights q: DEGREE uses the degrees; WEIGHTS quantises
//     q_s = llround(w_s / max w * 2^32) in IEEE double;
//   * Vose's construction in units where a column holds Q = sum q and node s
//     brings n * q_s; the small nodes (n q_s < Q) are served first-in
//     first-out in increasing id, the large ones from a stack filled in
//     increasing id (the top one keeps donating until it falls below Q, then
//     joins the back of the small queue);
//   * a column shared with its alias keeps col with threshold
//     floor(mass * 2^32 / Q); a full column has threshold 0xFFFFFFFF and
//     itself as alias.
//
// The device draws (snap_device.cuh, weighted_negative) take two words per
// attempt, reject the source, and fall back to the uniform rule after 16
// rejections.  The objective those draws descend generalises Section 3.3:
// c_ij = d_i P(j|i) + d_j P(i|j), with
// P(s|i) = (1 - rho_i^16) q_s / (Q - q_i) + rho_i^16 / (n - 1), rho_i = q_i / Q.
#include <cmath>
#include <cstdint>
#include <vector>

#include "snap_sampler.h"

namespace snap {

int sampler_weights(int32_t kind, const int64_t *row_ptr, const float *node_weights, int32_t v0, int32_t v1,
                    uint64_t *q) {
    const int32_t n = v1 - v0;
    if (kind == 1) {   // DEGREE
        uint64_t total = 0;
        for (int32_t s = 0; s < n; ++s) {
            q[s] = (uint64_t)(row_ptr[v0 + s + 1] - row_ptr[v0 + s]);
            total += q[s];
        }
        return total > 0 ? 0 : 2;
    }
    double top = 0.0;
    for (int32_t s = 0; s < n; ++s) {
        const double w = (double)node_weights[v0 + s];
        if (!(w >= 0.0) || std::isinf(w)) return 1;
        top = w > top ? w : top;
    }
    if (!(top > 0.0)) return 2;
    for (int32_t s = 0; s < n; ++s) q[s] = (uint64_t)std::llround((double)node_weights[v0 + s] / top * 4294967296.0);
    return 0;
}

void alias_table(const uint64_t *q, int32_t n, uint32_t *threshold, int32_t *alias) {
    unsigned __int128 total = 0;
    for (int32_t s = 0; s < n; ++s) total += q[s];
    const uint64_t Q = (uint64_t)total;
    std::vector<uint64_t> left((size_t)n);
    std::vector<int32_t> queue;   // small nodes, served from the front
    std::vector<int32_t> stack;   // large nodes, served from the top
    queue.reserve((size_t)n);
    stack.reserve((size_t)n);
    for (int32_t s = 0; s < n; ++s) {
        left[(size_t)s] = (uint64_t)n * q[s];
        threshold[s] = 0xFFFFFFFFu;
        alias[s] = s;
        (left[(size_t)s] < Q ? queue : stack).push_back(s);
    }
    size_t front = 0;
    while (front < queue.size() && !stack.empty()) {
        const int32_t small = queue[front++];
        const int32_t donor = stack.back();
        const uint64_t kept = left[(size_t)small];
        threshold[small] = (uint32_t)(((unsigned __int128)kept << 32) / Q);
        alias[small] = donor;
        left[(size_t)donor] -= Q - kept;
        if (left[(size_t)donor] < Q) {
            stack.pop_back();
            queue.push_back(donor);
        }
    }
}

void sampler_objective_factors(const int64_t *row_ptr, const uint64_t *q, int32_t v0, int32_t v1, float4 *out) {
    const int32_t n = v1 - v0;
    unsigned __int128 total = 0;
    for (int32_t s = 0; s < n; ++s) total += q[s];
    const double Q = (double)(uint64_t)total;
    for (int32_t s = 0; s < n; ++s) {
        const double d = (double)(row_ptr[v0 + s + 1] - row_ptr[v0 + s]);
        const double rho = (double)q[s] / Q;
        double r16 = rho * rho;
        r16 *= r16;
        r16 *= r16;
        r16 *= r16;
        const uint64_t rest = (uint64_t)total - q[s];
        // P(j|s) = scale_s * (q_j / Q) + floor_s
        const double scale = rest > 0 ? (1.0 - r16) * Q / (double)rest : 0.0;
        const double floor_p = n > 1 ? r16 / (double)(n - 1) : 0.0;
        out[s] = make_float4((float)(d * scale), (float)(d * floor_p), (float)((double)q[s] / Q), 0.0f);
    }
}

}  // namespace snap
