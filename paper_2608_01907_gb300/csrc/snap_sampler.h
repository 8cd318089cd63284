// snap_sampler.h -- host construction of the weighted-negative tables
// (sampler.cpp).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace snap {

// Integer weights of vertices [v0, v1): kind 1 = degree (row lengths of
// row_ptr), kind 2 = llround(w / max w * 2^32) of node_weights.  Returns 0,
// 1 (a weight is negative, NaN or infinite) or 2 (all weights are zero).
int sampler_weights(int32_t kind, const int64_t *row_ptr, const float *node_weights, int32_t v0, int32_t v1,
                    uint64_t *q);

// Alias table of n integer weights (sum > 0, n * max q < 2^64): thresholds
// and graph-local aliases.
void alias_table(const uint64_t *q, int32_t n, uint32_t *threshold, int32_t *alias);

// Per-vertex factors of the pair coefficient of the weighted objective:
// d_i P(j|i) = x_i * z_j + y_i with out[i] = {x_i, y_i, z_i, 0}.
void sampler_objective_factors(const int64_t *row_ptr, const uint64_t *q, int32_t v0, int32_t v1, float4 *out);

}  // namespace snap
