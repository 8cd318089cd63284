// snap_internal.h -- launchers shared by the translation units of the library.
// Not part of the public ABI (that is include/snap_layout.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace snap {

// Bits of the device status word.
enum : uint32_t {
    kStatusNonFinite = 1u,   // a force or position became NaN/Inf
    kStatusClamped = 2u,     // a fixed-point term was clamped
};

// Bits of the validation word written by launch_validate_csr.
enum : uint32_t {
    kBadColumn = 1u,      // column outside [0, n)
    kSelfLoop = 2u,       // j == i
    kUnsorted = 4u,       // row not strictly ascending (duplicate or unsorted)
    kAsymmetric = 8u,     // (i, j) present but (j, i) missing
};

// t-FDP constants (Section 3.1: alpha = 0.1, beta = 8, gamma = 2).
constexpr float kAlpha = 0.1f;
constexpr float kBeta = 8.0f;

// Fixed-point scale of the synchronous accumulator: value * 2^32 as int64.
constexpr float kFixScale = 4294967296.0f;
constexpr float kFixInv = 2.3283064365386963e-10f;   // 2^-32
constexpr float kFixClamp = 1048576.0f;              // |term| <= 2^20 before scaling

struct EpochArgs {
    const int64_t *row_ptr;   // n + 1
    const int32_t *col_idx;   // nnz (+ padding to a multiple of seg_len + 4)
    const int32_t *seg_row;   // row containing edge seg * seg_len, per segment
    float2 *pos;              // n
    int64_t nnz;
    int32_t n;
    int32_t k;
    int32_t seg_len;
    uint32_t epoch;
    uint64_t seed;
    float eta;
    uint32_t *status;
};

struct SyncArgs {
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const int32_t *seg_row;
    const float2 *pos;
    long long *disp;          // n x 2 int64 fixed point
    int64_t e_begin, e_end;   // edge range of this chunk
    int32_t n;
    int32_t k;
    int32_t seg_len;
    uint32_t epoch;
    uint64_t seed;
    uint32_t *status;
};

cudaError_t launch_hogwild_epoch(const EpochArgs &a, int red_mode, int grid, int block, cudaStream_t s);
cudaError_t launch_sync_chunk(const SyncArgs &a, int grid, int block, cudaStream_t s);
cudaError_t launch_sync_apply(float2 *pos, long long *disp, int32_t n, float eta, float limit,
                              uint32_t *status, int grid, int block, cudaStream_t s);
int hogwild_blocks_per_sm(int red_mode, int block);
int sync_blocks_per_sm(int block);

cudaError_t launch_segment_rows(const int64_t *row_ptr, int32_t n, int64_t nnz, int32_t seg_len,
                                int32_t *seg_row, int64_t num_segs, cudaStream_t s);
cudaError_t launch_validate_csr(const int64_t *row_ptr, const int32_t *col_idx, const int32_t *seg_row,
                                int32_t n, int64_t nnz, int32_t seg_len, uint32_t *flags,
                                cudaStream_t s);
// Objective partial sums (FP64), one per block, summed on the host in order.
cudaError_t launch_objective_edges(const int64_t *row_ptr, const int32_t *col_idx, const int32_t *seg_row,
                                   const float2 *pos, int64_t nnz, int32_t n, int32_t seg_len,
                                   double *partial, int grid, cudaStream_t s);
cudaError_t launch_objective_pairs_exact(const float2 *pos, const int32_t *deg, int32_t n,
                                         double *partial, int grid, cudaStream_t s);
cudaError_t launch_objective_pairs_sampled(const float2 *pos, const int32_t *deg, int32_t n,
                                           int64_t pairs, uint64_t seed, double *partial, int grid,
                                           cudaStream_t s);

}  // namespace snap
