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
    kCrossGraph = 16u,    // an edge joins two graphs of a batch
    kBadRowPtr = 32u,     // row_ptr decreases or leaves [0, nnz]
};

// t-FDP constants (Section 3.1: alpha = 0.1, beta = 8, gamma = 2).
constexpr float kAlpha = 0.1f;
constexpr float kBeta = 8.0f;

// Fixed-point scale of the synchronous accumulator: value * 2^32 as int64.
constexpr float kFixScale = 4294967296.0f;
constexpr float kFixInv = 2.3283064365386963e-10f;   // 2^-32
constexpr float kFixClamp = 1048576.0f;              // |term| <= 2^20 before scaling

// One graph of a batch: its vertices are [node_base, node_base + n), its
// directed edges [edge_base, edge_base + 2|E_g|) of the batch CSR.  Random
// words use the graph-local edge index and the graph's own seed, and the
// graph runs epoch (tick - start_tick) of its own schedule, so its layout
// draws exactly the numbers it would draw alone.  A graph is active while
// 0 <= tick - start_tick < total_epochs.
struct GraphInfo {
    int32_t node_base;
    int32_t n;
    int64_t edge_base;
    uint64_t seed;
    int32_t start_tick;
    int32_t total_epochs;
    double eta0;
    double eta_min;
    int32_t kind;      // schedule kind (0: linear decay, 1: constant)
    int32_t pad;
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
    const int32_t *node_graph;   // batch only
    const GraphInfo *graphs;
    const uint2 *alias;          // weighted negatives: n entries {threshold, alias (graph-local)}; else null
    double *energy;              // actual energy of the epoch is added here (null: not computed)
};

// Oriented bundle list: entry {j, CSR index of (i, j), CSR index of (j, i),
// i} (indices as unsigned 32-bit) for each partner j ranked below i,
// row-major (rows in vertex order, a row's entries in affine or ascending
// partner order).  The
// list is cut into chunks of T consecutive entries (a chunk may cross row
// boundaries; the last one may be short); chunk c goes to slot
// (mul * c + add) mod S, S = ceil(nnz / T), so neighbouring slots hold
// unrelated parts of the graph.  The slots of a slot group (32 slots; the
// last group may have fewer, W) store their entries interleaved: entry t of
// slot s is at (s / 32) * 32 * T + t * W + s % 32, so a warp on one slot
// group reads W consecutive entries per step.  The array holds S * T entries.
struct ChunkLayout {
    int32_t T;     // entries per chunk
    int64_t S;     // chunks (slots)
    int64_t mul;   // slot of chunk c: (mul * c + add) mod S, gcd(mul, S) = 1
    int64_t add;
    int32_t order = 0;   // entries within a row: 0 affine order of their partners, 1 ascending partner id
};

__host__ __device__ inline int64_t chunk_slot(const ChunkLayout &L, int64_t c) {
    return (int64_t)(((uint64_t)L.mul * (uint64_t)c + (uint64_t)L.add) % (uint64_t)L.S);
}

// Slots in the group of `slot` (32 except in the last group).
__host__ __device__ inline int64_t chunk_group_width(int64_t slot, int64_t S) {
    const int64_t rest = S - ((slot >> 5) << 5);
    return rest < 32 ? rest : 32;
}

__host__ __device__ inline int64_t chunk_entry_index(int64_t slot, int64_t S, int32_t T, int64_t t) {
    return (slot >> 5) * 32 * (int64_t)T + t * chunk_group_width(slot, S) + (slot & 31);
}

struct OrientedArgs {
    const int64_t *row_ptr;   // n + 1 row offsets of the oriented list (row-major positions)
    const int4 *ent;          // entries {j, index of (i, j), index of (j, i), i}, stored slot-interleaved
    const int2 *meta;         // per slot: {row of the chunk's first entry, chunk id}
    float2 *pos;
    int64_t num_segs;         // slots S
    int64_t nnz;              // entries of the list
    int32_t seg_len;          // entries per chunk T
    int32_t n;
    int64_t perm_mul;         // order of the 32-slot groups this epoch: (perm_mul * g + perm_add) mod groups
    int64_t perm_add;
    int32_t k;
    uint32_t epoch;           // single graph: the epoch; batch: the tick
    uint64_t seed;
    float eta;
    uint32_t *status;
    const int32_t *node_graph;   // batch only: graph of every vertex
    const GraphInfo *graphs;     // batch only
    float inflight_share;        // lanes in flight / slots (share of the chunks running at once)
    const uint2 *alias;          // weighted negatives (alias table, graph-local ids); null: uniform
    double *energy;              // actual energy of the epoch is added here (null: not computed)
    const int32_t *pieces;       // chunks each vertex's oriented row spans (HOGWILD_RED's write-back)
};

// Dispatches on a.alias (weighted negatives, epoch_weighted.cu) and a.energy
// (actual energy, epoch_energy.cu; single graphs only).
cudaError_t launch_oriented_epoch(const OrientedArgs &a, int red_mode, int grid, int block, cudaStream_t s);
cudaError_t launch_oriented_weighted(const OrientedArgs &a, int red_mode, int grid, int block, cudaStream_t s);
cudaError_t launch_oriented_energy(const OrientedArgs &a, int red_mode, int grid, int block, cudaStream_t s);
int oriented_weighted_blocks_per_sm(int red_mode, int k, int block, int multi);
int oriented_energy_blocks_per_sm(int red_mode, int k, int block, int weighted);


// One job of a multi-handle epoch: a single-graph HOGWILD handle's device
// arrays, its positions, and the epoch, step and seed it runs this launch.
struct JobDesc {
    const int64_t *row_ptr;
    const int4 *ent;
    const int2 *meta;
    float2 *pos;
    int64_t num_segs;
    int64_t seg_prefix;     // slots of the jobs before this one
    int64_t nnz;
    uint64_t seed;
    int32_t n;
    uint32_t epoch;
    float eta;
    int32_t seg_len;
    const uint2 *alias;     // the job's alias table, or null (uniform)
    const int32_t *pieces;  // the job's per-vertex piece counts (OrientedArgs::pieces)
};

struct MultiArgs {
    const JobDesc *jobs;
    int32_t num_jobs;
    int32_t k;
    int64_t total_segs;
    int64_t perm_mul;         // order of the 32-slot groups, as OrientedArgs
    int64_t perm_add;
    uint32_t *status;
    float inflight_share;
};

// weighted: some job of the launch draws weighted negatives.
cudaError_t launch_multi_epoch(const MultiArgs &a, int red_mode, int weighted, int grid, int block,
                               cudaStream_t s);
int multi_blocks_per_sm(int red_mode, int weighted, int k, int block);
cudaError_t launch_multi_weighted(const MultiArgs &a, int red_mode, int grid, int block, cudaStream_t s);
int multi_weighted_blocks_per_sm(int red_mode, int k, int block);
int oriented_blocks_per_sm(int red_mode, int k, int block, int multi, int weighted);
cudaError_t launch_sync_chunk(const SyncArgs &a, int grid, int block, cudaStream_t s);
// y += eta * D * 2^-32 (clipped to `limit` when > 0), D = 0.  For a batch
// (graphs != nullptr) eta and the clip come from each vertex's graph at
// `tick`, with limit = cap * eta_t / eta0 when cap > 0.
cudaError_t launch_sync_apply(float2 *pos, long long *disp, int32_t n, float eta, float limit,
                              uint32_t *status, int grid, int block, cudaStream_t s,
                              const int32_t *node_graph = nullptr, const GraphInfo *graphs = nullptr,
                              int32_t tick = 0, float cap = 0.0f);
int sync_blocks_per_sm(int block);

cudaError_t launch_degrees(const int64_t *row_ptr, int32_t n, int32_t *deg, cudaStream_t s);
cudaError_t launch_segment_rows(const int64_t *row_ptr, int32_t n, int64_t nnz, int32_t seg_len,
                                int32_t *seg_row, int64_t num_segs, cudaStream_t s);
cudaError_t launch_validate_csr(const int64_t *row_ptr, const int32_t *col_idx, const int32_t *seg_row,
                                int32_t n, int64_t nnz, int32_t seg_len, uint32_t *flags, cudaStream_t s,
                                const int32_t *node_graph, unsigned long long *upper_count, const int32_t *deg,
                                int32_t *orient);
// Construction of the oriented bundle list: the flags come from the
// validation pass (launch_validate_csr's orient), then exclusive scan,
// scatter into the chunked layout, offsets.
cudaError_t exclusive_scan_i32(void *temp, size_t *temp_bytes, const int32_t *in, int32_t *out, int64_t count,
                               cudaStream_t s);
cudaError_t launch_orient_scatter(const int64_t *row_ptr, const int32_t *col_idx, const int32_t *seg_row,
                                  const int32_t *deg, int64_t nnz, int32_t seg_len, const int32_t *pos,
                                  const ChunkLayout &to, int4 *ent, int2 *meta, int64_t capacity, uint32_t *flags,
                                  cudaStream_t s);
// pieces[v] = chunks of T entries that v's oriented row spans.
cudaError_t launch_row_pieces(const int64_t *act_rp, int32_t n, int32_t T, int32_t *pieces, cudaStream_t s);
cudaError_t launch_orient_rowptr(const int64_t *row_ptr, const int32_t *pos, int32_t n, int64_t *act_row_ptr,
                                 cudaStream_t s);
// Moves the oriented entries from layout `from` (T == 0: plain row-major) to
// layout `to` and writes `to`'s slot table.
cudaError_t launch_chunk_layout(const int4 *src, const ChunkLayout &from, int4 *dst, const ChunkLayout &to,
                                int2 *meta, const int64_t *act_rp, int32_t n, int64_t nnz, cudaStream_t s);
// Objective partial sums (FP64), one per block, summed on the host in order.
cudaError_t launch_objective_edges(const int64_t *row_ptr, const int32_t *col_idx, const int32_t *seg_row,
                                   const float2 *pos, int64_t nnz, int32_t seg_len, double *partial, int grid,
                                   cudaStream_t s);
cudaError_t launch_objective_oriented(const int64_t *row_ptr, const int4 *ent, const int2 *meta,
                                      const ChunkLayout &L, int64_t nnz, const float2 *pos, double *partial,
                                      int grid, cudaStream_t s);
// Pair sums of the objective; wt (nullable) holds the per-vertex factors of
// a weighted sampler ({x, y, z}: d_i P(j|i) = x_i z_j + y_i).
// Exact: sum over ordered pairs i != j of coef_ij U^r, coef = d_i + d_j or c_ij.
cudaError_t launch_objective_pairs_exact(const float2 *pos, const int32_t *deg, const float4 *wt, int32_t n,
                                         double *partial, int grid, cudaStream_t s);
// Batch: sum over graphs and ordered pairs of the graph of w_ij U^r, w_ij =
// (d_i + d_j) / (2 (n_g - 1)) or c_ij / 2; the host applies k / 2.
cudaError_t launch_objective_pairs_batch(const float2 *pos, const int32_t *deg, const float4 *wt,
                                         const int32_t *node_graph, const GraphInfo *graphs, int32_t n,
                                         double *partial, int grid, cudaStream_t s);
// Neighbourhood preservation (Section 4.1, r = 2) of `count` sampled
// vertices: out[q] = the Jaccard index of the 2-hop set and the nearest set
// of nodes[q], or -1 for a vertex without neighbours.  Every graph (all of
// [0, n) when graphs is null) has at most max_graph vertices.  Graphs of up
// to kNpMaxGraph vertices keep the 2-hop bitmap in shared memory; larger
// ones pass gbits, np_scratch_words(gbits_words, grid) words of global
// scratch: a bitmap row of gbits_words words per block, then per block a
// list of kNpCandidates keys (8 bytes) and ids (4 bytes).
constexpr int32_t kNpMaxGraph = 1 << 18;
constexpr int64_t kNpCandidates = 1 << 16;
inline int64_t np_scratch_words(int64_t gbits_words, int64_t grid) {
    return ((grid * gbits_words + 1) & ~(int64_t)1) + grid * kNpCandidates * 3;
}
cudaError_t launch_np_samples(const int64_t *row_ptr, const int32_t *col_idx, const float2 *pos, const int32_t *nodes,
                              int32_t count, const int32_t *node_graph, const GraphInfo *graphs, int32_t n,
                              int32_t max_graph, double *out, int grid, uint32_t *gbits, int64_t gbits_words,
                              cudaStream_t s);
cudaError_t launch_objective_pairs_sampled(const float2 *pos, const int32_t *deg, const float4 *wt, int32_t n,
                                           int64_t pairs, uint64_t seed, double *partial, int grid,
                                           cudaStream_t s);

}  // namespace snap
