/*
 * snap_layout.h -- C ABI of the GB300 (sm_103a) SNAP-tFDP layout library.
 *
 * SNAP-tFDP ("Massively Scalable Graph Layouts via Sparse Negative Sampling")
 * lays out an undirected graph G = (V, E) in 2D (Section 3.1).  One epoch
 * visits every directed edge (i, j) -- each undirected edge stored both ways,
 * Section 3.3 -- applies the bounded t-distribution attraction of Table 1 to
 * both endpoints, draws k negatives s uniformly from V \ {i} and applies the
 * short-range t-distribution repulsion to i and s (Algorithm 1).  In
 * expectation this descends the degree-weighted t-FDP energy of Eq. 4 with the
 * linear weight (d_i + d_j) / (2(|V|-1)) (Section 3.3, Eq. 5).
 *
 * Conventions shared by every entry point
 *   - All functions are plain C, thread-compatible (one handle must not be
 *     used from two host threads at once), and return snap_status.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the current device.  The library never takes ownership
 *     of a caller's buffer.
 *   - Positions are n x 2 float32, interleaved (x0, y0, x1, y1, ...), 8-byte
 *     aligned, owned by the caller.
 *   - cuda_stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; only the calls documented as
 *     synchronising wait for it.
 *   - On any non-OK status nothing is written to the caller's outputs, the
 *     handle stays valid and snap_last_error() describes the failure.
 *   - Faults detected inside kernels (non-finite force, fixed-point clamp) are
 *     recorded in a device status word and reported by the next call on the
 *     handle that observes them, or by snap_layout_check(), which waits.
 */
#ifndef SNAP_LAYOUT_H
#define SNAP_LAYOUT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SNAP_LAYOUT_ABI_VERSION 1

typedef struct snap_layout snap_layout;
typedef snap_layout *snap_layout_t;

typedef enum {
    SNAP_OK = 0,
    SNAP_ERR_INVALID_ARG = 1,    /* malformed CSR, bad size, null pointer, misaligned buffer */
    SNAP_ERR_OUT_OF_MEMORY = 2,  /* a device or host allocation failed; nothing leaked */
    SNAP_ERR_CUDA = 3,           /* a CUDA runtime call or launch failed */
    SNAP_ERR_TIMEOUT = 4,        /* reserved: no kernel of this library waits on a flag */
    SNAP_ERR_NOT_SUPPORTED = 5,  /* the option or call is not supported for this handle */
    SNAP_ERR_NUMERIC = 6         /* a kernel met a non-finite or out-of-range value */
} snap_status;

/* Parallel update semantics of an epoch. */
typedef enum {
    /* Lock-free updates in the spirit of HOGWILD! (Section 3.4).  Each
     * undirected edge {i, j} is placed in the bundle (row) of its
     * higher-ranked endpoint (larger degree, then smaller id); rows are cut
     * into chunks of segment_edges entries that lanes take in an order
     * reshuffled every epoch; a lane keeps the current row's source in
     * registers and applies both directed steps (i, j) and (j, i) of every
     * entry, each with its own negatives.  Partners are written back with
     * racy writes (64-bit exchanges): concurrent writers may overwrite each
     * other (the paper's description of its lock-free scheme). */
    SNAP_MODE_HOGWILD = 0,
    /* As HOGWILD, but every partner update is an atomic float add of the
     * change computed from a racy read (HOGWILD!'s component-wise atomic
     * updates: no lost updates, no locks); a row cut into L chunks merges the
     * chunks' source displacements by the expected number running together.
     * The default: faster than HOGWILD on GB300 (L2 handles atomic adds to
     * random addresses better than dependent plain stores) and closer to the
     * sequential algorithm on large graphs. */
    SNAP_MODE_HOGWILD_RED = 1,
    /* Deterministic synchronous mode: positions are frozen within each of S
     * row chunks, every force is quantised to int64 fixed point (2^-32) and
     * summed with integer atomics, then y += eta_t * D.  Bitwise reproducible
     * for a given input, independent of scheduling. */
    SNAP_MODE_SYNC = 2
} snap_mode;

/* Negative-sample distribution.  UNIFORM is the paper's (Algorithm 1: s
 * uniform over V \ {i}; the degree weighting of Eq. 4 then arises implicitly,
 * Section 3.3).  DEGREE and WEIGHTS draw s in proportion to its degree or to
 * a caller weight -- the non-uniform negatives the paper leaves to future
 * work (Section 6) -- through an alias table (snap_sampler_table): two
 * random words per attempt, an attempt yielding s = i rejected, the uniform
 * rule after 16 rejections.  The objective then uses the pair weight
 * w_ij = (d_i P(j|i) + d_j P(i|j)) / 2 with the sampler's P(s|i). */
typedef enum {
    SNAP_SAMPLER_UNIFORM = 0,
    SNAP_SAMPLER_DEGREE = 1,
    SNAP_SAMPLER_WEIGHTS = 2
} snap_sampler;

/* Step-size schedule.  The paper decays eta over epochs and updates it once
 * per epoch (Section 3.3, Algorithm 1) without stating the form; this library
 * uses  kind 0: eta_t = max(eta0 * (1 - t / total_epochs), eta_min)
 *       kind 1: eta_t = eta0 (constant).
 * t is the global epoch index, so a layout split over several calls (resume)
 * sees the same schedule as one call. */
typedef struct {
    int32_t kind;
    int32_t total_epochs;
    double eta0;
    double eta_min;
} snap_schedule;

typedef struct {
    int32_t mode;             /* snap_mode */
    int32_t sampler;          /* snap_sampler */
    const float *node_weights;/* host, n floats >= 0 (read during create only); SNAP_SAMPLER_WEIGHTS */
    int32_t sync_substeps;    /* S >= 1 row chunks per epoch in SNAP_MODE_SYNC */
    float sync_cap;           /* > 0: clip each node's sync step to cap*eta_t/eta0 */
    int32_t segment_edges;    /* work per lane segment, a multiple of 4 in [4, 4096]: in the HOGWILD
                                 modes the length of a chunk of the oriented list (entries of 2
                                 directed edges each; a chunk may span rows, and a graph with at most
                                 this many entries is one chunk, so one lane); in SYNC directed
                                 edges; 0 = default (HOGWILD: 4; SYNC: 16) */
    int32_t block_threads;    /* threads per block; 0 = default (256) */
    int32_t flags;            /* SNAP_FLAG_* bits */
    float max_inflight;       /* HOGWILD modes: at most this share of the graph's entries in flight at
                                 once (lanes = share x entries); 0 = default (0.005).  Concurrent
                                 updates of one vertex degrade Hogwild quality on small graphs */
} snap_options;

/* snap_options.flags: capture the launches of a snap_layout_epochs call with
 * epochs > 1 into a CUDA graph on first use and replay it on later calls
 * with the same positions pointer, epoch range, k, schedule and seed (up to 4
 * graphs are cached per handle). */
#define SNAP_FLAG_CUDA_GRAPH 1
/* snap_options.flags: a HOGWILD handle keeps its device CSR after building
 * the oriented list (SYNC handles always keep it), for
 * snap_layout_neighborhood_preservation and the NP half of the autotuner's
 * gate; snap_layout_device_bytes counts it. */
#define SNAP_FLAG_KEEP_CSR 2
/* snap_options.flags: store each oriented row's entries in ascending partner
 * id instead of the default affine order (which keeps entries of nearby
 * partners apart, Section 3.4's shuffle; the ascending order gathers
 * neighbouring partners back to back).  The autotuner may switch it. */
#define SNAP_FLAG_ASCENDING_ROWS 4

/* Fill *opts with the defaults (HOGWILD_RED, UNIFORM, S = 1, no cap). */
void snap_options_default(snap_options *opts);

/*
 * snap_layout_create -- validate a graph and make it resident on the device.
 *
 * Paper: the method needs only the directed edge list and the positions
 * (Section 3.3: nothing but the edges and the positions); the edge list is a CSR
 * here, each undirected edge stored as (i, j) and (j, i).
 *
 *   row_ptr   host, n+1 int64; row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz < 2^32
 *             (directed edges: up to 2^31 - 1 undirected edges).
 *   col_idx   host, nnz int32; each row strictly ascending, 0 <= j < n, j != i,
 *             and symmetric: j in row i  <=>  i in row j.
 *   degrees   host, n int32, or NULL.  If given it must equal the row lengths.
 *   n         number of vertices, 1 <= n < 2^31 - 1.
 *   opts      NULL for defaults.
 *   out       receives the handle; untouched on error.
 *
 * Copies the CSR to the device (the host arrays may be freed on return),
 * checks it there and, in the HOGWILD modes, builds the oriented list (each
 * undirected edge in the row of its higher-ranked endpoint, a row's entries
 * in a fixed affine order of their partners, cut into chunks of
 * segment_edges entries stored in a pseudo-random slot order) and frees the
 * CSR; for a weighted sampler it also builds the alias table.  Synchronises
 * the stream.  Errors: INVALID_ARG (malformed input, with the first
 * violation in snap_last_error), OUT_OF_MEMORY, CUDA.
 */
snap_status snap_layout_create(const int64_t *row_ptr, const int32_t *col_idx,
                               const int32_t *degrees, int32_t n,
                               const snap_options *opts, void *cuda_stream,
                               snap_layout_t *out);

/*
 * snap_layout_create_batch -- many graphs laid out together, in the same
 * launches (the paper lays out one graph at a time; batching is a
 * deployment form of the same method).
 *
 *   row_ptr, col_idx, n  host, the disjoint union of the graphs as one CSR
 *                        with the contract of snap_layout_create; graph g owns
 *                        vertices [graph_offsets[g], graph_offsets[g+1]) and
 *                        no edge may join two graphs (INVALID_ARG).
 *   graph_offsets        host, num_graphs + 1 int32, strictly increasing,
 *                        from 0 to n.
 *
 * On the returned handle snap_layout_epochs lays out every graph at once with
 * the call's schedule and seed; each graph draws its negatives from its own
 * vertices, and its random words use its own edge indices (offset from the
 * graph's first edge), so every graph draws exactly the numbers it would draw
 * in a handle of its own: in SNAP_MODE_SYNC with sync_substeps = 1 the result
 * equals the one-graph layouts bit for bit.  snap_layout_objective returns
 * the sum over graphs of their objectives (exact = 1 only).
 */
snap_status snap_layout_create_batch(const int64_t *row_ptr, const int32_t *col_idx, int32_t n,
                                     const int32_t *graph_offsets, int32_t num_graphs,
                                     const snap_options *opts, void *cuda_stream, snap_layout_t *out);

/*
 * snap_layout_epochs -- run epochs [epoch_begin, epoch_begin + epochs) of
 * Algorithm 1 on device positions, with the handle's mode.
 *
 *   positions    device, n x 2 float32, updated in place.
 *   neg_samples  k >= 0 (the paper's default is k = 3, Section 4.2); k <= 64.
 *   schedule     host struct, read during the call.
 *   seed         keys the counter-based Philox4x32-10 stream: word w of edge
 *                e in epoch t is component w mod 4 of
 *                Philox(ctr = (e_lo, e_hi, t, w div 4), key = (seed_lo, seed_hi)).
 *                The negatives of edge e = (i, j) consume its words in
 *                order; a uniform negative takes one word:
 *                u = floor(word * (n-1) / 2^32), s = u + (u >= i) (weighted
 *                samplers: see snap_sampler).
 *
 * Asynchronous: enqueues one kernel per epoch (HOGWILD modes) or 2 per chunk
 * (SYNC) and returns.  Errors: INVALID_ARG, CUDA, NUMERIC (from an earlier
 * call, observed without waiting).
 */
snap_status snap_layout_epochs(snap_layout_t h, float *positions, int32_t epoch_begin,
                               int32_t epochs, int32_t neg_samples,
                               const snap_schedule *schedule, uint64_t seed,
                               void *cuda_stream);

/*
 * snap_layout_sync_chunks -- run chunks [chunk_begin, chunk_end) of epoch
 * `epoch` of the synchronous mode (SNAP_MODE_SYNC handles only).
 *
 * Paper: none directly.  The synchronous mode is this library's
 * deterministic variant of Algorithm 1 (Section 3.3's update with positions
 * frozen within a chunk of rows); an epoch is sync_substeps chunk steps, each
 * summing the forces of its rows' edges and negatives from the positions at
 * the chunk's start and then applying eta_epoch times that sum (clipped to
 * sync_cap * eta_epoch / eta0 per vertex when sync_cap > 0).
 *
 *   positions    device, n x 2 float32, updated in place.
 *   epoch        the epoch index t (selects the step size and the random words).
 *   chunk_begin, chunk_end   0 <= chunk_begin <= chunk_end <= sync_substeps.
 *   neg_samples, schedule, seed   as for snap_layout_epochs.
 *
 * Calling it for chunks [0, c) and then [c, sync_substeps) gives bit for bit
 * the positions of one snap_layout_epochs call for that epoch, so an epoch
 * can be split at any chunk boundary (to interleave other work, or to look at
 * the positions between chunks).  Asynchronous, like snap_layout_epochs.
 * Errors: INVALID_ARG (not a SYNC handle, range outside [0, sync_substeps],
 * bad schedule or k), CUDA, NUMERIC (from an earlier call).
 */
snap_status snap_layout_sync_chunks(snap_layout_t h, float *positions, int32_t epoch,
                                    int32_t chunk_begin, int32_t chunk_end, int32_t neg_samples,
                                    const snap_schedule *schedule, uint64_t seed, void *cuda_stream);

/*
 * snap_layout_epochs_energy -- snap_layout_epochs that also reports the
 * actual energy of every epoch (Section 3.3, compared there with the
 * effective energy of Eq. 4 evaluated after each epoch): half the sum, over
 * the directed steps of the epoch, of U^a of the step's pair and U^r of each
 * drawn pair, each evaluated on the positions the update used (frozen
 * positions in SNAP_MODE_SYNC).  Summed in FP64 per block from FP32 terms.
 *
 *   actual_energy  device, epochs doubles, 8-byte aligned; overwritten
 *                  asynchronously on the stream (entry e = epoch epoch_begin + e).
 * The call is never captured into a CUDA graph.  Other arguments, ordering
 * and errors as snap_layout_epochs; NOT_SUPPORTED for a batch handle.
 */
snap_status snap_layout_epochs_energy(snap_layout_t h, float *positions, int32_t epoch_begin, int32_t epochs,
                                      int32_t neg_samples, const snap_schedule *schedule, uint64_t seed,
                                      double *actual_energy, void *cuda_stream);

/*
 * snap_layout_objective -- the energy the method descends (Eq. 4 with the
 * weight realised by uniform sampling, Section 3.3):
 *   U = sum_{(i,j) in E, i<j} U^a(r_ij) + k * sum_{i<j} w_ij U^r(r_ij),
 *   w_ij = (d_i + d_j) / (2(n-1))   (DEGREE / WEIGHTS samplers: the w_ij of snap_sampler),
 *   U^a(r) = alpha (r^2/2 + (beta/2) ln(1+r^2)),  U^r(r) = 1 / (2(1+r^2))
 * (the energies whose negative gradients are the Table 1 forces, Eq. 2).
 *
 *   positions     device, n x 2 float32 (read only).
 *   exact         1: all n(n-1)/2 pairs; 0: pair_samples uniform unordered
 *                 pairs (Philox counter (p_lo, p_hi, 0xFFFFFFFD, 0), key seed;
 *                 i = floor(w0 n / 2^32), j from w1 as a negative of i) scaled
 *                 to an unbiased estimate.  The attraction sum is always exact.
 *   out_attr, out_rep, out_total   host doubles.
 *
 * Synchronises the stream.  Per-term arithmetic is FP32, sums are FP64.
 */
snap_status snap_layout_objective(snap_layout_t h, const float *positions, int32_t neg_samples,
                                  int32_t exact, int64_t pair_samples, uint64_t seed,
                                  double *out_attr, double *out_rep, double *out_total,
                                  void *cuda_stream);

/* Wait for the stream and report any fault recorded by earlier kernels of
 * this handle (then clear it).  Returns OK, NUMERIC or CUDA. */
snap_status snap_layout_check(snap_layout_t h, void *cuda_stream);

/* Device bytes held by the handle (CSR, tables, scratch; positions excluded). */
int64_t snap_layout_device_bytes(snap_layout_t h);

/*
 * snap_layout_autotune -- choose the chunk size (oriented entries per lane)
 * and the block size of a HOGWILD handle: the fastest configuration whose
 * layout quality stays within `tolerance` of the configuration the handle
 * has on entry.  The choice stays on the handle.
 *
 * Candidates: the entry configuration and 4, 8, 16, 32 entries x 128/256
 * threads x the two row orders (affine, ascending partner id;
 * SNAP_FLAG_ASCENDING_ROWS).  Longer chunks apply more of one source's steps back to back,
 * which is faster but moves the visiting order away from Algorithm 1's
 * shuffled order and can cost energy (Section 3.4's lock-free scheme
 * bounds concurrency, not order).
 *   1. Timing: each candidate runs the schedule's epoch 0 untimed and epochs
 *      1-3 timed (CUDA events) on scratch_positions, in two passes over the
 *      candidates; the faster pass counts.  A candidate stays in the running
 *      only if it is at least 3% faster than the entry configuration.
 *   2. Quality gate (tolerance >= 0): candidates in increasing time are laid
 *      out from initial_positions for schedule->total_epochs epochs with
 *      `seed`, and the first whose Eq. 4 objective U satisfies
 *      U <= (1 + tolerance) U_entry is chosen (U_entry: the entry
 *      configuration's layout; the objective is exact for batches and
 *      n <= 16384, otherwise the same 2^24 sampled pairs for every
 *      candidate).  A candidate whose layout becomes non-finite is
 *      rejected.  The entry configuration always passes.  When the handle
 *      keeps its CSR (SNAP_FLAG_KEEP_CSR, or SYNC) and no graph has more
 *      than 262,144 vertices, a candidate must also keep the neighbourhood
 *      preservation NP (Section 4.1, r = 2; snap_layout_neighborhood_preservation
 *      on 1,024 vertices drawn from `seed`, the same for every candidate)
 *      at NP >= (1 - tolerance) NP_entry.
 *      tolerance < 0: no gate, the fastest remaining candidate is chosen.
 *
 *   initial_positions  device, n x 2 float32, read only (may be NULL when
 *                      tolerance < 0).
 *   scratch_positions  device, n x 2 float32; overwritten.
 *   neg_samples, schedule, seed   as for snap_layout_epochs.
 *   chosen_segment, chosen_block, chosen_row_order (0 affine, 1 ascending),
 *   chosen_ms (ms per epoch),
 *   chosen_objective (U of the chosen layout; NaN without the gate),
 *   chosen_np (NP of the chosen layout; NaN when NP is not gated)
 *                      host outputs, nullable.
 * Synchronises the stream.  Errors: INVALID_ARG, NOT_SUPPORTED (SYNC),
 * NUMERIC (the entry configuration's layout became non-finite), CUDA.  On
 * an error the handle keeps a valid configuration.
 */
snap_status snap_layout_autotune(snap_layout_t h, const float *initial_positions, float *scratch_positions,
                                 int32_t neg_samples, const snap_schedule *schedule, uint64_t seed,
                                 double tolerance, int32_t *chosen_segment, int32_t *chosen_block,
                                 int32_t *chosen_row_order, double *chosen_ms, double *chosen_objective,
                                 double *chosen_np, void *cuda_stream);

/*
 * snap_layout_neighborhood_preservation -- NP of a layout (Section 4.1,
 * "Metrics", r = 2) on sampled vertices: for vertex i, N_G = the vertices
 * within two hops (i excluded, k = |N_G|), N_L = the k vertices of i's graph
 * nearest to i in the layout (squared distance formed in FP64 from the FP32
 * positions, ties to the smaller id), NP_i = |N_G & N_L| / |N_G | N_L|;
 * vertices without neighbours are skipped.
 *
 *   positions   device, n x 2 float32 (read only).
 *   nodes       host, count vertex ids in [0, n) (repeats allowed).
 *   out_mean    host: mean NP_i over the samples with neighbours (0 if none).
 *   out_used    host, nullable: the number of those samples.
 *
 * Needs the handle's device CSR: SYNC handles keep it, HOGWILD handles only
 * with SNAP_FLAG_KEEP_CSR (else NOT_SUPPORTED).  Each sample reads its graph's
 * positions 13 times (an exact radix select of the k-th nearest).  Allocates
 * scratch (for graphs above 262,144 vertices a 2-hop bitmap of n bits per
 * concurrent sample, at most 1 GiB), synchronises the stream.  Errors:
 * INVALID_ARG, NOT_SUPPORTED, OUT_OF_MEMORY, CUDA, NUMERIC (from an earlier
 * call).
 */
snap_status snap_layout_neighborhood_preservation(snap_layout_t h, const float *positions, const int32_t *nodes,
                                                  int32_t count, double *out_mean, int32_t *out_used,
                                                  void *cuda_stream);

/* Release the handle and its device memory.  NULL is ignored.  Does not
 * synchronise: the memory is freed stream-ordered after the work of the
 * handle's latest call (all work on a handle is assumed to be ordered on the
 * stream of its latest call).  The handle's memory is allocated
 * stream-ordered on the stream given to create, from a memory pool of the
 * library's own on that device, which keeps freed memory for the next
 * handle (snap_memory_cached, snap_memory_trim). */
void snap_layout_destroy(snap_layout_t h);

/*
 * snap_memory_cached -- device memory that the library's pool on `device`
 * holds for reuse: freed by released handles and not given back yet.  A
 * later create or temporary allocation of the library takes it before it
 * maps new memory; other allocators do not see it as free
 * (cudaMemGetInfo counts it as used).  Implementation choice, no
 * counterpart in the paper: mapping device memory costs about as much as
 * the rest of a create on a graph of millions of edges.
 *
 *   device   CUDA device ordinal (>= 0).
 *   bytes    host; receives the count (0 if the library has not allocated
 *            on that device).
 *
 * Errors: INVALID_ARG (NULL bytes, device < 0), CUDA.
 */
snap_status snap_memory_cached(int32_t device, uint64_t *bytes);

/*
 * snap_memory_trim -- give the cached memory of the library's pool on
 * `device` back to the device, down to keep_bytes (0: all of it).  Memory of
 * live handles is never released.  Errors: INVALID_ARG (device < 0), CUDA.
 */
snap_status snap_memory_trim(int32_t device, uint64_t keep_bytes);

/*
 * snap_sampler_table -- the alias table of a weighted sampler for one graph
 * (host only; snap_layout_create builds the same table, per graph of a
 * batch).  Integer weights q: the degrees (DEGREE) or
 * llround(w / max w * 2^32) (WEIGHTS).  Vose's construction in exact integer
 * arithmetic: the small vertices (n q_s < sum q) are served first-in
 * first-out in increasing id, the large ones from a stack filled in
 * increasing id; a column shared with alias a keeps its vertex with
 * probability threshold / 2^32 (threshold = floor(kept * 2^32 / sum q)), a
 * full column has threshold 0xFFFFFFFF and itself as alias.
 *
 *   sampler    SNAP_SAMPLER_DEGREE or SNAP_SAMPLER_WEIGHTS.
 *   row_ptr    host, n + 1 (DEGREE; unused for WEIGHTS).
 *   node_weights  host, n floats >= 0 (WEIGHTS; unused for DEGREE).
 *   threshold, alias  host outputs, n each (alias: vertex ids).
 * Errors: INVALID_ARG (unknown sampler, NULL array, a negative, NaN or
 * infinite weight, all weights zero).
 */
snap_status snap_sampler_table(int32_t sampler, const int64_t *row_ptr, const float *node_weights, int32_t n,
                               uint32_t *threshold, int32_t *alias);

/*
 * snap_graph_reorder -- locality relabelling of a symmetric CSR (host only).
 * Breadth-first order from the highest-degree unvisited vertex, neighbours
 * enqueued in ascending id order, so that vertices close in the graph get
 * close ids and a source bundle's partners share cache lines.  Not part of
 * the paper's method (which shuffles the edge list, Algorithm 1); it changes
 * only labels, never the layout problem.
 *
 *   row_ptr, col_idx, n   host, same contract as snap_layout_create.
 *   perm_out     host, n int32: perm_out[old] = new label.
 *   row_ptr_out  host, n+1 int64;  col_idx_out  host, nnz int32 (rows ascending).
 * Errors: INVALID_ARG, OUT_OF_MEMORY.
 */
snap_status snap_graph_reorder(const int64_t *row_ptr, const int32_t *col_idx, int32_t n,
                               int32_t *perm_out, int64_t *row_ptr_out, int32_t *col_idx_out);

/*
 * snap_layout_run -- whole layout from host buffers in one call: create,
 * copy positions to the device, epochs [0, epochs), copy them back, destroy.
 *
 *   positions_host  host, n x 2 float32, in: initial layout, out: final layout.
 * Synchronises the stream.  Errors: as create and epochs.
 */
snap_status snap_layout_run(const int64_t *row_ptr, const int32_t *col_idx, int32_t n,
                            const snap_options *opts, float *positions_host, int32_t epochs,
                            int32_t neg_samples, const snap_schedule *schedule, uint64_t seed,
                            void *cuda_stream);

/*
 * snap_sync_epochs_noalloc -- the synchronous mode (SNAP_MODE_SYNC) for
 * callers that cannot allocate device memory: code running inside a host
 * framework that owns all device memory through its own pool or budget, or
 * latency-critical code that must not pay for an allocation's implicit
 * synchronisation.  The paper has no counterpart; it is a deployment variant
 * of the same computation.
 *
 * Allocates nothing: no cudaMalloc/cudaFree and no allocating library call.
 * The per-vertex int64 displacement scratch lives in a fixed device array
 * inside the library, sized for at most 262,144 vertices (4 MiB, present on
 * every GPU that loads the library until the process exits).
 *
 *   row_ptr, col_idx  DEVICE, caller-owned, on the current device: the
 *                     symmetric CSR of snap_layout_create (n + 1 int64 and
 *                     nnz int32 entries).
 *   nnz               number of entries of col_idx, 0 <= nnz < 2^32.
 *   n                 1 <= n <= 262,144, else INVALID_ARG.
 *   positions         device, n x 2 float32, on the current device, updated
 *                     in place.
 *   epoch_begin, epochs, neg_samples, schedule, seed
 *                     as snap_layout_epochs.
 *   substeps, cap     as snap_options.sync_substeps / sync_cap.
 *
 * Before any epoch runs, the CSR is checked on the device with the rules of
 * snap_layout_create (row_ptr[0] = 0, row_ptr[n] = nnz, non-decreasing;
 * columns in [0, n), no self-loop, rows strictly ascending, every edge's
 * reverse present); a violation returns INVALID_ARG with the positions
 * untouched.  A buffer that is not device memory of the current device is
 * INVALID_ARG too.  The result equals snap_layout_epochs on a
 * SNAP_MODE_SYNC handle with the same substeps and cap (with any segment
 * length: the sums are integer).  The first call on a device looks up the scratch's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls in the process share the scratch, which keeps the last
 * call's contents (each call clears it first): calls that overlap on the GPU
 * -- other streams, other host threads -- race and must be serialised by the
 * caller.  Waits for the stream (after the check and at the end) before
 * returning.  Errors: INVALID_ARG, CUDA, NUMERIC.
 */
snap_status snap_sync_epochs_noalloc(const int64_t *row_ptr, const int32_t *col_idx, int64_t nnz,
                                     int32_t n, float *positions, int32_t epoch_begin, int32_t epochs,
                                     int32_t neg_samples, const snap_schedule *schedule, uint64_t seed,
                                     int32_t substeps, float cap, void *cuda_stream);

/*
 * Multi-handle epochs -- continuous batching of independent layouts.  The
 * paper lays out one graph at a time; this runs one epoch of several layouts
 * (jobs) in ONE kernel launch, each job at its own epoch index, step size and
 * seed, so jobs that arrive while others run can join at the next launch and
 * leave when their schedule ends.  Each job's random words are those of its
 * own handle, so its result is independent of the other jobs except through
 * race timing (and identical when each job is processed by a single lane,
 * i.e. segment_edges >= its entries).
 *
 * snap_multi_create  allocates a job table for up to max_jobs jobs per call.
 * snap_multi_epoch   enqueues epoch epochs[q] of job q for q < count:
 *     handles[q]     single-graph handle in SNAP_MODE_HOGWILD or
 *                    SNAP_MODE_HOGWILD_RED (all the same mode), else
 *                    NOT_SUPPORTED / INVALID_ARG;
 *     positions[q]   device pointer to that job's n x 2 float32 positions;
 *     schedules[q], seeds[q]  as in snap_layout_epochs.
 *   Asynchronous; it waits only until the previous call's job table has
 *   reached the device.  Jobs without edges are skipped.
 * snap_multi_check   waits for the stream; NUMERIC if a position became
 *                    non-finite in any job since the last check.
 */
typedef struct snap_multi snap_multi;
typedef snap_multi *snap_multi_t;
snap_status snap_multi_create(int32_t max_jobs, snap_multi_t *out);
snap_status snap_multi_epoch(snap_multi_t m, const snap_layout_t *handles, float *const *positions,
                             const int32_t *epochs, const snap_schedule *schedules, const uint64_t *seeds,
                             int32_t count, int32_t neg_samples, void *cuda_stream);
snap_status snap_multi_check(snap_multi_t m, void *cuda_stream);
void snap_multi_destroy(snap_multi_t m);

/* Message for the last non-OK status returned on this host thread. */
const char *snap_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SNAP_LAYOUT_H */
