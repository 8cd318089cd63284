// capi.cu -- the C ABI declared in include/snap_layout.h: handle life cycle,
// argument checking, launch configuration and error reporting.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/snap_layout.h"
#include "snap_internal.h"
#include "snap_sampler.h"

using namespace snap;

namespace {

thread_local std::string g_last_error;

snap_status fail(snap_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

snap_status cuda_fail(cudaError_t err, const char *what) {
    if (err == cudaErrorMemoryAllocation)
        return fail(SNAP_ERR_OUT_OF_MEMORY, "%s: %s", what, cudaGetErrorString(err));
    return fail(SNAP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(err));
}

// Host-side fault injection for tests: SNAP_FAULT_INJECT=alloc:N makes the
// N-th device allocation of a public call fail (1-based; snap_layout_run
// counts create's allocations first, then its own).
struct AllocCounter {
    int fail_at = 0;
    int count = 0;
    void reset() {
        count = 0;
        fail_at = 0;
        const char *v = getenv("SNAP_FAULT_INJECT");
        if (v && strncmp(v, "alloc:", 6) == 0) fail_at = atoi(v + 6);
    }
};

thread_local AllocCounter g_alloc;

// NVTX range over one library call (host timeline; a no-op unless a
// profiler that collects NVTX is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
thread_local bool g_in_run = false;

// Handle memory is stream-ordered (allocated on the creating stream,
// cudaFreeAsync when released), so creating and destroying handles never
// synchronises the device -- a server admits and retires layouts while other
// layouts keep running.  It comes from a memory pool of the library's own
// per device that keeps freed memory mapped (no release threshold): a create
// after a destroy reuses it instead of mapping new memory, which is most of
// the cost of an allocation of a graph's size (R-MAT 2^22: create + destroy
// 11.5 -> 8.1 ms).  snap_memory_trim gives the cached memory back.
struct LibraryPools {
    std::mutex mu;
    cudaMemPool_t pool[64] = {};
};
LibraryPools g_pools;

cudaMemPool_t library_pool(int dev, bool create) {
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_pools.mu);
    if (!g_pools.pool[dev] && create) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools.pool[dev] = pool;
    }
    return g_pools.pool[dev];
}

cudaError_t dev_alloc(AllocCounter &ac, void **p, size_t bytes, cudaStream_t stream) {
    ++ac.count;
    if (ac.fail_at > 0 && ac.count == ac.fail_at) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    cudaMemPool_t pool = library_pool(dev, true);
    if (!pool) return cudaMallocAsync(p, bytes < 16 ? 16 : bytes, stream);   // the device's default pool
    return cudaMallocFromPoolAsync(p, bytes < 16 ? 16 : bytes, pool, stream);
}

// One non-blocking stream per device on which released memory is freed,
// after waiting for the last work that used it.
cudaStream_t free_stream() {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!streams[dev]) cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
    return streams[dev];
}

// Pinned 16-byte status slots, handed out to handles and reused; the pool's
// pages live until the process exits.
struct StatusSlots {
    std::mutex mu;
    std::vector<uint32_t *> free_slots;
    std::vector<std::pair<uint32_t *, cudaEvent_t>> quarantine;   // read-back may be in flight

    uint32_t *take() {
        std::lock_guard<std::mutex> lock(mu);
        for (size_t q = 0; q < quarantine.size();) {
            if (cudaEventQuery(quarantine[q].second) == cudaSuccess) {
                cudaEventDestroy(quarantine[q].second);
                free_slots.push_back(quarantine[q].first);
                quarantine[q] = quarantine.back();
                quarantine.pop_back();
            } else {
                ++q;
            }
        }
        cudaGetLastError();
        if (free_slots.empty()) {
            uint32_t *page = nullptr;
            if (cudaMallocHost((void **)&page, 4096 * 4 * sizeof(uint32_t)) != cudaSuccess) return nullptr;
            for (int q = 4095; q >= 0; --q) free_slots.push_back(page + 4 * q);
        }
        uint32_t *slot = free_slots.back();
        free_slots.pop_back();
        return slot;
    }

    // `pending` (or nullptr) completes once no copy into the slot is in flight;
    // the pool then owns and destroys it.
    void give(uint32_t *slot, cudaEvent_t pending) {
        if (!slot) return;
        std::lock_guard<std::mutex> lock(mu);
        if (pending)
            quarantine.emplace_back(slot, pending);
        else
            free_slots.push_back(slot);
    }
};

StatusSlots g_status_slots;

// SplitMix64 finaliser (Steele, Lea, Flood 2014): the per-epoch offset of
// the slot-group order.
uint64_t mix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

double step_size(const snap_schedule &s, int32_t t) {
    if (s.kind == 1) return s.eta0;
    const double T = s.total_epochs > 0 ? (double)s.total_epochs : 1.0;
    const double eta = s.eta0 * (1.0 - (double)t / T);
    return eta > s.eta_min ? eta : s.eta_min;
}

constexpr int kObjGrid = 152 * 4;

}  // namespace

namespace snap {
snap_status reorder_fail(snap_status st, const char *msg) { return fail(st, "%s", msg); }
}  // namespace snap

struct CapturedEpochs {
    const float *pos;
    int32_t epoch_begin, epochs, k;
    uint64_t seed;
    snap_schedule sched;
    cudaGraphExec_t exec;
};

struct snap_layout {
    int32_t n = 0;
    int64_t nnz = 0;
    snap_options opts{};
    int32_t seg_len = 32;
    int32_t block = 256;
    int64_t num_segs = 0;
    int64_t *d_row_ptr = nullptr;
    int32_t *d_col = nullptr;
    int32_t *d_seg_row = nullptr;
    int32_t *d_deg = nullptr;
    long long *d_disp = nullptr;
    // oriented bundle list (HOGWILD modes): one entry per undirected edge,
    // cut into chunks of act_seg_len entries stored in slot order (ChunkLayout)
    int64_t act_nnz = 0;
    int64_t act_num_segs = 0;
    int32_t act_seg_len = 32;
    ChunkLayout act_layout{0, 0, 0, 0};   // T == 0 while the list is still row-major
    int64_t perm_mul = 1;                 // slot-group order multiplier
    int64_t *d_act_row_ptr = nullptr;
    int4 *d_act_ent = nullptr;
    int2 *d_act_meta = nullptr;
    int64_t act_ent_bytes = 0, act_meta_bytes = 0;
    int32_t *d_act_pieces = nullptr;      // chunks each vertex's oriented row spans
    int32_t *d_orient = nullptr;          // during create: orientation flags from the validation pass
    int64_t act_pieces_bytes = 0;
    // batch of graphs (num_graphs > 1): graph of every vertex and per-graph table
    int32_t num_graphs = 1;
    std::vector<int32_t> graph_offsets;   // num_graphs + 1 vertex offsets
    int32_t *d_node_graph = nullptr;
    GraphInfo *d_graphs = nullptr;
    std::vector<GraphInfo> h_graphs;
    bool graphs_set = false;
    snap_schedule graphs_sched{};
    uint64_t graphs_seed = 0;
    // weighted negatives (SNAP_SAMPLER_DEGREE / _WEIGHTS): per-vertex alias
    // table {threshold, graph-local alias} and objective factors
    uint2 *d_alias = nullptr;
    float4 *d_objw = nullptr;
    uint32_t *d_status = nullptr;   // [0] fault bits, [1] validation bits
    double *d_partial = nullptr;    // 2 * kObjGrid
    uint32_t *h_status = nullptr;   // pinned mirror of d_status[0]
    cudaEvent_t status_event = nullptr;
    bool status_pending = false;
    int sms = 1;
    int grid_sync = 0, grid_apply = 0;
    int grid_oriented[2][6] = {{0}};   // [red][negative width: k if k <= 4, else 5], filled on first use
    int grid_energy[2][6] = {{0}};     // the same for epochs that sum the actual energy
    std::vector<int64_t> chunk_edges;   // S + 1 edge offsets of the sync chunks
    int64_t device_bytes = 0;
    // CUDA graphs of captured epoch sequences (SNAP_FLAG_CUDA_GRAPH)
    cudaStream_t capture_stream = nullptr;
    std::vector<CapturedEpochs> captured;

    // Work that last used the handle's memory: the creating stream until the
    // first call, then the stream of the latest call.
    cudaStream_t alloc_stream = nullptr;
    cudaEvent_t last_use = nullptr;

    void mark_use(cudaStream_t s) {
        if (last_use) cudaEventRecord(last_use, s);
    }

    void free_async(void *p) {
        if (!p) return;
        cudaStream_t fs = free_stream();
        if (fs && last_use) {
            cudaStreamWaitEvent(fs, last_use, 0);
            cudaFreeAsync(p, fs);
        } else {
            cudaFreeAsync(p, alloc_stream);
        }
    }

    void release_csr() {
        free_async(d_row_ptr);
        free_async(d_col);
        free_async(d_seg_row);
        d_row_ptr = nullptr;
        d_col = nullptr;
        d_seg_row = nullptr;
    }

    void release() {
        release_csr();
        free_async(d_orient);
        d_orient = nullptr;
        free_async(d_act_row_ptr);
        free_async(d_act_ent);
        free_async(d_act_meta);
        free_async(d_act_pieces);
        d_act_pieces = nullptr;
        free_async(d_alias);
        free_async(d_objw);
        d_alias = nullptr;
        d_objw = nullptr;
        free_async(d_node_graph);
        free_async(d_graphs);
        d_node_graph = nullptr;
        d_graphs = nullptr;
        d_act_row_ptr = nullptr;
        d_act_ent = nullptr;
        d_act_meta = nullptr;
        free_async(d_deg);
        free_async(d_disp);
        free_async(d_status);
        free_async(d_partial);
        if (status_pending && status_event) {
            g_status_slots.give(h_status, status_event);   // the pool destroys the event
            status_event = nullptr;
        } else {
            g_status_slots.give(h_status, nullptr);
        }
        status_pending = false;
        for (const CapturedEpochs &c : captured) cudaGraphExecDestroy(c.exec);
        captured.clear();
        if (capture_stream) cudaStreamDestroy(capture_stream);
        capture_stream = nullptr;
        if (status_event) cudaEventDestroy(status_event);
        if (last_use) cudaEventDestroy(last_use);
        last_use = nullptr;
        d_deg = nullptr;
        d_disp = nullptr;
        d_status = nullptr;
        d_partial = nullptr;
        h_status = nullptr;
        status_event = nullptr;
    }
};

static int64_t gcd64(int64_t a, int64_t b) {
    while (b) {
        const int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Multiplier coprime with m near its golden section (0 when m <= 1): an
// affine map with it sends neighbouring indices far apart.
static int64_t golden_multiplier(int64_t m) {
    if (m <= 1) return 0;
    int64_t x = (int64_t)(0.6180339887498949 * (double)m) | 1;
    while (gcd64(x, m) != 1) x += 2;
    x %= m;
    return x == 0 ? 1 : x;
}

// (Re)cuts the oriented list into chunks of `target` entries: the entries
// move from the current layout (row-major right after construction) into a
// fresh array in the new slot order, and the slot table is rebuilt.
// The chunked layout of `entries` oriented entries in chunks of `target`
// (at most one chunk's worth of entries) in row order `order`.
static ChunkLayout make_chunk_layout(int64_t entries, int32_t target, int32_t order) {
    if (entries > 0 && target > entries) target = (int32_t)entries;   // one chunk
    ChunkLayout to;
    to.T = target;
    to.order = order;
    to.S = (entries + target - 1) / target;
    to.mul = golden_multiplier(to.S);
    to.add = to.S > 1 ? to.S / 3 : 0;
    return to;
}

// Makes (ent, meta) in layout `to` the handle's oriented list.
static void install_chunks(snap_layout *h, int4 *ent, int2 *meta, const ChunkLayout &to, int64_t ent_bytes,
                           int64_t meta_bytes) {
    h->device_bytes += ent_bytes + meta_bytes - h->act_ent_bytes - h->act_meta_bytes;
    h->d_act_ent = ent;
    h->d_act_meta = meta;
    h->act_ent_bytes = ent_bytes;
    h->act_meta_bytes = meta_bytes;
    h->act_layout = to;
    h->act_seg_len = to.T;
    h->act_num_segs = to.S;
    h->perm_mul = golden_multiplier((to.S + 31) / 32);
}

static cudaError_t set_chunks(snap_layout *h, AllocCounter &ac, int32_t target, int32_t order, cudaStream_t stream) {
    if (h->last_use) cudaStreamWaitEvent(stream, h->last_use, 0);   // the old arrays' last readers
    const ChunkLayout to = make_chunk_layout(h->act_nnz, target, order);
    target = to.T;
    const int64_t ent_bytes = (int64_t)sizeof(int4) * (to.S > 0 ? to.S * (int64_t)target : 1);
    const int64_t meta_bytes = (int64_t)sizeof(int2) * (to.S > 0 ? to.S : 1);
    int4 *ent = nullptr;
    int2 *meta = nullptr;
    cudaError_t err = dev_alloc(ac, (void **)&ent, (size_t)ent_bytes, stream);
    if (err == cudaSuccess) err = dev_alloc(ac, (void **)&meta, (size_t)meta_bytes, stream);
    if (err == cudaSuccess)
        err = launch_chunk_layout(h->d_act_ent, h->act_layout, ent, to, meta, h->d_act_row_ptr, h->n, h->act_nnz,
                                  stream);
    if (err != cudaSuccess) {
        if (ent) cudaFreeAsync(ent, stream);
        if (meta) cudaFreeAsync(meta, stream);
        return err;
    }
    {
        // the per-vertex piece counts depend on the chunk size
        if (!h->d_act_pieces) {
            const int64_t pb = (int64_t)sizeof(int32_t) * (h->n > 0 ? h->n : 1);
            err = dev_alloc(ac, (void **)&h->d_act_pieces, (size_t)pb, stream);
            if (err == cudaSuccess) {
                h->act_pieces_bytes = pb;
                h->device_bytes += pb;
            }
        }
        if (err == cudaSuccess) err = launch_row_pieces(h->d_act_row_ptr, h->n, target, h->d_act_pieces, stream);
        if (err != cudaSuccess) {
            cudaFreeAsync(ent, stream);
            cudaFreeAsync(meta, stream);
            return err;
        }
    }
    cudaFreeAsync(h->d_act_ent, stream);
    if (h->d_act_meta) cudaFreeAsync(h->d_act_meta, stream);
    install_chunks(h, ent, meta, to, ent_bytes, meta_bytes);
    return cudaSuccess;
}

// Builds the oriented bundle list from the validated device CSR and then
// frees the CSR (the HOGWILD kernels and the objective need only the list).
// The oriented list of a validated CSR.  h->d_orient holds the orientation
// flags the validation pass wrote (nnz + 1 entries); it is consumed here.
static snap_status build_oriented(snap_layout *h, AllocCounter &ac, cudaStream_t stream) {
    const int32_t n = h->n;
    const int64_t nnz = h->nnz;
    h->act_nnz = nnz / 2;   // symmetric and loop-free: each undirected edge once
    if (h->act_seg_len == 0) {
        // Default chunk: 4 entries.  A lane applies a chunk's steps of one
        // source back to back; long bursts of one source's steps move the
        // layout away from Algorithm 1's shuffled order (R-MAT 2^17,
        // sequential, eta0 = 1: +0.8% energy at 4 entries, +5% at 32, +10% at
        // 128).  Concurrency is bounded separately (max_inflight).
        h->act_seg_len = 4;
    }
    const ChunkLayout to = make_chunk_layout(h->act_nnz, h->act_seg_len,
                                             (h->opts.flags & SNAP_FLAG_ASCENDING_ROWS) ? 1 : 0);
    const int64_t ent_bytes = (int64_t)sizeof(int4) * (to.S > 0 ? to.S * (int64_t)to.T : 1);
    const int64_t meta_bytes = (int64_t)sizeof(int2) * (to.S > 0 ? to.S : 1);
    const int64_t pieces_bytes = (int64_t)sizeof(int32_t) * (n > 0 ? n : 1);
    int32_t *pos = nullptr;
    int4 *ent = nullptr;
    int2 *meta = nullptr;
    void *temp = nullptr;
    size_t temp_bytes = 0;
    cudaError_t err = cudaSuccess;
    const char *what = "";
    auto alloc = [&](void **p, size_t bytes, bool keep, const char *nm) {
        if (err != cudaSuccess) return;
        err = dev_alloc(ac, p, bytes, stream);
        if (err != cudaSuccess) {
            what = nm;
        } else if (keep) {
            h->device_bytes += (int64_t)bytes;
        }
    };
    auto step = [&](cudaError_t e, const char *nm) {
        if (err == cudaSuccess && e != cudaSuccess) {
            err = e;
            what = nm;
        }
    };
    alloc((void **)&h->d_act_row_ptr, sizeof(int64_t) * ((size_t)n + 1), true, "oriented row offsets");
    alloc((void **)&ent, (size_t)ent_bytes, false, "oriented entries");
    alloc((void **)&meta, (size_t)meta_bytes, false, "slot descriptors");
    alloc((void **)&h->d_act_pieces, (size_t)pieces_bytes, true, "row pieces");
    alloc((void **)&pos, sizeof(int32_t) * ((size_t)nnz + 1), false, "orientation offsets");
    if (err == cudaSuccess)
        step(exclusive_scan_i32(nullptr, &temp_bytes, h->d_orient, pos, nnz + 1, stream), "scan size");
    alloc(&temp, temp_bytes, false, "scan scratch");
    if (err == cudaSuccess) {
        h->act_pieces_bytes = pieces_bytes;
        step(exclusive_scan_i32(temp, &temp_bytes, h->d_orient, pos, nnz + 1, stream), "orientation scan");
        step(launch_orient_scatter(h->d_row_ptr, h->d_col, h->d_seg_row, h->d_deg, nnz, h->seg_len, pos, to, ent,
                                   meta, h->act_nnz, h->d_status + 1, stream),
             "orientation scatter kernel");
        step(launch_orient_rowptr(h->d_row_ptr, pos, n, h->d_act_row_ptr, stream), "orientation offsets kernel");
        step(launch_row_pieces(h->d_act_row_ptr, n, to.T, h->d_act_pieces, stream), "row pieces kernel");
    }
    int64_t total = -1;
    if (err == cudaSuccess) {
        step(cudaMemcpyAsync(&total, h->d_act_row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream),
             "read oriented entry count");
        step(cudaMemcpyAsync(h->h_status + 1, h->d_status + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream),
             "read symmetry word");
        step(cudaStreamSynchronize(stream), "orientation");
    }
    cudaFreeAsync(h->d_orient, stream);
    h->d_orient = nullptr;
    if (pos) cudaFreeAsync(pos, stream);
    if (temp) cudaFreeAsync(temp, stream);
    if (err != cudaSuccess) {
        if (ent) cudaFreeAsync(ent, stream);
        if (meta) cudaFreeAsync(meta, stream);
        return cuda_fail(err, what);
    }
    h->act_ent_bytes = 0;
    h->act_meta_bytes = 0;
    install_chunks(h, ent, meta, to, ent_bytes, meta_bytes);
    // every owned edge has its reverse and half of the edges are owned: symmetric
    if ((h->h_status[1] & kAsymmetric) || (nnz & 1) || total != h->act_nnz)
        return fail(SNAP_ERR_INVALID_ARG, "the CSR is not symmetric: some (i, j) has no (j, i)");
    if (!(h->opts.flags & SNAP_FLAG_KEEP_CSR)) {
        h->device_bytes -= (int64_t)(sizeof(int64_t) * ((size_t)n + 1) +
                                     sizeof(int32_t) * (size_t)(h->num_segs * h->seg_len + 4) +
                                     sizeof(int32_t) * (size_t)(h->num_segs > 0 ? h->num_segs : 1));
        h->release_csr();
    }
    return SNAP_OK;
}

extern "C" {

void snap_options_default(snap_options *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->mode = SNAP_MODE_HOGWILD_RED;
    o->sampler = SNAP_SAMPLER_UNIFORM;
    o->node_weights = nullptr;
    o->sync_substeps = 1;
    o->sync_cap = 0.0f;
    o->segment_edges = 0;
    o->block_threads = 0;
    o->flags = 0;
    o->max_inflight = 0.0f;
}

const char *snap_last_error(void) { return g_last_error.c_str(); }

static snap_status check_csr_host(const int64_t *row_ptr, const int32_t *col_idx, const int32_t *degrees,
                                  int32_t n) {
    if (!row_ptr) return fail(SNAP_ERR_INVALID_ARG, "row_ptr is NULL");
    if (n < 1 || n == INT32_MAX) return fail(SNAP_ERR_INVALID_ARG, "n = %d out of range [1, 2^31-2]", n);
    if (row_ptr[0] != 0) return fail(SNAP_ERR_INVALID_ARG, "row_ptr[0] = %lld, expected 0", (long long)row_ptr[0]);
    // the rest of row_ptr is checked on the device (check_row_ptr_kernel)
    const int64_t nnz = row_ptr[n];
    if (nnz < 0) return fail(SNAP_ERR_INVALID_ARG, "row_ptr[n] = %lld is negative", (long long)nnz);
    if (nnz >= ((int64_t)1 << 32)) return fail(SNAP_ERR_INVALID_ARG, "nnz = %lld exceeds 2^32-1", (long long)nnz);
    if (nnz > 0 && !col_idx) return fail(SNAP_ERR_INVALID_ARG, "col_idx is NULL");
    if (degrees)
        for (int32_t i = 0; i < n; ++i)
            if ((int64_t)degrees[i] != row_ptr[i + 1] - row_ptr[i])
                return fail(SNAP_ERR_INVALID_ARG, "degrees[%d] = %d but row %d has %lld entries", i, degrees[i], i,
                            (long long)(row_ptr[i + 1] - row_ptr[i]));
    return SNAP_OK;
}

static snap_status check_options(const snap_options &o) {
    if (o.mode < SNAP_MODE_HOGWILD || o.mode > SNAP_MODE_SYNC)
        return fail(SNAP_ERR_INVALID_ARG, "unknown mode %d", o.mode);
    if (o.sampler < SNAP_SAMPLER_UNIFORM || o.sampler > SNAP_SAMPLER_WEIGHTS)
        return fail(SNAP_ERR_INVALID_ARG, "unknown sampler %d", o.sampler);
    if (o.sampler == SNAP_SAMPLER_WEIGHTS && !o.node_weights)
        return fail(SNAP_ERR_INVALID_ARG, "SNAP_SAMPLER_WEIGHTS needs node_weights");
    if (o.sync_substeps < 1 || o.sync_substeps > (1 << 20))
        return fail(SNAP_ERR_INVALID_ARG, "sync_substeps = %d out of range [1, 2^20]", o.sync_substeps);
    if (!(o.sync_cap >= 0.0f) || !std::isfinite(o.sync_cap))
        return fail(SNAP_ERR_INVALID_ARG, "sync_cap must be finite and >= 0");
    if (o.segment_edges != 0 && (o.segment_edges < 4 || o.segment_edges > 4096 || o.segment_edges % 4 != 0))
        return fail(SNAP_ERR_INVALID_ARG, "segment_edges = %d must be 0 or a multiple of 4 in [4, 4096]",
                    o.segment_edges);
    if (o.flags & ~(SNAP_FLAG_CUDA_GRAPH | SNAP_FLAG_KEEP_CSR | SNAP_FLAG_ASCENDING_ROWS))
        return fail(SNAP_ERR_INVALID_ARG, "unknown flags 0x%x", o.flags);
    if (!(o.max_inflight >= 0.0f) || !(o.max_inflight <= 1.0f))
        return fail(SNAP_ERR_INVALID_ARG, "max_inflight must be in [0, 1]");
    if (o.block_threads != 0 && (o.block_threads < 32 || o.block_threads > 256 || o.block_threads % 32 != 0))
        return fail(SNAP_ERR_INVALID_ARG, "block_threads = %d must be 0 or a multiple of 32 in [32, 256]",
                    o.block_threads);
    return SNAP_OK;
}

// Alias tables and objective factors of a weighted sampler, one per graph of
// the handle (graph-local ids), built on the host in exact integer arithmetic.
static snap_status sampler_tables(const snap_options &o, const int64_t *row_ptr, int32_t n,
                                  const int32_t *graph_offsets, int32_t num_graphs, std::vector<uint2> &table,
                                  std::vector<float4> &objw) {
    table.assign((size_t)n, make_uint2(0xFFFFFFFFu, 0u));
    objw.assign((size_t)n, make_float4(0.f, 0.f, 0.f, 0.f));
    std::vector<uint64_t> q;
    std::vector<uint32_t> thr;
    std::vector<int32_t> al;
    const int32_t graphs = graph_offsets ? num_graphs : 1;
    for (int32_t g = 0; g < graphs; ++g) {
        const int32_t v0 = graph_offsets ? graph_offsets[g] : 0;
        const int32_t v1 = graph_offsets ? graph_offsets[g + 1] : n;
        const int32_t ng = v1 - v0;
        q.assign((size_t)ng, 0);
        const int rc = sampler_weights(o.sampler, row_ptr, o.node_weights, v0, v1, q.data());
        if (rc == 1) return fail(SNAP_ERR_INVALID_ARG, "node_weights must be finite and >= 0");
        if (rc == 2) {
            if (row_ptr[v1] > row_ptr[v0])
                return fail(SNAP_ERR_INVALID_ARG, "the sampler's weights of graph %d are all zero", g);
            for (uint64_t &x : q) x = 1;   // no edges: the table is never used
        }
        thr.assign((size_t)ng, 0);
        al.assign((size_t)ng, 0);
        alias_table(q.data(), ng, thr.data(), al.data());
        for (int32_t s = 0; s < ng; ++s) table[(size_t)(v0 + s)] = make_uint2(thr[(size_t)s], (uint32_t)al[(size_t)s]);
        sampler_objective_factors(row_ptr, q.data(), v0, v1, objw.data() + v0);
    }
    return SNAP_OK;
}

static snap_status create_impl(const int64_t *row_ptr, const int32_t *col_idx, const int32_t *degrees, int32_t n,
                               const int32_t *graph_offsets, int32_t num_graphs, const snap_options *opts,
                               void *cuda_stream, snap_layout_t *out) {
    NvtxRange nvtx_range("snap_layout_create");
    if (!out) return fail(SNAP_ERR_INVALID_ARG, "out is NULL");
    snap_status st = check_csr_host(row_ptr, col_idx, degrees, n);
    if (st != SNAP_OK) return st;
    if (num_graphs < 1) return fail(SNAP_ERR_INVALID_ARG, "num_graphs = %d must be >= 1", num_graphs);
    if (graph_offsets) {
        if (graph_offsets[0] != 0 || graph_offsets[num_graphs] != n)
            return fail(SNAP_ERR_INVALID_ARG, "graph_offsets must start at 0 and end at n");
        for (int32_t g = 0; g < num_graphs; ++g)
            if (graph_offsets[g + 1] <= graph_offsets[g])
                return fail(SNAP_ERR_INVALID_ARG, "graph %d is empty or graph_offsets decreases", g);
    }
    snap_options o;
    snap_options_default(&o);
    if (opts) o = *opts;
    st = check_options(o);
    if (st != SNAP_OK) return st;
    std::vector<uint2> alias_host;
    std::vector<float4> objw_host;
    if (o.sampler != SNAP_SAMPLER_UNIFORM) {
        st = sampler_tables(o, row_ptr, n, graph_offsets, num_graphs, alias_host, objw_host);
        if (st != SNAP_OK) return st;
    }

    cudaStream_t stream = (cudaStream_t)cuda_stream;
    snap_layout *h = new (std::nothrow) snap_layout();
    if (!h) return fail(SNAP_ERR_OUT_OF_MEMORY, "host allocation of the handle failed");
    h->alloc_stream = stream;
    if (cudaEventCreateWithFlags(&h->last_use, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(SNAP_ERR_CUDA, "event creation failed");
    }
    cudaEventRecord(h->last_use, stream);
    h->n = n;
    h->nnz = row_ptr[n];
    h->opts = o;
    h->num_graphs = graph_offsets ? num_graphs : 1;
    if (graph_offsets && num_graphs > 1) h->graph_offsets.assign(graph_offsets, graph_offsets + num_graphs + 1);
    // CSR segments: the synchronous kernel's unit of work (and the
    // validation pass); the HOGWILD modes use chunks of oriented entries.
    // SYNC takes 16 edges by default: a chunk of 1/S of the edges in 32-edge
    // segments leaves a tail wave (R-MAT 2^22, S = 16: 7.08 ms per epoch at
    // 32, 6.78 at 16, 6.89 at 8, 7.72 at 4; the sums are integer, so the
    // result is the same for every length).
    h->seg_len = o.mode == SNAP_MODE_SYNC ? (o.segment_edges ? o.segment_edges : 16) : 32;
    h->act_seg_len = (o.mode != SNAP_MODE_SYNC && o.segment_edges) ? o.segment_edges : 0;   // 0: by size
    h->block = o.block_threads ? o.block_threads : 256;
    h->num_segs = (h->nnz + h->seg_len - 1) / h->seg_len;

    AllocCounter &ac = g_alloc;
    if (!g_in_run) ac.reset();
    cudaError_t err;
    const size_t col_entries = (size_t)(h->num_segs * h->seg_len + 4);
    const size_t disp_bytes = o.mode == SNAP_MODE_SYNC ? sizeof(long long) * 2 * (size_t)n : 0;
#define SNAP_ALLOC(ptr, bytes)                                                        \
    do {                                                                              \
        err = dev_alloc(ac, (void **)&(ptr), (bytes), stream);                        \
        if (err != cudaSuccess) {                                                     \
            h->release();                                                             \
            delete h;                                                                 \
            cudaGetLastError();                                                       \
            return cuda_fail(err, "device allocation of " #ptr);                      \
        }                                                                             \
        h->device_bytes += (int64_t)(bytes);                                          \
    } while (0)
    SNAP_ALLOC(h->d_row_ptr, sizeof(int64_t) * ((size_t)n + 1));
    SNAP_ALLOC(h->d_col, sizeof(int32_t) * col_entries);
    SNAP_ALLOC(h->d_seg_row, sizeof(int32_t) * (size_t)(h->num_segs > 0 ? h->num_segs : 1));
    SNAP_ALLOC(h->d_deg, sizeof(int32_t) * (size_t)n);
    SNAP_ALLOC(h->d_status, sizeof(uint32_t) * 4);
    SNAP_ALLOC(h->d_partial, sizeof(double) * 2 * kObjGrid);
    if (disp_bytes) SNAP_ALLOC(h->d_disp, disp_bytes);
    if (!alias_host.empty()) {
        SNAP_ALLOC(h->d_alias, sizeof(uint2) * (size_t)n);
        SNAP_ALLOC(h->d_objw, sizeof(float4) * (size_t)n);
    }
    if (h->num_graphs > 1) {
        SNAP_ALLOC(h->d_node_graph, sizeof(int32_t) * (size_t)n);
        SNAP_ALLOC(h->d_graphs, sizeof(GraphInfo) * (size_t)h->num_graphs);
    }
#undef SNAP_ALLOC

#define SNAP_CUDA(call, what)                                                         \
    do {                                                                              \
        err = (call);                                                                 \
        if (err != cudaSuccess) {                                                     \
            cudaStreamSynchronize(stream);                                            \
            h->release();                                                             \
            delete h;                                                                 \
            cudaGetLastError();                                                       \
            return cuda_fail(err, what);                                              \
        }                                                                             \
    } while (0)
    h->h_status = g_status_slots.take();
    SNAP_CUDA(h->h_status ? cudaSuccess : cudaErrorMemoryAllocation, "pinned status word");
    SNAP_CUDA(cudaEventCreateWithFlags(&h->status_event, cudaEventDisableTiming), "status event");
    SNAP_CUDA(cudaMemcpyAsync(h->d_row_ptr, row_ptr, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyHostToDevice,
                              stream), "copy row_ptr");
    if (h->nnz > 0)
        SNAP_CUDA(cudaMemcpyAsync(h->d_col, col_idx, sizeof(int32_t) * (size_t)h->nnz, cudaMemcpyHostToDevice,
                                  stream), "copy col_idx");
    SNAP_CUDA(cudaMemsetAsync(h->d_col + h->nnz, 0, sizeof(int32_t) * (col_entries - (size_t)h->nnz), stream),
              "clear col_idx padding");
    SNAP_CUDA(launch_degrees(h->d_row_ptr, n, h->d_deg, stream), "degree kernel");
    SNAP_CUDA(cudaMemsetAsync(h->d_status, 0, sizeof(uint32_t) * 4, stream), "clear status");
    std::vector<int32_t> node_graph;
    if (h->num_graphs > 1) {
        node_graph.resize((size_t)n);
        h->h_graphs.assign((size_t)h->num_graphs, GraphInfo{});
        for (int32_t g = 0; g < h->num_graphs; ++g) {
            for (int32_t v = graph_offsets[g]; v < graph_offsets[g + 1]; ++v) node_graph[(size_t)v] = g;
            GraphInfo &gi = h->h_graphs[(size_t)g];
            gi.node_base = graph_offsets[g];
            gi.n = graph_offsets[g + 1] - graph_offsets[g];
            gi.edge_base = row_ptr[graph_offsets[g]];
        }
        SNAP_CUDA(cudaMemcpyAsync(h->d_node_graph, node_graph.data(), sizeof(int32_t) * (size_t)n,
                                  cudaMemcpyHostToDevice, stream), "copy vertex graphs");
        SNAP_CUDA(cudaMemcpyAsync(h->d_graphs, h->h_graphs.data(), sizeof(GraphInfo) * h->h_graphs.size(),
                                  cudaMemcpyHostToDevice, stream), "copy graph table");
    }
    if (h->d_disp) SNAP_CUDA(cudaMemsetAsync(h->d_disp, 0, disp_bytes, stream), "clear displacement");
    if (h->d_alias) {
        SNAP_CUDA(cudaMemcpyAsync(h->d_alias, alias_host.data(), sizeof(uint2) * (size_t)n, cudaMemcpyHostToDevice,
                                  stream), "copy alias table");
        SNAP_CUDA(cudaMemcpyAsync(h->d_objw, objw_host.data(), sizeof(float4) * (size_t)n, cudaMemcpyHostToDevice,
                                  stream), "copy objective factors");
    }
    SNAP_CUDA(launch_segment_rows(h->d_row_ptr, n, h->nnz, h->seg_len, h->d_seg_row, h->num_segs, stream),
              "segment table kernel");
    // symmetry: here for the synchronous mode, in the orientation pass otherwise;
    // the HOGWILD modes also take the orientation flags from this pass
    unsigned long long *upper = o.mode == SNAP_MODE_SYNC
                                    ? reinterpret_cast<unsigned long long *>(h->d_status + 2)
                                    : nullptr;
    if (o.mode != SNAP_MODE_SYNC && h->nnz > 0) {
        err = dev_alloc(ac, (void **)&h->d_orient, sizeof(int32_t) * ((size_t)h->nnz + 1), stream);
        if (err != cudaSuccess) {
            h->release();
            delete h;
            cudaGetLastError();
            return cuda_fail(err, "device allocation of the orientation flags");
        }
    }
    SNAP_CUDA(launch_validate_csr(h->d_row_ptr, h->d_col, h->d_seg_row, n, h->nnz, h->seg_len, h->d_status + 1,
                                  stream, h->d_node_graph, upper, h->d_deg, h->d_orient), "validation kernel");
    SNAP_CUDA(cudaMemcpyAsync(h->h_status, h->d_status, sizeof(uint32_t) * 4, cudaMemcpyDeviceToHost, stream),
              "read validation word");
    SNAP_CUDA(cudaStreamSynchronize(stream), "create");
#undef SNAP_CUDA
    uint32_t vflags = h->h_status[1];
    if (upper && !vflags) {
        unsigned long long count = 0;
        memcpy(&count, h->h_status + 2, sizeof(count));
        if ((h->nnz & 1) || (int64_t)count != h->nnz / 2) vflags |= kAsymmetric;
    }
    if (vflags) {
        h->release();
        delete h;
        if (vflags & kBadRowPtr) return fail(SNAP_ERR_INVALID_ARG, "row_ptr decreases or leaves [0, nnz]");
        if (vflags & kBadColumn) return fail(SNAP_ERR_INVALID_ARG, "col_idx holds a column outside [0, n)");
        if (vflags & kSelfLoop) return fail(SNAP_ERR_INVALID_ARG, "col_idx holds a self-loop (j == i)");
        if (vflags & kUnsorted) return fail(SNAP_ERR_INVALID_ARG, "a row of col_idx is not strictly ascending");
        if (vflags & kCrossGraph) return fail(SNAP_ERR_INVALID_ARG, "an edge joins two graphs of the batch");
        return fail(SNAP_ERR_INVALID_ARG, "the CSR is not symmetric: some (i, j) has no (j, i)");
    }
    h->h_status[0] = 0;

    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    h->sms = sms;
    h->grid_sync = sms * sync_blocks_per_sm(h->block);
    h->grid_apply = sms * 8;
    cudaGetLastError();

    if (o.mode != SNAP_MODE_SYNC && h->nnz > 0) {
        st = build_oriented(h, ac, stream);
        if (st != SNAP_OK) {
            cudaStreamSynchronize(stream);
            h->release();
            delete h;
            cudaGetLastError();
            return st;
        }
    }

    const int32_t S = o.sync_substeps;
    h->chunk_edges.assign((size_t)S + 1, 0);
    {
        int32_t r = 0;
        h->chunk_edges[0] = 0;
        for (int32_t c = 1; c < S; ++c) {
            while (r < n && row_ptr[r] * (int64_t)S < (int64_t)c * h->nnz) ++r;
            h->chunk_edges[(size_t)c] = row_ptr[r];
        }
        h->chunk_edges[(size_t)S] = h->nnz;
    }
    *out = h;
    return SNAP_OK;
}

snap_status snap_sampler_table(int32_t sampler, const int64_t *row_ptr, const float *node_weights, int32_t n,
                               uint32_t *threshold, int32_t *alias) {
    if (sampler != SNAP_SAMPLER_DEGREE && sampler != SNAP_SAMPLER_WEIGHTS)
        return fail(SNAP_ERR_INVALID_ARG, "sampler %d has no table", sampler);
    if (n < 1 || !threshold || !alias) return fail(SNAP_ERR_INVALID_ARG, "NULL output or n < 1");
    if (sampler == SNAP_SAMPLER_DEGREE ? !row_ptr : !node_weights)
        return fail(SNAP_ERR_INVALID_ARG, "the sampler's input array is NULL");
    std::vector<uint64_t> q((size_t)n);
    const int rc = sampler_weights(sampler, row_ptr, node_weights, 0, n, q.data());
    if (rc == 1) return fail(SNAP_ERR_INVALID_ARG, "node_weights must be finite and >= 0");
    if (rc == 2) return fail(SNAP_ERR_INVALID_ARG, "all weights are zero");
    alias_table(q.data(), n, threshold, alias);
    return SNAP_OK;
}

snap_status snap_layout_create(const int64_t *row_ptr, const int32_t *col_idx, const int32_t *degrees, int32_t n,
                               const snap_options *opts, void *cuda_stream, snap_layout_t *out) {
    return create_impl(row_ptr, col_idx, degrees, n, nullptr, 1, opts, cuda_stream, out);
}

snap_status snap_layout_create_batch(const int64_t *row_ptr, const int32_t *col_idx, int32_t n,
                                     const int32_t *graph_offsets, int32_t num_graphs, const snap_options *opts,
                                     void *cuda_stream, snap_layout_t *out) {
    if (!graph_offsets) return fail(SNAP_ERR_INVALID_ARG, "graph_offsets is NULL");
    return create_impl(row_ptr, col_idx, nullptr, n, graph_offsets, num_graphs, opts, cuda_stream, out);
}

static snap_status poll_status(snap_layout *h) {
    if (h->status_pending && cudaEventQuery(h->status_event) == cudaSuccess) {
        h->status_pending = false;
        const uint32_t f = h->h_status[0];
        if (f) {
            h->h_status[0] = 0;
            cudaMemset(h->d_status, 0, sizeof(uint32_t));
            if (f & kStatusNonFinite) return fail(SNAP_ERR_NUMERIC, "an earlier epoch produced a non-finite position");
            return fail(SNAP_ERR_NUMERIC, "an earlier synchronous epoch clamped a fixed-point force term");
        }
    }
    cudaGetLastError();
    return SNAP_OK;
}

static snap_status check_schedule(const snap_schedule *s) {
    if (!s) return fail(SNAP_ERR_INVALID_ARG, "schedule is NULL");
    if (s->kind != 0 && s->kind != 1) return fail(SNAP_ERR_INVALID_ARG, "unknown schedule kind %d", s->kind);
    if (!(s->eta0 > 0.0) || !std::isfinite(s->eta0)) return fail(SNAP_ERR_INVALID_ARG, "eta0 must be finite and > 0");
    if (!(s->eta_min >= 0.0) || !std::isfinite(s->eta_min))
        return fail(SNAP_ERR_INVALID_ARG, "eta_min must be finite and >= 0");
    if (s->total_epochs < 1) return fail(SNAP_ERR_INVALID_ARG, "total_epochs must be >= 1");
    return SNAP_OK;
}

// Default share of a graph's entries in flight at once: 0.5% for both modes.
// Concurrent updates of one vertex cost Hogwild quality: atomic adds of
// changes computed from the same stale position overshoot, overwrites lose
// updates (LFR 260k / 6.9M, 5 seeds, NP against the oracle: HOGWILD_RED
// -1.4% at 1%, -0.7% at 0.5%, -0.4% at 0.3%; 30 epochs, SI of the planted
// communities against the oracle's, mean of 3 runs: HOGWILD -5.7% at 1%,
// -3.7% at 0.5% and at 0.25%; HOGWILD_RED -3.6% at 0.5%, -2.0% at 0.25%).
// 0.5% costs HOGWILD 6% of the LFR epoch and HOGWILD_RED none (0.25%:
// 1.5x slower); on the 34M-edge R-MAT graph every share exceeds the
// resident lanes.
static double default_inflight(int) { return 0.005; }

// Grid of a HOGWILD epoch: enough blocks for every chunk, at most the
// resident maximum, and at most max_inflight * entries lanes (one entry in
// flight per lane), so small graphs are not updated by too many lanes at
// once (each lane grid-strides over several chunks instead).
static int inflight_grid(const snap_layout *h, int gmax) {
    const int64_t want = (h->act_num_segs + h->block - 1) / h->block;
    int64_t grid = want < gmax ? want : gmax;
    const double frac = h->opts.max_inflight > 0.0f ? (double)h->opts.max_inflight
                                                     : default_inflight(h->opts.mode == SNAP_MODE_HOGWILD_RED);
    const int64_t lanes_cap = (int64_t)(frac * (double)h->act_nnz);
    const int64_t grid_cap = (lanes_cap + h->block - 1) / h->block;
    if (grid_cap < grid) grid = grid_cap;
    return grid > 0 ? (int)grid : 1;
}

// Enqueues chunks [c_begin, c_end) of epoch t of the synchronous mode: for
// each chunk, the frozen-position force sum of its rows (sync_chunk_kernel)
// and the apply step (sync_apply_kernel).
static cudaError_t enqueue_sync_chunks(snap_layout *h, float2 *pos, int32_t t, int32_t c_begin, int32_t c_end,
                                       int32_t neg_samples, const snap_schedule &sched, uint64_t seed,
                                       cudaStream_t stream, double *energy) {
    const double eta = step_size(sched, t);
    const double limit = h->opts.sync_cap > 0.0f ? (double)h->opts.sync_cap * eta / sched.eta0 : 0.0;
    cudaError_t err = cudaSuccess;
    for (int32_t c = c_begin; c < c_end && err == cudaSuccess; ++c) {
        const int64_t eb = h->chunk_edges[(size_t)c], ee = h->chunk_edges[(size_t)c + 1];
        if (ee > eb) {
            SyncArgs a;
            a.row_ptr = h->d_row_ptr;
            a.col_idx = h->d_col;
            a.seg_row = h->d_seg_row;
            a.pos = pos;
            a.disp = h->d_disp;
            a.e_begin = eb;
            a.e_end = ee;
            a.n = h->n;
            a.k = neg_samples;
            a.seg_len = h->seg_len;
            a.epoch = (uint32_t)t;
            a.seed = seed;
            a.status = h->d_status;
            a.node_graph = h->d_node_graph;
            a.graphs = h->num_graphs > 1 ? h->d_graphs : nullptr;
            a.alias = h->d_alias;
            a.energy = energy;
            const int64_t segs = (ee + h->seg_len - 1) / h->seg_len - eb / h->seg_len;
            const int64_t want = (segs + h->block - 1) / h->block;
            const int grid = (int)(want < h->grid_sync ? want : h->grid_sync);
            err = launch_sync_chunk(a, grid > 0 ? grid : 1, h->block, stream);
        }
        if (err == cudaSuccess)
            err = launch_sync_apply(pos, h->d_disp, h->n, (float)eta, (float)limit, h->d_status, h->grid_apply, 256,
                                    stream, h->d_node_graph, h->num_graphs > 1 ? h->d_graphs : nullptr, t,
                                    h->opts.sync_cap);
    }
    return err;
}

// Enqueues the launches of epochs [epoch_begin, epoch_begin + epochs) on `stream`.
static cudaError_t enqueue_epochs(snap_layout *h, float2 *pos, int32_t epoch_begin, int32_t epochs,
                                  int32_t neg_samples, const snap_schedule &sched, uint64_t seed,
                                  cudaStream_t stream, double *energy = nullptr) {
    const snap_schedule *schedule = &sched;
    cudaError_t err = cudaSuccess;
    for (int32_t ep = 0; ep < epochs; ++ep) {
        NvtxRange nvtx_epoch("epoch");
        const int32_t t = epoch_begin + ep;
        const double eta = step_size(*schedule, t);
        if (h->opts.mode == SNAP_MODE_SYNC) {
            err = enqueue_sync_chunks(h, pos, t, 0, h->opts.sync_substeps, neg_samples, *schedule, seed, stream,
                                      energy ? energy + ep : nullptr);
        } else {
            OrientedArgs a;
            a.row_ptr = h->d_act_row_ptr;
            a.ent = h->d_act_ent;
            a.meta = h->d_act_meta;
            a.pos = pos;
            a.num_segs = h->act_num_segs;
            a.nnz = h->act_nnz;
            a.seg_len = h->act_seg_len;
            a.perm_mul = h->perm_mul;
            a.perm_add = (int64_t)(mix64(seed ^ (0x5EC0ull * (uint64_t)(t + 1))) %
                                   (uint64_t)(h->act_num_segs > 0 ? (h->act_num_segs + 31) / 32 : 1));
            a.n = h->n;
            a.k = neg_samples;
            a.epoch = (uint32_t)t;
            a.seed = seed;
            a.eta = (float)eta;
            a.status = h->d_status;
            a.node_graph = h->d_node_graph;
            a.graphs = h->num_graphs > 1 ? h->d_graphs : nullptr;
            a.alias = h->d_alias;
            a.energy = energy ? energy + ep : nullptr;
            a.pieces = h->d_act_pieces;
            const int red = h->opts.mode == SNAP_MODE_HOGWILD_RED;
            const int g = neg_samples <= 4 ? neg_samples : 5;   // the kernels' negative width
            const int gmax = energy ? h->grid_energy[red][g] : h->grid_oriented[red][g];
            if (gmax <= 0) return cudaErrorInvalidConfiguration;   // the caller sizes the grid first
            if (h->act_num_segs == 0) continue;
            const int grid = inflight_grid(h, gmax);
            {
                // lanes beyond the chunk count are idle
                const double lanes = (double)grid * h->block;
                const double segs = (double)h->act_num_segs;
                a.inflight_share = (float)((lanes < segs ? lanes : segs) / segs);
            }
            err = launch_oriented_epoch(a, red, grid > 0 ? grid : 1, h->block, stream);
        }
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

// Resident-block grid of the HOGWILD epoch kernel for k negatives (an
// occupancy query, cached per mode and negative group; kept outside any
// stream capture).
static void resident_grid(snap_layout *h, int32_t neg_samples) {
    const int red = h->opts.mode == SNAP_MODE_HOGWILD_RED;
    const int g = neg_samples <= 4 ? neg_samples : 5;   // the kernels' negative width
    if (h->grid_oriented[red][g] == 0)
        h->grid_oriented[red][g] =
            h->sms * oriented_blocks_per_sm(red, neg_samples, h->block, h->num_graphs > 1, h->d_alias != nullptr);
}

// A batch: every graph runs the call's schedule and seed from epoch 0 (the
// per-graph table is rewritten only when they change).
static cudaError_t set_batch_schedule(snap_layout *h, const snap_schedule &sc, uint64_t seed, cudaStream_t stream) {
    if (h->num_graphs <= 1) return cudaSuccess;
    if (h->graphs_set && h->graphs_seed == seed && memcmp(&h->graphs_sched, &sc, sizeof(sc)) == 0)
        return cudaSuccess;
    for (GraphInfo &gi : h->h_graphs) {
        gi.seed = seed;
        gi.start_tick = 0;
        gi.total_epochs = sc.kind == 1 ? INT32_MAX : sc.total_epochs;
        gi.eta0 = sc.eta0;
        gi.eta_min = sc.eta_min;
        gi.kind = sc.kind;
    }
    const cudaError_t err = cudaMemcpyAsync(h->d_graphs, h->h_graphs.data(), sizeof(GraphInfo) * h->h_graphs.size(),
                                            cudaMemcpyHostToDevice, stream);
    if (err != cudaSuccess) return err;
    h->graphs_set = true;
    h->graphs_sched = sc;
    h->graphs_seed = seed;
    return cudaSuccess;
}

static snap_status epochs_impl(snap_layout_t h, float *positions, int32_t epoch_begin, int32_t epochs,
                               int32_t neg_samples, const snap_schedule *schedule, uint64_t seed, double *energy,
                               void *cuda_stream) {
    NvtxRange nvtx_range("snap_layout_epochs");
    if (!h) return fail(SNAP_ERR_INVALID_ARG, "handle is NULL");
    if (!positions) return fail(SNAP_ERR_INVALID_ARG, "positions is NULL");
    if (((uintptr_t)positions & 7u) != 0) return fail(SNAP_ERR_INVALID_ARG, "positions must be 8-byte aligned");
    if (epochs < 0 || epoch_begin < 0) return fail(SNAP_ERR_INVALID_ARG, "epoch_begin and epochs must be >= 0");
    if (neg_samples < 0 || neg_samples > 64) return fail(SNAP_ERR_INVALID_ARG, "neg_samples = %d out of [0, 64]",
                                                         neg_samples);
    snap_status st = check_schedule(schedule);
    if (st != SNAP_OK) return st;
    st = poll_status(h);
    if (st != SNAP_OK) return st;
    if (energy && epochs > 0) {
        const cudaError_t e = cudaMemsetAsync(energy, 0, sizeof(double) * (size_t)epochs, (cudaStream_t)cuda_stream);
        if (e != cudaSuccess) return cuda_fail(e, "clear actual energy");
    }
    if (h->nnz == 0 || epochs == 0) return SNAP_OK;

    cudaStream_t stream = (cudaStream_t)cuda_stream;
    float2 *pos = reinterpret_cast<float2 *>(positions);
    cudaError_t err = cudaSuccess;
    err = set_batch_schedule(h, *schedule, seed, stream);
    if (err != cudaSuccess) return cuda_fail(err, "copy graph table");
    if (h->opts.mode != SNAP_MODE_SYNC) {
        // occupancy query outside any capture
        const int red = h->opts.mode == SNAP_MODE_HOGWILD_RED;
        const int g = neg_samples <= 4 ? neg_samples : 5;   // the kernels' negative width
        resident_grid(h, neg_samples);
        if (energy && h->grid_energy[red][g] == 0)
            h->grid_energy[red][g] =
                h->sms * oriented_energy_blocks_per_sm(red, neg_samples, h->block, h->d_alias != nullptr);
    }
    if ((h->opts.flags & SNAP_FLAG_CUDA_GRAPH) && epochs > 1 && !energy) {
        cudaGraphExec_t exec = nullptr;
        for (const CapturedEpochs &c : h->captured)
            if (c.pos == positions && c.epoch_begin == epoch_begin && c.epochs == epochs && c.k == neg_samples &&
                c.seed == seed && memcmp(&c.sched, schedule, sizeof(snap_schedule)) == 0)
                exec = c.exec;
        if (!exec) {
            if (!h->capture_stream) {
                err = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
                if (err != cudaSuccess) return cuda_fail(err, "capture stream");
            }
            // the capture stream must see the work already queued on the caller's stream
            cudaGraph_t graph = nullptr;
            err = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal);
            if (err == cudaSuccess) {
                const cudaError_t e2 = enqueue_epochs(h, pos, epoch_begin, epochs, neg_samples, *schedule, seed,
                                                      h->capture_stream);
                err = cudaStreamEndCapture(h->capture_stream, &graph);
                if (e2 != cudaSuccess) err = e2;
            }
            if (err == cudaSuccess) err = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (err != cudaSuccess) {
                cudaGetLastError();
                return cuda_fail(err, "epoch graph capture");
            }
            if (h->captured.size() >= 4) {
                cudaGraphExecDestroy(h->captured.front().exec);
                h->captured.erase(h->captured.begin());
            }
            h->captured.push_back(CapturedEpochs{positions, epoch_begin, epochs, neg_samples, seed, *schedule, exec});
        }
        err = cudaGraphLaunch(exec, stream);
        if (err != cudaSuccess) return cuda_fail(err, "epoch graph launch");
    } else {
        err = enqueue_epochs(h, pos, epoch_begin, epochs, neg_samples, *schedule, seed, stream, energy);
        if (err != cudaSuccess) return cuda_fail(err, "epoch launch");
    }
    if (!h->status_pending) {
        err = cudaMemcpyAsync(h->h_status, h->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream);
        if (err == cudaSuccess) err = cudaEventRecord(h->status_event, stream);
        if (err != cudaSuccess) return cuda_fail(err, "status read-back");
        h->status_pending = true;
    }
    h->mark_use(stream);
    return SNAP_OK;
}

snap_status snap_layout_epochs(snap_layout_t h, float *positions, int32_t epoch_begin, int32_t epochs,
                               int32_t neg_samples, const snap_schedule *schedule, uint64_t seed,
                               void *cuda_stream) {
    return epochs_impl(h, positions, epoch_begin, epochs, neg_samples, schedule, seed, nullptr, cuda_stream);
}

snap_status snap_layout_epochs_energy(snap_layout_t h, float *positions, int32_t epoch_begin, int32_t epochs,
                                      int32_t neg_samples, const snap_schedule *schedule, uint64_t seed,
                                      double *actual_energy, void *cuda_stream) {
    if (!h) return fail(SNAP_ERR_INVALID_ARG, "handle is NULL");
    if (!actual_energy || ((uintptr_t)actual_energy & 7u) != 0)
        return fail(SNAP_ERR_INVALID_ARG, "actual_energy must be a non-NULL 8-byte aligned device buffer");
    if (h->num_graphs > 1) return fail(SNAP_ERR_NOT_SUPPORTED, "the actual energy is reported for single graphs");
    return epochs_impl(h, positions, epoch_begin, epochs, neg_samples, schedule, seed, actual_energy, cuda_stream);
}

snap_status snap_layout_sync_chunks(snap_layout_t h, float *positions, int32_t epoch, int32_t chunk_begin,
                                    int32_t chunk_end, int32_t neg_samples, const snap_schedule *schedule,
                                    uint64_t seed, void *cuda_stream) {
    NvtxRange nvtx_range("snap_layout_sync_chunks");
    if (!h) return fail(SNAP_ERR_INVALID_ARG, "handle is NULL");
    if (h->opts.mode != SNAP_MODE_SYNC) return fail(SNAP_ERR_INVALID_ARG, "the handle is not in SNAP_MODE_SYNC");
    if (!positions) return fail(SNAP_ERR_INVALID_ARG, "positions is NULL");
    if (((uintptr_t)positions & 7u) != 0) return fail(SNAP_ERR_INVALID_ARG, "positions must be 8-byte aligned");
    if (epoch < 0) return fail(SNAP_ERR_INVALID_ARG, "epoch must be >= 0");
    if (chunk_begin < 0 || chunk_end > h->opts.sync_substeps || chunk_begin > chunk_end)
        return fail(SNAP_ERR_INVALID_ARG, "chunk range [%d, %d) outside [0, %d]", chunk_begin, chunk_end,
                    h->opts.sync_substeps);
    if (neg_samples < 0 || neg_samples > 64)
        return fail(SNAP_ERR_INVALID_ARG, "neg_samples = %d out of [0, 64]", neg_samples);
    snap_status st = check_schedule(schedule);
    if (st != SNAP_OK) return st;
    st = poll_status(h);
    if (st != SNAP_OK) return st;
    if (h->nnz == 0 || chunk_begin == chunk_end) return SNAP_OK;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    cudaError_t err = set_batch_schedule(h, *schedule, seed, stream);
    if (err != cudaSuccess) return cuda_fail(err, "copy graph table");
    err = enqueue_sync_chunks(h, reinterpret_cast<float2 *>(positions), epoch, chunk_begin, chunk_end, neg_samples,
                              *schedule, seed, stream, nullptr);
    if (err != cudaSuccess) return cuda_fail(err, "sync chunk launch");
    if (!h->status_pending) {
        err = cudaMemcpyAsync(h->h_status, h->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream);
        if (err == cudaSuccess) err = cudaEventRecord(h->status_event, stream);
        if (err != cudaSuccess) return cuda_fail(err, "status read-back");
        h->status_pending = true;
    }
    h->mark_use(stream);
    return SNAP_OK;
}

snap_status snap_layout_check(snap_layout_t h, void *cuda_stream) {
    if (!h) return fail(SNAP_ERR_INVALID_ARG, "handle is NULL");
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    cudaError_t err = cudaStreamSynchronize(stream);
    if (err != cudaSuccess) return cuda_fail(err, "stream synchronise");
    err = cudaMemcpy(h->h_status, h->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) return cuda_fail(err, "status read");
    h->status_pending = false;
    const uint32_t f = h->h_status[0];
    if (f) {
        h->h_status[0] = 0;
        cudaMemset(h->d_status, 0, sizeof(uint32_t));
        if (f & kStatusNonFinite) return fail(SNAP_ERR_NUMERIC, "a kernel produced a non-finite position");
        return fail(SNAP_ERR_NUMERIC, "a synchronous epoch clamped a fixed-point force term");
    }
    return SNAP_OK;
}

// Eq. 4 on the device: the attraction sum over the edges and the weighted
// repulsion sum (all pairs, per graph for a batch, or pair_samples sampled
// pairs).  Arguments are checked by the callers.  Synchronises the stream.
static snap_status objective_impl(snap_layout *h, const float2 *pos, int32_t neg_samples, int32_t exact,
                                  int64_t pair_samples, uint64_t seed, double *out_attr, double *out_rep,
                                  cudaStream_t stream) {
    cudaError_t err = cudaMemsetAsync(h->d_partial, 0, sizeof(double) * 2 * kObjGrid, stream);
    if (err == cudaSuccess && h->nnz > 0) {
        if (h->d_col)
            err = launch_objective_edges(h->d_row_ptr, h->d_col, h->d_seg_row, pos, h->nnz, h->seg_len,
                                         h->d_partial, kObjGrid, stream);
        else if (h->act_num_segs > 0)
            err = launch_objective_oriented(h->d_act_row_ptr, h->d_act_ent, h->d_act_meta, h->act_layout, h->act_nnz, pos,
                                            h->d_partial, kObjGrid, stream);
    }
    if (err == cudaSuccess && h->n > 1) {
        if (h->num_graphs > 1)
            err = launch_objective_pairs_batch(pos, h->d_deg, h->d_objw, h->d_node_graph, h->d_graphs, h->n,
                                               h->d_partial + kObjGrid, kObjGrid, stream);
        else if (exact)
            err = launch_objective_pairs_exact(pos, h->d_deg, h->d_objw, h->n, h->d_partial + kObjGrid, kObjGrid,
                                               stream);
        else
            err = launch_objective_pairs_sampled(pos, h->d_deg, h->d_objw, h->n, pair_samples, seed,
                                                 h->d_partial + kObjGrid, kObjGrid, stream);
    }
    std::vector<double> part(2 * (size_t)kObjGrid);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(part.data(), h->d_partial, sizeof(double) * 2 * kObjGrid, cudaMemcpyDeviceToHost,
                              stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
    if (err != cudaSuccess) return cuda_fail(err, "objective");
    h->mark_use(stream);
    double attr = 0.0, pairsum = 0.0;
    for (int b = 0; b < kObjGrid; ++b) attr += part[(size_t)b];
    for (int b = 0; b < kObjGrid; ++b) pairsum += part[(size_t)kObjGrid + b];
    double rep = 0.0;
    if (h->num_graphs > 1) {
        rep = (double)neg_samples * 0.5 * pairsum;   // per-graph weights applied on the device
    } else if (h->n > 1) {
        const double n = (double)h->n;
        // unordered-pair sum of coef_ij U^r; w_ij = coef / (2 (n-1)) (uniform) or c_ij / 2 (weighted)
        const double unordered = exact ? 0.5 * pairsum : pairsum / (double)pair_samples * 0.5 * n * (n - 1.0);
        rep = (double)neg_samples * unordered * (h->d_objw ? 0.5 : 1.0 / (2.0 * (n - 1.0)));
    }
    *out_attr = attr;
    *out_rep = rep;
    return SNAP_OK;
}

snap_status snap_layout_objective(snap_layout_t h, const float *positions, int32_t neg_samples, int32_t exact,
                                  int64_t pair_samples, uint64_t seed, double *out_attr, double *out_rep,
                                  double *out_total, void *cuda_stream) {
    NvtxRange nvtx_range("snap_layout_objective");
    if (!h) return fail(SNAP_ERR_INVALID_ARG, "handle is NULL");
    if (!positions) return fail(SNAP_ERR_INVALID_ARG, "positions is NULL");
    if (((uintptr_t)positions & 7u) != 0) return fail(SNAP_ERR_INVALID_ARG, "positions must be 8-byte aligned");
    if (neg_samples < 0) return fail(SNAP_ERR_INVALID_ARG, "neg_samples must be >= 0");
    if (!exact && pair_samples <= 0) return fail(SNAP_ERR_INVALID_ARG, "pair_samples must be > 0 when exact = 0");
    if (h->num_graphs > 1 && !exact)
        return fail(SNAP_ERR_NOT_SUPPORTED, "the sampled objective is not available for a batch (use exact = 1)");
    snap_status st = poll_status(h);
    if (st != SNAP_OK) return st;
    double attr = 0.0, rep = 0.0;
    st = objective_impl(h, reinterpret_cast<const float2 *>(positions), neg_samples, exact, pair_samples, seed,
                        &attr, &rep, (cudaStream_t)cuda_stream);
    if (st != SNAP_OK) return st;
    if (out_attr) *out_attr = attr;
    if (out_rep) *out_rep = rep;
    if (out_total) *out_total = attr + rep;
    return SNAP_OK;
}

int64_t snap_layout_device_bytes(snap_layout_t h) { return h ? h->device_bytes : 0; }

snap_status snap_memory_cached(int32_t device, uint64_t *bytes) {
    if (!bytes) return fail(SNAP_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = 0;
    if (device < 0) return fail(SNAP_ERR_INVALID_ARG, "device %d < 0", device);
    cudaMemPool_t pool = library_pool(device, false);
    if (!pool) return SNAP_OK;   // nothing allocated on that device yet
    uint64_t reserved = 0, used = 0;
    cudaError_t err = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
    if (err == cudaSuccess) err = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
    if (err != cudaSuccess) return cuda_fail(err, "memory pool attributes");
    *bytes = reserved > used ? reserved - used : 0;
    return SNAP_OK;
}

snap_status snap_memory_trim(int32_t device, uint64_t keep_bytes) {
    if (device < 0) return fail(SNAP_ERR_INVALID_ARG, "device %d < 0", device);
    cudaMemPool_t pool = library_pool(device, false);
    if (!pool) return SNAP_OK;
    const cudaError_t err = cudaMemPoolTrimTo(pool, (size_t)keep_bytes);
    if (err != cudaSuccess) return cuda_fail(err, "memory pool trim");
    return SNAP_OK;
}

// One candidate configuration of the autotuner.
struct TuneCandidate {
    int32_t target, block, order;
    double ms;
};

// Puts a (chunk size, block, row order) configuration on the handle.
static cudaError_t apply_config(snap_layout *h, AllocCounter &ac, int32_t target, int32_t block, int32_t order,
                                cudaStream_t stream) {
    if (target != h->act_seg_len || order != h->act_layout.order) {
        const cudaError_t err = set_chunks(h, ac, target, order, stream);
        if (err != cudaSuccess) return err;
    }
    h->block = block;
    for (auto &row : h->grid_oriented)
        for (int &v : row) v = 0;
    for (auto &row : h->grid_energy)
        for (int &v : row) v = 0;
    for (const CapturedEpochs &c : h->captured) cudaGraphExecDestroy(c.exec);
    h->captured.clear();
    return cudaSuccess;
}

// Neighbourhood preservation (Section 4.1, r = 2) of a layout on sampled
// vertices, from the CSR the handle keeps (SYNC handles, or HOGWILD handles
// created with SNAP_FLAG_KEEP_CSR).  *mean: the mean over the samples that
// have neighbours, *used: their number.
static snap_status np_impl(snap_layout *h, const float2 *pos, const int32_t *nodes, int32_t count, double *mean,
                           int32_t *used, cudaStream_t stream) {
    if (!h->d_row_ptr || !h->d_col)
        return fail(SNAP_ERR_NOT_SUPPORTED, "the handle does not keep its CSR (create it with SNAP_FLAG_KEEP_CSR)");
    int32_t max_graph = h->n;
    if (h->num_graphs > 1) {
        max_graph = 0;
        for (const GraphInfo &gi : h->h_graphs) max_graph = gi.n > max_graph ? gi.n : max_graph;
    }
    for (int32_t q = 0; q < count; ++q)
        if (nodes[q] < 0 || nodes[q] >= h->n) return fail(SNAP_ERR_INVALID_ARG, "sample %d outside [0, n)", q);
    *mean = 0.0;
    *used = 0;
    if (count == 0) return SNAP_OK;
    AllocCounter ac;
    int32_t *d_nodes = nullptr;
    double *d_out = nullptr;
    uint32_t *d_bits = nullptr;
    int grid = h->sms * 8;
    int64_t words = 0;
    cudaError_t err = dev_alloc(ac, (void **)&d_nodes, sizeof(int32_t) * (size_t)count, stream);
    if (err == cudaSuccess) err = dev_alloc(ac, (void **)&d_out, sizeof(double) * (size_t)count, stream);
    if (err == cudaSuccess && max_graph > kNpMaxGraph) {
        // 2-hop bitmaps and candidate lists in global scratch, one of each per block,
        // at most 1 GiB in all
        words = ((int64_t)max_graph + 31) / 32;
        int64_t g = (int64_t)h->sms * 2;
        const int64_t per_block = (words + 1 + 3 * kNpCandidates) * (int64_t)sizeof(uint32_t);
        const int64_t cap = ((int64_t)1 << 30) / per_block;
        if (g > cap) g = cap;
        if (g > count) g = count;
        grid = (int)(g > 0 ? g : 1);
        err = dev_alloc(ac, (void **)&d_bits, sizeof(uint32_t) * (size_t)np_scratch_words(words, grid), stream);
    }
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(d_nodes, nodes, sizeof(int32_t) * (size_t)count, cudaMemcpyHostToDevice, stream);
    if (err == cudaSuccess)
        err = launch_np_samples(h->d_row_ptr, h->d_col, pos, d_nodes, count, h->d_node_graph,
                                h->num_graphs > 1 ? h->d_graphs : nullptr, h->n, max_graph, d_out, grid, d_bits, words,
                                stream);
    std::vector<double> out((size_t)count, 0.0);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(out.data(), d_out, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
    if (d_nodes) cudaFreeAsync(d_nodes, stream);
    if (d_out) cudaFreeAsync(d_out, stream);
    if (d_bits) cudaFreeAsync(d_bits, stream);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return err == cudaErrorMemoryAllocation ? fail(SNAP_ERR_OUT_OF_MEMORY, "NP scratch")
                                                : cuda_fail(err, "neighbourhood preservation");
    }
    double sum = 0.0;
    int32_t u = 0;
    for (double v : out)
        if (v >= 0.0) {
            sum += v;
            ++u;
        }
    *mean = u > 0 ? sum / u : 0.0;
    *used = u;
    return SNAP_OK;
}

snap_status snap_layout_neighborhood_preservation(snap_layout_t h, const float *positions, const int32_t *nodes,
                                                  int32_t count, double *out_mean, int32_t *out_used,
                                                  void *cuda_stream) {
    NvtxRange nvtx_range("snap_layout_neighborhood_preservation");
    if (!h) return fail(SNAP_ERR_INVALID_ARG, "handle is NULL");
    if (!positions || ((uintptr_t)positions & 7u) != 0)
        return fail(SNAP_ERR_INVALID_ARG, "positions must be a non-NULL 8-byte aligned device buffer");
    if (count < 0 || (count > 0 && !nodes)) return fail(SNAP_ERR_INVALID_ARG, "bad sample list");
    if (!out_mean) return fail(SNAP_ERR_INVALID_ARG, "out_mean is NULL");
    snap_status st = poll_status(h);
    if (st != SNAP_OK) return st;
    int32_t used = 0;
    st = np_impl(h, reinterpret_cast<const float2 *>(positions), nodes, count, out_mean, &used,
                 (cudaStream_t)cuda_stream);
    if (st == SNAP_OK && out_used) *out_used = used;
    if (st == SNAP_OK) h->mark_use((cudaStream_t)cuda_stream);
    return st;
}

snap_status snap_layout_autotune(snap_layout_t h, const float *initial_positions, float *scratch_positions,
                                 int32_t neg_samples, const snap_schedule *schedule, uint64_t seed, double tolerance,
                                 int32_t *chosen_segment, int32_t *chosen_block, int32_t *chosen_row_order,
                                 double *chosen_ms, double *chosen_objective, double *chosen_np,
                                 void *cuda_stream) {
    NvtxRange nvtx_range("snap_layout_autotune");
    if (!h) return fail(SNAP_ERR_INVALID_ARG, "handle is NULL");
    if (h->opts.mode == SNAP_MODE_SYNC) return fail(SNAP_ERR_NOT_SUPPORTED, "autotuning applies to the HOGWILD modes");
    if (!scratch_positions || ((uintptr_t)scratch_positions & 7u) != 0)
        return fail(SNAP_ERR_INVALID_ARG, "scratch_positions must be a non-NULL 8-byte aligned device buffer");
    const bool gate = tolerance >= 0.0;
    if (gate && (!initial_positions || ((uintptr_t)initial_positions & 7u) != 0))
        return fail(SNAP_ERR_INVALID_ARG, "initial_positions must be a non-NULL 8-byte aligned device buffer");
    if (gate && !std::isfinite(tolerance)) return fail(SNAP_ERR_INVALID_ARG, "tolerance must be finite");
    if (neg_samples < 0 || neg_samples > 64) return fail(SNAP_ERR_INVALID_ARG, "neg_samples out of [0, 64]");
    snap_status st = check_schedule(schedule);
    if (st != SNAP_OK) return st;
    st = poll_status(h);
    if (st != SNAP_OK) return st;
    if (h->act_nnz == 0) return fail(SNAP_ERR_INVALID_ARG, "the graph has no edges");
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    float2 *scratch = reinterpret_cast<float2 *>(scratch_positions);
    const size_t pos_bytes = sizeof(float2) * (size_t)h->n;
    const snap_schedule sched = *schedule;
    const int32_t gate_epochs = sched.total_epochs;

    // the configuration at entry is always a candidate and the gate's reference
    const int32_t entry_order = h->act_layout.order;
    std::vector<TuneCandidate> cand{{h->act_seg_len, h->block, entry_order, 0.0}};
    for (int32_t order : {0, 1})
        for (int32_t target : {4, 8, 16, 32})
            for (int32_t block : {128, 256})
                if (target != h->act_seg_len || block != h->block || order != entry_order)
                    cand.push_back({target, block, order, 0.0});

    cudaEvent_t e0 = nullptr, e1 = nullptr;
    AllocCounter ac;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err == cudaSuccess) err = set_batch_schedule(h, sched, seed, stream);
    // timing: per candidate the schedule's epoch 0 untimed and epochs 1-3
    // timed; two passes over the candidates, the faster pass counts
    for (TuneCandidate &c : cand) c.ms = 1e300;
    for (int pass = 0; pass < 2 && err == cudaSuccess; ++pass) {
        for (TuneCandidate &c : cand) {
            err = apply_config(h, ac, c.target, c.block, c.order, stream);
            if (err == cudaSuccess) resident_grid(h, neg_samples);
            if (err == cudaSuccess && gate)
                err = cudaMemcpyAsync(scratch, initial_positions, pos_bytes, cudaMemcpyDeviceToDevice, stream);
            if (err == cudaSuccess) err = enqueue_epochs(h, scratch, 0, 1, neg_samples, sched, seed, stream);
            if (err == cudaSuccess) err = cudaEventRecord(e0, stream);
            if (err == cudaSuccess) err = enqueue_epochs(h, scratch, 1, 3, neg_samples, sched, seed, stream);
            if (err == cudaSuccess) err = cudaEventRecord(e1, stream);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (err != cudaSuccess) break;
            c.ms = std::min(c.ms, ms / 3.0);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (err != cudaSuccess) {
        cudaGetLastError();
        apply_config(h, ac, cand.front().target, cand.front().block, cand.front().order, stream);
        return cuda_fail(err, "autotune timing");
    }
    // a candidate replaces the entry configuration only if it is at least 3%
    // faster (the timing's run-to-run spread is about 1-2%)
    const TuneCandidate entry = cand.front();
    cand.erase(std::remove_if(cand.begin() + 1, cand.end(),
                              [&](const TuneCandidate &c) { return c.ms > 0.97 * entry.ms; }),
               cand.end());
    std::stable_sort(cand.begin(), cand.end(),
                     [](const TuneCandidate &x, const TuneCandidate &y) { return x.ms < y.ms; });

    // quality gate: a candidate faster than the entry configuration is kept
    // only if its layout's Eq. 4 objective (same initial positions, schedule
    // and seed; exact for batches and small graphs, else the same sampled
    // pairs) is within (1 + tolerance) of the entry configuration's
    const bool exact = h->num_graphs > 1 || h->n <= 16384;
    const int64_t pairs = 16 << 20;
    const uint64_t pair_seed = seed ^ 0x5bd1e9955bd1e995ull;
    // NP half of the gate (Section 4.1, r = 2) when the handle keeps its CSR
    // and every graph fits the device NP kernel: 1,024 vertices drawn from
    // the seed, the same for every candidate
    bool np_on = gate && h->d_row_ptr && h->d_col;
    if (np_on) {
        int32_t max_graph = h->n;
        if (h->num_graphs > 1) {
            max_graph = 0;
            for (const GraphInfo &gi : h->h_graphs) max_graph = gi.n > max_graph ? gi.n : max_graph;
        }
        np_on = max_graph <= kNpMaxGraph;
    }
    std::vector<int32_t> np_nodes;
    if (np_on) {
        np_nodes.resize(1024);
        for (size_t q = 0; q < np_nodes.size(); ++q)
            np_nodes[q] = (int32_t)(mix64(seed ^ (0x4E50ull << 32) ^ (uint64_t)q) % (uint64_t)h->n);
    }
    auto layout_np = [&](double *npv) -> snap_status {
        int32_t used = 0;
        return np_impl(h, scratch, np_nodes.data(), (int32_t)np_nodes.size(), npv, &used, stream);
    };
    auto layout_objective = [&](const TuneCandidate &c, double *u) -> snap_status {
        cudaError_t e = apply_config(h, ac, c.target, c.block, c.order, stream);
        if (e == cudaSuccess) resident_grid(h, neg_samples);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(scratch, initial_positions, pos_bytes, cudaMemcpyDeviceToDevice, stream);
        if (e == cudaSuccess) e = enqueue_epochs(h, scratch, 0, gate_epochs, neg_samples, sched, seed, stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_fail(e, "autotune layout");
        }
        snap_status s2 = snap_layout_check(h, cuda_stream);
        if (s2 != SNAP_OK) return s2;
        double attr = 0.0, rep = 0.0;
        s2 = objective_impl(h, scratch, neg_samples, exact ? 1 : 0, pairs, pair_seed, &attr, &rep, stream);
        *u = attr + rep;
        return s2;
    };
    TuneCandidate best = cand.front();
    double best_u = NAN, best_np = NAN;
    auto same = [](const TuneCandidate &x, const TuneCandidate &y) {
        return x.target == y.target && x.block == y.block && x.order == y.order;
    };
    if (gate && !same(best, entry)) {
        double u_ref = 0.0, np_ref = NAN;
        st = layout_objective(entry, &u_ref);
        if (st == SNAP_OK && np_on) st = layout_np(&np_ref);
        for (const TuneCandidate &c : cand) {
            if (st != SNAP_OK) break;
            if (same(c, entry)) {
                best = c;
                best_u = u_ref;
                best_np = np_ref;
                break;
            }
            double u = 0.0, npv = NAN;
            st = layout_objective(c, &u);
            bool pass = st == SNAP_OK && std::isfinite(u) && u <= u_ref * (1.0 + tolerance);
            if (pass && np_on) {
                st = layout_np(&npv);
                pass = st == SNAP_OK && npv >= np_ref * (1.0 - tolerance);
            }
            if (pass) {
                best = c;
                best_u = u;
                best_np = npv;
                break;
            }
            if (st == SNAP_ERR_NUMERIC) st = SNAP_OK;   // a candidate that diverged is rejected
        }
        if (st != SNAP_OK) {
            apply_config(h, ac, entry.target, entry.block, entry.order, stream);
            return st;
        }
    } else if (gate) {
        st = layout_objective(best, &best_u);
        if (st == SNAP_OK && np_on) st = layout_np(&best_np);
        if (st != SNAP_OK) return st;
    }
    err = apply_config(h, ac, best.target, best.block, best.order, stream);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(err, "autotune");
    }
    h->mark_use(stream);
    if (chosen_segment) *chosen_segment = h->act_seg_len;
    if (chosen_block) *chosen_block = h->block;
    if (chosen_row_order) *chosen_row_order = h->act_layout.order;
    if (chosen_ms) *chosen_ms = best.ms;
    if (chosen_objective) *chosen_objective = best_u;
    if (chosen_np) *chosen_np = best_np;
    return snap_layout_check(h, cuda_stream);
}

void snap_layout_destroy(snap_layout_t h) {
    if (!h) return;
    h->release();
    delete h;
}

snap_status snap_layout_run(const int64_t *row_ptr, const int32_t *col_idx, int32_t n, const snap_options *opts,
                            float *positions_host, int32_t epochs, int32_t neg_samples, const snap_schedule *schedule,
                            uint64_t seed, void *cuda_stream) {
    NvtxRange nvtx_range("snap_layout_run");
    if (!positions_host) return fail(SNAP_ERR_INVALID_ARG, "positions_host is NULL");
    snap_status st = check_schedule(schedule);
    if (st != SNAP_OK) return st;
    snap_layout_t h = nullptr;
    g_alloc.reset();
    g_in_run = true;
    st = snap_layout_create(row_ptr, col_idx, nullptr, n, opts, cuda_stream, &h);
    g_in_run = false;
    if (st != SNAP_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    float *d_pos = nullptr;
    const size_t bytes = sizeof(float) * 2 * (size_t)n;
    cudaError_t err = dev_alloc(g_alloc, (void **)&d_pos, bytes, stream);
    if (err != cudaSuccess) {
        cudaGetLastError();
        snap_layout_destroy(h);
        return cuda_fail(err, "device allocation of positions");
    }
    err = cudaMemcpyAsync(d_pos, positions_host, bytes, cudaMemcpyHostToDevice, stream);
    if (err != cudaSuccess) {
        cudaFreeAsync(d_pos, stream);
        snap_layout_destroy(h);
        return cuda_fail(err, "copy positions to the device");
    }
    st = snap_layout_epochs(h, d_pos, 0, epochs, neg_samples, schedule, seed, cuda_stream);
    if (st == SNAP_OK) st = snap_layout_check(h, cuda_stream);
    if (st == SNAP_OK) {
        err = cudaMemcpyAsync(positions_host, d_pos, bytes, cudaMemcpyDeviceToHost, stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
        if (err != cudaSuccess) st = cuda_fail(err, "copy positions to the host");
    }
    cudaFreeAsync(d_pos, stream);
    snap_layout_destroy(h);
    return st;
}

// ---------------------------------------------------------------------------
// Multi-handle epochs (continuous batching)
// ---------------------------------------------------------------------------
}  // extern "C"

struct snap_multi {
    int32_t capacity = 0;
    JobDesc *d_jobs = nullptr;
    JobDesc *h_jobs = nullptr;      // pinned staging of the job table
    uint32_t *d_status = nullptr;
    uint32_t *h_status = nullptr;   // pinned
    cudaEvent_t copied = nullptr;
    bool copy_pending = false;
    int sms = 1;
    int grid[2][2][6] = {{{0}}};   // [red][weighted][negative width: k if k <= 4, else 5], filled on first use
    uint64_t calls = 0;

    void release() {
        cudaFree(d_jobs);
        cudaFree(d_status);
        if (h_jobs) cudaFreeHost(h_jobs);
        if (h_status) cudaFreeHost(h_status);
        if (copied) cudaEventDestroy(copied);
        d_jobs = nullptr;
        d_status = nullptr;
        h_jobs = nullptr;
        h_status = nullptr;
        copied = nullptr;
    }
};

extern "C" {

snap_status snap_multi_create(int32_t max_jobs, snap_multi_t *out) {
    if (!out) return fail(SNAP_ERR_INVALID_ARG, "out is NULL");
    if (max_jobs < 1 || max_jobs > (1 << 20)) return fail(SNAP_ERR_INVALID_ARG, "max_jobs out of [1, 2^20]");
    snap_multi *m = new (std::nothrow) snap_multi();
    if (!m) return fail(SNAP_ERR_OUT_OF_MEMORY, "host allocation failed");
    m->capacity = max_jobs;
    cudaError_t err = cudaMalloc((void **)&m->d_jobs, sizeof(JobDesc) * (size_t)max_jobs);
    if (err == cudaSuccess) err = cudaMalloc((void **)&m->d_status, sizeof(uint32_t) * 4);
    if (err == cudaSuccess) err = cudaMallocHost((void **)&m->h_jobs, sizeof(JobDesc) * (size_t)max_jobs);
    if (err == cudaSuccess) err = cudaMallocHost((void **)&m->h_status, sizeof(uint32_t) * 4);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&m->copied, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaMemset(m->d_status, 0, sizeof(uint32_t) * 4);
    int dev = 0;
    if (err == cudaSuccess) err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) {
        m->release();
        delete m;
        cudaGetLastError();
        return cuda_fail(err, "snap_multi_create");
    }
    *out = m;
    return SNAP_OK;
}

snap_status snap_multi_epoch(snap_multi_t m, const snap_layout_t *handles, float *const *positions,
                             const int32_t *epochs, const snap_schedule *schedules, const uint64_t *seeds,
                             int32_t count, int32_t neg_samples, void *cuda_stream) {
    NvtxRange nvtx_range("snap_multi_epoch");
    if (!m || !handles || !positions || !epochs || !schedules || !seeds)
        return fail(SNAP_ERR_INVALID_ARG, "NULL argument");
    if (count < 0 || count > m->capacity) return fail(SNAP_ERR_INVALID_ARG, "count = %d out of [0, %d]", count,
                                                      m->capacity);
    if (neg_samples < 0 || neg_samples > 64) return fail(SNAP_ERR_INVALID_ARG, "neg_samples out of [0, 64]");
    int red = -1;
    for (int32_t q = 0; q < count; ++q) {
        const snap_layout *h = handles[q];
        if (!h) return fail(SNAP_ERR_INVALID_ARG, "handle %d is NULL", q);
        if (h->opts.mode == SNAP_MODE_SYNC || h->num_graphs > 1)
            return fail(SNAP_ERR_NOT_SUPPORTED, "handle %d: multi-handle epochs take single-graph HOGWILD handles", q);
        const int r = h->opts.mode == SNAP_MODE_HOGWILD_RED;
        if (red >= 0 && r != red) return fail(SNAP_ERR_INVALID_ARG, "handles mix HOGWILD and HOGWILD_RED");
        red = r;
        if (!positions[q] || ((uintptr_t)positions[q] & 7u) != 0)
            return fail(SNAP_ERR_INVALID_ARG, "positions[%d] is NULL or misaligned", q);
        if (epochs[q] < 0) return fail(SNAP_ERR_INVALID_ARG, "epochs[%d] < 0", q);
        const snap_status st = check_schedule(&schedules[q]);
        if (st != SNAP_OK) return st;
    }
    if (m->copy_pending) {
        // the staging buffer may be rewritten once the previous table reached the device
        const cudaError_t e = cudaEventSynchronize(m->copied);
        if (e != cudaSuccess) return cuda_fail(e, "multi staging");
        m->copy_pending = false;
    }
    int64_t total = 0;
    int32_t used = 0;
    uint64_t mixkey = 0x243F6A8885A308D3ull ^ ++m->calls;
    for (int32_t q = 0; q < count; ++q) {
        const snap_layout *h = handles[q];
        if (h->act_num_segs == 0) continue;
        JobDesc &jd = m->h_jobs[used++];
        jd.row_ptr = h->d_act_row_ptr;
        jd.ent = h->d_act_ent;
        jd.meta = h->d_act_meta;
        jd.pos = reinterpret_cast<float2 *>(positions[q]);
        jd.num_segs = h->act_num_segs;
        jd.nnz = h->act_nnz;
        jd.seg_len = h->act_seg_len;
        jd.alias = h->d_alias;
        jd.pieces = h->d_act_pieces;
        jd.seg_prefix = total;
        jd.seed = seeds[q];
        jd.n = h->n;
        jd.epoch = (uint32_t)epochs[q];
        jd.eta = (float)step_size(schedules[q], epochs[q]);
        total += h->act_num_segs;
        mixkey = mix64(mixkey ^ seeds[q] ^ ((uint64_t)epochs[q] << 32));
    }
    if (used == 0 || red < 0) return SNAP_OK;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    cudaError_t err = cudaMemcpyAsync(m->d_jobs, m->h_jobs, sizeof(JobDesc) * (size_t)used, cudaMemcpyHostToDevice,
                                      stream);
    if (err == cudaSuccess) err = cudaEventRecord(m->copied, stream);
    if (err != cudaSuccess) return cuda_fail(err, "copy job table");
    m->copy_pending = true;
    MultiArgs a;
    a.jobs = m->d_jobs;
    a.num_jobs = used;
    a.k = neg_samples;
    a.total_segs = total;
    const int64_t groups = (total + 31) / 32;
    a.perm_mul = golden_multiplier(groups);
    a.perm_add = (int64_t)(mixkey % (uint64_t)groups);
    a.status = m->d_status;
    const int g = neg_samples <= 4 ? neg_samples : 5;   // the kernels' negative width
    int weighted = 0;
    for (int32_t q = 0; q < used; ++q) weighted |= m->h_jobs[q].alias != nullptr;
    if (m->grid[red][weighted][g] == 0)
        m->grid[red][weighted][g] = m->sms * multi_blocks_per_sm(red, weighted, neg_samples, 256);
    // at most the default share of the jobs' entries in flight (as inflight_grid does for one handle)
    int64_t entries = 0;
    for (int32_t q = 0; q < count; ++q) entries += handles[q]->act_nnz;
    const int64_t want = (total + 255) / 256;
    int64_t gcap = ((int64_t)(default_inflight(red) * (double)entries) + 255) / 256;
    int64_t gl = want < m->grid[red][weighted][g] ? want : m->grid[red][weighted][g];
    if (gcap < gl) gl = gcap;
    const int grid = (int)(gl > 0 ? gl : 1);
    a.inflight_share = (float)(((double)grid * 256.0 < (double)total ? (double)grid * 256.0 : (double)total) /
                               (double)total);
    err = launch_multi_epoch(a, red, weighted, grid > 0 ? grid : 1, 256, stream);
    if (err != cudaSuccess) return cuda_fail(err, "multi-handle epoch launch");
    for (int32_t q = 0; q < count; ++q) handles[q]->mark_use(stream);
    return SNAP_OK;
}

snap_status snap_multi_check(snap_multi_t m, void *cuda_stream) {
    if (!m) return fail(SNAP_ERR_INVALID_ARG, "NULL argument");
    cudaError_t err = cudaStreamSynchronize((cudaStream_t)cuda_stream);
    if (err == cudaSuccess) err = cudaMemcpy(m->h_status, m->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) return cuda_fail(err, "multi check");
    if (m->h_status[0]) {
        cudaMemset(m->d_status, 0, sizeof(uint32_t));
        return fail(SNAP_ERR_NUMERIC, "a multi-handle epoch produced a non-finite position");
    }
    return SNAP_OK;
}

void snap_multi_destroy(snap_multi_t m) {
    if (!m) return;
    if (m->copy_pending) cudaEventSynchronize(m->copied);
    m->release();
    delete m;
}

}  // extern "C"
