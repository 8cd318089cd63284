// capi.cu -- the C ABI declared in include/snap_layout.h: handle life cycle,
// argument checking, launch configuration and error reporting.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/snap_layout.h"
#include "snap_internal.h"

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
thread_local bool g_in_run = false;

cudaError_t dev_alloc(AllocCounter &ac, void **p, size_t bytes) {
    ++ac.count;
    if (ac.fail_at > 0 && ac.count == ac.fail_at) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes < 16 ? 16 : bytes);
}

// SplitMix64 finaliser (Steele, Lea, Flood 2014): the per-epoch offset of
// the segment order.
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
    // whole rows packed into segments of about act_seg_len entries
    int64_t act_nnz = 0;
    int64_t act_num_segs = 0;
    int32_t act_seg_len = 32;
    int64_t perm_mul = 1;
    int64_t *d_act_row_ptr = nullptr;
    int4 *d_act_ent = nullptr;
    int4 *d_act_seg = nullptr;
    uint32_t *d_status = nullptr;   // [0] fault bits, [1] validation bits
    double *d_partial = nullptr;    // 2 * kObjGrid
    uint32_t *h_status = nullptr;   // pinned mirror of d_status[0]
    cudaEvent_t status_event = nullptr;
    bool status_pending = false;
    int sms = 1;
    int grid_sync = 0, grid_apply = 0;
    int grid_oriented[2][5] = {{0}};   // [red][min(k, 4)], filled on first use
    std::vector<int64_t> chunk_edges;   // S + 1 edge offsets of the sync chunks
    int64_t device_bytes = 0;

    void release_csr() {
        cudaFree(d_row_ptr);
        cudaFree(d_col);
        cudaFree(d_seg_row);
        d_row_ptr = nullptr;
        d_col = nullptr;
        d_seg_row = nullptr;
    }

    void release() {
        release_csr();
        cudaFree(d_act_row_ptr);
        cudaFree(d_act_ent);
        cudaFree(d_act_seg);
        d_act_row_ptr = nullptr;
        d_act_ent = nullptr;
        d_act_seg = nullptr;
        cudaFree(d_deg);
        cudaFree(d_disp);
        cudaFree(d_status);
        cudaFree(d_partial);
        if (h_status) cudaFreeHost(h_status);
        if (status_event) cudaEventDestroy(status_event);
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

// Segments of the oriented list: whole rows packed greedily up to `target`
// entries; a row longer than `target` is cut into equal pieces.
static void pack_segments(const std::vector<int64_t> &rp, int32_t target, std::vector<int4> &out) {
    out.clear();
    const int32_t n = (int32_t)rp.size() - 1;
    int64_t open_begin = -1, open_end = 0;
    int32_t open_row = 0;
    auto close = [&]() {
        if (open_begin >= 0) out.push_back(make_int4((int)open_begin, (int)open_end, open_row, 1));
        open_begin = -1;
    };
    for (int32_t i = 0; i < n; ++i) {
        const int64_t len = rp[(size_t)i + 1] - rp[(size_t)i];
        if (len == 0) continue;
        if (len > target) {
            close();
            const int64_t pieces = (len + target - 1) / target;
            for (int64_t q = 0; q < pieces; ++q) {
                const int64_t b = rp[(size_t)i] + len * q / pieces;
                const int64_t e = rp[(size_t)i] + len * (q + 1) / pieces;
                out.push_back(make_int4((int)b, (int)e, i, (int)pieces));
            }
            continue;
        }
        if (open_begin >= 0 && open_end - open_begin + len > target) close();
        if (open_begin < 0) {
            open_begin = rp[(size_t)i];
            open_row = i;
        }
        open_end = rp[(size_t)i + 1];
    }
    close();
}

// Builds the oriented bundle list from the validated device CSR and then
// frees the CSR (the HOGWILD kernels and the objective need only the list).
static snap_status build_oriented(snap_layout *h, AllocCounter &ac, cudaStream_t stream) {
    const int32_t n = h->n;
    const int64_t nnz = h->nnz;
    h->act_nnz = nnz / 2;   // symmetric and loop-free: each undirected edge once
    if (h->act_seg_len == 0) {
        // Default segment size.  Concurrency degrades Hogwild quality when a
        // large share of the graph is in flight at once, so graphs that fill
        // the device's lanes (about 512 per SM) fewer than four times over at
        // 32 entries per segment get 128-entry segments; larger graphs get 32
        // (shorter tails, same quality: their in-flight share is small).
        const int64_t lanes = (int64_t)h->sms * 512;
        h->act_seg_len = h->act_nnz >= 4 * 32 * lanes ? 32 : 128;
    }
    int32_t *flags = nullptr, *pos = nullptr;
    void *temp = nullptr;
    size_t temp_bytes = 0;
    cudaError_t err = cudaSuccess;
    const char *what = "";
    auto alloc = [&](void **p, size_t bytes, bool keep, const char *nm) {
        if (err != cudaSuccess) return;
        err = dev_alloc(ac, p, bytes);
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
    alloc((void **)&h->d_act_ent, sizeof(int4) * (size_t)(h->act_nnz > 0 ? h->act_nnz : 1), true, "oriented entries");
    alloc((void **)&flags, sizeof(int32_t) * ((size_t)nnz + 1), false, "orientation flags");
    alloc((void **)&pos, sizeof(int32_t) * ((size_t)nnz + 1), false, "orientation offsets");
    if (err == cudaSuccess) step(exclusive_scan_i32(nullptr, &temp_bytes, flags, pos, nnz + 1, stream), "scan size");
    alloc(&temp, temp_bytes, false, "scan scratch");
    if (err == cudaSuccess) {
        step(launch_orient_flags(h->d_row_ptr, h->d_col, h->d_seg_row, h->d_deg, nnz, h->seg_len, flags, stream),
             "orientation flags kernel");
        step(exclusive_scan_i32(temp, &temp_bytes, flags, pos, nnz + 1, stream), "orientation scan");
        step(launch_orient_scatter(h->d_row_ptr, h->d_col, h->d_seg_row, h->d_deg, nnz, h->seg_len, pos,
                                   h->d_act_ent, stream), "orientation scatter kernel");
        step(launch_orient_rowptr(h->d_row_ptr, pos, n, h->d_act_row_ptr, stream), "orientation offsets kernel");
    }
    std::vector<int64_t> act_rp;
    if (err == cudaSuccess) {
        act_rp.resize((size_t)n + 1);
        step(cudaMemcpyAsync(act_rp.data(), h->d_act_row_ptr, sizeof(int64_t) * ((size_t)n + 1),
                             cudaMemcpyDeviceToHost, stream), "read oriented row offsets");
        step(cudaStreamSynchronize(stream), "orientation");
    }
    cudaFree(flags);
    cudaFree(pos);
    cudaFree(temp);
    if (err != cudaSuccess) return cuda_fail(err, what);
    if (act_rp[(size_t)n] != h->act_nnz)
        return fail(SNAP_ERR_CUDA, "orientation produced %lld entries, expected %lld", (long long)act_rp[(size_t)n],
                    (long long)h->act_nnz);
    std::vector<int4> segs;
    pack_segments(act_rp, h->act_seg_len, segs);
    h->act_num_segs = (int64_t)segs.size();
    alloc((void **)&h->d_act_seg, sizeof(int4) * (segs.empty() ? 1 : segs.size()), true, "oriented segments");
    if (err == cudaSuccess && !segs.empty()) {
        step(cudaMemcpyAsync(h->d_act_seg, segs.data(), sizeof(int4) * segs.size(), cudaMemcpyHostToDevice, stream),
             "copy oriented segments");
        step(cudaStreamSynchronize(stream), "copy oriented segments");
    }
    if (err != cudaSuccess) return cuda_fail(err, what);
    // segment order multiplier: coprime with the segment count, near its golden section
    int64_t m = (int64_t)(0.6180339887498949 * (double)h->act_num_segs) | 1;
    while (h->act_num_segs > 1 && gcd64(m, h->act_num_segs) != 1) m += 2;
    h->perm_mul = h->act_num_segs > 1 ? m % h->act_num_segs : 0;
    if (h->act_num_segs > 1 && h->perm_mul == 0) h->perm_mul = 1;
    h->device_bytes -= (int64_t)(sizeof(int64_t) * ((size_t)n + 1) +
                                 sizeof(int32_t) * (size_t)(h->num_segs * h->seg_len + 4) +
                                 sizeof(int32_t) * (size_t)(h->num_segs > 0 ? h->num_segs : 1));
    h->release_csr();
    return SNAP_OK;
}

extern "C" {

void snap_options_default(snap_options *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->mode = SNAP_MODE_HOGWILD;
    o->sampler = SNAP_SAMPLER_UNIFORM;
    o->node_weights = nullptr;
    o->sync_substeps = 1;
    o->sync_cap = 0.0f;
    o->segment_edges = 0;
    o->block_threads = 0;
}

const char *snap_last_error(void) { return g_last_error.c_str(); }

static snap_status check_csr_host(const int64_t *row_ptr, const int32_t *col_idx, const int32_t *degrees,
                                  int32_t n) {
    if (!row_ptr) return fail(SNAP_ERR_INVALID_ARG, "row_ptr is NULL");
    if (n < 1 || n == INT32_MAX) return fail(SNAP_ERR_INVALID_ARG, "n = %d out of range [1, 2^31-2]", n);
    if (row_ptr[0] != 0) return fail(SNAP_ERR_INVALID_ARG, "row_ptr[0] = %lld, expected 0", (long long)row_ptr[0]);
    for (int32_t i = 0; i < n; ++i)
        if (row_ptr[i + 1] < row_ptr[i])
            return fail(SNAP_ERR_INVALID_ARG, "row_ptr decreases at row %d", i);
    const int64_t nnz = row_ptr[n];
    if (nnz >= ((int64_t)1 << 31)) return fail(SNAP_ERR_INVALID_ARG, "nnz = %lld exceeds 2^31-1", (long long)nnz);
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
    if (o.sampler != SNAP_SAMPLER_UNIFORM)
        return fail(SNAP_ERR_NOT_SUPPORTED, "sampler %d is not implemented (only SNAP_SAMPLER_UNIFORM)", o.sampler);
    if (o.sync_substeps < 1 || o.sync_substeps > (1 << 20))
        return fail(SNAP_ERR_INVALID_ARG, "sync_substeps = %d out of range [1, 2^20]", o.sync_substeps);
    if (!(o.sync_cap >= 0.0f) || !std::isfinite(o.sync_cap))
        return fail(SNAP_ERR_INVALID_ARG, "sync_cap must be finite and >= 0");
    if (o.segment_edges != 0 && (o.segment_edges < 4 || o.segment_edges > 4096 || o.segment_edges % 4 != 0))
        return fail(SNAP_ERR_INVALID_ARG, "segment_edges = %d must be 0 or a multiple of 4 in [4, 4096]",
                    o.segment_edges);
    if (o.block_threads != 0 && (o.block_threads < 32 || o.block_threads > 256 || o.block_threads % 32 != 0))
        return fail(SNAP_ERR_INVALID_ARG, "block_threads = %d must be 0 or a multiple of 32 in [32, 256]",
                    o.block_threads);
    return SNAP_OK;
}

snap_status snap_layout_create(const int64_t *row_ptr, const int32_t *col_idx, const int32_t *degrees, int32_t n,
                               const snap_options *opts, void *cuda_stream, snap_layout_t *out) {
    if (!out) return fail(SNAP_ERR_INVALID_ARG, "out is NULL");
    snap_status st = check_csr_host(row_ptr, col_idx, degrees, n);
    if (st != SNAP_OK) return st;
    snap_options o;
    snap_options_default(&o);
    if (opts) o = *opts;
    st = check_options(o);
    if (st != SNAP_OK) return st;

    cudaStream_t stream = (cudaStream_t)cuda_stream;
    snap_layout *h = new (std::nothrow) snap_layout();
    if (!h) return fail(SNAP_ERR_OUT_OF_MEMORY, "host allocation of the handle failed");
    h->n = n;
    h->nnz = row_ptr[n];
    h->opts = o;
    // CSR segments: the synchronous kernel's unit of work (and the
    // validation pass); the HOGWILD modes use segments of oriented entries.
    h->seg_len = (o.mode == SNAP_MODE_SYNC && o.segment_edges) ? o.segment_edges : 32;
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
        err = dev_alloc(ac, (void **)&(ptr), (bytes));                                \
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
    SNAP_CUDA(cudaMallocHost((void **)&h->h_status, sizeof(uint32_t) * 4), "pinned status word");
    SNAP_CUDA(cudaEventCreateWithFlags(&h->status_event, cudaEventDisableTiming), "status event");
    std::vector<int32_t> deg((size_t)n);
    for (int32_t i = 0; i < n; ++i) deg[(size_t)i] = (int32_t)(row_ptr[i + 1] - row_ptr[i]);
    SNAP_CUDA(cudaMemcpyAsync(h->d_row_ptr, row_ptr, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyHostToDevice,
                              stream), "copy row_ptr");
    if (h->nnz > 0)
        SNAP_CUDA(cudaMemcpyAsync(h->d_col, col_idx, sizeof(int32_t) * (size_t)h->nnz, cudaMemcpyHostToDevice,
                                  stream), "copy col_idx");
    SNAP_CUDA(cudaMemsetAsync(h->d_col + h->nnz, 0, sizeof(int32_t) * (col_entries - (size_t)h->nnz), stream),
              "clear col_idx padding");
    SNAP_CUDA(cudaMemcpyAsync(h->d_deg, deg.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, stream),
              "copy degrees");
    SNAP_CUDA(cudaMemsetAsync(h->d_status, 0, sizeof(uint32_t) * 4, stream), "clear status");
    if (h->d_disp) SNAP_CUDA(cudaMemsetAsync(h->d_disp, 0, disp_bytes, stream), "clear displacement");
    SNAP_CUDA(launch_segment_rows(h->d_row_ptr, n, h->nnz, h->seg_len, h->d_seg_row, h->num_segs, stream),
              "segment table kernel");
    SNAP_CUDA(launch_validate_csr(h->d_row_ptr, h->d_col, h->d_seg_row, n, h->nnz, h->seg_len, h->d_status + 1,
                                  stream), "validation kernel");
    SNAP_CUDA(cudaMemcpyAsync(h->h_status, h->d_status, sizeof(uint32_t) * 4, cudaMemcpyDeviceToHost, stream),
              "read validation word");
    SNAP_CUDA(cudaStreamSynchronize(stream), "create");
#undef SNAP_CUDA
    const uint32_t vflags = h->h_status[1];
    if (vflags) {
        h->release();
        delete h;
        if (vflags & kBadColumn) return fail(SNAP_ERR_INVALID_ARG, "col_idx holds a column outside [0, n)");
        if (vflags & kSelfLoop) return fail(SNAP_ERR_INVALID_ARG, "col_idx holds a self-loop (j == i)");
        if (vflags & kUnsorted) return fail(SNAP_ERR_INVALID_ARG, "a row of col_idx is not strictly ascending");
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

snap_status snap_layout_epochs(snap_layout_t h, float *positions, int32_t epoch_begin, int32_t epochs,
                               int32_t neg_samples, const snap_schedule *schedule, uint64_t seed,
                               void *cuda_stream) {
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
    if (h->nnz == 0 || epochs == 0) return SNAP_OK;

    cudaStream_t stream = (cudaStream_t)cuda_stream;
    float2 *pos = reinterpret_cast<float2 *>(positions);
    cudaError_t err = cudaSuccess;
    for (int32_t ep = 0; ep < epochs; ++ep) {
        const int32_t t = epoch_begin + ep;
        const double eta = step_size(*schedule, t);
        if (h->opts.mode == SNAP_MODE_SYNC) {
            const double limit = h->opts.sync_cap > 0.0f ? (double)h->opts.sync_cap * eta / schedule->eta0 : 0.0;
            const int32_t S = h->opts.sync_substeps;
            for (int32_t c = 0; c < S && err == cudaSuccess; ++c) {
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
                    const int64_t segs = (ee + h->seg_len - 1) / h->seg_len - eb / h->seg_len;
                    const int64_t want = (segs + h->block - 1) / h->block;
                    const int grid = (int)(want < h->grid_sync ? want : h->grid_sync);
                    err = launch_sync_chunk(a, grid > 0 ? grid : 1, h->block, stream);
                }
                if (err == cudaSuccess)
                    err = launch_sync_apply(pos, h->d_disp, h->n, (float)eta, (float)limit, h->d_status,
                                            h->grid_apply, 256, stream);
            }
        } else {
            OrientedArgs a;
            a.row_ptr = h->d_act_row_ptr;
            a.ent = h->d_act_ent;
            a.seg = h->d_act_seg;
            a.pos = pos;
            a.num_segs = h->act_num_segs;
            a.perm_mul = h->perm_mul;
            a.perm_add = (int64_t)(mix64(seed ^ (0x5EC0ull * (uint64_t)(t + 1))) % (uint64_t)h->act_num_segs);
            a.n = h->n;
            a.k = neg_samples;
            a.epoch = (uint32_t)t;
            a.seed = seed;
            a.eta = (float)eta;
            a.status = h->d_status;
            const int red = h->opts.mode == SNAP_MODE_HOGWILD_RED;
            const int g = neg_samples < 4 ? neg_samples : 4;
            if (h->grid_oriented[red][g] == 0)
                h->grid_oriented[red][g] = h->sms * oriented_blocks_per_sm(red, neg_samples, h->block);
            const int gmax = h->grid_oriented[red][g];
            const int64_t want = (h->act_num_segs + h->block - 1) / h->block;
            if (h->act_num_segs == 0) continue;
            const int grid = (int)(want < gmax ? want : gmax);
            err = launch_oriented_epoch(a, red, grid > 0 ? grid : 1, h->block, stream);
        }
        if (err != cudaSuccess) return cuda_fail(err, "epoch launch");
    }
    if (!h->status_pending) {
        err = cudaMemcpyAsync(h->h_status, h->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream);
        if (err == cudaSuccess) err = cudaEventRecord(h->status_event, stream);
        if (err != cudaSuccess) return cuda_fail(err, "status read-back");
        h->status_pending = true;
    }
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

snap_status snap_layout_objective(snap_layout_t h, const float *positions, int32_t neg_samples, int32_t exact,
                                  int64_t pair_samples, uint64_t seed, double *out_attr, double *out_rep,
                                  double *out_total, void *cuda_stream) {
    if (!h) return fail(SNAP_ERR_INVALID_ARG, "handle is NULL");
    if (!positions) return fail(SNAP_ERR_INVALID_ARG, "positions is NULL");
    if (((uintptr_t)positions & 7u) != 0) return fail(SNAP_ERR_INVALID_ARG, "positions must be 8-byte aligned");
    if (neg_samples < 0) return fail(SNAP_ERR_INVALID_ARG, "neg_samples must be >= 0");
    if (!exact && pair_samples <= 0) return fail(SNAP_ERR_INVALID_ARG, "pair_samples must be > 0 when exact = 0");
    snap_status st = poll_status(h);
    if (st != SNAP_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const float2 *pos = reinterpret_cast<const float2 *>(positions);
    cudaError_t err = cudaMemsetAsync(h->d_partial, 0, sizeof(double) * 2 * kObjGrid, stream);
    if (err == cudaSuccess && h->nnz > 0) {
        if (h->d_col)
            err = launch_objective_edges(h->d_row_ptr, h->d_col, h->d_seg_row, pos, h->nnz, h->seg_len,
                                         h->d_partial, kObjGrid, stream);
        else if (h->act_num_segs > 0)
            err = launch_objective_oriented(h->d_act_row_ptr, h->d_act_ent, h->d_act_seg, h->act_num_segs, pos,
                                            h->d_partial, kObjGrid, stream);
    }
    if (err == cudaSuccess && h->n > 1) {
        if (exact)
            err = launch_objective_pairs_exact(pos, h->d_deg, h->n, h->d_partial + kObjGrid, kObjGrid, stream);
        else
            err = launch_objective_pairs_sampled(pos, h->d_deg, h->n, pair_samples, seed, h->d_partial + kObjGrid,
                                                 kObjGrid, stream);
    }
    std::vector<double> part(2 * (size_t)kObjGrid);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(part.data(), h->d_partial, sizeof(double) * 2 * kObjGrid, cudaMemcpyDeviceToHost,
                              stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
    if (err != cudaSuccess) return cuda_fail(err, "objective");
    double attr = 0.0, pairsum = 0.0;
    for (int b = 0; b < kObjGrid; ++b) attr += part[(size_t)b];
    for (int b = 0; b < kObjGrid; ++b) pairsum += part[(size_t)kObjGrid + b];
    double rep = 0.0;
    if (h->n > 1) {
        const double n = (double)h->n;
        // unordered-pair sum of (d_i + d_j) U^r
        const double unordered = exact ? 0.5 * pairsum : pairsum / (double)pair_samples * 0.5 * n * (n - 1.0);
        rep = (double)neg_samples * unordered / (2.0 * (n - 1.0));
    }
    if (out_attr) *out_attr = attr;
    if (out_rep) *out_rep = rep;
    if (out_total) *out_total = attr + rep;
    return SNAP_OK;
}

int64_t snap_layout_device_bytes(snap_layout_t h) { return h ? h->device_bytes : 0; }

void snap_layout_destroy(snap_layout_t h) {
    if (!h) return;
    h->release();
    delete h;
}

snap_status snap_layout_run(const int64_t *row_ptr, const int32_t *col_idx, int32_t n, const snap_options *opts,
                            float *positions_host, int32_t epochs, int32_t neg_samples, const snap_schedule *schedule,
                            uint64_t seed, void *cuda_stream) {
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
    cudaError_t err = dev_alloc(g_alloc, (void **)&d_pos, bytes);
    if (err != cudaSuccess) {
        cudaGetLastError();
        snap_layout_destroy(h);
        return cuda_fail(err, "device allocation of positions");
    }
    err = cudaMemcpyAsync(d_pos, positions_host, bytes, cudaMemcpyHostToDevice, stream);
    if (err != cudaSuccess) {
        cudaFree(d_pos);
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
    cudaFree(d_pos);
    snap_layout_destroy(h);
    return st;
}

}  // extern "C"
