// sync_noalloc.cu -- snap_sync_epochs_noalloc: the synchronous epoch for
// callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: code that runs inside a host
// framework which owns every byte of device memory through its own pool or
// memory budget, or latency-critical code that cannot afford the implicit
// device synchronisation an allocation may cause.  For them this entry
// point runs the synchronous mode on buffers the caller already owns (device
// CSR and positions) and keeps its only scratch -- the int64 fixed-point
// displacement per vertex and a status word -- in file-scope device arrays
// of fixed size.  Those arrays exist on every GPU that loads the library
// until the process exits (4 MiB + 16 bytes).
//
// The chunk kernel below computes every edge's terms with the same device
// function as the synchronous chunk kernel of a handle (sync_edge_terms in
// snap_device.cuh), but finds its chunk bounds and each segment's start row
// by binary search on the device instead of reading tables built at create.
// Before any epoch runs, a validation pass checks the caller's CSR on the
// device (the rules snap_layout_create applies) and the call returns
// INVALID_ARG without touching the positions if it fails, so no later kernel
// reads outside the caller's buffers.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/snap_layout.h"
#include "snap_device.cuh"
#include "snap_internal.h"

namespace snap {
// Records the message returned by snap_last_error (defined in capi.cu).
snap_status reorder_fail(snap_status st, const char *msg);
}  // namespace snap

namespace {

using namespace snap;

// Largest vertex count the fixed scratch holds: 2^18 = 262,144 vertices,
// 2 int64 per vertex = 4 MiB.
constexpr int32_t kNoallocMaxNodes = 1 << 18;
constexpr uint32_t kNoallocBadCsr = 8u;
constexpr int kMaxDevices = 64;
constexpr int kSegLen = 16;

// The scratch.  In host code these names are host-side stand-ins, not device
// addresses; the device addresses come from cudaGetSymbolAddress below.
static __device__ __align__(256) long long g_noalloc_disp[2 * kNoallocMaxNodes];
static __device__ __align__(256) uint32_t g_noalloc_status[4];

struct DeviceScratch {
    long long *disp = nullptr;
    uint32_t *status = nullptr;
    int sms = 0;
    bool ready = false;
};

std::mutex g_scratch_mu;
DeviceScratch g_scratch[kMaxDevices];

// Device addresses of the scratch arrays on the current device, looked up
// once per device (with that device current) on the first call there.
cudaError_t current_scratch(DeviceScratch &out) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    DeviceScratch &s = g_scratch[dev];
    if (!s.ready) {
        void *p = nullptr;
        err = cudaGetSymbolAddress(&p, g_noalloc_disp);
        if (err != cudaSuccess) return err;
        s.disp = static_cast<long long *>(p);
        err = cudaGetSymbolAddress(&p, g_noalloc_status);
        if (err != cudaSuccess) return err;
        s.status = static_cast<uint32_t *>(p);
        err = cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev);
        if (err != cudaSuccess) return err;
        if (s.sms <= 0) s.sms = 1;
        s.ready = true;
    }
    out = s;
    return cudaSuccess;
}

// First row r in [0, n] with row_ptr[r] * S >= c * nnz (chunk c's first row).
__device__ __forceinline__ int32_t chunk_first_row(const int64_t *row_ptr, int32_t n, int64_t nnz, int32_t S,
                                                   int32_t c) {
    if (c <= 0) return 0;
    if (c >= S) return n;
    const int64_t want = (int64_t)c * nnz;
    int32_t lo = 0, hi = n;   // row_ptr[hi] * S >= want always holds for hi = n
    while (lo < hi) {
        const int32_t mid = lo + (hi - lo) / 2;
        if (row_ptr[mid] * (int64_t)S >= want)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// Row holding edge e < nnz: the largest r with row_ptr[r] <= e.
__device__ __forceinline__ int32_t row_of_edge(const int64_t *row_ptr, int32_t n, int64_t e) {
    int32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int32_t mid = lo + (hi - lo) / 2;
        if (row_ptr[mid] <= e)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void flush_source(long long *disp, int32_t row, long long &accx, long long &accy) {
    if (accx | accy) {
        add_fixed(disp + 2 * (int64_t)row, accx);
        add_fixed(disp + 2 * (int64_t)row + 1, accy);
    }
    accx = accy = 0;
}

// Validation, part 1 (one thread per row): row_ptr[0] = 0, row_ptr[n] = nnz,
// and every row's bounds inside [0, nnz] and non-decreasing.  Reads only
// row_ptr[0..n].
__global__ void __launch_bounds__(256) check_rows_kernel(const int64_t *__restrict__ row_ptr, int32_t n, int64_t nnz,
                                                         uint32_t *status) {
    const int32_t stride = gridDim.x * blockDim.x;
    bool bad = false;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t lo = row_ptr[i], hi = row_ptr[i + 1];
        if (lo < 0 || hi < lo || hi > nnz) bad = true;
        if (i == 0 && lo != 0) bad = true;
        if (i == n - 1 && hi != nnz) bad = true;
    }
    if (bad) atomicOr(status, kNoallocBadCsr);
}

// Validation, part 2 (one thread per directed edge): the edge's row found by
// binary search must hold it, its column must lie in [0, n) and differ from
// the row, rows must be strictly ascending, and the reverse edge must exist.
// Every read is bounds-checked first (row_ptr indices in [0, n], col_idx
// indices in [0, nnz)), whatever part 1 finds.
__global__ void __launch_bounds__(256) check_edges_kernel(const int64_t *__restrict__ row_ptr,
                                                          const int32_t *__restrict__ col_idx, int32_t n, int64_t nnz,
                                                          uint32_t *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        const int32_t i = row_of_edge(row_ptr, n, e);
        const int64_t lo = row_ptr[i], hi = row_ptr[i + 1];
        if (!(lo <= e && e < hi)) {
            bad = true;
            continue;
        }
        const int32_t j = col_idx[e];
        if (j < 0 || j >= n || j == i) {
            bad = true;
            continue;
        }
        if (e > lo && col_idx[e - 1] >= j) bad = true;
        int64_t a = row_ptr[j], b = row_ptr[j + 1];
        if (a < 0 || b < a || b > nnz) {
            bad = true;
            continue;
        }
        while (a < b) {   // first position in row j with col >= i
            const int64_t mid = a + (b - a) / 2;
            if (col_idx[mid] < i)
                a = mid + 1;
            else
                b = mid;
        }
        if (a >= row_ptr[j + 1] || col_idx[a] != i) bad = true;
    }
    if (bad) atomicOr(status, kNoallocBadCsr);
}

// Chunk c of S of one synchronous epoch on a validated CSR: 16-edge segments,
// one lane each; the source's terms are summed in registers and flushed once
// per row run.
__global__ void __launch_bounds__(256) sync_chunk_noalloc_kernel(const int64_t *__restrict__ row_ptr,
                                                                 const int32_t *__restrict__ col_idx,
                                                                 const float2 *__restrict__ pos,
                                                                 long long *__restrict__ disp, int32_t n, int32_t k,
                                                                 int32_t S, int32_t c, uint32_t epoch, uint64_t seed,
                                                                 uint32_t *status) {
    const int64_t nnz = row_ptr[n];
    const int64_t e_begin = row_ptr[chunk_first_row(row_ptr, n, nnz, S, c)];
    const int64_t e_end = row_ptr[chunk_first_row(row_ptr, n, nnz, S, c + 1)];
    if (e_begin >= e_end) return;
    const int64_t seg_first = e_begin / kSegLen;
    const int64_t seg_last = (e_end + kSegLen - 1) / kSegLen;
    GraphCtx ctx;
    ctx.base = 0;
    ctx.nm1 = (uint32_t)(n - 1);
    ctx.edge_base = 0;
    ctx.epoch = epoch;
    ctx.eta = 0.0f;
    ctx.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    ctx.active = true;
    uint32_t flags = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t seg = seg_first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; seg < seg_last; seg += stride) {
        const int64_t e0 = max(seg * kSegLen, e_begin);
        const int64_t e1 = min(seg * kSegLen + kSegLen, e_end);
        int32_t row = row_of_edge(row_ptr, n, e0);
        int64_t row_end = row_ptr[row + 1];
        float2 yi = __ldg(pos + row);
        long long accx = 0, accy = 0;
        for (int64_t e = e0; e < e1; ++e) {
            if (e >= row_end) {
                flush_source(disp, row, accx, accy);
                while (row + 1 < n && row_ptr[row + 1] <= e) ++row;
                row_end = row_ptr[row + 1];
                yi = __ldg(pos + row);
            }
            sync_edge_terms(pos, disp, ctx, nullptr, row, yi, col_idx[e], e, k, false, accx, accy, flags);
        }
        flush_source(disp, row, accx, accy);
    }
    if (flags) atomicOr(status, flags);
}

// INVALID_ARG unless p is device (or managed) memory of the current device.
cudaError_t on_device(const void *p, int dev, bool &ok) {
    cudaPointerAttributes attr;
    const cudaError_t err = cudaPointerGetAttributes(&attr, p);
    if (err != cudaSuccess) return err;
    ok = (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) && attr.device == dev;
    return cudaSuccess;
}

snap_status noalloc_fail(snap_status st, const char *fmt, long long a = 0, long long b = 0) {
    char buf[256];
    snprintf(buf, sizeof(buf), fmt, a, b);
    return snap::reorder_fail(st, buf);
}

}  // namespace

extern "C" snap_status snap_sync_epochs_noalloc(const int64_t *row_ptr, const int32_t *col_idx, int64_t nnz,
                                                int32_t n, float *positions, int32_t epoch_begin, int32_t epochs,
                                                int32_t neg_samples, const snap_schedule *schedule, uint64_t seed,
                                                int32_t substeps, float cap, void *cuda_stream) {
    if (!row_ptr || !positions || !schedule || (nnz > 0 && !col_idx))
        return noalloc_fail(SNAP_ERR_INVALID_ARG, "snap_sync_epochs_noalloc: NULL argument");
    if (nnz < 0 || nnz >= ((int64_t)1 << 32))
        return noalloc_fail(SNAP_ERR_INVALID_ARG, "snap_sync_epochs_noalloc: nnz = %lld is outside [0, 2^32)",
                            (long long)nnz);
    if (n < 1 || n > kNoallocMaxNodes)
        return noalloc_fail(SNAP_ERR_INVALID_ARG,
                            "snap_sync_epochs_noalloc: n = %lld is outside [1, %lld], the vertex limit of its "
                            "fixed scratch",
                            (long long)n, (long long)kNoallocMaxNodes);
    if (((uintptr_t)positions & 7u) != 0 || ((uintptr_t)row_ptr & 7u) != 0 || ((uintptr_t)col_idx & 3u) != 0)
        return noalloc_fail(SNAP_ERR_INVALID_ARG, "snap_sync_epochs_noalloc: misaligned buffer");
    if (epoch_begin < 0 || epochs < 0 || neg_samples < 0 || neg_samples > 64)
        return noalloc_fail(SNAP_ERR_INVALID_ARG, "snap_sync_epochs_noalloc: bad epoch range or neg_samples");
    if (substeps < 1 || substeps > (1 << 20) || !(cap >= 0.0f) || !std::isfinite(cap))
        return noalloc_fail(SNAP_ERR_INVALID_ARG, "snap_sync_epochs_noalloc: bad substeps or cap");
    if ((schedule->kind != 0 && schedule->kind != 1) || !(schedule->eta0 > 0.0) || !std::isfinite(schedule->eta0) ||
        !(schedule->eta_min >= 0.0) || schedule->total_epochs < 1)
        return noalloc_fail(SNAP_ERR_INVALID_ARG, "snap_sync_epochs_noalloc: bad schedule");
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    bool ok_rp = false, ok_ci = true, ok_pos = false;
    if (err == cudaSuccess) err = on_device(row_ptr, dev, ok_rp);
    if (err == cudaSuccess && nnz > 0) err = on_device(col_idx, dev, ok_ci);
    if (err == cudaSuccess) err = on_device(positions, dev, ok_pos);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(SNAP_ERR_INVALID_ARG, "snap_sync_epochs_noalloc: a buffer is not device memory (%lld)",
                            (long long)err);
    }
    if (!ok_rp || !ok_ci || !ok_pos)
        return noalloc_fail(SNAP_ERR_INVALID_ARG,
                            "snap_sync_epochs_noalloc: row_ptr, col_idx and positions must be device memory of the "
                            "current device (%lld)",
                            (long long)dev);
    DeviceScratch sc;
    err = current_scratch(sc);
    if (err != cudaSuccess)
        return noalloc_fail(SNAP_ERR_CUDA, "snap_sync_epochs_noalloc: scratch set-up failed (%lld)", (long long)err);
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    // the scratch keeps the previous call's contents: start from zero
    err = cudaMemsetAsync(sc.disp, 0, sizeof(long long) * 2 * (size_t)n, stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(sc.status, 0, sizeof(uint32_t) * 4, stream);
    // validate the CSR before any kernel indexes by it
    if (err == cudaSuccess) {
        check_rows_kernel<<<(n + 255) / 256, 256, 0, stream>>>(row_ptr, n, nnz, sc.status);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess && nnz > 0) {
        const int64_t want = (nnz + 255) / 256;
        const int grid_e = (int)(want < (int64_t)sc.sms * 16 ? want : (int64_t)sc.sms * 16);
        check_edges_kernel<<<grid_e, 256, 0, stream>>>(row_ptr, col_idx, n, nnz, sc.status);
        err = cudaGetLastError();
    }
    uint32_t csr_flags = 0;
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(&csr_flags, sc.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
    if (err != cudaSuccess)
        return noalloc_fail(SNAP_ERR_CUDA, "snap_sync_epochs_noalloc: CUDA error %lld", (long long)err);
    if (csr_flags & kNoallocBadCsr)
        return noalloc_fail(SNAP_ERR_INVALID_ARG,
                            "snap_sync_epochs_noalloc: malformed CSR (row_ptr[0] != 0, row_ptr[n] != nnz, a "
                            "decreasing row_ptr, a column outside [0, n), a self-loop, an unsorted row or a missing "
                            "reverse edge)");
    if (nnz == 0) return SNAP_OK;
    float2 *pos = reinterpret_cast<float2 *>(positions);
    const int grid = sc.sms * 4;
    for (int32_t ep = 0; ep < epochs && err == cudaSuccess; ++ep) {
        const int32_t t = epoch_begin + ep;
        double eta = schedule->eta0;
        if (schedule->kind == 0) {
            eta = schedule->eta0 * (1.0 - (double)t / (double)schedule->total_epochs);
            if (eta < schedule->eta_min) eta = schedule->eta_min;
        }
        const double limit = cap > 0.0f ? (double)cap * eta / schedule->eta0 : 0.0;
        for (int32_t c = 0; c < substeps && err == cudaSuccess; ++c) {
            sync_chunk_noalloc_kernel<<<grid, 256, 0, stream>>>(row_ptr, col_idx, pos, sc.disp, n, neg_samples,
                                                                substeps, c, (uint32_t)t, seed, sc.status);
            err = cudaGetLastError();
            if (err == cudaSuccess)
                err = launch_sync_apply(pos, sc.disp, n, (float)eta, (float)limit, sc.status, sc.sms * 8, 256, stream);
        }
    }
    uint32_t flags = 0;
    if (err == cudaSuccess) err = cudaMemcpyAsync(&flags, sc.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
    if (err != cudaSuccess)
        return noalloc_fail(SNAP_ERR_CUDA, "snap_sync_epochs_noalloc: CUDA error %lld", (long long)err);
    if (flags & kStatusNonFinite)
        return noalloc_fail(SNAP_ERR_NUMERIC, "snap_sync_epochs_noalloc: a position became non-finite");
    if (flags & kStatusClamped)
        return noalloc_fail(SNAP_ERR_NUMERIC, "snap_sync_epochs_noalloc: a fixed-point force term was clamped");
    return SNAP_OK;
}
