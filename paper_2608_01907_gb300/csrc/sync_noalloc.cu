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
// The kernel below computes exactly the terms of the synchronous chunk
// kernel in epoch_kernels.cu (same force, Philox and fixed-point helpers),
// but finds its chunk bounds and each segment's start row by binary search
// on the device instead of reading tables built at create, and checks every
// column index against n (the CSR is not validated beforehand).
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
constexpr uint32_t kNoallocBadColumn = 8u;
constexpr int kMaxDevices = 64;
constexpr int kSegLen = 32;

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
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const uint32_t nm1 = (uint32_t)(n - 1);
    uint32_t flags = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t seg = seg_first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; seg < seg_last; seg += stride) {
        const int64_t e0 = max(seg * kSegLen, e_begin);
        const int64_t e1 = min(seg * kSegLen + kSegLen, e_end);
        int32_t row = row_of_edge(row_ptr, n, e0);
        int64_t row_end = row_ptr[row + 1];
        float2 yi = pos[row];
        long long accx = 0, accy = 0;
        for (int64_t e = e0; e < e1; ++e) {
            if (e >= row_end) {
                flush_source(disp, row, accx, accy);
                while (row + 1 < n && row_ptr[row + 1] <= e) ++row;
                row_end = row_ptr[row + 1];
                yi = pos[row];
            }
            const int32_t i = row;
            const int32_t j = col_idx[e];
            if (j < 0 || j >= n) {
                flags |= kNoallocBadColumn;
                continue;
            }
            const float2 yj = pos[j];
            const float2 f = attraction_on_i(yi.x - yj.x, yi.y - yj.y);
            const long long fx = to_fixed(f.x, flags), fy = to_fixed(f.y, flags);
            accx += fx;
            accy += fy;
            add_fixed(disp + 2 * (int64_t)j, -fx);
            add_fixed(disp + 2 * (int64_t)j + 1, -fy);
            for (int g = 0; g * 4 < k; ++g) {
                const int nm = k - 4 * g < 4 ? k - 4 * g : 4;
                const uint4 w = edge_words(e, epoch, (uint32_t)g, key);
                const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if (m < nm) {
                        const int32_t s = negative_of(ws[m], i, nm1);
                        const float2 ys = pos[s];
                        const float2 gr = repulsion_on_i(yi.x - ys.x, yi.y - ys.y);
                        const long long gx = to_fixed(gr.x, flags), gy = to_fixed(gr.y, flags);
                        accx += gx;
                        accy += gy;
                        add_fixed(disp + 2 * (int64_t)s, -gx);
                        add_fixed(disp + 2 * (int64_t)s + 1, -gy);
                    }
                }
            }
        }
        flush_source(disp, row, accx, accy);
    }
    if (flags) atomicOr(status, flags);
}

snap_status noalloc_fail(snap_status st, const char *fmt, long long a = 0, long long b = 0) {
    char buf[256];
    snprintf(buf, sizeof(buf), fmt, a, b);
    return snap::reorder_fail(st, buf);
}

}  // namespace

extern "C" snap_status snap_sync_epochs_noalloc(const int64_t *row_ptr, const int32_t *col_idx, int32_t n,
                                                float *positions, int32_t epoch_begin, int32_t epochs,
                                                int32_t neg_samples, const snap_schedule *schedule, uint64_t seed,
                                                int32_t substeps, float cap, void *cuda_stream) {
    if (!row_ptr || !col_idx || !positions || !schedule)
        return noalloc_fail(SNAP_ERR_INVALID_ARG, "snap_sync_epochs_noalloc: NULL argument");
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
    DeviceScratch sc;
    cudaError_t err = current_scratch(sc);
    if (err != cudaSuccess)
        return noalloc_fail(SNAP_ERR_CUDA, "snap_sync_epochs_noalloc: scratch set-up failed (%lld)", (long long)err);
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    // the scratch keeps the previous call's contents: start from zero
    err = cudaMemsetAsync(sc.disp, 0, sizeof(long long) * 2 * (size_t)n, stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(sc.status, 0, sizeof(uint32_t) * 4, stream);
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
    if (flags & kNoallocBadColumn)
        return noalloc_fail(SNAP_ERR_INVALID_ARG, "snap_sync_epochs_noalloc: a column index is outside [0, n)");
    if (flags & kStatusNonFinite)
        return noalloc_fail(SNAP_ERR_NUMERIC, "snap_sync_epochs_noalloc: a position became non-finite");
    if (flags & kStatusClamped)
        return noalloc_fail(SNAP_ERR_NUMERIC, "snap_sync_epochs_noalloc: a fixed-point force term was clamped");
    return SNAP_OK;
}
