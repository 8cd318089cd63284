// bench_probe.cu -- hardware ceilings for bench.py's rooflines (measurement
// only; not part of the layout library).
//
// The epoch kernels stream their edge entries from HBM and make random
// 8-byte accesses to an L2-resident position array: loads of positions and
// vector float atomic adds of displacements.  Each probe below exercises one
// of those hardware paths alone, with many independent accesses in flight
// per thread and nothing else in the kernel, on a caller-owned array:
//   op 0  streaming read: coalesced 16-byte loads (ld.global.cg) sweeping the
//         array; result in bytes per second (the L2 bandwidth when the array
//         fits in L2)
//   op 1  random loads: 8-byte loads of uniformly random slots (ld.global.cg),
//         8 independent per thread per iteration; loads per second
//   op 2  random atomic adds: 8-byte vector float adds without return
//         (red.global.add.v2.f32) to uniformly random slots, 8 per thread per
//         iteration; atomics per second
//   op 3  the two mixed: per thread and iteration 8 random loads and 8
//         random atomic adds to other slots, independent of each other (the
//         mix the epoch kernels issue, without their dependence); load +
//         atomic pairs per second
//   op 4  the synchronous mode's mix: the array is cut into a position part
//         (its first third, 8-byte slots) and a displacement part (the rest,
//         16-byte slots of two int64); per thread and iteration 8 random
//         position loads and 8 random displacement slots, each given two
//         64-bit integer atomic adds (atom.global.add.u64, no return);
//         load + two-atomic triples per second
// Slots come from a 64-bit mixing hash of (thread, iteration) reduced to
// [0, n) by a multiply-shift, so every access stays inside the array.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kDepth = 8;

__device__ __forceinline__ uint32_t mix_slot(uint64_t x, uint32_t n) {
    // SplitMix64 finaliser (Steele, Lea, Flood 2014), then multiply-shift to [0, n)
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (uint32_t)(((x & 0xFFFFFFFFull) * (uint64_t)n) >> 32);
}

__global__ void __launch_bounds__(256) stream_read_kernel(const float4 *a, int64_t n4, int iters, float *sink) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float acc = 0.f;
    for (int it = 0; it < iters; ++it) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(a + i);
            acc += v.x + v.y + v.z + v.w;
        }
    }
    if (acc == 12345.678f) sink[0] = acc;   // keeps the loads alive
}

__global__ void __launch_bounds__(256) random_load_kernel(const float2 *a, uint32_t n, int iters, float *sink) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.f;
    for (int it = 0; it < iters; ++it) {
        float2 v[kDepth];
#pragma unroll
        for (int d = 0; d < kDepth; ++d) v[d] = __ldcg(a + mix_slot((tid << 24) ^ ((uint64_t)it * kDepth + d), n));
#pragma unroll
        for (int d = 0; d < kDepth; ++d) acc += v[d].x;
    }
    if (acc == 12345.678f) sink[0] = acc;
}

__global__ void __launch_bounds__(256) random_red_kernel(float2 *a, uint32_t n, int iters) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int d = 0; d < kDepth; ++d) {
            float2 *p = a + mix_slot((tid << 24) ^ ((uint64_t)it * kDepth + d), n);
            asm volatile("red.relaxed.gpu.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(1e-7f), "f"(0.0f)
                         : "memory");
        }
    }
}

__global__ void __launch_bounds__(256) random_mixed_kernel(float2 *a, uint32_t n, int iters, float *sink) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.f;
    for (int it = 0; it < iters; ++it) {
        float2 v[kDepth];
#pragma unroll
        for (int d = 0; d < kDepth; ++d) v[d] = __ldcg(a + mix_slot((tid << 24) ^ ((uint64_t)it * kDepth + d), n));
#pragma unroll
        for (int d = 0; d < kDepth; ++d) {
            float2 *p = a + mix_slot(((tid << 24) ^ ((uint64_t)it * kDepth + d)) + 0x9E37ull, n);
            asm volatile("red.relaxed.gpu.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(1e-7f), "f"(0.0f)
                         : "memory");
        }
#pragma unroll
        for (int d = 0; d < kDepth; ++d) acc += v[d].x;
    }
    if (acc == 12345.678f) sink[0] = acc;
}

__global__ void __launch_bounds__(256) random_sync_mixed_kernel(const float2 *a, uint32_t n,
                                                                unsigned long long *disp, uint32_t nd, int iters,
                                                                float *sink) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.f;
    for (int it = 0; it < iters; ++it) {
        float2 v[kDepth];
#pragma unroll
        for (int d = 0; d < kDepth; ++d) v[d] = __ldcg(a + mix_slot((tid << 24) ^ ((uint64_t)it * kDepth + d), n));
#pragma unroll
        for (int q = 0; q < kDepth; ++q) {
            unsigned long long *p =
                disp + 2 * (uint64_t)mix_slot(((tid << 24) ^ ((uint64_t)it * kDepth + q)) + 0x9E37ull, nd);
            atomicAdd(p, 1ull);
            atomicAdd(p + 1, 1ull);
        }
#pragma unroll
        for (int q = 0; q < kDepth; ++q) acc += v[q].x;
    }
    if (acc == 12345.678f) sink[0] = acc;
}

}  // namespace

// Runs probe `op` (above) on the caller's device array `a` of `bytes` bytes
// (a multiple of 16, at least 48) with `grid` blocks of 256 threads, once to
// warm up and once timed with CUDA events on `cuda_stream`.  `sink` is one
// device float.  Returns the op's rate (bytes/s for op 0, accesses/s
// otherwise) or a negative value on error.
extern "C" double bench_probe_rate(float *a, int64_t bytes, int op, int iters, int grid, float *sink,
                                   void *cuda_stream) {
    if (!a || !sink || bytes < 48 || (bytes & 15) != 0 || op < 0 || op > 4 || iters <= 0 || grid <= 0) return -1.0;
    const int64_t n2 = bytes / 8;
    if (n2 > 0xFFFFFFFFll) return -1.0;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -2.0;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -2.0;
    }
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {
        if (rep == 1) cudaEventRecord(e0, s);
        if (op == 0)
            stream_read_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const float4 *>(a), bytes / 16, iters, sink);
        else if (op == 1)
            random_load_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const float2 *>(a), (uint32_t)n2, iters, sink);
        else if (op == 2)
            random_red_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<float2 *>(a), (uint32_t)n2, iters);
        else if (op == 3)
            random_mixed_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<float2 *>(a), (uint32_t)n2, iters, sink);
        else {
            const int64_t pos_bytes = bytes / 48 * 16;   // a third, a multiple of 16
            random_sync_mixed_kernel<<<grid, 256, 0, s>>>(
                reinterpret_cast<const float2 *>(a), (uint32_t)(pos_bytes / 8),
                reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(a) + pos_bytes),
                (uint32_t)((bytes - pos_bytes) / 16), iters, sink);
        }
        err = cudaGetLastError();
    }
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess || ms <= 0.f) return -3.0;
    const double secs = (double)ms * 1e-3;
    if (op == 0) return (double)bytes * (double)iters / secs;
    return (double)grid * 256.0 * (double)iters * (double)kDepth / secs;
}
