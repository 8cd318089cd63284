// probe_l2.cu -- measurement probe for the roofline of the epoch kernels
// (built as libsnap_probe.so, used by bench.py only; not part of the layout
// library's ABI).
//
// The epoch kernels are bound by random 8-byte accesses to an L2-resident
// position array, a pattern whose ceiling the HBM copy bandwidth does not
// describe.  This probe issues the same pattern with nothing else around it:
// every thread visits uniformly random float2 slots of an n-slot array and
// performs one of
//   op 0: load                      (gather)
//   op 1: load then store           (racy read-modify-write, as HOGWILD)
//   op 2: load then atomic add      (as HOGWILD_RED)
//   op 3: atomic add only
//   op 4: load then 64-bit atomic exchange (a racy write that is atomic)
//   op 5: 64-bit atomic exchange only
//   op 6: store only
//   op 7: load slot s, store a value depending on it into another slot s'
//   op 8: load slot s, atomic add of a value depending on it into slot s
//   op 9: load slot s of the lower half, atomic add of a dependent value
//         into slot s of the upper half (reads and writes never alias)
//   op 10: as op 8 with the load on the non-coherent path (ld.global.nc)
//   op 11: as op 1 with the load on the non-coherent path (ld.global.nc)
// with `depth` independent accesses in flight per thread.  Slots come from a
// 64-bit mixing hash of (thread, iteration), so no random-number state is
// carried.  The result is accesses per second measured by CUDA events.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace {

__device__ __forceinline__ uint32_t mix_slot(uint64_t x, uint32_t n) {
    // SplitMix64 finaliser (Steele, Lea, Flood 2014), then multiply-shift to [0, n)
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (uint32_t)(((x & 0xFFFFFFFFull) * (uint64_t)n) >> 32);
}

template <int OP, int DEPTH>
__global__ void __launch_bounds__(256) probe_kernel(float2 *a, uint32_t n, int iters, float *sink) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.f;
    for (int it = 0; it < iters; ++it) {
        uint32_t s[DEPTH];
        float2 v[DEPTH];
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) s[d] = mix_slot((tid << 20) ^ ((uint64_t)it * DEPTH + d), n);
        const uint32_t half = n / 2;
        if (OP == 9) {
#pragma unroll
            for (int d = 0; d < DEPTH; ++d) s[d] = s[d] % half;
        }
        if (OP == 10 || OP == 11) {
#pragma unroll
            for (int d = 0; d < DEPTH; ++d) v[d] = __ldg(a + s[d]);
        } else if (OP == 0 || OP == 1 || OP == 2 || OP == 4 || OP == 7 || OP == 8 || OP == 9) {
#pragma unroll
            for (int d = 0; d < DEPTH; ++d) v[d] = __ldcg(a + s[d]);
        } else {
#pragma unroll
            for (int d = 0; d < DEPTH; ++d) v[d] = make_float2((float)it, (float)d);
        }
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) {
            if (OP == 0) {
                acc += v[d].x;
            } else if (OP == 1 || OP == 6 || OP == 11) {
                v[d].x += 1e-7f;
                __stcg(a + s[d], v[d]);
            } else if (OP == 7) {
                v[d].x += 1e-7f;
                __stcg(a + mix_slot(((tid << 20) ^ ((uint64_t)it * DEPTH + d)) + 0x51ull, n), v[d]);
            } else if (OP == 8 || OP == 10) {
                atomicAdd(a + s[d], make_float2(v[d].x * 1e-7f, 0.f));
            } else if (OP == 9) {
                atomicAdd(a + s[d] + half, make_float2(v[d].x * 1e-7f, 0.f));
            } else if (OP == 4 || OP == 5) {
                v[d].x += 1e-7f;
                unsigned long long bits;
                memcpy(&bits, &v[d], 8);
                atomicExch(reinterpret_cast<unsigned long long *>(a + s[d]), bits);
            } else {
                atomicAdd(a + s[d], make_float2(1e-7f, 0.f));
            }
        }
    }
    if (acc == 12345.678f) sink[0] = acc;   // keeps the loads of op 0 alive
}

template <int OP>
cudaError_t launch_op(int depth, float2 *a, uint32_t n, int iters, float *sink, int grid, cudaStream_t s) {
    switch (depth) {
        case 1: probe_kernel<OP, 1><<<grid, 256, 0, s>>>(a, n, iters, sink); break;
        case 2: probe_kernel<OP, 2><<<grid, 256, 0, s>>>(a, n, iters, sink); break;
        case 4: probe_kernel<OP, 4><<<grid, 256, 0, s>>>(a, n, iters, sink); break;
        default: probe_kernel<OP, 8><<<grid, 256, 0, s>>>(a, n, iters, sink); break;
    }
    return cudaGetLastError();
}

}  // namespace

// Runs the probe on a caller-owned device array `a` of n float2 slots and
// returns accesses per second (each access = one slot visit with the op's
// load and/or write), or a negative value on error.
extern "C" double snap_probe_random_access(float *a, uint32_t n, int op, int depth, int iters, int grid,
                                           void *cuda_stream) {
    if (!a || n < 2 || op < 0 || op > 11 || iters <= 0 || grid <= 0) return -1.0;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    float *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return -2.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float2 *p = reinterpret_cast<float2 *>(a);
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {
        if (rep == 1) cudaEventRecord(e0, s);
        switch (op) {
            case 0: err = launch_op<0>(depth, p, n, iters, sink, grid, s); break;
            case 1: err = launch_op<1>(depth, p, n, iters, sink, grid, s); break;
            case 2: err = launch_op<2>(depth, p, n, iters, sink, grid, s); break;
            case 3: err = launch_op<3>(depth, p, n, iters, sink, grid, s); break;
            case 4: err = launch_op<4>(depth, p, n, iters, sink, grid, s); break;
            case 5: err = launch_op<5>(depth, p, n, iters, sink, grid, s); break;
            case 6: err = launch_op<6>(depth, p, n, iters, sink, grid, s); break;
            case 7: err = launch_op<7>(depth, p, n, iters, sink, grid, s); break;
            case 8: err = launch_op<8>(depth, p, n, iters, sink, grid, s); break;
            case 9: err = launch_op<9>(depth, p, n, iters, sink, grid, s); break;
            case 10: err = launch_op<10>(depth, p, n, iters, sink, grid, s); break;
            default: err = launch_op<11>(depth, p, n, iters, sink, grid, s); break;
        }
    }
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess || ms <= 0.f) return -3.0;
    const int d = depth == 1 || depth == 2 || depth == 4 ? depth : 8;
    return (double)grid * 256.0 * (double)iters * (double)d / ((double)ms * 1e-3);
}
