// epoch_kernels.cu -- launchers of one epoch (Algorithm 1, Section 3.3):
// the HOGWILD modes with uniform negatives, the multi-handle epoch of
// continuous batching, and the synchronous mode.  The kernels are in
// epoch_device.cuh; weighted negatives are instantiated in epoch_weighted.cu
// and epochs that report the actual energy in epoch_energy.cu, so that the
// three translation units compile in parallel.
#include "epoch_device.cuh"

namespace snap {

cudaError_t launch_oriented_epoch(const OrientedArgs &a, int red_mode, int grid, int block, cudaStream_t s) {
    if (a.energy) return launch_oriented_energy(a, red_mode, grid, block, s);
    if (a.alias) return launch_oriented_weighted(a, red_mode, grid, block, s);
    const bool multi = a.graphs != nullptr;
    if (red_mode)
        return multi ? launch_oriented_k<true, true, false, false>(a, grid, block, s)
                     : launch_oriented_k<true, false, false, false>(a, grid, block, s);
    return multi ? launch_oriented_k<false, true, false, false>(a, grid, block, s)
                 : launch_oriented_k<false, false, false, false>(a, grid, block, s);
}

int oriented_blocks_per_sm(int red_mode, int k, int block, int multi, int weighted) {
    if (weighted) return oriented_weighted_blocks_per_sm(red_mode, k, block, multi);
    if (red_mode)
        return multi ? oriented_occupancy_k<true, true, false, false>(k, block)
                     : oriented_occupancy_k<true, false, false, false>(k, block);
    return multi ? oriented_occupancy_k<false, true, false, false>(k, block)
                 : oriented_occupancy_k<false, false, false, false>(k, block);
}

cudaError_t launch_multi_epoch(const MultiArgs &a, int red_mode, int weighted, int grid, int block,
                               cudaStream_t s) {
    if (weighted) return launch_multi_weighted(a, red_mode, grid, block, s);
    return red_mode ? launch_multi_k<true, false>(a, grid, block, s) : launch_multi_k<false, false>(a, grid, block, s);
}

int multi_blocks_per_sm(int red_mode, int weighted, int k, int block) {
    if (weighted) return multi_weighted_blocks_per_sm(red_mode, k, block);
    return red_mode ? multi_occupancy_k<true, false>(k, block) : multi_occupancy_k<false, false>(k, block);
}

cudaError_t launch_sync_chunk(const SyncArgs &a, int grid, int block, cudaStream_t s) {
    if (a.graphs)
        sync_chunk_kernel<true><<<grid, block, 0, s>>>(a);
    else
        sync_chunk_kernel<false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sync_apply(float2 *pos, long long *disp, int32_t n, float eta, float limit,
                              uint32_t *status, int grid, int block, cudaStream_t s, const int32_t *node_graph,
                              const GraphInfo *graphs, int32_t tick, float cap) {
    if (graphs)
        sync_apply_kernel<true><<<grid, block, 0, s>>>(pos, disp, n, eta, limit, status, node_graph, graphs, tick, cap);
    else
        sync_apply_kernel<false><<<grid, block, 0, s>>>(pos, disp, n, eta, limit, status, nullptr, nullptr, 0, 0.0f);
    return cudaGetLastError();
}

int sync_blocks_per_sm(int block) { return occupancy_of(sync_chunk_kernel<false>, block); }

}  // namespace snap
