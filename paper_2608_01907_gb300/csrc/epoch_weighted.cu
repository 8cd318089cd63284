// epoch_weighted.cu -- HOGWILD epochs with weighted negatives (degree or
// caller weights through an alias table; see sampler.cpp), single graphs,
// batches and multi-handle epochs.  Kernels in epoch_device.cuh.
#include "epoch_device.cuh"

namespace snap {

cudaError_t launch_oriented_weighted(const OrientedArgs &a, int red_mode, int grid, int block, cudaStream_t s) {
    const bool multi = a.graphs != nullptr;
    if (red_mode)
        return multi ? launch_oriented_k<true, true, true, false>(a, grid, block, s)
                     : launch_oriented_k<true, false, true, false>(a, grid, block, s);
    return multi ? launch_oriented_k<false, true, true, false>(a, grid, block, s)
                 : launch_oriented_k<false, false, true, false>(a, grid, block, s);
}

int oriented_weighted_blocks_per_sm(int red_mode, int k, int block, int multi) {
    if (red_mode)
        return multi ? oriented_occupancy_k<true, true, true, false>(k, block)
                     : oriented_occupancy_k<true, false, true, false>(k, block);
    return multi ? oriented_occupancy_k<false, true, true, false>(k, block)
                 : oriented_occupancy_k<false, false, true, false>(k, block);
}

cudaError_t launch_multi_weighted(const MultiArgs &a, int red_mode, int grid, int block, cudaStream_t s) {
    return red_mode ? launch_multi_k<true, true>(a, grid, block, s) : launch_multi_k<false, true>(a, grid, block, s);
}

int multi_weighted_blocks_per_sm(int red_mode, int k, int block) {
    return red_mode ? multi_occupancy_k<true, true>(k, block) : multi_occupancy_k<false, true>(k, block);
}

}  // namespace snap
