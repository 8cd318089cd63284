// epoch_energy.cu -- HOGWILD epochs of a single graph that also sum the
// actual energy of the epoch (Section 3.3: the energy of the pairs the epoch
// visits and draws, each taken at the moment of its update), uniform or
// weighted negatives.  Kernels in epoch_device.cuh.
#include "epoch_device.cuh"

namespace snap {

cudaError_t launch_oriented_energy(const OrientedArgs &a, int red_mode, int grid, int block, cudaStream_t s) {
    if (a.alias)
        return red_mode ? launch_oriented_k<true, false, true, true>(a, grid, block, s)
                        : launch_oriented_k<false, false, true, true>(a, grid, block, s);
    return red_mode ? launch_oriented_k<true, false, false, true>(a, grid, block, s)
                    : launch_oriented_k<false, false, false, true>(a, grid, block, s);
}

int oriented_energy_blocks_per_sm(int red_mode, int k, int block, int weighted) {
    if (weighted)
        return red_mode ? oriented_occupancy_k<true, false, true, true>(k, block)
                        : oriented_occupancy_k<false, false, true, true>(k, block);
    return red_mode ? oriented_occupancy_k<true, false, false, true>(k, block)
                    : oriented_occupancy_k<false, false, false, true>(k, block);
}

}  // namespace snap
