// Instantiation of the batched propagation kernel: float, integrator kMidpoint, 3xTF32 tensor-core products.
#include "pm_batched.cuh"

namespace pm {

cudaError_t batched_launch_fm_tc(const BatchItem *items, int n_items, unsigned *queue, const FusedParams *params,
                              unsigned char *scratch, size_t stride, int grid, size_t smem, unsigned *status,
                              cudaStream_t st) {
    return launch_batched<float, kMidpoint, 1>(items, n_items, queue, params, scratch, stride, grid, smem, status, st);
}

int batched_blocks_per_sm_fm_tc(size_t smem) { return batched_occupancy_of<float, kMidpoint, 1>(smem); }

}  // namespace pm
