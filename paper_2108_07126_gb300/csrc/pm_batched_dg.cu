// Instantiation of the batched propagation kernel: double, integrator kGL2, CUDA-core products.
#include "pm_batched.cuh"

namespace pm {

cudaError_t batched_launch_dg(const BatchItem *items, int n_items, unsigned *queue, const FusedParams *params,
                              unsigned char *scratch, size_t stride, int grid, size_t smem, unsigned *status,
                              cudaStream_t st) {
    return launch_batched<double, kGL2, 0>(items, n_items, queue, params, scratch, stride, grid, smem, status, st);
}

int batched_blocks_per_sm_dg(size_t smem) { return batched_occupancy_of<double, kGL2, 0>(smem); }

}  // namespace pm
