// Instantiation of the batched propagation kernel: float, integrator kGL2, split BF16x3 tensor-core products.
#include "pm_batched.cuh"

namespace pm {

cudaError_t batched_launch_fg_bf(const BatchItem *items, int n_items, unsigned *queue, const FusedParams *params,
                              unsigned char *scratch, size_t stride, int grid, size_t smem, unsigned *status,
                              cudaStream_t st) {
    return launch_batched<float, kGL2, 2>(items, n_items, queue, params, scratch, stride, grid, smem, status, st);
}

int batched_blocks_per_sm_fg_bf(size_t smem) { return batched_occupancy_of<float, kGL2, 2>(smem); }

}  // namespace pm
