// Instantiation of the batched propagation kernel: float, integrator kMidpoint, tensor cores true.
#include "pm_batched.cuh"

namespace pm {

cudaError_t batched_launch_fm_tc(const BatchItem *items, int n_items, unsigned *queue, const FusedParams *params,
                                 unsigned char *scratch, size_t stride, int grid, size_t smem, cudaStream_t st) {
    return launch_batched<float, kMidpoint, true>(items, n_items, queue, params, scratch, stride, grid, smem, st);
}

int batched_blocks_per_sm_fm_tc(size_t smem) {
    int nb = 0;
    auto k = batched_kernel<float, kMidpoint, true>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 256, smem) != cudaSuccess) return 0;
    return nb;
}

}  // namespace pm
