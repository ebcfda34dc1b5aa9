// Instantiation of the batched propagation kernel: float, integrator kMidpoint, CUDA-core products.
#include "pm_batched.cuh"

namespace pm {

cudaError_t batched_launch_fm(const BatchItem *items, int n_items, unsigned *queue, const FusedParams *params,
                              unsigned char *scratch, size_t stride, int grid, size_t smem, unsigned *status,
                              cudaStream_t st) {
    return launch_batched<float, kMidpoint, 0>(items, n_items, queue, params, scratch, stride, grid, smem, status, st);
}

int batched_blocks_per_sm_fm(size_t smem) { return batched_occupancy_of<float, kMidpoint, 0>(smem); }

cudaError_t batch_basis_launch(int c128, int fp64, const BatchInst *insts, const int2 *table, int n_mats, int magnus,
                               double2 *full, void *packed, double *norms, cudaStream_t st) {
    if (n_mats <= 0) return cudaSuccess;
    if (c128 && fp64)
        batch_basis_kernel<double2, double><<<n_mats, 256, 0, st>>>(insts, table, magnus, full, (double *)packed, norms);
    else if (c128)
        batch_basis_kernel<double2, float><<<n_mats, 256, 0, st>>>(insts, table, magnus, full, (float *)packed, norms);
    else if (fp64)
        batch_basis_kernel<float2, double><<<n_mats, 256, 0, st>>>(insts, table, magnus, full, (double *)packed, norms);
    else
        batch_basis_kernel<float2, float><<<n_mats, 256, 0, st>>>(insts, table, magnus, full, (float *)packed, norms);
    return cudaGetLastError();
}

}  // namespace pm
