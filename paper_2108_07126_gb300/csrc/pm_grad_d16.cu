// Instantiations of the gradient kernels for padded dimension 16.
#include "pm_grad.cuh"

namespace pm {

template <typename Real, int INTEG>
static cudaError_t adjoint_launch(const GradParams &gp, int grid, int warps, size_t smem, cudaStream_t st) {
    auto k = adjoint_kernel<Real, 16, INTEG>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, warps * 32, smem, st>>>(gp);
    return cudaGetLastError();
}

template <typename Real, int INTEG>
static int adjoint_occupancy(int warps, size_t smem) {
    int nb = 0;
    auto k = adjoint_kernel<Real, 16, INTEG>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, warps * 32, smem);
    return e == cudaSuccess ? nb : 0;
}

cudaError_t grad_run_d16(int fp64, int integ, const ScanParams &sp, const GradParams &gp, int grid, int warps,
                         size_t smem, cudaStream_t st) {
    scan_blocks_kernel<16><<<1, 256, 0, st>>>(sp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    scan_leaves_kernel<16><<<sp.n_blocks, 256, 0, st>>>(sp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    switch (integ * 2 + (fp64 ? 1 : 0)) {
        case 0: return adjoint_launch<float, kMidpoint>(gp, grid, warps, smem, st);
        case 1: return adjoint_launch<double, kMidpoint>(gp, grid, warps, smem, st);
        case 2: return adjoint_launch<float, kGL2>(gp, grid, warps, smem, st);
        case 3: return adjoint_launch<double, kGL2>(gp, grid, warps, smem, st);
        case 4: return adjoint_launch<float, kSimpson>(gp, grid, warps, smem, st);
        case 5: return adjoint_launch<double, kSimpson>(gp, grid, warps, smem, st);
    }
    return cudaErrorInvalidValue;
}

// exclusive prefixes and suffixes of every leaf from the forward pass's leaf and block products
cudaError_t scan_run_d16(const ScanParams &sp, cudaStream_t st) {
    scan_blocks_kernel<16><<<1, 256, 0, st>>>(sp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    scan_leaves_kernel<16><<<sp.n_blocks, 256, 0, st>>>(sp);
    return cudaGetLastError();
}

int adjoint_blocks_per_sm_d16(int fp64, int integ, int warps, size_t smem) {
    switch (integ * 2 + (fp64 ? 1 : 0)) {
        case 0: return adjoint_occupancy<float, kMidpoint>(warps, smem);
        case 1: return adjoint_occupancy<double, kMidpoint>(warps, smem);
        case 2: return adjoint_occupancy<float, kGL2>(warps, smem);
        case 3: return adjoint_occupancy<double, kGL2>(warps, smem);
        case 4: return adjoint_occupancy<float, kSimpson>(warps, smem);
        case 5: return adjoint_occupancy<double, kSimpson>(warps, smem);
    }
    return 0;
}

size_t adjoint_smem_d16(int fp64, int K, int warps) {
    return fp64 ? adjoint_smem_bytes<double, 16>(K, warps) : adjoint_smem_bytes<float, 16>(K, warps);
}

}  // namespace pm
