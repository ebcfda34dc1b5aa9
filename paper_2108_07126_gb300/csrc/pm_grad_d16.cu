// Instantiations of the gradient kernels for padded dimension 16.
#include "pm_grad.cuh"

namespace pm {

cudaError_t grad_run_d16(int fp64, const ScanParams &sp, const GradParams &gp, int grid, int warps, size_t smem,
                         cudaStream_t st) {
    scan_blocks_kernel<16><<<1, 256, 0, st>>>(sp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    scan_leaves_kernel<16><<<sp.n_blocks, 256, 0, st>>>(sp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (fp64) {
        auto k = adjoint_kernel<double, 16>;
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        k<<<grid, warps * 32, smem, st>>>(gp);
    } else {
        auto k = adjoint_kernel<float, 16>;
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        k<<<grid, warps * 32, smem, st>>>(gp);
    }
    return cudaGetLastError();
}

// exclusive prefixes and suffixes of every leaf from the forward pass's leaf and block products
cudaError_t scan_run_d16(const ScanParams &sp, cudaStream_t st) {
    scan_blocks_kernel<16><<<1, 256, 0, st>>>(sp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    scan_leaves_kernel<16><<<sp.n_blocks, 256, 0, st>>>(sp);
    return cudaGetLastError();
}

int adjoint_blocks_per_sm_d16(int fp64, int warps, size_t smem) {
    int nb = 0;
    cudaError_t e;
    if (fp64) {
        auto k = adjoint_kernel<double, 16>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, warps * 32, smem);
    } else {
        auto k = adjoint_kernel<float, 16>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, warps * 32, smem);
    }
    return e == cudaSuccess ? nb : 0;
}

size_t adjoint_smem_d16(int fp64, int K, int warps) {
    return fp64 ? adjoint_smem_bytes<double, 16>(K, warps) : adjoint_smem_bytes<float, 16>(K, warps);
}

}  // namespace pm
