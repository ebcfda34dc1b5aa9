// Instantiations of the large-dimension propagation kernel for padded dimension 256.
#include "pm_grad_large.cuh"
#include "pm_large.cuh"

namespace pm {

cudaError_t large_dispatch_d256(int fp64, int integ, const FusedParams &p, void *scratch, int grid, size_t smem,
                               cudaStream_t st, int tc) {
    if (tc == 2 && !fp64) {  // split BF16x3 on tcgen05
        switch (integ) {
            case kMidpoint: return launch_large<float, 256, kMidpoint, 2>(p, scratch, grid, smem, st);
            case kGL2: return launch_large<float, 256, kGL2, 2>(p, scratch, grid, smem, st);
            case kSimpson: return launch_large<float, 256, kSimpson, 2>(p, scratch, grid, smem, st);
        }
        return cudaErrorInvalidValue;
    }
    if (tc && !fp64) {
        switch (integ) {
            case kMidpoint: return launch_large<float, 256, kMidpoint, 1>(p, scratch, grid, smem, st);
            case kGL2: return launch_large<float, 256, kGL2, 1>(p, scratch, grid, smem, st);
            case kSimpson: return launch_large<float, 256, kSimpson, 1>(p, scratch, grid, smem, st);
        }
        return cudaErrorInvalidValue;
    }
    switch (integ * 2 + (fp64 ? 1 : 0)) {
        case 0: return launch_large<float, 256, kMidpoint>(p, scratch, grid, smem, st);
        case 1: return launch_large<double, 256, kMidpoint>(p, scratch, grid, smem, st);
        case 2: return launch_large<float, 256, kGL2>(p, scratch, grid, smem, st);
        case 3: return launch_large<double, 256, kGL2>(p, scratch, grid, smem, st);
        case 4: return launch_large<float, 256, kSimpson>(p, scratch, grid, smem, st);
        case 5: return launch_large<double, 256, kSimpson>(p, scratch, grid, smem, st);
    }
    return cudaErrorInvalidValue;
}

int large_blocks_per_sm_d256(int fp64, int integ, size_t smem, int tc) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    auto q = [&](auto k) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kLargeThreads, smem);
    };
    if (tc == 2 && !fp64) {
        switch (integ) {
            case kMidpoint: q(large_kernel<float, 256, kMidpoint, 2>); break;
            case kGL2: q(large_kernel<float, 256, kGL2, 2>); break;
            case kSimpson: q(large_kernel<float, 256, kSimpson, 2>); break;
        }
        return e == cudaSuccess ? nb : 0;
    }
    if (tc && !fp64) {
        switch (integ) {
            case kMidpoint: q(large_kernel<float, 256, kMidpoint, 1>); break;
            case kGL2: q(large_kernel<float, 256, kGL2, 1>); break;
            case kSimpson: q(large_kernel<float, 256, kSimpson, 1>); break;
        }
        return e == cudaSuccess ? nb : 0;
    }
    switch (integ * 2 + (fp64 ? 1 : 0)) {
        case 0: q(large_kernel<float, 256, kMidpoint>); break;
        case 1: q(large_kernel<double, 256, kMidpoint>); break;
        case 2: q(large_kernel<float, 256, kGL2>); break;
        case 3: q(large_kernel<double, 256, kGL2>); break;
        case 4: q(large_kernel<float, 256, kSimpson>); break;
        case 5: q(large_kernel<double, 256, kSimpson>); break;
    }
    return e == cudaSuccess ? nb : 0;
}

cudaError_t large_prefix_d256(const double2 *leaf, int n, double2 *a, double2 *b, double2 **x, cudaStream_t st) {
    return leaf_prefixes<256>(leaf, n, a, b, x, st);
}

size_t large_smem_d256(int fp64, int n_basis, int tc) {
    if (fp64) return large_smem_bytes<double, 256>(n_basis);
    if (tc == 2) return large_smem_bytes<float, 256, large_tcm<float, 256, 2>()>(n_basis);
    return tc ? large_smem_bytes<float, 256, large_tcm<float, 256, 1>()>(n_basis) : large_smem_bytes<float, 256>(n_basis);
}

cudaError_t grad_large_run_d256(int fp64, int integ, const double2 *leaf, int L, double2 *pre, double2 *suf,
                               const GradParams &gp, void *scratch, void *U_out, int out_c128, int d_out,
                               cudaStream_t st) {
    return grad_large_run<256>(fp64, integ, leaf, L, pre, suf, gp, scratch, U_out, out_c128, d_out, st);
}

size_t adjoint_large_smem_d256(int fp64) {
    return fp64 ? adjoint_large_smem_bytes<double, 256>() : adjoint_large_smem_bytes<float, 256>();
}

}  // namespace pm
