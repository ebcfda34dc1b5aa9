// Instantiations of the fused propagation kernel for padded dimension 8
// (mode cheb: 0 = Taylor exponential, 1 = Chebyshev exponential, 2 = Taylor trajectory).
#include "pm_fused.cuh"

namespace pm {

cudaError_t fused_dispatch_d8(int fp64, int integ, const FusedParams &p, int grid, int warps, size_t smem,
                               cudaStream_t st, int cheb) {
    switch (cheb * 6 + integ * 2 + (fp64 ? 1 : 0)) {
        case 0: return launch_fused<float, 8, kMidpoint>(p, grid, warps, smem, st);
        case 1: return launch_fused<double, 8, kMidpoint>(p, grid, warps, smem, st);
        case 2: return launch_fused<float, 8, kGL2>(p, grid, warps, smem, st);
        case 3: return launch_fused<double, 8, kGL2>(p, grid, warps, smem, st);
        case 4: return launch_fused<float, 8, kSimpson>(p, grid, warps, smem, st);
        case 5: return launch_fused<double, 8, kSimpson>(p, grid, warps, smem, st);
        case 6: return launch_fused<float, 8, kMidpoint, 1>(p, grid, warps, smem, st);
        case 7: return launch_fused<double, 8, kMidpoint, 1>(p, grid, warps, smem, st);
        case 8: return launch_fused<float, 8, kGL2, 1>(p, grid, warps, smem, st);
        case 9: return launch_fused<double, 8, kGL2, 1>(p, grid, warps, smem, st);
        case 10: return launch_fused<float, 8, kSimpson, 1>(p, grid, warps, smem, st);
        case 11: return launch_fused<double, 8, kSimpson, 1>(p, grid, warps, smem, st);
        case 12: return launch_fused<float, 8, kMidpoint, 2>(p, grid, warps, smem, st);
        case 13: return launch_fused<double, 8, kMidpoint, 2>(p, grid, warps, smem, st);
        case 14: return launch_fused<float, 8, kGL2, 2>(p, grid, warps, smem, st);
        case 15: return launch_fused<double, 8, kGL2, 2>(p, grid, warps, smem, st);
        case 16: return launch_fused<float, 8, kSimpson, 2>(p, grid, warps, smem, st);
        case 17: return launch_fused<double, 8, kSimpson, 2>(p, grid, warps, smem, st);
    }
    return cudaErrorInvalidValue;
}

int fused_blocks_per_sm_d8(int fp64, int integ, int warps, size_t smem, int cheb) {
    switch (cheb * 6 + integ * 2 + (fp64 ? 1 : 0)) {
        case 0: return fused_max_blocks_per_sm<float, 8, kMidpoint>(warps, smem);
        case 1: return fused_max_blocks_per_sm<double, 8, kMidpoint>(warps, smem);
        case 2: return fused_max_blocks_per_sm<float, 8, kGL2>(warps, smem);
        case 3: return fused_max_blocks_per_sm<double, 8, kGL2>(warps, smem);
        case 4: return fused_max_blocks_per_sm<float, 8, kSimpson>(warps, smem);
        case 5: return fused_max_blocks_per_sm<double, 8, kSimpson>(warps, smem);
        case 6: return fused_max_blocks_per_sm<float, 8, kMidpoint, 1>(warps, smem);
        case 7: return fused_max_blocks_per_sm<double, 8, kMidpoint, 1>(warps, smem);
        case 8: return fused_max_blocks_per_sm<float, 8, kGL2, 1>(warps, smem);
        case 9: return fused_max_blocks_per_sm<double, 8, kGL2, 1>(warps, smem);
        case 10: return fused_max_blocks_per_sm<float, 8, kSimpson, 1>(warps, smem);
        case 11: return fused_max_blocks_per_sm<double, 8, kSimpson, 1>(warps, smem);
        case 12: return fused_max_blocks_per_sm<float, 8, kMidpoint, 2>(warps, smem);
        case 13: return fused_max_blocks_per_sm<double, 8, kMidpoint, 2>(warps, smem);
        case 14: return fused_max_blocks_per_sm<float, 8, kGL2, 2>(warps, smem);
        case 15: return fused_max_blocks_per_sm<double, 8, kGL2, 2>(warps, smem);
        case 16: return fused_max_blocks_per_sm<float, 8, kSimpson, 2>(warps, smem);
        case 17: return fused_max_blocks_per_sm<double, 8, kSimpson, 2>(warps, smem);
    }
    return 0;
}

size_t fused_smem_d8(int fp64, int n_basis, int warps) {
    return fp64 ? fused_smem_bytes<double, 8>(n_basis, warps) : fused_smem_bytes<float, 8>(n_basis, warps);
}

int fused_groups_per_warp_d8(int fp64) { return fp64 ? Geo<double, 8>::GPW : Geo<float, 8>::GPW; }

int fused_max_warps_d8(int fp64) { return fp64 ? Geo<double, 8>::MAXW : Geo<float, 8>::MAXW; }

}  // namespace pm
