// Internal helpers of pm_api.cu shared with other translation units of the library.
#pragma once

#include "pm_common.cuh"

namespace pm {

// Taylor class table and 1/k! coefficients for unit roundoff u (force_m = 0: any degree).
int fill_classes(double u, int force_m, FusedParams &p);

// Fused propagation kernel for padded dimension Dp (2, 4, 8, 16).
cudaError_t fused_launch(int Dp, int fp64, int integ, const FusedParams &p, int grid, int warps, size_t smem,
                         cudaStream_t st);
int fused_occupancy(int Dp, int fp64, int integ, int warps, size_t smem);
size_t fused_smem_size(int Dp, int fp64, int n_basis, int warps);
int fused_groups(int Dp, int fp64);

// Basis of set_hamiltonians from raw[1 + K][d][d] (complex128 if c128, else complex64):
// full FP64 basis, packed FP64 / FP32 forms, FP64 1-norms and max-abs per matrix.
cudaError_t basis_build(const void *raw, int c128, int d, int Dp, int K, int magnus, int nb, double2 *full,
                        double *p64, float *p32, double *bnorm, double *bmax, cudaStream_t st);

}  // namespace pm
