// Batched propagation: many independent problems (instances) of uneven
// dimension and step count in one persistent launch.
//
// The host cuts every instance into `nblk` pieces (work items) sized by its
// cost, sorts the items by cost (largest first) and launches one block per SM.
// Each block repeatedly takes the next item from an atomic queue and runs the
// body that fits the instance's padded dimension: the warp-level fused body for
// D <= 16 (the item is one block's share of the instance's leaves), or the
// block-level body for D >= 32 (the item is one leaf).  Instances combine their
// pieces through per-instance pairwise arrival trees (the second arrival at a
// node multiplies, the first leaves), so no block ever waits for another and
// the item order is free.  The root of each instance's tree writes its U(T).
#pragma once

#include "pm_large.cuh"

namespace pm {

struct BatchItem {
    int inst, blk, nblk, Dp;
};

// per-instance set-up data for the basis kernel
struct BatchInst {
    const void *H0, *Hk;    // caller's device arrays (dtype of the call)
    int d, Dp, K, nb;
    size_t full_off;        // element offsets into the batch basis arrays
    size_t packed_off;
    size_t norm_off;
};

// One block per (instance, basis matrix): the FP64 basis matrix (H0, H_k, i[H0,H_k],
// i[H_a,H_b]; Sec. 4, Eq. magnus_coeffs), then its packed real form and FP64 1-norm.
template <typename InT, typename Real>
__global__ void batch_basis_kernel(const BatchInst *insts, const int2 *table, int magnus, double2 *full,
                                   Real *packed, double *norms) {
    const int2 te = table[blockIdx.x];
    const BatchInst bi = insts[te.x];
    const int e = te.y, d = bi.d, Dp = bi.Dp, K = bi.K;
    auto mat = [&](int raw) -> const InT * {
        return raw == 0 ? (const InT *)bi.H0 : (const InT *)bi.Hk + (size_t)(raw - 1) * d * d;
    };
    int a = -1, b = -1, src = -1;
    if (e < 1 + K) src = e;
    else if (e < 1 + 2 * K) { a = 0; b = e - K; }
    else {
        int pidx = e - (1 + 2 * K);
        for (int x = 0; x < K && a < 0; ++x) {
            const int cnt = K - 1 - x;
            if (pidx < cnt) { a = 1 + x; b = 2 + x + pidx; }
            else pidx -= cnt;
        }
    }
    (void)magnus;
    double2 *B = full + bi.full_off + (size_t)e * Dp * Dp;
    for (int t = threadIdx.x; t < Dp * Dp; t += blockDim.x) {
        const int i = t / Dp, j = t % Dp;
        double2 v = make_double2(0.0, 0.0);
        if (i < d && j < d) {
            if (src >= 0) {
                const InT x = mat(src)[i * d + j];
                v = make_double2((double)x.x, (double)x.y);
            } else {
                const InT *A = mat(a), *Bm = mat(b);
                double re = 0.0, im = 0.0;
                for (int l = 0; l < d; ++l) {
                    const double ax = A[i * d + l].x, ay = A[i * d + l].y;
                    const double bx = Bm[l * d + j].x, by = Bm[l * d + j].y;
                    const double cx = Bm[i * d + l].x, cy = Bm[i * d + l].y;
                    const double dx = A[l * d + j].x, dy = A[l * d + j].y;
                    re += ax * bx - ay * by - (cx * dx - cy * dy);
                    im += ax * by + ay * bx - (cx * dy + cy * dx);
                }
                v = make_double2(-im, re);  // i [A, B]
            }
        }
        B[t] = v;
    }
    __syncthreads();
    Real *P = packed + bi.packed_off + (size_t)e * Dp * Dp;
    for (int t = threadIdx.x; t < Dp * Dp; t += blockDim.x) {
        const int i = t / Dp, j = t % Dp;
        P[t] = (Real)((i <= j) ? B[t].x : B[t].y);
    }
    // 1-norm (max column sum of |B_ij|), widened by the FP32 rounding of the packed copy
    __shared__ double colsum[128];
    for (int j = threadIdx.x; j < Dp; j += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < Dp; ++i) s += hypot(B[i * Dp + j].x, B[i * Dp + j].y);
        colsum[j] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int j = 0; j < Dp; ++j) m = fmax(m, colsum[j]);
        norms[bi.norm_off + e] = m * (1.0 + 4.0 * 5.960464477539063e-08 * Dp);
    }
}

// The bodies run as separate (not inlined) functions: each keeps its own register allocation.
// Inlined into one switch they shared 255 registers and spilled 1.3 KB per thread, and the
// d = 64 items (most of the work of a mixed sweep) ran 1.5x slower than as single problems.
template <typename Real, int D, int INTEG>
static __device__ __noinline__ void batch_fused_item(const FusedParams &p, int blk, int nblk, unsigned char *smem) {
    fused_body<Real, D, INTEG>(p, blk, nblk, smem);
}

template <typename Real, int D, int INTEG, int TCM>
static __device__ __noinline__ void batch_large_item(const FusedParams &p, unsigned char *ws, int blk, int nblk,
                                                     unsigned char *smem, umma::Ctx *uc) {
    large_body<Real, D, INTEG, TCM>(p, (typename Cx<Real>::T *)ws, blk, nblk, smem, uc);
    large_arrival_tree<Real, D>(p, ws, blk, nblk, smem);
}

// the CUDA-core D = 64 items, inlined into the kernel: most of a mixed sweep's work, and as a
// separate function their products ran 20 % slower than in the single-problem kernel
template <typename Real, int D, int INTEG>
static __device__ __forceinline__ void batch_large_item_inl(const FusedParams &p, unsigned char *ws, int blk, int nblk,
                                                            unsigned char *smem) {
    large_body<Real, D, INTEG, 0>(p, (typename Cx<Real>::T *)ws, blk, nblk, smem, nullptr);
    large_arrival_tree<Real, D>(p, ws, blk, nblk, smem);
}

// D = 32 / 64 on the tensor cores: the shared-memory body of pm_tc_small.cuh, then the arrival tree
template <int D, int INTEG, int F>
static __device__ __noinline__ void batch_tc_item(const FusedParams &p, unsigned char *ws, int blk, int nblk,
                                                  unsigned char *smem, umma::Ctx *uc) {
    tcs::body<D, INTEG, F>(p, blk, nblk, smem, *uc);
    large_arrival_tree<float, D>(p, ws, blk, nblk, smem);
}

// TC: 0 = every product on the CUDA cores; 1 / 2 = D >= 32 products on the tcgen05 tensor cores in
// 3xTF32 / split BF16x3 (FP32 only), except for instances whose parameters set tc_off (the
// autotuner's choice for their dimension class).  A tensor-core kernel allocates the 512 columns
// of tensor memory once per block for all of its items.
template <typename Real, int INTEG, int TC>
__global__ void __launch_bounds__(256, 1) batched_kernel(const BatchItem *__restrict__ items, int n_items,
                                                         unsigned *queue, const FusedParams *__restrict__ params,
                                                         unsigned char *scratch, size_t scratch_stride,
                                                         unsigned *status) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    constexpr bool kTc = TC != 0 && std::is_same<Real, float>::value;
    constexpr int F = TC == 2 ? umma::kBF16x3 : umma::kTF32x3;
    __shared__ __align__(8) uint64_t s_mbar[umma::kBars];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    umma::Ctx cx;
    if constexpr (kTc) umma::setup(cx, s_mbar, &s_tmem, &s_abort, status);
    unsigned char *ws = scratch + (size_t)blockIdx.x * scratch_stride;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const BatchItem w = items[it];
        const FusedParams &p = params[w.inst];
        const bool tc = kTc && !p.tc_off;
        switch (w.Dp) {
            case 2: batch_fused_item<Real, 2, INTEG>(p, w.blk, w.nblk, smem); break;
            case 4: batch_fused_item<Real, 4, INTEG>(p, w.blk, w.nblk, smem); break;
            case 8: batch_fused_item<Real, 8, INTEG>(p, w.blk, w.nblk, smem); break;
            case 16: batch_fused_item<Real, 16, INTEG>(p, w.blk, w.nblk, smem); break;
            case 32:
                if constexpr (kTc) {
                    if (tc) {
                        batch_tc_item<32, INTEG, F>(p, ws, w.blk, w.nblk, smem, &cx);
                        break;
                    }
                }
                batch_large_item<Real, 32, INTEG, 0>(p, ws, w.blk, w.nblk, smem, nullptr);
                break;
            case 64:
                if constexpr (kTc) {
                    if (tc) {
                        batch_tc_item<64, INTEG, F>(p, ws, w.blk, w.nblk, smem, &cx);
                        break;
                    }
                }
                batch_large_item_inl<Real, 64, INTEG>(p, ws, w.blk, w.nblk, smem);
                break;
            case 128:
                if constexpr (kTc) {
                    if (tc) {
                        batch_large_item<Real, 128, INTEG, TC == 2 ? 3 : 2>(p, ws, w.blk, w.nblk, smem, &cx);
                        break;
                    }
                }
                batch_large_item<Real, 128, INTEG, 0>(p, ws, w.blk, w.nblk, smem, nullptr);
                break;
        }
        __syncthreads();
    }
    if constexpr (kTc) umma::teardown(cx);
}

template <typename Real, int INTEG, int TC>
cudaError_t launch_batched(const BatchItem *items, int n_items, unsigned *queue, const FusedParams *params,
                           unsigned char *scratch, size_t scratch_stride, int grid, size_t smem, unsigned *status,
                           cudaStream_t st) {
    auto k = batched_kernel<Real, INTEG, TC>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, 256, smem, st>>>(items, n_items, queue, params, scratch, scratch_stride, status);
    return cudaGetLastError();
}

template <typename Real, int INTEG, int TC>
int batched_occupancy_of(size_t smem) {
    int nb = 0;
    auto k = batched_kernel<Real, INTEG, TC>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 256, smem) != cudaSuccess) return 0;
    return nb;
}

}  // namespace pm
