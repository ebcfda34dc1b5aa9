// Fused propagation kernel for padded dimensions D in {2, 4, 8, 16}.
//
// One launch computes U(T) = U_N ... U_1 (Sec. 2, Eq. slices):
//   1. every group of lanes owns one leaf: a contiguous range of slices;
//   2. per slice: effective coefficients from the control samples (Sec. 4,
//      Eq. magnus_coeffs for the Magnus exponents), the FP64 norm bound
//      nu_j = sum_e |gamma_e| ||B_e||_1 >= ||G_j||_1 (Sec. 3.2, per slice),
//      the exponent G_j = sum_e gamma_e B_e from the shared-memory basis,
//      exp(-i G_j) by a Taylor polynomial of degree m evaluated with
//      Paterson-Stockmeyer on A = -i G_j / 2^s, then s squarings;
//   3. leaf product R <- U_j R (later slices on the left);
//   4. leaves of a block combined pairwise in shared memory (Sec. 2.2);
//   5. block partials combined pairwise in FP64 through global memory: the
//      second block to arrive at a tree node multiplies, the first leaves.
//      No block ever waits for another one.
#pragma once

#include "pm_common.cuh"

namespace pm {

// Lane tiling of one D x D complex product over the LANES lanes of a group.
// Lane (rb, cb) owns rows rb + r * (D/TR) and columns cb + c * (D/TC).
template <int D> struct Tiling;
template <> struct Tiling<2> { static constexpr int LANES = 1, TR = 2, TC = 2, LD = 2; };
template <> struct Tiling<4> { static constexpr int LANES = 2, TR = 2, TC = 4, LD = 4; };
template <> struct Tiling<8> { static constexpr int LANES = 8, TR = 2, TC = 4, LD = 9; };
template <> struct Tiling<16> { static constexpr int LANES = 32, TR = 2, TC = 4, LD = 17; };

template <int D> struct Geo {
    using T = Tiling<D>;
    static constexpr int LANES = T::LANES, TR = T::TR, TC = T::TC, LD = T::LD;
    static constexpr int GPW = 32 / LANES;   // groups per warp
    static constexpr int RBN = D / TR;       // row stride of a lane's rows
    static constexpr int CBN = D / TC;       // column stride of a lane's columns
    static constexpr int DD = D * D;
    static constexpr int SLOT = ((D * LD + 1) / 2) * 2;  // complex elements per slot, even
    static constexpr int NSLOT = 5;                      // X, X^2, X^3, T (work), R (leaf product)
};

// smem bytes of one warp's workspace for a given basis size
template <typename Real, int D>
__host__ __device__ inline size_t warp_ws_bytes(int n_basis) {
    using G = Geo<D>;
    size_t slots = (size_t)G::GPW * G::NSLOT * G::SLOT * sizeof(typename Cx<Real>::T);
    size_t gam = (size_t)n_basis * 32 * sizeof(Real);
    size_t cls = 32 * sizeof(int);
    return (slots + gam + cls + 15) & ~(size_t)15;
}

template <typename Real, int D>
__host__ __device__ inline size_t basis_smem_bytes(int n_basis) {
    size_t b = (size_t)n_basis * D * D * sizeof(Real) + (size_t)n_basis * sizeof(double);
    return (b + 15) & ~(size_t)15;
}

template <typename Real, int D>
__host__ __device__ inline size_t fused_smem_bytes(int n_basis, int warps) {
    return basis_smem_bytes<Real, D>(n_basis) + (size_t)warps * warp_ws_bytes<Real, D>(n_basis);
}

// acc = A * B for the lane's tile; A, B are D x D complex matrices with row stride LD
template <typename Real, int D>
__device__ __forceinline__ void mm_tile(const typename Cx<Real>::T *__restrict__ A,
                                        const typename Cx<Real>::T *__restrict__ B, int rb, int cb,
                                        typename Cx<Real>::T (&acc)[Geo<D>::TR][Geo<D>::TC]) {
    using G = Geo<D>;
    using C = typename Cx<Real>::T;
#pragma unroll
    for (int r = 0; r < G::TR; ++r)
#pragma unroll
        for (int c = 0; c < G::TC; ++c) acc[r][c] = Cx<Real>::make(0, 0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        C a[G::TR], b[G::TC];
#pragma unroll
        for (int r = 0; r < G::TR; ++r) a[r] = A[(rb + r * G::RBN) * G::LD + k];
#pragma unroll
        for (int c = 0; c < G::TC; ++c) b[c] = B[k * G::LD + cb + c * G::CBN];
#pragma unroll
        for (int r = 0; r < G::TR; ++r)
#pragma unroll
            for (int c = 0; c < G::TC; ++c) cfma(acc[r][c], a[r], b[c]);
    }
}

template <typename Real, int D>
__device__ __forceinline__ void st_tile(typename Cx<Real>::T *S, int rb, int cb,
                                        const typename Cx<Real>::T (&t)[Geo<D>::TR][Geo<D>::TC]) {
    using G = Geo<D>;
#pragma unroll
    for (int r = 0; r < G::TR; ++r)
#pragma unroll
        for (int c = 0; c < G::TC; ++c) S[(rb + r * G::RBN) * G::LD + cb + c * G::CBN] = t[r][c];
}

template <typename Real> __device__ __forceinline__ Real coef(const FusedParams &p, int k);
template <> __device__ __forceinline__ float coef<float>(const FusedParams &p, int k) { return p.coef_f[k]; }
template <> __device__ __forceinline__ double coef<double>(const FusedParams &p, int k) { return p.coef_d[k]; }

// Effective coefficients gamma_e of one slice (Sec. 4, Eq. magnus_coeffs with the
// commutator sign of Omega_2): basis order H0, H_k, i[H0,H_k], i[H_k,H_k'] (k < k').
template <typename Real, int INTEG>
__device__ __forceinline__ void slice_coefficients(const FusedParams &p, int64_t j, bool active,
                                                   Real *gam /* stride 32 */) {
    const Real *c = (const Real *)p.ctrl;
    const int K = p.K;
    const Real h = (Real)p.dt;
    if (!active) {
        for (int e = 0; e < p.n_basis; ++e) gam[e * 32] = Real(0);
        return;
    }
    gam[0] = h;
    if (INTEG == kMidpoint) {
        for (int k = 0; k < K; ++k) gam[(1 + k) * 32] = h * c[(int64_t)k * p.S + j];
        return;
    }
    Real c1[kMaxControls], c2[kMaxControls];
    Real w1, wc;  // weight of the averaged controls and of the commutators
    if (INTEG == kGL2) {
        for (int k = 0; k < K; ++k) {
            c1[k] = c[(int64_t)k * p.S + 2 * j];
            c2[k] = c[(int64_t)k * p.S + 2 * j + 1];
            gam[(1 + k) * 32] = (h * Real(0.5)) * (c1[k] + c2[k]);
        }
        wc = (Real)(1.7320508075688772 / 12.0) * h * h;
        (void)w1;
    } else {  // Simpson: c1 = start, c2 = end; centre sample only in Omega_1
        for (int k = 0; k < K; ++k) {
            const Real a = c[(int64_t)k * p.S + 2 * j];
            const Real m = c[(int64_t)k * p.S + 2 * j + 1];
            const Real b = c[(int64_t)k * p.S + 2 * j + 2];
            c1[k] = a;
            c2[k] = b;
            gam[(1 + k) * 32] = (h / Real(6)) * (a + Real(4) * m + b);
        }
        wc = h * h / Real(12);
        (void)w1;
    }
    for (int k = 0; k < K; ++k) gam[(1 + K + k) * 32] = wc * (c2[k] - c1[k]);
    int e = 1 + 2 * K;
    for (int k = 0; k < K; ++k)
        for (int l = k + 1; l < K; ++l, ++e) gam[e * 32] = wc * (c1[k] * c2[l] - c2[k] * c1[l]);
}

// Class index for a norm bound: first class with cap >= nu (binary search in FP64).
__device__ __forceinline__ int find_class(const FusedParams &p, double nu, unsigned *flags) {
    const int n = p.n_cls;
    if (!(nu <= p.cls_cap[n - 1])) {
        *flags |= (isnan(nu) || isinf(nu)) ? kDevNonfinite : kDevCapped;
        return n - 1;
    }
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (nu <= p.cls_cap[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

template <typename Real, int D, int INTEG>
__global__ void __launch_bounds__(256) fused_small_kernel(const FusedParams p) {
    using G = Geo<D>;
    using C = typename Cx<Real>::T;
    constexpr int LANES = G::LANES, GPW = G::GPW, TR = G::TR, TC = G::TC, LD = G::LD, DD = G::DD;
    constexpr int SLOT = G::SLOT, NSLOT = G::NSLOT;

    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_second;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int g = lane / LANES, gl = lane % LANES;
    const int rb = gl / G::CBN, cb = gl % G::CBN;
    const int nb = p.n_basis;

    Real *basis = (Real *)smem;
    double *bnorm = (double *)(basis + (size_t)nb * DD);
    const size_t boff = basis_smem_bytes<Real, D>(nb);
    const size_t wsb = warp_ws_bytes<Real, D>(nb);
    unsigned char *wbase = smem + boff + (size_t)warp * wsb;
    C *slots = (C *)wbase + (size_t)g * NSLOT * SLOT;
    C *S1 = slots, *S2 = slots + SLOT, *S3 = slots + 2 * SLOT, *ST = slots + 3 * SLOT, *SR = slots + 4 * SLOT;
    Real *gam = (Real *)(wbase + (size_t)GPW * NSLOT * SLOT * sizeof(C));
    int *cls = (int *)(gam + (size_t)nb * 32);

    // ---- basis and its norms into shared memory
    {
        const Real *src = (const Real *)p.packed;
        for (int i = tid; i < nb * DD; i += blockDim.x) basis[i] = src[i];
        for (int i = tid; i < nb; i += blockDim.x) bnorm[i] = p.bnorm1[i];
    }

    // ---- leaf of this group
    const int64_t n_leaves = (int64_t)gridDim.x * W * GPW;
    const int64_t leaf = ((int64_t)blockIdx.x * W + warp) * GPW + g;
    const int64_t j0 = p.n_steps * leaf / n_leaves;
    const int len = (int)(p.n_steps * (leaf + 1) / n_leaves - j0);
    const int wlen = (int)__reduce_max_sync(0xffffffffu, (unsigned)len);

    // R = I
    {
        C t[TR][TC];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c)
                t[r][c] = Cx<Real>::make((rb + r * G::RBN) == (cb + c * G::CBN) ? Real(1) : Real(0), Real(0));
        st_tile<Real, D>(SR, rb, cb, t);
    }
    __syncthreads();

    unsigned flags = 0;
    unsigned long long n_exp = 0, n_tree = 0;
    int m_max = 0, s_max = 0;

    for (int t0 = 0; t0 < wlen; t0 += LANES) {
        // -- tile preparation: lane gl handles slice j0 + t0 + gl of its group
        {
            const bool act = (t0 + gl) < len;
            Real *gcol = gam + lane;
            slice_coefficients<Real, INTEG>(p, j0 + t0 + gl, act, gcol);
            double nu = 0.0;
            for (int e = 0; e < nb; ++e) nu = fma(fabs((double)gcol[e * 32]), bnorm[e], nu);
            cls[lane] = find_class(p, nu, &flags);
        }
        __syncwarp();
        const int nr = min(LANES, wlen - t0);
        for (int rr = 0; rr < nr; ++rr) {
            const int cw = (int)__reduce_max_sync(0xffffffffu, (unsigned)cls[g * LANES + rr]);
            const int code = p.cls_code[cw];
            const int q = cls_q(code), rh = cls_r(code);
            const int s = cls_s(code) + p.extra_squarings;

            // -- exponent: packed G = sum_e gamma_e P_e (lane's tile of the packed array)
            Real gp[TR][TC];
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TC; ++c) gp[r][c] = Real(0);
            {
                const Real *gcol = gam + g * LANES + rr;
                for (int e = 0; e < nb; ++e) {
                    const Real ge = gcol[e * 32];
                    const Real *Pe = basis + e * DD;
#pragma unroll
                    for (int r = 0; r < TR; ++r)
#pragma unroll
                        for (int c = 0; c < TC; ++c)
                            gp[r][c] = fma(ge, Pe[(rb + r * G::RBN) * D + cb + c * G::CBN], gp[r][c]);
                }
            }
            Real *gpk = (Real *)ST;
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TC; ++c) gpk[(rb + r * G::RBN) * D + cb + c * G::CBN] = gp[r][c];
            __syncwarp();

            // -- unpack the Hermitian G into A = -i G / 2^s (row stride LD)
            const Real sc = (Real)ldexp(1.0, -s);
            C x1[TR][TC], x2[TR][TC], x3[TR][TC];
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TC; ++c) {
                    const int i = rb + r * G::RBN, jj = cb + c * G::CBN;
                    const Real re = (i <= jj) ? gpk[i * D + jj] : gpk[jj * D + i];
                    const Real im = (i > jj) ? gpk[i * D + jj] : ((i < jj) ? -gpk[jj * D + i] : Real(0));
                    x1[r][c] = Cx<Real>::make(im * sc, -re * sc);
                }
            __syncwarp();
            st_tile<Real, D>(S1, rb, cb, x1);
            __syncwarp();

            // -- powers X^2, X^3
            if (q >= 2) {
                mm_tile<Real, D>(S1, S1, rb, cb, x2);
                st_tile<Real, D>(S2, rb, cb, x2);
                __syncwarp();
            }
            if (q >= 3) {
                mm_tile<Real, D>(S2, S1, rb, cb, x3);
                st_tile<Real, D>(S3, rb, cb, x3);
                __syncwarp();
            }
            const C *Sq = (q == 1) ? S1 : ((q == 2) ? S2 : S3);

            // -- Horner over blocks: T = a_{q r} X^q + B_{r-1}; T = X^q T + B_b
            //    with B_b = sum_{l<q} a_{q b + l} X^l
            C tt[TR][TC];
            {
                const Real atop = coef<Real>(p, q * rh);
#pragma unroll
                for (int r = 0; r < TR; ++r)
#pragma unroll
                    for (int c = 0; c < TC; ++c) {
                        const C xq = (q == 1) ? x1[r][c] : ((q == 2) ? x2[r][c] : x3[r][c]);
                        tt[r][c] = Cx<Real>::make(atop * xq.x, atop * xq.y);
                    }
            }
            for (int b = rh - 1; b >= 0; --b) {
                if (b < rh - 1) {
                    st_tile<Real, D>(ST, rb, cb, tt);
                    __syncwarp();
                    mm_tile<Real, D>(Sq, ST, rb, cb, tt);
                    __syncwarp();
                }
                const Real a0 = coef<Real>(p, q * b);
                const Real a1 = (q >= 2) ? coef<Real>(p, q * b + 1) : Real(0);
                const Real a2 = (q >= 3) ? coef<Real>(p, q * b + 2) : Real(0);
#pragma unroll
                for (int r = 0; r < TR; ++r)
#pragma unroll
                    for (int c = 0; c < TC; ++c) {
                        const bool diag = (rb + r * G::RBN) == (cb + c * G::CBN);
                        C v = tt[r][c];
                        if (q == 1) {
                            v.x = fma(a0, diag ? Real(1) : Real(0), v.x);
                        } else {
                            v.x = fma(a1, x1[r][c].x, v.x + (diag ? a0 : Real(0)));
                            v.y = fma(a1, x1[r][c].y, v.y);
                            if (q >= 3) {
                                v.x = fma(a2, x2[r][c].x, v.x);
                                v.y = fma(a2, x2[r][c].y, v.y);
                            }
                        }
                        tt[r][c] = v;
                    }
            }

            // -- squarings
            for (int i = 0; i < s; ++i) {
                st_tile<Real, D>(ST, rb, cb, tt);
                __syncwarp();
                mm_tile<Real, D>(ST, ST, rb, cb, tt);
                __syncwarp();
            }

            // -- leaf product R <- U_j R
            st_tile<Real, D>(ST, rb, cb, tt);
            __syncwarp();
            mm_tile<Real, D>(ST, SR, rb, cb, tt);
            __syncwarp();
            st_tile<Real, D>(SR, rb, cb, tt);
            __syncwarp();

            if (gl == 0 && (t0 + rr) < len) {
                n_exp += (unsigned long long)((q - 1) + (rh - 1) + s);
                n_tree += 1;
                m_max = max(m_max, cls_m(code));
                s_max = max(s_max, s);
            }
        }
        __syncwarp();
    }

    // ---- statistics and status (before this block's tree arrival)
    if (gl == 0) {
        if (n_tree) {
            atomicAdd(&p.counters[0], n_exp);
            atomicAdd(&p.counters[1], n_tree);
            atomicMax(&p.counters[2], (unsigned long long)m_max);
            atomicMax(&p.counters[3], (unsigned long long)s_max);
        }
    }
    if (flags) atomicOr(&p.status[0], flags);

    // ---- in-block pairwise tree over the leaves (Sec. 2.2): leaf l+h is later than leaf l
    __syncthreads();
    const int n_leaf = W * GPW;
    const int gid = warp * GPW + g;  // block-wide group id
    auto leaf_R = [&](int l) -> C * {
        return (C *)(smem + boff + (size_t)(l / GPW) * wsb) + (size_t)(l % GPW) * NSLOT * SLOT + 4 * SLOT;
    };
    for (int h = 1; h < n_leaf; h <<= 1) {
        const int left = gid * 2 * h;
        const bool v = left + h < n_leaf;
        C acc[TR][TC];
        if (v) mm_tile<Real, D>(leaf_R(left + h), leaf_R(left), rb, cb, acc);
        __syncthreads();
        if (v) st_tile<Real, D>(leaf_R(left), rb, cb, acc);
        __syncthreads();
    }

    // ---- block partial in FP64 to global memory
    {
        const C *R0 = leaf_R(0);
        double2 *dst = p.partials + (size_t)blockIdx.x * DD;
        for (int t = tid; t < DD; t += blockDim.x) {
            const C v = R0[(t / D) * LD + (t % D)];
            dst[t] = make_double2((double)v.x, (double)v.y);
        }
    }
    __threadfence();
    __syncthreads();

    // ---- pairwise tree over blocks: second arrival at a node multiplies right * left
    using GD = Geo<D>;
    double2 *bufL = (double2 *)(smem + boff);  // warp 0's workspace, free by now
    double2 *bufR = bufL + D * LD;
    int idx = blockIdx.x, n = gridDim.x, level = 0, toff = 0;
    while (n > 1) {
        const int parent = idx >> 1;
        if ((idx | 1) < n) {
            if (tid == 0) s_second = (atomicAdd(&p.tickets[toff + parent], 1u) != 0u);
            __syncthreads();
            if (!s_second) return;
            if (tid == 0) p.tickets[toff + parent] = 0u;  // ready for the next launch
            __threadfence();
            const double2 *gL = p.partials + (size_t)((idx & ~1) << level) * DD;
            const double2 *gR = p.partials + (size_t)((idx | 1) << level) * DD;
            for (int t = tid; t < DD; t += blockDim.x) {
                bufL[(t / D) * LD + t % D] = __ldcg(gL + t);
                bufR[(t / D) * LD + t % D] = __ldcg(gR + t);
            }
            __syncthreads();
            if (warp == 0 && g == 0) {
                double2 acc[GD::TR][GD::TC];
                mm_tile<double, D>(bufR, bufL, rb, cb, acc);
                double2 *dst = p.partials + (size_t)((idx & ~1) << level) * DD;
#pragma unroll
                for (int r = 0; r < GD::TR; ++r)
#pragma unroll
                    for (int c = 0; c < GD::TC; ++c)
                        __stcg(dst + (rb + r * GD::RBN) * D + cb + c * GD::CBN, acc[r][c]);
            }
            __threadfence();
            __syncthreads();
        }
        idx = parent;
        n = (n + 1) >> 1;
        toff += n;
        ++level;
    }

    // ---- root: U(T) to the output buffer, statistics snapshot
    {
        const int d = p.d_out;
        for (int t = tid; t < d * d; t += blockDim.x) {
            const double2 v = __ldcg(p.partials + (t / d) * D + (t % d));
            if (p.out_c128) ((double2 *)p.U_out)[t] = v;
            else ((float2 *)p.U_out)[t] = make_float2((float)v.x, (float)v.y);
        }
        if (tid == 0) {
            __threadfence();
            for (int i = 0; i < 4; ++i) {
                p.counters[4 + i] = atomicExch(&p.counters[i], 0ull);
            }
            p.status[1] = atomicExch(&p.status[0], 0u);
        }
    }
}

// host-side launcher (explicitly instantiated per D in pm_fused_d*.cu)
template <typename Real, int D, int INTEG>
cudaError_t launch_fused(const FusedParams &p, int grid, int warps, size_t smem, cudaStream_t st) {
    auto k = fused_small_kernel<Real, D, INTEG>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, warps * 32, smem, st>>>(p);
    return cudaGetLastError();
}

template <typename Real, int D, int INTEG>
int fused_max_blocks_per_sm(int warps, size_t smem) {
    int nb = 0;
    auto k = fused_small_kernel<Real, D, INTEG>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, warps * 32, smem) != cudaSuccess) return 0;
    return nb;
}

}  // namespace pm
