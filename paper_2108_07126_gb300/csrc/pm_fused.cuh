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
//
// Shared-memory layout per block: the packed basis (row stride D) and its
// norms, then per warp: GPW groups x 4 complex D x LD slots (X / Horner
// operand, X^2, X^3, leaf product R), the second packed exponent of a pair
// (FP32 d = 16 only), the coefficient tile and class tile.  The FP32 d = 16
// Taylor path keeps the slots in the row / column chunk layouts of
// pm_pp16.cuh while a leaf runs and converts the leaf product to the slot
// layout for the tree.
#pragma once

#include <type_traits>

#include "pm_common.cuh"
#include "pm_pp16.cuh"

namespace pm {

// Lane tiling of one D x D complex product over the LANES lanes of a group.
// Lane (rb, cb) owns rows rb + r * RBN (r < TR) and columns col(cb, c) (c < TC);
// V complex numbers move per shared-memory access (V = 2: 16-byte float4).
template <typename Real, int D> struct Tiling;
// MAXW: most warps of a standalone fused block (its launch bound; the host picks fewer when the
// shared memory does not fit them).
template <> struct Tiling<float, 16> { static constexpr int LANES = 32, TR = 4, TC = 2, LD = 18, V = 2, GPAD = 16, MAXW = 12; };
template <> struct Tiling<float, 8> { static constexpr int LANES = 4, TR = 4, TC = 4, LD = 8, V = 2, GPAD = 16, MAXW = 8; };
template <> struct Tiling<float, 4> { static constexpr int LANES = 1, TR = 4, TC = 4, LD = 4, V = 2, GPAD = 16, MAXW = 8; };
template <> struct Tiling<float, 2> { static constexpr int LANES = 1, TR = 2, TC = 2, LD = 2, V = 2, GPAD = 16, MAXW = 8; };
template <> struct Tiling<double, 16> { static constexpr int LANES = 32, TR = 2, TC = 4, LD = 17, V = 1, GPAD = 0, MAXW = 8; };
template <> struct Tiling<double, 8> { static constexpr int LANES = 8, TR = 2, TC = 4, LD = 9, V = 1, GPAD = 16, MAXW = 8; };
template <> struct Tiling<double, 4> { static constexpr int LANES = 2, TR = 2, TC = 4, LD = 4, V = 1, GPAD = 16, MAXW = 8; };
template <> struct Tiling<double, 2> { static constexpr int LANES = 1, TR = 2, TC = 2, LD = 2, V = 1, GPAD = 16, MAXW = 8; };

template <typename Real, int D> struct Geo {
    using T = Tiling<Real, D>;
    using C = typename Cx<Real>::T;
    static constexpr int LANES = T::LANES, TR = T::TR, TC = T::TC, LD = T::LD, V = T::V, MAXW = T::MAXW;
    static constexpr int GPW = 32 / LANES;        // groups per warp
    static constexpr int RBN = D / TR;            // row blocks: rows rb + r * RBN
    static constexpr int CBW = D / TC;            // column blocks
    static constexpr int DD = D * D;
    static constexpr int SLOT = D * LD;           // complex elements per slot
    static constexpr int NSLOT = 4;               // X (then Horner operand), X^2, X^3, R
    static constexpr int GSTRIDE = NSLOT * SLOT * (int)sizeof(C) + T::GPAD;  // bytes per group
    static constexpr int NCH = DD / (4 * LANES);  // 4-entry chunks of the packed exponent per lane
    // row stride of the packed exponent scratch (FP32 d = 16: 19, fewest bank conflicts for the
    // assembly's stores and the packed-FMA path's transposed unpack reads together)
    static constexpr int PS = (sizeof(Real) == 4 && D == 16) ? 19 : ((D >= 4) ? D + 1 : D);
    // slices assembled per pass over the shared-memory basis: the FP32 d = 16 kernel is bound by
    // shared-memory wavefronts, and assembling two slices per pass halves the basis reads of the
    // assembly; the second packed exponent waits in a buffer of XB bytes per group
    static constexpr int APASS = (sizeof(Real) == 4 && D == 16) ? 2 : 1;
    static constexpr int XB = APASS == 2 ? ((D * PS * (int)sizeof(Real) + 15) & ~15) : 0;
    static_assert(LANES == RBN * CBW, "tiling must cover the matrix");
    static_assert(NCH >= 1 && NCH * 4 * LANES == DD, "assembly chunks must cover the matrix");
    static_assert(TC % V == 0 && LD % V == 0, "vector accesses must stay aligned");
    __host__ __device__ static constexpr int col(int cb, int c) { return V == 2 ? cb * TC + c : cb + c * CBW; }
};

template <typename Real, int D>
__host__ __device__ inline size_t warp_ws_bytes(int n_basis) {
    using G = Geo<Real, D>;
    size_t b = (size_t)G::GPW * (G::GSTRIDE + G::XB) + (size_t)n_basis * 32 * sizeof(Real) + 32 * sizeof(int);
    return (b + 15) & ~(size_t)15;
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

// ---------------------------------------------------------------- tile primitives

template <typename C, int V> struct Vec;
template <> struct Vec<float2, 2> {
    __device__ static inline void ld(const float2 *p, float2 (&o)[2]) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        o[0] = make_float2(v.x, v.y);
        o[1] = make_float2(v.z, v.w);
    }
    __device__ static inline void st(float2 *p, const float2 a, const float2 b) {
        *reinterpret_cast<float4 *>(p) = make_float4(a.x, a.y, b.x, b.y);
    }
};
template <typename C> struct Vec<C, 1> {
    __device__ static inline void ld(const C *p, C (&o)[1]) { o[0] = *p; }
};

// acc = A * B for the lane's tile; A, B are D x D complex matrices with row stride LD
template <typename Real, int D>
__device__ __forceinline__ void mm_tile(const typename Cx<Real>::T *__restrict__ A,
                                        const typename Cx<Real>::T *__restrict__ B, int rb, int cb,
                                        typename Cx<Real>::T (&acc)[Geo<Real, D>::TR][Geo<Real, D>::TC]) {
    using G = Geo<Real, D>;
    using C = typename G::C;
    constexpr int TR = G::TR, TC = G::TC, V = G::V, LD = G::LD;
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
        for (int c = 0; c < TC; ++c) acc[r][c] = Cx<Real>::make(0, 0);
#pragma unroll
    for (int k = 0; k < D; k += V) {
        C a[TR][V], b[V][TC];
#pragma unroll
        for (int r = 0; r < TR; ++r) Vec<C, V>::ld(A + (rb + r * G::RBN) * LD + k, a[r]);
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int c = 0; c < TC; c += V) {
                C t[V];
                Vec<C, V>::ld(B + (k + v) * LD + G::col(cb, c), t);
#pragma unroll
                for (int w = 0; w < V; ++w) b[v][c + w] = t[w];
            }
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TC; ++c) cfma(acc[r][c], a[r][v], b[v][c]);
    }
}

// acc += A * B
template <typename Real, int D>
__device__ __forceinline__ void mm_tile_add(const typename Cx<Real>::T *__restrict__ A,
                                            const typename Cx<Real>::T *__restrict__ B, int rb, int cb,
                                            typename Cx<Real>::T (&acc)[Geo<Real, D>::TR][Geo<Real, D>::TC]) {
    using G = Geo<Real, D>;
    using C = typename G::C;
    constexpr int TR = G::TR, TC = G::TC, V = G::V, LD = G::LD;
#pragma unroll
    for (int k = 0; k < D; k += V) {
        C a[TR][V], b[V][TC];
#pragma unroll
        for (int r = 0; r < TR; ++r) Vec<C, V>::ld(A + (rb + r * G::RBN) * LD + k, a[r]);
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int c = 0; c < TC; c += V) {
                C t[V];
                Vec<C, V>::ld(B + (k + v) * LD + G::col(cb, c), t);
#pragma unroll
                for (int w = 0; w < V; ++w) b[v][c + w] = t[w];
            }
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TC; ++c) cfma(acc[r][c], a[r][v], b[v][c]);
    }
}

template <typename Real, int D>
__device__ __forceinline__ void st_tile(typename Cx<Real>::T *S, int rb, int cb,
                                        const typename Cx<Real>::T (&t)[Geo<Real, D>::TR][Geo<Real, D>::TC]) {
    using G = Geo<Real, D>;
#pragma unroll
    for (int r = 0; r < G::TR; ++r) {
        if constexpr (G::V == 2) {
#pragma unroll
            for (int c = 0; c < G::TC; c += 2)
                Vec<float2, 2>::st(S + (rb + r * G::RBN) * G::LD + G::col(cb, c), t[r][c], t[r][c + 1]);
        } else {
#pragma unroll
            for (int c = 0; c < G::TC; ++c) S[(rb + r * G::RBN) * G::LD + G::col(cb, c)] = t[r][c];
        }
    }
}

template <typename Real> __device__ __forceinline__ Real coef(const FusedParams &p, int k);
template <> __device__ __forceinline__ float coef<float>(const FusedParams &p, int k) { return p.coef_f[k]; }
template <> __device__ __forceinline__ double coef<double>(const FusedParams &p, int k) { return p.coef_d[k]; }

template <typename Real> __device__ __forceinline__ Real pow2neg(int s);
template <> __device__ __forceinline__ float pow2neg<float>(int s) { return __int_as_float((127 - s) << 23); }
template <> __device__ __forceinline__ double pow2neg<double>(int s) {
    return __longlong_as_double((long long)(1023 - s) << 52);
}

// Effective coefficients gamma_e of one slice (Sec. 4, Eq. magnus_coeffs with the
// commutator sign of Omega_2): basis order H0, H_k, i[H0,H_k], i[H_k,H_k'] (k < k').
// P: any parameter block with ctrl, S, K, dt, n_basis and slot_of (FusedParams, GradParams).
template <typename Real, int INTEG, int STRIDE = 32, typename P = FusedParams>
__device__ __forceinline__ void slice_coefficients(const P &p, int64_t j, bool active, Real *gam) {
    const Real *c = (const Real *)p.ctrl;
    const int K = p.K;
    const Real h = (Real)p.dt;
    if (!active) {
        for (int e = 0; e < p.n_basis; ++e) gam[e * STRIDE] = Real(0);
        return;
    }
    // coefficients of identically zero basis matrices are dropped
    auto put = [&](int e, Real v) {
        const int sl = p.slot_of[e];
        if (sl >= 0) gam[sl * STRIDE] = v;
    };
    put(0, h);
    if (INTEG == kMidpoint) {
        for (int k = 0; k < K; ++k) put(1 + k, h * c[(int64_t)k * p.S + j]);
        return;
    }
    Real c1[kMaxControls], c2[kMaxControls];
    Real wc;  // weight of the commutator coefficients
    if (INTEG == kGL2) {
        for (int k = 0; k < K; ++k) {
            c1[k] = c[(int64_t)k * p.S + 2 * j];
            c2[k] = c[(int64_t)k * p.S + 2 * j + 1];
            put(1 + k, (h * Real(0.5)) * (c1[k] + c2[k]));
        }
        wc = (Real)(1.7320508075688772 / 12.0) * h * h;
    } else {  // Simpson: c1 = slice start, c2 = slice end; the centre sample enters Omega_1 only
        for (int k = 0; k < K; ++k) {
            const Real a = c[(int64_t)k * p.S + 2 * j];
            const Real m = c[(int64_t)k * p.S + 2 * j + 1];
            const Real b = c[(int64_t)k * p.S + 2 * j + 2];
            c1[k] = a;
            c2[k] = b;
            put(1 + k, (h / Real(6)) * (a + Real(4) * m + b));
        }
        wc = h * h / Real(12);
    }
    for (int k = 0; k < K; ++k) put(1 + K + k, wc * (c2[k] - c1[k]));
    int e = 1 + 2 * K;
    for (int k = 0; k < K; ++k)
        for (int l = k + 1; l < K; ++l, ++e) put(e, wc * (c1[k] * c2[l] - c2[k] * c1[l]));
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

// 4 consecutive packed entries of a basis matrix
template <typename Real> __device__ __forceinline__ void ld4(const Real *p, Real (&o)[4]);
template <> __device__ __forceinline__ void ld4<float>(const float *p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <> __device__ __forceinline__ void ld4<double>(const double *p, double (&o)[4]) {
    const double2 a = *reinterpret_cast<const double2 *>(p);
    const double2 b = *reinterpret_cast<const double2 *>(p + 2);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

// The whole propagation of one problem, executed by thread block `blk` of the
// `nblk` blocks assigned to it (the grid of fused_small_kernel, or the blocks
// of one instance of the batched kernel).  smem: the dynamic shared memory.
// EXPM: 0 = Taylor exponential, 1 = Chebyshev exponential, 2 = Taylor in
// trajectory mode (every leaf starts from its exclusive prefix p.traj_pin and
// writes U(t_n) or psi(t_n) at the output slices; no tree, no statistics).
template <typename Real, int D, int INTEG, int EXPM = 0>
__device__ __forceinline__ void fused_body(const FusedParams &p, int blk, int nblk, unsigned char *smem) {
    using G = Geo<Real, D>;
    using C = typename G::C;
    constexpr int LANES = G::LANES, GPW = G::GPW, TR = G::TR, TC = G::TC, LD = G::LD, DD = G::DD;
    constexpr int SLOT = G::SLOT, NCH = G::NCH, PS = G::PS;
    constexpr int AP = EXPM == 2 ? 1 : G::APASS;  // slices assembled per pass over the basis
    // FP32 d = 16 Taylor path: the products run on packed two-wide FMAs (pm_pp16.cuh) with the
    // working matrices in its row / column layouts; the leaf product is kept in the column layout
    // and converted to the slot layout of the tree after the last slice of the leaf
    constexpr bool PP = std::is_same<Real, float>::value && D == 16 && EXPM == 0;
    static_assert(!PP || G::SLOT * (int)sizeof(C) >= pp16::MAT_BYTES, "a slot holds one pp16 matrix");

    __shared__ int s_second;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int W = (p.warps > 0 && p.warps < (int)(blockDim.x >> 5)) ? p.warps : (int)(blockDim.x >> 5);
    const bool active_warp = warp < W;  // warps beyond W own no leaf and no shared workspace
    const int g = lane / LANES, gl = lane % LANES;
    const int rb = gl / G::CBW, cb = gl % G::CBW;
    const int nb = p.n_basis;

    Real *basis = (Real *)smem;
    double *bnorm = (double *)(basis + (size_t)nb * DD);
    const size_t boff = basis_smem_bytes<Real, D>(nb);
    const size_t wsb = warp_ws_bytes<Real, D>(nb);
    unsigned char *wbase = smem + boff + (size_t)warp * wsb;
    C *slots = (C *)(wbase + (size_t)g * G::GSTRIDE);
    C *S1 = slots, *S2 = slots + SLOT, *S3 = slots + 2 * SLOT, *SR = slots + 3 * SLOT;
    Real *xpk = (Real *)(wbase + (size_t)GPW * G::GSTRIDE + (size_t)g * G::XB);  // second packed exponent
    Real *gam = (Real *)(wbase + (size_t)GPW * (G::GSTRIDE + G::XB));
    int *cls = (int *)(gam + (size_t)nb * 32);

    // ---- basis and its norms into shared memory
    {
        const Real *src = (const Real *)p.packed;
        for (int i = tid; i < nb * DD; i += blockDim.x) basis[i] = src[i];
        for (int i = tid; i < nb; i += blockDim.x) bnorm[i] = p.bnorm1[i];
    }

    // ---- leaf of this group
    const int64_t n_leaves = (int64_t)nblk * W * GPW;
    const int64_t leaf = ((int64_t)blk * W + warp) * GPW + g;
    const int64_t j0 = active_warp ? p.n_steps * leaf / n_leaves : 0;
    const int len = active_warp ? (int)(p.n_steps * (leaf + 1) / n_leaves - j0) : 0;
    const int wlen = (int)__reduce_max_sync(0xffffffffu, (unsigned)len);

    // R = I (trajectory mode: R = the product of all slices before the leaf)
    if (active_warp) {
        C t[TR][TC];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c) {
                const int i = rb + r * G::RBN, jj = G::col(cb, c);
                if constexpr (EXPM == 2) {
                    const double2 v = p.traj_pin[(size_t)leaf * DD + i * D + jj];
                    t[r][c] = Cx<Real>::make((Real)v.x, (Real)v.y);
                } else {
                    t[r][c] = Cx<Real>::make(i == jj ? Real(1) : Real(0), Real(0));
                }
            }
        if constexpr (PP) {
            pp16::Tile id;
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    id.re[r][c] = pp16::orow(lane >> 3, r) == 2 * (lane & 7) + c ? 1.f : 0.f;
                    id.im[r][c] = 0.f;
                }
            pp16::st_col(reinterpret_cast<float4 *>(SR), lane >> 3, lane & 7, id);
        } else {
            st_tile<Real, D>(SR, rb, cb, t);
        }
    }
    __syncthreads();

    // trajectory mode: after slice j, R = U(t_{j+1}); keep it at the output slices
    auto traj_emit = [&](int64_t j, const C (&R)[TR][TC]) {
        const int64_t n1 = j + 1;
        if (n1 % p.traj_every != 0 && n1 != p.n_steps) return;
        const int64_t o = j / p.traj_every;
        const int d = p.d_out;
        if (p.traj_psi0 == nullptr) {
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TC; ++c) {
                    const int i = rb + r * G::RBN, jj = G::col(cb, c);
                    if (i < d && jj < d) {
                        const size_t at = ((size_t)o * d + i) * d + jj;
                        if (p.out_c128) ((double2 *)p.traj_out)[at] = make_double2((double)R[r][c].x, (double)R[r][c].y);
                        else ((float2 *)p.traj_out)[at] = make_float2((float)R[r][c].x, (float)R[r][c].y);
                    }
                }
        } else {  // psi(t_n) = R psi_0, rows gl, gl + LANES, ... (R is in SR)
            for (int i = gl; i < d; i += LANES) {
                Real re = 0, im = 0;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const C a = SR[i * LD + k];
                    const double2 b = p.traj_psi0[k];
                    re = fma(a.x, (Real)b.x, fma(-a.y, (Real)b.y, re));
                    im = fma(a.x, (Real)b.y, fma(a.y, (Real)b.x, im));
                }
                const size_t at = (size_t)o * d + i;
                if (p.out_c128) ((double2 *)p.traj_out)[at] = make_double2((double)re, (double)im);
                else ((float2 *)p.traj_out)[at] = make_float2((float)re, (float)im);
            }
        }
    };

    unsigned flags = 0;
    unsigned long long n_exp = 0, n_tree = 0;
    int m_max = 0, s_max = 0;

    for (int t0 = 0; t0 < wlen; t0 += LANES) {
        // -- tile preparation: lane gl handles slice j0 + t0 + gl of its group
        {
            const bool act = (t0 + gl) < len;
            Real *gcol = gam + lane;
            slice_coefficients<Real, INTEG>(p, j0 + t0 + gl, act, gcol);
            if (EXPM != 1) {
                double nu = 0.0;
                for (int e = 0; e < nb; ++e) nu = fma(fabs((double)gcol[e * 32]), bnorm[e], nu);
                cls[lane] = find_class(p, nu, &flags);
            } else {
                cls[lane] = 0;  // Chebyshev: one global degree, fixed before the launch
            }
        }
        __syncwarp();
        const int nr = min(LANES, wlen - t0);
        for (int rr = 0; rr < nr; ++rr) {
            const int cw = (int)__reduce_max_sync(0xffffffffu, (unsigned)cls[g * LANES + rr]);
            const int code = p.cls_code[cw];
            const int q = cls_q(code), rh = cls_r(code);
            const int s = cls_s(code) + p.extra_squarings;

            // -- exponent in packed form: lane owns chunks gl + LANES * t of 4 entries.  With two
            //    slices per pass (AP = 2; not in trajectory mode, whose registers are full) the even
            //    slice of a pair also assembles the odd one into xpk, and the odd slice starts there.
            const bool second = AP == 2 && (rr & 1);
            const bool both = AP == 2 && !(rr & 1) && rr + 1 < nr;
            const Real *gpk = second ? xpk : (const Real *)S2;  // S2 is scratch until X^2 is formed
            if (!second) {
                Real acc[NCH][4], acc2[AP == 2 ? NCH : 1][4];
#pragma unroll
                for (int t = 0; t < NCH; ++t)
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[t][u] = Real(0);
                const Real *gcol = gam + g * LANES + rr;
                bool two = false;
                if constexpr (AP == 2) two = both;
                if (two) {
#pragma unroll
                    for (int t = 0; t < (int)(sizeof(acc2) / sizeof(acc2[0])); ++t)
#pragma unroll
                        for (int u = 0; u < 4; ++u) acc2[t][u] = Real(0);
                    for (int e = 0; e < nb; ++e) {
                        Real ge[2];  // slices rr and rr + 1 (rr is even: one 8-byte load)
                        if constexpr (AP == 2) {
                            const float2 gv = *reinterpret_cast<const float2 *>(gcol + e * 32);
                            ge[0] = gv.x;
                            ge[1] = gv.y;
                        }
                        const Real *Pe = basis + e * DD;
#pragma unroll
                        for (int t = 0; t < NCH; ++t) {
                            Real v[4];
                            ld4<Real>(Pe + 4 * (gl + LANES * t), v);
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                acc[t][u] = fma(ge[0], v[u], acc[t][u]);
                                if constexpr (AP == 2) acc2[t][u] = fma(ge[1], v[u], acc2[t][u]);
                            }
                        }
                    }
                } else {
                    for (int e = 0; e < nb; ++e) {
                        const Real ge = gcol[e * 32];
                        const Real *Pe = basis + e * DD;
#pragma unroll
                        for (int t = 0; t < NCH; ++t) {
                            Real v[4];
                            ld4<Real>(Pe + 4 * (gl + LANES * t), v);
#pragma unroll
                            for (int u = 0; u < 4; ++u) acc[t][u] = fma(ge, v[u], acc[t][u]);
                        }
                    }
                }
                Real *dst = (Real *)S2;
#pragma unroll
                for (int t = 0; t < NCH; ++t)
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int pos = 4 * (gl + LANES * t) + u;
                        dst[(pos / D) * PS + (pos % D)] = acc[t][u];
                        if constexpr (AP == 2)
                            if (two) xpk[(pos / D) * PS + (pos % D)] = acc2[t][u];
                    }
            }
            __syncwarp();

            if constexpr (PP) {
                // -- packed-pair products (pm_pp16.cuh).  Slots: S1 = R(X), S2 = R(X^2), S3 = R(X^3);
                //    the Horner / squaring operand T takes the two slots that the powers leave free
                //    (Ta: C(T), Tb: R(T)); SR holds C(R) of the leaf product.
                using pp16::Tile;
                const int pa = lane >> 3, pb = lane & 7;
                float4 *M1 = reinterpret_cast<float4 *>(S1), *M2 = reinterpret_cast<float4 *>(S2);
                float4 *M3 = reinterpret_cast<float4 *>(S3), *MR = reinterpret_cast<float4 *>(SR);
                const Real sc = pow2neg<Real>(s);
                Tile x1, x2, tt;
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int i = pp16::orow(pa, r), jj = 2 * pb + c;
                        const Real va = gpk[i * PS + jj], vb = gpk[jj * PS + i];
                        const Real re = (i <= jj) ? va : vb;
                        const Real im = (i > jj) ? va : ((i < jj) ? -vb : Real(0));
                        x1.re[r][c] = im * sc;
                        x1.im[r][c] = -re * sc;
                        x2.re[r][c] = x2.im[r][c] = 0.f;
                    }
                pp16::st_row(M1, pa, pb, x1);
                __syncwarp();

                const Real atop = coef<Real>(p, q * rh);
                const float4 *Mq = (q == 1) ? M1 : ((q == 2) ? M2 : M3);
                float4 *Ta = (q == 1) ? M2 : M1;
                float4 *Tb = (q == 3) ? M2 : M3;
                auto add_block = [&](int bl) {
                    const Real a0 = coef<Real>(p, q * bl);
                    const Real a1 = (q >= 2) ? coef<Real>(p, q * bl + 1) : Real(0);
                    const Real a2 = (q >= 3) ? coef<Real>(p, q * bl + 2) : Real(0);
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            const bool diag = pp16::orow(pa, r) == 2 * pb + c;
                            Real vr = tt.re[r][c] + (diag ? a0 : Real(0)), vi = tt.im[r][c];
                            if (q >= 2) {
                                vr = fma(a1, x1.re[r][c], vr);
                                vi = fma(a1, x1.im[r][c], vi);
                            }
                            if (q >= 3) {
                                vr = fma(a2, x2.re[r][c], vr);
                                vi = fma(a2, x2.im[r][c], vi);
                            }
                            tt.re[r][c] = vr;
                            tt.im[r][c] = vi;
                        }
                };
                auto start_horner = [&](const Tile &top) {
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            tt.re[r][c] = atop * top.re[r][c];
                            tt.im[r][c] = atop * top.im[r][c];
                        }
                    add_block(rh - 1);
                };
                const int n_pow = q - 1, n_hor = rh - 1;
                const int n_prod = n_pow + n_hor + s + 1;
                int bl = rh - 1;
                if (n_pow == 0) start_horner(x1);
                for (int pi = 0; pi < n_prod; ++pi) {
                    Tile acc;
                    if (pi < n_pow) {
                        // X^2 = X X, X^3 = X^2 X: B = X from its row layout (anti-Hermitian)
                        pp16::mm<true>(pi == 0 ? M1 : M2, M1, pa, pb, acc);
                        if (pi == 0) {
                            x2 = acc;
                            pp16::st_row(M2, pa, pb, acc);
                        } else {
                            pp16::st_row(M3, pa, pb, acc);
                        }
                        if (pi == n_pow - 1) start_horner(acc);
                        __syncwarp();
                        continue;
                    }
                    // T in the layouts the next product reads: C(T) as the right operand of a
                    // Horner step or squaring, R(T) as the left operand of a squaring or the leaf
                    const bool leafp = pi == n_prod - 1;
                    const bool horner = pi < n_pow + n_hor;
                    if (!leafp) pp16::st_col(Ta, pa, pb, tt);
                    if (!horner) pp16::st_row(Tb, pa, pb, tt);
                    __syncwarp();
                    //   T <- X^q T + B_b, T <- T T, R <- T R (later slice on the left)
                    pp16::mm<false>(horner ? Mq : Tb, leafp ? MR : Ta, pa, pb, acc);
                    __syncwarp();
                    if (leafp) {
                        pp16::st_col(MR, pa, pb, acc);
                        __syncwarp();
                    } else {
                        tt = acc;
                        if (horner) add_block(--bl);
                    }
                }
                if (gl == 0 && (t0 + rr) < len) {
                    n_exp += (unsigned long long)((q - 1) + (rh - 1) + s);
                    n_tree += 1;
                    m_max = max(m_max, cls_m(code));
                    s_max = max(s_max, s);
                }
                continue;
            }


            if constexpr (EXPM == 1) {
                // -- Chebyshev (Sec. 2.1, Algorithm 1): X = G / beta, D_k = a_k I + 2 X D_{k+1} - D_{k+2},
                //    exp(-i G) ~ D_0 - D_2; one product per degree, then the leaf product
                const Real ib = (Real)*p.cheb_inv_beta;
                const int mch = *p.cheb_m;
                const C *ak = (const C *)p.cheb_coef;
                C dk1[TR][TC], dk2[TR][TC], U[TR][TC];
#pragma unroll
                for (int r = 0; r < TR; ++r)
#pragma unroll
                    for (int c = 0; c < TC; ++c) {
                        const int i = rb + r * G::RBN, jj = G::col(cb, c);
                        const Real a = gpk[i * PS + jj], b = gpk[jj * PS + i];
                        const Real re = (i <= jj) ? a : b;
                        const Real im = (i > jj) ? a : ((i < jj) ? -b : Real(0));
                        U[r][c] = Cx<Real>::make(re * ib, im * ib);
                    }
                st_tile<Real, D>(S1, rb, cb, U);
                {
                    const C am = ak[mch];
#pragma unroll
                    for (int r = 0; r < TR; ++r)
#pragma unroll
                        for (int c = 0; c < TC; ++c) {
                            const bool diag = (rb + r * G::RBN) == G::col(cb, c);
                            dk1[r][c] = diag ? am : Cx<Real>::make(0, 0);
                            dk2[r][c] = Cx<Real>::make(0, 0);
                        }
                }
                __syncwarp();
                for (int k = mch - 1; k >= 0; --k) {
                    st_tile<Real, D>(S2, rb, cb, dk1);
                    __syncwarp();
                    C acc[TR][TC];
                    mm_tile<Real, D>(S1, S2, rb, cb, acc);
                    __syncwarp();
                    const C a_k = ak[k];
#pragma unroll
                    for (int r = 0; r < TR; ++r)
#pragma unroll
                        for (int c = 0; c < TC; ++c) {
                            const bool diag = (rb + r * G::RBN) == G::col(cb, c);
                            C v = Cx<Real>::make(Real(2) * acc[r][c].x - dk2[r][c].x,
                                                 Real(2) * acc[r][c].y - dk2[r][c].y);
                            if (diag) {
                                v.x += a_k.x;
                                v.y += a_k.y;
                            }
                            if (k == 0) {
                                U[r][c] = Cx<Real>::make(v.x - dk2[r][c].x, v.y - dk2[r][c].y);
                            } else {
                                dk2[r][c] = dk1[r][c];
                                dk1[r][c] = v;
                            }
                        }
                }
                // leaf product R <- U_j R (skipped for padding slices, which would multiply by ~I)
                st_tile<Real, D>(S2, rb, cb, U);
                __syncwarp();
                {
                    C acc[TR][TC];
                    mm_tile<Real, D>(S2, SR, rb, cb, acc);
                    __syncwarp();
                    if ((t0 + rr) < len) st_tile<Real, D>(SR, rb, cb, acc);
                    __syncwarp();
                }
                if (gl == 0 && (t0 + rr) < len) {
                    n_exp += (unsigned long long)mch;
                    n_tree += 1;
                    m_max = max(m_max, mch);
                }
                continue;
            }

            // -- unpack the Hermitian G into A = -i G / 2^s at the lane's tile
            const Real sc = pow2neg<Real>(s);
            C x1[TR][TC], x2[TR][TC], tt[TR][TC];
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TC; ++c) {
                    const int i = rb + r * G::RBN, jj = G::col(cb, c);
                    const Real a = gpk[i * PS + jj], b = gpk[jj * PS + i];
                    const Real re = (i <= jj) ? a : b;
                    const Real im = (i > jj) ? a : ((i < jj) ? -b : Real(0));
                    x1[r][c] = Cx<Real>::make(im * sc, -re * sc);
                }
            st_tile<Real, D>(S1, rb, cb, x1);
            __syncwarp();

            // -- every complex product of the slice goes through one call site (one copy of
            //    the unrolled product in the instruction stream):
            //      X^2 (q >= 2), X^3 (q >= 3)           powers of X = A
            //      T <- X^q T + B_b  (rh - 1 times)     Horner over blocks, with
            //                                           T = a_{q rh} X^q + B_{rh-1} to start and
            //                                           B_b = sum_{l<q} a_{q b + l} X^l
            //      T <- T T          (s times)          squarings
            //      R <- T R                             leaf product (later slice on the left)
            const Real atop = coef<Real>(p, q * rh);
            const C *Sq = (q == 1) ? S1 : ((q == 2) ? S2 : S3);
            C *ST = (q == 1) ? S2 : S1;  // operand slot of Horner, squarings and the leaf product
            auto add_block = [&](int b) {
                const Real a0 = coef<Real>(p, q * b);
                const Real a1 = (q >= 2) ? coef<Real>(p, q * b + 1) : Real(0);
                const Real a2 = (q >= 3) ? coef<Real>(p, q * b + 2) : Real(0);
#pragma unroll
                for (int r = 0; r < TR; ++r)
#pragma unroll
                    for (int c = 0; c < TC; ++c) {
                        const bool diag = (rb + r * G::RBN) == G::col(cb, c);
                        C v = tt[r][c];
                        v.x += diag ? a0 : Real(0);
                        if (q >= 2) {
                            v.x = fma(a1, x1[r][c].x, v.x);
                            v.y = fma(a1, x1[r][c].y, v.y);
                        }
                        if (q >= 3) {
                            v.x = fma(a2, x2[r][c].x, v.x);
                            v.y = fma(a2, x2[r][c].y, v.y);
                        }
                        tt[r][c] = v;
                    }
            };
            auto start_horner = [&](const C (&top)[TR][TC]) {
#pragma unroll
                for (int r = 0; r < TR; ++r)
#pragma unroll
                    for (int c = 0; c < TC; ++c) tt[r][c] = Cx<Real>::make(atop * top[r][c].x, atop * top[r][c].y);
                add_block(rh - 1);
            };
            const int n_pow = q - 1, n_hor = rh - 1;
            const int n_prod = n_pow + n_hor + s + 1;
            int blk = rh - 1;
            if (n_pow == 0) start_horner(x1);
            for (int pi = 0; pi < n_prod; ++pi) {
                const C *A, *B;
                if (pi < n_pow) {
                    A = (pi == 0) ? S1 : S2;
                    B = S1;
                } else {
                    st_tile<Real, D>(ST, rb, cb, tt);
                    __syncwarp();
                    if (pi < n_pow + n_hor) {
                        A = Sq;
                        B = ST;
                    } else {
                        A = ST;
                        B = (pi < n_prod - 1) ? ST : SR;
                    }
                }
                C acc[TR][TC];
                mm_tile<Real, D>(A, B, rb, cb, acc);
                __syncwarp();
                if (pi < n_pow) {
                    if (pi == 0) {
#pragma unroll
                        for (int r = 0; r < TR; ++r)
#pragma unroll
                            for (int c = 0; c < TC; ++c) x2[r][c] = acc[r][c];
                    }
                    st_tile<Real, D>(pi == 0 ? S2 : S3, rb, cb, acc);
                    if (pi == n_pow - 1) start_horner(acc);
                    __syncwarp();
                } else if (pi < n_pow + n_hor) {
#pragma unroll
                    for (int r = 0; r < TR; ++r)
#pragma unroll
                        for (int c = 0; c < TC; ++c) tt[r][c] = acc[r][c];
                    add_block(--blk);
                } else if (pi < n_prod - 1) {
#pragma unroll
                    for (int r = 0; r < TR; ++r)
#pragma unroll
                        for (int c = 0; c < TC; ++c) tt[r][c] = acc[r][c];
                } else {
                    st_tile<Real, D>(SR, rb, cb, acc);
                    __syncwarp();
                    if constexpr (EXPM == 2) {
                        if ((t0 + rr) < len) traj_emit(j0 + t0 + rr, acc);
                    }
                }
            }

            if (gl == 0 && (t0 + rr) < len) {
                n_exp += (unsigned long long)((q - 1) + (rh - 1) + s);
                n_tree += 1;
                m_max = max(m_max, cls_m(code));
                s_max = max(s_max, s);
            }
        }
        __syncwarp();
    }

    // packed-pair path: the leaf product from C(R) into the slot layout of the tree
    if constexpr (PP) {
        if (active_warp) {
            pp16::Tile t;
            pp16::ld_col(reinterpret_cast<const float4 *>(SR), lane >> 3, lane & 7, t);
            __syncwarp();
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 2; ++c)
                    SR[pp16::orow(lane >> 3, r) * LD + 2 * (lane & 7) + c] = make_float2(t.re[r][c], t.im[r][c]);
            __syncwarp();
        }
    }

    // trajectory mode: the forward pass already combined the leaves and recorded statistics
    if constexpr (EXPM == 2) return;

    // ---- FP32: pull the leaf product back towards the unitary group.  The slices of a
    //      drift-dominated run repeat nearly the same rounding errors, so the deviation of
    //      R^dagger R from I grows linearly along a leaf; one Newton-Schulz step of the polar
    //      iteration, R <- R (3 I - R^dagger R) / 2, squares it away (the exact product is unitary).
    if constexpr (std::is_same<Real, float>::value) {
        if (p.unitary_step && active_warp) {
            __syncwarp();
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TC; ++c) {
                    const int i = rb + r * G::RBN, jj = G::col(cb, c);
                    const C v = SR[i * LD + jj];
                    S1[jj * LD + i] = Cx<Real>::make(v.x, -v.y);  // R^dagger
                }
            __syncwarp();
            C m[TR][TC];
            mm_tile<Real, D>(S1, SR, rb, cb, m);  // R^dagger R
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TC; ++c) {
                    const bool diag = (rb + r * G::RBN) == G::col(cb, c);
                    m[r][c] = Cx<Real>::make((diag ? Real(3) : Real(0)) - m[r][c].x, -m[r][c].y);
                }
            st_tile<Real, D>(S2, rb, cb, m);
            __syncwarp();
            mm_tile<Real, D>(SR, S2, rb, cb, m);  // R (3 I - R^dagger R)
            __syncwarp();
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TC; ++c) m[r][c] = Cx<Real>::make(Real(0.5) * m[r][c].x, Real(0.5) * m[r][c].y);
            st_tile<Real, D>(SR, rb, cb, m);
            __syncwarp();
        }
    }

    // ---- optional: every leaf product in FP64 (checkpoints of the adjoint pass)
    if (p.leaf_out && active_warp) {
        double2 *dst = p.leaf_out + (size_t)leaf * DD;
        for (int t = gl; t < DD; t += LANES) {
            const C v = SR[(t / D) * LD + (t % D)];
            dst[t] = make_double2((double)v.x, (double)v.y);
        }
    }

    // ---- statistics and status (before this block's tree arrival)
    if (gl == 0 && n_tree) {
        atomicAdd(&p.counters[0], n_exp);
        atomicAdd(&p.counters[1], n_tree);
        atomicMax(&p.counters[2], (unsigned long long)m_max);
        atomicMax(&p.counters[3], (unsigned long long)s_max);
    }
    if (flags) atomicOr(&p.status[0], flags);

    // ---- in-block pairwise tree over the leaves (Sec. 2.2): leaf l+h is later than leaf l
    __syncthreads();
    const int n_leaf = W * GPW;
    const int gid = warp * GPW + g;  // block-wide group id
    auto leaf_R = [&](int l) -> C * {
        return (C *)(smem + boff + (size_t)(l / GPW) * wsb + (size_t)(l % GPW) * G::GSTRIDE) + 3 * SLOT;
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
        double2 *dst = p.partials + (size_t)blk * DD;
        double2 *keep = p.block_out ? p.block_out + (size_t)blk * DD : nullptr;
        for (int t = tid; t < DD; t += blockDim.x) {
            const C v = R0[(t / D) * LD + (t % D)];
            dst[t] = make_double2((double)v.x, (double)v.y);
            if (keep) keep[t] = dst[t];
        }
    }
    __threadfence();
    __syncthreads();

    // ---- pairwise tree over blocks in FP64: second arrival at a node multiplies right * left
    using GD = Geo<double, D>;
    double2 *bufL = (double2 *)(smem + boff);  // warp 0's workspace, free by now
    double2 *bufR = bufL + D * GD::LD;
    const int rb64 = (lane % GD::LANES) / GD::CBW, cb64 = (lane % GD::LANES) % GD::CBW;
    int idx = blk, n = nblk, level = 0, toff = 0;
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
                bufL[(t / D) * GD::LD + t % D] = __ldcg(gL + t);
                bufR[(t / D) * GD::LD + t % D] = __ldcg(gR + t);
            }
            __syncthreads();
            if (warp == 0 && lane < GD::LANES) {
                double2 acc[GD::TR][GD::TC];
                mm_tile<double, D>(bufR, bufL, rb64, cb64, acc);
                double2 *dst = p.partials + (size_t)((idx & ~1) << level) * DD;
#pragma unroll
                for (int r = 0; r < GD::TR; ++r)
#pragma unroll
                    for (int c = 0; c < GD::TC; ++c)
                        __stcg(dst + (rb64 + r * GD::RBN) * D + GD::col(cb64, c), acc[r][c]);
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
            for (int i = 0; i < 4; ++i) p.counters[4 + i] = atomicExch(&p.counters[i], 0ull);
            p.status[1] = atomicExch(&p.status[0], 0u);
        }
    }
}

template <typename Real, int D, int INTEG, int EXPM = 0>
__global__ void __launch_bounds__(Geo<Real, D>::MAXW * 32, 1) fused_small_kernel(const FusedParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    fused_body<Real, D, INTEG, EXPM>(p, blockIdx.x, gridDim.x, smem);
}

// host-side launcher (explicitly instantiated per D in pm_fused_d*.cu)
template <typename Real, int D, int INTEG, int EXPM = 0>
cudaError_t launch_fused(const FusedParams &p, int grid, int warps, size_t smem, cudaStream_t st) {
    auto k = fused_small_kernel<Real, D, INTEG, EXPM>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, warps * 32, smem, st>>>(p);
    return cudaGetLastError();
}

template <typename Real, int D, int INTEG, int EXPM = 0>
int fused_max_blocks_per_sm(int warps, size_t smem) {
    int nb = 0;
    auto k = fused_small_kernel<Real, D, INTEG, EXPM>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, warps * 32, smem) != cudaSuccess) return 0;
    return nb;
}

}  // namespace pm
