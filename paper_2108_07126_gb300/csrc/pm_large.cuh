// Propagation kernel for padded dimensions D in {32, 64, 128, 256}.
//
// Same method as the fused small-D kernel (per slice: effective coefficients,
// FP64 norm bound, exponent assembly, Taylor / Paterson-Stockmeyer on
// A = -i G / 2^s, s squarings, leaf product; then the pairwise tree over the
// block partials), but one thread block owns one leaf and a D x D complex
// matrix no longer fits a warp's shared memory.  The working matrices (X,
// X^2, X^3, Horner operand, leaf product, product output) live in a per-block
// region of global memory that stays in L2; every complex product is a
// block-wide tiled GEMM that stages k-panels of both operands in shared
// memory (cp.async, double-buffered) and accumulates register tiles.
#pragma once

#include <type_traits>

#include "pm_fused.cuh"
#include "pm_tc_small.cuh"
#include "pm_umma.cuh"

namespace pm {

constexpr int kLargeThreads = 256;
constexpr int kLargeSlots = 6;  // X, X^2, X^3, leaf product R, two ping-pong product buffers

template <typename Real, int D> struct LargeTile;
// threads = (RBAND / TR) x (D / TC) = 256; passes = D / RBAND row bands per product
template <> struct LargeTile<float, 32> { static constexpr int TR = 2, TC = 2, PASS = 1, KP = 16; };
template <> struct LargeTile<float, 64> { static constexpr int TR = 4, TC = 4, PASS = 1, KP = 16; };
template <> struct LargeTile<float, 128> { static constexpr int TR = 4, TC = 4, PASS = 4, KP = 16; };
template <> struct LargeTile<double, 32> { static constexpr int TR = 2, TC = 2, PASS = 1, KP = 8; };
template <> struct LargeTile<double, 64> { static constexpr int TR = 4, TC = 4, PASS = 1, KP = 8; };
template <> struct LargeTile<double, 128> { static constexpr int TR = 4, TC = 4, PASS = 4, KP = 8; };
template <> struct LargeTile<float, 256> { static constexpr int TR = 4, TC = 4, PASS = 16, KP = 16; };
template <> struct LargeTile<double, 256> { static constexpr int TR = 4, TC = 4, PASS = 16, KP = 8; };

template <typename Real, int D> struct LGeo {
    using T = LargeTile<Real, D>;
    using C = typename Cx<Real>::T;
    static constexpr int TR = T::TR, TC = T::TC, PASS = T::PASS, KP = T::KP;
    static constexpr int RBAND = D / PASS;       // output rows per pass
    static constexpr int TY = RBAND / TR;        // thread rows
    static constexpr int TX = D / TC;            // thread columns
    static_assert(TY * TX == kLargeThreads, "one output tile per thread per pass");
    static constexpr int DD = D * D;
    static constexpr int APAD = 16 / (int)sizeof(C), BPAD = 0;  // A rows padded by 16 bytes
    static constexpr int AS = RBAND * (KP + APAD);  // A panel elements
    static constexpr int BS = KP * (D + BPAD);      // B panel elements
    static constexpr size_t PANEL_BYTES = (size_t)2 * (AS + BS) * sizeof(C);  // double-buffered
};

// TCM: 0 = CUDA-core products, 2 = 3xTF32 with tcgen05 (D = 128, 256: 128 x 128 output blocks),
// 3 = split BF16x3 with tcgen05 (D = 128, 256), 4 / 5 = 3xTF32 / split BF16x3 with tcgen05 in the
// shared-memory body of pm_tc_small.cuh (D = 32, 64)
template <int TCM> __host__ __device__ constexpr int tcm_format() { return (TCM == 3 || TCM == 5) ? umma::kBF16x3 : umma::kTF32x3; }

template <typename Real, int D, int TCM = 0>
__host__ __device__ inline size_t large_panel_bytes() {
    // the FP64 top tree and the tensor-core products run through the same panels
    size_t b = LGeo<Real, D>::PANEL_BYTES;
    if (LGeo<double, D>::PANEL_BYTES > b) b = LGeo<double, D>::PANEL_BYTES;
    if (TCM >= 2 && umma::kSmemBytes > b) b = umma::kSmemBytes;
    return b;
}

// FP32 at D <= 64 on the CUDA cores keeps all six working matrices in shared memory
// (6 D^2 complex64 = 192 KB at D = 64) instead of the global scratch region.
template <typename Real, int D, int TCM>
__host__ __device__ constexpr bool large_resident() {
    return std::is_same<Real, float>::value && D <= 64 && TCM == 0;
}

// bytes in front of the coefficient tile: the resident matrices, or the staging panels
template <typename Real, int D, int TCM = 0>
__host__ __device__ inline size_t large_front_bytes() {
    const size_t res = large_resident<Real, D, TCM>() ? (size_t)kLargeSlots * D * D * sizeof(typename Cx<Real>::T) : 0;
    const size_t pan = large_panel_bytes<Real, D, TCM>();
    return res > pan ? res : pan;
}

template <typename Real, int D, int TCM = 0>
__host__ __device__ inline size_t large_smem_bytes(int n_basis) {
    if constexpr (TCM >= 4) {
        // the tensor-core body, and the FP64 / FP32 panels of the arrival tree that may follow it
        size_t b = tcs::smem_bytes<D, tcm_format<TCM>()>(n_basis);
        if (LGeo<double, D>::PANEL_BYTES > b) b = LGeo<double, D>::PANEL_BYTES;
        return (b + 15) & ~(size_t)15;
    }
    size_t b = large_front_bytes<Real, D, TCM>() + (size_t)(n_basis + 1) * sizeof(Real) + 64;
    return (b + 15) & ~(size_t)15;
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::); }

// Cout = A * B (D x D complex, row-major, global memory), by the whole block.
// Cout must not alias A or B.
template <typename Real, int D>
__device__ void cta_mm(const typename Cx<Real>::T *__restrict__ A, const typename Cx<Real>::T *__restrict__ B,
                       typename Cx<Real>::T *__restrict__ Cout, unsigned char *panels) {
    using G = LGeo<Real, D>;
    using C = typename G::C;
    constexpr int TR = G::TR, TC = G::TC, KP = G::KP, RBAND = G::RBAND, TY = G::TY;
    constexpr int ALD = KP + G::APAD, BLD = D + G::BPAD;
    constexpr int CPE = 16 / sizeof(C);  // complex elements per 16-byte copy
    C *As[2] = {(C *)panels, (C *)panels + G::AS};
    C *Bs[2] = {(C *)panels + 2 * G::AS, (C *)panels + 2 * G::AS + G::BS};
    const int tid = threadIdx.x;
    const int ty = tid / G::TX, tx = tid % G::TX;

    for (int pass = 0; pass < G::PASS; ++pass) {
        const int row0 = pass * RBAND;
        auto load = [&](int buf, int k0) {
            // A band: RBAND x KP; B panel: KP x D (16-byte pieces)
            for (int e = tid; e < RBAND * KP / CPE; e += kLargeThreads) {
                const int r = e / (KP / CPE), c = (e % (KP / CPE)) * CPE;
                cp_async16(As[buf] + r * ALD + c, A + (size_t)(row0 + r) * D + k0 + c);
            }
            for (int e = tid; e < KP * D / CPE; e += kLargeThreads) {
                const int r = e / (D / CPE), c = (e % (D / CPE)) * CPE;
                cp_async16(Bs[buf] + r * BLD + c, B + (size_t)(k0 + r) * D + c);
            }
            cp_async_commit();
        };
        C acc[TR][TC];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c) acc[r][c] = Cx<Real>::make(0, 0);
        load(0, 0);
        for (int kp = 0; kp < D / KP; ++kp) {
            const int buf = kp & 1;
            if (kp + 1 < D / KP) {
                load(buf ^ 1, (kp + 1) * KP);
                cp_async_wait_one();
            } else {
                cp_async_wait_all();
            }
            __syncthreads();
            const C *a_s = As[buf], *b_s = Bs[buf];
#pragma unroll 4
            for (int k = 0; k < KP; ++k) {
                C a[TR], b[TC];
#pragma unroll
                for (int r = 0; r < TR; ++r) a[r] = a_s[(ty + r * TY) * ALD + k];
#pragma unroll
                for (int c = 0; c < TC; ++c) b[c] = b_s[k * BLD + tx + c * G::TX];
#pragma unroll
                for (int r = 0; r < TR; ++r)
#pragma unroll
                    for (int c = 0; c < TC; ++c) cfma(acc[r][c], a[r], b[c]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c) Cout[(size_t)(row0 + ty + r * TY) * D + tx + c * G::TX] = acc[r][c];
    }
    __syncthreads();
}

// Cout = A * B for D x D complex64 matrices already in shared memory (row stride D), by the
// whole block: thread (ty, tx) = (tid / 16, tid % 16) owns rows ty + 16 r and the TC consecutive
// columns TC tx .. TC tx + TC - 1.  Per pair of k the A reads are two broadcast rows per warp
// (16-byte loads) and the B reads one contiguous 16 TC-complex row segment.  Cout must not
// alias A or B; ends with a block barrier.
template <int D>
__device__ __forceinline__ void smem_mm(const float2 *__restrict__ A, const float2 *__restrict__ B,
                                        float2 *__restrict__ Cout) {
    // thread (ty, tx): rows ty + 16 r, column pairs 32 p + 2 tx (p < TC / 2), so the 16-byte B loads
    // and C stores of a quarter warp cover 128 contiguous bytes
    constexpr int TR = D / 16, TC = D / 16;
    static_assert(TR * TC * kLargeThreads == D * D && TC % 2 == 0 && 16 * TC == D, "thread tiling");
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    float2 acc[TR][TC];
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
        for (int c = 0; c < TC; ++c) acc[r][c] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int k = 0; k < D; k += 2) {
        float2 a[TR][2], b[2][TC];
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            const float4 v = *reinterpret_cast<const float4 *>(A + (ty + 16 * r) * D + k);
            a[r][0] = make_float2(v.x, v.y);
            a[r][1] = make_float2(v.z, v.w);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int c = 0; c < TC; c += 2) {
                const float4 v = *reinterpret_cast<const float4 *>(B + (k + u) * D + 16 * c + 2 * tx);
                b[u][c] = make_float2(v.x, v.y);
                b[u][c + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TC; ++c) cfma(acc[r][c], a[r][u], b[u][c]);
    }
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
        for (int c = 0; c < TC; c += 2)
            *reinterpret_cast<float4 *>(Cout + (ty + 16 * r) * D + 16 * c + 2 * tx) =
                make_float4(acc[r][c].x, acc[r][c].y, acc[r][c + 1].x, acc[r][c + 1].y);
    __syncthreads();
}

// the complex product used by the large kernel: CUDA cores, or tcgen05 with tensor-memory
// accumulators (FP32 only; TCM = 2 3xTF32, 3 split BF16x3): D = 128 in one 128 x 128 block, D = 256
// in four 128 x 128 output blocks over K = 256
template <typename Real, int D, int TCM>
__device__ __forceinline__ void large_mm(const typename Cx<Real>::T *A, const typename Cx<Real>::T *B,
                                         typename Cx<Real>::T *Cout, unsigned char *panels, umma::Ctx *uc) {
    if constexpr ((TCM == 2 || TCM == 3) && std::is_same<Real, float>::value) {
        constexpr int F = TCM == 3 ? umma::kBF16x3 : umma::kTF32x3;
        if constexpr (D == 128) {
            umma::cmul128<F>(A, B, Cout, panels, *uc);
        } else {
            static_assert(D == 256, "tcgen05 block product covers D = 128 and 256");
#pragma unroll 1
            for (int blk = 0; blk < 4; ++blk) {
                const int i0 = (blk >> 1) * 128, j0 = (blk & 1) * 128;
                umma::cmul128<F, 256, 256>(A + (size_t)i0 * 256, B + j0, Cout + (size_t)i0 * 256 + j0, panels, *uc);
            }
        }
    } else if constexpr (large_resident<Real, D, TCM>()) {
        smem_mm<D>(A, B, Cout);
    } else {
        cta_mm<Real, D>(A, B, Cout, panels);
    }
}

// One leaf (slices [N blk / nblk, N (blk + 1) / nblk)) of one problem by one
// thread block; writes the leaf product to p.partials[blk] (FP64).
// ws: this block's 6 D x D scratch matrices.
template <typename Real, int D, int INTEG, int TCM>
__device__ __forceinline__ void large_body(const FusedParams &p, typename Cx<Real>::T *ws, int blk, int nblk,
                                           unsigned char *smem, umma::Ctx *uc = nullptr) {
    using G = LGeo<Real, D>;
    using C = typename G::C;
    constexpr int DD = G::DD;

    __shared__ int s_code;
    unsigned char *panels = smem;
    Real *gam = (Real *)(smem + large_front_bytes<Real, D, TCM>());
    const int tid = threadIdx.x, nb = p.n_basis;
    constexpr bool kResident = large_resident<Real, D, TCM>();
    if constexpr (kResident) ws = (C *)smem;  // the working matrices live in shared memory

    C *SX = ws, *SX2 = ws + DD, *SX3 = ws + 2 * DD;
    // leaf product and the two Horner / squaring buffers rotate through the last three slots
    C *SR = ws + 3 * DD, *P0 = ws + 4 * DD, *P1 = ws + 5 * DD;
    // packed exponent: in shared memory (rows padded to D + 1, conflict-free transposed reads)
    // when the tensor-core stages leave room, else in a free scratch slot
    constexpr bool kGpkShared = (TCM >= 2 && D <= 128) || kResident;  // D = 256: 263 KB, too large
    static_assert(DD % (4 * kLargeThreads) == 0, "element passes take four elements per thread and step");
    constexpr int GLD = kGpkShared ? D + 1 : D;
    const Real *packed = (const Real *)p.packed;

    const int64_t j0 = p.n_steps * blk / nblk;
    const int len = (int)(p.n_steps * (blk + 1) / nblk - j0);

    // R = I, or in trajectory mode the product of every slice before the leaf (FP64 prefix)
    const bool traj = p.traj_out != nullptr;
    for (int e = tid; e < DD; e += kLargeThreads) {
        if (traj) {
            const double2 v = p.traj_pin[(size_t)blk * DD + e];
            SR[e] = Cx<Real>::make((Real)v.x, (Real)v.y);
        } else {
            SR[e] = Cx<Real>::make((e / D) == (e % D) ? Real(1) : Real(0), Real(0));
        }
    }
    unsigned flags = 0;
    unsigned long long n_exp = 0;
    int m_max = 0, s_max = 0;

    // the paper's Chebyshev exponential (Sec. 2.1, Algorithm 1) when the pre-pass set its degree
    const bool cheb = p.cheb_m != nullptr;
    const int mch = cheb ? *p.cheb_m : 0;
    const Real ib = cheb ? (Real)*p.cheb_inv_beta : Real(0);

    for (int t = 0; t < len; ++t) {
        const int64_t j = j0 + t;
        if (tid == 0) {
            slice_coefficients<Real, INTEG, 1>(p, j, true, gam);
            double nu = 0.0;
            for (int e = 0; e < nb; ++e) nu = fma(fabs((double)gam[e]), p.bnorm1[e], nu);
            s_code = cheb ? 0 : p.cls_code[find_class(p, nu, &flags)];  // Chebyshev: one degree, set before
        }
        __syncthreads();
        const int code = s_code;
        const int q = cls_q(code), rh = cls_r(code), s = cls_s(code) + p.extra_squarings;
        const Real sc = pow2neg<Real>(s);
        // tensor cores (D <= 128): the idle operand stages; otherwise the free slot P0 (in shared
        // memory for the resident bodies, in the global scratch otherwise)
        Real *gpk = (TCM >= 2 && D <= 128) ? (Real *)panels : (Real *)P0;

        // packed exponent sum_b gamma_b P_b: EP groups of four entries per thread and step, the
        // basis loop unrolled, so that 4 EP independent 16-byte loads from L2 are in flight (the
        // basis is read once per slice and does not fit in shared memory)
        {
            constexpr int NE4 = DD / 4, EP = (NE4 / kLargeThreads) < 4 ? (NE4 / kLargeThreads) : 4;
            static_assert(EP >= 1 && NE4 % (EP * kLargeThreads) == 0, "assembly steps cover the matrix");
            for (int e0 = tid; e0 < NE4; e0 += EP * kLargeThreads) {
                Real v[EP][4];
#pragma unroll
                for (int q = 0; q < EP; ++q)
#pragma unroll
                    for (int u = 0; u < 4; ++u) v[q][u] = Real(0);
#pragma unroll 4
                for (int b = 0; b < nb; ++b) {
                    const Real g = gam[b];
                    Real w[EP][4];
#pragma unroll
                    for (int q = 0; q < EP; ++q) ld4<Real>(packed + (size_t)b * DD + 4 * (e0 + q * kLargeThreads), w[q]);
#pragma unroll
                    for (int q = 0; q < EP; ++q)
#pragma unroll
                        for (int u = 0; u < 4; ++u) v[q][u] = fma(g, w[q][u], v[q][u]);
                }
#pragma unroll
                for (int q = 0; q < EP; ++q) {
                    const int e4 = e0 + q * kLargeThreads, i = (4 * e4) / D, jj = (4 * e4) % D;
#pragma unroll
                    for (int u = 0; u < 4; ++u) gpk[i * GLD + jj + u] = v[q][u];
                }
            }
        }
        __syncthreads();
        // Hermitian unpack (upper triangle: Re, strict lower: Im) into A = -i G / 2^s, or into
        // X = G / beta for the Chebyshev series
        for (int e = tid; e < DD; e += kLargeThreads) {
            const int i = e / D, jj = e % D;
            const Real a = gpk[i * GLD + jj], b = gpk[jj * GLD + i];
            const Real re = (i <= jj) ? a : b;
            const Real im = (i > jj) ? a : ((i < jj) ? -b : Real(0));
            SX[e] = cheb ? Cx<Real>::make(re * ib, im * ib) : Cx<Real>::make(im * sc, -re * sc);
        }
        __syncthreads();
        if (cheb) {
            // Clenshaw: D_m = a_m I, D_{m+1} = 0; D_k = a_k I + 2 X D_{k+1} - D_{k+2}; U = D_0 - D_2
            const C *ak = (const C *)p.cheb_coef;
            C *d1 = SX2, *d2 = SX3, *nw = P0;
            for (int e = tid; e < DD; e += kLargeThreads) {
                const bool diag = (e / D) == (e % D);
                d1[e] = diag ? ak[mch] : Cx<Real>::make(Real(0), Real(0));
                d2[e] = Cx<Real>::make(Real(0), Real(0));
            }
            __syncthreads();
            for (int k = mch - 1; k >= 0; --k) {
                large_mm<Real, D, TCM>(SX, d1, nw, panels, uc);
                const C a_k = ak[k];
                for (int e = tid; e < DD; e += kLargeThreads) {
                    const C x = nw[e], y = d2[e];
                    C v = Cx<Real>::make(Real(2) * x.x - y.x, Real(2) * x.y - y.y);
                    if ((e / D) == (e % D)) {
                        v.x += a_k.x;
                        v.y += a_k.y;
                    }
                    nw[e] = (k == 0) ? Cx<Real>::make(v.x - y.x, v.y - y.y) : v;
                }
                __syncthreads();
                if (k > 0) {  // D_{k+2} <- D_{k+1}, D_{k+1} <- D_k
                    C *t2 = d2;
                    d2 = d1;
                    d1 = nw;
                    nw = t2;
                }
            }
            // leaf product R <- U_j R into P1 (U_j is in one of SX2, SX3, P0), which becomes R
            large_mm<Real, D, TCM>(nw, SR, P1, panels, uc);
            {
                C *old = SR;
                SR = P1;
                P1 = old;
            }
            if (tid == 0) {
                n_exp += (unsigned long long)mch;
                m_max = max(m_max, mch);
            }
            continue;
        }
        if (q >= 2) large_mm<Real, D, TCM>(SX, SX, SX2, panels, uc);
        if (q >= 3) large_mm<Real, D, TCM>(SX2, SX, SX3, panels, uc);
        const C *Xq = (q == 1) ? SX : ((q == 2) ? SX2 : SX3);
        // Horner over blocks with two ping-pong buffers:
        //   T = a_{q r} X^q + B_{r-1};  T <- X^q T + B_b;  B_b = sum_{l<q} a_{q b + l} X^l
        // (four elements per thread and step: all loads before the stores, T may alias src)
        auto add_block = [&](C *T, const C *src, Real scale, int b) {
            const Real a0 = coef<Real>(p, q * b);
            const Real a1 = (q >= 2) ? coef<Real>(p, q * b + 1) : Real(0);
            const Real a2 = (q >= 3) ? coef<Real>(p, q * b + 2) : Real(0);
            for (int e0 = tid; e0 < DD; e0 += 4 * kLargeThreads) {
                C v[4], x1[4], x2[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = e0 + u * kLargeThreads;
                    v[u] = src[e];
                    if (q >= 2) x1[u] = SX[e];
                    if (q >= 3) x2[u] = SX2[e];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = e0 + u * kLargeThreads;
                    C w = Cx<Real>::make(v[u].x * scale, v[u].y * scale);
                    w.x += ((e / D) == (e % D)) ? a0 : Real(0);
                    if (q >= 2) {
                        w.x = fma(a1, x1[u].x, w.x);
                        w.y = fma(a1, x1[u].y, w.y);
                    }
                    if (q >= 3) {
                        w.x = fma(a2, x2[u].x, w.x);
                        w.y = fma(a2, x2[u].y, w.y);
                    }
                    T[e] = w;
                }
            }
            __syncthreads();
        };
        C *cur = P0, *nxt = P1;
        add_block(cur, Xq, coef<Real>(p, q * rh), rh - 1);
        for (int b = rh - 2; b >= 0; --b) {
            large_mm<Real, D, TCM>(Xq, cur, nxt, panels, uc);
            add_block(nxt, nxt, Real(1), b);
            C *t2 = cur; cur = nxt; nxt = t2;
        }
        for (int i = 0; i < s; ++i) {
            large_mm<Real, D, TCM>(cur, cur, nxt, panels, uc);
            C *t2 = cur; cur = nxt; nxt = t2;
        }
        // leaf product R <- U_j R into the free buffer, which becomes R; the old R slot is free
        large_mm<Real, D, TCM>(cur, SR, nxt, panels, uc);
        {
            C *old = SR;
            SR = nxt;
            P0 = cur;
            P1 = old;
        }
        // trajectory mode: R = U(t_{j+1}); keep it at the output slices (R is complete: the
        // product ends with a block barrier)
        if (traj && ((j + 1) % p.traj_every == 0 || j + 1 == p.n_steps)) {
            const int64_t o = j / p.traj_every;
            const int d = p.d_out;
            if (p.traj_psi0 == nullptr) {
                for (int e = tid; e < d * d; e += kLargeThreads) {
                    const C v = SR[(e / d) * D + e % d];
                    const size_t at = (size_t)o * d * d + e;
                    if (p.out_c128) ((double2 *)p.traj_out)[at] = make_double2((double)v.x, (double)v.y);
                    else ((float2 *)p.traj_out)[at] = make_float2((float)v.x, (float)v.y);
                }
            } else {
                for (int i = tid; i < d; i += kLargeThreads) {
                    Real re = 0, im = 0;
                    for (int k = 0; k < d; ++k) {
                        const C a = SR[i * D + k];
                        const double2 b = p.traj_psi0[k];
                        re = fma(a.x, (Real)b.x, fma(-a.y, (Real)b.y, re));
                        im = fma(a.x, (Real)b.y, fma(a.y, (Real)b.x, im));
                    }
                    const size_t at = (size_t)o * d + i;
                    if (p.out_c128) ((double2 *)p.traj_out)[at] = make_double2((double)re, (double)im);
                    else ((float2 *)p.traj_out)[at] = make_float2((float)re, (float)im);
                }
            }
        }
        if (tid == 0) {
            n_exp += (unsigned long long)((q - 1) + (rh - 1) + s);
            m_max = max(m_max, cls_m(code));
            s_max = max(s_max, s);
        }
    }

    // trajectory mode: the forward pass already combined the leaves and recorded statistics
    if (traj) {
        __syncthreads();
        return;
    }

    // FP32: one Newton-Schulz step of the polar iteration on the leaf product,
    // R <- R (3 I - R^dagger R) / 2 (the exact product is unitary; repeated rounding, and the
    // truncating accumulation of the tensor cores, drift R off the unitary group along a leaf)
    if constexpr (std::is_same<Real, float>::value) {
        if (p.unitary_step && len > 0) {
            for (int e = tid; e < DD; e += kLargeThreads) {
                const C v = SR[(e % D) * D + e / D];
                P0[e] = Cx<Real>::make(v.x, -v.y);  // R^dagger
            }
            __syncthreads();
            large_mm<Real, D, TCM>(P0, SR, P1, panels, uc);  // R^dagger R
            for (int e = tid; e < DD; e += kLargeThreads) {
                const C v = P1[e];
                P1[e] = Cx<Real>::make(((e / D) == (e % D) ? Real(3) : Real(0)) - v.x, -v.y);
            }
            __syncthreads();
            large_mm<Real, D, TCM>(SR, P1, P0, panels, uc);  // R (3 I - R^dagger R)
            for (int e = tid; e < DD; e += kLargeThreads) {
                const C v = P0[e];
                SR[e] = Cx<Real>::make(Real(0.5) * v.x, Real(0.5) * v.y);
            }
            __syncthreads();
        }
    }

    if (tid == 0 && len > 0) {
        atomicAdd(&p.counters[0], n_exp);
        atomicAdd(&p.counters[1], (unsigned long long)len);
        atomicMax(&p.counters[2], (unsigned long long)m_max);
        atomicMax(&p.counters[3], (unsigned long long)s_max);
    }
    if (flags) atomicOr(&p.status[0], flags);

    // block partial (the leaf product) in FP64
    {
        double2 *dst = p.partials + (size_t)blk * DD;
        for (int e = tid; e < DD; e += kLargeThreads) {
            const C v = SR[e];
            dst[e] = make_double2((double)v.x, (double)v.y);
            if (p.leaf_out) p.leaf_out[(size_t)blk * DD + e] = dst[e];
            if (p.block_out) p.block_out[(size_t)blk * DD + e] = dst[e];
        }
    }
    __threadfence();
    __syncthreads();
}

// products of the tensor-core precisions in the standalone large kernel (TC: 0 none, 1 3xTF32,
// 2 split BF16x3): tcgen05 in the shared-memory body for D = 32, 64, tcgen05 with working
// matrices in a global scratch region for D = 128, 256
template <typename Real, int D, int TC>
__host__ __device__ constexpr int large_tcm() {
    return (TC == 0 || !std::is_same<Real, float>::value) ? 0 : (D <= 64 ? (TC == 2 ? 5 : 4) : (TC == 2 ? 3 : 2));
}

// blocks per SM the large kernel is compiled for: two for the tensor-core body at D = 32
template <typename Real, int D, int TC>
__host__ __device__ constexpr int large_min_blocks() {
    return large_tcm<Real, D, TC>() >= 4 ? tcs::Cfg<D, tcm_format<large_tcm<Real, D, TC>()>()>::MIN_BLOCKS : 1;
}

template <typename Real, int D, int INTEG, int TC = 0>
__global__ void __launch_bounds__(kLargeThreads, large_min_blocks<Real, D, TC>())
    large_kernel(const FusedParams p, void *scratch) {
    extern __shared__ __align__(16) unsigned char smem[];
    using C = typename Cx<Real>::T;
    constexpr int TCM = large_tcm<Real, D, TC>();
    C *ws = (C *)scratch + (size_t)blockIdx.x * kLargeSlots * D * D;
    if constexpr (TCM >= 4) {
        __shared__ __align__(8) uint64_t s_mbar[umma::kBars];
        __shared__ uint32_t s_tmem;
        __shared__ int s_abort;
        umma::Ctx cx;
        constexpr int F = tcm_format<TCM>();
        umma::setup(cx, s_mbar, &s_tmem, &s_abort, p.status, tcs::tmem_cols<D, F>());
        tcs::body<D, INTEG, F>(p, blockIdx.x, gridDim.x, smem, cx);
        umma::teardown(cx);
    } else if constexpr (TCM >= 2) {
        __shared__ __align__(8) uint64_t s_mbar[umma::kBars];
        __shared__ uint32_t s_tmem;
        __shared__ int s_abort;
        umma::Ctx cx;
        umma::setup(cx, s_mbar, &s_tmem, &s_abort, p.status);
        large_body<Real, D, INTEG, TCM>(p, ws, blockIdx.x, gridDim.x, smem, &cx);
        umma::teardown(cx);
    } else {
        large_body<Real, D, INTEG, TCM>(p, ws, blockIdx.x, gridDim.x, smem);
    }
    // the pairwise tree over the block partials runs in tree_level_kernel launches
}

// Pairwise tree over the nblk leaf products of one problem without waiting:
// the second block to reach a node multiplies (later on the left, through the
// block's scratch), the first one leaves; the root writes U_out and snapshots
// the statistics.  As in the single-problem tree, the levels with at most 8
// nodes multiply in FP64 and the levels below in Real (the partials stay FP64
// in global memory): an FP64 product of two 64 x 64 matrices costs an SM
// ~0.5 M cycles on GB300's FP64 pipe, as much as the FP32 work of ~5 slices.
template <typename Real, int D>
__device__ void large_arrival_tree(const FusedParams &p, void *ws_bytes, int blk, int nblk, unsigned char *smem) {
    constexpr int DD = D * D;
    __shared__ int s_second;
    const int tid = threadIdx.x;
    double2 *L2 = (double2 *)ws_bytes, *R2 = L2 + DD;
    int idx = blk, n = nblk, level = 0, toff = 0;
    while (n > 1) {
        const int parent = idx >> 1;
        if ((idx | 1) < n) {
            if (tid == 0) s_second = (atomicAdd(&p.tickets[toff + parent], 1u) != 0u);
            __syncthreads();
            if (!s_second) return;
            if (tid == 0) p.tickets[toff + parent] = 0u;
            __threadfence();
            double2 *gL = p.partials + (size_t)((idx & ~1) << level) * DD;
            const double2 *gR = p.partials + (size_t)((idx | 1) << level) * DD;
            if (std::is_same<Real, double>::value || n <= 8) {
                for (int e = tid; e < DD; e += kLargeThreads) {
                    L2[e] = __ldcg(gL + e);
                    R2[e] = __ldcg(gR + e);
                }
                __syncthreads();
                cta_mm<double, D>(R2, L2, gL, smem);
            } else {
                float2 *Lf = (float2 *)ws_bytes, *Rf = Lf + DD, *Cf = Rf + DD;
                for (int e = tid; e < DD; e += kLargeThreads) {
                    const double2 l = __ldcg(gL + e), r = __ldcg(gR + e);
                    Lf[e] = make_float2((float)l.x, (float)l.y);
                    Rf[e] = make_float2((float)r.x, (float)r.y);
                }
                __syncthreads();
                cta_mm<float, D>(Rf, Lf, Cf, smem);
                for (int e = tid; e < DD; e += kLargeThreads) gL[e] = make_double2((double)Cf[e].x, (double)Cf[e].y);
            }
            __threadfence();
            __syncthreads();
        }
        idx = parent;
        n = (n + 1) >> 1;
        toff += n;
        ++level;
    }
    const int d = p.d_out;
    for (int e = tid; e < d * d; e += kLargeThreads) {
        const double2 v = __ldcg(p.partials + (e / d) * D + (e % d));
        if (p.out_c128) ((double2 *)p.U_out)[e] = v;
        else ((float2 *)p.U_out)[e] = make_float2((float)v.x, (float)v.y);
    }
    if (tid == 0) {
        __threadfence();
        for (int i = 0; i < 4; ++i) p.counters[4 + i] = atomicExch(&p.counters[i], 0ull);
        p.status[1] = atomicExch(&p.status[0], 0u);
    }
    __syncthreads();
}

// One level of the pairwise tree over block partials (Sec. 2.2) for large D:
// out[i] = in[2i+1] * in[2i] (the later partial on the left), an odd last
// partial is carried.  Storage is FP64; the products are computed in Real
// (FP64 for the top levels, FP32 below them in the FP32 modes).  Each block
// computes one 32 x 32 tile of one product, so a level spreads over the GPU.
// The last level (one output) also writes U_out and snapshots the statistics.
template <typename Real, int D>
__global__ void __launch_bounds__(256) tree_level_kernel(const double2 *__restrict__ in, int n_in,
                                                         double2 *__restrict__ out, const FusedParams p) {
    using C = typename Cx<Real>::T;
    constexpr int T = 32, KP = 16;
    __shared__ C As[T][KP + 1], Bs[KP][T + 1];
    const int tiles = D / T;
    const int ti = blockIdx.x / tiles, tj = blockIdx.x % tiles, pair = blockIdx.y;
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    const size_t DD = (size_t)D * D;
    const bool has_pair = 2 * pair + 1 < n_in;
    const double2 *L = in + (size_t)(2 * pair) * DD;      // earlier
    const double2 *R = in + (size_t)(2 * pair + 1) * DD;  // later
    double2 *O = out + (size_t)pair * DD;
    C acc[2][2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) acc[r][c] = Cx<Real>::make(0, 0);
    if (has_pair) {
        for (int k0 = 0; k0 < D; k0 += KP) {
            for (int e = threadIdx.x; e < T * KP; e += blockDim.x) {
                const int r = e / KP, k = e % KP;
                const double2 a = R[(size_t)(ti * T + r) * D + k0 + k];
                As[r][k] = Cx<Real>::make((Real)a.x, (Real)a.y);
                const int kb = e / T, cb = e % T;
                const double2 b = L[(size_t)(k0 + kb) * D + tj * T + cb];
                Bs[kb][cb] = Cx<Real>::make((Real)b.x, (Real)b.y);
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const C a0 = As[ty][k], a1 = As[ty + 16][k];
                const C b0 = Bs[k][tx], b1 = Bs[k][tx + 16];
                cfma(acc[0][0], a0, b0);
                cfma(acc[0][1], a0, b1);
                cfma(acc[1][0], a1, b0);
                cfma(acc[1][1], a1, b1);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int i = ti * T + ty + 16 * r, j = tj * T + tx + 16 * c;
            const double2 v = has_pair ? make_double2((double)acc[r][c].x, (double)acc[r][c].y)
                                       : L[(size_t)i * D + j];
            O[(size_t)i * D + j] = v;
            if (gridDim.y == 1 && n_in <= 2) {  // last level: the propagator itself
                const int d = p.d_out;
                if (i < d && j < d) {
                    if (p.out_c128) ((double2 *)p.U_out)[i * d + j] = v;
                    else ((float2 *)p.U_out)[i * d + j] = make_float2((float)v.x, (float)v.y);
                }
            }
        }
    if (gridDim.y == 1 && n_in <= 2 && blockIdx.x == 0 && threadIdx.x == 0) {
        for (int i = 0; i < 4; ++i) p.counters[4 + i] = atomicExch(&p.counters[i], 0ull);
        p.status[1] = atomicExch(&p.status[0], 0u);
    }
}

// Exclusive prefixes of the leaf products for the trajectory pass, by a Hillis-Steele scan in
// FP64: x_0 = I, x_b = leaf_{b-1}; at each level out_i = in_i in_{i-off} for i >= off (the later
// factor on the left), off = 1, 2, 4, ...; the result is prefix_b = leaf_{b-1} ... leaf_0.
template <int D>
__global__ void __launch_bounds__(256) prefix_init_kernel(const double2 *__restrict__ leaf, int n,
                                                          double2 *__restrict__ x) {
    const size_t DD = (size_t)D * D;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * DD; e += (size_t)gridDim.x * blockDim.x) {
        const size_t b = e / DD, t = e % DD;
        x[e] = (b == 0) ? make_double2((t / D) == (t % D) ? 1.0 : 0.0, 0.0) : leaf[(b - 1) * DD + t];
    }
}

// one level: block (tile, i) computes one 32 x 32 tile of out_i
template <int D>
__global__ void __launch_bounds__(256) prefix_level_kernel(const double2 *__restrict__ in, int n, int off,
                                                           double2 *__restrict__ out) {
    constexpr int T = 32, KP = 16;
    __shared__ double2 As[T][KP + 1], Bs[KP][T + 1];
    const int tiles = D / T;
    const int ti = blockIdx.x / tiles, tj = blockIdx.x % tiles, i = blockIdx.y;
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    const size_t DD = (size_t)D * D;
    const double2 *Lt = in + (size_t)i * DD;  // later factor (left)
    double2 *O = out + (size_t)i * DD;
    if (i < off) {
        for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
            const size_t at = (size_t)(ti * T + e / T) * D + tj * T + e % T;
            O[at] = Lt[at];
        }
        return;
    }
    const double2 *Rt = in + (size_t)(i - off) * DD;  // earlier factor (right)
    double2 acc[2][2] = {{make_double2(0.0, 0.0), make_double2(0.0, 0.0)}, {make_double2(0.0, 0.0), make_double2(0.0, 0.0)}};
    for (int k0 = 0; k0 < D; k0 += KP) {
        for (int e = threadIdx.x; e < T * KP; e += blockDim.x) {
            const int r = e / KP, k = e % KP;
            As[r][k] = Lt[(size_t)(ti * T + r) * D + k0 + k];
            const int kb = e / T, cb = e % T;
            Bs[kb][cb] = Rt[(size_t)(k0 + kb) * D + tj * T + cb];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const double2 a0 = As[ty][k], a1 = As[ty + 16][k], b0 = Bs[k][tx], b1 = Bs[k][tx + 16];
            cfma(acc[0][0], a0, b0);
            cfma(acc[0][1], a0, b1);
            cfma(acc[1][0], a1, b0);
            cfma(acc[1][1], a1, b1);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) O[(size_t)(ti * T + ty + 16 * r) * D + tj * T + tx + 16 * c] = acc[r][c];
}

// exclusive prefixes of n leaf products into x (one of the two buffers a, b; returned)
template <int D>
cudaError_t leaf_prefixes(const double2 *leaf, int n, double2 *a, double2 *b, double2 **x, cudaStream_t st) {
    prefix_init_kernel<D><<<1024, 256, 0, st>>>(leaf, n, a);
    cudaError_t e = cudaGetLastError();
    double2 *cur = a, *nxt = b;
    for (int off = 1; off < n && e == cudaSuccess; off <<= 1) {
        prefix_level_kernel<D><<<dim3((D / 32) * (D / 32), n), 256, 0, st>>>(cur, n, off, nxt);
        e = cudaGetLastError();
        double2 *t = cur;
        cur = nxt;
        nxt = t;
    }
    *x = cur;
    return e;
}

// Forward kernel, then the tree levels: FP64 products for the top three levels (and everywhere in
// FP64 mode), Real products below.  The per-block scratch doubles as the second tree buffer.
template <typename Real, int D, int INTEG, int TC = 0>
cudaError_t launch_large(const FusedParams &p, void *scratch, int grid, size_t smem, cudaStream_t st) {
    auto k = large_kernel<Real, D, INTEG, TC>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kLargeThreads, smem, st>>>(p, scratch);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (p.traj_out) return cudaSuccess;  // trajectory pass: no tree
    double2 *bufs[2] = {p.partials, (double2 *)scratch};
    int cur = 0, n = grid;
    do {
        const int n_out = (n + 1) / 2;
        const dim3 g((D / 32) * (D / 32), n_out);
        if (std::is_same<Real, double>::value || n <= 8)
            tree_level_kernel<double, D><<<g, 256, 0, st>>>(bufs[cur], n, bufs[cur ^ 1], p);
        else
            tree_level_kernel<float, D><<<g, 256, 0, st>>>(bufs[cur], n, bufs[cur ^ 1], p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        cur ^= 1;
        n = n_out;
    } while (n > 1);
    return cudaSuccess;
}

}  // namespace pm
