// Propagation kernel for padded dimensions D in {32, 64, 128}.
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

#include "pm_fused.cuh"

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

template <typename Real, int D>
__host__ __device__ inline size_t large_panel_bytes() {
    // the FP64 top tree runs its products through the same panels
    return LGeo<Real, D>::PANEL_BYTES > LGeo<double, D>::PANEL_BYTES ? LGeo<Real, D>::PANEL_BYTES
                                                                      : LGeo<double, D>::PANEL_BYTES;
}

template <typename Real, int D>
__host__ __device__ inline size_t large_smem_bytes(int n_basis) {
    size_t b = large_panel_bytes<Real, D>() + (size_t)(n_basis + 1) * sizeof(Real) + 64;
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
                for (int c = 0; c < TC; ++c) b[c] = b_s[k * BLD + tx * TC + c];
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
            for (int c = 0; c < TC; ++c) Cout[(size_t)(row0 + ty + r * TY) * D + tx * TC + c] = acc[r][c];
    }
    __syncthreads();
}

template <typename Real, int D, int INTEG>
__global__ void __launch_bounds__(kLargeThreads, 1) large_kernel(const FusedParams p, void *scratch) {
    using G = LGeo<Real, D>;
    using C = typename G::C;
    constexpr int DD = G::DD;

    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_code, s_second;
    unsigned char *panels = smem;
    Real *gam = (Real *)(smem + large_panel_bytes<Real, D>());
    const int tid = threadIdx.x, nb = p.n_basis;

    C *ws = (C *)scratch + (size_t)blockIdx.x * kLargeSlots * DD;
    C *SX = ws, *SX2 = ws + DD, *SX3 = ws + 2 * DD, *SR = ws + 3 * DD, *P0 = ws + 4 * DD, *P1 = ws + 5 * DD;
    Real *gpk = (Real *)P0;  // packed exponent scratch, free once X is formed
    const Real *packed = (const Real *)p.packed;

    const int64_t j0 = p.n_steps * blockIdx.x / gridDim.x;
    const int len = (int)(p.n_steps * (blockIdx.x + 1) / gridDim.x - j0);

    for (int e = tid; e < DD; e += kLargeThreads) SR[e] = Cx<Real>::make((e / D) == (e % D) ? Real(1) : Real(0), Real(0));
    unsigned flags = 0;
    unsigned long long n_exp = 0;
    int m_max = 0, s_max = 0;

    for (int t = 0; t < len; ++t) {
        const int64_t j = j0 + t;
        if (tid == 0) {
            slice_coefficients<Real, INTEG, 1>(p, j, true, gam);
            double nu = 0.0;
            for (int e = 0; e < nb; ++e) nu = fma(fabs((double)gam[e]), p.bnorm1[e], nu);
            s_code = p.cls_code[find_class(p, nu, &flags)];
        }
        __syncthreads();
        const int code = s_code;
        const int q = cls_q(code), rh = cls_r(code), s = cls_s(code) + p.extra_squarings;
        const Real sc = pow2neg<Real>(s);

        // packed exponent, then A = -i G / 2^s into SX
        for (int e = tid; e < DD; e += kLargeThreads) {
            Real v = 0;
            for (int b = 0; b < nb; ++b) v = fma(gam[b], __ldg(packed + (size_t)b * DD + e), v);
            gpk[e] = v;
        }
        __syncthreads();
        for (int e = tid; e < DD; e += kLargeThreads) {
            const int i = e / D, jj = e % D;
            const Real a = gpk[i * D + jj], b = gpk[jj * D + i];
            const Real re = (i <= jj) ? a : b;
            const Real im = (i > jj) ? a : ((i < jj) ? -b : Real(0));
            SX[e] = Cx<Real>::make(im * sc, -re * sc);
        }
        __syncthreads();
        if (q >= 2) cta_mm<Real, D>(SX, SX, SX2, panels);
        if (q >= 3) cta_mm<Real, D>(SX2, SX, SX3, panels);
        const C *Xq = (q == 1) ? SX : ((q == 2) ? SX2 : SX3);
        // Horner over blocks with two ping-pong buffers P0 / P1:
        //   T = a_{q r} X^q + B_{r-1};  T <- X^q T + B_b;  B_b = sum_{l<q} a_{q b + l} X^l
        auto add_block = [&](C *T, const C *src, Real scale, int b) {
            const Real a0 = coef<Real>(p, q * b);
            const Real a1 = (q >= 2) ? coef<Real>(p, q * b + 1) : Real(0);
            const Real a2 = (q >= 3) ? coef<Real>(p, q * b + 2) : Real(0);
            for (int e = tid; e < DD; e += kLargeThreads) {
                C v = src[e];
                v.x *= scale;
                v.y *= scale;
                v.x += ((e / D) == (e % D)) ? a0 : Real(0);
                if (q >= 2) {
                    const C x = SX[e];
                    v.x = fma(a1, x.x, v.x);
                    v.y = fma(a1, x.y, v.y);
                }
                if (q >= 3) {
                    const C x = SX2[e];
                    v.x = fma(a2, x.x, v.x);
                    v.y = fma(a2, x.y, v.y);
                }
                T[e] = v;
            }
            __syncthreads();
        };
        C *cur = P0, *nxt = P1;
        add_block(cur, Xq, coef<Real>(p, q * rh), rh - 1);
        for (int b = rh - 2; b >= 0; --b) {
            cta_mm<Real, D>(Xq, cur, nxt, panels);
            add_block(nxt, nxt, Real(1), b);
            C *t2 = cur; cur = nxt; nxt = t2;
        }
        for (int i = 0; i < s; ++i) {
            cta_mm<Real, D>(cur, cur, nxt, panels);
            C *t2 = cur; cur = nxt; nxt = t2;
        }
        // leaf product R <- U_j R
        cta_mm<Real, D>(cur, SR, nxt, panels);
        for (int e = tid; e < DD; e += kLargeThreads) SR[e] = nxt[e];
        __syncthreads();
        if (tid == 0) {
            n_exp += (unsigned long long)((q - 1) + (rh - 1) + s);
            m_max = max(m_max, cls_m(code));
            s_max = max(s_max, s);
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
        double2 *dst = p.partials + (size_t)blockIdx.x * DD;
        for (int e = tid; e < DD; e += kLargeThreads) {
            const C v = SR[e];
            dst[e] = make_double2((double)v.x, (double)v.y);
            if (p.leaf_out) p.leaf_out[(size_t)blockIdx.x * DD + e] = dst[e];
            if (p.block_out) p.block_out[(size_t)blockIdx.x * DD + e] = dst[e];
        }
    }
    __threadfence();
    __syncthreads();

    // pairwise tree over blocks in FP64 (second arrival multiplies right * left); the product runs
    // through this block's scratch, viewed as FP64 matrices
    double2 *wsd = (double2 *)((unsigned char *)scratch + (size_t)blockIdx.x * kLargeSlots * DD * sizeof(C));
    int idx = blockIdx.x, n = gridDim.x, level = 0, toff = 0;
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
            double2 *L2 = wsd, *R2 = wsd + DD;
            for (int e = tid; e < DD; e += kLargeThreads) {
                L2[e] = __ldcg(gL + e);
                R2[e] = __ldcg(gR + e);
            }
            __syncthreads();
            cta_mm<double, D>(R2, L2, gL, panels);
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
}

template <typename Real, int D, int INTEG>
cudaError_t launch_large(const FusedParams &p, void *scratch, int grid, size_t smem, cudaStream_t st) {
    auto k = large_kernel<Real, D, INTEG>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kLargeThreads, smem, st>>>(p, scratch);
    return cudaGetLastError();
}

}  // namespace pm
