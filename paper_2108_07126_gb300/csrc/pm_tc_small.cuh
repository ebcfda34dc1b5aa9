// Complex FP32 products for padded dimensions D = 32 and 64 on the tcgen05 tensor cores, and the
// block-level propagation body that runs on them.
//
// A complex product C = A B consists of four real products.  With the real and imaginary parts
// of A stacked along M ([Re A; Im A], 2 D rows) and those of B^T stacked along N ([Re B^T; Im B^T],
// 2 D rows), one chain of M = 128, N = 2 D MMAs over k computes all four at once: accumulator lane
// r < D holds row r of Re A Re B (columns 0 .. D - 1) and of Re A Im B (columns D .. 2 D - 1);
// lane D + r holds the same row of Im A Re B and Im A Im B.  The epilogue combines them with
// round-to-nearest FP32 adds: Re C = Re A Re B - Im A Im B, Im C = Re A Im B + Im A Re B.  Every
// operand value is staged exactly once; at D = 32 lanes 64 .. 127 see zero rows of A.
//
// Operand precision as for D = 128 (pm_umma.cuh): 3xTF32 (x = hi + lo, three MMAs per chunk) or
// split BF16x3 (x = b0 + b1 + b2, six MMAs per chunk), every term rounded to nearest.  A chunk is
// one MMA K step (8 complex k for TF32, 16 for BF16) and accumulates into a fresh set of
// tensor-memory columns, which is read back with tcgen05.ld and added into FP32 register sums with
// round-to-nearest adds (the accumulator itself truncates).  The staging of chunk c + 1 and the
// read-back of chunk c - 1 overlap the MMAs of chunk c.  Every wait is bounded (umma::wait_idx).
//
// The working matrices of the body live in shared memory in planar form: a real and an imaginary
// plane of D rows padded to D + 1 floats, so that a warp touching one column of 32 consecutive
// rows hits 32 distinct banks (staging of B^T, epilogue stores).
#pragma once

#include "pm_fused.cuh"
#include "pm_umma.cuh"

namespace pm {
namespace tcs {

// per-format chunk geometry: K = complex k per chunk (= one MMA K step), VPL = values per
// 16-byte core-matrix row, TERMS = split terms per value
template <int F> struct Fmt;
template <> struct Fmt<umma::kTF32x3> { static constexpr int TERMS = 2, KC = 8, VPL = 4; };
template <> struct Fmt<umma::kBF16x3> { static constexpr int TERMS = 3, KC = 16, VPL = 8; };

// One operand plane: 128 rows x 2 core-matrix columns (32 bytes of k per row).  Core matrix
// (row group g, k group kg) sits at g * kSBO + kg * kLBO; row r of it at + 16 (r % 8).
constexpr int kRows = 128, kLBO = 128, kSBO = 256;
constexpr int kPlane = kRows / 8 * kSBO;  // 4 KB

template <int F> __host__ __device__ constexpr int stage_bytes() { return 2 * Fmt<F>::TERMS * kPlane; }

template <int D> struct PGeo {
    static constexpr int LD = D + 1;          // row stride of a plane (floats)
    static constexpr int PL = D * LD;         // floats per plane
    static constexpr int MAT = 2 * PL;        // floats per planar complex matrix
};

// Pipeline per (D, format): two operand stages and two accumulator sets of 2 D tensor-memory
// columns; chunk c is staged into stage c % 2 and accumulated into set c % 2 while chunk c - 1 is
// read back.  All working matrices stay in shared memory.  At D = 32 the body fits two blocks per
// SM.  (Deeper pipelines, a dedicated issuing warp and read-back every 16 or 32 k were measured
// slower at these sizes: the per-chunk costs -- operand split and staging, read-back, and the
// issue of an MMA, which holds the issuing thread for about its execution time -- do not overlap
// enough to pay for their synchronisation.)
template <int D, int F> struct Cfg {
    static constexpr int NCH = D / Fmt<F>::KC;
    static constexpr int NST = 2;
    static constexpr int NMAT_SMEM = 5;  // X, X^2, X^3, Horner / squaring matrix, leaf product
    static constexpr int MIN_BLOCKS = D == 32 ? 2 : 1;
};

template <int D, int F>
__host__ __device__ constexpr size_t smem_bytes(int n_basis) {
    return (size_t)Cfg<D, F>::NST * stage_bytes<F>() +
           (size_t)Cfg<D, F>::NMAT_SMEM * PGeo<D>::MAT * sizeof(float) + (size_t)(n_basis + 1) * sizeof(float) + 64;
}

// tensor-memory columns: NST accumulator sets of 2 D columns
template <int D, int F> __host__ __device__ constexpr uint32_t tmem_cols() { return Cfg<D, F>::NST * 2 * D; }

// shared-memory matrix descriptor of a plane: K-major, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(kLBO >> 4) << 16) | ((uint64_t)(kSBO >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// Stage chunk c (complex k in [c K, c K + K)) of A and B into stage buffer st: operand o = 0 (A,
// row r of the M stack = row r % D of Re A or Im A) or 1 (B, row r of the N stack = column r % D
// of Re B or Im B), k group g.  One item = one 16-byte core-matrix row in every term plane; the
// 32 lanes of a warp take 32 consecutive rows of one operand and k group.
// ptid: index among the NP staging threads (NP a multiple of 32, so a warp's 32 items stay inside
// one operand and k group).
template <int D, int F, int NP>
__device__ __forceinline__ void stage_chunk(const float *A, const float *B, unsigned char *st, int c, int ptid) {
    using G = PGeo<D>;
    constexpr int LD = G::LD, PL = G::PL, VPL = Fmt<F>::VPL, TERMS = Fmt<F>::TERMS;
    constexpr int NI = 2 * (2 * D) * 2;
    static_assert(NP % 32 == 0 && (2 * D) % 32 == 0, "warp-uniform operand and k group");
    const int k0 = c * Fmt<F>::KC;
#pragma unroll
    for (int i = 0; i < (NI + NP - 1) / NP; ++i) {
        const int it = ptid + NP * i;
        if (it >= NI) break;  // warp-uniform
        const int r = it % (2 * D), o = (it / (2 * D)) & 1, g = it / (4 * D);
        const int rr = r < D ? r : r - D, kk = k0 + g * VPL;
        const float *pl = (o ? B : A) + (r < D ? 0 : PL);
        float v[VPL];
        if (o == 0) {
#pragma unroll
            for (int t = 0; t < VPL; ++t) v[t] = pl[rr * LD + kk + t];
        } else {
#pragma unroll
            for (int t = 0; t < VPL; ++t) v[t] = pl[(kk + t) * LD + rr];
        }
        unsigned char *dst = st + o * TERMS * kPlane + (r >> 3) * kSBO + g * kLBO + (r & 7) * 16;
        if constexpr (F == umma::kTF32x3) {
            float4 hi, lo;
            float *ph = &hi.x, *pl2 = &lo.x;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                ph[t] = umma::tf32_rn(v[t]);
                pl2[t] = umma::tf32_rn(v[t] - ph[t]);
            }
            *(float4 *)dst = hi;
            *(float4 *)(dst + kPlane) = lo;
        } else {
            uint4 w[3];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                uint32_t x[3];
                umma::split3_pair(v[2 * h], v[2 * h + 1], x);
#pragma unroll
                for (int t = 0; t < 3; ++t) (&w[t].x)[h] = x[t];
            }
#pragma unroll
            for (int t = 0; t < 3; ++t) *(uint4 *)(dst + t * kPlane) = w[t];
        }
    }
}

// C = A B for planar complex D x D FP32 matrices in shared memory.  C may alias A or B (every
// operand read happens before the first store of C).  Called by all 256 threads: all of them stage
// and read back, thread 0 issues the MMAs; uses the mbarriers kBarSDone + 0, 1 of cx and
// accumulator columns [0, 4 D) of its tensor memory; ends with a block barrier.
template <int D, int F>
static __device__ __noinline__ void cmul(const float *A, const float *B, float *C, unsigned char *stages,
                                         umma::Ctx &cx) {
    using G = PGeo<D>;
    constexpr int LD = G::LD, PL = G::PL, NCH = Cfg<D, F>::NCH, SB = stage_bytes<F>();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = warp & 3, h = warp >> 2;  // tensor-memory lane quadrant, column half
    const bool active = 32 * q < 2 * D;     // warp-uniform: lanes beyond 2 D hold zero rows
    if (*(volatile int *)cx.abort) return;  // uniform: set before the last block barrier
    const uint32_t base0 = cx.cnt[umma::kBarSDone], base1 = cx.cnt[umma::kBarSDone + 1];
    float s[D];
#pragma unroll
    for (int j = 0; j < D; ++j) s[j] = 0.f;

    auto issue = [&](int c) {
        const uint32_t sb = umma::smem_u32(stages + (c & 1) * SB);
        const uint32_t d = cx.tmem + (uint32_t)((c & 1) * 2 * D);
        constexpr uint32_t id = umma::idesc<F>(false, 2 * D);
        if constexpr (F == umma::kTF32x3) {
            const uint32_t ah = sb, al = sb + kPlane, bh = sb + 2 * kPlane, bl = sb + 3 * kPlane;
            umma::mma<F>(d, sdesc(al), sdesc(bh), id, 0u);  // small terms first, fresh accumulator
            umma::mma<F>(d, sdesc(ah), sdesc(bl), id, 1u);
            umma::mma<F>(d, sdesc(ah), sdesc(bh), id, 1u);
        } else {
            constexpr int TT[6] = {2, 1, 0, 1, 0, 0}, UU[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
            for (int w = 0; w < 6; ++w)
                umma::mma<F>(d, sdesc(sb + TT[w] * kPlane), sdesc(sb + (3 + UU[w]) * kPlane), id, w > 0 ? 1u : 0u);
        }
        umma::commit(cx.bar + umma::kBarSDone + (c & 1));
    };
    // chunk c's sums from accumulator set c % 2 into the register sums
    auto gather = [&](int c) {
        umma::wait_idx(cx, umma::kBarSDone + (c & 1), ((c & 1) ? base1 : base0) + (uint32_t)(c >> 1));
        umma::fence_after();
        if (active && !__any_sync(0xffffffffu, *(volatile int *)cx.abort)) {
            const uint32_t tb = cx.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((c & 1) * 2 * D + h * D);
#pragma unroll
            for (int cc = 0; cc < D; cc += 32) {
                float v0[16], v1[16];
                umma::ld16(tb + (uint32_t)cc, v0);
                umma::ld16(tb + (uint32_t)cc + 16u, v1);
                umma::wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    s[cc + j] = __fadd_rn(s[cc + j], v0[j]);
                    s[cc + 16 + j] = __fadd_rn(s[cc + 16 + j], v1[j]);
                }
            }
        }
        umma::fence_before();
    };

    stage_chunk<D, F, 256>(A, B, stages, 0, tid);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        umma::fence_after();
        issue(0);
    }
    for (int c = 1; c <= NCH; ++c) {
        // stage c % 2 was last read by the MMAs of chunk c - 2, whose completion every thread saw
        // in gather(c - 2); accumulator set c % 2 was last read in gather(c - 2), before this barrier
        if (c < NCH) {
            stage_chunk<D, F, 256>(A, B, stages + (c & 1) * SB, c, tid);
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        }
        __syncthreads();
        if (c < NCH && tid == 0) {
            umma::fence_after();
            issue(c);
        }
        gather(c - 1);
    }
    cx.cnt[umma::kBarSDone] += (uint32_t)((NCH + 1) / 2);
    cx.cnt[umma::kBarSDone + 1] += (uint32_t)(NCH / 2);
    const bool ab = __syncthreads_or(*(volatile int *)cx.abort);
    const int L = 32 * q + lane;
    const bool im_row = L >= D;
    const int r = im_row ? L - D : L;
    if (!ab && active && !im_row) {
        // Re A Re B -> Re C, Re A Im B -> Im C
        float *dst = C + (h ? PL : 0) + r * LD;
#pragma unroll
        for (int j = 0; j < D; ++j) dst[j] = s[j];
    }
    __syncthreads();
    if (!ab && active && im_row) {
        // Im A Re B -> + Im C, Im A Im B -> - Re C
        float *dst = C + (h ? 0 : PL) + r * LD;
        if (h) {
#pragma unroll
            for (int j = 0; j < D; ++j) dst[j] = __fsub_rn(dst[j], s[j]);
        } else {
#pragma unroll
            for (int j = 0; j < D; ++j) dst[j] = __fadd_rn(dst[j], s[j]);
        }
    }
    __syncthreads();
}

// One leaf (slices [N blk / nblk, N (blk + 1) / nblk)) of one problem by one thread block of 256
// threads, products on the tensor cores: the method of large_body (effective coefficients, FP64
// norm bound and Taylor class, assembly of the packed exponent, Paterson-Stockmeyer on
// A = -i G / 2^s, s squarings, leaf product; or the Chebyshev series when p.cheb_m is set), then
// one Newton-Schulz step on the leaf product and its FP64 copy to p.partials[blk].  smem:
// smem_bytes<D, F>(n_basis); cx: set up with at least tmem_cols<D, F>() columns.
template <int D, int INTEG, int F>
__device__ void body(const FusedParams &p, int blk, int nblk, unsigned char *smem, umma::Ctx &cx) {
    using G = PGeo<D>;
    using K = Cfg<D, F>;
    constexpr int LD = G::LD, PL = G::PL, MAT = G::MAT, DD = D * D;
    constexpr int SB = stage_bytes<F>();
    static_assert(DD % (4 * 256) == 0, "element passes take four entries per thread and step");
    __shared__ int s_code;
    unsigned char *stages = smem;
    float *mats = (float *)(smem + K::NST * SB);
    float *X = mats, *X2 = mats + MAT, *X3 = mats + 2 * MAT, *Tm = mats + 3 * MAT;
    float *R = mats + 4 * MAT;
    float *gam = mats + K::NMAT_SMEM * MAT;
    const int tid = threadIdx.x, nb = p.n_basis;
    const float *packed = (const float *)p.packed;

    // the A planes' rows 2 D .. 127 must read as zeros (D = 32); staging never writes them
    for (int e = tid; e < K::NST * SB / 16; e += 256) reinterpret_cast<float4 *>(stages)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t j0 = p.n_steps * blk / nblk;
    const int len = (int)(p.n_steps * (blk + 1) / nblk - j0);
    for (int e = tid; e < DD; e += 256) {
        const int i = e / D, jj = e % D;
        R[i * LD + jj] = (i == jj) ? 1.f : 0.f;
        R[PL + i * LD + jj] = 0.f;
    }
    unsigned flags = 0;
    unsigned long long n_exp = 0;
    int m_max = 0, s_max = 0;
    const bool cheb = p.cheb_m != nullptr;
    const int mch = cheb ? *p.cheb_m : 0;
    const float ib = cheb ? (float)*p.cheb_inv_beta : 0.f;
    __syncthreads();

    auto mul = [&](const float *A, const float *B, float *C) { cmul<D, F>(A, B, C, stages, cx); };
    auto leaf_product = [&](const float *U) { mul(U, R, R); };  // R <- U R (later slice on the left)

    for (int t = 0; t < len; ++t) {
        const int64_t j = j0 + t;
        if (tid == 0) {
            slice_coefficients<float, INTEG, 1>(p, j, true, gam);
            double nu = 0.0;
            for (int e = 0; e < nb; ++e) nu = fma(fabs((double)gam[e]), p.bnorm1[e], nu);
            s_code = cheb ? 0 : p.cls_code[find_class(p, nu, &flags)];
        }
        __syncthreads();
        const int code = s_code;
        const int q = cls_q(code), rh = cls_r(code), s = cls_s(code) + p.extra_squarings;
        const float sc = pow2neg<float>(s);
        // packed exponent sum_b gamma_b P_b (real D x D: upper triangle Re G, strict lower Im G) into
        // the free Horner matrix, four entries per thread and step, the basis read once from L2
        float *gpk = Tm;
        for (int e0 = tid; e0 < DD / 4; e0 += 256) {
            float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
            for (int b = 0; b < nb; ++b) {
                float w[4];
                ld4<float>(packed + (size_t)b * DD + 4 * e0, w);
                const float g = gam[b];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = fmaf(g, w[u], v[u]);
            }
            const int i = (4 * e0) / D, jj = (4 * e0) % D;
#pragma unroll
            for (int u = 0; u < 4; ++u) gpk[i * LD + jj + u] = v[u];
        }
        __syncthreads();
        // Hermitian unpack into A = -i G / 2^s (Taylor) or X = G / beta (Chebyshev)
        for (int e = tid; e < DD; e += 256) {
            const int i = e / D, jj = e % D;
            const float a = gpk[i * LD + jj], b = gpk[jj * LD + i];
            const float re = (i <= jj) ? a : b;
            const float im = (i > jj) ? a : ((i < jj) ? -b : 0.f);
            X[i * LD + jj] = cheb ? re * ib : im * sc;
            X[PL + i * LD + jj] = cheb ? im * ib : -re * sc;
        }
        __syncthreads();
        if (cheb) {
            // Clenshaw (Sec. 2.1, Algorithm 1): D_m = a_m I, D_{m+1} = 0;
            // D_k = a_k I + 2 X D_{k+1} - D_{k+2}; exp(-i G) = D_0 - D_2
            const float2 *ak = (const float2 *)p.cheb_coef;
            float *d1 = X2, *d2 = X3, *nw = Tm;
            for (int e = tid; e < DD; e += 256) {
                const int i = e / D, jj = e % D, o = i * LD + jj;
                d1[o] = (i == jj) ? ak[mch].x : 0.f;
                d1[PL + o] = (i == jj) ? ak[mch].y : 0.f;
                d2[o] = 0.f;
                d2[PL + o] = 0.f;
            }
            __syncthreads();
            for (int k = mch - 1; k >= 0; --k) {
                mul(X, d1, nw);
                const float2 a_k = ak[k];
                for (int e = tid; e < DD; e += 256) {
                    const int i = e / D, jj = e % D, o = i * LD + jj;
                    float vr = 2.f * nw[o] - d2[o], vi = 2.f * nw[PL + o] - d2[PL + o];
                    if (i == jj) {
                        vr += a_k.x;
                        vi += a_k.y;
                    }
                    nw[o] = (k == 0) ? vr - d2[o] : vr;
                    nw[PL + o] = (k == 0) ? vi - d2[PL + o] : vi;
                }
                __syncthreads();
                if (k > 0) {
                    float *t2 = d2;
                    d2 = d1;
                    d1 = nw;
                    nw = t2;
                }
            }
            leaf_product(nw);
            if (tid == 0) {
                n_exp += (unsigned long long)mch;
                m_max = max(m_max, mch);
            }
            continue;
        }
        if (q >= 2) mul(X, X, X2);
        if (q >= 3) mul(X2, X, X3);
        const float *Xq = (q == 1) ? X : ((q == 2) ? X2 : X3);
        // Horner over blocks: T = a_{q r} X^q + B_{r-1}; T <- X^q T + B_b, B_b = sum_{l<q} a_{q b + l} X^l
        auto add_block = [&](const float *src, float scale, int b) {
            const float a0 = coef<float>(p, q * b);
            const float a1 = (q >= 2) ? coef<float>(p, q * b + 1) : 0.f;
            const float a2 = (q >= 3) ? coef<float>(p, q * b + 2) : 0.f;
            for (int e = tid; e < DD; e += 256) {
                const int i = e / D, jj = e % D, o = i * LD + jj;
                float vr = src[o] * scale, vi = src[PL + o] * scale;
                if (i == jj) vr += a0;
                if (q >= 2) {
                    vr = fmaf(a1, X[o], vr);
                    vi = fmaf(a1, X[PL + o], vi);
                }
                if (q >= 3) {
                    vr = fmaf(a2, X2[o], vr);
                    vi = fmaf(a2, X2[PL + o], vi);
                }
                Tm[o] = vr;
                Tm[PL + o] = vi;
            }
            __syncthreads();
        };
        add_block(Xq, coef<float>(p, q * rh), rh - 1);
        for (int b = rh - 2; b >= 0; --b) {
            mul(Xq, Tm, Tm);
            add_block(Tm, 1.f, b);
        }
        for (int i = 0; i < s; ++i) mul(Tm, Tm, Tm);
        leaf_product(Tm);
        if (tid == 0) {
            n_exp += (unsigned long long)((q - 1) + (rh - 1) + s);
            m_max = max(m_max, cls_m(code));
            s_max = max(s_max, s);
        }
    }

    // one Newton-Schulz step of the polar iteration, R <- R (3 I - R^dagger R) / 2 (the exact
    // product is unitary; the truncating accumulation and FP32 rounding drift R off it)
    if (p.unitary_step && len > 0) {
        for (int e = tid; e < DD; e += 256) {
            const int i = e / D, jj = e % D;
            X[i * LD + jj] = R[jj * LD + i];
            X[PL + i * LD + jj] = -R[PL + jj * LD + i];
        }
        __syncthreads();
        mul(X, R, X2);  // R^dagger R
        for (int e = tid; e < DD; e += 256) {
            const int i = e / D, jj = e % D, o = i * LD + jj;
            X2[o] = ((i == jj) ? 3.f : 0.f) - X2[o];
            X2[PL + o] = -X2[PL + o];
        }
        __syncthreads();
        mul(R, X2, R);
        for (int e = tid; e < DD; e += 256) {
            const int i = e / D, jj = e % D, o = i * LD + jj;
            R[o] *= 0.5f;
            R[PL + o] *= 0.5f;
        }
        __syncthreads();
    }

    if (tid == 0 && len > 0) {
        atomicAdd(&p.counters[0], n_exp);
        atomicAdd(&p.counters[1], (unsigned long long)len);
        atomicMax(&p.counters[2], (unsigned long long)m_max);
        atomicMax(&p.counters[3], (unsigned long long)s_max);
    }
    if (flags) atomicOr(&p.status[0], flags);
    double2 *dst = p.partials + (size_t)blk * DD;
    for (int e = tid; e < DD; e += 256) {
        const int i = e / D, jj = e % D;
        dst[e] = make_double2((double)R[i * LD + jj], (double)R[PL + i * LD + jj]);
    }
    __threadfence();
    __syncthreads();
}

}  // namespace tcs
}  // namespace pm
