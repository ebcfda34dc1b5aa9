// Complex 128 x 128 FP32 matrix product on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), with FP32 accuracy from the
// three-term TF32 split (Ootomo & Yokota): x = hi + lo with hi = rn_tf32(x),
// lo = rn_tf32(x - hi); a b ~ hi_a hi_b + hi_a lo_b + lo_a hi_b.  Re C = Re A Re B - Im A Im B uses the negate-A bit
// of the instruction descriptor for the second term.
//
// One thread block of 256 threads: all threads stage k-chunks of both
// operands from global memory (L2) into shared memory in the canonical
// no-swizzle K-major layout (8-row x 16-byte core matrices) as the four
// planes hi / lo of Re / Im, three stages deep; thread 0 issues the MMAs of a
// chunk and commits them to the stage's mbarrier.  A chunk accumulates Re C in
// tensor-memory columns [0, 128) and Im C in [128, 256) of set c % 2 (set 1 at
// column 256); the threads read the finished set back with tcgen05.ld (warp w
// reads lanes 32 (w % 4) .. + 31, half of the columns), add it into register
// sums and finally store C row-major.  Every wait is bounded: after about a second without
// progress the block records kDevTimeout and skips its remaining products.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>

#include "pm_common.cuh"

namespace pm {
namespace umma {

constexpr int kStages = 3;
constexpr int KC = 16;                         // complex k per stage
constexpr int kLBO = 128;                      // bytes between core matrices along K
constexpr int kTmemCols = 512;                 // two sets of Re and Im accumulators, 128 columns each
constexpr long long kWaitCycles = 2000000000ll;

// operand formats: 3xTF32 (two TF32 terms per value, K = 8 per MMA) and split BF16x3 (three BF16
// terms per value, K = 16 per MMA); a plane holds one term of Re or Im of 128 rows x KC k
constexpr int kTF32x3 = 0, kBF16x3 = 1;
template <int F> struct Fmt;
template <> struct Fmt<kTF32x3> {
    static constexpr int TERMS = 2, ELEM = 4, KMMA = 8;
    static constexpr int PLANE = 128 * KC * ELEM;          // 8 KB
    static constexpr int SBO = (KC * ELEM / 16) * 128;     // 4 core matrices along K per 8 rows
};
template <> struct Fmt<kBF16x3> {
    static constexpr int TERMS = 3, ELEM = 2, KMMA = 16;
    static constexpr int PLANE = 128 * KC * ELEM;          // 4 KB
    static constexpr int SBO = (KC * ELEM / 16) * 128;     // 2 core matrices along K per 8 rows
};
template <int F> constexpr int stage_bytes() { return 4 * Fmt<F>::TERMS * Fmt<F>::PLANE; }  // A and B, Re and Im
constexpr int kStageBytes = 64 * 1024;  // the larger of the two formats (3xTF32: 8 planes of 8 KB)
static_assert(stage_bytes<kTF32x3>() <= kStageBytes && stage_bytes<kBF16x3>() <= kStageBytes, "stage size");
constexpr size_t kSmemBytes = (size_t)kStages * kStageBytes;

struct Ctx {
    uint32_t tmem;     // tensor-memory base address of the accumulators
    uint64_t *mbar;    // kStages mbarriers in shared memory
    uint32_t phase;    // bit s: parity of the next completion of barrier s (identical in all threads)
    int *abort;        // shared: a wait timed out, the remaining products are skipped
    unsigned *status;  // device status word of the call
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle, relative leading-dimension offset
template <int F>
__device__ __forceinline__ uint64_t desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(kLBO >> 4) << 16) |
           ((uint64_t)(Fmt<F>::SBO >> 4) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: D F32, A and B TF32 (kind::tf32) or BF16 (kind::f16), both K-major,
// M = N = 128, optional negated A
template <int F>
__host__ __device__ constexpr uint32_t idesc(bool neg_a) {
    return (1u << 4) | ((F == kTF32x3 ? 2u : 1u) << 7) | ((F == kTF32x3 ? 2u : 1u) << 10) | ((neg_a ? 1u : 0u) << 13) |
           ((uint32_t)(128 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

template <int F>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    if constexpr (F == kTF32x3)
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(id), "r"(acc));
    else
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// bounded wait for the completion of phase `parity` of an mbarrier
__device__ __forceinline__ bool wait(uint64_t *bar, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Block-level set-up and tear-down (all threads of the block call both).
__device__ __forceinline__ void setup(Ctx &cx, uint64_t *mbar, uint32_t *tmem_slot, int *abort, unsigned *status) {
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar + s)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    cx.tmem = *tmem_slot;
    cx.mbar = mbar;
    cx.phase = 0;
    cx.abort = abort;
    cx.status = status;
}

__device__ __forceinline__ void teardown(const Ctx &cx) {
    fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(cx.tmem), "r"(kTmemCols)
                     : "memory");
}

// round-to-nearest TF32 value of x (FP32 bit pattern with the low 13 bits clear)
__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// hi = rn_tf32(x), lo = rn_tf32(x - hi) of Re and Im of one complex operand into the four planes
// (Re hi, Re lo, Im hi, Im lo) at byte offset o.  Rounding both parts to nearest keeps the split
// unbiased (the tensor core would truncate a raw FP32 operand, and the truncations of all operands
// shrink them the same way).
__device__ __forceinline__ void put_split(unsigned char *planes, int o, float2 v) {
    constexpr int P = Fmt<kTF32x3>::PLANE;
    const float hr = tf32_rn(v.x), hi = tf32_rn(v.y);
    *(float *)(planes + o) = hr;
    *(float *)(planes + P + o) = tf32_rn(v.x - hr);
    *(float *)(planes + 2 * P + o) = hi;
    *(float *)(planes + 3 * P + o) = tf32_rn(v.y - hi);
}

// BF16x3: x = b0 + b1 + b2 with b0 = rn_bf16(x), b1 = rn_bf16(x - b0), b2 = rn_bf16(x - b0 - b1)
// (the differences are exact in FP32); two consecutive k of Re and Im into the six planes
// (Re b0, b1, b2, Im b0, b1, b2) at byte offset o, one 4-byte word (two BF16) per plane.
__device__ __forceinline__ void split3(float x, uint16_t (&b)[3]) {
    float r = x;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const __nv_bfloat16 h = __float2bfloat16_rn(r);
        b[t] = __bfloat16_as_ushort(h);
        r -= __bfloat162float(h);
    }
}
__device__ __forceinline__ void put_split3(unsigned char *planes, int o, float2 v0, float2 v1) {
    constexpr int P = Fmt<kBF16x3>::PLANE;
    uint16_t r0[3], r1[3], i0[3], i1[3];
    split3(v0.x, r0);
    split3(v1.x, r1);
    split3(v0.y, i0);
    split3(v1.y, i1);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        *(uint32_t *)(planes + t * P + o) = (uint32_t)r0[t] | ((uint32_t)r1[t] << 16);
        *(uint32_t *)(planes + (3 + t) * P + o) = (uint32_t)i0[t] | ((uint32_t)i1[t] << 16);
    }
}

__device__ __forceinline__ void wait_stage(Ctx &cx, int s) {
    if (!*(volatile int *)cx.abort && !wait(cx.mbar + s, (cx.phase >> s) & 1u)) {
        *(volatile int *)cx.abort = 1;
        atomicOr(cx.status, kDevTimeout);
    }
    cx.phase ^= 1u << s;
}

// C = A B; A, B, C: 128 x 128 complex FP32, row-major, global memory (C may not alias A or B).
// Called by all 256 threads of the block; `stages` is kSmemBytes of shared memory.
//
// The tensor core truncates when it adds a product into its accumulator, so a long
// accumulation chain is biased (every same-sign sum, e.g. the diagonal of X^2, comes out
// small).  Each k-chunk therefore starts a fresh accumulator, alternating between two
// tensor-memory sets, and the threads add the finished chunk into FP32 register sums with
// round-to-nearest while the tensor core works on the next chunk.  Thread (warp w, lane l)
// owns row 32 (w % 4) + l, columns [64 (w / 4), 64 (w / 4) + 64) of Re C and Im C.
template <int F>
static __device__ __noinline__ void cmul128(const float2 *__restrict__ A, const float2 *__restrict__ B,
                                            float2 *__restrict__ Cout, unsigned char *stages, Ctx &cx) {
    constexpr int NCH = 128 / KC;
    constexpr int P = Fmt<F>::PLANE, SBO = Fmt<F>::SBO;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (*(volatile int *)cx.abort) return;  // uniform: set before the last block barrier
    const uint32_t ID = idesc<F>(false), IDN = idesc<F>(true);
    const int row = (warp & 3) * 32 + lane, col0 = (warp >> 2) * 64;
    const uint32_t tl = cx.tmem + ((uint32_t)((warp & 3) * 32) << 16);
    float sre[64], sim[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) sre[j] = sim[j] = 0.f;
    // chunk c's partial sums from tensor-memory set c % 2 into the register sums
    auto gather = [&](int c) {
        wait_stage(cx, c % kStages);  // its commit: every MMA of chunk c is done
        fence_after();
        if (!__syncthreads_or(*(volatile int *)cx.abort)) {  // block-uniform: tcgen05.ld is warp-collective
            const uint32_t base = tl + (uint32_t)((c & 1) * 256 + col0);
#pragma unroll
            for (int cc = 0; cc < 64; cc += 16) {
                float re[16], im[16];
                ld16(base + (uint32_t)cc, re);
                ld16(base + 128u + (uint32_t)cc, im);
                wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    sre[cc + j] = __fadd_rn(sre[cc + j], re[j]);
                    sim[cc + j] = __fadd_rn(sim[cc + j], im[j]);
                }
            }
        }
        fence_before();
    };
    // Staging: the 32 lanes of a warp fill one core matrix (8 rows x 16 bytes) of every plane per
    // store instruction, lane -> (row % 8, 4-byte column), so the 32 stores hit 32 banks.
    //  3xTF32: thread element i of a chunk: row g * 8 + lane % 8, k = kg * 4 + lane / 8, q = 8 warp + i
    //  BF16x3: thread element i: row g * 8 + lane % 8, k = 2 kp, 2 kp + 1 with kp = kq * 4 + lane / 8,
    //          q = 4 warp + i, g = q / 2, kq = q % 2 (two BF16 per 4-byte word)
    float2 ra[8], rb[8];  // the chunk being staged, loaded one chunk ahead
    auto load = [&](int c, float2 (&xa)[8], float2 (&xb)[8]) {
        const int k0 = c * KC;
        if constexpr (F == kTF32x3) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int q = warp * 8 + i, g = q >> 2, kg = q & 3;
                const int r = g * 8 + (lane & 7), kk = kg * 4 + (lane >> 3);
                xa[i] = __ldcg(A + r * 128 + k0 + kk);
                xb[i] = __ldcg(B + (k0 + kk) * 128 + r);  // B^T: row n = r
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int q = warp * 4 + i, g = q >> 1, kq = q & 1;
                const int r = g * 8 + (lane & 7), kk = 2 * (kq * 4 + (lane >> 3));
                const float4 av = __ldcg(reinterpret_cast<const float4 *>(A + r * 128 + k0 + kk));
                xa[2 * i] = make_float2(av.x, av.y);
                xa[2 * i + 1] = make_float2(av.z, av.w);
                xb[2 * i] = __ldcg(B + (k0 + kk) * 128 + r);
                xb[2 * i + 1] = __ldcg(B + (k0 + kk + 1) * 128 + r);
            }
        }
    };
    load(0, ra, rb);
    for (int c = 0; c < NCH; ++c) {
        // stage c % kStages was last read by the MMAs of chunk c - kStages, gathered already
        const int s = c % kStages;
        float2 na[8], nb[8];
        if (c + 1 < NCH) load(c + 1, na, nb);
        unsigned char *st = stages + (size_t)s * kStageBytes;
        if constexpr (F == kTF32x3) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int q = warp * 8 + i, g = q >> 2, kg = q & 3;
                const int o = g * SBO + kg * kLBO + (lane & 7) * 16 + (lane >> 3) * 4;
                put_split(st, o, ra[i]);
                put_split(st + 4 * P, o, rb[i]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int q = warp * 4 + i, g = q >> 1, kq = q & 1;
                const int o = g * SBO + kq * kLBO + (lane & 7) * 16 + (lane >> 3) * 4;
                put_split3(st, o, ra[2 * i], ra[2 * i + 1]);
                put_split3(st + 6 * P, o, rb[2 * i], rb[2 * i + 1]);
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            ra[i] = na[i];
            rb[i] = nb[i];
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();  // also: set c % 2 was read out (chunk c - 2 gathered) by every thread
        if (tid == 0) {
            fence_after();
            const uint32_t sb = smem_u32(st);
            const uint32_t dr = cx.tmem + (uint32_t)((c & 1) * 256), di = dr + 128;
            if constexpr (F == kTF32x3) {
#pragma unroll
                for (int ks = 0; ks < KC / 8; ++ks) {
                    const uint32_t o = (uint32_t)ks * 2 * kLBO;
                    const uint64_t arh = desc<F>(sb + o), arl = desc<F>(sb + P + o);
                    const uint64_t aih = desc<F>(sb + 2 * P + o), ail = desc<F>(sb + 3 * P + o);
                    const uint64_t brh = desc<F>(sb + 4 * P + o), brl = desc<F>(sb + 5 * P + o);
                    const uint64_t bih = desc<F>(sb + 6 * P + o), bil = desc<F>(sb + 7 * P + o);
                    const uint32_t acc = ks > 0 ? 1u : 0u;  // fresh accumulator for every chunk
                    // small terms first: Re += Re A Re B - Im A Im B
                    mma<F>(dr, arl, brh, ID, acc);
                    mma<F>(dr, arh, brl, ID, 1u);
                    mma<F>(dr, arh, brh, ID, 1u);
                    mma<F>(dr, ail, bih, IDN, 1u);
                    mma<F>(dr, aih, bil, IDN, 1u);
                    mma<F>(dr, aih, bih, IDN, 1u);
                    // Im += Re A Im B + Im A Re B
                    mma<F>(di, arl, bih, ID, acc);
                    mma<F>(di, arh, bil, ID, 1u);
                    mma<F>(di, arh, bih, ID, 1u);
                    mma<F>(di, ail, brh, ID, 1u);
                    mma<F>(di, aih, brl, ID, 1u);
                    mma<F>(di, aih, brh, ID, 1u);
                }
            } else {
                // one K = 16 step; planes: A Re b0..b2, A Im b0..b2, B Re b0..b2, B Im b0..b2
                uint64_t ar[3], ai[3], br[3], bi[3];
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    ar[t] = desc<F>(sb + t * P);
                    ai[t] = desc<F>(sb + (3 + t) * P);
                    br[t] = desc<F>(sb + (6 + t) * P);
                    bi[t] = desc<F>(sb + (9 + t) * P);
                }
                // the six terms x_t y_u with t + u <= 2, small first
                constexpr int TT[6] = {2, 1, 0, 1, 0, 0}, UU[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
                for (int w = 0; w < 6; ++w) mma<F>(dr, ar[TT[w]], br[UU[w]], ID, w > 0 ? 1u : 0u);
#pragma unroll
                for (int w = 0; w < 6; ++w) mma<F>(dr, ai[TT[w]], bi[UU[w]], IDN, 1u);
#pragma unroll
                for (int w = 0; w < 6; ++w) mma<F>(di, ar[TT[w]], bi[UU[w]], ID, w > 0 ? 1u : 0u);
#pragma unroll
                for (int w = 0; w < 6; ++w) mma<F>(di, ai[TT[w]], br[UU[w]], ID, 1u);
            }
            commit(cx.mbar + s);
        }
        if (c >= 1) gather(c - 1);  // overlaps the MMAs of chunk c
    }
    gather(NCH - 1);
    if (!__syncthreads_or(*(volatile int *)cx.abort)) {
        float4 *dst = reinterpret_cast<float4 *>(Cout + row * 128 + col0);
#pragma unroll
        for (int j = 0; j < 32; ++j) dst[j] = make_float4(sre[2 * j], sim[2 * j], sre[2 * j + 1], sim[2 * j + 1]);
    }
    __syncthreads();
}

}  // namespace umma
}  // namespace pm
