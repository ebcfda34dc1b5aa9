// Complex 128 x 128 FP32 matrix product on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), with FP32 accuracy from a split
// of every operand into narrower terms: three-term TF32 (Ootomo & Yokota:
// x = hi + lo, hi = rn_tf32(x), lo = rn_tf32(x - hi); a b ~ hi hi + hi lo +
// lo hi) or split BF16x3 (x = b0 + b1 + b2; six products).  Re C = Re A Re B -
// Im A Im B uses the negate-A bit of the instruction descriptor.
//
// One thread block of 256 threads, warp-specialised: warps 1..7 stage 16-k
// chunks of A and B^T from global memory (L2) into three shared-memory stages
// in the canonical no-swizzle K-major layout (8-row x 16-byte core matrices),
// one plane per term of Re / Im, and signal a "full" mbarrier; thread 0
// issues the chunk's MMAs into a fresh accumulator set in tensor memory (two
// sets of Re / Im x 128 columns) and commits them to the stage's "done"
// mbarrier; all eight warps read the finished set back with tcgen05.ld (warp w
// reads lanes 32 (w % 4) .. + 31, half of the columns), add it into FP32
// register sums with round-to-nearest (the tensor-core accumulator truncates)
// and release the set on a "free" mbarrier.  Staging, MMA execution and
// read-back of neighbouring chunks overlap; no block-wide barrier inside the
// product.  Every wait is bounded: after about a second without progress the
// block records kDevTimeout and skips its remaining products.
#pragma once

#include <cstdint>

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

// mbarriers of the product pipeline: done[3] (the MMAs of a stage finished, one tcgen05.commit),
// full[3] (a stage was written, one arrival per producer warp), free[2] (an accumulator set was
// read back, one arrival per warp)
constexpr int kProducerWarps = 7;
// 8, 9: done barriers of the small-dimension product of pm_tc_small.cuh (one commit each)
constexpr int kBarDone = 0, kBarFull = 3, kBarFree = 6, kBarsBig = 8, kBarSDone = 8, kBars = 10;

struct Ctx {
    uint32_t tmem;          // tensor-memory base address of the accumulators
    uint32_t ncols;         // tensor-memory columns allocated by setup
    uint64_t *bar;          // kBars mbarriers in shared memory
    uint32_t cnt[kBars];    // completions of each barrier consumed so far (identical in all threads)
    int *abort;             // shared: a wait timed out, the remaining products are skipped
    unsigned *status;       // device status word of the call
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle, relative leading-dimension offset
template <int F>
__device__ __forceinline__ uint64_t desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(kLBO >> 4) << 16) |
           ((uint64_t)(Fmt<F>::SBO >> 4) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: D F32, A and B TF32 (kind::tf32) or BF16 (kind::f16), both K-major,
// M = 128, N = 128 or 256, optional negated A
template <int F>
__host__ __device__ constexpr uint32_t idesc(bool neg_a, int n = 128) {
    return (1u << 4) | ((F == kTF32x3 ? 2u : 1u) << 7) | ((F == kTF32x3 ? 2u : 1u) << 10) | ((neg_a ? 1u : 0u) << 13) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
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
__device__ __forceinline__ void setup(Ctx &cx, uint64_t *bar, uint32_t *tmem_slot, int *abort, unsigned *status,
                                      uint32_t ncols = kTmemCols) {
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int b = 0; b < kBars; ++b) {
            const int count = (b < kBarFull || b >= kBarsBig) ? 1 : (b < kBarFree ? kProducerWarps : 8);
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar + b)), "r"(count) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    cx.tmem = *tmem_slot;
    cx.ncols = ncols;
    cx.bar = bar;
    for (int b = 0; b < kBars; ++b) cx.cnt[b] = 0;
    cx.abort = abort;
    cx.status = status;
}

__device__ __forceinline__ void teardown(const Ctx &cx) {
    fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(cx.tmem), "r"(cx.ncols)
                     : "memory");
}

// round-to-nearest TF32 value of x (ties away from zero): add half a unit of the 10-bit mantissa
// to the magnitude bits and clear the 13 low bits (integer pipe; a carry moves into the exponent
// as it should).  Finite inputs only.
__device__ __forceinline__ float tf32_rn(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// hi = rn_tf32(x), lo = rn_tf32(x - hi) of Re and Im of four consecutive k of one row into the
// 16-byte row of a core matrix in four planes, at byte offset o: Re hi at planes + o, then Re lo,
// Im hi, Im lo at the plane offsets PRL, PIH, PIL.  Rounding both parts to nearest keeps the split
// unbiased (the tensor core would truncate a raw FP32 operand, and the truncations of all operands
// shrink them the same way).
template <int PRL, int PIH, int PIL>
__device__ __forceinline__ void put_split(unsigned char *planes, int o, const float2 (&v)[4]) {
    float4 rh, rl, ih, il;
    float *prh = &rh.x, *prl = &rl.x, *pih = &ih.x, *pil = &il.x;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        prh[t] = tf32_rn(v[t].x);
        prl[t] = tf32_rn(v[t].x - prh[t]);
        pih[t] = tf32_rn(v[t].y);
        pil[t] = tf32_rn(v[t].y - pih[t]);
    }
    *(float4 *)(planes + o) = rh;
    *(float4 *)(planes + PRL + o) = rl;
    *(float4 *)(planes + PIH + o) = ih;
    *(float4 *)(planes + PIL + o) = il;
}

// BF16x3: x = b0 + b1 + b2 with b0 = rn_bf16(x), b1 = rn_bf16(x - b0), b2 = rn_bf16(x - b0 - b1)
// (the differences are exact in FP32).  Round to nearest even: add 0x7FFF plus the lowest kept
// bit to the FP32 bits and keep the upper half (integer pipe; finite inputs only).
__device__ __forceinline__ uint32_t bf16_rne_bits(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}
// the three terms of x and y, packed two BF16 per word (x in the low half)
__device__ __forceinline__ void split3_pair(float x, float y, uint32_t (&w)[3]) {
    float rx = x, ry = y;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const uint32_t hx = bf16_rne_bits(rx), hy = bf16_rne_bits(ry);
        w[t] = hx | (hy << 16);
        rx -= __uint_as_float(hx << 16);
        ry -= __uint_as_float(hy << 16);
    }
}
// eight consecutive k of Re and Im of one row into the 16-byte row of a core matrix in six planes
// at byte offset o.  RS / IS: bytes between the planes of consecutive terms of Re / Im; IM: offset
// of the Im planes.
template <int RS, int IM, int IS>
__device__ __forceinline__ void put_split3(unsigned char *planes, int o, const float2 (&v)[8]) {
    uint4 re[3], im[3];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        uint32_t wr[3], wi[3];
        split3_pair(v[2 * h].x, v[2 * h + 1].x, wr);
        split3_pair(v[2 * h].y, v[2 * h + 1].y, wi);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            (&re[t].x)[h] = wr[t];
            (&im[t].x)[h] = wi[t];
        }
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        *(uint4 *)(planes + t * RS + o) = re[t];
        *(uint4 *)(planes + IM + t * IS + o) = im[t];
    }
}

// bounded wait for completion number k (0-based) of barrier b
__device__ __forceinline__ void wait_idx(Ctx &cx, int b, uint32_t k) {
    if (!*(volatile int *)cx.abort && !wait(cx.bar + b, k & 1u)) {
        *(volatile int *)cx.abort = 1;
        atomicOr(cx.status, kDevTimeout);
    }
}

__device__ __forceinline__ void arrive(uint64_t *bar) {
    asm volatile("{\n.reg .b64 arrst;\nmbarrier.arrive.shared::cta.b64 arrst, [%0];\n}\n" ::"r"(smem_u32(bar)) : "memory");
}

// C = A B for one 128 x 128 block of complex FP32 output: A is 128 x KDIM, B is KDIM x 128, all
// row-major in global memory with row stride LD (C may not alias A or B).  LD = KDIM = 128 is the
// whole d = 128 product; d = 256 takes four blocks with LD = KDIM = 256.  Called by all 256
// threads of the block; `stages` is kSmemBytes of shared memory.  Thread (warp w, lane l) owns
// row 32 (w % 4) + l, columns [64 (w / 4), 64 (w / 4) + 64) of Re C and Im C.
template <int F, int LD = 128, int KDIM = 128>
static __device__ __noinline__ void cmul128(const float2 *__restrict__ A, const float2 *__restrict__ B,
                                            float2 *__restrict__ Cout, unsigned char *stages, Ctx &cx) {
    constexpr int NCH = KDIM / KC;
    constexpr int P = Fmt<F>::PLANE, SBO = Fmt<F>::SBO;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (*(volatile int *)cx.abort) return;  // uniform: set before the last block barrier
    const uint32_t ID = idesc<F>(false), IDN = idesc<F>(true), ID2 = idesc<F>(false, 256);
    const int row = (warp & 3) * 32 + lane, col0 = (warp >> 2) * 64;
    const uint32_t tl = cx.tmem + ((uint32_t)((warp & 3) * 32) << 16);
    // completions of each barrier before this product: chunk c is use c / 3 of stage c % 3 and
    // use c / 2 of accumulator set c % 2
    uint32_t base[kBarsBig];
#pragma unroll
    for (int b = 0; b < kBarsBig; ++b) base[b] = cx.cnt[b];
    float sre[64], sim[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) sre[j] = sim[j] = 0.f;

    // chunk c's partial sums from tensor-memory set c % 2 into the register sums, then release the set
    auto gather = [&](int c) {
        wait_idx(cx, kBarDone + c % kStages, base[kBarDone + c % kStages] + c / kStages);
        fence_after();
        if (!__any_sync(0xffffffffu, *(volatile int *)cx.abort)) {  // warp-uniform: tcgen05.ld is collective
            const uint32_t tb = tl + (uint32_t)((c & 1) * 256 + col0);
#pragma unroll
            for (int cc = 0; cc < 64; cc += 16) {
                float re[16], im[16];
                ld16(tb + (uint32_t)cc, re);
                ld16(tb + 128u + (uint32_t)cc, im);
                wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    sre[cc + j] = __fadd_rn(sre[cc + j], re[j]);
                    sim[cc + j] = __fadd_rn(sim[cc + j], im[j]);
                }
            }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) arrive(cx.bar + kBarFree + (c & 1));
    };

    // producer warp p = warp - 1 stages warp-items q = p, p + 7, ... of a chunk.  A warp-item is 32
    // rows x one 16-byte core-matrix column of every plane (4 TF32 or 8 BF16 along k): lane l takes
    // row 32 rg + l, so each quarter warp writes one whole core matrix (conflict-free 16-byte stores).
    // Items 0 .. NA - 1 are rows of A (k contiguous in global memory), NA .. 2 NA - 1 rows of B^T
    // (32 consecutive columns of B per load instruction).  The loads of chunk c + 1 go out right
    // after chunk c is published, so their latency overlaps the read-back of chunk c - 1 and the
    // MMAs of chunk c.
    constexpr int VPL = 16 / Fmt<F>::ELEM;  // k per core-matrix row
    constexpr int NKG = KC / VPL;           // core-matrix columns per chunk
    constexpr int NA = 4 * NKG, NITEM = 2 * NA;
    constexpr int NIT = (NITEM + kProducerWarps - 1) / kProducerWarps;
    float2 v[NIT][VPL];  // the next chunk's operands
    auto load = [&](int c) {
        const int p = warp - 1, k0 = c * KC;
#pragma unroll
        for (int i = 0; i < NIT; ++i) {
            const int q = p + kProducerWarps * i;
            const int qa = q % NA, r = (qa / NKG) * 32 + lane, kk = k0 + (qa % NKG) * VPL;
            if (q < NA) {
                // written by this block before its last barrier: plain (coherent) loads
                const float4 *src = reinterpret_cast<const float4 *>(A + (size_t)r * LD + kk);
#pragma unroll
                for (int h = 0; h < VPL / 2; ++h) {
                    const float4 a = src[h];
                    v[i][2 * h] = make_float2(a.x, a.y);
                    v[i][2 * h + 1] = make_float2(a.z, a.w);
                }
            } else if (q < NITEM) {
#pragma unroll
                for (int t = 0; t < VPL; ++t) v[i][t] = __ldcg(B + (size_t)(kk + t) * LD + r);
            }
        }
    };
    auto stage = [&](int c) {
        const int p = warp - 1;
        unsigned char *st = stages + (size_t)(c % kStages) * kStageBytes;
#pragma unroll
        for (int i = 0; i < NIT; ++i) {
            const int q = p + kProducerWarps * i;
            const int qa = q % NA;
            const int o = ((qa / NKG) * 4 + (lane >> 3)) * SBO + (qa % NKG) * kLBO + (lane & 7) * 16;
            if constexpr (F == kTF32x3) {
                if (q < NA) put_split<P, 2 * P, 3 * P>(st, o, v[i]);                    // A: Re hi, Re lo, Im hi, Im lo
                else if (q < NITEM) put_split<2 * P, P, 3 * P>(st + 4 * P, o, v[i]);  // B: Re hi, Im hi, Re lo, Im lo
            } else {
                if (q < NA) put_split3<P, 3 * P, P>(st, o, v[i]);                       // A: Re b0..b2, Im b0..b2
                else if (q < NITEM) put_split3<2 * P, P, 2 * P>(st + 6 * P, o, v[i]);   // B: Re b_t, Im b_t pairs
            }
        }
    };

    // thread 0: the MMAs of chunk c into accumulator set c % 2.  The B planes of a term hold Re and
    // Im back to back (256 rows), so one N = 256 MMA of a Re A term adds Re A Re B into the Re
    // columns and Re A Im B into the Im columns of the set; the Im A terms take two N = 128 MMAs.
    auto issue = [&](int c) {
        const int s = c % kStages;
        const uint32_t sb = smem_u32(stages + (size_t)s * kStageBytes);
        const uint32_t dr = cx.tmem + (uint32_t)((c & 1) * 256), di = dr + 128;
        if constexpr (F == kTF32x3) {
#pragma unroll
            for (int ks = 0; ks < KC / 8; ++ks) {
                const uint32_t o = (uint32_t)ks * 2 * kLBO;
                const uint64_t arh = desc<F>(sb + o), arl = desc<F>(sb + P + o);
                const uint64_t aih = desc<F>(sb + 2 * P + o), ail = desc<F>(sb + 3 * P + o);
                const uint64_t brh = desc<F>(sb + 4 * P + o), bih = desc<F>(sb + 5 * P + o);  // [Re; Im] hi
                const uint64_t brl = desc<F>(sb + 6 * P + o), bil = desc<F>(sb + 7 * P + o);  // [Re; Im] lo
                const uint32_t acc = ks > 0 ? 1u : 0u;  // fresh accumulator for every chunk
                // small terms first: [Re | Im] += Re A [Re B | Im B]
                mma<F>(dr, arl, brh, ID2, acc);
                mma<F>(dr, arh, brl, ID2, 1u);
                mma<F>(dr, arh, brh, ID2, 1u);
                // Re -= Im A Im B, Im += Im A Re B
                mma<F>(dr, ail, bih, IDN, 1u);
                mma<F>(dr, aih, bil, IDN, 1u);
                mma<F>(dr, aih, bih, IDN, 1u);
                mma<F>(di, ail, brh, ID, 1u);
                mma<F>(di, aih, brl, ID, 1u);
                mma<F>(di, aih, brh, ID, 1u);
            }
        } else {
            // one K = 16 step; planes: A Re b0..b2, A Im b0..b2, then B Re b_t, Im b_t for t = 0..2
            uint64_t ar[3], ai[3], br[3], bi[3];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                ar[t] = desc<F>(sb + t * P);
                ai[t] = desc<F>(sb + (3 + t) * P);
                br[t] = desc<F>(sb + (6 + 2 * t) * P);
                bi[t] = desc<F>(sb + (7 + 2 * t) * P);
            }
            // the six terms x_t y_u with t + u <= 2, small first
            constexpr int TT[6] = {2, 1, 0, 1, 0, 0}, UU[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
            for (int w = 0; w < 6; ++w) mma<F>(dr, ar[TT[w]], br[UU[w]], ID2, w > 0 ? 1u : 0u);
#pragma unroll
            for (int w = 0; w < 6; ++w) mma<F>(dr, ai[TT[w]], bi[UU[w]], IDN, 1u);
#pragma unroll
            for (int w = 0; w < 6; ++w) mma<F>(di, ai[TT[w]], br[UU[w]], ID, 1u);
        }
        commit(cx.bar + kBarDone + s);
    };

    if (warp != 0) load(0);
    for (int c = 0; c < NCH; ++c) {
        const int s = c % kStages;
        if (warp != 0) {
            // stage s was last read by the MMAs of chunk c - 3 (earlier products are drained)
            if (c >= kStages) wait_idx(cx, kBarDone + s, base[kBarDone + s] + (c - kStages) / kStages);
            stage(c);
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) arrive(cx.bar + kBarFull + s);
            if (c + 1 < NCH) load(c + 1);
        } else if (lane == 0) {
            wait_idx(cx, kBarFull + s, base[kBarFull + s] + c / kStages);
            // accumulator set c % 2 was read back by every warp (chunk c - 2)
            if (c >= 2) wait_idx(cx, kBarFree + (c & 1), base[kBarFree + (c & 1)] + (c - 2) / 2);
            fence_after();
            issue(c);
        }
        __syncwarp();
        if (c >= 1) gather(c - 1);  // overlaps the MMAs of chunk c and the staging of chunk c + 1
    }
    gather(NCH - 1);
    // every thread consumed the same completions: 3, 3, 2 uses of the stages, 4 of each set
#pragma unroll
    for (int b = 0; b < kStages; ++b) {
        const uint32_t uses = (NCH - b + kStages - 1) / kStages;
        cx.cnt[kBarDone + b] += uses;
        cx.cnt[kBarFull + b] += uses;
    }
    cx.cnt[kBarFree] += NCH / 2;
    cx.cnt[kBarFree + 1] += NCH / 2;
    if (!__syncthreads_or(*(volatile int *)cx.abort)) {
        // C goes out through the idle operand stages (every MMA of the product has completed):
        // each thread writes its 64 columns of its row there (rows padded to kCRow bytes, so a
        // quarter warp's 16-byte stores hit distinct banks), then each warp copies whole rows to
        // global memory with coalesced 512-byte stores (storing each thread's row directly means
        // 16-byte stores 1 KB apart across a warp, several times slower)
        constexpr int kCRow = 128 * 8 + 16;
        static_assert(128 * kCRow <= (int)kSmemBytes, "C fits in the operand stages");
        float4 *crow = reinterpret_cast<float4 *>(stages + row * kCRow + col0 * 8);
#pragma unroll
        for (int j = 0; j < 32; ++j) crow[j] = make_float4(sre[2 * j], sim[2 * j], sre[2 * j + 1], sim[2 * j + 1]);
        __syncthreads();
        for (int r = warp; r < 128; r += 8) {
            const float4 *src = reinterpret_cast<const float4 *>(stages + r * kCRow);
            float4 *dst = reinterpret_cast<float4 *>(Cout + (size_t)r * LD);
            dst[lane] = src[lane];
            dst[lane + 32] = src[lane + 32];
        }
    }
    __syncthreads();
}

}  // namespace umma
}  // namespace pm
