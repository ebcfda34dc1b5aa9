// 16 x 16 complex FP32 products with packed two-wide fused multiply-adds (fma.rn.f32x2), the
// product engine of the fused kernel's FP32 d = 16 Taylor path.
//
// Layouts in shared memory: 16 physical rows of 8 chunks of 16 bytes (row stride RS = 9 chunks,
// 2304 bytes per matrix); matrix row or column i sits in physical row prow(i) = i / 2 + 8 (i % 2),
// which keeps every load and store below free of bank conflicts.
//   row layout    R(M): chunk (i, p) = (Re M[i][2p], Re M[i][2p+1], Im M[i][2p], Im M[i][2p+1])
//   column layout C(M): chunk (j, p) = (Re M[2p][j], Re M[2p+1][j], Im M[2p][j], Im M[2p+1][j])
// C = A B reads R(A) and C(B).  One packed FMA multiplies the k-pair (2p, 2p+1) of a row of A with
// the same k-pair of a column of B, so the two halves of an accumulator hold the even-k and the
// odd-k partial sums; they are added once per output.  For an anti-Hermitian B (the scaled exponent
// X = -i G / 2^s with G Hermitian) C(B) is R(B) with its real parts negated, so R(X) serves as both
// operands of X X and X^2 X.
//
// Lane l = 8 a + b of the warp owns rows {2a, 2a+1, 2a+8, 2a+9} and columns {2b, 2b+1} of the
// output.  Per k-pair a lane loads four A chunks (one address per quarter warp) and two B chunks
// (eight consecutive chunks per quarter warp) and issues 32 packed FMAs: half the FMA instructions
// of the scalar product, which leaves issue slots for the rest of the slice.
#pragma once

#include <cstdint>

namespace pm {
namespace pp16 {

constexpr int RS = 9;                   // chunks per physical row (8 + 1 pad)
constexpr int MAT_BYTES = 16 * RS * 16;  // one matrix in either layout

typedef unsigned long long u64;

__device__ __forceinline__ int prow(int i) { return (i >> 1) + 8 * (i & 1); }
// output row r (0..3) of lane group a
__device__ __forceinline__ int orow(int a, int r) { return 2 * a + (r & 1) + 8 * (r >> 1); }

__device__ __forceinline__ u64 pack2(float x, float y) {
    u64 v;
    asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(x), "f"(y));
    return v;
}
__device__ __forceinline__ float hsum(u64 v) {
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
    return x + y;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// a lane's 4 x 2 output tile
struct Tile {
    float re[4][2], im[4][2];
};

// out = A B for the lane's tile.  A: R(A).  B: C(B), or (AH) R(B) of an anti-Hermitian B.
template <bool AH>
__device__ __forceinline__ void mm(const float4 *__restrict__ A, const float4 *__restrict__ B, int a, int b,
                                   Tile &out) {
    const ulonglong2 *pa[4], *pb[2];
#pragma unroll
    for (int r = 0; r < 4; ++r) pa[r] = reinterpret_cast<const ulonglong2 *>(A + prow(orow(a, r)) * RS);
#pragma unroll
    for (int c = 0; c < 2; ++c) pb[c] = reinterpret_cast<const ulonglong2 *>(B + prow(2 * b + c) * RS);
    const u64 m1 = pack2(-1.f, -1.f);
    u64 sr[4][2], si[4][2];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) sr[r][c] = si[r][c] = 0ull;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        u64 ar[4], ai[4], x[2], y[2], n[2];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const ulonglong2 v = pa[r][p];
            ar[r] = v.x;
            ai[r] = v.y;
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const ulonglong2 v = pb[c][p];
            x[c] = v.x;
            y[c] = v.y;
            // general B: (x, y) = (Re, Im) of the column, Re C needs -Im B.  Anti-Hermitian B given
            // by its rows: the column is (-x, y); Re C is accumulated with the sign flipped
            n[c] = AH ? mul2(v.x, m1) : mul2(v.y, m1);
        }
        // the two FMAs into one accumulator are 16 instructions apart (latency of the packed FMA)
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                sr[r][c] = fma2(ar[r], x[c], sr[r][c]);  // AH: -(Re C)
                si[r][c] = fma2(ar[r], y[c], si[r][c]);
            }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                sr[r][c] = fma2(ai[r], AH ? y[c] : n[c], sr[r][c]);
                si[r][c] = fma2(ai[r], AH ? n[c] : x[c], si[r][c]);
            }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float re = hsum(sr[r][c]);
            out.re[r][c] = AH ? -re : re;
            out.im[r][c] = hsum(si[r][c]);
        }
}

// store the tile in the row layout R(M)
__device__ __forceinline__ void st_row(float4 *M, int a, int b, const Tile &t) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
        M[prow(orow(a, r)) * RS + b] = make_float4(t.re[r][0], t.re[r][1], t.im[r][0], t.im[r][1]);
}

// store the tile in the column layout C(M)
__device__ __forceinline__ void st_col(float4 *M, int a, int b, const Tile &t) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        float4 *col = M + prow(2 * b + c) * RS;
        col[a] = make_float4(t.re[0][c], t.re[1][c], t.im[0][c], t.im[1][c]);
        col[a + 4] = make_float4(t.re[2][c], t.re[3][c], t.im[2][c], t.im[3][c]);
    }
}

// load the tile from the column layout C(M)
__device__ __forceinline__ void ld_col(const float4 *M, int a, int b, Tile &t) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const float4 *col = M + prow(2 * b + c) * RS;
        const float4 u = col[a], v = col[a + 4];
        t.re[0][c] = u.x;
        t.re[1][c] = u.y;
        t.im[0][c] = u.z;
        t.im[1][c] = u.w;
        t.re[2][c] = v.x;
        t.re[3][c] = v.y;
        t.im[2][c] = v.z;
        t.im[3][c] = v.w;
    }
}

}  // namespace pp16
}  // namespace pm
