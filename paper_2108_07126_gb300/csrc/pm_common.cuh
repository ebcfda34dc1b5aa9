// Shared device-side definitions of the propagator kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pm {

// ---------------------------------------------------------------- complex helpers
template <typename Real> struct Cx;
template <> struct Cx<float> {
    using T = float2;
    __host__ __device__ static inline float2 make(float a, float b) { return make_float2(a, b); }
};
template <> struct Cx<double> {
    using T = double2;
    __host__ __device__ static inline double2 make(double a, double b) { return make_double2(a, b); }
};

// acc += a * b (complex), four fused multiply-adds
template <typename C>
__device__ __forceinline__ void cfma(C &acc, const C a, const C b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

// ---------------------------------------------------------------- Taylor classes
// A class is one (degree m, Paterson-Stockmeyer split m = q * r, squarings s)
// choice with its capacity: slices whose norm bound nu satisfies
// nu <= cap use it.  Classes are sorted by capacity and cost.
constexpr int kMaxClasses = 96;
constexpr int kMaxDegree = 12;  // q <= 3 powers: m in {1, 2, 4, 6, 9, 12}
constexpr int kMaxControls = 16;
constexpr int kMaxBasis = 1 + 2 * kMaxControls + kMaxControls * (kMaxControls - 1) / 2;

__host__ __device__ inline int cls_m(int code) { return code & 0xff; }
__host__ __device__ inline int cls_q(int code) { return (code >> 8) & 0xff; }
__host__ __device__ inline int cls_r(int code) { return (code >> 16) & 0xff; }
__host__ __device__ inline int cls_s(int code) { return (code >> 24) & 0xff; }
__host__ __device__ inline int cls_pack(int m, int q, int r, int s) { return m | (q << 8) | (r << 16) | (s << 24); }

// device status bits (mirrors PARAMENT_DEV_* in parament.h)
constexpr unsigned kDevNonfinite = 0x1u;
constexpr unsigned kDevCapped = 0x2u;
constexpr unsigned kDevTimeout = 0x4u;  // a bounded tensor-core wait gave up: the result is invalid

enum Integrator { kMidpoint = 0, kGL2 = 1, kSimpson = 2 };

// counters[0..3] live: exp products, tree products, max degree, max squarings
// counters[4..7] copy of the live values at the end of the latest launch
// status[0] live, status[1] copy
struct FusedParams {
    const void *ctrl;          // Real [K][S]
    int64_t S;                 // samples per control (row stride of ctrl)
    int64_t n_steps;
    int K;
    int n_basis;               // basis matrices kept in the kernel (identically zero ones dropped)
    int n_coef;                // effective coefficients per slice: 1 + K or 1 + K (K + 3) / 2
    int d_out;                 // true dimension (<= padded D)
    int out_c128;              // U_out is complex128 (else complex64)
    double dt;
    const void *packed;        // Real [n_basis][D][D] packed Hermitian basis
    const double *bnorm1;      // [n_basis] FP64 1-norms of the basis matrices
    double2 *partials;         // [gridDim.x][D][D] block partial products (FP64)
    unsigned *tickets;         // >= gridDim.x zero-initialised arrival counters
    void *U_out;               // d_out x d_out
    double2 *leaf_out;         // optional [n_leaves][D][D]: every leaf product (FP64)
    double2 *block_out;        // optional [gridDim.x][D][D]: every block product (FP64)
    unsigned long long *counters;
    unsigned *status;
    int extra_squarings;
    int unitary_step;          // FP32: one Newton-Schulz step R <- R (3 I - R^dagger R) / 2 on every leaf product
    int warps;                 // warps of a block that own leaves (0 = all; the others only join the barriers)
    int tc_off;                // batched tensor-core kernel: run this instance's products on the CUDA cores
    const int *cheb_m;         // Chebyshev mode: degree, 1 / beta and coefficients (device, written by
    const double *cheb_inv_beta;  //   cheb_coef_kernel)
    const void *cheb_coef;     // Real complex [m + 1]: a_k = (-i)^k J_k(beta)
    const double2 *traj_pin;   // trajectory mode: exclusive prefix of every leaf, FP64 [n_leaves][D][D]
    void *traj_out;            // trajectory mode: U(t_n) [n_out][d][d] or psi(t_n) [n_out][d] (U_out's dtype)
    const double2 *traj_psi0;  // trajectory mode: psi_0 padded to D in FP64, or null for U(t_n)
    int64_t traj_every;        // trajectory mode: outputs after slices every, 2 every, ..., and the last
    int n_cls;
    double cls_cap[kMaxClasses];
    int cls_code[kMaxClasses];
    short slot_of[kMaxBasis];  // coefficient index -> kept basis slot, -1 if the matrix is zero
    double coef_d[kMaxDegree + 1];  // 1/k!
    float coef_f[kMaxDegree + 1];
};

}  // namespace pm
