// Adjoint gradient of the gate-fidelity loss L = 1 - |Tr(V^dagger U)|^2 / d^2
// with respect to every control sample (all three integrators).
//
// U = S_j U_j P_{j-1} with the exclusive prefix P_{j-1} = U_{j-1} ... U_1 and
// suffix S_j = U_N ... U_{j+1}; with z = Tr(V^dagger U) and X_j = -i G_j,
//   dz/dc = Tr(Lambda_j L_{X_j}(dX_j/dc)) = Tr(L_{X_j}(Lambda_j) dX_j/dc),
//   Lambda_j = P_{j-1} V^dagger S_j,  dX_j/dc = -i sum_e (d gamma_e / dc) B_e,
//   dL/dc = -(2/d^2) Re(conj(z) dz/dc),
// where L_X(E) is the Frechet derivative of exp at X (L_X is self-adjoint under
// the trace pairing).  M_j = L_{X_j}(Lambda_j) is the upper-right block of
// exp([[X_j, Lambda_j], [0, X_j]]) (Van Loan), evaluated with the same Taylor /
// Paterson-Stockmeyer / squaring scheme as the forward exponential on
// block-upper-triangular matrices ([[A, B], [0, A]] [[C, D], [0, C]] =
// [[AC, AD + BC], [0, AC]]).
//
// Prefixes and suffixes come from the forward tree: the fused forward kernel
// stores every leaf product and every block product; scan_blocks_kernel turns
// the block products into exclusive block prefixes / suffixes (and U(T), z, L);
// scan_leaves_kernel does the same for the leaves inside each block; the
// adjoint kernel then walks each leaf: a forward sweep P_j = U_j P_{j-1} that
// stores the prefixes of a sub-chunk (re-computed from checkpoints when a leaf
// is longer than the sub-chunk buffer), and a backward sweep
// W_{j-1} = W_j U_j from W = V^dagger S (leaf end), Lambda_j = P_{j-1} W_j.
#pragma once

#include "pm_fused.cuh"

namespace pm {

struct GradParams {
    const void *ctrl;        // Real [K][S] control samples
    int64_t S;               // samples per control (N, 2N or 2N + 1)
    int64_t n_steps;
    int K;
    int n_basis;             // kept basis matrices
    int n_coef;              // effective coefficients per slice (kept or not)
    double dt;
    short slot_of[kMaxBasis];
    const void *packed;      // Real [n_basis][D][D] packed basis (kept matrices)
    const double *bnorm1;    // [n_basis]
    const double2 *pin;      // [L][D][D] exclusive prefix of each leaf
    const double2 *sout;     // [L][D][D] exclusive suffix of each leaf
    const double2 *vdag;     // [D][D] V^dagger (padded with zeros)
    const double *z;         // z = Tr(V^dagger U): z[0] + i z[1]
    void *grad;              // Real [K][S], zeroed before the launch (Simpson end points add up)
    void *pbuf;              // Real complex [groups][c_sub][D][D]: prefixes of one sub-chunk
    void *ckpt;              // Real complex [groups][n_ckpt][D][D]: sub-chunk checkpoints
    int c_sub, n_ckpt;
    int64_t n_leaves;
    double d_true;           // the unpadded dimension d
    unsigned *status;
    int n_cls;
    double cls_cap[kMaxClasses];
    int cls_code[kMaxClasses];
    int n_dcls;
    double dcls_cap[kMaxClasses];
    int dcls_code[kMaxClasses];
    double coef_d[kMaxDegree + 1];
    float coef_f[kMaxDegree + 1];
};

struct ScanParams {
    const double2 *leafpart;  // [n_blocks * leaves_per_block][D][D]
    const double2 *blockpart; // [n_blocks][D][D]
    int n_blocks, leaves_per_block;
    double2 *bpin, *bsout;    // [n_blocks][D][D]
    double2 *pin, *sout;      // [L][D][D]
    const double2 *vdag;      // [D][D], or null (no z, no loss)
    double *z;                // [3]: Re z, Im z, loss
    void *U_out;              // optional d x d
    int out_c128, d_out;
};

// ---------------------------------------------------------------- scans (FP64, whole-block products)

// C = A * B for row-major D x D matrices in shared memory, threads [t0, t0 + nt)
template <int D>
__device__ __forceinline__ void half_mm(const double2 *A, const double2 *B, double2 *Cm, int t, int nt) {
    for (int e = t; e < D * D; e += nt) {
        const int i = e / D, j = e % D;
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int k = 0; k < D; ++k) cfma(acc, A[i * D + k], B[k * D + j]);
        Cm[e] = acc;
    }
}

// Exclusive prefix (first half of the block) and suffix (second half) of a
// sequence of n matrices, seeded with pre / suf; both halves run in lockstep.
template <int D>
__device__ void scan_pair(const double2 *seq, int n, const double2 *pre, const double2 *suf, double2 *out_pre,
                          double2 *out_suf, double2 *sm /* 4 D*D */) {
    constexpr int DD = D * D;
    const int half = blockDim.x / 2;
    const bool second = threadIdx.x >= half;
    const int t = second ? threadIdx.x - half : threadIdx.x;
    double2 *acc = sm + (second ? DD : 0);
    double2 *tmp = sm + 2 * DD + (second ? DD : 0);
    for (int e = t; e < DD; e += half) acc[e] = second ? suf[e] : pre[e];
    __syncthreads();
    for (int it = 0; it < n; ++it) {
        const int idx = second ? n - 1 - it : it;
        double2 *dst = (second ? out_suf : out_pre) + (size_t)idx * DD;
        for (int e = t; e < DD; e += half) dst[e] = acc[e];
        const double2 *m = seq + (size_t)idx * DD;
        // prefix: acc <- m acc (later on the left); suffix: acc <- acc m
        for (int e = t; e < DD; e += half) {
            const int i = e / D, j = e % D;
            double2 v = make_double2(0.0, 0.0);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                if (second) cfma(v, acc[i * D + k], __ldg(m + k * D + j));
                else cfma(v, __ldg(m + i * D + k), acc[k * D + j]);
            }
            tmp[e] = v;
        }
        __syncthreads();
        for (int e = t; e < DD; e += half) acc[e] = tmp[e];
        __syncthreads();
    }
}

template <int D>
__global__ void __launch_bounds__(256) scan_blocks_kernel(const ScanParams sp) {
    constexpr int DD = D * D;
    __shared__ double2 sm[6 * DD];
    double2 *ident = sm + 4 * DD;
    for (int e = threadIdx.x; e < DD; e += blockDim.x)
        ident[e] = make_double2((e / D) == (e % D) ? 1.0 : 0.0, 0.0);
    __syncthreads();
    scan_pair<D>(sp.blockpart, sp.n_blocks, ident, ident, sp.bpin, sp.bsout, sm);
    // U(T) = (last block) * prefix of the last block; z = Tr(V^dagger U)
    double2 *U = sm + 5 * DD;
    const double2 *last = sp.blockpart + (size_t)(sp.n_blocks - 1) * DD;
    const double2 *lp = sp.bpin + (size_t)(sp.n_blocks - 1) * DD;
    __syncthreads();
    for (int e = threadIdx.x; e < DD; e += blockDim.x) {
        const int i = e / D, j = e % D;
        double2 v = make_double2(0.0, 0.0);
        for (int k = 0; k < D; ++k) cfma(v, last[i * D + k], lp[k * D + j]);
        U[e] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0 && sp.vdag) {
        double2 z = make_double2(0.0, 0.0);
        for (int i = 0; i < D; ++i)
            for (int k = 0; k < D; ++k) cfma(z, sp.vdag[i * D + k], U[k * D + i]);
        sp.z[0] = z.x;
        sp.z[1] = z.y;
        const double d = (double)sp.d_out;
        sp.z[2] = 1.0 - (z.x * z.x + z.y * z.y) / (d * d);
    }
    if (sp.U_out) {
        const int d = sp.d_out;
        for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
            const double2 v = U[(e / d) * D + (e % d)];
            if (sp.out_c128) ((double2 *)sp.U_out)[e] = v;
            else ((float2 *)sp.U_out)[e] = make_float2((float)v.x, (float)v.y);
        }
    }
}

template <int D>
__global__ void __launch_bounds__(256) scan_leaves_kernel(const ScanParams sp) {
    constexpr int DD = D * D;
    __shared__ double2 sm[4 * DD];
    const int b = blockIdx.x;
    const size_t first = (size_t)b * sp.leaves_per_block;
    scan_pair<D>(sp.leafpart + first * DD, sp.leaves_per_block, sp.bpin + (size_t)b * DD,
                 sp.bsout + (size_t)b * DD, sp.pin + first * DD, sp.sout + first * DD, sm);
}

// ---------------------------------------------------------------- the adjoint kernel

// per group: 10 complex D x LD slots, then the traces Tr(M B_e) of one slice (kMaxBasis complex,
// rounded up to 16 bytes: the slots of the next group take 16-byte vector accesses)
template <typename Real, int D>
__host__ __device__ constexpr size_t adjoint_group_bytes() {
    using G = Geo<Real, D>;
    return (size_t)10 * G::SLOT * sizeof(typename G::C) +
           (((size_t)kMaxBasis * sizeof(typename G::C) + 15) & ~(size_t)15) + Tiling<Real, D>::GPAD;
}

template <typename Real, int D>
__host__ __device__ inline size_t adjoint_smem_bytes(int K, int warps) {
    using G = Geo<Real, D>;
    (void)K;
    return (size_t)warps * G::GPW * adjoint_group_bytes<Real, D>();
}

template <typename Real> __device__ __forceinline__ Real gcoef(const GradParams &p, int k);
template <> __device__ __forceinline__ float gcoef<float>(const GradParams &p, int k) { return p.coef_f[k]; }
template <> __device__ __forceinline__ double gcoef<double>(const GradParams &p, int k) { return p.coef_d[k]; }

template <typename Real, int D, int INTEG>
__global__ void __launch_bounds__(256, 1) adjoint_kernel(const GradParams p) {
    using G = Geo<Real, D>;
    static_assert(adjoint_group_bytes<Real, D>() % 16 == 0 && (G::SLOT * sizeof(typename G::C)) % 16 == 0,
                  "group workspaces and slots must stay 16-byte aligned");
    using C = typename G::C;
    constexpr int LANES = G::LANES, GPW = G::GPW, TR = G::TR, TC = G::TC, LD = G::LD, DD = G::DD;
    constexpr int SLOT = G::SLOT, NCH = G::NCH, PS = G::PS;

    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int g = lane / LANES, gl = lane % LANES;
    const int rb = gl / G::CBW, cb = gl % G::CBW;
    const int K = p.K, nb = p.n_basis;

    C *slots = (C *)(smem + (size_t)(warp * GPW + g) * adjoint_group_bytes<Real, D>());
    C *SX = slots, *SX2 = slots + SLOT, *SX3 = slots + 2 * SLOT;
    C *SD1 = slots + 3 * SLOT, *SD2 = slots + 4 * SLOT, *SD3 = slots + 5 * SLOT;
    C *STL = slots + 6 * SLOT, *STR = slots + 7 * SLOT, *SW = slots + 8 * SLOT, *SP = slots + 9 * SLOT;
    C *Ttr = slots + 10 * SLOT;  // Tr(M B_e) of the kept basis matrices

    const Real *ctrl = (const Real *)p.ctrl;
    const Real *packed = (const Real *)p.packed;
    const Real h = (Real)p.dt;
    const int64_t N = p.n_steps;
    const int64_t TG = (int64_t)gridDim.x * W * GPW;
    const int64_t gid = ((int64_t)blockIdx.x * W + warp) * GPW + g;
    C *pbuf = (C *)p.pbuf + (size_t)gid * p.c_sub * DD;
    C *ckpt = (C *)p.ckpt + (size_t)gid * p.n_ckpt * DD;
    const Real zr = (Real)p.z[0], zi = (Real)p.z[1];
    const Real gscale = (Real)(-2.0 / (p.d_true * p.d_true));
    unsigned flags = 0;

    // lane tile helpers
    auto ld_glob = [&](C *S, const double2 *src, bool valid) {  // FP64 global D x D -> slot
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c) {
                const int i = rb + r * G::RBN, j = G::col(cb, c);
                const double2 v = valid ? src[i * D + j] : make_double2(i == j ? 1.0 : 0.0, 0.0);
                S[i * LD + j] = Cx<Real>::make((Real)v.x, (Real)v.y);
            }
    };
    auto copy_out = [&](C *dst, const C *S) {  // slot -> global (Real complex, row-major D x D)
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c) {
                const int i = rb + r * G::RBN, j = G::col(cb, c);
                dst[i * D + j] = S[i * LD + j];
            }
    };
    auto copy_in = [&](C *S, const C *src) {
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c) {
                const int i = rb + r * G::RBN, j = G::col(cb, c);
                S[i * LD + j] = src[i * D + j];
            }
    };

    // Exponent of slice j into SX as A = -i G_j / 2^s; returns the class (warp-uniform)
    auto prep = [&](int64_t j, bool active, bool deriv) -> int {
        Real gam[kMaxBasis];
        for (int e = 0; e < nb; ++e) gam[e] = Real(0);
        slice_coefficients<Real, INTEG, 1>(p, j, active, gam);
        double nu = 0.0;
        for (int e = 0; e < nb; ++e) nu = fma(fabs((double)gam[e]), p.bnorm1[e], nu);
        int c;
        {
            const int n = deriv ? p.n_dcls : p.n_cls;
            const double *cap = deriv ? p.dcls_cap : p.cls_cap;
            if (!(nu <= cap[n - 1])) {
                flags |= (isnan(nu) || isinf(nu)) ? kDevNonfinite : kDevCapped;
                c = n - 1;
            } else {
                int lo = 0, hi = n - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (nu <= cap[mid]) hi = mid; else lo = mid + 1;
                }
                c = lo;
            }
        }
        c = (int)__reduce_max_sync(0xffffffffu, (unsigned)c);
        const int code = deriv ? p.dcls_code[c] : p.cls_code[c];
        // packed exponent (lane chunks), then the Hermitian unpack into SX
        Real acc[NCH][4];
#pragma unroll
        for (int t = 0; t < NCH; ++t)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[t][u] = Real(0);
        for (int e = 0; e < nb; ++e) {
            const Real ge = gam[e];
#pragma unroll
            for (int t = 0; t < NCH; ++t)
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    acc[t][u] = fma(ge, __ldg(packed + (size_t)e * DD + 4 * (gl + LANES * t) + u), acc[t][u]);
        }
        Real *gpk = (Real *)STR;
#pragma unroll
        for (int t = 0; t < NCH; ++t)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int pos = 4 * (gl + LANES * t) + u;
                gpk[(pos / D) * PS + (pos % D)] = acc[t][u];
            }
        __syncwarp();
        const Real sc = pow2neg<Real>(cls_s(code));
        C x1[TR][TC];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c2 = 0; c2 < TC; ++c2) {
                const int i = rb + r * G::RBN, jj = G::col(cb, c2);
                const Real a = gpk[i * PS + jj], b = gpk[jj * PS + i];
                const Real re = (i <= jj) ? a : b;
                const Real im = (i > jj) ? a : ((i < jj) ? -b : Real(0));
                x1[r][c2] = Cx<Real>::make(im * sc, -re * sc);
            }
        __syncwarp();
        st_tile<Real, D>(SX, rb, cb, x1);
        __syncwarp();
        return code;
    };

    // exp of [[A, Lambda], [0, A]] (A in SX, Lambda in SD1, both already scaled by 2^-s):
    // upper-left block -> U, upper-right -> M (only when deriv)
    auto block_exp = [&](int code, bool deriv, C (&U)[TR][TC], C (&M)[TR][TC]) {
        const int q = cls_q(code), rh = cls_r(code), s = cls_s(code);
        C t1[TR][TC], t2[TR][TC];
        if (q >= 2) {
            mm_tile<Real, D>(SX, SX, rb, cb, t1);
            st_tile<Real, D>(SX2, rb, cb, t1);
            if (deriv) {  // D2 = A D1 + D1 A
                mm_tile<Real, D>(SX, SD1, rb, cb, t2);
                mm_tile_add<Real, D>(SD1, SX, rb, cb, t2);
                st_tile<Real, D>(SD2, rb, cb, t2);
            }
            __syncwarp();
        }
        if (q >= 3) {
            mm_tile<Real, D>(SX2, SX, rb, cb, t1);
            st_tile<Real, D>(SX3, rb, cb, t1);
            if (deriv) {  // D3 = A D2 + D1 A^2
                mm_tile<Real, D>(SX, SD2, rb, cb, t2);
                mm_tile_add<Real, D>(SD1, SX2, rb, cb, t2);
                st_tile<Real, D>(SD3, rb, cb, t2);
            }
            __syncwarp();
        }
        const C *Xq = (q == 1) ? SX : ((q == 2) ? SX2 : SX3);
        const C *Dq = (q == 1) ? SD1 : ((q == 2) ? SD2 : SD3);
        auto add_block = [&](int b) {
            const Real a0 = gcoef<Real>(p, q * b);
            const Real a1 = (q >= 2) ? gcoef<Real>(p, q * b + 1) : Real(0);
            const Real a2 = (q >= 3) ? gcoef<Real>(p, q * b + 2) : Real(0);
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TC; ++c) {
                    const int i = rb + r * G::RBN, j = G::col(cb, c);
                    C u = U[r][c], m = M[r][c];
                    u.x += (i == j) ? a0 : Real(0);
                    if (q >= 2) {
                        const C x = SX[i * LD + j];
                        u.x = fma(a1, x.x, u.x);
                        u.y = fma(a1, x.y, u.y);
                        if (deriv) {
                            const C d1 = SD1[i * LD + j];
                            m.x = fma(a1, d1.x, m.x);
                            m.y = fma(a1, d1.y, m.y);
                        }
                    }
                    if (q >= 3) {
                        const C x = SX2[i * LD + j];
                        u.x = fma(a2, x.x, u.x);
                        u.y = fma(a2, x.y, u.y);
                        if (deriv) {
                            const C d2 = SD2[i * LD + j];
                            m.x = fma(a2, d2.x, m.x);
                            m.y = fma(a2, d2.y, m.y);
                        }
                    }
                    U[r][c] = u;
                    M[r][c] = m;
                }
        };
        {
            const Real atop = gcoef<Real>(p, q * rh);
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int c = 0; c < TC; ++c) {
                    const int i = rb + r * G::RBN, j = G::col(cb, c);
                    const C x = Xq[i * LD + j];
                    U[r][c] = Cx<Real>::make(atop * x.x, atop * x.y);
                    if (deriv) {
                        const C dq = Dq[i * LD + j];
                        M[r][c] = Cx<Real>::make(atop * dq.x, atop * dq.y);
                    } else {
                        M[r][c] = Cx<Real>::make(Real(0), Real(0));
                    }
                }
            add_block(rh - 1);
        }
        for (int b = rh - 2; b >= 0; --b) {
            st_tile<Real, D>(STL, rb, cb, U);
            if (deriv) st_tile<Real, D>(STR, rb, cb, M);
            __syncwarp();
            mm_tile<Real, D>(Xq, STL, rb, cb, U);
            if (deriv) {
                mm_tile<Real, D>(Xq, STR, rb, cb, M);
                mm_tile_add<Real, D>(Dq, STL, rb, cb, M);
            }
            __syncwarp();
            add_block(b);
        }
        for (int i = 0; i < s; ++i) {
            st_tile<Real, D>(STL, rb, cb, U);
            if (deriv) st_tile<Real, D>(STR, rb, cb, M);
            __syncwarp();
            mm_tile<Real, D>(STL, STL, rb, cb, U);
            if (deriv) {
                mm_tile<Real, D>(STL, STR, rb, cb, M);
                mm_tile_add<Real, D>(STR, STL, rb, cb, M);
            }
            __syncwarp();
        }
    };

    // P <- U P  (U in registers, P in SP)
    auto advance_prefix = [&](const C (&U)[TR][TC]) {
        st_tile<Real, D>(STL, rb, cb, U);
        __syncwarp();
        C t[TR][TC];
        mm_tile<Real, D>(STL, SP, rb, cb, t);
        __syncwarp();
        st_tile<Real, D>(SP, rb, cb, t);
        __syncwarp();
    };

    const int64_t L = p.n_leaves;
    const int c_sub = p.c_sub;
    for (int64_t round = 0;; ++round) {
        const int64_t leaf = gid + round * TG;
        const bool has_leaf = leaf < L;
        if (!__any_sync(0xffffffffu, has_leaf)) break;
        const int64_t j0 = has_leaf ? N * leaf / L : 0;
        const int len = has_leaf ? (int)(N * (leaf + 1) / L - j0) : 0;
        const int wlen = (int)__reduce_max_sync(0xffffffffu, (unsigned)len);
        const int nsub = (wlen + c_sub - 1) / c_sub;
        C U[TR][TC], M[TR][TC];

        // checkpoint pass: prefixes at the start of every sub-chunk
        if (nsub > 1) {
            ld_glob(SP, p.pin + (size_t)(has_leaf ? leaf : 0) * DD, has_leaf);
            __syncwarp();
            for (int t = 0; t < wlen; ++t) {
                if (t % c_sub == 0) copy_out(ckpt + (size_t)(t / c_sub) * DD, SP);
                const int code = prep(j0 + t, t < len, false);
                block_exp(code, false, U, M);
                advance_prefix(U);
            }
        }

        // W = V^dagger S (suffix after the leaf)
        ld_glob(STL, p.vdag, true);
        ld_glob(STR, p.sout + (size_t)(has_leaf ? leaf : 0) * DD, has_leaf);
        __syncwarp();
        mm_tile<Real, D>(STL, STR, rb, cb, U);
        st_tile<Real, D>(SW, rb, cb, U);
        __syncwarp();

        for (int sub = nsub - 1; sub >= 0; --sub) {
            const int a = sub * c_sub;
            const int nt = min(c_sub, wlen - a);
            if (nsub > 1) copy_in(SP, ckpt + (size_t)sub * DD);
            else ld_glob(SP, p.pin + (size_t)(has_leaf ? leaf : 0) * DD, has_leaf);
            __syncwarp();
            // forward sweep over the sub-chunk: store P_{j-1}, advance
            for (int t = 0; t < nt; ++t) {
                copy_out(pbuf + (size_t)t * DD, SP);
                const int code = prep(j0 + a + t, a + t < len, false);
                block_exp(code, false, U, M);
                advance_prefix(U);
            }
            // backward sweep
            for (int t = nt - 1; t >= 0; --t) {
                const bool act = a + t < len;
                const int64_t j = j0 + a + t;
                copy_in(SP, pbuf + (size_t)t * DD);
                const int code = prep(j, act, true);
                __syncwarp();
                // Lambda = P_{j-1} W, scaled like A
                {
                    const Real sc = pow2neg<Real>(cls_s(code));
                    C t1[TR][TC];
                    mm_tile<Real, D>(SP, SW, rb, cb, t1);
#pragma unroll
                    for (int r = 0; r < TR; ++r)
#pragma unroll
                        for (int c = 0; c < TC; ++c) t1[r][c] = Cx<Real>::make(t1[r][c].x * sc, t1[r][c].y * sc);
                    st_tile<Real, D>(SD1, rb, cb, t1);
                    __syncwarp();
                }
                block_exp(code, true, U, M);
                // T_e = Tr(M B_e) for every kept basis matrix, from its packed real form
                // (upper triangle: Re, strict lower: Im); element (i, jj) of M meets B_e[jj][i]
                for (int e = 0; e < nb; ++e) {
                    const Real *Pe = packed + (size_t)e * DD;
                    Real tr = 0, ti = 0;
#pragma unroll
                    for (int r = 0; r < TR; ++r)
#pragma unroll
                        for (int c = 0; c < TC; ++c) {
                            const int i = rb + r * G::RBN, jj = G::col(cb, c);
                            const Real a = __ldg(Pe + jj * D + i), b = __ldg(Pe + i * D + jj);
                            const Real br = (jj <= i) ? a : b;
                            const Real bi = (jj > i) ? a : ((jj < i) ? -b : Real(0));
                            tr = fma(M[r][c].x, br, fma(-M[r][c].y, bi, tr));
                            ti = fma(M[r][c].x, bi, fma(M[r][c].y, br, ti));
                        }
#pragma unroll
                    for (int off = LANES / 2; off > 0; off >>= 1) {
                        tr += __shfl_xor_sync(0xffffffffu, tr, off);
                        ti += __shfl_xor_sync(0xffffffffu, ti, off);
                    }
                    if (gl == 0) Ttr[e] = Cx<Real>::make(tr, ti);
                }
                __syncwarp();
                // dL/dc = -(2/d^2) (Re z Im Q - Im z Re Q),  Q = sum_e (d gamma_e / dc) T_e
                if (act) {
                    auto T = [&](int raw) -> C {
                        const int sl = p.slot_of[raw];
                        return sl >= 0 ? Ttr[sl] : Cx<Real>::make(Real(0), Real(0));
                    };
                    auto emit = [&](int k, int64_t sidx, C q) {
                        Real *gr = (Real *)p.grad + (size_t)k * p.S + sidx;
                        const Real v = gscale * (zr * q.y - zi * q.x);
                        if (INTEG == kSimpson) atomicAdd(gr, v);  // end points are shared by two slices
                        else *gr = v;
                    };
                    auto axpy = [](C &q, Real a, C t) {
                        q.x = fma(a, t.x, q.x);
                        q.y = fma(a, t.y, q.y);
                    };
                    const int R = (INTEG == kMidpoint) ? 1 : ((INTEG == kGL2) ? 2 : 3);
                    for (int w = gl; w < K * R; w += LANES) {
                        const int k = w / R, role = w % R;
                        C q = Cx<Real>::make(Real(0), Real(0));
                        if (INTEG == kMidpoint) {
                            axpy(q, h, T(1 + k));
                            emit(k, j, q);
                        } else {
                            // samples of the slice: GL4 nodes (2j, 2j + 1); Simpson (2j, 2j + 1, 2j + 2)
                            const Real wc = (INTEG == kGL2) ? (Real)(1.7320508075688772 / 12.0) * h * h : h * h / Real(12);
                            const Real w1 = (INTEG == kGL2) ? h * Real(0.5) : h / Real(6);
                            const int64_t s1 = 2 * j, s2 = (INTEG == kGL2) ? 2 * j + 1 : 2 * j + 2;
                            if (INTEG == kSimpson && role == 1) {  // centre sample: Omega_1 only
                                axpy(q, Real(4) * h / Real(6), T(1 + k));
                                emit(k, 2 * j + 1, q);
                                continue;
                            }
                            const bool first = (role == 0);  // c1 (first node / start) or c2 (second node / end)
                            axpy(q, w1, T(1 + k));
                            axpy(q, first ? -wc : wc, T(1 + K + k));
                            // pairs (a, b), a < b: gamma = wc (c1_a c2_b - c2_a c1_b)
                            int e = 1 + 2 * K;
                            for (int a = 0; a < K; ++a)
                                for (int b = a + 1; b < K; ++b, ++e) {
                                    if (a != k && b != k) continue;
                                    Real coef;
                                    if (first) coef = (k == a) ? wc * ctrl[(int64_t)b * p.S + s2] : -wc * ctrl[(int64_t)a * p.S + s2];
                                    else coef = (k == b) ? wc * ctrl[(int64_t)a * p.S + s1] : -wc * ctrl[(int64_t)b * p.S + s1];
                                    axpy(q, coef, T(e));
                                }
                            emit(k, first ? s1 : s2, q);
                        }
                    }
                }
                __syncwarp();
                // W <- W U_j
                st_tile<Real, D>(STL, rb, cb, U);
                __syncwarp();
                mm_tile<Real, D>(SW, STL, rb, cb, U);
                __syncwarp();
                st_tile<Real, D>(SW, rb, cb, U);
                __syncwarp();
            }
        }
    }
    if (flags) atomicOr(p.status, flags);
}

}  // namespace pm
