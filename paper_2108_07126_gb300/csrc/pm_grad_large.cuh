// Adjoint gradient for padded dimensions D in {32, 64, 128, 256}: the method of pm_grad.cuh with
// one thread block per leaf and block-wide complex products (cta_mm) on a per-block scratch region
// in global memory.
//
// Forward: large_kernel keeps every leaf product (one leaf per block, FP64).  Scans (FP64,
// Hillis-Steele, one tiled launch per level): the exclusive prefix of every leaf, with one more
// element whose prefix is U(T); the exclusive suffix of every leaf, S_b = leaf_{L-1} ... leaf_{b+1}.
// z = Tr(V^dagger U(T)) and the loss.  Adjoint (adjoint_large_kernel): per leaf a forward sweep
// that stores the prefixes P_{j-1} of a sub-chunk (checkpoints every c_sub slices when the leaf is
// longer), and a backward sweep W_{j-1} = W_j U_j from W = V^dagger S (leaf end), with
// Lambda_j = P_{j-1} W_j, M_j = L_{X_j}(Lambda_j) the upper-right block of
// exp([[X_j, Lambda_j], [0, X_j]]) (Van Loan; same Taylor / Paterson-Stockmeyer / squaring scheme
// as the forward exponential on block-upper-triangular matrices), the traces Tr(M_j B_e) and the
// derivatives of the effective coefficients (Sec. 4, Eq. magnus_coeffs).
#pragma once

#include "pm_grad.cuh"
#include "pm_large.cuh"

namespace pm {

// ---------------------------------------------------------------- FP64 scans over leaf products

// x_b = leaf_{b+1} for b < n - 1, x_{n-1} = I
template <int D>
__global__ void __launch_bounds__(256) suffix_init_kernel(const double2 *__restrict__ leaf, int n,
                                                          double2 *__restrict__ x) {
    const size_t DD = (size_t)D * D;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * DD;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t b = e / DD, t = e % DD;
        x[e] = (b + 1 == (size_t)n) ? make_double2((t / D) == (t % D) ? 1.0 : 0.0, 0.0) : leaf[(b + 1) * DD + t];
    }
}

// one level of the right-to-left inclusive scan: out_i = in_{i+off} in_i for i + off < n (the later
// factor on the left), else in_i; block (tile, i) computes one 32 x 32 tile of out_i
template <int D>
__global__ void __launch_bounds__(256) suffix_level_kernel(const double2 *__restrict__ in, int n, int off,
                                                           double2 *__restrict__ out) {
    constexpr int T = 32, KP = 16;
    __shared__ double2 As[T][KP + 1], Bs[KP][T + 1];
    const int tiles = D / T;
    const int ti = blockIdx.x / tiles, tj = blockIdx.x % tiles, i = blockIdx.y;
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    const size_t DD = (size_t)D * D;
    const double2 *Rt = in + (size_t)i * DD;  // earlier factor (right)
    double2 *O = out + (size_t)i * DD;
    if (i + off >= n) {
        for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
            const size_t at = (size_t)(ti * T + e / T) * D + tj * T + e % T;
            O[at] = Rt[at];
        }
        return;
    }
    const double2 *Lt = in + (size_t)(i + off) * DD;  // later factor (left)
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

// exclusive suffixes of n leaf products into x (one of the two buffers a, b; returned)
template <int D>
cudaError_t leaf_suffixes(const double2 *leaf, int n, double2 *a, double2 *b, double2 **x, cudaStream_t st) {
    suffix_init_kernel<D><<<1024, 256, 0, st>>>(leaf, n, a);
    cudaError_t e = cudaGetLastError();
    double2 *cur = a, *nxt = b;
    for (int off = 1; off < n && e == cudaSuccess; off <<= 1) {
        suffix_level_kernel<D><<<dim3((D / 32) * (D / 32), n), 256, 0, st>>>(cur, n, off, nxt);
        e = cudaGetLastError();
        double2 *t = cur;
        cur = nxt;
        nxt = t;
    }
    *x = cur;
    return e;
}

// z = Tr(V^dagger U), loss = 1 - |z|^2 / d^2 (z[0], z[1], z[2]), and U (d x d) into U_out if given
template <int D>
__global__ void __launch_bounds__(256) z_loss_kernel(const double2 *__restrict__ U, const double2 *__restrict__ vdag,
                                                     double *z, void *U_out, int out_c128, int d_out) {
    __shared__ double red[2][8];
    double zr = 0.0, zi = 0.0;
    for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
        const int i = e / D, k = e % D;
        const double2 a = vdag[i * D + k], b = U[k * D + i];
        zr = fma(a.x, b.x, fma(-a.y, b.y, zr));
        zi = fma(a.x, b.y, fma(a.y, b.x, zi));
    }
    for (int off = 16; off > 0; off >>= 1) {
        zr += __shfl_xor_sync(0xffffffffu, zr, off);
        zi += __shfl_xor_sync(0xffffffffu, zi, off);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = zr;
        red[1][threadIdx.x >> 5] = zi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sr = 0.0, si = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            sr += red[0][w];
            si += red[1][w];
        }
        z[0] = sr;
        z[1] = si;
        const double dd = (double)d_out;
        z[2] = 1.0 - (sr * sr + si * si) / (dd * dd);
    }
    if (U_out) {
        for (int e = threadIdx.x; e < d_out * d_out; e += blockDim.x) {
            const double2 v = U[(e / d_out) * D + (e % d_out)];
            if (out_c128) ((double2 *)U_out)[e] = v;
            else ((float2 *)U_out)[e] = make_float2((float)v.x, (float)v.y);
        }
    }
}

// ---------------------------------------------------------------- the block-level adjoint kernel

constexpr int kGradSlots = 14;  // D x D complex matrices per block in the scratch region

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename Real, int D> struct AdjLayout {
    using C = typename Cx<Real>::T;
    static constexpr size_t GAM = LGeo<Real, D>::PANEL_BYTES;                 // after the cta_mm panels
    static constexpr size_t TRC = GAM + align16(kMaxBasis * sizeof(Real));    // Tr(M B_e)
    static constexpr size_t RED = TRC + align16(kMaxBasis * sizeof(C));       // per-warp partial traces
    static constexpr size_t BYTES = RED + align16((size_t)kMaxBasis * 8 * sizeof(C));
};

template <typename Real, int D>
__host__ __device__ constexpr size_t adjoint_large_smem_bytes() { return AdjLayout<Real, D>::BYTES; }

// One block per leaf (grid = p.n_leaves); scratch: kGradSlots D x D complex matrices per block.
template <typename Real, int D, int INTEG>
__global__ void __launch_bounds__(256, 1) adjoint_large_kernel(const GradParams p, void *scratch) {
    using C = typename Cx<Real>::T;
    using AL = AdjLayout<Real, D>;
    constexpr int DD = D * D, NT = 256;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *panels = smem;
    Real *gam = (Real *)(smem + AL::GAM);
    C *Ttr = (C *)(smem + AL::TRC);
    C *red = (C *)(smem + AL::RED);
    __shared__ int s_code;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = p.n_basis, K = p.K;
    const Real *ctrl = (const Real *)p.ctrl;
    const Real *packed = (const Real *)p.packed;
    const Real h = (Real)p.dt;

    C *ws = (C *)scratch + (size_t)blockIdx.x * kGradSlots * DD;
    C *X = ws, *X2 = ws + DD, *X3 = ws + 2 * DD, *D1 = ws + 3 * DD, *D2 = ws + 4 * DD, *D3 = ws + 5 * DD;
    // temporaries and running matrices rotate through these slots by pointer swaps
    C *TL = ws + 6 * DD, *TR = ws + 7 * DD, *T3 = ws + 8 * DD, *W = ws + 9 * DD, *P = ws + 10 * DD;
    C *U = ws + 11 * DD, *M = ws + 12 * DD;
    Real *gpk = (Real *)(ws + 13 * DD);
    C *pbuf = (C *)p.pbuf + (size_t)blockIdx.x * p.c_sub * DD;
    C *ckpt = (C *)p.ckpt + (size_t)blockIdx.x * p.n_ckpt * DD;

    const int64_t N = p.n_steps, L = p.n_leaves, leaf = blockIdx.x;
    const int64_t j0 = N * leaf / L;
    const int len = (int)(N * (leaf + 1) / L - j0);
    if (len <= 0) return;  // uniform over the block
    const Real zr = (Real)p.z[0], zi = (Real)p.z[1];
    const Real gscale = (Real)(-2.0 / (p.d_true * p.d_true));
    unsigned flags = 0;

    auto mm = [&](const C *A, const C *B, C *Cm) { cta_mm<Real, D>(A, B, Cm, panels); };  // ends with a barrier
    auto ld_glob = [&](C *S, const double2 *src) {
        for (int e = tid; e < DD; e += NT) S[e] = Cx<Real>::make((Real)src[e].x, (Real)src[e].y);
        __syncthreads();
    };
    auto copy = [&](C *dst, const C *src) {
        for (int e = tid; e < DD; e += NT) dst[e] = src[e];
        __syncthreads();
    };
    auto sum_into = [&](C *dst, const C *a, const C *b) {  // dst = a + b
        for (int e = tid; e < DD; e += NT) dst[e] = Cx<Real>::make(a[e].x + b[e].x, a[e].y + b[e].y);
        __syncthreads();
    };

    // Exponent of slice j into X as A = -i G_j / 2^s; returns the Taylor class (derivative
    // classes when deriv: the Frechet series loses one power of the truncation bound)
    auto prep = [&](int64_t j, bool deriv) -> int {
        if (tid == 0) {
            for (int e = 0; e < nb; ++e) gam[e] = Real(0);
            slice_coefficients<Real, INTEG, 1>(p, j, true, gam);
            double nu = 0.0;
            for (int e = 0; e < nb; ++e) nu = fma(fabs((double)gam[e]), p.bnorm1[e], nu);
            const int n = deriv ? p.n_dcls : p.n_cls;
            const double *cap = deriv ? p.dcls_cap : p.cls_cap;
            int c;
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
            s_code = deriv ? p.dcls_code[c] : p.cls_code[c];
        }
        __syncthreads();
        const int code = s_code;
        for (int e = tid; e < DD; e += NT) {
            Real v = Real(0);
            for (int b = 0; b < nb; ++b) v = fma(gam[b], __ldg(packed + (size_t)b * DD + e), v);
            gpk[e] = v;
        }
        __syncthreads();
        const Real sc = pow2neg<Real>(cls_s(code));
        for (int e = tid; e < DD; e += NT) {
            const int i = e / D, jj = e % D;
            const Real a = gpk[i * D + jj], b = gpk[jj * D + i];
            const Real re = (i <= jj) ? a : b;
            const Real im = (i > jj) ? a : ((i < jj) ? -b : Real(0));
            X[e] = Cx<Real>::make(im * sc, -re * sc);
        }
        __syncthreads();
        return code;
    };

    // exp of [[A, Lambda], [0, A]] (A in X, Lambda in D1, both scaled by 2^-s): upper-left block
    // -> U, upper-right -> M (only when deriv); block-upper-triangular products
    // [[A, B], [0, A]] [[C, E], [0, C]] = [[AC, AE + BC], [0, AC]]
    auto block_exp = [&](int code, bool deriv) {
        const int q = cls_q(code), rh = cls_r(code), s = cls_s(code);
        if (q >= 2) {
            mm(X, X, X2);
            if (deriv) {  // D2 = A D1 + D1 A
                mm(X, D1, TL);
                mm(D1, X, TR);
                sum_into(D2, TL, TR);
            }
        }
        if (q >= 3) {
            mm(X2, X, X3);
            if (deriv) {  // D3 = A D2 + D1 A^2
                mm(X, D2, TL);
                mm(D1, X2, TR);
                sum_into(D3, TL, TR);
            }
        }
        const C *Xq = (q == 1) ? X : ((q == 2) ? X2 : X3);
        const C *Dq = (q == 1) ? D1 : ((q == 2) ? D2 : D3);
        // U += B_b = sum_{l<q} a_{qb+l} A^l, M += its derivative sum_{1<=l<q} a_{qb+l} D_l
        auto add_block = [&](int b, bool first) {
            const Real a0 = gcoef<Real>(p, q * b);
            const Real a1 = (q >= 2) ? gcoef<Real>(p, q * b + 1) : Real(0);
            const Real a2 = (q >= 3) ? gcoef<Real>(p, q * b + 2) : Real(0);
            for (int e = tid; e < DD; e += NT) {
                C u, m;
                if (first) {  // the first block: T = a_{q rh} X^q + B_{rh-1}
                    const Real top = gcoef<Real>(p, q * rh);
                    u = Cx<Real>::make(top * Xq[e].x, top * Xq[e].y);
                    m = deriv ? Cx<Real>::make(top * Dq[e].x, top * Dq[e].y) : Cx<Real>::make(Real(0), Real(0));
                } else {
                    u = U[e];
                    m = deriv ? M[e] : Cx<Real>::make(Real(0), Real(0));
                }
                if ((e / D) == (e % D)) u.x += a0;
                if (q >= 2) {
                    u.x = fma(a1, X[e].x, u.x);
                    u.y = fma(a1, X[e].y, u.y);
                    if (deriv) {
                        m.x = fma(a1, D1[e].x, m.x);
                        m.y = fma(a1, D1[e].y, m.y);
                    }
                }
                if (q >= 3) {
                    u.x = fma(a2, X2[e].x, u.x);
                    u.y = fma(a2, X2[e].y, u.y);
                    if (deriv) {
                        m.x = fma(a2, D2[e].x, m.x);
                        m.y = fma(a2, D2[e].y, m.y);
                    }
                }
                U[e] = u;
                if (deriv) M[e] = m;
            }
            __syncthreads();
        };
        add_block(rh - 1, true);
        for (int b = rh - 2; b >= 0; --b) {
            mm(Xq, U, TL);  // X^q T
            if (deriv) {    // X^q M + D^q T
                mm(Xq, M, TR);
                mm(Dq, U, T3);
                sum_into(M, TR, T3);
            }
            C *t = U;
            U = TL;
            TL = t;
            add_block(b, false);
        }
        for (int i = 0; i < s; ++i) {
            mm(U, U, TL);
            if (deriv) {  // U M + M U
                mm(U, M, TR);
                mm(M, U, T3);
                sum_into(M, TR, T3);
            }
            C *t = U;
            U = TL;
            TL = t;
        }
    };
    auto advance_prefix = [&]() {  // P <- U P
        mm(U, P, TL);
        C *t = P;
        P = TL;
        TL = t;
    };

    const int c_sub = p.c_sub;
    const int nsub = (len + c_sub - 1) / c_sub;
    // checkpoint pass: prefixes at the start of every sub-chunk
    if (nsub > 1) {
        ld_glob(P, p.pin + (size_t)leaf * DD);
        for (int t = 0; t < len; ++t) {
            if (t % c_sub == 0) copy(ckpt + (size_t)(t / c_sub) * DD, P);
            block_exp(prep(j0 + t, false), false);
            advance_prefix();
        }
    }
    // W = V^dagger S (suffix after the leaf)
    ld_glob(TL, p.vdag);
    ld_glob(TR, p.sout + (size_t)leaf * DD);
    mm(TL, TR, W);

    for (int sub = nsub - 1; sub >= 0; --sub) {
        const int a = sub * c_sub;
        const int nt = min(c_sub, len - a);
        if (nsub > 1) copy(P, ckpt + (size_t)sub * DD);
        else ld_glob(P, p.pin + (size_t)leaf * DD);
        // forward sweep over the sub-chunk: store P_{j-1}, advance
        for (int t = 0; t < nt; ++t) {
            copy(pbuf + (size_t)t * DD, P);
            block_exp(prep(j0 + a + t, false), false);
            advance_prefix();
        }
        // backward sweep
        for (int t = nt - 1; t >= 0; --t) {
            const int64_t j = j0 + a + t;
            copy(P, pbuf + (size_t)t * DD);
            const int code = prep(j, true);
            // Lambda = P_{j-1} W, scaled like A
            mm(P, W, D1);
            {
                const Real sc = pow2neg<Real>(cls_s(code));
                for (int e = tid; e < DD; e += NT) D1[e] = Cx<Real>::make(D1[e].x * sc, D1[e].y * sc);
                __syncthreads();
            }
            block_exp(code, true);
            // T_e = Tr(M B_e) for every kept basis matrix from its packed real form (upper
            // triangle: Re, strict lower: Im); element (i, jj) of M meets B_e[jj][i]
            for (int e = 0; e < nb; ++e) {
                const Real *Pe = packed + (size_t)e * DD;
                Real tr = 0, ti = 0;
                for (int el = tid; el < DD; el += NT) {
                    const int i = el / D, jj = el % D;
                    const Real av = __ldg(Pe + jj * D + i), bv = __ldg(Pe + i * D + jj);
                    const Real br = (jj <= i) ? av : bv;
                    const Real bi = (jj > i) ? av : ((jj < i) ? -bv : Real(0));
                    const C m = M[el];
                    tr = fma(m.x, br, fma(-m.y, bi, tr));
                    ti = fma(m.x, bi, fma(m.y, br, ti));
                }
                for (int off = 16; off > 0; off >>= 1) {
                    tr += __shfl_xor_sync(0xffffffffu, tr, off);
                    ti += __shfl_xor_sync(0xffffffffu, ti, off);
                }
                if (lane == 0) red[e * 8 + warp] = Cx<Real>::make(tr, ti);
            }
            __syncthreads();
            for (int e = tid; e < nb; e += NT) {
                Real sr = 0, si = 0;
                for (int w = 0; w < NT / 32; ++w) {
                    sr += red[e * 8 + w].x;
                    si += red[e * 8 + w].y;
                }
                Ttr[e] = Cx<Real>::make(sr, si);
            }
            __syncthreads();
            // dL/dc = -(2/d^2) (Re z Im Q - Im z Re Q),  Q = sum_e (d gamma_e / dc) T_e
            {
                auto T = [&](int raw) -> C {
                    const int sl = p.slot_of[raw];
                    return sl >= 0 ? Ttr[sl] : Cx<Real>::make(Real(0), Real(0));
                };
                auto emit = [&](int k, int64_t sidx, C qv) {
                    Real *gr = (Real *)p.grad + (size_t)k * p.S + sidx;
                    const Real v = gscale * (zr * qv.y - zi * qv.x);
                    if (INTEG == kSimpson) atomicAdd(gr, v);  // end points are shared by two slices
                    else *gr = v;
                };
                auto axpy = [](C &qv, Real av, C tv) {
                    qv.x = fma(av, tv.x, qv.x);
                    qv.y = fma(av, tv.y, qv.y);
                };
                const int R = (INTEG == kMidpoint) ? 1 : ((INTEG == kGL2) ? 2 : 3);
                for (int w = tid; w < K * R; w += NT) {
                    const int k = w / R, role = w % R;
                    C qv = Cx<Real>::make(Real(0), Real(0));
                    if (INTEG == kMidpoint) {
                        axpy(qv, h, T(1 + k));
                        emit(k, j, qv);
                    } else {
                        // samples of the slice: GL4 nodes (2j, 2j + 1); Simpson (2j, 2j + 1, 2j + 2)
                        const Real wc = (INTEG == kGL2) ? (Real)(1.7320508075688772 / 12.0) * h * h : h * h / Real(12);
                        const Real w1 = (INTEG == kGL2) ? h * Real(0.5) : h / Real(6);
                        const int64_t s1 = 2 * j, s2 = (INTEG == kGL2) ? 2 * j + 1 : 2 * j + 2;
                        if (INTEG == kSimpson && role == 1) {  // centre sample: Omega_1 only
                            axpy(qv, Real(4) * h / Real(6), T(1 + k));
                            emit(k, 2 * j + 1, qv);
                            continue;
                        }
                        const bool first = (role == 0);  // c1 (first node / start) or c2 (second node / end)
                        axpy(qv, w1, T(1 + k));
                        axpy(qv, first ? -wc : wc, T(1 + K + k));
                        // pairs (a, b), a < b: gamma = wc (c1_a c2_b - c2_a c1_b)
                        int e = 1 + 2 * K;
                        for (int aa = 0; aa < K; ++aa)
                            for (int bb = aa + 1; bb < K; ++bb, ++e) {
                                if (aa != k && bb != k) continue;
                                Real coef;
                                if (first) coef = (k == aa) ? wc * ctrl[(int64_t)bb * p.S + s2] : -wc * ctrl[(int64_t)aa * p.S + s2];
                                else coef = (k == bb) ? wc * ctrl[(int64_t)aa * p.S + s1] : -wc * ctrl[(int64_t)bb * p.S + s1];
                                axpy(qv, coef, T(e));
                            }
                        emit(k, first ? s1 : s2, qv);
                    }
                }
            }
            __syncthreads();
            // W <- W U_j
            mm(W, U, TL);
            C *tw = W;
            W = TL;
            TL = tw;
        }
    }
    if (flags) atomicOr(p.status, flags);
}

template <typename Real, int INTEG, int D>
cudaError_t adjoint_large_launch(const GradParams &gp, void *scratch, cudaStream_t st) {
    auto k = adjoint_large_kernel<Real, D, INTEG>;
    const size_t smem = adjoint_large_smem_bytes<Real, D>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)gp.n_leaves, 256, smem, st>>>(gp, scratch);
    return cudaGetLastError();
}

// Scans, z and the adjoint for padded dimension D: leaf[L] the forward leaf products (FP64);
// pre (2 (L + 1) D^2) and suf (2 L D^2) ping-pong buffers; gp.pin / gp.sout / gp.z are set here.
template <int D>
cudaError_t grad_large_run(int fp64, int integ, const double2 *leaf, int L, double2 *pre, double2 *suf,
                           GradParams gp, void *scratch, void *U_out, int out_c128, int d_out, cudaStream_t st) {
    const size_t DD = (size_t)D * D;
    double2 *xp = nullptr, *xs = nullptr;
    cudaError_t e = leaf_prefixes<D>(leaf, L + 1, pre, pre + (size_t)(L + 1) * DD, &xp, st);
    if (e == cudaSuccess) e = leaf_suffixes<D>(leaf, L, suf, suf + (size_t)L * DD, &xs, st);
    if (e != cudaSuccess) return e;
    z_loss_kernel<D><<<1, 256, 0, st>>>(xp + (size_t)L * DD, gp.vdag, (double *)gp.z, U_out, out_c128, d_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    gp.pin = xp;
    gp.sout = xs;
    switch (integ * 2 + (fp64 ? 1 : 0)) {
        case 0: return adjoint_large_launch<float, kMidpoint, D>(gp, scratch, st);
        case 1: return adjoint_large_launch<double, kMidpoint, D>(gp, scratch, st);
        case 2: return adjoint_large_launch<float, kGL2, D>(gp, scratch, st);
        case 3: return adjoint_large_launch<double, kGL2, D>(gp, scratch, st);
        case 4: return adjoint_large_launch<float, kSimpson, D>(gp, scratch, st);
        case 5: return adjoint_large_launch<double, kSimpson, D>(gp, scratch, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pm
