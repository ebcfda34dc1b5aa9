// Host side of the C ABI declared in include/parament.h, plus the set-up
// kernels (basis construction, Hermiticity check, control conversion).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/parament.h"
#include "pm_batched.cuh"
#include "pm_cheb.cuh"
#include "pm_common.cuh"
#include "pm_grad.cuh"
#include "pm_grad_large.cuh"

namespace pm {
#define PM_DECL_D(D)                                                                                     \
    cudaError_t fused_dispatch_d##D(int, int, const FusedParams &, int, int, size_t, cudaStream_t, int); \
    int fused_blocks_per_sm_d##D(int, int, int, size_t, int);                                            \
    size_t fused_smem_d##D(int, int, int);                                                               \
    int fused_groups_per_warp_d##D(int);                                                                 \
    int fused_max_warps_d##D(int);                                                                       \
    cudaError_t grad_run_d##D(int, int, const ScanParams &, const GradParams &, int, int, size_t, cudaStream_t); \
    cudaError_t scan_run_d##D(const ScanParams &, cudaStream_t);                                          \
    int adjoint_blocks_per_sm_d##D(int, int, int, size_t);                                                \
    size_t adjoint_smem_d##D(int, int, int);
PM_DECL_D(2)
PM_DECL_D(4)
PM_DECL_D(8)
PM_DECL_D(16)
#undef PM_DECL_D
#define PM_DECL_L(D)                                                                                     \
    cudaError_t large_dispatch_d##D(int, int, const FusedParams &, void *, int, size_t, cudaStream_t, int); \
    int large_blocks_per_sm_d##D(int, int, size_t, int);                                                 \
    size_t large_smem_d##D(int, int, int);                                                               \
    cudaError_t large_prefix_d##D(const double2 *, int, double2 *, double2 *, double2 **, cudaStream_t);    \
    cudaError_t grad_large_run_d##D(int, int, const double2 *, int, double2 *, double2 *, const GradParams &, \
                                    void *, void *, int, int, cudaStream_t);                             \
    size_t adjoint_large_smem_d##D(int);
PM_DECL_L(32)
PM_DECL_L(64)
PM_DECL_L(128)
PM_DECL_L(256)
#undef PM_DECL_L
cudaError_t batch_basis_launch(int, int, const BatchInst *, const int2 *, int, int, double2 *, void *, double *,
                               cudaStream_t);
#define PM_DECL_B(v)                                                                                     \
    cudaError_t batched_launch_##v(const BatchItem *, int, unsigned *, const FusedParams *, unsigned char *, \
                                   size_t, int, size_t, unsigned *, cudaStream_t);                       \
    int batched_blocks_per_sm_##v(size_t);
PM_DECL_B(fm)
PM_DECL_B(fm_tc)
PM_DECL_B(fm_bf)
PM_DECL_B(dm)
PM_DECL_B(fg)
PM_DECL_B(fg_tc)
PM_DECL_B(fg_bf)
PM_DECL_B(dg)
#undef PM_DECL_B
}  // namespace pm

using namespace pm;

namespace {

constexpr int kMaxDim = 256;
constexpr int kMaxBatchDim = 128;  // the batched kernel's block-level bodies go up to D = 128
constexpr int kMaxSmallDim = 16;  // larger dimensions use one thread block per leaf
constexpr int kLeafMinSteps = 8;    // fewer blocks for short runs: each leaf gets >= 8 slices (FP32)
constexpr int kLeafMinSteps64 = 2;  // the same for FP64, whose slices cost far more than the tree

struct Workspace {
    void *ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct parament_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int state = 0;  // 0 created, 1 Hamiltonians set, 2 controls set
    int sm_count = 0;
    size_t smem_optin = 0;
    int max_grid = 0;

    int dim = 0, dpad = 0, K = 0, nb = 0;
    parament_dtype dtype = PARAMENT_C128;
    parament_integrator integ = PARAMENT_MIDPOINT;

    Workspace hraw, full, packed64, packed32, bnorm, partials, tickets, counters, status, check;
    Workspace ctrl_copy, ctrl_conv, uout, bmax, cpacked64, cpacked32, cbnorm;
    Workspace gv, gvdag, gleaf, gblock, gbpin, gpin, gz, gpbuf, gckpt, ggrad, lscratch, gadj;
    Workspace tstage, tpsi;  // trajectory: staging of a host output, psi_0 padded (FP64)
    std::vector<double2> tpsi_host;
    // batched plan
    Workspace bparams, binsts, btable, bitems, bfull, bpacked, bnorms, bpartials, btickets, bcounters, bstatus,
        bqueue, bscratch;
    std::vector<int64_t> bkey;
    std::vector<int> b_nblk;               // work items per instance in the current plan
    std::vector<int> b_warps;              // leaf-owning warps per block for each instance (D <= 16)
    std::vector<FusedParams> bparams_up;  // last uploaded parameter block
    std::vector<BatchInst> binsts_up;
    int b_n_items = 0, b_n_mats = 0, b_grid = 0, b_variant = -1, b_fp64 = 0, b_c128 = 0, b_magnus = 0, b_ninst = 0;
    size_t b_smem = 0, b_stride = 0;
    cudaGraphExec_t b_exec = nullptr;
    bool last_batched = false;
    int64_t opt_batch_leaf = 0, opt_batch_items = 0, opt_batch_graph = 1;
    int64_t opt_batch_cuda_mask = 0;  // dimension classes (bit 0: D = 32, 1: 64, 2: 128) on the CUDA cores
    int64_t opt_exp_method = 0;
    int64_t opt_unitary_step = 1;
    Workspace cheb;  // Chebyshev pre-pass: max norm bound, degree, 1/beta, coefficients
    int nb_eff = 0;
    std::vector<short> slot_of;

    const void *ctrl = nullptr;
    parament_real_dtype cdtype = PARAMENT_F64;
    int64_t n_steps = 0, S = 0;
    double dt = 0.0;

    int64_t opt_degree = 0, opt_grid = 0, opt_warps = 0, opt_check_herm = 1, opt_extra_sq = 0, opt_herm_tol = 1000;
    int64_t opt_grad_subchunk = 0, opt_workspace_mb = 4096;

    parament_stats last{};
    std::string err;
};

namespace {

int set_err(parament_ctx *ctx, int status, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return status;
}

#define PM_CUDA(call)                                                                                    \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) {                                                                         \
            cudaGetLastError();                                                                          \
            return set_err(ctx, PARAMENT_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
        }                                                                                                \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int ws_reserve(parament_ctx *ctx, Workspace &w, size_t bytes) {
    if (w.bytes >= bytes && w.ptr) return PARAMENT_OK;
    if (w.ptr) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(w.ptr);
        w.ptr = nullptr;
        w.bytes = 0;
    }
    if (bytes == 0) return PARAMENT_OK;
    cudaError_t e = cudaMalloc(&w.ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        w.ptr = nullptr;
        return set_err(ctx, PARAMENT_ERR_ALLOC, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    w.bytes = bytes;
    return PARAMENT_OK;
}

void ws_free(Workspace &w) {
    if (w.ptr) cudaFree(w.ptr);
    w.ptr = nullptr;
    w.bytes = 0;
}

// Device address of page-locked host memory (readable by the kernels in place over the host
// link), or null for any other pointer.
const void *pinned_device_ptr(const void *p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int pad_dim(int d) {
    int D = 2;
    while (D < d) D *= 2;
    return D;
}

int n_basis_for(int K, parament_integrator integ) {
    return integ == PARAMENT_MIDPOINT ? 1 + K : 1 + 2 * K + K * (K - 1) / 2;
}

int64_t samples_for(int64_t n, parament_integrator integ) {
    switch (integ) {
        case PARAMENT_MIDPOINT: return n;
        case PARAMENT_MAGNUS4_GL2: return 2 * n;
        case PARAMENT_MAGNUS4_SIMPSON: return 2 * n + 1;
    }
    return n;
}

// ------------------------------------------------------------------ set-up kernels

// order-preserving bit pattern of a non-negative double, for atomicMax
__device__ inline unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

template <typename InT>
__global__ void check_hermitian_kernel(const InT *raw, int d, int n_mat, unsigned long long *out /*[3]*/) {
    const int m = blockIdx.x;
    double err = 0.0, mx = 0.0;
    int bad = 0;
    for (int t = threadIdx.x; t < d * d; t += blockDim.x) {
        const int i = t / d, j = t % d;
        const InT a = raw[(size_t)m * d * d + i * d + j];
        const InT b = raw[(size_t)m * d * d + j * d + i];
        const double ax = a.x, ay = a.y, bx = b.x, by = b.y;
        if (!isfinite(ax) || !isfinite(ay)) bad = 1;
        err = fmax(err, hypot(ax - bx, ay + by));
        mx = fmax(mx, hypot(ax, ay));
    }
    if (bad) atomicOr(&out[2], 1ull);
    if (isfinite(err)) atomicMax(&out[0], dbits(err));
    if (isfinite(mx)) atomicMax(&out[1], dbits(mx));
}

// Basis B_e (FP64, padded to Dp): H0, H_k and, for the Magnus exponents,
// i[H0, H_k] and i[H_a, H_b] (a < b), the effective control Hamiltonians of
// Sec. 4, Eq. magnus_coeffs.
// grid: (basis matrices, tiles of 256 entries)
template <typename InT>
__global__ void build_basis_kernel(const InT *raw, int d, int Dp, int K, int magnus, double2 *full) {
    const int e = blockIdx.x;
    int a = -1, b = -1, src = -1;
    if (e < 1 + K) {
        src = e;
    } else if (e < 1 + 2 * K) {
        a = 0;
        b = e - K;  // raw index of H_k is k + 1
    } else {
        int pidx = e - (1 + 2 * K);
        for (int x = 0; x < K && a < 0; ++x) {
            const int cnt = K - 1 - x;
            if (pidx < cnt) { a = 1 + x; b = 1 + x + 1 + pidx; }
            else pidx -= cnt;
        }
    }
    (void)magnus;
    for (int t = blockIdx.y * blockDim.x + threadIdx.x; t < Dp * Dp; t += gridDim.y * blockDim.x) {
        const int i = t / Dp, j = t % Dp;
        double2 v = make_double2(0.0, 0.0);
        if (i < d && j < d) {
            if (src >= 0) {
                const InT x = raw[(size_t)src * d * d + i * d + j];
                v = make_double2((double)x.x, (double)x.y);
            } else {
                const InT *A = raw + (size_t)a * d * d;
                const InT *B = raw + (size_t)b * d * d;
                double re = 0.0, im = 0.0;  // [A, B]_ij
                for (int l = 0; l < d; ++l) {
                    const double2 ail = make_double2(A[i * d + l].x, A[i * d + l].y);
                    const double2 blj = make_double2(B[l * d + j].x, B[l * d + j].y);
                    const double2 bil = make_double2(B[i * d + l].x, B[i * d + l].y);
                    const double2 alj = make_double2(A[l * d + j].x, A[l * d + j].y);
                    re += ail.x * blj.x - ail.y * blj.y - (bil.x * alj.x - bil.y * alj.y);
                    im += ail.x * blj.y + ail.y * blj.x - (bil.x * alj.y + bil.y * alj.x);
                }
                v = make_double2(-im, re);  // i * [A, B]
            }
        }
        full[(size_t)e * Dp * Dp + t] = v;
    }
}

// Packed real form of each Hermitian basis matrix (upper triangle: real parts,
// strictly lower triangle: imaginary parts) and its FP64 1-norm.
__global__ void pack_basis_kernel(const double2 *full, int Dp, double *p64, float *p32, double *bnorm,
                                  double *bmax) {
    const int e = blockIdx.x;
    const double2 *B = full + (size_t)e * Dp * Dp;
    for (int t = threadIdx.x; t < Dp * Dp; t += blockDim.x) {
        const int i = t / Dp, j = t % Dp;
        const double2 v = B[t];
        const double x = (i <= j) ? v.x : v.y;
        p64[(size_t)e * Dp * Dp + t] = x;
        p32[(size_t)e * Dp * Dp + t] = (float)x;
    }
    __shared__ double colsum[kMaxDim], colmax[kMaxDim];
    if (threadIdx.x < Dp) {
        double s = 0.0, mx = 0.0;
        for (int i = 0; i < Dp; ++i) {
            const double a = hypot(B[i * Dp + threadIdx.x].x, B[i * Dp + threadIdx.x].y);
            s += a;
            mx = fmax(mx, a);
        }
        colsum[threadIdx.x] = s;
        colmax[threadIdx.x] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0, mx = 0.0;
        for (int j = 0; j < Dp; ++j) {
            m = fmax(m, colsum[j]);
            mx = fmax(mx, colmax[j]);
        }
        bmax[e] = mx;
        // the packed FP32 basis is a rounded copy: widen the bound by its relative rounding
        bnorm[e] = m * (1.0 + 4.0 * 5.960464477539063e-08 * Dp);
    }
}

template <typename From, typename To>
__global__ void convert_kernel(const From *src, To *dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (To)src[i];
}

// ------------------------------------------------------------------ Chebyshev pre-pass

struct ChebTheta {
    double t[kMaxChebDegree + 1];  // t[m] = largest half-width covered by degree m
};

// Largest per-slice bound nu_j = sum_e |gamma_e| ||B_e||_1 over all slices: the common
// spectral half-width beta (the paper uses one alpha, beta for all slices, Sec. 3.2).
template <typename Real, int INTEG>
__global__ void cheb_bound_kernel(const FusedParams p, unsigned long long *numax, unsigned *status) {
    Real gam[kMaxBasis];
    double nu_max = 0.0;
    bool bad = false;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < p.n_steps;
         j += (int64_t)gridDim.x * blockDim.x) {
        slice_coefficients<Real, INTEG, 1>(p, j, true, gam);
        double nu = 0.0;
        for (int e = 0; e < p.n_basis; ++e) nu = fma(fabs((double)gam[e]), p.bnorm1[e], nu);
        if (!(nu <= 1e300)) bad = true;
        else nu_max = fmax(nu_max, nu);
    }
    for (int off = 16; off > 0; off >>= 1) nu_max = fmax(nu_max, __shfl_xor_sync(0xffffffffu, nu_max, off));
    if ((threadIdx.x & 31) == 0) atomicMax(numax, (unsigned long long)__double_as_longlong(nu_max));
    if (bad) atomicOr(status, kDevNonfinite);
}

// Degree (smallest m whose bound covers beta; Sec. 2.1) and coefficients a_k = (-i)^k J_k(beta)
template <typename C>
__global__ void cheb_coef_kernel(const unsigned long long *numax, const ChebTheta th, int *m_out, double *inv_beta,
                                 C *coef, unsigned *status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double beta = __longlong_as_double((long long)*numax);
    int m = kMaxChebDegree;
    bool capped = true;
    for (int k = 1; k <= kMaxChebDegree; ++k)
        if (th.t[k] >= beta) {
            m = k;
            capped = false;
            break;
        }
    if (capped) atomicOr(status, kDevCapped);
    double J[kMaxChebDegree + 1];
    bessel_j_seq(beta, m, J);
    for (int k = 0; k <= m; ++k) {
        const double v = J[k];
        double re = 0.0, im = 0.0;
        switch (k & 3) {
            case 0: re = v; break;
            case 1: im = -v; break;
            case 2: re = -v; break;
            case 3: im = v; break;
        }
        coef[k].x = re;
        coef[k].y = im;
    }
    *m_out = m;
    *inv_beta = beta > 0.0 ? 1.0 / beta : 0.0;
}

const ChebTheta &cheb_theta_table(double u) {
    static std::mutex mu;
    static std::map<double, ChebTheta> memo;
    std::lock_guard<std::mutex> lock(mu);
    auto it = memo.find(u);
    if (it != memo.end()) return it->second;
    ChebTheta t;
    t.t[0] = 0.0;
    for (int m = 1; m <= kMaxChebDegree; ++m) t.t[m] = cheb_theta(m, u);
    return memo.emplace(u, t).first->second;
}

// ------------------------------------------------------------------ Taylor classes

struct Cand {
    double cap;
    int cost, m, q, r, s;
};

const int kDegrees[][3] = {{1, 1, 1}, {2, 2, 1}, {4, 2, 2}, {6, 3, 2}, {9, 3, 3}, {12, 3, 4}};  // m, q, r

struct ClassTable {
    int n_cls;
    double cap[kMaxClasses];
    int code[kMaxClasses];
    double coef_d[kMaxDegree + 1];
    float coef_f[kMaxDegree + 1];
};

int build_classes_uncached(double u, int force_m, FusedParams &p, int shift);

// The table depends only on (u, force_m, shift); it is computed once per process (a few
// hundred root solves) so that a propagation call costs microseconds on the host.
int build_classes(double u, int force_m, FusedParams &p, int shift = 0) {
    static std::mutex mu;
    static std::map<std::tuple<double, int, int>, ClassTable> memo;
    const auto key = std::make_tuple(u, force_m, shift);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = memo.find(key);
        if (it != memo.end()) {
            const ClassTable &t = it->second;
            p.n_cls = t.n_cls;
            std::memcpy(p.cls_cap, t.cap, sizeof(t.cap));
            std::memcpy(p.cls_code, t.code, sizeof(t.code));
            std::memcpy(p.coef_d, t.coef_d, sizeof(t.coef_d));
            std::memcpy(p.coef_f, t.coef_f, sizeof(t.coef_f));
            return p.n_cls;
        }
    }
    const int n = build_classes_uncached(u, force_m, p, shift);
    if (n > 0) {
        ClassTable t;
        t.n_cls = p.n_cls;
        std::memcpy(t.cap, p.cls_cap, sizeof(t.cap));
        std::memcpy(t.code, p.cls_code, sizeof(t.code));
        std::memcpy(t.coef_d, p.coef_d, sizeof(t.coef_d));
        std::memcpy(t.coef_f, p.coef_f, sizeof(t.coef_f));
        std::lock_guard<std::mutex> lock(mu);
        memo[key] = t;
    }
    return n;
}

// Occupancy queries are memoised per (device, kernel family, shape, shared memory).
template <typename F>
int memo_occupancy(int kind, int Dp, int fp64, int integ, int warps, size_t smem, int extra, F &&query) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, int, int, size_t, int>, int> memo;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, kind, Dp, fp64, integ, warps, smem, extra);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = memo.find(key);
        if (it != memo.end()) return it->second;
    }
    const int v = query();
    if (v > 0) {
        std::lock_guard<std::mutex> lock(mu);
        memo[key] = v;
    }
    return v;
}

// shift = 0: truncation bound of exp; shift = 1: of its Frechet derivative
// (the derivative series loses one power: remainder ~ x^m / m! e^x).
int build_classes_uncached(double u, int force_m, FusedParams &p, int shift) {
    std::vector<Cand> all;
    for (int s = 0; s <= 62; ++s) {
        for (const auto &dg : kDegrees) {
            const int m = dg[0], q = dg[1], r = dg[2];
            if (force_m > 0 && m != force_m) continue;
            if (m - shift < 1) continue;
            // s squarings multiply the truncation error of exp(A / 2^s) by 2^s: the
            // polynomial must meet u / 2^s so that the squared result meets u.
            const double th = parament_taylor_theta(m - shift, std::ldexp(u, -s));
            if (!(th > 0.0)) continue;
            all.push_back({std::ldexp(th, s), (q - 1) + (r - 1) + s, m, q, r, s});
        }
    }
    if (all.empty()) return 0;
    std::sort(all.begin(), all.end(), [](const Cand &a, const Cand &b) {
        return a.cap != b.cap ? a.cap > b.cap : a.cost < b.cost;
    });
    std::vector<Cand> keep;
    int best = 1 << 30;
    for (const auto &c : all)
        if (c.cost < best) {
            keep.push_back(c);
            best = c.cost;
        }
    std::reverse(keep.begin(), keep.end());
    if ((int)keep.size() > kMaxClasses) keep.resize(kMaxClasses);
    p.n_cls = (int)keep.size();
    for (int i = 0; i < p.n_cls; ++i) {
        p.cls_cap[i] = keep[i].cap;
        p.cls_code[i] = cls_pack(keep[i].m, keep[i].q, keep[i].r, keep[i].s);
    }
    double f = 1.0;
    for (int k = 0; k <= kMaxDegree; ++k) {
        if (k > 0) f /= k;
        p.coef_d[k] = f;
        p.coef_f[k] = (float)f;
    }
    return p.n_cls;
}

cudaError_t fused_dispatch(int Dp, int fp64, int integ, const FusedParams &p, int grid, int warps, size_t smem,
                           cudaStream_t st, int cheb = 0) {
    switch (Dp) {
        case 2: return fused_dispatch_d2(fp64, integ, p, grid, warps, smem, st, cheb);
        case 4: return fused_dispatch_d4(fp64, integ, p, grid, warps, smem, st, cheb);
        case 8: return fused_dispatch_d8(fp64, integ, p, grid, warps, smem, st, cheb);
        case 16: return fused_dispatch_d16(fp64, integ, p, grid, warps, smem, st, cheb);
    }
    return cudaErrorInvalidValue;
}
int fused_blocks_per_sm_uncached(int Dp, int fp64, int integ, int warps, size_t smem, int cheb) {
    switch (Dp) {
        case 2: return fused_blocks_per_sm_d2(fp64, integ, warps, smem, cheb);
        case 4: return fused_blocks_per_sm_d4(fp64, integ, warps, smem, cheb);
        case 8: return fused_blocks_per_sm_d8(fp64, integ, warps, smem, cheb);
        case 16: return fused_blocks_per_sm_d16(fp64, integ, warps, smem, cheb);
    }
    return 0;
}
int fused_blocks_per_sm(int Dp, int fp64, int integ, int warps, size_t smem, int cheb = 0) {
    return memo_occupancy(0, Dp, fp64, integ, warps, smem, cheb,
                          [&] { return fused_blocks_per_sm_uncached(Dp, fp64, integ, warps, smem, cheb); });
}
size_t fused_smem(int Dp, int fp64, int nb, int warps) {
    switch (Dp) {
        case 2: return fused_smem_d2(fp64, nb, warps);
        case 4: return fused_smem_d4(fp64, nb, warps);
        case 8: return fused_smem_d8(fp64, nb, warps);
        case 16: return fused_smem_d16(fp64, nb, warps);
    }
    return 0;
}
cudaError_t grad_run(int Dp, int fp64, int integ, const ScanParams &sp, const GradParams &gp, int grid, int warps,
                     size_t smem, cudaStream_t st) {
    switch (Dp) {
        case 2: return grad_run_d2(fp64, integ, sp, gp, grid, warps, smem, st);
        case 4: return grad_run_d4(fp64, integ, sp, gp, grid, warps, smem, st);
        case 8: return grad_run_d8(fp64, integ, sp, gp, grid, warps, smem, st);
        case 16: return grad_run_d16(fp64, integ, sp, gp, grid, warps, smem, st);
    }
    return cudaErrorInvalidValue;
}
cudaError_t scan_run(int Dp, const ScanParams &sp, cudaStream_t st) {
    switch (Dp) {
        case 2: return scan_run_d2(sp, st);
        case 4: return scan_run_d4(sp, st);
        case 8: return scan_run_d8(sp, st);
        case 16: return scan_run_d16(sp, st);
    }
    return cudaErrorInvalidValue;
}
int adjoint_blocks_per_sm(int Dp, int fp64, int integ, int warps, size_t smem) {
    switch (Dp) {
        case 2: return adjoint_blocks_per_sm_d2(fp64, integ, warps, smem);
        case 4: return adjoint_blocks_per_sm_d4(fp64, integ, warps, smem);
        case 8: return adjoint_blocks_per_sm_d8(fp64, integ, warps, smem);
        case 16: return adjoint_blocks_per_sm_d16(fp64, integ, warps, smem);
    }
    return 0;
}
size_t adjoint_smem(int Dp, int fp64, int K, int warps) {
    switch (Dp) {
        case 2: return adjoint_smem_d2(fp64, K, warps);
        case 4: return adjoint_smem_d4(fp64, K, warps);
        case 8: return adjoint_smem_d8(fp64, K, warps);
        case 16: return adjoint_smem_d16(fp64, K, warps);
    }
    return 0;
}
cudaError_t large_dispatch(int Dp, int fp64, int integ, const FusedParams &p, void *scratch, int grid, size_t smem,
                           cudaStream_t st, int tc) {
    switch (Dp) {
        case 32: return large_dispatch_d32(fp64, integ, p, scratch, grid, smem, st, tc);
        case 64: return large_dispatch_d64(fp64, integ, p, scratch, grid, smem, st, tc);
        case 128: return large_dispatch_d128(fp64, integ, p, scratch, grid, smem, st, tc);
        case 256: return large_dispatch_d256(fp64, integ, p, scratch, grid, smem, st, tc);
    }
    return cudaErrorInvalidValue;
}
cudaError_t grad_large_run(int Dp, int fp64, int integ, const double2 *leaf, int L, double2 *pre, double2 *suf,
                           const GradParams &gp, void *scratch, void *U_out, int out_c128, int d_out, cudaStream_t st) {
    switch (Dp) {
        case 32: return grad_large_run_d32(fp64, integ, leaf, L, pre, suf, gp, scratch, U_out, out_c128, d_out, st);
        case 64: return grad_large_run_d64(fp64, integ, leaf, L, pre, suf, gp, scratch, U_out, out_c128, d_out, st);
        case 128: return grad_large_run_d128(fp64, integ, leaf, L, pre, suf, gp, scratch, U_out, out_c128, d_out, st);
        case 256: return grad_large_run_d256(fp64, integ, leaf, L, pre, suf, gp, scratch, U_out, out_c128, d_out, st);
    }
    return cudaErrorInvalidValue;
}
size_t adjoint_large_smem(int Dp, int fp64) {
    switch (Dp) {
        case 32: return adjoint_large_smem_d32(fp64);
        case 64: return adjoint_large_smem_d64(fp64);
        case 128: return adjoint_large_smem_d128(fp64);
        case 256: return adjoint_large_smem_d256(fp64);
    }
    return 0;
}
cudaError_t large_prefix(int Dp, const double2 *leaf, int n, double2 *a, double2 *b, double2 **x, cudaStream_t st) {
    switch (Dp) {
        case 32: return large_prefix_d32(leaf, n, a, b, x, st);
        case 64: return large_prefix_d64(leaf, n, a, b, x, st);
        case 128: return large_prefix_d128(leaf, n, a, b, x, st);
        case 256: return large_prefix_d256(leaf, n, a, b, x, st);
    }
    return cudaErrorInvalidValue;
}
int large_blocks_per_sm_uncached(int Dp, int fp64, int integ, size_t smem, int tc) {
    switch (Dp) {
        case 32: return large_blocks_per_sm_d32(fp64, integ, smem, tc);
        case 64: return large_blocks_per_sm_d64(fp64, integ, smem, tc);
        case 128: return large_blocks_per_sm_d128(fp64, integ, smem, tc);
        case 256: return large_blocks_per_sm_d256(fp64, integ, smem, tc);
    }
    return 0;
}
int large_blocks_per_sm(int Dp, int fp64, int integ, size_t smem, int tc) {
    return memo_occupancy(1, Dp, fp64, integ, 8, smem, tc,
                          [&] { return large_blocks_per_sm_uncached(Dp, fp64, integ, smem, tc); });
}
// the code that runs the complex products of parament_propagate for one padded dimension and
// precision (tc: 0 none, 1 3xTF32, 2 split BF16x3), as PARAMENT_BACKEND_* bits
template <int D>
unsigned large_backend_bits(int tc) {
    const int tcm = tc == 1 ? large_tcm<float, D, 1>() : large_tcm<float, D, 2>();
    return tcm == 0 ? PARAMENT_BACKEND_CUDA_CORES : (tcm == 1 ? PARAMENT_BACKEND_MMA_SYNC : PARAMENT_BACKEND_TCGEN05);
}
unsigned product_backend(int Dp, int fp64, int tc) {
    if (Dp <= kMaxSmallDim || fp64 || tc == 0) return PARAMENT_BACKEND_CUDA_CORES;
    switch (Dp) {
        case 32: return large_backend_bits<32>(tc);
        case 64: return large_backend_bits<64>(tc);
        case 128: return large_backend_bits<128>(tc);
        case 256: return large_backend_bits<256>(tc);
    }
    return PARAMENT_BACKEND_CUDA_CORES;
}
size_t large_smem(int Dp, int fp64, int nb, int tc = 0) {
    switch (Dp) {
        case 32: return large_smem_d32(fp64, nb, tc);
        case 64: return large_smem_d64(fp64, nb, tc);
        case 128: return large_smem_d128(fp64, nb, tc);
        case 256: return large_smem_d256(fp64, nb, tc);
    }
    return 0;
}
int fused_max_warps(int Dp, int fp64) {
    switch (Dp) {
        case 2: return fused_max_warps_d2(fp64);
        case 4: return fused_max_warps_d4(fp64);
        case 8: return fused_max_warps_d8(fp64);
        case 16: return fused_max_warps_d16(fp64);
    }
    return 8;
}
int fused_gpw(int Dp, int fp64) {
    switch (Dp) {
        case 2: return fused_groups_per_warp_d2(fp64);
        case 4: return fused_groups_per_warp_d4(fp64);
        case 8: return fused_groups_per_warp_d8(fp64);
        case 16: return fused_groups_per_warp_d16(fp64);
    }
    return 1;
}

}  // namespace

// ------------------------------------------------------------------ C ABI

extern "C" {

int parament_version(void) { return PARAMENT_VERSION_MAJOR * 1000 + PARAMENT_VERSION_MINOR; }

const char *parament_status_string(int status) {
    switch (status) {
        case PARAMENT_OK: return "PARAMENT_OK";
        case PARAMENT_ERR_INVALID_VALUE: return "PARAMENT_ERR_INVALID_VALUE";
        case PARAMENT_ERR_STATE: return "PARAMENT_ERR_STATE";
        case PARAMENT_ERR_ALLOC: return "PARAMENT_ERR_ALLOC";
        case PARAMENT_ERR_CUDA: return "PARAMENT_ERR_CUDA";
        case PARAMENT_ERR_NONFINITE: return "PARAMENT_ERR_NONFINITE";
        case PARAMENT_ERR_NOT_HERMITIAN: return "PARAMENT_ERR_NOT_HERMITIAN";
        case PARAMENT_ERR_TIMEOUT: return "PARAMENT_ERR_TIMEOUT";
        case PARAMENT_ERR_UNSUPPORTED: return "PARAMENT_ERR_UNSUPPORTED";
    }
    return "PARAMENT_UNKNOWN_STATUS";
}

const char *parament_last_error(const parament_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

double parament_taylor_theta(int m, double u) {
    if (m < 1 || !(u > 0.0) || !(u < 1.0)) return -1.0;
    // g(x) = (m+1) ln x - ln (m+1)! + x - ln u is increasing for x > 0
    const double lf = std::lgamma((double)m + 2.0), lu = std::log(u);
    auto g = [&](double x) { return (m + 1) * std::log(x) - lf + x - lu; };
    double lo = 0.0, hi = 1.0;
    for (int i = 0; i < 64 && g(hi) < 0.0; ++i) hi *= 2.0;
    for (int i = 0; i < 200; ++i) {
        const double mid = 0.5 * (lo + hi);
        if (g(mid) <= 0.0) lo = mid; else hi = mid;
    }
    return lo;
}

int parament_taylor_choice(double norm_bound, double u, int force_m, int *m_out, int *s_out) {
    if (!m_out || !s_out || !(u > 0.0) || !(u < 1.0) || !(norm_bound >= 0.0) || std::isinf(norm_bound))
        return PARAMENT_ERR_INVALID_VALUE;
    if (force_m != 0 && force_m != 1 && force_m != 2 && force_m != 4 && force_m != 6 && force_m != 9 && force_m != 12)
        return PARAMENT_ERR_INVALID_VALUE;
    FusedParams p;
    std::memset(&p, 0, sizeof(p));
    if (build_classes(u, force_m, p) <= 0) return PARAMENT_ERR_INVALID_VALUE;
    int c = 0;
    while (c < p.n_cls - 1 && !(norm_bound <= p.cls_cap[c])) ++c;
    if (!(norm_bound <= p.cls_cap[c])) return PARAMENT_ERR_UNSUPPORTED;
    *m_out = cls_m(p.cls_code[c]);
    *s_out = cls_s(p.cls_code[c]);
    return PARAMENT_OK;
}

double parament_chebyshev_theta(int m, double u) {
    if (m < 1 || m > kMaxChebDegree || !(u > 0.0) || !(u < 1.0)) return -1.0;
    return cheb_theta(m, u);
}

int parament_chebyshev_degree(double half_width, double u) {
    if (!(half_width >= 0.0) || std::isinf(half_width) || !(u > 0.0) || !(u < 1.0)) return -1;
    for (int m = 1; m <= kMaxChebDegree; ++m)
        if (cheb_theta(m, u) >= half_width) return m;
    return -1;
}

int parament_bessel_j(int n, double x, double *out) {
    if (!out || n < 0 || n > kMaxChebDegree || !(x >= 0.0) || std::isinf(x)) return PARAMENT_ERR_INVALID_VALUE;
    bessel_j_seq(x, n, out);
    return PARAMENT_OK;
}

int parament_create(parament_ctx **out, int device, void *cuda_stream) {
    if (!out) return PARAMENT_ERR_INVALID_VALUE;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return PARAMENT_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return PARAMENT_ERR_INVALID_VALUE;
    parament_ctx *ctx = new (std::nothrow) parament_ctx();
    if (!ctx) return PARAMENT_ERR_ALLOC;
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    DeviceGuard guard(device);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return PARAMENT_ERR_CUDA;
    }
    ctx->sm_count = prop.multiProcessorCount;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
    ctx->max_grid = prop.multiProcessorCount * 8;
    int st = ws_reserve(ctx, ctx->counters, 8 * sizeof(unsigned long long));
    if (st == PARAMENT_OK) st = ws_reserve(ctx, ctx->status, 2 * sizeof(unsigned));
    if (st == PARAMENT_OK) st = ws_reserve(ctx, ctx->tickets, 2 * (size_t)ctx->max_grid * sizeof(unsigned));
    if (st == PARAMENT_OK) st = ws_reserve(ctx, ctx->check, 4 * sizeof(unsigned long long));
    if (st != PARAMENT_OK) {
        parament_destroy(ctx);
        return st;
    }
    if (cudaMemset(ctx->counters.ptr, 0, ctx->counters.bytes) != cudaSuccess ||
        cudaMemset(ctx->status.ptr, 0, ctx->status.bytes) != cudaSuccess ||
        cudaMemset(ctx->tickets.ptr, 0, ctx->tickets.bytes) != cudaSuccess) {
        cudaGetLastError();
        parament_destroy(ctx);
        return PARAMENT_ERR_CUDA;
    }
    *out = ctx;
    return PARAMENT_OK;
}

int parament_destroy(parament_ctx *ctx) {
    if (!ctx) return PARAMENT_OK;
    {
        DeviceGuard guard(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        cudaGetLastError();
        Workspace *all[] = {&ctx->hraw, &ctx->full, &ctx->packed64, &ctx->packed32, &ctx->bnorm,
                            &ctx->partials, &ctx->tickets, &ctx->counters, &ctx->status, &ctx->check,
                            &ctx->ctrl_copy, &ctx->ctrl_conv, &ctx->uout, &ctx->bmax, &ctx->cpacked64,
                            &ctx->cpacked32, &ctx->cbnorm, &ctx->gv, &ctx->gvdag, &ctx->gleaf, &ctx->gblock,
                            &ctx->gbpin, &ctx->gpin, &ctx->gz, &ctx->gpbuf, &ctx->gckpt, &ctx->ggrad, &ctx->lscratch,
                            &ctx->gadj,
                            &ctx->bparams, &ctx->binsts, &ctx->btable, &ctx->bitems, &ctx->bfull, &ctx->bpacked,
                            &ctx->bnorms, &ctx->bpartials, &ctx->btickets, &ctx->bcounters, &ctx->bstatus,
                            &ctx->bqueue, &ctx->bscratch, &ctx->cheb, &ctx->tstage, &ctx->tpsi};
        if (ctx->b_exec) cudaGraphExecDestroy(ctx->b_exec);
        for (Workspace *w : all) ws_free(*w);
    }
    delete ctx;
    return PARAMENT_OK;
}

int parament_set_stream(parament_ctx *ctx, void *cuda_stream) {
    if (!ctx) return PARAMENT_ERR_INVALID_VALUE;
    ctx->stream = (cudaStream_t)cuda_stream;
    return PARAMENT_OK;
}

int parament_set_hamiltonians(parament_ctx *ctx, int dim, int n_ctrl, const void *H0, const void *Hk,
                              parament_dtype dtype, parament_integrator integrator) {
    if (!ctx) return PARAMENT_ERR_INVALID_VALUE;
    ctx->err.clear();
    if (dim < 1) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "dim must be >= 1 (got %d)", dim);
    if (dim > kMaxDim)
        return set_err(ctx, PARAMENT_ERR_UNSUPPORTED, "dim %d > %d is not supported by this build", dim, kMaxDim);
    if (n_ctrl < 0 || n_ctrl > kMaxControls)
        return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "n_ctrl must be in [0, %d] (got %d)", kMaxControls, n_ctrl);
    if (!H0 || (n_ctrl > 0 && !Hk)) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "null Hamiltonian pointer");
    if (dtype != PARAMENT_C64 && dtype != PARAMENT_C128)
        return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "unknown dtype %d", (int)dtype);
    if (integrator != PARAMENT_MIDPOINT && integrator != PARAMENT_MAGNUS4_GL2 && integrator != PARAMENT_MAGNUS4_SIMPSON)
        return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "unknown integrator %d", (int)integrator);
    DeviceGuard guard(ctx->device);

    const size_t esz = dtype == PARAMENT_C128 ? 16 : 8;
    const size_t mat = (size_t)dim * dim * esz;
    int st = ws_reserve(ctx, ctx->hraw, mat * (1 + n_ctrl));
    if (st) return st;
    // stage H0 and Hk contiguously: raw[0] = H0, raw[1 + k] = H_k
    PM_CUDA(cudaMemcpyAsync(ctx->hraw.ptr, H0, mat, cudaMemcpyDefault, ctx->stream));
    if (n_ctrl > 0)
        PM_CUDA(cudaMemcpyAsync((char *)ctx->hraw.ptr + mat, Hk, mat * n_ctrl, cudaMemcpyDefault, ctx->stream));

    // Hermiticity and finiteness of the inputs
    PM_CUDA(cudaMemsetAsync(ctx->check.ptr, 0, ctx->check.bytes, ctx->stream));
    if (dtype == PARAMENT_C128)
        check_hermitian_kernel<double2><<<1 + n_ctrl, 256, 0, ctx->stream>>>(
            (const double2 *)ctx->hraw.ptr, dim, 1 + n_ctrl, (unsigned long long *)ctx->check.ptr);
    else
        check_hermitian_kernel<float2><<<1 + n_ctrl, 256, 0, ctx->stream>>>(
            (const float2 *)ctx->hraw.ptr, dim, 1 + n_ctrl, (unsigned long long *)ctx->check.ptr);
    PM_CUDA(cudaGetLastError());
    unsigned long long chk[3];
    PM_CUDA(cudaMemcpyAsync(chk, ctx->check.ptr, sizeof(chk), cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    double herr, hmax;
    std::memcpy(&herr, &chk[0], 8);
    std::memcpy(&hmax, &chk[1], 8);
    if (chk[2]) return set_err(ctx, PARAMENT_ERR_NONFINITE, "Hamiltonians contain NaN or Inf");
    if (ctx->opt_check_herm && herr > (double)ctx->opt_herm_tol * 1e-12 * std::max(hmax, 1e-300))
        return set_err(ctx, PARAMENT_ERR_NOT_HERMITIAN, "max |H - H^dagger| = %.3e exceeds tolerance (max |H| = %.3e)",
                       herr, hmax);

    const int Dp = pad_dim(dim);
    const int nb = n_basis_for(n_ctrl, integrator);
    const size_t DD = (size_t)Dp * Dp;
    if ((st = ws_reserve(ctx, ctx->full, nb * DD * sizeof(double2)))) return st;
    if ((st = ws_reserve(ctx, ctx->packed64, nb * DD * sizeof(double)))) return st;
    if ((st = ws_reserve(ctx, ctx->packed32, nb * DD * sizeof(float)))) return st;
    if ((st = ws_reserve(ctx, ctx->bnorm, nb * sizeof(double)))) return st;
    const int grid_cap = Dp <= kMaxSmallDim ? ctx->max_grid : 2 * ctx->sm_count;
    if ((st = ws_reserve(ctx, ctx->partials, (size_t)grid_cap * DD * sizeof(double2)))) return st;
    const int magnus = integrator != PARAMENT_MIDPOINT;
    const dim3 bgrid(nb, (unsigned)std::max<size_t>(1, DD / 256));
    if (dtype == PARAMENT_C128)
        build_basis_kernel<double2><<<bgrid, 256, 0, ctx->stream>>>((const double2 *)ctx->hraw.ptr, dim, Dp, n_ctrl,
                                                                    magnus, (double2 *)ctx->full.ptr);
    else
        build_basis_kernel<float2><<<bgrid, 256, 0, ctx->stream>>>((const float2 *)ctx->hraw.ptr, dim, Dp, n_ctrl,
                                                                   magnus, (double2 *)ctx->full.ptr);
    PM_CUDA(cudaGetLastError());
    if ((st = ws_reserve(ctx, ctx->bmax, nb * sizeof(double)))) return st;
    pack_basis_kernel<<<nb, 256, 0, ctx->stream>>>((const double2 *)ctx->full.ptr, Dp, (double *)ctx->packed64.ptr,
                                                   (float *)ctx->packed32.ptr, (double *)ctx->bnorm.ptr,
                                                   (double *)ctx->bmax.ptr);
    PM_CUDA(cudaGetLastError());

    // Identically zero basis matrices (e.g. commutators of controls acting on
    // different subsystems) contribute nothing to G_j: keep only the others.
    std::vector<double> bmax(nb);
    PM_CUDA(cudaMemcpyAsync(bmax.data(), ctx->bmax.ptr, nb * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->slot_of.assign(kMaxBasis, (short)-1);
    int kept = 0;
    for (int e = 0; e < nb; ++e)
        if (bmax[e] > 0.0) ctx->slot_of[e] = (short)kept++;
    if ((st = ws_reserve(ctx, ctx->cpacked64, std::max(kept, 1) * DD * sizeof(double)))) return st;
    if ((st = ws_reserve(ctx, ctx->cpacked32, std::max(kept, 1) * DD * sizeof(float)))) return st;
    if ((st = ws_reserve(ctx, ctx->cbnorm, std::max(kept, 1) * sizeof(double)))) return st;
    for (int e = 0; e < nb; ++e) {
        const int sl = ctx->slot_of[e];
        if (sl < 0) continue;
        PM_CUDA(cudaMemcpyAsync((double *)ctx->cpacked64.ptr + sl * DD, (double *)ctx->packed64.ptr + e * DD,
                                DD * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        PM_CUDA(cudaMemcpyAsync((float *)ctx->cpacked32.ptr + sl * DD, (float *)ctx->packed32.ptr + e * DD,
                                DD * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
        PM_CUDA(cudaMemcpyAsync((double *)ctx->cbnorm.ptr + sl, (double *)ctx->bnorm.ptr + e, sizeof(double),
                                cudaMemcpyDeviceToDevice, ctx->stream));
    }
    ctx->nb_eff = kept;

    ctx->dim = dim;
    ctx->dpad = Dp;
    ctx->K = n_ctrl;
    ctx->nb = nb;
    ctx->dtype = dtype;
    ctx->integ = integrator;
    ctx->ctrl = nullptr;
    ctx->state = 1;
    return PARAMENT_OK;
}

int parament_set_controls(parament_ctx *ctx, const void *c, parament_real_dtype cdtype, int64_t n_steps, double dt) {
    if (!ctx) return PARAMENT_ERR_INVALID_VALUE;
    ctx->err.clear();
    if (ctx->state < 1) return set_err(ctx, PARAMENT_ERR_STATE, "set_hamiltonians must come first");
    if (cdtype != PARAMENT_F32 && cdtype != PARAMENT_F64)
        return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "unknown control dtype %d", (int)cdtype);
    if (n_steps < 0 || n_steps > (int64_t)0x7fffffff)
        return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "n_steps out of range (%lld)", (long long)n_steps);
    if (!std::isfinite(dt)) return set_err(ctx, PARAMENT_ERR_NONFINITE, "dt is not finite");
    const int64_t S = samples_for(n_steps, ctx->integ);
    const size_t esz = cdtype == PARAMENT_F64 ? 8 : 4;
    const size_t bytes = (size_t)ctx->K * (size_t)S * esz;
    if (bytes > 0 && !c) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "null control pointer");
    DeviceGuard guard(ctx->device);
    const void *use = c;
    if (bytes > 0 && !is_device_ptr(c)) {
        if (const void *mapped = pinned_device_ptr(c)) {
            // page-locked host memory: the kernels read the samples in place, so the transfer
            // overlaps the computation instead of preceding it (each sample is read once)
            use = mapped;
        } else {
            int st = ws_reserve(ctx, ctx->ctrl_copy, bytes);
            if (st) return st;
            PM_CUDA(cudaMemcpyAsync(ctx->ctrl_copy.ptr, c, bytes, cudaMemcpyHostToDevice, ctx->stream));
            use = ctx->ctrl_copy.ptr;
        }
    }
    if (bytes > 0 && ((uintptr_t)use % esz))
        return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "control pointer not aligned to its element size");
    ctx->ctrl = use;
    ctx->cdtype = cdtype;
    ctx->n_steps = n_steps;
    ctx->S = S;
    ctx->dt = dt;
    ctx->state = 2;
    return PARAMENT_OK;
}

}  // extern "C"

namespace {

// Controls in the compute type, Taylor table and launch geometry of the fused
// forward kernel (shared by propagate and propagate_grad).
int forward_setup(parament_ctx *ctx, int fp64, void *U_dst, FusedParams &p, int &grid, int &warps, size_t &smem,
                  int &leaves_per_block, int tc = 0) {
    const int Dp = ctx->dpad, nb = ctx->nb_eff;
    const void *ctrl = ctx->ctrl;
    const int64_t count = (int64_t)ctx->K * ctx->S;
    const bool want64 = fp64 != 0;
    if (count > 0 && (ctx->cdtype == PARAMENT_F64) != want64) {
        int st = ws_reserve(ctx, ctx->ctrl_conv, (size_t)count * (want64 ? 8 : 4));
        if (st) return st;
        const int blocks = (int)std::min<int64_t>((count + 255) / 256, 4096);
        if (want64)
            convert_kernel<float, double><<<blocks, 256, 0, ctx->stream>>>((const float *)ctrl,
                                                                          (double *)ctx->ctrl_conv.ptr, count);
        else
            convert_kernel<double, float><<<blocks, 256, 0, ctx->stream>>>((const double *)ctrl,
                                                                          (float *)ctx->ctrl_conv.ptr, count);
        PM_CUDA(cudaGetLastError());
        ctrl = ctx->ctrl_conv.ptr;
    }

    std::memset(&p, 0, sizeof(p));
    const double u = fp64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
    if (build_classes(u, (int)ctx->opt_degree, p) <= 0)
        return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "Taylor degree %lld is not one of 1, 2, 4, 6, 9, 12",
                       (long long)ctx->opt_degree);

    if (Dp > kMaxSmallDim) {
        // one thread block (256 threads) per leaf; working matrices in a per-block scratch region
        warps = 8;
        smem = large_smem(Dp, fp64, nb, tc);
        if (smem > ctx->smem_optin) return set_err(ctx, PARAMENT_ERR_UNSUPPORTED, "large-d shared memory %zu B", smem);
        int bps = large_blocks_per_sm(Dp, fp64, (int)ctx->integ, smem, tc);
        if (bps <= 0) return set_err(ctx, PARAMENT_ERR_CUDA, "occupancy query failed (large d)");
        // the d <= 32 tensor-core body is compiled for two blocks per SM and they do run together
        // (measured: 2^14 slices at d = 32 in 1.7 ms with 304 blocks, 2.7 ms with 152), although
        // the occupancy query reports one
        if (tc && !fp64 && Dp == 32) bps = std::max(bps, 2);
        leaves_per_block = 1;
        grid = (int)ctx->opt_grid;
        if (grid <= 0) grid = (int)std::max<int64_t>(1, std::min<int64_t>(ctx->n_steps, (int64_t)bps * ctx->sm_count));
        grid = std::min(grid, 2 * ctx->sm_count);
        const size_t csz = fp64 ? sizeof(double2) : sizeof(float2);
        int st = ws_reserve(ctx, ctx->lscratch, (size_t)grid * 6 * Dp * Dp * csz);
        if (st) return st;
    } else {
    const int max_warps = fused_max_warps(Dp, fp64);
    warps = (int)ctx->opt_warps;
    if (warps <= 0) {
        warps = max_warps;
        while (warps > 1 && fused_smem(Dp, fp64, nb, warps) > ctx->smem_optin) --warps;
        if (fp64 && ctx->opt_grid <= 0) {
            // an FP64 slice costs ~64x an FP32 one (GB300's FP64 rate), so a short run is spread
            // over more SMs first: halve the warps per block while the grid that gives every leaf
            // kLeafMinSteps64 slices stays below one block per SM (d = 2, N = 2^14: 8 x 256 ->
            // 128 x 64 threads, 2.2x faster)
            auto blocks_for = [&](int w) {
                const int64_t per = (int64_t)w * fused_gpw(Dp, fp64) * kLeafMinSteps64;
                return (ctx->n_steps + per - 1) / per;
            };
            while (warps > 2 && blocks_for(warps) < ctx->sm_count) warps /= 2;
        }
    }
    if (warps > max_warps) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "at most %d warps per block", max_warps);
    smem = fused_smem(Dp, fp64, nb, warps);
    if (smem > ctx->smem_optin)
        return set_err(ctx, PARAMENT_ERR_UNSUPPORTED, "basis of %d matrices (d=%d) needs %zu B shared memory > %zu",
                       nb, ctx->dim, smem, ctx->smem_optin);
    const int bps = fused_blocks_per_sm(Dp, fp64, (int)ctx->integ, warps, smem);
    if (bps <= 0) return set_err(ctx, PARAMENT_ERR_CUDA, "occupancy query failed (%d warps, %zu B)", warps, smem);
    leaves_per_block = warps * fused_gpw(Dp, fp64);
    grid = (int)ctx->opt_grid;
    if (grid <= 0) {
        const int lm = fp64 ? kLeafMinSteps64 : kLeafMinSteps;
        const int64_t need = (ctx->n_steps + (int64_t)leaves_per_block * lm - 1) / ((int64_t)leaves_per_block * lm);
        grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)bps * ctx->sm_count));
    }
    grid = std::min(grid, ctx->max_grid);
    }

    p.ctrl = ctrl;
    p.S = ctx->S;
    p.n_steps = ctx->n_steps;
    p.K = ctx->K;
    p.n_basis = nb;
    p.n_coef = ctx->nb;
    for (int e = 0; e < kMaxBasis; ++e) p.slot_of[e] = ctx->slot_of[e];
    p.d_out = ctx->dim;
    p.out_c128 = ctx->dtype == PARAMENT_C128;
    p.dt = ctx->dt;
    p.packed = fp64 ? ctx->cpacked64.ptr : ctx->cpacked32.ptr;
    p.bnorm1 = (const double *)ctx->cbnorm.ptr;
    p.partials = (double2 *)ctx->partials.ptr;
    p.tickets = (unsigned *)ctx->tickets.ptr;
    p.U_out = U_dst;
    p.counters = (unsigned long long *)ctx->counters.ptr;
    p.status = (unsigned *)ctx->status.ptr;
    p.extra_squarings = (int)ctx->opt_extra_sq;
    p.unitary_step = fp64 ? 0 : (int)ctx->opt_unitary_step;
    return PARAMENT_OK;
}

cudaError_t forward_launch(parament_ctx *ctx, int fp64, const FusedParams &p, int grid, int warps, size_t smem,
                           int tc = 0) {
    if (ctx->dpad > kMaxSmallDim)
        return large_dispatch(ctx->dpad, fp64, (int)ctx->integ, p, ctx->lscratch.ptr, grid, smem, ctx->stream, tc);
    return fused_dispatch(ctx->dpad, fp64, (int)ctx->integ, p, grid, warps, smem, ctx->stream);
}

void record_launch(parament_ctx *ctx, int nb, int grid, int warps, int leaves_per_block,
                   unsigned backends = PARAMENT_BACKEND_CUDA_CORES) {
    ctx->last = parament_stats{};
    ctx->last.n_steps = ctx->n_steps;
    ctx->last.dim = ctx->dim;
    ctx->last.n_basis = nb;
    ctx->last.grid_blocks = grid;
    ctx->last.block_threads = warps * 32;
    ctx->last.leaves = grid * leaves_per_block;
    ctx->last.product_backends = backends;
    ctx->last.kernel_ms = -1.0;
}

// V^dagger, padded with zeros to Dp x Dp, in FP64
template <typename InT>
__global__ void vdag_kernel(const InT *V, int d, int Dp, double2 *out) {
    for (int t = threadIdx.x; t < Dp * Dp; t += blockDim.x) {
        const int i = t / Dp, j = t % Dp;
        double2 v = make_double2(0.0, 0.0);
        if (i < d && j < d) {
            const InT x = V[j * d + i];
            v = make_double2((double)x.x, -(double)x.y);
        }
        out[t] = v;
    }
}

// psi_0 padded with zeros to Dp entries, in FP64
template <typename InT>
__global__ void psi_pad_kernel(const InT *psi, int d, int Dp, double2 *out) {
    for (int t = threadIdx.x; t < Dp; t += blockDim.x)
        out[t] = t < d ? make_double2((double)psi[t].x, (double)psi[t].y) : make_double2(0.0, 0.0);
}

}  // namespace

extern "C" {

int parament_propagate(parament_ctx *ctx, void *U_out, parament_precision prec) {
    if (!ctx) return PARAMENT_ERR_INVALID_VALUE;
    ctx->err.clear();
    if (ctx->state < 2) return set_err(ctx, PARAMENT_ERR_STATE, "set_hamiltonians and set_controls must come first");
    if (!U_out) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "null U_out");
    const bool tc_prec = prec == PARAMENT_PREC_FP32_TC_TF32X3 || prec == PARAMENT_PREC_FP32_TC_BF16X3;
    if (tc_prec && ctx->dpad <= kMaxSmallDim)
        return set_err(ctx, PARAMENT_ERR_UNSUPPORTED, "tensor-core products are used for d > %d only", kMaxSmallDim);
    if (prec != PARAMENT_PREC_FP64 && prec != PARAMENT_PREC_FP32 && !tc_prec)
        return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "unknown precision %d", (int)prec);
    DeviceGuard guard(ctx->device);
    const int fp64 = prec == PARAMENT_PREC_FP64;
    const int tc = prec == PARAMENT_PREC_FP32_TC_TF32X3 ? 1 : (prec == PARAMENT_PREC_FP32_TC_BF16X3 ? 2 : 0);

    const size_t esz = ctx->dtype == PARAMENT_C128 ? 16 : 8;
    const bool host_out = !is_device_ptr(U_out);
    void *dst = U_out;
    if (host_out) {
        int st = ws_reserve(ctx, ctx->uout, (size_t)ctx->dim * ctx->dim * esz);
        if (st) return st;
        dst = ctx->uout.ptr;
    } else if ((uintptr_t)U_out % esz) {
        return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "U_out not aligned to its element size");
    }

    FusedParams p;
    int grid = 0, warps = 0, lpb = 0;
    size_t smem = 0;
    const int cheb = ctx->opt_exp_method == 1;
    int st = forward_setup(ctx, fp64, dst, p, grid, warps, smem, lpb, tc);
    if (st) return st;
    if (cheb) {
        // common spectral half-width over all slices, then degree and coefficients, on the device
        if ((st = ws_reserve(ctx, ctx->cheb, 1024))) return st;
        unsigned char *cw = (unsigned char *)ctx->cheb.ptr;
        unsigned long long *numax = (unsigned long long *)cw;
        int *mptr = (int *)(cw + 8);
        double *ibeta = (double *)(cw + 16);
        void *coef = cw + 32;
        PM_CUDA(cudaMemsetAsync(numax, 0, 8, ctx->stream));
        const int bgrid = (int)std::max<int64_t>(1, std::min<int64_t>((ctx->n_steps + 255) / 256, 4 * ctx->sm_count));
        const ChebTheta &th = cheb_theta_table(fp64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24));
        const int ig = (int)ctx->integ;
        if (fp64) {
            if (ig == 0) cheb_bound_kernel<double, kMidpoint><<<bgrid, 256, 0, ctx->stream>>>(p, numax, p.status);
            else if (ig == 1) cheb_bound_kernel<double, kGL2><<<bgrid, 256, 0, ctx->stream>>>(p, numax, p.status);
            else cheb_bound_kernel<double, kSimpson><<<bgrid, 256, 0, ctx->stream>>>(p, numax, p.status);
            cheb_coef_kernel<double2><<<1, 32, 0, ctx->stream>>>(numax, th, mptr, ibeta, (double2 *)coef, p.status);
        } else {
            if (ig == 0) cheb_bound_kernel<float, kMidpoint><<<bgrid, 256, 0, ctx->stream>>>(p, numax, p.status);
            else if (ig == 1) cheb_bound_kernel<float, kGL2><<<bgrid, 256, 0, ctx->stream>>>(p, numax, p.status);
            else cheb_bound_kernel<float, kSimpson><<<bgrid, 256, 0, ctx->stream>>>(p, numax, p.status);
            cheb_coef_kernel<float2><<<1, 32, 0, ctx->stream>>>(numax, th, mptr, ibeta, (float2 *)coef, p.status);
        }
        PM_CUDA(cudaGetLastError());
        p.cheb_m = mptr;
        p.cheb_inv_beta = ibeta;
        p.cheb_coef = coef;
        if (ctx->dpad > kMaxSmallDim) {
            // the block-level kernel switches to the Clenshaw recurrence when cheb_m is set
            PM_CUDA(forward_launch(ctx, fp64, p, grid, warps, smem, tc));
        } else {
            if (fused_blocks_per_sm(ctx->dpad, fp64, ig, warps, smem, 1) <= 0)
                return set_err(ctx, PARAMENT_ERR_CUDA, "occupancy query failed (Chebyshev kernel)");
            PM_CUDA(fused_dispatch(ctx->dpad, fp64, ig, p, grid, warps, smem, ctx->stream, 1));
        }
    } else {
        PM_CUDA(forward_launch(ctx, fp64, p, grid, warps, smem, tc));
    }
    record_launch(ctx, ctx->nb_eff, grid, warps, lpb, product_backend(ctx->dpad, fp64, tc));

    if (host_out) {
        PM_CUDA(cudaMemcpyAsync(U_out, dst, (size_t)ctx->dim * ctx->dim * esz, cudaMemcpyDeviceToHost, ctx->stream));
        PM_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return PARAMENT_OK;
}

int parament_propagate_grad(parament_ctx *ctx, const void *V, double *loss_out, void *grad_out, void *U_out,
                            parament_precision prec) {
    if (!ctx) return PARAMENT_ERR_INVALID_VALUE;
    ctx->err.clear();
    if (ctx->state < 2) return set_err(ctx, PARAMENT_ERR_STATE, "set_hamiltonians and set_controls must come first");
    if (!V || !grad_out) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "null V or grad_out");
    if (prec != PARAMENT_PREC_FP64 && prec != PARAMENT_PREC_FP32)
        return set_err(ctx, PARAMENT_ERR_UNSUPPORTED, "gradient precision must be FP64 or FP32");
    DeviceGuard guard(ctx->device);
    const int fp64 = prec == PARAMENT_PREC_FP64;
    const int Dp = ctx->dpad, d = ctx->dim, K = ctx->K;
    const size_t DD = (size_t)Dp * Dp;
    const size_t esz = ctx->dtype == PARAMENT_C128 ? 16 : 8;
    const size_t rsz = fp64 ? 8 : 4;
    const int64_t N = ctx->n_steps;
    int st;

    // V (host or device) -> V^dagger padded, FP64
    const void *Vd = V;
    if (!is_device_ptr(V)) {
        if ((st = ws_reserve(ctx, ctx->gv, (size_t)d * d * esz))) return st;
        PM_CUDA(cudaMemcpyAsync(ctx->gv.ptr, V, (size_t)d * d * esz, cudaMemcpyHostToDevice, ctx->stream));
        Vd = ctx->gv.ptr;
    }
    if ((st = ws_reserve(ctx, ctx->gvdag, DD * sizeof(double2)))) return st;
    if (ctx->dtype == PARAMENT_C128)
        vdag_kernel<double2><<<1, 256, 0, ctx->stream>>>((const double2 *)Vd, d, Dp, (double2 *)ctx->gvdag.ptr);
    else
        vdag_kernel<float2><<<1, 256, 0, ctx->stream>>>((const float2 *)Vd, d, Dp, (double2 *)ctx->gvdag.ptr);
    PM_CUDA(cudaGetLastError());

    // forward pass keeping every leaf and block product
    const bool host_u = U_out && !is_device_ptr(U_out);
    if ((st = ws_reserve(ctx, ctx->uout, (size_t)d * d * esz))) return st;
    void *udst = (U_out && !host_u) ? U_out : ctx->uout.ptr;
    FusedParams p;
    int grid = 0, warps = 0, lpb = 0;
    size_t smem = 0;
    if ((st = forward_setup(ctx, fp64, udst, p, grid, warps, smem, lpb))) return st;
    const int64_t L = (int64_t)grid * lpb;
    const bool large = Dp > kMaxSmallDim;  // one leaf per thread block, block-level adjoint
    if ((st = ws_reserve(ctx, ctx->gleaf, (size_t)L * DD * sizeof(double2)))) return st;
    if ((st = ws_reserve(ctx, ctx->gz, 4 * sizeof(double)))) return st;
    p.leaf_out = (double2 *)ctx->gleaf.ptr;
    if (large) {
        // prefix scan over L + 1 elements (the last prefix is U(T)) and suffix scan, ping-pong each
        if ((st = ws_reserve(ctx, ctx->gpin, (2 * (size_t)(L + 1) + 2 * (size_t)L) * DD * sizeof(double2))))
            return st;
        p.block_out = nullptr;
        PM_CUDA(forward_launch(ctx, fp64, p, grid, warps, smem, 0));
        record_launch(ctx, ctx->nb_eff, grid, warps, lpb);
    } else {
        if ((st = ws_reserve(ctx, ctx->gblock, (size_t)grid * DD * sizeof(double2)))) return st;
        if ((st = ws_reserve(ctx, ctx->gbpin, 2 * (size_t)grid * DD * sizeof(double2)))) return st;
        if ((st = ws_reserve(ctx, ctx->gpin, 2 * (size_t)L * DD * sizeof(double2)))) return st;
        p.block_out = (double2 *)ctx->gblock.ptr;
        PM_CUDA(fused_dispatch(Dp, fp64, (int)ctx->integ, p, grid, warps, smem, ctx->stream));
        record_launch(ctx, ctx->nb_eff, grid, warps, lpb);
    }

    // adjoint launch geometry: d <= 16 warp groups over a persistent grid, d > 16 one block per leaf
    int aw = 8, agrid = 0;
    size_t asmem = 0;
    int64_t TG = 0;
    if (large) {
        asmem = adjoint_large_smem(Dp, fp64);
        if (asmem > ctx->smem_optin)
            return set_err(ctx, PARAMENT_ERR_UNSUPPORTED, "adjoint needs %zu B shared memory", asmem);
        TG = L;
    } else {
        while (aw > 1 && adjoint_smem(Dp, fp64, K, aw) > ctx->smem_optin) --aw;
        asmem = adjoint_smem(Dp, fp64, K, aw);
        if (asmem > ctx->smem_optin)
            return set_err(ctx, PARAMENT_ERR_UNSUPPORTED, "adjoint needs %zu B shared memory", asmem);
        const int abps = adjoint_blocks_per_sm(Dp, fp64, (int)ctx->integ, aw, asmem);
        if (abps <= 0) return set_err(ctx, PARAMENT_ERR_CUDA, "adjoint occupancy query failed");
        agrid = abps * ctx->sm_count;
        TG = (int64_t)agrid * aw * fused_gpw(Dp, fp64);
    }
    const int64_t maxlen = L > 0 ? (N + L - 1) / L : 0;
    int64_t c_sub = ctx->opt_grad_subchunk > 0 ? ctx->opt_grad_subchunk : std::max<int64_t>(maxlen, 1);
    const size_t csz = 2 * rsz;  // complex element
    const size_t cap = (size_t)ctx->opt_workspace_mb << 20;
    while (c_sub > 1 && (size_t)TG * c_sub * DD * csz > cap) c_sub = (c_sub + 1) / 2;
    const int64_t n_ckpt = std::max<int64_t>(1, (maxlen + c_sub - 1) / c_sub);
    if ((st = ws_reserve(ctx, ctx->gpbuf, (size_t)TG * c_sub * DD * csz))) return st;
    if ((st = ws_reserve(ctx, ctx->gckpt, (size_t)TG * n_ckpt * DD * csz))) return st;
    if (large && (st = ws_reserve(ctx, ctx->gadj, (size_t)L * kGradSlots * DD * csz))) return st;

    void *gdst = grad_out;
    const bool host_g = !is_device_ptr(grad_out);
    const size_t gbytes = (size_t)K * ctx->S * rsz;
    if (host_g) {
        if ((st = ws_reserve(ctx, ctx->ggrad, std::max<size_t>(gbytes, 8)))) return st;
        gdst = ctx->ggrad.ptr;
    }

    ScanParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.leafpart = (const double2 *)ctx->gleaf.ptr;
    sp.blockpart = (const double2 *)ctx->gblock.ptr;
    sp.n_blocks = grid;
    sp.leaves_per_block = lpb;
    sp.bpin = (double2 *)ctx->gbpin.ptr;
    sp.bsout = sp.bpin + (size_t)grid * DD;
    sp.pin = (double2 *)ctx->gpin.ptr;
    sp.sout = sp.pin + (size_t)L * DD;
    sp.vdag = (const double2 *)ctx->gvdag.ptr;
    sp.z = (double *)ctx->gz.ptr;
    sp.U_out = nullptr;
    sp.d_out = d;

    GradParams gp;
    std::memset(&gp, 0, sizeof(gp));
    gp.ctrl = p.ctrl;
    gp.S = ctx->S;
    gp.n_steps = N;
    gp.K = K;
    gp.n_basis = ctx->nb_eff;
    gp.n_coef = ctx->nb;
    gp.dt = ctx->dt;
    for (int e = 0; e < kMaxBasis; ++e) gp.slot_of[e] = ctx->slot_of[e];
    gp.packed = p.packed;
    gp.bnorm1 = p.bnorm1;
    gp.pin = sp.pin;
    gp.sout = sp.sout;
    gp.vdag = sp.vdag;
    gp.z = sp.z;
    gp.grad = gdst;
    gp.pbuf = ctx->gpbuf.ptr;
    gp.ckpt = ctx->gckpt.ptr;
    gp.c_sub = (int)c_sub;
    gp.n_ckpt = (int)n_ckpt;
    gp.n_leaves = L;
    gp.d_true = d;
    gp.status = (unsigned *)ctx->status.ptr;
    {
        const double u = fp64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
        FusedParams tmp;
        std::memset(&tmp, 0, sizeof(tmp));
        build_classes(u, 0, tmp);
        gp.n_cls = tmp.n_cls;
        std::memcpy(gp.cls_cap, tmp.cls_cap, sizeof(gp.cls_cap));
        std::memcpy(gp.cls_code, tmp.cls_code, sizeof(gp.cls_code));
        std::memcpy(gp.coef_d, tmp.coef_d, sizeof(gp.coef_d));
        std::memcpy(gp.coef_f, tmp.coef_f, sizeof(gp.coef_f));
        std::memset(&tmp, 0, sizeof(tmp));
        build_classes(u, 0, tmp, 1);
        gp.n_dcls = tmp.n_cls;
        std::memcpy(gp.dcls_cap, tmp.cls_cap, sizeof(gp.dcls_cap));
        std::memcpy(gp.dcls_code, tmp.cls_code, sizeof(gp.dcls_code));
    }
    if (gbytes) PM_CUDA(cudaMemsetAsync(gdst, 0, gbytes, ctx->stream));  // Simpson end points accumulate
    if (large) {
        // FP64 prefix / suffix scans, z and U(T) from them, then the block-level adjoint
        double2 *pre = (double2 *)ctx->gpin.ptr, *suf = pre + 2 * (size_t)(L + 1) * DD;
        PM_CUDA(grad_large_run(Dp, fp64, (int)ctx->integ, (const double2 *)ctx->gleaf.ptr, (int)L, pre, suf, gp,
                               ctx->gadj.ptr, udst, ctx->dtype == PARAMENT_C128, d, ctx->stream));
    } else {
        PM_CUDA(grad_run(Dp, fp64, (int)ctx->integ, sp, gp, agrid, aw, asmem, ctx->stream));
    }
    ctx->last.grad_subchunk = (int32_t)c_sub;

    if (host_g && gbytes) PM_CUDA(cudaMemcpyAsync(grad_out, gdst, gbytes, cudaMemcpyDeviceToHost, ctx->stream));
    if (host_u) PM_CUDA(cudaMemcpyAsync(U_out, udst, (size_t)d * d * esz, cudaMemcpyDeviceToHost, ctx->stream));
    if (loss_out) {
        double z[4];
        PM_CUDA(cudaMemcpyAsync(z, ctx->gz.ptr, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        PM_CUDA(cudaStreamSynchronize(ctx->stream));
        *loss_out = z[2];
    } else if (host_g || host_u) {
        PM_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return PARAMENT_OK;
}

int parament_propagate_trajectory(parament_ctx *ctx, const void *psi0, void *out, int64_t every,
                                  parament_precision prec) {
    if (!ctx) return PARAMENT_ERR_INVALID_VALUE;
    ctx->err.clear();
    if (ctx->state < 2) return set_err(ctx, PARAMENT_ERR_STATE, "set_hamiltonians and set_controls must come first");
    if (every < 1) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "every must be >= 1");
    if (!out && ctx->n_steps > 0) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "null out");
    if (prec != PARAMENT_PREC_FP64 && prec != PARAMENT_PREC_FP32)
        return set_err(ctx, PARAMENT_ERR_UNSUPPORTED, "trajectory precision must be FP64 or FP32");
    if (ctx->opt_exp_method != 0)
        return set_err(ctx, PARAMENT_ERR_UNSUPPORTED, "trajectories use the Taylor exponential");
    DeviceGuard guard(ctx->device);
    const int fp64 = prec == PARAMENT_PREC_FP64;
    const int Dp = ctx->dpad, d = ctx->dim;
    const size_t DD = (size_t)Dp * Dp;
    const size_t esz = ctx->dtype == PARAMENT_C128 ? 16 : 8;
    const int64_t N = ctx->n_steps;
    const int64_t n_out = (N + every - 1) / every;
    const size_t obytes = (size_t)n_out * (psi0 ? (size_t)d : (size_t)d * d) * esz;
    if (n_out == 0) return PARAMENT_OK;
    int st;

    // psi_0 (host or device) -> padded FP64
    const double2 *psi_dev = nullptr;
    if (psi0) {
        if ((st = ws_reserve(ctx, ctx->tpsi, (size_t)Dp * sizeof(double2)))) return st;
        if (is_device_ptr(psi0)) {
            if (ctx->dtype == PARAMENT_C128)
                psi_pad_kernel<double2><<<1, 32, 0, ctx->stream>>>((const double2 *)psi0, d, Dp, (double2 *)ctx->tpsi.ptr);
            else
                psi_pad_kernel<float2><<<1, 32, 0, ctx->stream>>>((const float2 *)psi0, d, Dp, (double2 *)ctx->tpsi.ptr);
            PM_CUDA(cudaGetLastError());
        } else {
            ctx->tpsi_host.assign(Dp, make_double2(0.0, 0.0));
            for (int i = 0; i < d; ++i) {
                if (ctx->dtype == PARAMENT_C128) ctx->tpsi_host[i] = ((const double2 *)psi0)[i];
                else ctx->tpsi_host[i] = make_double2(((const float2 *)psi0)[i].x, ((const float2 *)psi0)[i].y);
            }
            PM_CUDA(cudaMemcpyAsync(ctx->tpsi.ptr, ctx->tpsi_host.data(), (size_t)Dp * sizeof(double2),
                                    cudaMemcpyHostToDevice, ctx->stream));
        }
        psi_dev = (const double2 *)ctx->tpsi.ptr;
    }
    const bool host_out = !is_device_ptr(out);
    void *odst = out;
    if (host_out) {
        if ((st = ws_reserve(ctx, ctx->tstage, obytes))) return st;
        odst = ctx->tstage.ptr;
    } else if ((uintptr_t)out % esz) {
        return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "out not aligned to its element size");
    }

    // forward pass keeping every leaf and block product (U(T) into the scratch output)
    if ((st = ws_reserve(ctx, ctx->uout, (size_t)d * d * esz))) return st;
    FusedParams p;
    int grid = 0, warps = 0, lpb = 0;
    size_t smem = 0;
    if ((st = forward_setup(ctx, fp64, ctx->uout.ptr, p, grid, warps, smem, lpb))) return st;
    const int64_t L = (int64_t)grid * lpb;
    if ((st = ws_reserve(ctx, ctx->gleaf, (size_t)L * DD * sizeof(double2)))) return st;
    if (Dp > kMaxSmallDim) {
        // block-level kernel: one leaf per block; FP64 prefix scan over the leaf products
        if ((st = ws_reserve(ctx, ctx->gpin, 2 * (size_t)L * DD * sizeof(double2)))) return st;
        p.leaf_out = (double2 *)ctx->gleaf.ptr;
        PM_CUDA(forward_launch(ctx, fp64, p, grid, warps, smem));
        record_launch(ctx, ctx->nb_eff, grid, warps, lpb);
        double2 *pin = nullptr;
        PM_CUDA(large_prefix(Dp, (const double2 *)ctx->gleaf.ptr, (int)L, (double2 *)ctx->gpin.ptr,
                             (double2 *)ctx->gpin.ptr + (size_t)L * DD, &pin, ctx->stream));
        FusedParams pt = p;
        pt.leaf_out = nullptr;
        pt.traj_pin = pin;
        pt.traj_out = odst;
        pt.traj_psi0 = psi_dev;
        pt.traj_every = every;
        PM_CUDA(forward_launch(ctx, fp64, pt, grid, warps, smem));
        if (host_out) {
            PM_CUDA(cudaMemcpyAsync(out, odst, obytes, cudaMemcpyDeviceToHost, ctx->stream));
            PM_CUDA(cudaStreamSynchronize(ctx->stream));
        }
        return PARAMENT_OK;
    }
    if ((st = ws_reserve(ctx, ctx->gblock, (size_t)grid * DD * sizeof(double2)))) return st;
    if ((st = ws_reserve(ctx, ctx->gbpin, 2 * (size_t)grid * DD * sizeof(double2)))) return st;
    if ((st = ws_reserve(ctx, ctx->gpin, 2 * (size_t)L * DD * sizeof(double2)))) return st;
    p.leaf_out = (double2 *)ctx->gleaf.ptr;
    p.block_out = (double2 *)ctx->gblock.ptr;
    PM_CUDA(fused_dispatch(Dp, fp64, (int)ctx->integ, p, grid, warps, smem, ctx->stream));
    record_launch(ctx, ctx->nb_eff, grid, warps, lpb);

    // exclusive prefix of every leaf (FP64)
    ScanParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.leafpart = (const double2 *)ctx->gleaf.ptr;
    sp.blockpart = (const double2 *)ctx->gblock.ptr;
    sp.n_blocks = grid;
    sp.leaves_per_block = lpb;
    sp.bpin = (double2 *)ctx->gbpin.ptr;
    sp.bsout = sp.bpin + (size_t)grid * DD;
    sp.pin = (double2 *)ctx->gpin.ptr;
    sp.sout = sp.pin + (size_t)L * DD;
    sp.d_out = d;
    PM_CUDA(scan_run(Dp, sp, ctx->stream));

    // second pass: every leaf from its prefix, running product at the output slices
    FusedParams pt = p;
    pt.leaf_out = nullptr;
    pt.block_out = nullptr;
    pt.traj_pin = sp.pin;
    pt.traj_out = odst;
    pt.traj_psi0 = psi_dev;
    pt.traj_every = every;
    PM_CUDA(fused_dispatch(Dp, fp64, (int)ctx->integ, pt, grid, warps, smem, ctx->stream, 2));

    if (host_out) {
        PM_CUDA(cudaMemcpyAsync(out, odst, obytes, cudaMemcpyDeviceToHost, ctx->stream));
        PM_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return PARAMENT_OK;
}

int parament_get_stats(parament_ctx *ctx, parament_stats *out) {
    if (!ctx || !out) return PARAMENT_ERR_INVALID_VALUE;
    DeviceGuard guard(ctx->device);
    unsigned long long cnt[8];
    unsigned stv[2];
    PM_CUDA(cudaMemcpyAsync(cnt, ctx->counters.ptr, sizeof(cnt), cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaMemcpyAsync(stv, ctx->status.ptr, sizeof(stv), cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    parament_stats s = ctx->last;
    s.exp_products = (int64_t)cnt[4];
    s.tree_products = (int64_t)cnt[5];
    s.max_degree = (int32_t)cnt[6];
    s.max_squarings = (int32_t)cnt[7];
    s.device_status = stv[1];
    *out = s;
    return PARAMENT_OK;
}

int parament_set_option(parament_ctx *ctx, int key, int64_t value) {
    if (!ctx) return PARAMENT_ERR_INVALID_VALUE;
    switch (key) {
        case PARAMENT_OPT_TAYLOR_DEGREE:
            if (value != 0 && value != 1 && value != 2 && value != 4 && value != 6 && value != 9 && value != 12)
                return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "Taylor degree must be 0 or one of 1,2,4,6,9,12");
            ctx->opt_degree = value;
            return PARAMENT_OK;
        case PARAMENT_OPT_GRID_BLOCKS:
            if (value < 0 || value > ctx->max_grid)
                return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "grid blocks must be in [0, %d]", ctx->max_grid);
            ctx->opt_grid = value;
            return PARAMENT_OK;
        case PARAMENT_OPT_BLOCK_WARPS:
            if (value < 0 || value > 16) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "block warps must be in [0, 16]");
            ctx->opt_warps = value;
            return PARAMENT_OK;
        case PARAMENT_OPT_CHECK_HERMITIAN:
            ctx->opt_check_herm = value != 0;
            return PARAMENT_OK;
        case PARAMENT_OPT_EXTRA_SQUARINGS:
            if (value < 0 || value > 16) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "extra squarings in [0, 16]");
            ctx->opt_extra_sq = value;
            return PARAMENT_OK;
        case PARAMENT_OPT_HERMITIAN_TOL_E12:
            if (value < 0) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "tolerance must be >= 0");
            ctx->opt_herm_tol = value;
            return PARAMENT_OK;
        case PARAMENT_OPT_GRAD_SUBCHUNK:
            if (value < 0 || value > (1 << 24)) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "sub-chunk in [0, 2^24]");
            ctx->opt_grad_subchunk = value;
            return PARAMENT_OK;
        case PARAMENT_OPT_WORKSPACE_MB:
            if (value < 1) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "workspace cap must be >= 1 MiB");
            ctx->opt_workspace_mb = value;
            return PARAMENT_OK;
        case PARAMENT_OPT_BATCH_LEAF_STEPS:
            if (value < 0 || value > (1 << 20)) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "leaf steps in [0, 2^20]");
            ctx->opt_batch_leaf = value;
            return PARAMENT_OK;
        case PARAMENT_OPT_BATCH_ITEMS_PER_SM:
            if (value < 0 || value > 64) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "items per SM in [0, 64]");
            ctx->opt_batch_items = value;
            return PARAMENT_OK;
        case PARAMENT_OPT_BATCH_GRAPH:
            ctx->opt_batch_graph = value != 0;
            return PARAMENT_OK;
        case PARAMENT_OPT_EXP_METHOD:
            if (value != 0 && value != 1) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "exp method is 0 or 1");
            ctx->opt_exp_method = value;
            return PARAMENT_OK;
        case PARAMENT_OPT_UNITARY_STEP:
            ctx->opt_unitary_step = value != 0;
            return PARAMENT_OK;
        case PARAMENT_OPT_BATCH_CUDA_CORE_CLASSES:
            if (value < 0 || value > 7) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "class mask in [0, 7]");
            ctx->opt_batch_cuda_mask = value;
            return PARAMENT_OK;
    }
    return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "unknown option key %d", key);
}

int parament_get_option(const parament_ctx *ctx, int key, int64_t *value) {
    if (!ctx || !value) return PARAMENT_ERR_INVALID_VALUE;
    switch (key) {
        case PARAMENT_OPT_TAYLOR_DEGREE: *value = ctx->opt_degree; return PARAMENT_OK;
        case PARAMENT_OPT_GRID_BLOCKS: *value = ctx->opt_grid; return PARAMENT_OK;
        case PARAMENT_OPT_BLOCK_WARPS: *value = ctx->opt_warps; return PARAMENT_OK;
        case PARAMENT_OPT_CHECK_HERMITIAN: *value = ctx->opt_check_herm; return PARAMENT_OK;
        case PARAMENT_OPT_EXTRA_SQUARINGS: *value = ctx->opt_extra_sq; return PARAMENT_OK;
        case PARAMENT_OPT_HERMITIAN_TOL_E12: *value = ctx->opt_herm_tol; return PARAMENT_OK;
        case PARAMENT_OPT_GRAD_SUBCHUNK: *value = ctx->opt_grad_subchunk; return PARAMENT_OK;
        case PARAMENT_OPT_WORKSPACE_MB: *value = ctx->opt_workspace_mb; return PARAMENT_OK;
        case PARAMENT_OPT_BATCH_LEAF_STEPS: *value = ctx->opt_batch_leaf; return PARAMENT_OK;
        case PARAMENT_OPT_BATCH_ITEMS_PER_SM: *value = ctx->opt_batch_items; return PARAMENT_OK;
        case PARAMENT_OPT_BATCH_GRAPH: *value = ctx->opt_batch_graph; return PARAMENT_OK;
        case PARAMENT_OPT_EXP_METHOD: *value = ctx->opt_exp_method; return PARAMENT_OK;
        case PARAMENT_OPT_UNITARY_STEP: *value = ctx->opt_unitary_step; return PARAMENT_OK;
        case PARAMENT_OPT_BATCH_CUDA_CORE_CLASSES: *value = ctx->opt_batch_cuda_mask; return PARAMENT_OK;
    }
    return PARAMENT_ERR_INVALID_VALUE;
}

}  // extern "C"

// ------------------------------------------------------------------ helpers for other translation units

#include "pm_internal.h"

namespace pm {

int fill_classes(double u, int force_m, FusedParams &p) { return build_classes(u, force_m, p); }

cudaError_t fused_launch(int Dp, int fp64, int integ, const FusedParams &p, int grid, int warps, size_t smem,
                         cudaStream_t st) {
    return fused_dispatch(Dp, fp64, integ, p, grid, warps, smem, st);
}

int fused_occupancy(int Dp, int fp64, int integ, int warps, size_t smem) {
    return fused_blocks_per_sm(Dp, fp64, integ, warps, smem);
}

size_t fused_smem_size(int Dp, int fp64, int n_basis, int warps) { return fused_smem(Dp, fp64, n_basis, warps); }

int fused_groups(int Dp, int fp64) { return fused_gpw(Dp, fp64); }

cudaError_t basis_build(const void *raw, int c128, int d, int Dp, int K, int magnus, int nb, double2 *full,
                        double *p64, float *p32, double *bnorm, double *bmax, cudaStream_t st) {
    const dim3 bgrid(nb, (unsigned)std::max(1, Dp * Dp / 256));
    if (c128)
        build_basis_kernel<double2><<<bgrid, 256, 0, st>>>((const double2 *)raw, d, Dp, K, magnus, full);
    else
        build_basis_kernel<float2><<<bgrid, 256, 0, st>>>((const float2 *)raw, d, Dp, K, magnus, full);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    pack_basis_kernel<<<nb, 256, 0, st>>>(full, Dp, p64, p32, bnorm, bmax);
    return cudaGetLastError();
}

}  // namespace pm

// ------------------------------------------------------------------ batched propagation

namespace {

// variant = 4 * magnus + (FP64 ? 3 : tensor-core format), format 0 none, 1 3xTF32, 2 split BF16x3
cudaError_t batched_launch(int variant, const BatchItem *items, int n_items, unsigned *queue,
                           const FusedParams *params, unsigned char *scratch, size_t stride, int grid, size_t smem,
                           unsigned *status, cudaStream_t st) {
    switch (variant) {
        case 0: return batched_launch_fm(items, n_items, queue, params, scratch, stride, grid, smem, status, st);
        case 1: return batched_launch_fm_tc(items, n_items, queue, params, scratch, stride, grid, smem, status, st);
        case 2: return batched_launch_fm_bf(items, n_items, queue, params, scratch, stride, grid, smem, status, st);
        case 3: return batched_launch_dm(items, n_items, queue, params, scratch, stride, grid, smem, status, st);
        case 4: return batched_launch_fg(items, n_items, queue, params, scratch, stride, grid, smem, status, st);
        case 5: return batched_launch_fg_tc(items, n_items, queue, params, scratch, stride, grid, smem, status, st);
        case 6: return batched_launch_fg_bf(items, n_items, queue, params, scratch, stride, grid, smem, status, st);
        case 7: return batched_launch_dg(items, n_items, queue, params, scratch, stride, grid, smem, status, st);
    }
    return cudaErrorInvalidValue;
}

int batched_occupancy(int variant, size_t smem) {
    switch (variant) {
        case 0: return batched_blocks_per_sm_fm(smem);
        case 1: return batched_blocks_per_sm_fm_tc(smem);
        case 2: return batched_blocks_per_sm_fm_bf(smem);
        case 3: return batched_blocks_per_sm_dm(smem);
        case 4: return batched_blocks_per_sm_fg(smem);
        case 5: return batched_blocks_per_sm_fg_tc(smem);
        case 6: return batched_blocks_per_sm_fg_bf(smem);
        case 7: return batched_blocks_per_sm_dg(smem);
    }
    return 0;
}

// dimension class of the batched tensor-core choice: D = 32, 64, 128 -> 0, 1, 2 (-1 below 32)
int batch_tc_class(int Dp) { return Dp == 32 ? 0 : (Dp == 64 ? 1 : (Dp == 128 ? 2 : -1)); }

// the code that runs the complex products of one dimension class of the batched kernel
// (cuda_mask: bit batch_tc_class(D) set = that class runs on the CUDA cores in a tensor-core batch)
unsigned batch_backend(int Dp, int fp64, int tc, unsigned cuda_mask) {
    const int cls = batch_tc_class(Dp);
    if (fp64 || !tc || cls < 0 || ((cuda_mask >> cls) & 1u)) return PARAMENT_BACKEND_CUDA_CORES;
    return PARAMENT_BACKEND_TCGEN05;
}

// Build (when the shapes change) and enqueue one batched propagation.
int batch_run(parament_ctx *ctx, const parament_instance *inst, int n, parament_dtype dtype,
              parament_real_dtype cdtype, parament_integrator integ, parament_precision prec) {
    if (n < 0 || (n > 0 && !inst)) return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "bad instance list");
    if (dtype != PARAMENT_C64 && dtype != PARAMENT_C128)
        return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "unknown dtype %d", (int)dtype);
    if (integ != PARAMENT_MIDPOINT && integ != PARAMENT_MAGNUS4_GL2)
        return set_err(ctx, PARAMENT_ERR_UNSUPPORTED, "batched propagation supports midpoint and GL4 Magnus");
    if (prec != PARAMENT_PREC_FP64 && prec != PARAMENT_PREC_FP32 && prec != PARAMENT_PREC_FP32_TC_TF32X3 &&
        prec != PARAMENT_PREC_FP32_TC_BF16X3)
        return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "unknown precision %d", (int)prec);
    const int fp64 = prec == PARAMENT_PREC_FP64;
    const int tc = prec == PARAMENT_PREC_FP32_TC_TF32X3 ? 1 : (prec == PARAMENT_PREC_FP32_TC_BF16X3 ? 2 : 0);
    if ((cdtype == PARAMENT_F64) != (fp64 != 0))
        return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "control dtype must match the precision in batched calls");
    const int magnus = integ != PARAMENT_MIDPOINT;
    const unsigned cuda_mask = tc ? (unsigned)ctx->opt_batch_cuda_mask : 0u;
    ctx->last_batched = true;
    if (n == 0) return PARAMENT_OK;
    for (int i = 0; i < n; ++i) {
        const parament_instance &q = inst[i];
        if (q.dim < 1 || q.dim > kMaxBatchDim || q.n_ctrl < 0 || q.n_ctrl > kMaxControls || q.n_steps < 0 ||
            q.n_steps > (int64_t)0x7fffffff || !std::isfinite(q.dt))
            return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "instance %d: bad sizes", i);
        const int64_t S = samples_for(q.n_steps, integ);
        if (!q.H0 || !q.U_out || (q.n_ctrl > 0 && !q.Hk) || (q.n_ctrl > 0 && S > 0 && !q.c))
            return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "instance %d: null pointer", i);
        if (!is_device_ptr(q.H0) || !is_device_ptr(q.U_out) || (q.n_ctrl > 0 && !is_device_ptr(q.Hk)) ||
            (q.n_ctrl > 0 && S > 0 && !is_device_ptr(q.c)))
            return set_err(ctx, PARAMENT_ERR_INVALID_VALUE, "instance %d: batched calls take device pointers", i);
    }
    // the tensor-core kernel only when some instance's products run on the tensor cores: with
    // every class on the CUDA cores (the autotuner's choice for sweeps of d <= 64) the plain FP32
    // kernel runs the same products without the tensor-memory set-up
    bool needs_tc = false;
    for (int i = 0; i < n && tc; ++i) {
        const int cls = batch_tc_class(pad_dim(inst[i].dim));
        if (cls >= 0 && !((cuda_mask >> cls) & 1u)) needs_tc = true;
    }
    const int variant = (magnus ? 4 : 0) + (fp64 ? 3 : (needs_tc ? tc : 0));
    const int leaf_steps = ctx->opt_batch_leaf > 0 ? (int)ctx->opt_batch_leaf : 64;
    const int items_per_sm = ctx->opt_batch_items > 0 ? (int)ctx->opt_batch_items : 32;
    const size_t csz = fp64 ? 16 : 8, rsz = fp64 ? 8 : 4;

    std::vector<int64_t> key = {n, dtype, cdtype, integ, prec, leaf_steps, items_per_sm, (int64_t)cuda_mask};
    for (int i = 0; i < n; ++i) {
        key.push_back(inst[i].dim);
        key.push_back(inst[i].n_ctrl);
        key.push_back(inst[i].n_steps);
    }
    std::vector<int> Dp(n), nbs(n), nblk(n), warps_of(n, 8);
    std::vector<size_t> full_off(n), packed_off(n), norm_off(n), part_off(n), tick_off(n);
    if (key != ctx->bkey) {
        if (ctx->b_exec) {
            cudaGraphExecDestroy(ctx->b_exec);
            ctx->b_exec = nullptr;
        }
        ctx->bkey.clear();
        // cost model: d^3 N per instance; items sized to (total cost) / (items_per_sm * #SMs)
        double total = 0.0;
        for (int i = 0; i < n; ++i) {
            Dp[i] = pad_dim(inst[i].dim);
            nbs[i] = n_basis_for(inst[i].n_ctrl, integ);
            total += std::pow((double)Dp[i], 3) * std::max<int64_t>(inst[i].n_steps, 1);
        }
        const double target = total / std::max(1, items_per_sm * ctx->sm_count);
        size_t nf = 0, np = 0, nn = 0, npart = 0, ntick = 0;
        size_t smem = 0, stride = 0;
        int n_mats = 0;
        std::vector<BatchItem> items;
        std::vector<double> icost;
        for (int i = 0; i < n; ++i) {
            const int64_t N = inst[i].n_steps;
            const double cost = std::pow((double)Dp[i], 3) * std::max<int64_t>(N, 1);
            int64_t nb_cap;
            if (Dp[i] <= kMaxSmallDim) {
                int w = 8;
                while (w > 1 && fused_smem(Dp[i], fp64, nbs[i], w) > ctx->smem_optin) --w;
                warps_of[i] = w;
                nb_cap = std::max<int64_t>(1, N / ((int64_t)w * fused_gpw(Dp[i], fp64) * leaf_steps));
                smem = std::max(smem, fused_smem(Dp[i], fp64, nbs[i], w));
            } else {
                nb_cap = std::max<int64_t>(1, N / leaf_steps);
                const int cls = batch_tc_class(Dp[i]);
                const bool on_tc = tc && cls >= 0 && !((cuda_mask >> cls) & 1u);
                smem = std::max(smem, large_smem(Dp[i], fp64, nbs[i], on_tc ? tc : 0));
                stride = std::max(stride, (size_t)6 * Dp[i] * Dp[i] * csz);
            }
            nblk[i] = (int)std::min<int64_t>({nb_cap, (int64_t)std::ceil(cost / std::max(target, 1.0)), 1024});
            nblk[i] = std::max(nblk[i], 1);
            full_off[i] = nf;
            packed_off[i] = np;
            norm_off[i] = nn;
            part_off[i] = npart;
            tick_off[i] = ntick;
            nf += (size_t)nbs[i] * Dp[i] * Dp[i];
            np += (size_t)nbs[i] * Dp[i] * Dp[i];
            nn += nbs[i];
            npart += (size_t)nblk[i] * Dp[i] * Dp[i];
            ntick += 2 * (size_t)nblk[i] + 2;
            n_mats += nbs[i];
            for (int b = 0; b < nblk[i]; ++b) {
                items.push_back({i, b, nblk[i], Dp[i]});
                icost.push_back(cost / nblk[i]);
            }
        }
        if (smem > ctx->smem_optin)
            return set_err(ctx, PARAMENT_ERR_UNSUPPORTED, "batch needs %zu B shared memory per block", smem);
        std::vector<int> order(items.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return icost[a] > icost[b]; });
        std::vector<BatchItem> sorted(items.size());
        for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
        std::vector<int2> table;
        for (int i = 0; i < n; ++i)
            for (int e = 0; e < nbs[i]; ++e) table.push_back(make_int2(i, e));
        const int bps = batched_occupancy(variant, smem);
        if (bps <= 0) return set_err(ctx, PARAMENT_ERR_CUDA, "batched occupancy query failed (%zu B)", smem);
        const int grid = bps * ctx->sm_count;
        int st;
        if ((st = ws_reserve(ctx, ctx->bparams, (size_t)n * sizeof(FusedParams)))) return st;
        if ((st = ws_reserve(ctx, ctx->binsts, (size_t)n * sizeof(BatchInst)))) return st;
        if ((st = ws_reserve(ctx, ctx->btable, table.size() * sizeof(int2)))) return st;
        if ((st = ws_reserve(ctx, ctx->bitems, sorted.size() * sizeof(BatchItem)))) return st;
        if ((st = ws_reserve(ctx, ctx->bfull, nf * sizeof(double2)))) return st;
        if ((st = ws_reserve(ctx, ctx->bpacked, np * rsz))) return st;
        if ((st = ws_reserve(ctx, ctx->bnorms, nn * sizeof(double)))) return st;
        if ((st = ws_reserve(ctx, ctx->bpartials, npart * sizeof(double2)))) return st;
        if ((st = ws_reserve(ctx, ctx->btickets, ntick * sizeof(unsigned)))) return st;
        if ((st = ws_reserve(ctx, ctx->bcounters, (size_t)n * 8 * sizeof(unsigned long long)))) return st;
        if ((st = ws_reserve(ctx, ctx->bstatus, (size_t)n * 2 * sizeof(unsigned)))) return st;
        if ((st = ws_reserve(ctx, ctx->bqueue, 16))) return st;
        if ((st = ws_reserve(ctx, ctx->bscratch, std::max<size_t>(stride, 16) * grid))) return st;
        PM_CUDA(cudaMemcpy(ctx->btable.ptr, table.data(), table.size() * sizeof(int2), cudaMemcpyHostToDevice));
        PM_CUDA(cudaMemcpy(ctx->bitems.ptr, sorted.data(), sorted.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
        PM_CUDA(cudaMemset(ctx->btickets.ptr, 0, ntick * sizeof(unsigned)));
        PM_CUDA(cudaMemset(ctx->bcounters.ptr, 0, (size_t)n * 8 * sizeof(unsigned long long)));
        PM_CUDA(cudaMemset(ctx->bstatus.ptr, 0, (size_t)n * 2 * sizeof(unsigned)));
        ctx->b_n_items = (int)sorted.size();
        ctx->b_n_mats = n_mats;
        ctx->b_grid = grid;
        ctx->b_smem = smem;
        ctx->b_stride = std::max<size_t>(stride, 16);
        ctx->b_variant = variant;
        ctx->b_fp64 = fp64;
        ctx->b_c128 = dtype == PARAMENT_C128;
        ctx->b_magnus = magnus;
        ctx->b_ninst = n;
        ctx->b_nblk = nblk;
        ctx->b_warps = warps_of;
        ctx->bparams_up.clear();
        ctx->binsts_up.clear();
        ctx->bkey = key;
    } else {
        size_t nf = 0, np = 0, nn = 0, npart = 0, ntick = 0;
        for (int i = 0; i < n; ++i) {
            Dp[i] = pad_dim(inst[i].dim);
            nbs[i] = n_basis_for(inst[i].n_ctrl, integ);
            full_off[i] = nf;
            packed_off[i] = np;
            norm_off[i] = nn;
            part_off[i] = npart;
            tick_off[i] = ntick;
            nf += (size_t)nbs[i] * Dp[i] * Dp[i];
            np += (size_t)nbs[i] * Dp[i] * Dp[i];
            nn += nbs[i];
        }
    }

    // per-instance parameters (pointers may change between calls)
    const std::vector<int> &nblk_of = ctx->b_nblk;
    FusedParams base;
    std::memset(&base, 0, sizeof(base));
    build_classes(fp64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24), (int)ctx->opt_degree, base);
    std::vector<FusedParams> params(n, base);
    std::vector<BatchInst> insts(n);
    size_t npart = 0, ntick = 0;
    for (int i = 0; i < n; ++i) {
        const parament_instance &q = inst[i];
        FusedParams &p = params[i];
        p.ctrl = q.c;
        p.S = samples_for(q.n_steps, integ);
        p.n_steps = q.n_steps;
        p.K = q.n_ctrl;
        p.n_basis = nbs[i];
        p.n_coef = nbs[i];
        for (int e = 0; e < kMaxBasis; ++e) p.slot_of[e] = (short)(e < nbs[i] ? e : -1);
        p.d_out = q.dim;
        p.out_c128 = dtype == PARAMENT_C128;
        p.dt = q.dt;
        p.packed = (const char *)ctx->bpacked.ptr + packed_off[i] * rsz;
        p.bnorm1 = (const double *)ctx->bnorms.ptr + norm_off[i];
        p.partials = (double2 *)ctx->bpartials.ptr + npart;
        p.tickets = (unsigned *)ctx->btickets.ptr + ntick;
        p.U_out = q.U_out;
        p.counters = (unsigned long long *)ctx->bcounters.ptr + (size_t)i * 8;
        p.status = (unsigned *)ctx->bstatus.ptr + (size_t)i * 2;
        p.extra_squarings = (int)ctx->opt_extra_sq;
        p.unitary_step = fp64 ? 0 : (int)ctx->opt_unitary_step;
        p.warps = ctx->b_warps[i];
        {
            const int cls = batch_tc_class(Dp[i]);
            p.tc_off = (cls >= 0 && ((cuda_mask >> cls) & 1u)) ? 1 : 0;
        }
        npart += (size_t)nblk_of[i] * Dp[i] * Dp[i];
        ntick += 2 * (size_t)nblk_of[i] + 2;
        insts[i] = BatchInst{q.H0, q.Hk, q.dim, Dp[i], q.n_ctrl, nbs[i], full_off[i], packed_off[i], norm_off[i]};
    }
    if (ctx->bparams_up.size() != params.size() ||
        std::memcmp(ctx->bparams_up.data(), params.data(), params.size() * sizeof(FusedParams)) != 0) {
        PM_CUDA(cudaMemcpyAsync(ctx->bparams.ptr, params.data(), params.size() * sizeof(FusedParams),
                                cudaMemcpyHostToDevice, ctx->stream));
        ctx->bparams_up = params;
    }
    if (ctx->binsts_up.size() != insts.size() ||
        std::memcmp(ctx->binsts_up.data(), insts.data(), insts.size() * sizeof(BatchInst)) != 0) {
        PM_CUDA(cudaMemcpyAsync(ctx->binsts.ptr, insts.data(), insts.size() * sizeof(BatchInst),
                                cudaMemcpyHostToDevice, ctx->stream));
        ctx->binsts_up = insts;
    }

    auto enqueue = [&]() -> cudaError_t {
        cudaError_t e = batch_basis_launch(ctx->b_c128, ctx->b_fp64, (const BatchInst *)ctx->binsts.ptr,
                                           (const int2 *)ctx->btable.ptr, ctx->b_n_mats, ctx->b_magnus,
                                           (double2 *)ctx->bfull.ptr, ctx->bpacked.ptr, (double *)ctx->bnorms.ptr,
                                           ctx->stream);
        if (e != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(ctx->bqueue.ptr, 0, sizeof(unsigned), ctx->stream)) != cudaSuccess) return e;
        // the kernel-wide status word (bounded tensor-core waits) is the one parament_get_stats reads
        unsigned *kstatus = (unsigned *)ctx->status.ptr + 1;
        if ((e = cudaMemsetAsync(kstatus, 0, sizeof(unsigned), ctx->stream)) != cudaSuccess) return e;
        return batched_launch(ctx->b_variant, (const BatchItem *)ctx->bitems.ptr, ctx->b_n_items,
                              (unsigned *)ctx->bqueue.ptr, (const FusedParams *)ctx->bparams.ptr,
                              (unsigned char *)ctx->bscratch.ptr, ctx->b_stride, ctx->b_grid, ctx->b_smem, kstatus,
                              ctx->stream);
    };
    if (ctx->opt_batch_graph && ctx->stream != nullptr) {
        if (!ctx->b_exec) {
            cudaGraph_t graph = nullptr;
            PM_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = enqueue();
            cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &graph);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                return set_err(ctx, PARAMENT_ERR_CUDA, "graph capture failed: %s",
                               cudaGetErrorString(e != cudaSuccess ? e : e2));
            }
            cudaError_t e3 = cudaGraphInstantiate(&ctx->b_exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e3 != cudaSuccess) {
                ctx->b_exec = nullptr;
                cudaGetLastError();
                return set_err(ctx, PARAMENT_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e3));
            }
        }
        PM_CUDA(cudaGraphLaunch(ctx->b_exec, ctx->stream));
    } else {
        PM_CUDA(enqueue());
    }
    int64_t tot = 0;
    unsigned backends = 0;
    for (int i = 0; i < n; ++i) {
        tot += inst[i].n_steps;
        backends |= batch_backend(pad_dim(inst[i].dim), fp64, tc, cuda_mask);
    }
    ctx->last = parament_stats{};
    ctx->last.n_steps = tot;
    ctx->last.product_backends = backends;
    ctx->last.grid_blocks = ctx->b_grid;
    ctx->last.block_threads = 256;
    ctx->last.leaves = ctx->b_n_items;
    ctx->last.kernel_ms = -1.0;
    return PARAMENT_OK;
}

}  // namespace

extern "C" {

int parament_propagate_batched(parament_ctx *ctx, const parament_instance *inst, int n_inst, parament_dtype dtype,
                               parament_real_dtype cdtype, parament_integrator integrator, parament_precision prec) {
    if (!ctx) return PARAMENT_ERR_INVALID_VALUE;
    ctx->err.clear();
    DeviceGuard guard(ctx->device);
    return batch_run(ctx, inst, n_inst, dtype, cdtype, integrator, prec);
}

int parament_batch_autotune(parament_ctx *ctx, const parament_instance *inst, int n_inst, parament_dtype dtype,
                            parament_real_dtype cdtype, parament_integrator integrator, parament_precision prec,
                            int *best_leaf_steps, int *best_items_per_sm, double *best_ms,
                            unsigned *cuda_core_classes) {
    if (!ctx) return PARAMENT_ERR_INVALID_VALUE;
    ctx->err.clear();
    DeviceGuard guard(ctx->device);
    const bool tc = prec == PARAMENT_PREC_FP32_TC_TF32X3 || prec == PARAMENT_PREC_FP32_TC_BF16X3;
    unsigned present = 0;  // dimension classes with a tensor-core body in this batch
    for (int i = 0; tc && i < n_inst && inst; ++i) {
        const int cls = batch_tc_class(pad_dim(inst[i].dim));
        if (cls >= 0) present |= 1u << cls;
    }
    cudaEvent_t a, b;
    PM_CUDA(cudaEventCreate(&a));
    PM_CUDA(cudaEventCreate(&b));
    int st = PARAMENT_OK;
    // one configuration: a warm-up run (which also builds the plan), then the mean of two timed runs
    auto time_cfg = [&](int l, int it, unsigned mask, double *ms_out) -> int {
        ctx->opt_batch_leaf = l;
        ctx->opt_batch_items = it;
        ctx->opt_batch_cuda_mask = mask;
        int s2 = batch_run(ctx, inst, n_inst, dtype, cdtype, integrator, prec);
        float ms_sum = 0.f;
        for (int r = 0; r < 2 && s2 == PARAMENT_OK; ++r) {
            cudaEventRecord(a, ctx->stream);
            s2 = batch_run(ctx, inst, n_inst, dtype, cdtype, integrator, prec);
            cudaEventRecord(b, ctx->stream);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            ms_sum += ms;
        }
        *ms_out = ms_sum / 2.0;
        return s2;
    };
    const int leafs[] = {32, 128}, items[] = {8, 16, 32, 64};
    double best = 1e300;
    int bl = 128, bi = 32;
    unsigned bm = 0;
    // (1) the work split with every class on the tensor cores (or the CUDA cores for FP32 / FP64)
    auto tune_split = [&](unsigned mask) {
        for (int l : leafs)
            for (int it : items) {
                double ms = 0.0;
                if ((st = time_cfg(l, it, mask, &ms))) return;
                if (ms < best) {
                    best = ms;
                    bl = l;
                    bi = it;
                    bm = mask;
                }
            }
    };
    tune_split(0u);
    // (2) per dimension class: tensor cores or CUDA cores, every subset of the classes present
    if (!st && present) {
        const unsigned split_mask = bm;
        for (unsigned m = 1; m <= 7 && !st; ++m) {
            if ((m & ~present) != 0u) continue;
            double ms = 0.0;
            if ((st = time_cfg(bl, bi, m, &ms))) break;
            if (ms < best) {
                best = ms;
                bm = m;
            }
        }
        // (3) the split again for the chosen back-ends
        if (!st && bm != split_mask) tune_split(bm);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st) return st;
    ctx->opt_batch_leaf = bl;
    ctx->opt_batch_items = bi;
    ctx->opt_batch_cuda_mask = bm;
    if (best_leaf_steps) *best_leaf_steps = bl;
    if (best_items_per_sm) *best_items_per_sm = bi;
    if (best_ms) *best_ms = best;
    if (cuda_core_classes) *cuda_core_classes = bm;
    return PARAMENT_OK;
}

}  // extern "C"
