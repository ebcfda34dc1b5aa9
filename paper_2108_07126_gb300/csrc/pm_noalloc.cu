// parament_propagate_noalloc: one propagation that allocates no memory.
//
// For callers that cannot call cudaMalloc: an application or framework that
// owns every byte of device memory through its own allocator, or a
// latency-critical loop that cannot afford the device-wide synchronisation
// that cudaMalloc / cudaFree imply.  The caller passes device inputs and the
// output buffer; every intermediate (staged Hamiltonians, the basis, the
// block partial products, the tree-arrival counters, statistics and status
// words) lives in the file-scope array below, which each GPU that loads the
// library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/parament.h"
#include "pm_internal.h"

namespace {

constexpr int kNaMaxDim = PARAMENT_NOALLOC_MAX_DIM;
constexpr int kNaMaxBasis = PARAMENT_NOALLOC_MAX_BASIS;
constexpr int kNaMaxBlocks = PARAMENT_NOALLOC_MAX_BLOCKS;
constexpr size_t kMat = (size_t)kNaMaxDim * kNaMaxDim;  // entries of one padded matrix

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// byte offsets of the regions inside the scratch array
constexpr size_t kOffRaw = 0;                                                    // [1 + K][d][d] inputs
constexpr size_t kOffFull = kOffRaw + align256((1 + pm::kMaxControls) * kMat * 16);
constexpr size_t kOffP64 = kOffFull + align256(kNaMaxBasis * kMat * 16);
constexpr size_t kOffP32 = kOffP64 + align256(kNaMaxBasis * kMat * 8);
constexpr size_t kOffNorm = kOffP32 + align256(kNaMaxBasis * kMat * 4);
constexpr size_t kOffMax = kOffNorm + align256(kNaMaxBasis * 8);
constexpr size_t kOffPart = kOffMax + align256(kNaMaxBasis * 8);
constexpr size_t kOffTick = kOffPart + align256(kNaMaxBlocks * kMat * 16);
constexpr size_t kOffCnt = kOffTick + align256(2 * kNaMaxBlocks * 4);
constexpr size_t kOffStat = kOffCnt + align256(8 * 8);
constexpr size_t kScratchBytes = kOffStat + align256(2 * 4);
static_assert(kScratchBytes == PARAMENT_NOALLOC_SCRATCH_BYTES, "header and scratch layout disagree");

// Shared by every call on a device; holds the latest call's contents.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char *g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device:
// in host code the symbol itself is only a host-side stand-in).
int scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return PARAMENT_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return PARAMENT_ERR_CUDA;
        }
        g_addr[dev] = (unsigned char *)p;
    }
    *out = g_addr[dev];
    return PARAMENT_OK;
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int parament_propagate_noalloc(int dim, int n_ctrl, const void *H0, const void *Hk, parament_dtype dtype,
                                          parament_integrator integrator, const void *c,
                                          parament_real_dtype cdtype, int64_t n_steps, double dt, void *U_out,
                                          parament_precision prec, void *cuda_stream, uint32_t *device_status) {
    if (dim < 1 || n_ctrl < 0 || n_ctrl > pm::kMaxControls) return PARAMENT_ERR_INVALID_VALUE;
    if (dim > kNaMaxDim) return PARAMENT_ERR_UNSUPPORTED;
    if (dtype != PARAMENT_C64 && dtype != PARAMENT_C128) return PARAMENT_ERR_INVALID_VALUE;
    if (cdtype != PARAMENT_F32 && cdtype != PARAMENT_F64) return PARAMENT_ERR_INVALID_VALUE;
    if (integrator != PARAMENT_MIDPOINT && integrator != PARAMENT_MAGNUS4_GL2 &&
        integrator != PARAMENT_MAGNUS4_SIMPSON)
        return PARAMENT_ERR_INVALID_VALUE;
    if (prec != PARAMENT_PREC_FP64 && prec != PARAMENT_PREC_FP32) return PARAMENT_ERR_UNSUPPORTED;
    const int fp64 = prec == PARAMENT_PREC_FP64;
    if ((cdtype == PARAMENT_F64) != (fp64 != 0)) return PARAMENT_ERR_INVALID_VALUE;  // no conversion buffer
    if (n_steps < 0 || n_steps > (int64_t)0x7fffffff) return PARAMENT_ERR_INVALID_VALUE;
    if (!std::isfinite(dt)) return PARAMENT_ERR_NONFINITE;
    const int magnus = integrator != PARAMENT_MIDPOINT;
    const int nb = magnus ? 1 + 2 * n_ctrl + n_ctrl * (n_ctrl - 1) / 2 : 1 + n_ctrl;
    if (nb > kNaMaxBasis) return PARAMENT_ERR_UNSUPPORTED;
    const int64_t S = integrator == PARAMENT_MIDPOINT ? n_steps
                      : (integrator == PARAMENT_MAGNUS4_GL2 ? 2 * n_steps : 2 * n_steps + 1);
    const bool need_c = n_ctrl > 0 && S > 0;
    if (!H0 || !U_out || (n_ctrl > 0 && !Hk) || (need_c && !c)) return PARAMENT_ERR_INVALID_VALUE;
    if (!on_device(H0) || !on_device(U_out) || (n_ctrl > 0 && !on_device(Hk)) || (need_c && !on_device(c)))
        return PARAMENT_ERR_INVALID_VALUE;
    // the kernel stores U as float2 / double2 and reads c as float / double: misaligned pointers
    // would fault in the kernel, so they are refused here
    const size_t esz_u = dtype == PARAMENT_C128 ? 16 : 8, esz_c = fp64 ? 8 : 4;
    if ((uintptr_t)U_out % esz_u != 0 || (need_c && (uintptr_t)c % esz_c != 0)) return PARAMENT_ERR_INVALID_VALUE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PARAMENT_ERR_CUDA;
    }
    unsigned char *base = nullptr;
    int st = scratch_address(dev, &base);
    if (st != PARAMENT_OK) return st;
    int sms = 0, optin = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return PARAMENT_ERR_CUDA;
    }
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const int Dp = dim <= 2 ? 2 : (dim <= 4 ? 4 : (dim <= 8 ? 8 : 16));
    const size_t DD = (size_t)Dp * Dp;
    const size_t esz = dtype == PARAMENT_C128 ? 16 : 8;
    const size_t mat = (size_t)dim * dim * esz;

#define NA_CUDA(call)                     \
    do {                                  \
        if ((call) != cudaSuccess) {      \
            cudaGetLastError();           \
            return PARAMENT_ERR_CUDA;     \
        }                                 \
    } while (0)

    // stage H0 and H_k contiguously, then the basis (no pruning, no Hermiticity check)
    NA_CUDA(cudaMemcpyAsync(base + kOffRaw, H0, mat, cudaMemcpyDeviceToDevice, stream));
    if (n_ctrl > 0) NA_CUDA(cudaMemcpyAsync(base + kOffRaw + mat, Hk, mat * n_ctrl, cudaMemcpyDeviceToDevice, stream));
    NA_CUDA(pm::basis_build(base + kOffRaw, dtype == PARAMENT_C128, dim, Dp, n_ctrl, magnus, nb,
                            (double2 *)(base + kOffFull), (double *)(base + kOffP64), (float *)(base + kOffP32),
                            (double *)(base + kOffNorm), (double *)(base + kOffMax), stream));
    // arrival counters, statistics and status must start at zero
    NA_CUDA(cudaMemsetAsync(base + kOffTick, 0, kScratchBytes - kOffTick, stream));

    pm::FusedParams p;
    std::memset(&p, 0, sizeof(p));
    const double u = fp64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
    if (pm::fill_classes(u, 0, p) <= 0) return PARAMENT_ERR_INVALID_VALUE;

    int warps = 8;
    while (warps > 1 && pm::fused_smem_size(Dp, fp64, nb, warps) > (size_t)optin) --warps;
    const size_t smem = pm::fused_smem_size(Dp, fp64, nb, warps);
    if (smem > (size_t)optin) return PARAMENT_ERR_UNSUPPORTED;
    const int bps = pm::fused_occupancy(Dp, fp64, (int)integrator, warps, smem);
    if (bps <= 0) return PARAMENT_ERR_CUDA;
    const int64_t per_block = (int64_t)warps * pm::fused_groups(Dp, fp64) * 8;
    int64_t grid = (n_steps + per_block - 1) / per_block;
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, std::min<int64_t>((int64_t)bps * sms, kNaMaxBlocks)));

    p.ctrl = c;
    p.S = S;
    p.n_steps = n_steps;
    p.K = n_ctrl;
    p.n_basis = nb;
    p.n_coef = nb;
    for (int e = 0; e < pm::kMaxBasis; ++e) p.slot_of[e] = (short)(e < nb ? e : -1);
    p.d_out = dim;
    p.out_c128 = dtype == PARAMENT_C128;
    p.dt = dt;
    p.packed = fp64 ? (const void *)(base + kOffP64) : (const void *)(base + kOffP32);
    p.bnorm1 = (const double *)(base + kOffNorm);
    p.partials = (double2 *)(base + kOffPart);
    p.tickets = (unsigned *)(base + kOffTick);
    p.U_out = U_out;
    p.counters = (unsigned long long *)(base + kOffCnt);
    p.status = (unsigned *)(base + kOffStat);
    p.extra_squarings = 0;
    p.unitary_step = fp64 ? 0 : 1;  // as parament_propagate with its default options
    NA_CUDA(pm::fused_launch(Dp, fp64, (int)integrator, p, (int)grid, warps, smem, stream));
    if (device_status) {
        // the root of the product tree moved the status bits of this call to the second word
        NA_CUDA(cudaMemcpyAsync(device_status, base + kOffStat + sizeof(unsigned), sizeof(unsigned),
                                cudaMemcpyDeviceToHost, stream));
        NA_CUDA(cudaStreamSynchronize(stream));
    }
#undef NA_CUDA
    (void)DD;
    return PARAMENT_OK;
}
