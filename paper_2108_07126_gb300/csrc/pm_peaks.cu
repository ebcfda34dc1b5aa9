// Measured peaks of the pipes the propagator runs on (parament_measure_peaks): FP32 and FP64
// fused multiply-adds on the CUDA cores and dense TF32 / BF16 MMAs on the tcgen05 tensor cores.
// The benchmark divides its achieved rates by these instead of by unit counts and nominal ratios.
//
// FMA: every thread runs 4, 8 or 16 independent multiply-add chains over 1, 2 or 4 blocks of 512
// threads per SM; the best of these shapes is the pipe's rate (flops = 2 x multiply-adds), both
// event-timed and per SM clock cycle (scaled to the maximum SM clock).  Tensor: one block per SM, one thread issues a long stream of M = 128, N = 256 MMAs on
// zero operands in shared memory (TF32: K = 8, BF16: K = 16) into one tensor-memory accumulator and
// waits for the last one with a bounded wait; flops = 2 x M x N x K x MMAs x SMs.  Times are CUDA
// events around each launch on the given stream (median of three after a warm-up launch).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "../../include/parament.h"
#include "pm_umma.cuh"

namespace {

template <typename T, int CH>
__global__ void __launch_bounds__(512) fma_kernel(int iters, T a, T b, T *sink, unsigned long long *cycles) {
    const long long t0 = clock64();
    T x[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = (T)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int i = 0; i < CH; ++i) x[i] = fma(x[i], a, b);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += x[i];
    if (s == (T)-1.2345) sink[blockIdx.x] = s;  // keeps the chains live; never true for these inputs
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(cycles, (unsigned long long)(clock64() - t0));
}

template <int F>
__global__ void __launch_bounds__(128, 1) mma_kernel(int n_mma, unsigned *status) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    for (int i = threadIdx.x; i < 32768 / 16; i += blockDim.x) reinterpret_cast<float4 *>(sm)[i] = make_float4(0, 0, 0, 0);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(pm::umma::smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n" ::"r"(
                         pm::umma::smem_u32(&tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    pm::umma::fence_before();
    __syncthreads();
    pm::umma::fence_after();
    const uint32_t tm = tslot;
    if (threadIdx.x == 0) {
        // K-major, no swizzle: 16-byte core-matrix rows, k groups 128 B apart, 8-row groups 256 B
        // apart; A (128 rows) at 0, B (256 rows) at 8 KB, both inside the 32 KB of zeros
        const uint32_t a = pm::umma::smem_u32(sm), b = a + 8192;
        auto desc = [](uint32_t addr) {
            return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
                   ((uint64_t)1 << 46);
        };
        const uint32_t id = pm::umma::idesc<F>(false, 256);
        for (int i = 0; i < n_mma; ++i) pm::umma::mma<F>(tm, desc(a), desc(b), id, i > 0 ? 1u : 0u);
        pm::umma::commit(&bar);
        if (!pm::umma::wait(&bar, 0)) atomicOr(status, 1u);
    }
    pm::umma::fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tm) : "memory");
}

// median of three event-timed launches after one warm-up launch, in ms
template <typename L>
cudaError_t time_ms(L launch, cudaStream_t st, double *ms) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) return e;
    float t[3] = {0.f, 0.f, 0.f};
    launch();
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
        cudaEventRecord(a, st);
        launch();
        cudaEventRecord(b, st);
        e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t[r], a, b);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::sort(t, t + 3);
    *ms = t[1];
    return e;
}

// Best rate over chain counts 4, 8, 16 and 1, 2, 4 blocks of 512 threads per SM (the same
// multiply-adds per thread for every shape).  *best: event-timed TFLOP/s at the clock the GPU ran;
// *best_clk: flops per SM clock cycle (the longest block's clock64 count, all blocks resident at
// once) times the maximum SM clock -- the rate at the clock the timed kernels run at.
template <typename T>
cudaError_t fma_peak(int sms, int iters, T *sink, unsigned long long *cyc, double clk_hz, cudaStream_t st,
                     double *best, double *best_clk) {
    cudaError_t e = cudaSuccess;
    *best = *best_clk = 0.0;
    for (int bps = 1; bps <= 4 && e == cudaSuccess; bps *= 2) {
        const int blocks = bps * sms;
        const double flops = 2.0 * 8 * 16.0 * iters * (double)blocks * 512;
        auto one = [&](auto kern, int it) -> cudaError_t {
            double ms = 0.0;
            cudaError_t e2 = time_ms([&] { kern<<<blocks, 512, 0, st>>>(it, (T)0.999, (T)1e-3, sink, cyc); }, st, &ms);
            if (e2 != cudaSuccess) return e2;
            unsigned long long c = 0;
            e2 = cudaMemsetAsync(cyc, 0, sizeof(c), st);  // one more launch for the cycle count alone
            if (e2 == cudaSuccess) {
                kern<<<blocks, 512, 0, st>>>(it, (T)0.999, (T)1e-3, sink, cyc);
                e2 = cudaMemcpyAsync(&c, cyc, sizeof(c), cudaMemcpyDeviceToHost, st);
            }
            if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
            if (e2 != cudaSuccess) return e2;
            *best = std::max(*best, flops / (ms * 1e-3) / 1e12);
            if (c > 0) *best_clk = std::max(*best_clk, flops / (double)c * clk_hz / 1e12);
            return cudaSuccess;
        };
        e = one(fma_kernel<T, 4>, iters * 2);
        if (e == cudaSuccess) e = one(fma_kernel<T, 8>, iters);
        if (e == cudaSuccess) e = one(fma_kernel<T, 16>, iters / 2);
    }
    return e;
}

}  // namespace

extern "C" int parament_measure_peaks(int device, void *cuda_stream, parament_peaks *out) {
    if (!out) return PARAMENT_ERR_INVALID_VALUE;
    std::memset(out, 0, sizeof(*out));
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return PARAMENT_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int sms = 0, clk_khz = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, device);
    void *sink = nullptr;
    unsigned *status = nullptr;
    unsigned long long *cyc = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync(&sink, 4096 * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&cyc, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&status, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(unsigned), st);
    double ms = 0.0;
    const double clk_hz = clk_khz * 1e3;
    if (e == cudaSuccess)
        e = fma_peak<float>(sms, 128, (float *)sink, cyc, clk_hz, st, &out->fp32_tflops, &out->fp32_tflops_max_clock);
    if (e == cudaSuccess)
        e = fma_peak<double>(sms, 16, (double *)sink, cyc, clk_hz, st, &out->fp64_tflops, &out->fp64_tflops_max_clock);
    const int n_mma = 8192;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(mma_kernel<pm::umma::kTF32x3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 32768);
    if (e == cudaSuccess) {
        e = time_ms([&] { mma_kernel<pm::umma::kTF32x3><<<sms, 128, 32768, st>>>(n_mma, status); }, st, &ms);
        out->tf32_tflops = 2.0 * 128 * 256 * 8 * (double)n_mma * sms / (ms * 1e-3) / 1e12;
    }
    if (e == cudaSuccess) e = cudaFuncSetAttribute(mma_kernel<pm::umma::kBF16x3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 32768);
    if (e == cudaSuccess) {
        e = time_ms([&] { mma_kernel<pm::umma::kBF16x3><<<sms, 128, 32768, st>>>(n_mma, status); }, st, &ms);
        out->bf16_tflops = 2.0 * 128 * 256 * 16 * (double)n_mma * sms / (ms * 1e-3) / 1e12;
    }
    unsigned stv = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&stv, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (sink) cudaFreeAsync(sink, st);
    if (status) cudaFreeAsync(status, st);
    if (cyc) cudaFreeAsync(cyc, st);
    cudaStreamSynchronize(st);
    out->sm_count = sms;
    out->max_sm_clock_mhz = clk_khz / 1000.0;
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PARAMENT_ERR_CUDA;
    }
    return stv ? PARAMENT_ERR_TIMEOUT : PARAMENT_OK;
}
