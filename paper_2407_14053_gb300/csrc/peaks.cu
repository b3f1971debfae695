// Throughput microbenchmarks of the two arithmetic pipes the compositing
// kernels lean on: FP32 fused multiply-add (scalar and packed FP32x2) and
// the ex2 approximation of the special-function unit.  The benchmark's
// roofline divides the compositing stage's algorithmic FLOPs and ex2 counts
// by these measured rates.  No counterpart in the paper.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/directl.h"
#include "dl_internal.cuh"

namespace dl {
namespace {

constexpr int kChains = 8;     // independent dependency chains per thread
constexpr int kPeakThreads = 256;

// kChains independent FMA chains of `iters` steps each: 2 * kChains * iters
// FLOP per thread.  The result is stored only when it equals an impossible
// sentinel, so the chains cannot be removed.
__global__ void __launch_bounds__(kPeakThreads) fma_kernel(float seed, int iters, float* sink) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + float(threadIdx.x + c);
    const float m = 0.999999f, k = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, k);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == -1.2345f) sink[threadIdx.x] = s;
}

// The same with packed FP32x2 FMAs: 4 * kChains * iters FLOP per thread.
__global__ void __launch_bounds__(kPeakThreads) fma2_kernel(float seed, int iters, float* sink) {
    float2 a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = make_float2(seed + float(c), seed - float(threadIdx.x));
    const float2 m = make_float2(0.999999f, 0.999998f), k = make_float2(1e-7f, 2e-7f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = __ffma2_rn(a[c], m, k);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c].x + a[c].y;
    if (s == -1.2345f) sink[threadIdx.x] = s;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// kChains independent chains y <- 2^y - 1.5 (values stay in (-1.5, 0.5]):
// kChains * iters ex2 per thread (and as many adds, on the FMA pipe).
__global__ void __launch_bounds__(kPeakThreads) ex2_kernel(float seed, int iters, float* sink) {
    float y[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) y[c] = seed - 0.01f * float(c + (threadIdx.x & 7));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) y[c] = ex2_approx(y[c]) - 1.5f;
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += y[c];
    if (s == -1.2345f) sink[threadIdx.x] = s;
}

template <class K>
cudaError_t time_kernel(K kernel, int blocks, int iters, float* sink, cudaStream_t s, float* ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        kernel<<<blocks, kPeakThreads, 0, s>>>(-0.25f, iters, sink);  // warm-up
        e = cudaGetLastError();
    }
    float best = 1e30f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) {
            kernel<<<blocks, kPeakThreads, 0, s>>>(-0.25f, iters, sink);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess) best = std::min(best, t);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *ms = best;
    return e;
}

}  // namespace
}  // namespace dl

extern "C" dl_status dl_measure_peaks(int32_t device, double* fp32_tflops, double* fp32x2_tflops,
                                      double* ex2_per_s) {
    using namespace dl;
    if (!fp32_tflops || !fp32x2_tflops || !ex2_per_s) return DL_ERR_INVALID_ARG;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return DL_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return DL_ERR_CUDA;
    }
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, device) != cudaSuccess) {
        cudaGetLastError();
        return DL_ERR_CUDA;
    }
    // every SM filled with resident threads, several waves of work each
    const int blocks = sms * std::max(1, per_sm / kPeakThreads) * 4;
    const double threads = double(blocks) * kPeakThreads;
    float* sink = nullptr;
    if (cudaMalloc(&sink, kPeakThreads * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return DL_ERR_OOM;
    }
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    float ms = 0.f;
    const int it_fma = 4096, it_ex2 = 1024;
    if (e == cudaSuccess) e = time_kernel(fma_kernel, blocks, it_fma, sink, s, &ms);
    if (e == cudaSuccess) *fp32_tflops = threads * 2.0 * kChains * it_fma / (ms * 1e-3) / 1e12;
    if (e == cudaSuccess) e = time_kernel(fma2_kernel, blocks, it_fma, sink, s, &ms);
    if (e == cudaSuccess) *fp32x2_tflops = threads * 4.0 * kChains * it_fma / (ms * 1e-3) / 1e12;
    if (e == cudaSuccess) e = time_kernel(ex2_kernel, blocks, it_ex2, sink, s, &ms);
    if (e == cudaSuccess) *ex2_per_s = threads * double(kChains) * it_ex2 / (ms * 1e-3);
    if (s) cudaStreamDestroy(s);
    cudaFree(sink);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return DL_ERR_CUDA;
    }
    return DL_OK;
}
