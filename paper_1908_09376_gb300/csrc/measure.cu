// Measured arithmetic rates of the current GPU, for the roofline of the
// kernels bound by arithmetic rather than memory (the middle factor made on
// the fly: one sine, one cosine and, for the FIO phases, one reciprocal
// square root per entry on the SFU, and about twenty FP32 FMA-pipe
// operations; the plain FP64 form, bound by FP64 FMAs).  Throughput loops,
// timed with CUDA events:
//   - FP32 and FP64 FMA: eight independent fused multiply-add chains per thread;
//   - SFU: eight independent chains of rsqrt.approx per thread (one SFU
//     operation each; the add that keeps the chains finite runs on the FMA
//     pipe, which has four times the rate).
// The grid is eight CTAs of 256 threads per SM, so every SM is full.
#include <cuda_runtime.h>

#include "internal.hpp"

#define MCK(call)                                                                                    \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) midbf::fail(MIDBF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fma_rate(float* out, int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = (float)(threadIdx.x + q) * 1e-3f;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int q = 0; q < kChains; ++q) a[q] = fmaf(a[q], b, c);
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += a[q];
    if (s == 12345.0f) out[blockIdx.x] = s;   // keeps the chains alive; never true for these inputs
}

__global__ void __launch_bounds__(256) k_dfma_rate(double* out, int iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = (double)(threadIdx.x + q) * 1e-3;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int q = 0; q < kChains; ++q) a[q] = fma(a[q], b, c);
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += a[q];
    if (s == 12345.0) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_sfu_rate(float* out, int iters, float c) {
    float a[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = 1.0f + (float)(threadIdx.x + q) * 1e-3f;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int q = 0; q < kChains; ++q) {
            float y;
            asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[q]));
            a[q] = y + c;   // stays in [c, c + 1] for c >= 1
        }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += a[q];
    if (s == 12345.0f) out[blockIdx.x] = s;
}

}  // namespace

extern "C" int midbf_pipe_rates(void* stream, double* fma_per_s, double* sfu_per_s, double* dfma_per_s) {
    float* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MIDBF_OK;
    try {
        if (!fma_per_s || !sfu_per_s) midbf::fail(MIDBF_EINVAL, "null argument");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        int dev = 0, nsm = 0;
        MCK(cudaGetDevice(&dev));
        MCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const int grid = 8 * nsm, threads = 256;
        MCK(cudaMalloc(&out, grid * sizeof(double)));
        MCK(cudaEventCreate(&e0));
        MCK(cudaEventCreate(&e1));
        auto time = [&](auto launch) {
            launch();   // warm-up
            float best = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                MCK(cudaEventRecord(e0, s));
                launch();
                MCK(cudaEventRecord(e1, s));
                MCK(cudaEventSynchronize(e1));
                float ms = 0.f;
                MCK(cudaEventElapsedTime(&ms, e0, e1));
                best = std::min(best, ms);
            }
            return (double)best * 1e-3;
        };
        const int it_fma = 4096, it_sfu = 1024;
        const double t_fma = time([&] { k_fma_rate<<<grid, threads, 0, s>>>(out, it_fma, 0.999f, 1e-3f); });
        MCK(cudaGetLastError());
        const double t_sfu = time([&] { k_sfu_rate<<<grid, threads, 0, s>>>(out, it_sfu, 1.0f); });
        MCK(cudaGetLastError());
        const int it_dfma = 256;
        const double t_dfma =
            time([&] { k_dfma_rate<<<grid, threads, 0, s>>>(reinterpret_cast<double*>(out), it_dfma, 0.999, 1e-3); });
        MCK(cudaGetLastError());
        const double n = (double)grid * threads * kChains;
        *fma_per_s = n * it_fma / t_fma;
        *sfu_per_s = n * it_sfu / t_sfu;
        if (dfma_per_s) *dfma_per_s = n * it_dfma / t_dfma;
    } catch (const midbf::Error& e) {
        midbf::set_last_error(e.what());
        rc = e.code;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    return rc;
}
