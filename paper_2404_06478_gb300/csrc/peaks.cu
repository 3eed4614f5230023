// peaks.cu — throughput microbenchmarks of the arithmetic pipes the pair
// passes use (FP32 FMA, packed f32x2 FMA, MUFU ex2 / rsqrt / lg2), so that
// the roofline of the ALU-bound kernels is measured on the device instead of
// assumed.  Each kernel runs many independent dependency chains per thread at
// full occupancy; results are operations per second (one FMA = one op).
#include "api_internal.h"

namespace laue {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kPeakThreads) peak_ffma(float* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int k = 0; k < iters; ++k)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.f) out[0] = s;
}

__global__ void __launch_bounds__(kPeakThreads) peak_ffma2(float* out, int iters, float a, float b) {
    unsigned long long x[kChains], A, B;
    asm("mov.b64 %0, {%1, %1};" : "=l"(A) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(B) : "f"(b));
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float v = threadIdx.x * 1e-3f + c;
        asm("mov.b64 %0, {%1, %1};" : "=l"(x[c]) : "f"(v));
    }
    for (int k = 0; k < iters; ++k)
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(A), "l"(B));
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == 12345.f) out[0] = s;
}

template <int OP>
__global__ void __launch_bounds__(kPeakThreads) peak_mufu(float* out, int iters) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.5f + threadIdx.x * 1e-4f + c * 1e-2f;
    for (int k = 0; k < iters; ++k)
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (OP == 0) x[c] = ex2(-x[c]);          // stays in (0.25, 1)
            if (OP == 1) x[c] = rsq(x[c]);           // fixed point 1
            if (OP == 2) x[c] = lg2(x[c] + 2.0f);    // one extra FADD per op
        }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.f) out[0] = s;
}

}  // namespace laue

using namespace laue;

// out_host[0..4] = FFMA, f32x2 FMA (counted as 2 ops), ex2, rsqrt, lg2 ops per
// second; out_host[5] = SM count.  Needs >= 4 bytes of workspace.
extern "C" int laue_alu_peaks(laue_handle* h, double* out_host, void* stream) {
    if (!h || !out_host) return LAUE_ERR_INVALID_ARG;
    if (!h->ws) return laue_fail(h, LAUE_ERR_WORKSPACE, "no workspace set");
    cudaStream_t s = (cudaStream_t)stream;
    float* sink = (float*)((char*)h->ws + 64);
    int blocks = h->sm_count * 8;
    double threads = (double)blocks * kPeakThreads;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto timed = [&](auto launch, double ops) {
        launch();  // warm-up
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ops / (ms * 1e-3);
    };
    const int it = 4096;
    out_host[0] = timed([&] { peak_ffma<<<blocks, kPeakThreads, 0, s>>>(sink, it, 0.9999f, 1e-4f); },
                        threads * it * kChains);
    out_host[1] = timed([&] { peak_ffma2<<<blocks, kPeakThreads, 0, s>>>(sink, it, 0.9999f, 1e-4f); },
                        threads * it * kChains * 2);
    out_host[2] = timed([&] { peak_mufu<0><<<blocks, kPeakThreads, 0, s>>>(sink, it / 4); },
                        threads * (it / 4) * kChains);
    out_host[3] = timed([&] { peak_mufu<1><<<blocks, kPeakThreads, 0, s>>>(sink, it / 4); },
                        threads * (it / 4) * kChains);
    out_host[4] = timed([&] { peak_mufu<2><<<blocks, kPeakThreads, 0, s>>>(sink, it / 4); },
                        threads * (it / 4) * kChains);
    out_host[5] = h->sm_count;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return laue_cuda_check(h, cudaGetLastError(), "peak kernels");
}
