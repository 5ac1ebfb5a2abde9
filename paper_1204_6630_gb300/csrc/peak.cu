// FP32 fused multiply-add throughput of the device: the denominator of the
// counting kernel's roofline, measured rather than derived from the SM count
// and a nominal clock.  Not part of the paper's method (it is how its pair
// rate is put in proportion to the hardware).
//
// Every thread advances 16 independent dependent chains v = fma(v, s, c);
// blocks of 512 threads, 4 per SM, keep every scheduler's FMA pipe fed.  The
// scalar variant issues one fma.rn.f32 per FMA, the packed variant one
// fma.rn.f32x2 per two.  The result is the best of several timed launches
// (CUDA events), counted as 2 flops per FMA.
#include <stdint.h>

#include "tpcf.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 512;
constexpr int kBlocksPerSm = 4;

__device__ unsigned int g_peak_sink;

__global__ void __launch_bounds__(kThreads) fma_chains_kernel(int iters, float s, float c) {
    float v[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) v[k] = 1e-3f * (float)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(v[k]) : "f"(s), "f"(c));
    }
    unsigned int x = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) x ^= __float_as_uint(v[k]);
    if (x == 0x7f7fffffu) g_peak_sink = x;  // never true: keeps the chains alive
}

__global__ void __launch_bounds__(kThreads) fma2_chains_kernel(int iters, float s, float c) {
    unsigned long long v[kChains], ss, cc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(ss) : "f"(s));
    asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        const float a = 1e-3f * (float)(threadIdx.x + k), b = a + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(v[k]) : "f"(a), "f"(b));
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(v[k]) : "l"(ss), "l"(cc));
    }
    unsigned long long x = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) x ^= v[k];
    if (x == 0x7f7fffff7f7fffffull) g_peak_sink = (unsigned int)x;
}

}  // namespace

extern "C" int tpcf_fp32_peak(int device, int packed, double* tflops) {
    if (!tflops || (packed != 0 && packed != 1)) return TPCF_EINVAL;
    *tflops = 0.0;
    int ndev = 0, sms = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return TPCF_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return TPCF_ECUDA;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return TPCF_ECUDA;
    int rc = TPCF_OK;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) rc = TPCF_ECUDA;
    // about 20 ms per launch at 2 GHz: 2048 threads x 16 chains x iters FMAs per SM at 128 per cycle
    const int iters = packed ? 4096 : 8192;
    const int blocks = sms * kBlocksPerSm;
    double best_ms = 1e300;
    for (int rep = 0; rep < 6 && rc == TPCF_OK; ++rep) {  // the first launch is a warm-up
        if (cudaEventRecord(a, st) != cudaSuccess) { rc = TPCF_ECUDA; break; }
        if (packed) fma2_chains_kernel<<<blocks, kThreads, 0, st>>>(iters, 0.99999994f, 1e-7f);
        else fma_chains_kernel<<<blocks, kThreads, 0, st>>>(iters, 0.99999994f, 1e-7f);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(b, st) != cudaSuccess ||
            cudaEventSynchronize(b) != cudaSuccess) {
            rc = TPCF_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms > 0.f && ms < best_ms) best_ms = ms;
    }
    if (rc == TPCF_OK) {
        const double fmas = (double)blocks * kThreads * kChains * (double)iters * (packed ? 2.0 : 1.0);
        *tflops = 2.0 * fmas / (best_ms * 1e-3) / 1e12;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaStreamDestroy(st);
    return rc;
}
