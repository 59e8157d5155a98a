/*
 * FP32 arithmetic peak of the device, measured: the denominator of the ALU
 * roofline of the fused window kernel, whose filter taps, pair sums and
 * moments all run on the FP32 FMA pipe.
 *
 * sf_fma_probe runs eight independent fma chains per thread (scalar fma.rn.f32,
 * or packed fma.rn.f32x2 pairs) on 2048 threads per SM, so the FMA pipe never
 * waits on a dependency.  sf_fp32_peak times each form with CUDA events (best
 * of three launches after a warm-up) and returns 2 flops per lane-FMA per
 * second.  The paper has no counterpart: it is a measurement of the machine.
 */
#include <cuda_runtime.h>

#include <string>

#include "sf.h"

namespace {

typedef unsigned long long u64;

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__device__ __forceinline__ u64 pk(float a, float b)
{
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c)
{
    u64 d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

/* x <- x * a + b keeps every chain bounded for a just below 1; the final
 * store is conditional on a value the chains never reach, so nothing is
 * dead code */
template <bool PAIR>
__global__ void __launch_bounds__(kProbeThreads)
sf_fma_probe(float *sink, int iters, float a, float b)
{
    const float seed = (float)(threadIdx.x & 7) * 0.125f;
    if constexpr (PAIR) {
        u64 x[kProbeChains];
        const u64 A = pk(a, a), B = pk(b, b);
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) x[k] = pk(seed + k, seed - k);
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kProbeChains; ++k) x[k] = fma2(x[k], A, B);
        u64 s = x[0];
#pragma unroll
        for (int k = 1; k < kProbeChains; ++k) s ^= x[k];
        if ((unsigned)s == 0x7f800001u) sink[blockIdx.x] = (float)(s >> 32);
    } else {
        float x[kProbeChains];
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) x[k] = seed + k;
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kProbeChains; ++k)
                asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[k]) : "f"(a), "f"(b));
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) s += x[k];
        if (s == -1.0e30f) sink[blockIdx.x] = s;
    }
}

thread_local std::string g_probe_err;

sf_status probe_fail(cudaError_t e, const char *what)
{
    g_probe_err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return SF_ECUDA;
}

}  // namespace

extern "C" sf_status sf_fp32_peak(int32_t device, double *tflops_scalar, double *tflops_pair)
{
    if (!tflops_scalar || !tflops_pair) {
        g_probe_err = "sf_fp32_peak: null output pointer";
        return SF_EINVAL;
    }
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return probe_fail(e, "cudaGetDevice");
    if ((e = cudaSetDevice(device)) != cudaSuccess) return probe_fail(e, "cudaSetDevice");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = sms * (2048 / kProbeThreads);
    float *sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sf_status rc = SF_OK;
    const int iters = 1 << 15;
    double best[2] = {0.0, 0.0};
    if ((e = cudaMalloc(&sink, sizeof(float) * blocks)) != cudaSuccess) {
        rc = probe_fail(e, "cudaMalloc");
        goto done;
    }
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        rc = probe_fail(e, "stream/event creation");
        goto done;
    }
    for (int form = 0; form < 2; ++form) {
        /* lane-FMAs per launch: chains (x2 lanes for the pairs) per iteration */
        const double lane_fma = (double)blocks * kProbeThreads * kProbeChains * (form ? 2 : 1) * iters;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, st);
            if (form == 0) sf_fma_probe<false><<<blocks, kProbeThreads, 0, st>>>(sink, iters, 0.9999f, 1e-4f);
            else sf_fma_probe<true><<<blocks, kProbeThreads, 0, st>>>(sink, iters, 0.9999f, 1e-4f);
            cudaEventRecord(e1, st);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
                rc = probe_fail(e, "probe launch");
                goto done;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms > 0.f) {
                const double tf = 2.0 * lane_fma / (ms * 1e-3) / 1e12;
                if (tf > best[form]) best[form] = tf;
            }
        }
    }
    *tflops_scalar = best[0];
    *tflops_pair = best[1];
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}

extern "C" const char *sf_fp32_peak_error(void) { return g_probe_err.c_str(); }
