/*
 * Elementwise kernels of the weighted convolution (Eq. 1):
 *   sf_w_product  p = d * w, the numerator's input;
 *   sf_w_ratio    c = num / den where den != 0, else 0 (no weight in the
 *                 filter's support).
 * Both move four floats per thread per step (16-byte loads and stores) with a
 * grid-stride loop, and handle a ragged tail element by element.
 */
#include <cuda_runtime.h>

namespace {

typedef long long i64;

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) sf_w_product(const float *__restrict__ d, const float *__restrict__ w,
                                                       float *__restrict__ p, i64 n)
{
    const i64 n4 = n / 4;
    const i64 stride = (i64)gridDim.x * kThreads;
    for (i64 i = (i64)blockIdx.x * kThreads + threadIdx.x; i < n4; i += stride) {
        const float4 a = reinterpret_cast<const float4 *>(d)[i];
        const float4 b = reinterpret_cast<const float4 *>(w)[i];
        reinterpret_cast<float4 *>(p)[i] = make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
    }
    for (i64 i = 4 * n4 + (i64)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) p[i] = d[i] * w[i];
}

__device__ __forceinline__ float safe_ratio(float a, float b) { return b != 0.f ? a / b : 0.f; }

__global__ void __launch_bounds__(kThreads) sf_w_ratio(const float *__restrict__ num, const float *__restrict__ den,
                                                     float *__restrict__ out, i64 n)
{
    const i64 n4 = n / 4;
    const i64 stride = (i64)gridDim.x * kThreads;
    for (i64 i = (i64)blockIdx.x * kThreads + threadIdx.x; i < n4; i += stride) {
        const float4 a = reinterpret_cast<const float4 *>(num)[i];
        const float4 b = reinterpret_cast<const float4 *>(den)[i];
        reinterpret_cast<float4 *>(out)[i] =
            make_float4(safe_ratio(a.x, b.x), safe_ratio(a.y, b.y), safe_ratio(a.z, b.z), safe_ratio(a.w, b.w));
    }
    for (i64 i = 4 * n4 + (i64)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride)
        out[i] = safe_ratio(num[i], den[i]);
}

unsigned grid_for(i64 n)
{
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const i64 want = (n / 4 + kThreads - 1) / kThreads;
    const i64 cap = (i64)nsm * 8;
    return (unsigned)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace

cudaError_t sf_launch_w_product(const float *d, const float *w, float *p, long long n, cudaStream_t st)
{
    sf_w_product<<<grid_for(n), kThreads, 0, st>>>(d, w, p, n);
    return cudaGetLastError();
}

cudaError_t sf_launch_w_ratio(const float *num, const float *den, float *out, long long n, cudaStream_t st)
{
    sf_w_ratio<<<grid_for(n), kThreads, 0, st>>>(num, den, out, n);
    return cudaGetLastError();
}
