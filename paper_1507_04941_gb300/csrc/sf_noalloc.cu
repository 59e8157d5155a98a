/*
 * sf_filter_noalloc: the filtered cube of one Gaussian filter for callers that
 * cannot allocate device memory.
 *
 * Some callers must not call cudaMalloc / cudaFree at all: code running while
 * a CUDA graph is being captured into a pool they do not own, allocation-free
 * real-time loops whose memory is budgeted up front, or hosts embedding this
 * library inside another runtime that owns every allocation.  They cannot
 * create an sf_ctx (sf_create allocates the scratch cubes and loads kernels).
 * This entry point needs no context: it runs three one-dimensional passes
 * (x, y, z) with the two intermediate cubes kept in one fixed scratch array
 * that lives in this file, and the caller passes only the input cube and the
 * output cube.
 *
 * The scratch array is a file-scope __device__ array of SF_NOALLOC_BYTES
 * (64 MiB), so every GPU that loads the library holds it until the process
 * exits.  It bounds the cube to SF_NOALLOC_BYTES / 8 voxels (8,388,608 FP32
 * voxels, two intermediate cubes); larger cubes are rejected with SF_EINVAL.
 * Every call shares the array: two calls whose work overlaps on the GPU (on
 * different streams, or from different host threads) race on it and give
 * wrong results.  Nothing in the array needs clearing between calls: each
 * pass writes every element the next pass reads.
 *
 * The first call on a device looks up the device address of the array with
 * cudaGetSymbolAddress (the array's name in host code is only a host-side
 * stand-in); make that first call before any stream capture.
 */
#include "sf.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include <cstdio>

#define SF_NOALLOC_BYTES ((size_t)64 << 20)

void sf_set_global_error(const char *msg);   /* sf_runtime.cpp: sf_last_error(NULL) */

/* the scratch: two intermediate FP32 cubes, shared by every call */
static __device__ __align__(256) unsigned char g_noalloc_scratch[SF_NOALLOC_BYTES];

namespace {

constexpr size_t kScratchBytes = SF_NOALLOC_BYTES;
constexpr int kMaxR = 32;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

struct Taps1D {
    float g[2 * kMaxR + 1];
    int r;
};

/* out[x][y][z] = sum_o g[o] in[x + o*step_axis] along one axis, zero outside */
__global__ void __launch_bounds__(256)
noalloc_pass(const float *__restrict__ in, float *__restrict__ out, long long nx, long long ny,
             long long nz, int axis, Taps1D t)
{
    const long long n = nx * ny * nz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long z = i % nz, y = (i / nz) % ny, x = i / (nz * ny);
        const long long pos = axis == 0 ? x : axis == 1 ? y : z;
        const long long len = axis == 0 ? nx : axis == 1 ? ny : nz;
        const long long stride = axis == 0 ? ny * nz : axis == 1 ? nz : 1;
        float s = 0.f;
        for (int o = -t.r; o <= t.r; ++o) {
            const long long q = pos + o;
            if (q >= 0 && q < len) s = fmaf(t.g[o + t.r], __ldg(in + i + (long long)o * stride), s);
        }
        out[i] = s;
    }
}

Taps1D make_taps(double sigma, double truncation)
{
    Taps1D t{};
    t.r = sigma > 0.0 ? (int)std::ceil(truncation * sigma) : 0;
    if (t.r == 0) {
        t.g[0] = 1.f;
        return t;
    }
    double w[2 * kMaxR + 1], total = 0.0;
    for (int o = -t.r; o <= t.r; ++o) {
        w[o + t.r] = std::exp(-(double)o * o / (2.0 * sigma * sigma));
        total += w[o + t.r];
    }
    for (int o = -t.r; o <= t.r; ++o) t.g[o + t.r] = (float)(w[o + t.r] / total);
    return t;
}

}  // namespace

extern "C" sf_status sf_filter_noalloc(const float *d_cube, int64_t nx, int64_t ny, int64_t nz,
                                       float sigma_xy, float sigma_z, float truncation,
                                       float *d_filtered, void *stream)
{
    char msg[256];
    if (!d_cube || !d_filtered) {
        sf_set_global_error("sf_filter_noalloc: NULL buffer");
        return SF_EINVAL;
    }
    if (nx < 1 || ny < 1 || nz < 1) {
        sf_set_global_error("sf_filter_noalloc: cube dimensions must be >= 1");
        return SF_EINVAL;
    }
    if (!(truncation > 0.f) || !(sigma_xy >= 0.f) || !(sigma_z >= 0.f) ||
        !std::isfinite(sigma_xy) || !std::isfinite(sigma_z) || !std::isfinite(truncation)) {
        sf_set_global_error("sf_filter_noalloc: sigmas must be finite and >= 0, truncation > 0");
        return SF_EINVAL;
    }
    const double nvox = (double)nx * (double)ny * (double)nz;
    if (nvox * 2.0 * sizeof(float) > (double)kScratchBytes) {
        snprintf(msg, sizeof(msg),
                 "sf_filter_noalloc: %.0f voxels exceed the fixed scratch (%zu bytes holds two "
                 "float32 cubes of at most %zu voxels)",
                 nvox, kScratchBytes, kScratchBytes / (2 * sizeof(float)));
        sf_set_global_error(msg);
        return SF_EINVAL;
    }
    if ((sigma_xy > 0.f && std::ceil((double)truncation * sigma_xy) > kMaxR) ||
        (sigma_z > 0.f && std::ceil((double)truncation * sigma_z) > kMaxR)) {
        sf_set_global_error("sf_filter_noalloc: filter radius above 32");
        return SF_EINVAL;
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        sf_set_global_error("sf_filter_noalloc: cudaGetDevice failed (no usable CUDA device)");
        return SF_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        snprintf(msg, sizeof(msg), "sf_filter_noalloc: device %d beyond the %d devices it serves", dev,
                 kMaxDevices);
        sf_set_global_error(msg);
        return SF_ECUDA;
    }
    void *scratch = nullptr;
    {
        /* set-up once per device, with that device current: the host-side name
         * of the array is not a device address, so ask the runtime for it */
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                sf_set_global_error("sf_filter_noalloc: cudaGetSymbolAddress of the scratch failed");
                return SF_ECUDA;
            }
            g_scratch_ptr[dev] = p;
        }
        scratch = g_scratch_ptr[dev];
    }
    float *t1 = (float *)scratch;
    float *t2 = t1 + (size_t)nx * ny * nz;
    const Taps1D gxy = make_taps(sigma_xy, truncation), gz = make_taps(sigma_z, truncation);
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = nx * ny * nz;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    noalloc_pass<<<blocks, 256, 0, st>>>(d_cube, t1, nx, ny, nz, 0, gxy);
    noalloc_pass<<<blocks, 256, 0, st>>>(t1, t2, nx, ny, nz, 1, gxy);
    noalloc_pass<<<blocks, 256, 0, st>>>(t2, d_filtered, nx, ny, nz, 2, gz);
    if (cudaGetLastError() != cudaSuccess) {
        sf_set_global_error("sf_filter_noalloc: kernel launch failed");
        return SF_ECUDA;
    }
    return SF_OK;
}
