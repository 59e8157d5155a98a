/*
 * Kernels compiled ahead of time (their shape does not depend on the filter
 * radii): window statistics of a filtered cube and the threshold / mask
 * packing of one filtered cube.  Both back the step-by-step entry points
 * sf_stats and sf_threshold and the composed path of sf_detect.
 */
#include <cuda_runtime.h>

namespace {

typedef long long i64;

/* moments of a set of values; T = float, or double for the FP64 combine of
 * the per-thread FP32 partial sums */
template <class T>
struct Mom {
    T n, mean, m2;
};

template <class T>
__device__ __forceinline__ Mom<T> merge(Mom<T> a, Mom<T> b)
{
    if (b.n == 0) return a;
    if (a.n == 0) return b;
    const T n = a.n + b.n;
    const T d = b.mean - a.mean;
    const T wb = b.n / n;
    return Mom<T>{n, fma(d, wb, a.mean), a.m2 + b.m2 + d * d * a.n * wb};
}

constexpr int kStatThreads = 256;

/* Window mean and population standard deviation (Sec. 3.3): one CTA per
 * window.  Each thread sums its values shifted by its first value (FP32), the
 * per-thread moments are merged pairwise (Chan et al.) in T across the warp
 * and then across warps in a fixed order. */
template <class T>
__global__ void __launch_bounds__(kStatThreads)
sf_window_stats_kernel(const float *__restrict__ c, i64 nx, i64 ny, i64 nz, int wx, int wy, int wz,
                       int nwy, int nwz, int ddof, float *__restrict__ mean, float *__restrict__ stdv)
{
    __shared__ T red[kStatThreads / 32][3];
    const int w = blockIdx.x;
    const int a = w / (nwy * nwz), b = (w / nwz) % nwy, e = w % nwz;
    const i64 x0 = (i64)a * wx, y0 = (i64)b * wy, z0 = (i64)e * wz;
    const int ex = (int)min((i64)wx, nx - x0), ey = (int)min((i64)wy, ny - y0),
              ez = (int)min((i64)wz, nz - z0);
    float K = 0.f, s1 = 0.f, s2 = 0.f, cnt = 0.f;
    /* warps over the window's (x, y) rows, lanes over z: coalesced, one
     * division per row */
    const int lane0 = threadIdx.x & 31, warp0 = threadIdx.x >> 5;
    for (int row = warp0; row < ex * ey; row += kStatThreads / 32) {
        const int dx = row / ey, dy = row - dx * ey;
        const float *p = c + ((x0 + dx) * ny + (y0 + dy)) * nz + z0;
        for (int dz = lane0; dz < ez; dz += 32) {
            const float v = __ldg(p + dz);
            if (cnt == 0.f) K = v;
            const float d = v - K;
            s1 += d;
            s2 = fmaf(d, d, s2);
            cnt += 1.f;
        }
    }
    Mom<T> m{0, 0, 0};
    if (cnt > 0.f) {
        const T mu = (T)s1 / (T)cnt;
        m = Mom<T>{(T)cnt, (T)K + mu, fmax((T)s2 - (T)s1 * mu, (T)0)};
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        Mom<T> o{__shfl_xor_sync(0xffffffffu, m.n, off), __shfl_xor_sync(0xffffffffu, m.mean, off),
                 __shfl_xor_sync(0xffffffffu, m.m2, off)};
        m = (lane & off) ? merge(o, m) : merge(m, o);
    }
    if (lane == 0) {
        red[warp][0] = m.n;
        red[warp][1] = m.mean;
        red[warp][2] = m.m2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Mom<T> t{0, 0, 0};
        for (int q = 0; q < kStatThreads / 32; ++q) t = merge(t, Mom<T>{red[q][0], red[q][1], red[q][2]});
        mean[w] = (float)t.mean;
        stdv[w] = (float)(t.n > ddof ? sqrt(t.m2 / (t.n - ddof)) : (T)0);
    }
}

constexpr int kThrThreads = 256;

/* One warp per (x, y) row, walking its mask words: lane l tests voxel
 * z = 32*word + l against mean + k*std of its window and the warp ballot is
 * the word (OR-ed into the word already there when accumulating). */
__global__ void __launch_bounds__(kThrThreads)
sf_threshold_kernel(const float *__restrict__ c, i64 nx, i64 ny, i64 nz, int wx, int wy, int wz,
                    int nwy, int nwz, const float *__restrict__ mean, const float *__restrict__ stdv,
                    float k, unsigned int *__restrict__ mask, int accumulate, i64 nw32, i64 nrows)
{
    const i64 xy = (i64)blockIdx.x * (kThrThreads / 32) + (threadIdx.x >> 5);
    if (xy >= nrows) return;
    const int lane = threadIdx.x & 31;
    const i64 x = xy / ny, y = xy - x * ny;
    const int wbase = (int)(((x / wx) * nwy + y / wy) * nwz);
    const float *row = c + xy * nz;
    unsigned int *mrow = mask + xy * nw32;
    for (int zw = 0; zw < (int)nw32; ++zw) {
        const int z = zw * 32 + lane;
        bool fire = false;
        if (z < nz) {
            const int wi = wbase + z / wz;
            fire = __ldg(row + z) > fmaf(k, __ldg(stdv + wi), __ldg(mean + wi));
        }
        const unsigned int bits = __ballot_sync(0xffffffffu, fire);
        if (lane == 0) {
            if (!accumulate) mrow[zw] = bits;
            else if (bits) atomicOr(mrow + zw, bits);
        }
    }
}

}  // namespace

cudaError_t sf_launch_stats(const float *c, long long nx, long long ny, long long nz, int wx, int wy,
                            int wz, int nwx, int nwy, int nwz, float *mean, float *stdv, int fp64, int ddof,
                            cudaStream_t st)
{
    const long long nwin = (long long)nwx * nwy * nwz;
    if (fp64)
        sf_window_stats_kernel<double><<<(unsigned)nwin, kStatThreads, 0, st>>>(c, nx, ny, nz, wx, wy, wz, nwy,
                                                                                 nwz, ddof, mean, stdv);
    else
        sf_window_stats_kernel<float><<<(unsigned)nwin, kStatThreads, 0, st>>>(c, nx, ny, nz, wx, wy, wz, nwy,
                                                                               nwz, ddof, mean, stdv);
    return cudaGetLastError();
}

cudaError_t sf_launch_threshold(const float *c, long long nx, long long ny, long long nz, int wx,
                                int wy, int wz, int nwy, int nwz, const float *mean,
                                const float *stdv, float k, unsigned int *mask, int accumulate,
                                cudaStream_t st)
{
    const long long nw32 = (nz + 31) / 32;
    const long long nrows = nx * ny;
    const long long per = kThrThreads / 32;
    const long long blocks = (nrows + per - 1) / per;
    sf_threshold_kernel<<<(unsigned)blocks, kThrThreads, 0, st>>>(c, nx, ny, nz, wx, wy, wz, nwy, nwz,
                                                                   mean, stdv, k, mask, accumulate,
                                                                   nw32, nrows);
    return cudaGetLastError();
}
