/*
 * Device code of the Gaussian source-finder hot path, compiled at plan time
 * for sm_103a by the host runtime.  The runtime prepends sf_kernel_abi.h and
 * a prelude of #defines that fix the filter radii, window shape, storage type
 * and launch shape of one plan, so every loop over filter taps is fully
 * unrolled with the taps read from the kernel's parameter bank.
 *
 * Method (Westerlund & Harris): Eq. 2 convolution with a separable 3D
 * Gaussian (x pass, then y and z passes), zero outside the cube; the local
 * mean / standard deviation of each filtered cube over windows (Sec. 3.3);
 * voxel selection c > mean + k*std; OR of the selections of all filters.
 *
 * Kernels (one per compiled program, chosen by the prelude):
 *   SF_KERNEL_XPASS   sf_xpass      x pass for up to four sigma_xy at once.
 *                                   Each thread owns V consecutive z of one
 *                                   (y, z) lane and marches along x with a
 *                                   register ring of the last 2R+1+PF planes,
 *                                   so every input element is read once.
 *   SF_KERNEL_DETECT  sf_window_detect  one CTA per statistics window: per
 *                                   input cube a TMA-staged slab per x-plane,
 *                                   y filter in shared memory, z filters in
 *                                   registers, moments and plane maxima (pass
 *                                   1), then the flagged planes filtered again
 *                                   and thresholded (pass 2); one packed store
 *                                   per mask word.
 *   SF_KERNEL_PERSIST sf_persist    the x pass and the windows of many cubes
 *                                   in one persistent launch (a work queue
 *                                   with per-cube completion counters).
 *   SF_KERNEL_FILTER  sf_yz_filter  y and z passes of one filter writing the
 *                                   float32 filtered cube.
 */

typedef unsigned int u32;
typedef unsigned short u16;
typedef long long i64;
typedef unsigned long long u64;

template <class T> struct sf_is_f32 { static constexpr bool v = false; };
template <> struct sf_is_f32<float> { static constexpr bool v = true; };

template <class T> __device__ __forceinline__ float sf_dec16(u32 b);
template <> __device__ __forceinline__ float sf_dec16<sf_f16>(u32 b)
{
    const u16 h = (u16)b;
    float f;
    asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(h));
    return f;
}
template <> __device__ __forceinline__ float sf_dec16<sf_bf16>(u32 b)
{
    return __uint_as_float(b << 16);
}
template <class T> __device__ __forceinline__ u32 sf_enc16(float f);
template <> __device__ __forceinline__ u32 sf_enc16<sf_f16>(float f)
{
    u16 h;
    asm("cvt.rn.f16.f32 %0, %1;" : "=h"(h) : "f"(f));
    return (u32)h;
}
template <> __device__ __forceinline__ u32 sf_enc16<sf_bf16>(float f)
{
    u16 h;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(f));
    return (u32)h;
}

/* N consecutive elements of storage type T -> float (GLOBAL: read-only path). */
template <class T, int N, bool GLOBAL>
__device__ __forceinline__ void sf_ld(const T *p, float *o)
{
    if constexpr (sf_is_f32<T>::v) {
        if constexpr (N == 4) {
            float4 v;
            if constexpr (GLOBAL) v = __ldg(reinterpret_cast<const float4 *>(p));
            else v = *reinterpret_cast<const float4 *>(p);
            o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
        } else if constexpr (N == 2) {
            float2 v;
            if constexpr (GLOBAL) v = __ldg(reinterpret_cast<const float2 *>(p));
            else v = *reinterpret_cast<const float2 *>(p);
            o[0] = v.x; o[1] = v.y;
        } else {
            static_assert(N == 1, "vector width");
            if constexpr (GLOBAL) o[0] = __ldg(reinterpret_cast<const float *>(p));
            else o[0] = *reinterpret_cast<const float *>(p);
        }
    } else {
        if constexpr (N == 8) {
            uint4 v;
            if constexpr (GLOBAL) v = __ldg(reinterpret_cast<const uint4 *>(p));
            else v = *reinterpret_cast<const uint4 *>(p);
            o[0] = sf_dec16<T>(v.x & 0xffffu); o[1] = sf_dec16<T>(v.x >> 16);
            o[2] = sf_dec16<T>(v.y & 0xffffu); o[3] = sf_dec16<T>(v.y >> 16);
            o[4] = sf_dec16<T>(v.z & 0xffffu); o[5] = sf_dec16<T>(v.z >> 16);
            o[6] = sf_dec16<T>(v.w & 0xffffu); o[7] = sf_dec16<T>(v.w >> 16);
        } else if constexpr (N == 4) {
            uint2 v;
            if constexpr (GLOBAL) v = __ldg(reinterpret_cast<const uint2 *>(p));
            else v = *reinterpret_cast<const uint2 *>(p);
            o[0] = sf_dec16<T>(v.x & 0xffffu); o[1] = sf_dec16<T>(v.x >> 16);
            o[2] = sf_dec16<T>(v.y & 0xffffu); o[3] = sf_dec16<T>(v.y >> 16);
        } else if constexpr (N == 2) {
            u32 v;
            if constexpr (GLOBAL) v = __ldg(reinterpret_cast<const unsigned int *>(p));
            else v = *reinterpret_cast<const unsigned int *>(p);
            o[0] = sf_dec16<T>(v & 0xffffu); o[1] = sf_dec16<T>(v >> 16);
        } else {
            static_assert(N == 1, "vector width");
            u16 v;
            if constexpr (GLOBAL) v = __ldg(reinterpret_cast<const unsigned short *>(p));
            else v = *reinterpret_cast<const unsigned short *>(p);
            o[0] = sf_dec16<T>((u32)v);
        }
    }
}

/* N floats -> N consecutive elements of storage type T (round to nearest). */
template <class T, int N>
__device__ __forceinline__ void sf_st(T *p, const float *v)
{
    if constexpr (sf_is_f32<T>::v) {
        if constexpr (N == 4) *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
        else if constexpr (N == 2) *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
        else *reinterpret_cast<float *>(p) = v[0];
    } else {
        if constexpr (N == 8) {
            uint4 w;
            w.x = sf_enc16<T>(v[0]) | (sf_enc16<T>(v[1]) << 16);
            w.y = sf_enc16<T>(v[2]) | (sf_enc16<T>(v[3]) << 16);
            w.z = sf_enc16<T>(v[4]) | (sf_enc16<T>(v[5]) << 16);
            w.w = sf_enc16<T>(v[6]) | (sf_enc16<T>(v[7]) << 16);
            *reinterpret_cast<uint4 *>(p) = w;
        } else if constexpr (N == 4) {
            uint2 w;
            w.x = sf_enc16<T>(v[0]) | (sf_enc16<T>(v[1]) << 16);
            w.y = sf_enc16<T>(v[2]) | (sf_enc16<T>(v[3]) << 16);
            *reinterpret_cast<uint2 *>(p) = w;
        } else if constexpr (N == 2) {
            *reinterpret_cast<unsigned int *>(p) = sf_enc16<T>(v[0]) | (sf_enc16<T>(v[1]) << 16);
        } else {
            *reinterpret_cast<unsigned short *>(p) = (unsigned short)sf_enc16<T>(v[0]);
        }
    }
}

/* ---- packed FP32 pairs (f32x2): one instruction for two lanes of work ---- */
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_pack(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float f2_lo(f2 v)
{
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return a;
}
__device__ __forceinline__ float f2_hi(f2 v)
{
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return b;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

/* ======================================================================= */
#if defined(SF_KERNEL_XPASS) || defined(SF_KERNEL_PERSIST) || defined(SF_KERNEL_XBATCH)
/* Prelude: SFX_NOUT, SFX_R0..SFX_R3 (radii, 0 = unused), SFX_RM (max radius),
 * SFX_PF (prefetch depth), typedef sfx_t; the stand-alone kernel adds SFX_V and
 * SFX_THREADS. */
struct sfx_taps { float g[SFX_NOUT][SFX_RM + 1]; };   /* g[k][|o|] */
__host__ __device__ constexpr int sfx_r(int k)
{
    return k == 0 ? SFX_R0 : k == 1 ? SFX_R1 : k == 2 ? SFX_R2 : SFX_R3;
}

/* x pass of one lane (V consecutive z of one (y, z) position) over output
 * planes [xb, xe): a register ring of the last 2R+1+PF input planes, every
 * input element read once, pair sums shared by the NOUT outputs.  Input
 * planes are `plane` elements apart; output k is written at
 * dst[k] + x * oplane + lane_off (a null dst[k] is skipped). */
template <int V>
__device__ __forceinline__ void sfx_lane(const sfx_t *__restrict__ p, void *const *dst, i64 lane_off,
                                         i64 nx, i64 plane, i64 oplane, i64 xb, i64 xe, const sfx_taps &t)
{
    constexpr int RM = SFX_RM, K = 2 * RM + 1 + SFX_PF;
    const i64 xlim = min(nx, xe + RM);            /* inputs used: [xb-RM, xe+RM) */
    /* slot i of the ring holds input plane xb-RM+i (mod K) */
    float ring[K][V];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const i64 xi = xb - RM + i;
        if (xi >= 0 && xi < xlim) sf_ld<sfx_t, V, true>(p + xi * plane, ring[i]);
        else {
#pragma unroll
            for (int v = 0; v < V; ++v) ring[i][v] = 0.f;
        }
    }
    for (i64 x0 = xb; x0 < xe; x0 += K) {
#pragma unroll
        for (int u = 0; u < K; ++u) {
            const i64 x = x0 + u;
            if (x < xe) {
                float ps[RM + 1][V];
#pragma unroll
                for (int v = 0; v < V; ++v) ps[0][v] = ring[(u + RM) % K][v];
#pragma unroll
                for (int j = 1; j <= RM; ++j)
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        ps[j][v] = ring[(u + RM - j) % K][v] + ring[(u + RM + j) % K][v];
#pragma unroll
                for (int k = 0; k < SFX_NOUT; ++k) {
                    float acc[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) acc[v] = t.g[k][0] * ps[0][v];
#pragma unroll
                    for (int j = 1; j <= sfx_r(k); ++j)
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] = fmaf(t.g[k][j], ps[j][v], acc[v]);
                    if (dst[k] != nullptr)
                        sf_st<sfx_t, V>(reinterpret_cast<sfx_t *>(dst[k]) + x * oplane + lane_off, acc);
                }
                /* slot u is free: refill it with plane x - RM + K */
                const i64 xi = x - RM + K;
                if (xi < xlim) sf_ld<sfx_t, V, true>(p + xi * plane, ring[u]);
                else {
#pragma unroll
                    for (int v = 0; v < V; ++v) ring[u][v] = 0.f;
                }
            }
        }
    }
}

/* Staged form: the input planes of a lane stream through D slots of shared
 * memory filled by cp.async (zero fill outside [0, xlim)), D - 1 planes ahead
 * of use, so the loads in flight cost no registers; the register ring then
 * holds exactly the 2R+1 planes the filter reads.  Each thread only ever
 * reads the slots its own copies wrote, so a cp.async.wait_group is the whole
 * synchronisation; a slot is refilled one step after it was read.  sb / sp:
 * the thread's slot 0 (shared address / pointer), slots THREADS*V elements
 * apart. */
template <int V>
__device__ __forceinline__ void sfx_stage(u32 dst, const void *src, bool in)
{
    constexpr int VB = V * (int)sizeof(sfx_t);
    static_assert(VB == 4 || VB == 8 || VB == 16, "cp.async sizes");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(dst), "l"(src), "n"(VB),
                 "r"(in ? VB : 0)
                 : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int V, int THREADS, int D>
__device__ __forceinline__ void sfx_lane_staged(const sfx_t *__restrict__ p, void *const *dst,
                                                i64 lane_off, i64 nx, i64 plane, i64 oplane, i64 xb, i64 xe,
                                                const sfx_taps &t, u32 sb, const unsigned char *sp)
{
    static_assert(D >= 3, "staging depth");
    constexpr int RM = SFX_RM, K = 2 * RM + 1;
    constexpr u32 STRIDE = THREADS * V * (u32)sizeof(sfx_t);
    const i64 xlim = min(nx, xe + RM);                 /* inputs used: [xb-RM, xlim) */
    /* step s of the stream consumes input plane xb - RM + s */
    auto stage = [&](i64 s, int slot) {
        const i64 xi = xb - RM + s;
        const bool in = xi >= 0 && xi < xlim;
        sfx_stage<V>(sb + (u32)slot * STRIDE, in ? p + xi * plane : p, in);
    };
#pragma unroll
    for (int i = 0; i < D - 1; ++i) stage(i, i);
    float ring[K][V];                                  /* ring[s % K] = plane of step s */
    const i64 S = (xe - xb) + 2 * RM;
    int slot = 0;
    for (i64 s0 = 0; s0 < S; s0 += K) {
#pragma unroll
        for (int u = 0; u < K; ++u) {
            const i64 s = s0 + u;
            if (s < S) {
                asm volatile("cp.async.wait_group %0;\n" ::"n"(D - 2) : "memory");
                sf_ld<sfx_t, V, false>(reinterpret_cast<const sfx_t *>(sp + slot * STRIDE), ring[u]);
                stage(s + D - 1, slot == 0 ? D - 1 : slot - 1);
                slot = slot + 1 == D ? 0 : slot + 1;
                if (s >= 2 * RM) {
                    /* output plane x = xb + s - 2R, centred on ring slot c */
                    const i64 x = xb + s - 2 * RM;
                    const int c = (u + RM + 1) % K;
                    float o[SFX_NOUT][V];
                    if constexpr (V % 2 == 0) {
                        constexpr int H = V / 2 > 0 ? V / 2 : 1;
                        f2 acc[SFX_NOUT][H];
#pragma unroll
                        for (int h = 0; h < H; ++h) {
                            const f2 m = f2_pack(ring[c][2 * h], ring[c][2 * h + 1]);
#pragma unroll
                            for (int k = 0; k < SFX_NOUT; ++k)
                                acc[k][h] = f2_mul(f2_pack(t.g[k][0], t.g[k][0]), m);
                        }
#pragma unroll
                        for (int j = 1; j <= RM; ++j)
#pragma unroll
                            for (int h = 0; h < H; ++h) {
                                const int a0 = (c + j) % K, a1 = (c + K - j) % K;
                                const f2 ps = f2_add(f2_pack(ring[a0][2 * h], ring[a0][2 * h + 1]),
                                                     f2_pack(ring[a1][2 * h], ring[a1][2 * h + 1]));
#pragma unroll
                                for (int k = 0; k < SFX_NOUT; ++k)
                                    if (j <= sfx_r(k))
                                        acc[k][h] = f2_fma(f2_pack(t.g[k][j], t.g[k][j]), ps, acc[k][h]);
                            }
#pragma unroll
                        for (int k = 0; k < SFX_NOUT; ++k)
#pragma unroll
                            for (int h = 0; h < H; ++h) {
                                o[k][2 * h] = f2_lo(acc[k][h]);
                                o[k][2 * h + 1] = f2_hi(acc[k][h]);
                            }
                    } else {
#pragma unroll
                        for (int v = 0; v < V; ++v) {
#pragma unroll
                            for (int k = 0; k < SFX_NOUT; ++k) o[k][v] = t.g[k][0] * ring[c][v];
#pragma unroll
                            for (int j = 1; j <= RM; ++j) {
                                const float ps = ring[(c + j) % K][v] + ring[(c + K - j) % K][v];
#pragma unroll
                                for (int k = 0; k < SFX_NOUT; ++k)
                                    if (j <= sfx_r(k)) o[k][v] = fmaf(t.g[k][j], ps, o[k][v]);
                            }
                        }
                    }
#pragma unroll
                    for (int k = 0; k < SFX_NOUT; ++k)
                        if (dst[k] != nullptr)
                            sf_st<sfx_t, V>(reinterpret_cast<sfx_t *>(dst[k]) + x * oplane + lane_off, o[k]);
                }
            }
        }
    }
    /* copies of planes past the end may still be in flight */
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
#endif

#ifdef SF_KERNEL_XPASS
#if SFX_D > 0
extern __shared__ __align__(16) unsigned char sfx_smem[];
#endif
extern "C" __global__ void __launch_bounds__(SFX_THREADS)
sf_xpass(const __grid_constant__ sf_xargs a, const __grid_constant__ sfx_taps t)
{
    const i64 lane = (i64)blockIdx.x * SFX_THREADS + threadIdx.x;
    if (lane >= a.lanes) return;
    const i64 xb = a.xoff + (i64)blockIdx.y * a.xseg;
    const i64 xe = min(a.nx, xb + a.xseg);
    const sfx_t *p = reinterpret_cast<const sfx_t *>(a.src) + lane * SFX_V;
    /* outputs with a padded z stride (ozs > nz; planned with V dividing nz,
     * so a lane stays within a row): the lane's first element (y, z) moves
     * to y * ozs + z; the padding is never written */
    i64 olane = lane * SFX_V, oplane = a.plane;
    if (a.ozs != a.nz) {
        const i64 e = lane * SFX_V, y = e / a.nz;
        olane = y * a.ozs + (e - y * a.nz);
        oplane = (a.plane / a.nz) * a.ozs;
    }
#if SFX_D > 0
    constexpr u32 VB = SFX_V * (u32)sizeof(sfx_t);
    sfx_lane_staged<SFX_V, SFX_THREADS, SFX_D>(
        p, a.dst, olane, a.nx, a.plane, oplane, xb, xe, t,
        (u32)__cvta_generic_to_shared(sfx_smem) + threadIdx.x * VB, sfx_smem + threadIdx.x * VB);
#else
    sfx_lane<SFX_V>(p, a.dst, olane, a.nx, a.plane, oplane, xb, xe, t);
#endif
}
#endif /* SF_KERNEL_XPASS */

#ifdef SF_KERNEL_XBATCH
/* sf_xpass_batch: the staged x pass of every cube of a batch in one launch
 * (SFX_THREADS threads, SFX_D slots per thread, lanes of two elements, or one
 * where the y-z plane is odd).  Block b finds its cube by bisection of the
 * block0 column of the table. */
extern __shared__ __align__(16) unsigned char sfx_smem[];

template <int V>
__device__ __forceinline__ void sfx_batch_lane(const sf_xcube &q, i64 lane, i64 olane, i64 oplane, const sfx_taps &t)
{
    constexpr u32 VB = V * (u32)sizeof(sfx_t);
    const sfx_t *p = reinterpret_cast<const sfx_t *>(q.src) + lane * V;
    sfx_lane_staged<V, SFX_THREADS, SFX_D>(p, q.dst, olane, q.nx, q.plane, oplane, q.x0, q.x1, t,
                                           (u32)__cvta_generic_to_shared(sfx_smem) + threadIdx.x * VB,
                                           sfx_smem + threadIdx.x * VB);
}

extern "C" __global__ void __launch_bounds__(SFX_THREADS, 6)
sf_xpass_batch(const __grid_constant__ sf_xbargs a, const __grid_constant__ sfx_taps t)
{
    const int blk = (int)blockIdx.x;
    int lo = 0, hi = a.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.cubes[mid].block0 <= blk) lo = mid;
        else hi = mid - 1;
    }
    const sf_xcube &q = a.cubes[lo];
    const i64 lane = (i64)(blk - q.block0) * SFX_THREADS + threadIdx.x;
    if (lane >= q.lanes) return;
    /* outputs with a padded z stride (ozs > nz; v divides nz, so a lane
     * stays within a row): the lane's first element (y, z) moves to
     * y * ozs + z; the padding is never written */
    i64 olane = lane * q.v, oplane = q.plane;
    if (q.ozs != q.nz) {
        const i64 e = lane * q.v, y = e / q.nz;
        olane = y * q.ozs + (e - y * q.nz);
        oplane = (q.plane / q.nz) * q.ozs;
    }
    if constexpr (sizeof(sfx_t) == 4) {
        if (q.v == 2) sfx_batch_lane<2>(q, lane, olane, oplane, t);
        else sfx_batch_lane<1>(q, lane, olane, oplane, t);
    } else {
        if (q.v == 2) sfx_batch_lane<2>(q, lane, olane, oplane, t);
        else {
            /* two-byte lanes are below the cp.async size: register ring */
            const sfx_t *p = reinterpret_cast<const sfx_t *>(q.src) + lane;
            sfx_lane<1>(p, q.dst, olane, q.nx, q.plane, oplane, q.x0, q.x1, t);
        }
    }
}
#endif /* SF_KERNEL_XBATCH */

/* ======================================================================= */
#if defined(SF_KERNEL_DETECT) || defined(SF_KERNEL_FILTER) || defined(SF_KERNEL_PERSIST) || defined(SF_KERNEL_TC)
#ifndef SFD_X2
#define SFD_X2 0
#endif
#ifndef SFD_WEIGHTED
#define SFD_WEIGHTED 0   /* Eq. 1: inputs come as (denominator, numerator) pairs */
#endif
/* Prelude: SFD_WY, SFD_WZ (tile of one plane), SFD_P (z outputs per thread),
 * SFD_THREADS (= WY*WZ/P), SFD_NSRC, SFD_NZF, SFD_RYM, SFD_RZM, SFD_HZ (z halo,
 * multiple of 4 and of SFD_CH), SFD_CH (elements per cp.async, 0 = synchronous
 * element loads), SFD_SROW, SFD_UROW, SFD_PY, SFD_SOURCES(X) with
 * X(index, RY, NZ, RZ0, RZ1, RZ2, RZ3), typedef sfd_t; DETECT adds SFD_WX,
 * SFD_TMA and the shared-memory offsets.
 *
 * Thread layout of the z pass: warp w, lane l owns row 8*(w % (WY/8)) + (l&7)
 * and the chunk of P consecutive z numbered 4*(w / (WY/8)) + (l>>3); the eight
 * lanes of one shared-memory phase read eight rows of one chunk, conflict-free
 * because the row strides hold an odd number of 16-byte words. */

constexpr int SFD_UW = SFD_WZ + 2 * SFD_HZ;   /* staged columns: z0-HZ .. z0+WZ+HZ */
constexpr int SFD_NWARP = SFD_THREADS / 32;

struct sfd_taps {
    float gy[SFD_NSRC][SFD_RYM + 1];             /* y taps by |offset| */
    float gz[SFD_NSRC][SFD_NZF][SFD_RZM + 1];    /* z taps by |offset| */
};

__device__ __forceinline__ u32 sf_smem_addr(const void *p)
{
    return (u32)__cvta_generic_to_shared(p);
}

template <int BYTES>
__device__ __forceinline__ void sf_cp_async(u32 dst, const void *src, u32 n)
{
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(dst), "l"(src),
                     "n"(BYTES), "r"(n)
                     : "memory");
}
__device__ __forceinline__ void sf_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void sf_cp_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

/* Stage rows y0-RY .. y0+WY+RY-1 and columns z0-HZ .. z0+WZ+HZ-1 of plane x
 * of `src` into `slab` (row stride SFD_SROW); zeros outside the cube. */
template <int RY>
__device__ __forceinline__ void sfd_load_slab(sfd_t *slab, const sfd_t *__restrict__ src, i64 x,
                                              i64 y0, i64 z0, i64 nx, i64 ny, i64 nz)
{
    /* one warp per slab row, lanes over the row's chunks: no index division */
    constexpr int ROWS = SFD_WY + 2 * RY;
    constexpr int NWARPS = SFD_THREADS / 32;
    const int lane = threadIdx.x & 31;
    const bool xin = x >= 0 && x < nx;
    if constexpr (SFD_CH > 0) {
        constexpr int CHE = SFD_CH > 0 ? SFD_CH : 1;   /* non-dependent: keep it defined */
        constexpr int NCH = SFD_UW / CHE;
        constexpr int BYTES = CHE * (int)sizeof(sfd_t);
        for (int r = threadIdx.x >> 5; r < ROWS; r += NWARPS) {
            const i64 y = y0 - RY + r;
            const bool rin = xin && y >= 0 && y < ny;
            const sfd_t *row = rin ? src + (x * ny + y) * nz : src;
            const u32 dst = sf_smem_addr(slab + r * SFD_SROW);
            for (int ch = lane; ch < NCH; ch += 32) {
                const i64 z = z0 - SFD_HZ + (i64)ch * CHE;
                const bool in = rin && z >= 0 && z + CHE <= nz;
                sf_cp_async<BYTES>(dst + (u32)(ch * BYTES), in ? row + z : src, in ? BYTES : 0u);
            }
        }
    } else {
        /* element loads for 16-bit storage with an odd nz (no 4-byte chunks) */
        for (int r = threadIdx.x >> 5; r < ROWS; r += NWARPS) {
            const i64 y = y0 - RY + r;
            const bool rin = xin && y >= 0 && y < ny;
            const sfd_t *row = rin ? src + (x * ny + y) * nz : src;
            for (int c = lane; c < SFD_UW; c += 32) {
                const i64 z = z0 - SFD_HZ + c;
                sfd_t v;
                if (rin && z >= 0 && z < nz) v = row[z];
                else *reinterpret_cast<u16 *>(&v) = 0;
                slab[r * SFD_SROW + c] = v;
            }
        }
    }
}

/* U[y][c] = sum_j gy[|j|] slab[y + RY + j][c] for the WY output rows and all
 * SFD_UW staged columns (the z halo is needed by the z pass). */
template <int SI, int RY>
__device__ __forceinline__ void sfd_yfilter(const sfd_t *slab, float *U, const sfd_taps &t)
{
    constexpr int NQ = SFD_UW / 4;
    constexpr int NRB = SFD_WY / SFD_PY;
    for (int task = threadIdx.x; task < NRB * NQ; task += SFD_THREADS) {
        const int rb = task / NQ, q = task - rb * NQ;
        float acc[SFD_PY][4];
#pragma unroll
        for (int i = 0; i < SFD_PY; ++i)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[i][c] = 0.f;
#pragma unroll
        for (int r = 0; r < SFD_PY + 2 * RY; ++r) {
            float v[4];
            sf_ld<sfd_t, 4, false>(slab + (rb * SFD_PY + r) * SFD_SROW + 4 * q, v);
#pragma unroll
            for (int i = 0; i < SFD_PY; ++i) {
                const int j = r - i;   /* slab row r feeds output row i at offset j-RY */
                if (j >= 0 && j <= 2 * RY) {
                    const float g = t.gy[SI][j >= RY ? j - RY : RY - j];
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[i][c] = fmaf(g, v[c], acc[i][c]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < SFD_PY; ++i) sf_st<float, 4>(U + (rb * SFD_PY + i) * SFD_UROW + 4 * q, acc[i]);
    }
}

__host__ __device__ constexpr int sfd_max4(int a, int b, int c, int d)
{
    return (a > b ? a : b) > (c > d ? c : d) ? (a > b ? a : b) : (c > d ? c : d);
}
__host__ __device__ constexpr int sfd_pick(int f, int a, int b, int c, int d)
{
    return f == 0 ? a : f == 1 ? b : f == 2 ? c : d;
}

/* four consecutive staged elements as two pairs (low, high) */
template <class T>
__device__ __forceinline__ void sf_ld_pairs(const T *p, f2 &lo, f2 &hi)
{
    if constexpr (sf_is_f32<T>::v) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(p);
        lo = v.x;
        hi = v.y;
    } else {
        float o[4];
        sf_ld<T, 4, false>(p, o);
        lo = f2_pack(o[0], o[1]);
        hi = f2_pack(o[2], o[3]);
    }
}

/* y filter with column pairs: the same taps as sfd_yfilter, two columns per
 * instruction. */
template <int SI, int RY>
__device__ __forceinline__ void sfd_yfilter2(const sfd_t *slab, float *U, const sfd_taps &t)
{
    constexpr int NQ = SFD_UW / 4;
    constexpr int NRB = SFD_WY / SFD_PY;
    for (int task = threadIdx.x; task < NRB * NQ; task += SFD_THREADS) {
        const int rb = task / NQ, q = task - rb * NQ;
        f2 acc[SFD_PY][2];
#pragma unroll
        for (int i = 0; i < SFD_PY; ++i) acc[i][0] = acc[i][1] = 0ull;
#pragma unroll
        for (int r = 0; r < SFD_PY + 2 * RY; ++r) {
            f2 v0, v1;
            sf_ld_pairs<sfd_t>(slab + (rb * SFD_PY + r) * SFD_SROW + 4 * q, v0, v1);
#pragma unroll
            for (int i = 0; i < SFD_PY; ++i) {
                const int j = r - i;
                if (j >= 0 && j <= 2 * RY) {
                    const float g = t.gy[SI][j >= RY ? j - RY : RY - j];
                    const f2 G = f2_pack(g, g);
                    acc[i][0] = f2_fma(G, v0, acc[i][0]);
                    acc[i][1] = f2_fma(G, v1, acc[i][1]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < SFD_PY; ++i)
            *reinterpret_cast<ulonglong2 *>(U + (rb * SFD_PY + i) * SFD_UROW + 4 * q) =
                make_ulonglong2(acc[i][0], acc[i][1]);
    }
}

/* z filters with output pairs (z, z+1): pair sums of aligned element pairs for
 * even taps, of pairs shifted by one element for odd taps. */
template <int SI, int RY, int NZ, int RZ0, int RZ1, int RZ2, int RZ3>
__device__ __forceinline__ void sfd_zfilter2(const sfd_t *slab, const float *U, int row, int chunk,
                                             float (&c)[SFD_NZF][SFD_P], const sfd_taps &t)
{
    static_assert(SFD_P % 2 == 0, "output pairs");
    constexpr int RZM = sfd_max4(RZ0, RZ1, RZ2, RZ3);
    constexpr int LO = (SFD_HZ - RZM) & ~3;
    constexpr int HI = SFD_HZ + SFD_P - 1 + RZM;
    constexpr int NQ = (HI - LO) / 4 + 1;
    f2 E[2 * NQ];          /* E[k] = (in[2k], in[2k+1]) */
    if constexpr (RY > 0) {
        const float *p = U + row * SFD_UROW + SFD_P * chunk + LO;
#pragma unroll
        for (int q = 0; q < NQ; ++q) sf_ld_pairs<float>(p + 4 * q, E[2 * q], E[2 * q + 1]);
    } else {
        const sfd_t *p = slab + row * SFD_SROW + SFD_P * chunk + LO;
#pragma unroll
        for (int q = 0; q < NQ; ++q) sf_ld_pairs<sfd_t>(p + 4 * q, E[2 * q], E[2 * q + 1]);
    }
    f2 O[2 * NQ - 1];      /* O[k] = (in[2k+1], in[2k+2]) */
#pragma unroll
    for (int k = 0; k < 2 * NQ - 1; ++k) O[k] = f2_pack(f2_hi(E[k]), f2_lo(E[k + 1]));
    f2 acc[SFD_NZF][SFD_P / 2];
#pragma unroll
    for (int j = 0; j <= RZM; ++j) {
#pragma unroll
        for (int m = 0; m < SFD_P / 2; ++m) {
            const int ci = SFD_HZ + 2 * m - LO;       /* even */
            f2 ps;
            if (j == 0) ps = E[ci / 2];
            else if ((j & 1) == 0) ps = f2_add(E[(ci - j) / 2], E[(ci + j) / 2]);
            else ps = f2_add(O[(ci - j - 1) / 2], O[(ci + j - 1) / 2]);
#pragma unroll
            for (int f = 0; f < NZ; ++f) {
                if (j <= sfd_pick(f, RZ0, RZ1, RZ2, RZ3)) {
                    const float g = t.gz[SI][f][j];
                    const f2 G = f2_pack(g, g);
                    acc[f][m] = j == 0 ? f2_mul(G, ps) : f2_fma(G, ps, acc[f][m]);
                }
            }
        }
    }
#pragma unroll
    for (int f = 0; f < NZ; ++f)
#pragma unroll
        for (int m = 0; m < SFD_P / 2; ++m) {
            c[f][2 * m] = f2_lo(acc[f][m]);
            c[f][2 * m + 1] = f2_hi(acc[f][m]);
        }
}

/* SFD_P consecutive z outputs (z0 + P*chunk ...) of row `row` for the NZ
 * spectral filters of input SI: c[f][i] = sum_o gz_f[|o|] u[z + o].  The
 * symmetric taps are applied to pair sums u[z-o] + u[z+o] shared by the NZ
 * filters of this input. */
template <int SI, int RY, int NZ, int RZ0, int RZ1, int RZ2, int RZ3>
__device__ __forceinline__ void sfd_zfilter(const sfd_t *slab, const float *U, int row, int chunk,
                                            float (&c)[SFD_NZF][SFD_P], const sfd_taps &t)
{
    constexpr int RZM = sfd_max4(RZ0, RZ1, RZ2, RZ3);
    constexpr int LO = (SFD_HZ - RZM) & ~3;           /* first staged column used (aligned) */
    constexpr int HI = SFD_HZ + SFD_P - 1 + RZM;       /* last staged column used */
    constexpr int NQ = (HI - LO) / 4 + 1;
    float in[NQ * 4];
    if constexpr (RY > 0) {
        const float *p = U + row * SFD_UROW + SFD_P * chunk + LO;
#pragma unroll
        for (int q = 0; q < NQ; ++q) sf_ld<float, 4, false>(p + 4 * q, in + 4 * q);
    } else {
        const sfd_t *p = slab + row * SFD_SROW + SFD_P * chunk + LO;
#pragma unroll
        for (int q = 0; q < NQ; ++q) sf_ld<sfd_t, 4, false>(p + 4 * q, in + 4 * q);
    }
#pragma unroll
    for (int i = 0; i < SFD_P; ++i) {
        const int ci = SFD_HZ + i - LO;
        float ps[RZM + 1];
        ps[0] = in[ci];
#pragma unroll
        for (int j = 1; j <= RZM; ++j) ps[j] = in[ci - j] + in[ci + j];
#pragma unroll
        for (int f = 0; f < NZ; ++f) {
            float acc = t.gz[SI][f][0] * ps[0];
#pragma unroll
            for (int j = 1; j <= sfd_pick(f, RZ0, RZ1, RZ2, RZ3); ++j)
                acc = fmaf(t.gz[SI][f][j], ps[j], acc);
            c[f][i] = acc;
        }
    }
}
#endif

/* ======================================================================= */
#if defined(SF_KERNEL_DETECT) || defined(SF_KERNEL_PERSIST) || defined(SF_KERNEL_TC)
/*
 * sf_window_detect: one CTA per statistics window (grid = number of windows).
 * For every input cube of the plan (the cube itself, then each x-filtered
 * scratch cube), with the window's x-planes streamed through a double-buffered
 * slab in shared memory:
 *   pass 1  y and z filters of every plane, per-thread moments of the
 *           filtered values, and the maximum of each plane per filter;
 *           the moments are merged (Chan et al.) into the window mean and
 *           standard deviation and the thresholds T_f = mean_f + k std_f;
 *   pass 2  only the planes whose maximum exceeds T_f for some filter can
 *           hold a selected voxel: those planes are filtered again (the same
 *           arithmetic, so the same values) and c_f > T_f is OR-ed into the
 *           window's mask words kept in shared memory.
 * The mask words of the window are written once at the end.  Slabs arrive by
 * TMA (cp.async.bulk.tensor, zero fill outside the cube) when the cube's
 * rows are 16-byte multiples, else by cp.async.  Every wait on a TMA
 * transaction is bounded by %globaltimer (the limit comes with the
 * arguments); on expiry the CTA records the failure in *err and leaves.
 */
struct __align__(64) sf_tmap { unsigned long long opaque[16]; };

struct sfw_maps { sf_tmap m[SFD_NSRC]; };

constexpr int SFW_RG = SFD_WY / 8;                 /* row groups of 8 */
constexpr int SFW_LPW = 32 / SFD_P;                /* lanes per 32-z mask word */
constexpr int SFW_NW = SFD_WZ / 32;                /* mask words per window row */
#ifndef SFD_ZMAP
#define SFD_ZMAP 0
#endif
constexpr int SFW_RPW = 32 / (SFD_WZ / SFD_P);     /* rows per warp (layout 1) */
/* lanes of one mask word: stride SFW_LST, position sfw_la(lane) */
constexpr int SFW_LST = SFD_ZMAP == 1 ? 1 : 8;
__device__ __forceinline__ int sfw_la(int lane)
{
    return SFD_ZMAP == 1 ? lane % SFW_LPW : (lane >> 3) % SFW_LPW;
}
constexpr int SFW_SLAB_STRIDE = (SFD_OFF_SLAB1 - SFD_OFF_SLAB0) / (int)sizeof(sfd_t);

/* the type of the moment merge: FP32, or FP64 for the combine of the
 * per-thread FP32 partial sums (configuration stats_fp64) */
#ifndef SFD_STATS64
#define SFD_STATS64 0
#endif
#ifndef SFD_DDOF
#define SFD_DDOF 0   /* std over n - SFD_DDOF (1: sample std) */
#endif
#if SFD_STATS64
typedef double sfd_st;
#else
typedef float sfd_st;
#endif
struct sfd_mom { sfd_st n, mean, m2; };

__device__ __forceinline__ sfd_mom sfd_merge(sfd_mom a, sfd_mom b)
{
    if (b.n == 0) return a;
    if (a.n == 0) return b;
    const sfd_st n = a.n + b.n;
    const sfd_st d = b.mean - a.mean;
    const sfd_st wb = b.n / n;
    sfd_mom r;
    r.n = n;
    r.mean = fma(d, wb, a.mean);
    r.m2 = a.m2 + b.m2 + d * d * a.n * wb;
    return r;
}

__device__ __forceinline__ unsigned long long sfw_clock()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool sfw_try_wait(u32 bar, u32 parity)
{
    u32 ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

/* wait for phase `parity` of the barrier; false after `limit` ns */
__device__ __forceinline__ bool sfw_wait(u32 bar, u32 parity, unsigned long long limit)
{
    if (sfw_try_wait(bar, parity)) return true;
    const unsigned long long t0 = sfw_clock();
    while (!sfw_try_wait(bar, parity))
        if (sfw_clock() - t0 > limit) return false;
    return true;
}

/* plane maxima: a three-input max and one warp-wide reduction instruction
 * (sm_100a and later), or the two-input max and a shuffle tree */
#ifndef SFD_FASTMAX
#define SFD_FASTMAX 1
#endif
__device__ __forceinline__ float sfw_max3(float a, float b, float c)
{
#if SFD_FASTMAX
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
#else
    return fmaxf(a, fmaxf(b, c));
#endif
}
__device__ __forceinline__ float sfw_warp_max(float v)
{
#if SFD_FASTMAX
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
#else
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
#endif
}

struct sfw_state {
    sfd_t *slab0;
    float *U;
    float *pmax;    /* [WX][NWARP][NZF] */
    u32 *mask;      /* [WX][WY][NW] */
    sfd_st *red;    /* [NWARP][NZF][3] */
    float *thr;     /* [NZF] */
    u32 *flags;     /* [2] planes flagged for pass 2 (bit p) */
    u32 bar;        /* two mbarriers, 8 bytes apart */
    u32 phase;      /* bit b: parity of the next completion of barrier b */
    i64 x0, y0, z0;
    int npl, wid, row, chunk;
    u32 vmask;      /* valid outputs among this thread's P */
    int it;         /* slab loads issued so far (buffer = it & 1) */
    bool dead;
    bool tma;       /* slabs arrive by TMA (else cp.async) */
    unsigned long long limit;   /* bounded waits give up after this many ns */
};

/* TMA or cp.async slabs: fixed by the plan, or per cube in the persistent kernel */
__device__ __forceinline__ bool sfw_tma(const sfw_state &S)
{
#if defined(SF_KERNEL_PERSIST)
    return S.tma;
#else
    (void)S;
    return SFD_TMA != 0;
#endif
}

/* Load plane x0+p of input s into buffer b. */
template <int IDX, int RY>
__device__ __forceinline__ void sfw_load(const sf_dargs &a, const sf_tmap *mp, sfw_state &S, int p,
                                         int b)
{
    sfd_t *dst = S.slab0 + b * SFW_SLAB_STRIDE;
    if (sfw_tma(S)) {
        if (threadIdx.x != 0) return;
        constexpr u32 BYTES = (u32)(SFD_SROW * (SFD_WY + 2 * RY) * sizeof(sfd_t));
        const u32 bar = S.bar + 8u * (u32)b;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(BYTES)
                     : "memory");
        const int cz = (int)(S.z0 - SFD_HZ), cy = (int)(S.y0 - RY), cx = (int)(S.x0 + p);
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(sf_smem_addr(dst)),
            "l"(reinterpret_cast<unsigned long long>(mp + IDX)), "r"(cz), "r"(cy), "r"(cx),
            "r"(bar)
            : "memory");
    } else {
        sfd_load_slab<RY>(dst, reinterpret_cast<const sfd_t *>(a.src[IDX]), S.x0 + p, S.y0, S.z0,
                          a.nx, a.ny, a.nz);
        sf_cp_commit();
    }
}

/* Wait for buffer b (loaded by this CTA); `more` = another load is in flight. */
__device__ __forceinline__ bool sfw_wait_buf(sfw_state &S, int b, bool more)
{
    if (sfw_tma(S)) {
        const bool ok = sfw_wait(S.bar + 8u * (u32)b, (S.phase >> b) & 1u, S.limit);
        S.phase ^= 1u << b;
        return ok;
    }
    if (more) sf_cp_wait<1>();
    else sf_cp_wait<0>();
    return true;
}

/* filtered values of this thread's outputs for plane buffer b */
template <int IDX, int RY, int NZ, int RZ0, int RZ1, int RZ2, int RZ3>
__device__ __forceinline__ void sfw_plane(const sfd_taps &t, sfw_state &S, int b,
                                          float (&c)[SFD_NZF][SFD_P])
{
    const sfd_t *slab = S.slab0 + b * SFW_SLAB_STRIDE;
#if SFD_X2
    if constexpr (RY > 0) {
        sfd_yfilter2<IDX, RY>(slab, S.U, t);
        __syncthreads();
    }
    sfd_zfilter2<IDX, RY, NZ, RZ0, RZ1, RZ2, RZ3>(slab, S.U, S.row, S.chunk, c, t);
#else
    if constexpr (RY > 0) {
        sfd_yfilter<IDX, RY>(slab, S.U, t);
        __syncthreads();
    }
    sfd_zfilter<IDX, RY, NZ, RZ0, RZ1, RZ2, RZ3>(slab, S.U, S.row, S.chunk, c, t);
#endif
}

/* the next input's first load, issued while this input finishes */
template <int IDX> __device__ __forceinline__ void sfw_first_load(const sf_dargs &a, const sf_tmap *mp,
                                                                  sfw_state &S, int b);

template <int IDX, int RY, int NZ, int RZ0, int RZ1, int RZ2, int RZ3>
__device__ __forceinline__ void sfw_input(const sf_dargs &a, const sfd_taps &t, const sf_tmap *mp,
                                          sfw_state &S)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr u32 FULL = SFD_P == 32 ? 0xffffffffu : ((1u << SFD_P) - 1u);
    constexpr int NEXT = SFD_WEIGHTED ? IDX + 2 : IDX + 1;   /* the next input (pair) */
    const bool full = S.vmask == FULL;
    /* per-thread shifted sums: K = the thread's first value of the window */
    float K[SFD_NZF], s1[SFD_NZF], s2[SFD_NZF];
    int cnt = 0;
#pragma unroll
    for (int f = 0; f < SFD_NZF; ++f) { K[f] = 0.f; s1[f] = 0.f; s2[f] = 0.f; }
    float T[SFD_NZF];
#pragma unroll
    for (int f = 0; f < SFD_NZF; ++f) T[f] = 0.f;
    u32 fl0 = 0u, fl1 = 0u;
    /* first flagged plane after `after` (-1: the first one), -1 when none */
    auto next_flag = [&](int after) -> int {
        const int from = after + 1;
        if (from < 32) {
            const u32 m = fl0 & ~((1u << from) - 1u);
            if (m) return __ffs(m) - 1;
        }
        const int lo = from - 32;
        const u32 m1 = lo <= 0 ? fl1 : (lo >= 32 ? 0u : (fl1 & ~((1u << lo) - 1u)));
        return m1 ? 32 + __ffs(m1) - 1 : -1;
    };

    /* One loop over the items of both passes, so the filter code exists once:
     * pass 1 visits planes 0..npl-1 (plane 0 was issued already), pass 2 the
     * flagged planes. */
    bool pass2 = false;
    int p = 0;
    f2 s1p[SFD_NZF], s2p[SFD_NZF];   /* packed partial sums of the full-tile path */
#pragma unroll
    for (int f = 0; f < SFD_NZF; ++f) s1p[f] = s2p[f] = 0ull;
    while (true) {
        const int b = S.it & 1;
        int np = -1;
        if (!pass2) np = p + 1 < S.npl ? p + 1 : -1;
        else np = next_flag(p);
        float c[SFD_NZF][SFD_P];
#if SFD_WEIGHTED
        {
            /* Eq. 1: the denominator source IDX, then the numerator source
             * IDX+1 of the same plane, each through the buffer ring; the
             * denominator's filtered values wait in registers */
            const bool ok = sfw_wait_buf(S, b, false);
            if (__syncthreads_or(!ok)) { S.dead = true; return; }
            sfw_load<IDX + 1, RY>(a, mp, S, p, b ^ 1);
            float cd[SFD_NZF][SFD_P];
            sfw_plane<IDX, RY, NZ, RZ0, RZ1, RZ2, RZ3>(t, S, b, cd);
            ++S.it;
            const int b2 = b ^ 1;
            const bool ok2 = sfw_wait_buf(S, b2, false);
            if (__syncthreads_or(!ok2)) { S.dead = true; return; }
            if (np >= 0) sfw_load<IDX, RY>(a, mp, S, np, b);
            else if (pass2 && NEXT < SFD_NSRC) sfw_first_load<NEXT>(a, mp, S, b);
            sfw_plane<IDX + 1, RY, NZ, RZ0, RZ1, RZ2, RZ3>(t, S, b2, c);
#pragma unroll
            for (int f = 0; f < NZ; ++f)
#pragma unroll
                for (int i = 0; i < SFD_P; ++i) c[f][i] = cd[f][i] != 0.f ? c[f][i] / cd[f][i] : 0.f;
        }
#else
        /* wait for this plane, then (everyone being past the previous plane)
         * start the next load into the other buffer */
        const bool ok = sfw_wait_buf(S, b, false);
        if (__syncthreads_or(!ok)) { S.dead = true; return; }
        if (np >= 0) sfw_load<IDX, RY>(a, mp, S, np, b ^ 1);
        else if (pass2 && NEXT < SFD_NSRC) sfw_first_load<NEXT>(a, mp, S, b ^ 1);
        sfw_plane<IDX, RY, NZ, RZ0, RZ1, RZ2, RZ3>(t, S, b, c);
#endif
        if (!pass2) {
            if (p == 0) {
#pragma unroll
                for (int f = 0; f < NZ; ++f) K[f] = c[f][0];
            }
#pragma unroll
            for (int f = 0; f < NZ; ++f) {
                float mx = -3.402823466e38f;
                if (full) {
                    const f2 NK = f2_pack(-K[f], -K[f]);
#pragma unroll
                    for (int i = 0; i < SFD_P; i += 2) {
                        const f2 d = f2_add(f2_pack(c[f][i], c[f][i + 1]), NK);
                        s1p[f] = f2_add(s1p[f], d);
                        s2p[f] = f2_fma(d, d, s2p[f]);
                        mx = sfw_max3(mx, c[f][i], c[f][i + 1]);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < SFD_P; ++i)
                        if (S.vmask & (1u << i)) {
                            const float d = c[f][i] - K[f];
                            s1[f] += d;
                            s2[f] = fmaf(d, d, s2[f]);
                            mx = fmaxf(mx, c[f][i]);
                        }
                }
                mx = sfw_warp_max(mx);
                if (lane == 0) S.pmax[(p * SFD_NWARP + warp) * SFD_NZF + f] = mx;
            }
            cnt += __popc(S.vmask);
        } else {
            u32 bits = 0;
#pragma unroll
            for (int f = 0; f < NZ; ++f)
#pragma unroll
                for (int i = 0; i < SFD_P; ++i) bits |= (c[f][i] > T[f] ? 1u : 0u) << i;
            bits &= S.vmask;
            /* the SFW_LPW lanes of one 32-z word combine their pieces */
            u32 word = bits << (SFD_P * sfw_la(lane));
#pragma unroll
            for (int off = SFW_LST; off < SFW_LST * SFW_LPW; off <<= 1)
                word |= __shfl_xor_sync(0xffffffffu, word, off);
            if (sfw_la(lane) == 0) {
                u32 *mw = S.mask + (p * SFD_WY + S.row) * SFW_NW + (S.chunk * SFD_P) / 32;
                *mw |= word;
            }
        }
        ++S.it;

        if (!pass2 && np < 0) {
            /* end of pass 1: window statistics, thresholds, flagged planes */
#pragma unroll
            for (int f = 0; f < NZ; ++f) {
                s1[f] += f2_lo(s1p[f]) + f2_hi(s1p[f]);
                s2[f] += f2_lo(s2p[f]) + f2_hi(s2p[f]);
                sfd_mom m{0, 0, 0};
#if SFD_STATS64
                {
                    /* FP64 combine: the thread's FP32 sums about its own shift
                     * K are moved to the warp's shift R (lane 0's K),
                     *   sum (c - R)   = s1 + n (K - R),
                     *   sum (c - R)^2 = s2 + (K - R)(2 s1 + n (K - R)),
                     * summed over the warp in FP64, then turned into moments */
                    const float R = __shfl_sync(0xffffffffu, K[f], 0);
                    const double n = (double)cnt, dk = (double)K[f] - (double)R;
                    double t1 = (double)s1[f] + n * dk;
                    double t2 = (double)s2[f] + dk * (2.0 * (double)s1[f] + n * dk);
                    float nw = (float)cnt;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        t1 += __shfl_xor_sync(0xffffffffu, t1, off);
                        t2 += __shfl_xor_sync(0xffffffffu, t2, off);
                        nw += __shfl_xor_sync(0xffffffffu, nw, off);
                    }
                    if (nw > 0.f) {
                        const double mu = t1 / (double)nw;
                        m = sfd_mom{(double)nw, (double)R + mu, fmax(t2 - t1 * mu, 0.0)};
                    }
                }
#else
                if (cnt > 0) {
                    const sfd_st n = (sfd_st)cnt, mu = (sfd_st)s1[f] / n;
                    m = sfd_mom{n, (sfd_st)K[f] + mu, fmax((sfd_st)s2[f] - (sfd_st)s1[f] * mu, (sfd_st)0)};
                }
                /* rolled: once per input and window, and every input's copy
                 * of the kernel carries it (smaller code, fewer fetch stalls) */
#pragma unroll 1
                for (int off = 1; off < 32; off <<= 1) {
                    sfd_mom o;
                    o.n = __shfl_xor_sync(0xffffffffu, m.n, off);
                    o.mean = __shfl_xor_sync(0xffffffffu, m.mean, off);
                    o.m2 = __shfl_xor_sync(0xffffffffu, m.m2, off);
                    m = (lane & off) ? sfd_merge(o, m) : sfd_merge(m, o);
                }
#endif
                if (lane == 0) {
                    sfd_st *w = S.red + (warp * SFD_NZF + f) * 3;
                    w[0] = m.n; w[1] = m.mean; w[2] = m.m2;
                }
            }
            __syncthreads();
            if (threadIdx.x < NZ) {
                const int f = threadIdx.x;
                sfd_mom m{0, 0, 0};
                for (int w = 0; w < SFD_NWARP; ++w) {
                    const sfd_st *q = S.red + (w * SFD_NZF + f) * 3;
                    m = sfd_merge(m, sfd_mom{q[0], q[1], q[2]});
                }
                const sfd_st sd = m.n > SFD_DDOF ? sqrt(m.m2 / (m.n - SFD_DDOF)) : (sfd_st)0;
                /* the threshold in the merge's precision, rounded once */
                S.thr[f] = (float)fma((sfd_st)a.k, sd, m.mean);
                if (a.mean != nullptr) {
                    const i64 o = (i64)a.fidx[IDX][f] * a.nwin + S.wid;
                    a.mean[o] = (float)m.mean;
                    a.stdv[o] = (float)sd;
                }
            }
            __syncthreads();
            if (warp == 0) {
                for (int base = 0; base < SFD_WX; base += 32) {
                    const int q = base + lane;
                    bool hot = false;
                    if (q < S.npl)
                        for (int w = 0; w < SFD_NWARP; ++w)
#pragma unroll
                            for (int f = 0; f < NZ; ++f)
                                hot |= S.pmax[(q * SFD_NWARP + w) * SFD_NZF + f] > S.thr[f];
                    const u32 bits = __ballot_sync(0xffffffffu, hot);
                    if (lane == 0) S.flags[base >> 5] = bits;
                }
            }
            __syncthreads();
            fl0 = S.flags[0];
            fl1 = SFD_WX > 32 ? S.flags[1] : 0u;
#pragma unroll
            for (int f = 0; f < NZ; ++f) T[f] = S.thr[f];
            pass2 = true;
            p = next_flag(-1);
            if (p < 0) {
                /* nothing can be selected in this window for this input */
                if (NEXT < SFD_NSRC) sfw_first_load<NEXT>(a, mp, S, S.it & 1);
                return;
            }
            sfw_load<IDX, RY>(a, mp, S, p, S.it & 1);
            continue;
        }
        if (pass2 && np < 0) return;
        p = np;
    }
}

#define SFW_FIRST(IDX, RY, NZ, RZ0, RZ1, RZ2, RZ3)                                               \
    template <> __device__ __forceinline__ void sfw_first_load<IDX>(const sf_dargs &a,             \
                                                                    const sf_tmap *mp,            \
                                                                    sfw_state &S, int b)           \
    {                                                                                              \
        sfw_load<IDX, RY>(a, mp, S, 0, b);                                                         \
    }
SFD_SOURCES(SFW_FIRST)
#undef SFW_FIRST
template <int IDX> __device__ __forceinline__ void sfw_first_load(const sf_dargs &, const sf_tmap *,
                                                                  sfw_state &, int)
{
}

/* one input, or (Eq. 1) one (denominator, numerator) pair starting at an
 * even index */
template <int IDX, int RY, int NZ, int RZ0, int RZ1, int RZ2, int RZ3>
__device__ __forceinline__ void sfw_run(const sf_dargs &a, const sfd_taps &t, const sf_tmap *mp,
                                        sfw_state &S)
{
    if constexpr (SFD_WEIGHTED == 0 || IDX % 2 == 0) sfw_input<IDX, RY, NZ, RZ0, RZ1, RZ2, RZ3>(a, t, mp, S);
}

/* shared-memory carve-up, thread roles and barrier set-up (once per CTA) */
__device__ __forceinline__ void sfw_init(sfw_state &S, unsigned char *raw, bool barriers = true)
{
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<unsigned long long>(raw) + 127ull) & ~127ull);
    S.slab0 = reinterpret_cast<sfd_t *>(sm + SFD_OFF_SLAB0);
    S.U = reinterpret_cast<float *>(sm + SFD_OFF_U);
    S.pmax = reinterpret_cast<float *>(sm + SFD_OFF_PMAX);
    S.mask = reinterpret_cast<u32 *>(sm + SFD_OFF_MASK);
    S.red = reinterpret_cast<sfd_st *>(sm + SFD_OFF_RED);
    S.thr = reinterpret_cast<float *>(sm + SFD_OFF_THR);
    S.flags = reinterpret_cast<u32 *>(sm + SFD_OFF_FLAGS);
    S.bar = sf_smem_addr(sm + SFD_OFF_MBAR);
    S.phase = 0;
    S.dead = false;
    S.tma = SFD_TMA != 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#if SFD_ZMAP == 1
    /* warp w owns whole rows: lane l takes row w*RPW + (l/CA) % RPW and chunk
     * (l % CA) + CA*(l / (CA*RPW)); an 8-lane phase reads four chunks of two rows */
    S.row = warp * SFW_RPW + (lane / SFW_LPW) % SFW_RPW;
    S.chunk = lane % SFW_LPW + SFW_LPW * (lane / (SFW_LPW * SFW_RPW));
#else
    S.row = (warp % SFW_RG) * 8 + (lane & 7);
    S.chunk = (warp / SFW_RG) * 4 + (lane >> 3);
#endif
    if (!barriers) return;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(S.bar) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(S.bar + 8u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

/* One statistics window (index wid of the window grid of the cube `a`
 * describes): both passes for every input, then the window's mask words.
 * Returns false when a bounded wait expired (the CTA must stop). */
__device__ __forceinline__ bool sfw_window(const sf_dargs &a, const sfd_taps &t, const sf_tmap *mp,
                                           sfw_state &S, int wid)
{
    const int lane = threadIdx.x & 31;
    S.wid = wid;
    S.limit = (unsigned long long)a.wait_ns;
    const int wz = wid % a.nwz, wy = (wid / a.nwz) % a.nwy, wx = wid / (a.nwz * a.nwy);
    S.x0 = a.xorg + (i64)wx * SFD_WX;
    S.y0 = (i64)wy * SFD_WY;
    S.z0 = (i64)wz * SFD_WZ;
    const i64 left = a.nx - S.x0;
    S.npl = left < SFD_WX ? (int)left : SFD_WX;
    const bool rowv = S.y0 + S.row < a.ny;
    const i64 zb = S.z0 + (i64)SFD_P * S.chunk;
    S.vmask = 0;
#pragma unroll
    for (int i = 0; i < SFD_P; ++i)
        if (rowv && zb + i < a.nz) S.vmask |= 1u << i;
    S.it = 0;

    __syncthreads();   /* the previous window's mask words have been written out */
    for (int i = threadIdx.x; i < SFD_WX * SFD_WY * SFW_NW; i += SFD_THREADS) S.mask[i] = 0u;
    __syncthreads();
    sfw_first_load<0>(a, mp, S, 0);

#define SFW_RUN(IDX, RY, NZ, RZ0, RZ1, RZ2, RZ3)                                                 \
    if (!S.dead) sfw_run<IDX, RY, NZ, RZ0, RZ1, RZ2, RZ3>(a, t, mp, S);
    SFD_SOURCES(SFW_RUN)
#undef SFW_RUN

    if (S.dead) {
        /* a slab transaction did not complete in time: report it, give the
         * copies still in flight a bounded time to land, and stop */
        if (threadIdx.x == 0) {
            atomicOr(a.err, 1);
            if (S.tma) {
                sfw_wait(S.bar, (S.phase >> 0) & 1u, S.limit);
                sfw_wait(S.bar + 8u, (S.phase >> 1) & 1u, S.limit);
            }
        }
        if (!S.tma) sf_cp_wait<0>();
        return false;
    }
    __syncthreads();
    /* mask words of the window: one owner lane per (row, word) */
    if (sfw_la(lane) == 0 && rowv) {
        const int wd = (S.chunk * SFD_P) / 32;
        const i64 gw = (S.z0 >> 5) + wd;
        if (gw < a.nw32)
            for (int p = 0; p < S.npl; ++p)
                a.mask[((S.x0 - a.xorg + p) * a.ny + S.y0 + S.row) * a.nw32 + gw] =
                    S.mask[(p * SFD_WY + S.row) * SFW_NW + wd];
    }
    return true;
}
#endif

#ifdef SF_KERNEL_DETECT
extern "C" __global__ void __launch_bounds__(SFD_THREADS, SFD_MINB)
sf_window_detect(const __grid_constant__ sf_dargs a, const __grid_constant__ sfd_taps t,
                 const __grid_constant__ sfw_maps mp)
{
    extern __shared__ __align__(128) unsigned char sfw_raw[];
    sfw_state S;
    sfw_init(S, sfw_raw);
    sfw_window(a, t, mp.m, S, a.wid0 + (int)blockIdx.x);
}
#endif /* SF_KERNEL_DETECT */

/* ======================================================================= */
#ifdef SF_KERNEL_PERSIST
#ifndef SFP_XITEMS
#define SFP_XITEMS 1
#endif
/*
 * sf_persist: every unit's windows, and (SFP_XITEMS) its x pass, in one
 * persistent launch.  Without x items the x pass of the batch runs as
 * sf_xpass_batch just before, in the same graph.
 * CTAs pull items from a global counter.  Items are ordered so that all x
 * items of a unit come before its window items; a window item waits (bounded
 * by %globaltimer) until the unit's x items are all complete.  x items never
 * wait, and an item is only ever taken by a running CTA, so every wait ends.
 * HBM-bound x items and ALU-bound window items of different units run side by
 * side on the SMs.
 */
__device__ __forceinline__ bool sfp_wait_count(const int *ctr, int need, unsigned long long limit)
{
    unsigned long long t0 = 0ull;
    while (true) {
        int v;
        asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= need) return true;
        const unsigned long long now = sfw_clock();
        if (t0 == 0ull) t0 = now;
        else if (now - t0 > limit) return false;
        __nanosleep(200);
    }
}

extern "C" __global__ void __launch_bounds__(SFD_THREADS, SFD_MINB)
sf_persist(const __grid_constant__ sf_pargs pa, const __grid_constant__ sfd_taps t,
           const __grid_constant__ sfx_taps xt)
{
    extern __shared__ __align__(128) unsigned char sfp_raw[];
    __shared__ int s_item;
    u32 phase = 0;   /* mbarrier parities, carried from one window item to the next */
    {
        sfw_state S0;
        sfw_init(S0, sfp_raw);
    }
    const sf_tmap *maps = reinterpret_cast<const sf_tmap *>(pa.maps);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(pa.head, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= pa.n_items) break;
        const sf_item it = pa.items[item];
        const sf_unit &u = pa.units[it.unit];
        if (it.kind == 0) {
#if SFP_XITEMS
            /* x pass of lanes [index*xlanes, (index+1)*xlanes) over the unit's planes */
            const i64 l0 = (i64)it.index * u.xlanes;
            const i64 l1 = min(u.lanes, l0 + u.xlanes);
            const sfx_t *src = reinterpret_cast<const sfx_t *>(u.xsrc);
            void *dst[SFX_NOUT];
#pragma unroll
            for (int k = 0; k < SFX_NOUT; ++k) dst[k] = u.xdst[k];
            const i64 nx = u.args.nx, plane = u.plane, x0 = u.x0, x1 = u.x1;
            if (u.xv == 2) {
                for (i64 l = l0 + threadIdx.x; l < l1; l += SFD_THREADS)
                    sfx_lane<2>(src + 2 * l, dst, 2 * l, nx, plane, plane, x0, x1, xt);
            } else {
                for (i64 l = l0 + threadIdx.x; l < l1; l += SFD_THREADS)
                    sfx_lane<1>(src + l, dst, l, nx, plane, plane, x0, x1, xt);
            }
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(pa.xdone + it.unit, 1);
#endif
        } else {
            bool ok = true;
            if (SFP_XITEMS && threadIdx.x == 0) {
                ok = sfp_wait_count(pa.xdone + it.unit, u.n_xitems + pa.xextra,
                                    (unsigned long long)pa.wait_ns);
                /* the x-filtered planes were written through the generic proxy
                 * by other CTAs; order them before this CTA's TMA reads */
                asm volatile("fence.proxy.async.global;" ::: "memory");
            }
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) atomicOr(pa.err, 1);
                return;
            }
            sfw_state S;
            sfw_init(S, sfp_raw, false);
            S.phase = phase;
            S.tma = u.tma != 0;
            const int per = u.args.nwy * u.args.nwz;
            const int wid = (u.wx0 + it.index / per) * per + it.index % per;
            if (!sfw_window(u.args, t, maps + u.map_base, S, wid)) return;
            phase = S.phase;
        }
    }
}
#endif /* SF_KERNEL_PERSIST */

/* ======================================================================= */
#ifdef SF_KERNEL_TC
/*
 * sf_window_tc: the window kernel for 16-bit storage with both spectral (z)
 * and spatial (y) filters on the tensor cores (tcgen05, kind::f16, FP32
 * accumulation in tensor memory).  16-bit values are exact tensor-core
 * operands; every tap is split into two 16-bit parts (hi + lo; the z taps
 * scaled by 2^SFT_SCALE so their low parts stay normal), which carries the
 * taps to about 2^-22.
 *
 * y filter (inputs with sigma_xy > 0), one x-plane at a time: the plane's
 * slab (rows y0-R .. y0+31+R padded to KY, 128 staged columns) arrives by TMA
 * in the 128-byte swizzled layout with z contiguous, which the MMA reads as
 * an MN-major A operand: U^T[z][y] = sum_k slab[k][z] Ty[y][k], M = 128 (z),
 * N = 32 (y), K = KY, into a TMEM accumulator.  Each thread then reads its z
 * column and writes the 32 values, rounded to the storage type, into the z
 * filter's A tile (the y-filtered rows of the plane).
 *
 * z filter, per group of four planes (M = 128 = 4 planes x 32 rows): the
 * z filter of a row is banded: outputs 16j..16j+15 of the window read the
 * staged columns 16j + HZ - R .. 16j + 15 + HZ + R, i.e. the 16-column slices
 * j + s_lo .. j + s_hi, so every output tile multiplies the same 16 x 64
 * Toeplitz tile T[n][k] = g[k - n - HZ] by up to four K-slices of the A tile:
 * one M=128 N=16 K=16 MMA per slice and tap part.  Inputs with sigma_xy = 0
 * load the A tile (four planes) by TMA directly.
 *
 * The z accumulators feed the same per-window work as the CUDA-core kernel:
 * shifted moments and plane maxima (pass 1), the window statistics and
 * thresholds, then the selection bits of the flagged planes (pass 2).
 * Thread (warp w, lane l) owns TMEM lane quarter w % 4 (plane w % 4 of the
 * group, row l) and filter w / 4: 64 outputs per group.  One thread issues
 * the MMAs and commits them to mbarriers; every wait is bounded.
 */
#ifndef SFT_SCALE
#define SFT_SCALE 10
#endif
constexpr int SFT_M = 128;
constexpr int SFT_PLANES = SFT_M / SFD_WY;          /* planes per group (4) */
constexpr int SFT_ATOM = SFT_M * 128;                /* bytes of one 64-column atom of the A tile */
constexpr int SFT_TM_COLS = 256;                     /* z accumulators at 0 and 128; y at 128, 192 */
constexpr int SFT_KYM = (SFD_WY + 2 * SFD_RYM + 15) / 16 * 16;   /* padded slab rows */
constexpr int SFT_SLAB_BYTES = 2 * SFT_KYM * 128;    /* one slab buffer: two 64-column atoms */
constexpr int SFT_NS = 3;                            /* slab buffers: copies two planes ahead */
static_assert(SFD_WY == 32 && SFD_WZ == 64 && SFD_THREADS == 256, "window 32 x 64, 256 threads");
static_assert(SFD_NZF <= 2, "at most two spectral filters per input");
static_assert(SFD_HZ + SFD_RZM <= 48, "band within the 64-column Toeplitz tile");
static_assert(SFT_KYM <= 64, "y filter rows within one 128-byte row of the y tile");

struct sft_tiles {
    unsigned char z[SFT_NZT][2][SFT_ZROWS * 32];       /* z Toeplitz tall tiles: ZROWS x 16, hi and lo */
    unsigned char y[SFT_NYT > 0 ? SFT_NYT : 1][2][4096]; /* y Toeplitz tiles: 32 x 64, hi and lo */
    int zt[SFD_NSRC][SFD_NZF];                          /* z tile of each (input, filter) */
    int yt[SFD_NSRC];                                   /* y tile of each input (-1: none) */
};
struct sft_maps { sf_tmap m[SFD_NSRC]; };
constexpr int SFT_ZT_BYTES = (int)sizeof(((sft_tiles *)0)->z);   /* z tiles: resident */
constexpr int SFT_YT_BYTES = 2 * 4096;                              /* one y tile: staged per input */

__device__ __forceinline__ u32 sft_sw128(u32 row, u32 kbyte)
{
    return (row >> 3) * 1024u + (row & 7u) * 128u + ((((kbyte >> 4) ^ (row & 7u)) & 7u) << 4) + (kbyte & 15u);
}
/* shared-memory matrix descriptor without swizzle (K-major: lbo = stride
 * between the two core matrices along K, sbo = stride between 8-row groups) */
__device__ __forceinline__ unsigned long long sft_desc_plain(u32 addr, u32 lbo, u32 sbo)
{
    return (unsigned long long)((addr >> 4) & 0x3fffu) | ((unsigned long long)((lbo >> 4) & 0x3fffu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}
/* shared-memory matrix descriptor, 128-byte swizzle, version 1: lbo = stride
 * between 64-element atoms along M/N (MN-major operands), sbo = stride
 * between 8-row groups */
__device__ __forceinline__ unsigned long long sft_desc(u32 addr, u32 lbo, u32 sbo)
{
    return (unsigned long long)((addr >> 4) & 0x3fffu) | ((unsigned long long)((lbo >> 4) & 0x3fffu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46) | (2ull << 61);
}
/* kind::f16 instruction descriptors: D FP32, A/B FP16 (0) or BF16 (1);
 * z: both K-major, N = 32 (two output tiles), M = 128; y: A MN-major, N = 64
 * (the 32 outputs against the hi part, then against the lo part), M = 128 */
constexpr u32 SFT_AB = SFT_BF16 ? 1u : 0u;
constexpr u32 SFT_IDESC_Z = (1u << 4) | (SFT_AB << 7) | (SFT_AB << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
constexpr u32 SFT_IDESC_Y =
    (1u << 4) | (SFT_AB << 7) | (SFT_AB << 10) | (1u << 15) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

/* z MMAs: 32 outputs (two 16-output tiles, pair p) per MMA.  Outputs
 * 32p .. 32p+31 read the K-slices sft_zlo(r, p) .. sft_zhi(r, p).  The B
 * operand of (p, slice S) is rows t0 .. t0+31 of the filter's tall tile
 * Tt[t][kk] = g[kk - t + C] (no swizzle, K-major: 8-row groups of two
 * 8 x 16-byte core matrices, 256 bytes apart), t0 = 32p + HZ + C - 16S,
 * C the smallest multiple of 8 that keeps every t0 >= 0. */
__host__ __device__ constexpr int sft_zlo(int r, int p) { return (32 * p + SFD_HZ - r) / 16; }
__host__ __device__ constexpr int sft_zhi(int r, int p) { return (32 * p + 31 + SFD_HZ + r) / 16; }
__host__ __device__ constexpr int sft_zc(int r)
{
    const int m0 = 16 * sft_zhi(r, 0) - SFD_HZ, m1 = 16 * sft_zhi(r, 1) - 32 - SFD_HZ;
    const int m = m0 > m1 ? m0 : m1;
    return m <= 0 ? 0 : (m + 7) / 8 * 8;
}
__host__ __device__ constexpr int sft_zt0(int r, int p, int S) { return 32 * p + SFD_HZ + sft_zc(r) - 16 * S; }
__host__ __device__ constexpr int sft_ky(int ry) { return (SFD_WY + 2 * ry + 15) / 16 * 16; }

struct sft_state {
    unsigned char *A;      /* z-filter A tile: 1024-aligned, two 16 KB atoms */
    unsigned char *T;      /* tap tiles (z then y) */
    unsigned char *slab;   /* y-filter slabs: SFT_NS buffers of SFT_SLAB_BYTES */
    float *pmax;           /* [WX][NZF] */
    u32 *mask;             /* [WX][WY][2] */
    sfd_st *red;           /* [8 warps][3] */
    float *thr;            /* [NZF] */
    u32 *flags;            /* [2] */
    u32 bar_s;             /* slab copies (SFT_NS), 8 bytes apart */
    u32 bar_a;             /* A-tile copies (two buffers: the A tile, and the slab region) */
    u32 bar_z;             /* z-MMA commits (2) */
    u32 bar_y;             /* y-MMA commits (2) */
    u32 ph_s, ph_a, ph_z, ph_y;   /* parity of the next completion, bit per barrier */
    u32 tmem;              /* accumulator base */
    u32 pend;              /* completions awaited: bits 0-2 slabs, 3-4 A tiles, 5-6 z, 7-8 y */
    i64 x0, y0, z0;
    int npl, wid;
    int it;                /* slab copies issued (buffer = it % SFT_NS) */
    int ic;                /* slab planes consumed (buffer = ic % SFT_NS) */
    int ity;               /* y-MMAs issued (accumulator = ity & 1) */
    unsigned long long limit;
    int *err;
    bool dead;
};

/* a bounded wait; on expiry the waiting site is recorded in *err (bit 1:
 * A-tile copy, 2: slab copy, 3: z MMA, 4: y MMA) beside bit 0 */
__device__ __forceinline__ bool sft_wait(sft_state &S, u32 bar, u32 &ph, int b, int site)
{
    const bool ok = sfw_wait(bar + 8u * (u32)b, (ph >> b) & 1u, S.limit);
    ph ^= 1u << b;
    if (!ok) atomicOr(S.err, 1 | (1 << site));
    return ok;
}

/* the slab of plane x0+p of a y-filtered input into buffer b: two boxes
 * {64 columns, KY rows, 1 plane}, 128-byte swizzle */
template <int IDX, int RY>
__device__ __forceinline__ void sft_load_slab(const sft_maps &mp, sft_state &S, int p, int b)
{
    if (threadIdx.x != 0) return;
    constexpr int KY = sft_ky(RY);
    unsigned char *dst = S.slab + b * SFT_SLAB_BYTES;
    const u32 bar = S.bar_s + 8u * (u32)b;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((u32)(2 * KY * 128))
                 : "memory");
    const int cy = (int)(S.y0 - RY), cx = (int)(S.x0 + p);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int cz = (int)(S.z0 - SFD_HZ) + 64 * a;
        asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(sf_smem_addr(dst + a * KY * 128)),
                     "l"(reinterpret_cast<unsigned long long>(&mp.m[IDX])), "r"(cz), "r"(cy), "r"(cx), "r"(bar)
                     : "memory");
    }
}

/* the two atoms of A buffer ab: the A tile (0), or the slab region, idle
 * while a sigma_xy = 0 input runs (1) */
__device__ __forceinline__ unsigned char *sft_abuf(const sft_state &S, int ab) { return ab ? S.slab : S.A; }

/* A tile of group g of a sigma_xy = 0 input into A buffer ab: two swizzled
 * boxes {64, 32, 4} */
template <int IDX>
__device__ __forceinline__ void sft_load_a(const sft_maps &mp, sft_state &S, int g, int ab)
{
    if (threadIdx.x != 0) return;
    const u32 bar = S.bar_a + 8u * (u32)ab;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((u32)(2 * SFT_ATOM))
                 : "memory");
    const int cy = (int)S.y0, cx = (int)(S.x0 + SFT_PLANES * g);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int cz = (int)(S.z0 - SFD_HZ) + 64 * a;
        asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(sf_smem_addr(sft_abuf(S, ab) + a * SFT_ATOM)),
                     "l"(reinterpret_cast<unsigned long long>(&mp.m[IDX])), "r"(cz), "r"(cy), "r"(cx), "r"(bar)
                     : "memory");
    }
}

/* the y-filter MMAs of the plane in slab buffer b into y accumulator yb */
template <int RY>
__device__ __forceinline__ void sft_mma_y(const sft_state &S, const sft_tiles &bt, int SI, int b, int yb)
{
    constexpr int KY = sft_ky(RY);
    /* base descriptors once, compile-time offsets per slice and part */
    const unsigned long long a0 = sft_desc(sf_smem_addr(S.slab + b * SFT_SLAB_BYTES), (u32)(KY * 128), 1024u);
    const unsigned long long t0 = sft_desc(sf_smem_addr(S.T + SFT_ZT_BYTES), 16u, 1024u);   /* this input's y tile */
    (void)bt;
    (void)SI;
    /* the tile's hi and lo parts are 32 rows each, contiguous in the same
     * swizzled layout: one N = 64 MMA per K-slice takes both, into columns
     * 0-31 (hi) and 32-63 (lo) of the accumulator, which the read-out adds */
    const u32 d = S.tmem + 128u + (u32)(yb * 64);
    u32 acc = 0u;
#pragma unroll
    for (int s = 0; s < KY / 16; ++s) {
        const unsigned long long ad = a0 + (unsigned long long)((s * 2048) >> 4);
        const unsigned long long bd = t0 + (unsigned long long)((s * 32) >> 4);
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                     "l"(ad), "l"(bd), "r"(SFT_IDESC_Y), "r"(acc));
        acc = 1u;
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(S.bar_y + 8u * (u32)yb)
                 : "memory");
}

/* the z-filter MMAs of one group into z accumulator buf: for every filter and
 * 16-output tile j, the K-slices j + s_lo .. j + s_hi against the filter's
 * Toeplitz tile, hi and lo parts */
template <int SI, int NZ, int RZ0, int RZ1>
__device__ __forceinline__ void sft_mma_z(const sft_state &S, const sft_tiles &bt, int buf, const unsigned char *A)
{
    /* base descriptors once; every slice's start is a compile-time offset
     * added to the 14-bit address field (shared addresses stay below 2^18) */
    const unsigned long long a0 = sft_desc(sf_smem_addr(A), 16u, 1024u);
#pragma unroll
    for (int f = 0; f < NZ; ++f) {
        constexpr int RA = RZ0, RB = RZ1;
        const unsigned long long t0 =
            sft_desc_plain(sf_smem_addr(S.T + bt.zt[SI][f] * 2 * SFT_ZROWS * 32), 128u, 256u);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const u32 d = S.tmem + (u32)(buf * 128 + f * 64 + p * 32);
            const int lo = f == 0 ? sft_zlo(RA, p) : sft_zlo(RB, p), hi = f == 0 ? sft_zhi(RA, p) : sft_zhi(RB, p);
            u32 acc = 0u;
#pragma unroll
            for (int ts = 0; ts < 7; ++ts) {
                if (ts < lo || ts > hi) continue;
                const int t0r = f == 0 ? sft_zt0(RA, p, ts) : sft_zt0(RB, p, ts);
                const unsigned long long ad = a0 + (unsigned long long)(((ts >> 2) * SFT_ATOM + (ts & 3) * 32) >> 4);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const unsigned long long bd = t0 + (unsigned long long)((h * SFT_ZROWS * 32 + (t0r / 8) * 256) >> 4);
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                                 "l"(ad), "l"(bd), "r"(SFT_IDESC_Z), "r"(acc));
                    acc = 1u;
                }
            }
        }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(S.bar_z + 8u * (u32)buf)
                 : "memory");
}

/* 16 accumulator columns of this thread's lane */
__device__ __forceinline__ void sft_ld16(u32 addr, float (&v)[16])
{
    u32 r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

/* the y-filtered plane in y accumulator yb into rows [32 slot, 32 slot + 32)
 * of the A tile, rounded to the storage type: thread (w, l) takes column
 * z = 32 (w % 4) + l, rows 16 (w / 4) .. +15 */
__device__ __forceinline__ bool sft_convert(sft_state &S, int slot, int yb)
{
    const bool ok = sft_wait(S, S.bar_y, S.ph_y, yb, 4);
    S.pend &= ~(128u << yb);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int z = 32 * (warp & 3) + lane, half = warp >> 2;
    float v[16];
    sft_ld16(S.tmem + ((u32)((warp & 3) * 32) << 16) + 128u + (u32)(yb * 64 + half * 16), v);
    {
        float vl[16];   /* the lo part's products */
        sft_ld16(S.tmem + ((u32)((warp & 3) * 32) << 16) + 128u + (u32)(yb * 64 + 32 + half * 16), vl);
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] += vl[q];
    }
    unsigned char *col = S.A + (z >> 6) * SFT_ATOM;
    const u32 kb = (u32)((z & 63) * 2);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const u32 m = (u32)(slot * SFD_WY + half * 16 + q);
        *reinterpret_cast<u16 *>(col + sft_sw128(m, kb)) = (u16)sf_enc16<sfd_t>(v[q]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    return ok;
}

/* first plane (y-filtered input) or A tile (sigma_xy = 0) of group g */
template <int IDX, int RY>
__device__ __forceinline__ void sft_start(const sft_maps &mp, sft_state &S, int g)
{
    /* the slab copies of a y-filtered input start inside its plane loop */
    if (g < 0 || RY > 0) return;
    sft_load_a<IDX>(mp, S, g, 0);
    S.pend |= 8u;
}

template <int IDX, int RY, int NZ, int RZ0, int RZ1, int RZ2, int RZ3>
__device__ __forceinline__ void sft_input(const sf_dargs &a, const sfd_taps &t, const sft_maps &mp,
                                          const sft_tiles &bt, const uint4 *__restrict__ tct, sft_state &S)
{
    static_assert(NZ <= 2, "two spectral filters per input");
    (void)t;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int slot = warp & 3, f = warp >> 2;
    const bool mine = f < NZ;
    const i64 y = S.y0 + lane;
    const bool rowv = y < a.ny;
    const bool zfull = S.z0 + SFD_WZ <= a.nz;
    const int ngr = (S.npl + SFT_PLANES - 1) / SFT_PLANES;
    const float inv = 1.f / (float)(1 << SFT_SCALE);
    float K = 0.f, s1 = 0.f, s2 = 0.f;
    f2 s1p = 0ull, s2p = 0ull;
    int cnt = 0;
    bool haveK = false;
    float T = 0.f;
    u32 fl0 = 0u, fl1 = 0u;
    int pass = 0;
    if constexpr (RY > 0) {
        /* this input's y tile (hi and lo parts) into the y-tile slot: every
         * y MMA of the previous input has completed (its planes were read out) */
        const uint4 *src = tct + (SFT_ZT_BYTES + bt.yt[IDX] * SFT_YT_BYTES) / 16;
        uint4 *dst = reinterpret_cast<uint4 *>(S.T + SFT_ZT_BYTES);
        for (int i = threadIdx.x; i < SFT_YT_BYTES / 16; i += SFD_THREADS) dst[i] = __ldg(src + i);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }

    auto next_group = [&](int after) -> int {
        for (int g = after + 1; g < ngr; ++g) {
            if (pass == 0) return g;
            const int p = g * SFT_PLANES;
            const u32 m = (p < 32 ? (fl0 >> p) : (fl1 >> (p - 32))) & 0xfu;
            if (m) return g;
        }
        return -1;
    };
    /* read the z accumulator of group g (buffer b) once its MMAs completed */
    /* plane p takes part in this pass (every plane in pass 1) */
    auto flagged = [&](int p) -> bool {
        return pass == 0 || (((p < 32 ? (fl0 >> p) : (fl1 >> (p - 32))) & 1u) != 0u);
    };
    auto epilogue = [&](int g, int b) {
        const bool ok = sft_wait(S, S.bar_z, S.ph_z, b, 3);
        S.pend &= ~(32u << b);
        if (!ok) S.dead = true;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int p = g * SFT_PLANES + slot;
        /* pass 2 reads flagged planes only: the rows of the others are not
         * filtered in that pass (and could not select anything) */
        const bool pv = p < S.npl && rowv && mine && (pass == 0 || flagged(p));
        float mx = -3.402823466e38f;
        u32 w0 = 0u, w1 = 0u;
        if (mine) {
            /* not unrolled: this read-out is inlined at every call site of
             * every input, and four copies of it per site made the kernel's
             * code outgrow the instruction caches */
#pragma unroll 1
            for (int j = 0; j < 4; ++j) {
                float v[16];
                sft_ld16(S.tmem + ((u32)(slot * 32) << 16) + (u32)(b * 128 + f * 64 + j * 16), v);
                if (!pv) continue;
                if (pass == 0) {
                    if (!haveK) { K = v[0]; haveK = true; }
                    if (zfull) {
                        const f2 NK = f2_pack(-K, -K);
#pragma unroll
                        for (int q = 0; q < 16; q += 2) {
                            const f2 d = f2_add(f2_pack(v[q], v[q + 1]), NK);
                            s1p = f2_add(s1p, d);
                            s2p = f2_fma(d, d, s2p);
                            mx = sfw_max3(mx, v[q], v[q + 1]);
                        }
                        cnt += 16;
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            if (S.z0 + 16 * j + q < a.nz) {
                                const float d = v[q] - K;
                                s1 += d;
                                s2 = fmaf(d, d, s2);
                                ++cnt;
                                mx = fmaxf(mx, v[q]);
                            }
                    }
                } else {
                    u32 bits = 0u;
#pragma unroll
                    for (int q = 0; q < 16; ++q) bits |= (v[q] > T ? 1u : 0u) << q;
                    if (!zfull) {
                        const i64 left = a.nz - (S.z0 + 16 * j);
                        bits &= left >= 16 ? 0xffffu : (left <= 0 ? 0u : ((1u << left) - 1u));
                    }
                    if (j < 2) w0 |= bits << (16 * j);
                    else w1 |= bits << (16 * (j - 2));
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (pass == 0) {
            if (mine) {
                mx = sfw_warp_max(mx);
                if (lane == 0 && p < S.npl) S.pmax[p * SFD_NZF + f] = mx;
            }
        } else if (pv && (w0 | w1)) {
            atomicOr(&S.mask[(p * SFD_WY + lane) * 2 + 0], w0);
            atomicOr(&S.mask[(p * SFD_WY + lane) * 2 + 1], w1);
        }
    };
    /* the z MMAs of group g once its A tile is complete */
    /* one barrier: the A tile is complete and every thread is alive (false:
     * a wait expired somewhere, the input stops) */
    auto issue_z = [&](int g, int buf, int ab) -> bool {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (__syncthreads_or(S.dead)) {
            S.dead = true;
            return false;
        }
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            sft_mma_z<IDX, NZ, RZ0, RZ1>(S, bt, buf, sft_abuf(S, ab));
        }
        S.pend |= 32u << buf;
        (void)g;
        return true;
    };

    sft_start<IDX, RY>(mp, S, next_group(-1));
    for (;;) {
        int pend_g = -1, pend_b = 0;
        int gi = next_group(-1);
        if constexpr (RY == 0) {
            /* A tiles double-buffered: the copy of group gn lands while the
             * z MMAs of group gi run and the previous group is read out */
            int nbuf = 0, ab = 0;
            while (gi >= 0) {
                const int gn = next_group(gi);
                const bool ok = sft_wait(S, S.bar_a, S.ph_a, ab, 1);
                S.pend &= ~(8u << ab);
                if (!ok) S.dead = true;
                const int cur = nbuf;
                nbuf ^= 1;
                if (!issue_z(gi, cur, ab)) return;
                if (gn >= 0 && threadIdx.x == 0) {
                    /* the other A buffer was read by the previous group's z MMAs:
                     * refill it once they completed (a peek: the epilogue waits
                     * on the same completion) */
                    bool ok2 = true;
                    if (pend_g >= 0) ok2 = sfw_wait(S.bar_z + 8u * (u32)pend_b, (S.ph_z >> pend_b) & 1u, S.limit);
                    if (!ok2) {
                        atomicOr(S.err, 1 | (1 << 3));
                        S.dead = true;
                    } else {
                        sft_load_a<IDX>(mp, S, gn, ab ^ 1);
                        S.pend |= 8u << (ab ^ 1);
                    }
                }
                if (pend_g >= 0) epilogue(pend_g, pend_b);
                pend_g = gi;
                pend_b = cur;
                ab ^= 1;
                gi = gn;
            }
        } else {
            /* slab copies run two planes ahead through SFT_NS buffers: lp is
             * the next plane of this pass to copy */
            /* the next plane of this pass after p (-1: the first): pass 2
             * filters only the flagged planes of its groups */
            auto next_plane = [&](int p) -> int {
                int g = p < 0 ? -1 : p / SFT_PLANES, q = p + 1;
                for (;;) {
                    if (g >= 0 && q < (g + 1) * SFT_PLANES && q < S.npl) {
                        if (flagged(q)) return q;
                        ++q;
                        continue;
                    }
                    g = next_group(g);
                    if (g < 0) return -1;
                    q = g * SFT_PLANES;
                }
            };
            int lp = next_plane(-1);
            auto load_next = [&]() {
                if (lp < 0) return;
                const int b = S.it % SFT_NS;
                sft_load_slab<IDX, RY>(mp, S, lp, b);
                S.pend |= 1u << b;
                ++S.it;
                lp = next_plane(lp);
            };
            load_next();
            load_next();
            while (gi >= 0) {
                const int gn = next_group(gi);
                const int p0 = gi * SFT_PLANES;
                const int np = min(SFT_PLANES, S.npl - p0);
                int yprev = -1, iprev = -1;
                for (int i = 0; i < np; ++i) {
                    if (!flagged(p0 + i)) continue;
                    const int b = S.ic % SFT_NS;
                    const bool ok = sft_wait(S, S.bar_s, S.ph_s, b, 2);
                    S.pend &= ~(1u << b);
                    if (__syncthreads_or(!ok)) { S.dead = true; return; }
                    const int yb = S.ity & 1;
                    if (threadIdx.x == 0) {
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        sft_mma_y<RY>(S, bt, IDX, b, yb);
                    }
                    S.pend |= 128u << yb;
                    ++S.ity;
                    ++S.ic;
                    /* the previous group's z accumulator, then the previous
                     * plane into the A tile (its z MMAs are complete by then) */
                    if (pend_g >= 0) {
                        epilogue(pend_g, pend_b);
                        pend_g = -1;
                    }
                    if (yprev >= 0 && !sft_convert(S, iprev, yprev)) S.dead = true;
                    yprev = yb;
                    iprev = i;
                    /* the buffer of the plane before is free: its y MMAs completed
                     * (converted above, or at the end of the previous group) */
                    load_next();
                }
                if (!sft_convert(S, iprev, yprev)) S.dead = true;
                /* planes past the window's end: zero rows (excluded from every sum) */
                for (int e = threadIdx.x + np * SFD_WY * 16; e < SFT_PLANES * SFD_WY * 16; e += SFD_THREADS) {
                    const u32 m = (u32)(e / 16);
                    const int k = 8 * (e % 16);
                    *reinterpret_cast<uint4 *>(S.A + (k >> 6) * SFT_ATOM + sft_sw128(m, (u32)((k & 63) * 2))) =
                        make_uint4(0u, 0u, 0u, 0u);
                }
                if (!issue_z(gi, 0, 0)) return;
                pend_g = gi;
                pend_b = 0;
                gi = gn;
            }
        }
        if (pend_g >= 0) epilogue(pend_g, pend_b);
        if (__syncthreads_or(S.dead)) { S.dead = true; return; }
        if (pass == 1) break;

        /* end of pass 1: statistics, thresholds, flagged planes */
        s1 += f2_lo(s1p) + f2_hi(s1p);
        s2 += f2_lo(s2p) + f2_hi(s2p);
        sfd_mom m{0, 0, 0};
        if (cnt > 0) {
            const sfd_st n = (sfd_st)cnt, mu = (sfd_st)s1 / n;
            m = sfd_mom{n, (sfd_st)K + mu, fmax((sfd_st)s2 - (sfd_st)s1 * mu, (sfd_st)0)};
        }
        /* rolled: once per input and window (smaller code) */
#pragma unroll 1
        for (int off = 1; off < 32; off <<= 1) {
            sfd_mom o;
            o.n = __shfl_xor_sync(0xffffffffu, m.n, off);
            o.mean = __shfl_xor_sync(0xffffffffu, m.mean, off);
            o.m2 = __shfl_xor_sync(0xffffffffu, m.m2, off);
            m = (lane & off) ? sfd_merge(o, m) : sfd_merge(m, o);
        }
        if (lane == 0) {
            sfd_st *w = S.red + warp * 3;
            w[0] = m.n; w[1] = m.mean; w[2] = m.m2;
        }
        __syncthreads();
        if (threadIdx.x < NZ) {
            const int ff = threadIdx.x;
            sfd_mom mm{0, 0, 0};
            for (int w = 0; w < 4; ++w) {
                const sfd_st *q = S.red + (ff * 4 + w) * 3;
                mm = sfd_merge(mm, sfd_mom{q[0], q[1], q[2]});
            }
            const sfd_st sd = mm.n > SFD_DDOF ? sqrt(mm.m2 / (mm.n - SFD_DDOF)) : (sfd_st)0;
            S.thr[ff] = (float)fma((sfd_st)a.k, sd, mm.mean);
            if (a.mean != nullptr) {
                const i64 o = (i64)a.fidx[IDX][ff] * a.nwin + S.wid;
                a.mean[o] = (float)mm.mean * inv;
                a.stdv[o] = (float)sd * inv;
            }
        }
        __syncthreads();
        if (warp == 0) {
            for (int base = 0; base < SFD_WX; base += 32) {
                const int q = base + lane;
                bool hot = false;
                if (q < S.npl)
#pragma unroll
                    for (int ff = 0; ff < NZ; ++ff) hot |= S.pmax[q * SFD_NZF + ff] > S.thr[ff];
                const u32 bits = __ballot_sync(0xffffffffu, hot);
                if (lane == 0) S.flags[base >> 5] = bits;
            }
        }
        __syncthreads();
        fl0 = S.flags[0];
        fl1 = SFD_WX > 32 ? S.flags[1] : 0u;
        if (mine) T = S.thr[f];
        pass = 1;
        sft_start<IDX, RY>(mp, S, next_group(-1));
    }
}

__device__ __forceinline__ bool sft_window(const sf_dargs &a, const sfd_taps &t, const sft_maps &mp,
                                           const uint4 *__restrict__ tct,
                                           const sft_tiles &bt, sft_state &S, int wid)
{
    S.wid = wid;
    S.limit = (unsigned long long)a.wait_ns;
    const int wz = wid % a.nwz, wy = (wid / a.nwz) % a.nwy, wx = wid / (a.nwz * a.nwy);
    S.x0 = a.xorg + (i64)wx * SFD_WX;
    S.y0 = (i64)wy * SFD_WY;
    S.z0 = (i64)wz * SFD_WZ;
    const i64 left = a.nx - S.x0;
    S.npl = left < SFD_WX ? (int)left : SFD_WX;
    for (int i = threadIdx.x; i < SFD_WX * SFD_WY * 2; i += SFD_THREADS) S.mask[i] = 0u;
    __syncthreads();
#define SFT_RUN(IDX, RY, NZ, RZ0, RZ1, RZ2, RZ3) \
    if (!S.dead) sft_input<IDX, RY, NZ, RZ0, RZ1, RZ2, RZ3>(a, t, mp, bt, tct, S);
    SFD_SOURCES(SFT_RUN)
#undef SFT_RUN
    if (S.dead) return false;
    __syncthreads();
    /* mask words: thread (row, word) of every plane */
    const int row = threadIdx.x >> 1, wd = threadIdx.x & 1;
    if (row < SFD_WY && S.y0 + row < a.ny) {
        const i64 gw = (S.z0 >> 5) + wd;
        if (gw < a.nw32)
            for (int p = 0; p < S.npl; ++p)
                a.mask[((S.x0 - a.xorg + p) * a.ny + S.y0 + row) * a.nw32 + gw] = S.mask[(p * SFD_WY + row) * 2 + wd];
    }
    return true;
}

extern "C" __global__ void __launch_bounds__(SFD_THREADS, 2)
sf_window_tc(const __grid_constant__ sf_dargs a, const __grid_constant__ sfd_taps t,
             const __grid_constant__ sft_maps mp, const __grid_constant__ sft_tiles bt, const uint4 *__restrict__ tct)
{
    extern __shared__ __align__(1024) unsigned char sft_raw[];
    __shared__ u32 s_tmem;
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<unsigned long long>(sft_raw) + 1023ull) & ~1023ull);
    sft_state S;
    S.A = sm + SFT_OFF_A;
    S.T = sm + SFT_OFF_T;
    S.slab = sm + SFT_OFF_SLAB;
    S.pmax = reinterpret_cast<float *>(sm + SFT_OFF_PMAX);
    S.mask = reinterpret_cast<u32 *>(sm + SFT_OFF_MASK);
    S.red = reinterpret_cast<sfd_st *>(sm + SFT_OFF_RED);
    S.thr = reinterpret_cast<float *>(sm + SFT_OFF_THR);
    S.flags = reinterpret_cast<u32 *>(sm + SFT_OFF_FLAGS);
    S.bar_s = sf_smem_addr(sm + SFT_OFF_MBAR);
    S.bar_a = S.bar_s + 8u * SFT_NS;
    S.bar_z = S.bar_a + 16u;
    S.bar_y = S.bar_z + 16u;
    S.ph_s = S.ph_a = S.ph_z = S.ph_y = 0u;
    S.pend = 0u;
    S.it = S.ic = S.ity = 0;
    S.dead = false;
    S.limit = (unsigned long long)a.wait_ns;
    S.err = a.err;
    /* the tap tiles, already in the swizzled layout */
    {
        /* from the device copy: the same bytes as bt's tiles */
        uint4 *dst = reinterpret_cast<uint4 *>(S.T);
        for (int i = threadIdx.x; i < SFT_ZT_BYTES / 16; i += SFD_THREADS) dst[i] = __ldg(tct + i);
    }
    if (threadIdx.x == 0) {
        for (int b = 0; b < SFT_NS + 6; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(S.bar_s + 8u * (u32)b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sf_smem_addr(&s_tmem)),
                     "r"((u32)SFT_TM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    S.tmem = s_tmem;
    const bool ok = sft_window(a, t, mp, tct, bt, S, a.wid0 + (int)blockIdx.x);
    if (!ok && threadIdx.x == 0) {
        /* a bounded wait expired: report it, then give the copies and MMAs in
         * flight a bounded time to land before the buffers go away */
        atomicOr(a.err, 1);
        for (int b = 0; b < SFT_NS; ++b)
            if ((S.pend >> b) & 1u) sfw_wait(S.bar_s + 8u * (u32)b, (S.ph_s >> b) & 1u, S.limit);
        for (int b = 0; b < 2; ++b) {
            if ((S.pend >> (3 + b)) & 1u) sfw_wait(S.bar_a + 8u * (u32)b, (S.ph_a >> b) & 1u, S.limit);
            if ((S.pend >> (5 + b)) & 1u) sfw_wait(S.bar_z + 8u * (u32)b, (S.ph_z >> b) & 1u, S.limit);
            if ((S.pend >> (7 + b)) & 1u) sfw_wait(S.bar_y + 8u * (u32)b, (S.ph_y >> b) & 1u, S.limit);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem), "r"((u32)SFT_TM_COLS)
                     : "memory");
}
#endif /* SF_KERNEL_TC */

/* ======================================================================= */
#ifdef SF_KERNEL_FILTER
/* one CTA per (x, y tile, z tile): y and z passes of a single filter */
extern "C" __global__ void __launch_bounds__(SFD_THREADS)
sf_yz_filter(const __grid_constant__ sf_fargs a, const __grid_constant__ sfd_taps t)
{
    extern __shared__ __align__(128) unsigned char sff_sm[];
    sfd_t *slab = reinterpret_cast<sfd_t *>(sff_sm);
    float *U = reinterpret_cast<float *>(sff_sm + SFD_OFF_U);
    const i64 x = blockIdx.x;
    const i64 y0 = (i64)blockIdx.y * SFD_WY, z0 = (i64)blockIdx.z * SFD_WZ;
    const sfd_t *src = reinterpret_cast<const sfd_t *>(a.src);
#define SFF_LOAD(IDX, RY, NZ, RZ0, RZ1, RZ2, RZ3) sfd_load_slab<RY>(slab, src, x, y0, z0, a.nx, a.ny, a.nz);
    SFD_SOURCES(SFF_LOAD)
#undef SFF_LOAD
    sf_cp_commit();
    sf_cp_wait<0>();
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int RG = SFD_WY / 8;
    const int row = (warp % RG) * 8 + (lane & 7);
    const int chunk = (warp / RG) * 4 + (lane >> 3);
    float c[SFD_NZF][SFD_P];
#if SFD_X2
#define SFF_RUN(IDX, RY, NZ, RZ0, RZ1, RZ2, RZ3)                                \
    if constexpr (RY > 0) {                                                     \
        sfd_yfilter2<IDX, RY>(slab, U, t);                                      \
        __syncthreads();                                                        \
    }                                                                           \
    sfd_zfilter2<IDX, RY, NZ, RZ0, RZ1, RZ2, RZ3>(slab, U, row, chunk, c, t);
#else
#define SFF_RUN(IDX, RY, NZ, RZ0, RZ1, RZ2, RZ3)                                \
    if constexpr (RY > 0) {                                                     \
        sfd_yfilter<IDX, RY>(slab, U, t);                                       \
        __syncthreads();                                                        \
    }                                                                           \
    sfd_zfilter<IDX, RY, NZ, RZ0, RZ1, RZ2, RZ3>(slab, U, row, chunk, c, t);
#endif
    SFD_SOURCES(SFF_RUN)
#undef SFF_RUN
    const i64 y = y0 + row, zb = z0 + 8 * chunk;
    if (y >= a.ny) return;
    float *out = a.out + (x * a.ny + y) * a.nz + zb;
    if (zb + 8 <= a.nz && (a.nz & 3) == 0) {
        sf_st<float, 4>(out, c[0]);
        sf_st<float, 4>(out + 4, c[0] + 4);
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (zb + i < a.nz) out[i] = c[0][i];
    }
}
#endif /* SF_KERNEL_FILTER */
