/*
 * Per-voxel local statistics of a filtered cube (Sec. 3.3: the mean and
 * standard deviation of each voxel come from a user-specified range of the
 * filtered data around it), read as the box [x-sx, x+sx] x [y-sy, y+sy] x
 * [z-sz, z+sz] clipped to the cube, with n the number of voxels of the clipped
 * box; population statistics.  The box sums are separable, as in the paper's
 * three directional sums:
 *
 *   sf_local_yz  one CTA per (x, 32-row, 64-column) tile: the tile with its y
 *                and z halo is staged in shared memory, shifted by one of its
 *                values s_t (entries outside the cube are 0: they are not in
 *                any box); box sums of (c - s_t) and (c - s_t)^2 along z and
 *                then along y are formed as running sums restarted every 16
 *                outputs (direct sums per output for half-widths up to 16),
 *                and each voxel's y-z box mean A and second central
 *                moment M = sum (c - A)^2 are written as two float32 cubes;
 *   sf_local_x   one thread per (y, z) and 32-plane x segment, marching along
 *                x with compensated (Kahan) running sums over the x box of
 *                (A - s), (A - s)^2 and M, started from a direct sum with s
 *                the segment's first A; the box statistics then
 *                follow from the parallel-axis rule
 *                  mean = s + sum(A - s)/X,
 *                  M2   = sum M + n_yz (sum (A - s)^2 - (sum (A - s))^2 / X)
 *                (X planes of n_yz voxels each), var = M2 / (X n_yz); either
 *                the mean / std cubes are written or the selection
 *                c > mean + k std is packed into the mask words by a warp
 *                ballot (one warp = 32 consecutive z of one row), OR-ed into
 *                the words already there when the mask accumulates a bank.
 * Shifting by a value of the data keeps the second moments from cancelling
 * when the local mean is large against the local spread.
 */
#include <cuda_runtime.h>

namespace {

typedef long long i64;

constexpr int kYT = 32;          /* tile rows (y) */
constexpr int kZT = 64;          /* tile columns (z) */
constexpr int kPZ = kZT + 1;     /* row stride of the z sums (odd: conflict-free) */
constexpr int kSeg = 16;         /* outputs per running-sum segment */
constexpr int kDirect = 2;       /* half-widths up to this: direct sums per output */
constexpr int kYSeg = 8;         /* rows per y running-sum segment */
constexpr int kYZThreads = 256;
constexpr int kXThreads = 128;
constexpr int kXSeg = 32;        /* x planes per re-anchored segment */

__host__ __device__ inline int stage_cols(int sz) { return (kZT + 2 * sz) | 1; }   /* odd: fewer bank conflicts */

__device__ __forceinline__ i64 clipped(i64 v, int h, i64 n)
{
    const i64 lo = v - h < 0 ? 0 : v - h, hi = v + h >= n ? n - 1 : v + h;
    return hi - lo + 1;
}

__global__ void __launch_bounds__(kYZThreads) sf_local_yz(const float *__restrict__ c, float *__restrict__ A,
                                                        float *__restrict__ M, i64 nx, i64 ny, i64 nz, int sy,
                                                        int sz)
{
    extern __shared__ float sm[];
    const int rows = kYT + 2 * sy, cols = stage_cols(sz);
    float *T = sm;                       /* [rows][cols] staged c - s_t */
    float *Pz = T + rows * cols;         /* [rows][kPZ] z box sums of c - s_t */
    float *Qz = Pz + rows * kPZ;         /* [rows][kPZ] z box sums of (c - s_t)^2 */
    const i64 x = blockIdx.z, y0 = (i64)blockIdx.y * kYT, z0 = (i64)blockIdx.x * kZT;
    (void)nx;
    /* the tile's shift: the value nearest its centre inside the cube */
    const i64 yc = min(ny - 1, y0 + kYT / 2), zc = min(nz - 1, z0 + kZT / 2);
    const float st = c[(x * ny + yc) * nz + zc];
    /* staging by cp.async (4 bytes, zero fill outside the cube), then each
     * thread shifts the elements its own copies wrote */
    const unsigned int tbase = (unsigned int)__cvta_generic_to_shared(T);
    for (int r = threadIdx.x >> 5; r < rows; r += kYZThreads / 32) {
        const i64 y = y0 - sy + r;
        const bool yin = y >= 0 && y < ny;
        const float *src = c + (x * ny + (yin ? y : 0)) * nz;
        for (int q = threadIdx.x & 31; q < cols; q += 32) {
            const i64 z = z0 - sz + q;
            const bool in = yin && z >= 0 && z < nz && q < kZT + 2 * sz;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(tbase + 4u * (unsigned)(r * cols + q)),
                         "l"(in ? src + z : c), "r"(in ? 4 : 0)
                         : "memory");
        }
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    for (int r = threadIdx.x >> 5; r < rows; r += kYZThreads / 32) {
        const i64 y = y0 - sy + r;
        const bool yin = y >= 0 && y < ny;
        for (int q = threadIdx.x & 31; q < cols; q += 32) {
            const i64 z = z0 - sz + q;
            if (yin && z >= 0 && z < nz && q < kZT + 2 * sz) T[r * cols + q] -= st;
        }
    }
    __syncthreads();
    /* z: output column j of staged row r sums staged columns j .. j + 2 sz */
    constexpr int nseg_z = kZT / kSeg;
    for (int task = threadIdx.x; task < rows * nseg_z; task += kYZThreads) {
        /* consecutive lanes take consecutive rows: with an odd row stride the
         * shared loads of a warp hit 32 different banks */
        const int seg = task / rows, r = task - seg * rows, j0 = seg * kSeg;
        const float *row = T + r * cols;
        float p = 0.f, q = 0.f;
#pragma unroll 4
        for (int o = 0; o <= 2 * sz; ++o) {
            const float v = row[j0 + o];
            p += v;
            q = fmaf(v, v, q);
        }
        Pz[r * kPZ + j0] = p;
        Qz[r * kPZ + j0] = q;
        for (int j = j0 + 1; j < j0 + kSeg; ++j) {
            if (sz <= kDirect) {
                /* short boxes: a direct sum per output (exact for one voxel) */
                p = 0.f;
                q = 0.f;
                for (int o = 0; o <= 2 * sz; ++o) {
                    const float v = row[j + o];
                    p += v;
                    q = fmaf(v, v, q);
                }
            } else {
                const float vin = row[j + 2 * sz], vout = row[j - 1];
                p += vin - vout;
                q = fmaf(-vout, vout, fmaf(vin, vin, q));
            }
            Pz[r * kPZ + j] = p;
            Qz[r * kPZ + j] = q;
        }
    }
    __syncthreads();
    /* y: output row i sums staged rows i .. i + 2 sy */
    constexpr int nseg_y = kYT / kYSeg;
    /* clipped box counts factor into a y and a z part (32-bit) */
    const int nyi = (int)ny, nzi = (int)nz;
    auto cnt = [](int v, int h, int n) { return min(v + h, n - 1) - max(v - h, 0) + 1; };
    for (int task = threadIdx.x; task < kZT * nseg_y; task += kYZThreads) {
        const int j = task % kZT, i0 = (task / kZT) * kYSeg;
        const int z = (int)z0 + j;
        const bool zin = z < nzi;
        const float cz = (float)cnt(z, sz, nzi);
        float *pa = A + (x * ny + y0 + i0) * nz + z;
        float *pm = M + (x * ny + y0 + i0) * nz + z;
        float p = 0.f, q = 0.f;
#pragma unroll 4
        for (int o = 0; o <= 2 * sy; ++o) {
            p += Pz[(i0 + o) * kPZ + j];
            q += Qz[(i0 + o) * kPZ + j];
        }
        for (int i = i0; i < i0 + kYSeg; ++i) {
            if (i > i0 && sy <= kDirect) {
                p = 0.f;
                q = 0.f;
                for (int o = 0; o <= 2 * sy; ++o) {
                    p += Pz[(i + o) * kPZ + j];
                    q += Qz[(i + o) * kPZ + j];
                }
            } else if (i > i0) {
                p += Pz[(i + 2 * sy) * kPZ + j] - Pz[(i - 1) * kPZ + j];
                q += Qz[(i + 2 * sy) * kPZ + j] - Qz[(i - 1) * kPZ + j];
            }
            const int y = (int)y0 + i;
            if (y < nyi && zin) {
                const float n = (float)cnt(y, sy, nyi) * cz;
                *pa = st + p / n;
                /* a rounded product (no contraction into an fma): for a
                 * one-voxel box q and p*p round alike and M is exactly 0 */
                *pm = fmaxf(q - __fmul_rn(p, p / n), 0.f);
            }
            pa += nz;
            pm += nz;
        }
    }
}

/* compensated running sum */
struct Kahan {
    float s = 0.f, comp = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        const float y = v - comp;
        const float t = s + y;
        comp = (t - s) - y;
        s = t;
    }
};

/* MODE 0: mean / std cubes; 1: mask words set; 2: mask words OR-ed */
template <int MODE>
__global__ void __launch_bounds__(kXThreads, 10)
    sf_local_x(const float *__restrict__ c, const float *__restrict__ A, const float *__restrict__ M, i64 nx,
               i64 ny, i64 nz, i64 nw32, int sx, int sy, int sz, float k, float *__restrict__ mean,
               float *__restrict__ stdv, unsigned int *__restrict__ mask)
{
    const i64 lane = (i64)blockIdx.x * kXThreads + threadIdx.x;
    const i64 per_row = nw32 * 32;
    const i64 y = lane / per_row;
    if (y >= ny) return;   /* whole warps: a row holds a multiple of 32 lanes */
    const int zw = (int)((lane - y * per_row) >> 5);
    const int bit = (int)(lane & 31);
    const i64 z = (i64)zw * 32 + bit;
    const bool valid = z < nz;
    const i64 plane = ny * nz;
    const i64 off = y * nz + (valid ? z : 0);
    const float *pa = A + off, *pm = M + off, *pc = c + off;
    const float nyz = (float)(clipped(y, sy, ny) * clipped(z, sz, nz));
    const int nxi = (int)nx;
    const i64 x0 = (i64)blockIdx.y * kXSeg;
    const i64 x1 = x0 + kXSeg < nx ? x0 + kXSeg : nx;
    /* segment blockIdx.y of kXSeg planes: the sums start from a direct sum
     * over the box of the segment's first plane, shifted by that plane's A,
     * so the running updates neither drift nor cancel */
    const float s = pa[x0 * plane];
    Kahan sa, sb, sm;   /* sums over the x box of A - s, (A - s)^2, M */
    {
        const i64 lo = x0 - sx < 0 ? 0 : x0 - sx, hi = x0 + sx >= nx ? nx - 1 : x0 + sx;
        for (i64 xi = lo; xi <= hi; ++xi) {
            const float d = pa[xi * plane] - s;
            sa.add(d);
            sb.add(d * d);
            sm.add(pm[xi * plane]);
        }
    }
    /* pointers to the planes entering (x + sx) and leaving (x - sx - 1) the
     * box, and to plane x; unused ones stay at plane 0 */
    const float *ain_p = pa + (x0 + sx) * plane, *min_p = pm + (x0 + sx) * plane;
    const float *aout_p = pa + (x0 - sx - 1) * plane, *mout_p = pm + (x0 - sx - 1) * plane;
    const float *c_p = pc + x0 * plane;
#pragma unroll 4
    for (i64 x = x0; x < x1; ++x) {
        /* the step's loads, unconditional (unused ones read plane 0) so they
         * issue together */
        const int xi = (int)x;
        const bool hin = x > x0 && xi + sx < nxi, hout = x > x0 && xi - sx - 1 >= 0;
        const float ain = hin ? ain_p[0] : pa[0], min_ = hin ? min_p[0] : pm[0];
        const float aout = hout ? aout_p[0] : pa[0], mout = hout ? mout_p[0] : pm[0];
        const float cv = MODE != 0 ? c_p[0] : 0.f;
        ain_p += plane;
        min_p += plane;
        aout_p += plane;
        mout_p += plane;
        c_p += plane;
        if (hin) {
            const float d = ain - s;
            sa.add(d);
            sb.add(d * d);
            sm.add(min_);
        }
        if (hout) {
            const float d = aout - s;
            sa.add(-d);
            sb.add(-(d * d));
            sm.add(-mout);
        }
        float X, mu, m2;
        if (sx == 0) {
            /* the x box is the plane itself */
            X = 1.f;
            mu = pa[x * plane];
            m2 = pm[x * plane];
        } else {
            X = (float)(min(xi + sx, nxi - 1) - max(xi - sx, 0) + 1);
            const float da = sa.s / X;
            mu = s + da;
            /* a rounded product (no contraction into an fma) */
            m2 = sm.s + nyz * fmaxf(sb.s - __fmul_rn(sa.s, da), 0.f);
        }
        const float sd = sqrtf(m2 / (X * nyz));
        if (MODE == 0) {
            if (valid) {
                mean[x * plane + off] = mu;
                stdv[x * plane + off] = sd;
            }
        } else {
            const unsigned int bits = __ballot_sync(0xffffffffu, valid && cv > fmaf(k, sd, mu));
            if (bit == 0) {
                unsigned int *w = mask + (x * ny + y) * nw32 + zw;
                if (MODE == 2) {
                    if (bits) atomicOr(w, bits);   /* nothing waits on it */
                } else {
                    *w = bits;
                }
            }
        }
    }
}

}  // namespace

/* shared memory of sf_local_yz for half-widths (sy, sz) */
size_t sf_local_yz_smem(int sy, int sz)
{
    const size_t rows = (size_t)kYT + 2 * (size_t)sy;
    return sizeof(float) * rows * ((size_t)stage_cols(sz) + 2 * kPZ);
}

cudaError_t sf_launch_local_yz(const float *c, float *A, float *M, long long nx, long long ny, long long nz, int sy,
                               int sz, cudaStream_t st)
{
    const size_t smem = sf_local_yz_smem(sy, sz);
    cudaError_t e = cudaFuncSetAttribute(sf_local_yz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((nz + kZT - 1) / kZT), (unsigned)((ny + kYT - 1) / kYT), (unsigned)nx);
    sf_local_yz<<<grid, kYZThreads, smem, st>>>(c, A, M, nx, ny, nz, sy, sz);
    return cudaGetLastError();
}

cudaError_t sf_launch_local_x(const float *c, const float *A, const float *M, long long nx, long long ny,
                              long long nz, long long nw32, int sx, int sy, int sz, float k, float *mean,
                              float *stdv, unsigned int *mask, int mode, cudaStream_t st)
{
    const long long lanes = ny * nw32 * 32;
    const dim3 grid((unsigned)((lanes + kXThreads - 1) / kXThreads), (unsigned)((nx + kXSeg - 1) / kXSeg));
    if (mode == 0) sf_local_x<0><<<grid, kXThreads, 0, st>>>(c, A, M, nx, ny, nz, nw32, sx, sy, sz, k, mean, stdv, mask);
    else if (mode == 1) sf_local_x<1><<<grid, kXThreads, 0, st>>>(c, A, M, nx, ny, nz, nw32, sx, sy, sz, k, mean, stdv, mask);
    else sf_local_x<2><<<grid, kXThreads, 0, st>>>(c, A, M, nx, ny, nz, nw32, sx, sy, sz, k, mean, stdv, mask);
    return cudaGetLastError();
}
