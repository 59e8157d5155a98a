/*
 * Per-voxel local statistics of a filtered cube (Sec. 3.3: the mean and
 * standard deviation of each voxel come from a user-specified range of the
 * filtered data around it), read as the box [x-sx, x+sx] x [y-sy, y+sy] x
 * [z-sz, z+sz] clipped to the cube, with n the number of voxels of the clipped
 * box; population statistics (sample statistics, over n - 1, on request).
 * The box sums are separable, as in the paper's three directional sums:
 *
 *   sf_local_yz  one CTA per (x, 128-column z tile, y segment of up to 256
 *                rows) marching along y in steps of 16 rows.  Each step
 *                stages 16 rows of the tile with their z halo (cp.async, zeros
 *                outside the cube), forms the z box sums of (c - s) and
 *                (c - s)^2 of every row (s: the mean of the tile's centre
 *                row) as running sums over 16-column segments started from
 *                16-column block sums, and pushes them into a ring of the
 *                last 2 sy + 17 rows.  The y box sums run down the ring, two
 *                lanes per column (one per sum), restarted from a direct sum
 *                at every step of 16 rows.  A sum of squares whose chain has
 *                carried a total above kBudget times its current value is
 *                recomputed directly (the rounding left by large values that
 *                entered and left would otherwise dominate).  Each voxel's y-z
 *                box mean A and second central moment M = sum (c - A)^2 are
 *                written as two float32 cubes.  Half-widths up to 2 use
 *                direct sums for every output; a one-voxel y-z box is a copy
 *                (A = c, M = 0);
 *   sf_local_x   one thread per (y, z) and x segment, marching along x with
 *                compensated (Neumaier) running sums over the x box of (A - s),
 *                (A - s)^2 and M, started from a direct sum with s the
 *                segment's first A; the box statistics then follow from the
 *                parallel-axis rule
 *                  mean = s + sum(A - s)/X,
 *                  M2   = sum M + n_yz (sum (A - s)^2 - (sum (A - s))^2 / X)
 *                (X planes of n_yz voxels each), var = M2 / (X n_yz); either
 *                the mean / std cubes are written or the selection
 *                c > mean + k std is packed into the mask words by a warp
 *                ballot (V z per thread, V mask words per warp), OR-ed into
 *                the words already there when the mask accumulates a bank.
 * Shifting by values of the data keeps the second moments from cancelling
 * when the local mean is large against the local spread.  The FP32 sums still
 * lose precision where the box's spread is small against the distance from
 * its mean to the shift, which thin boxes on smooth data reach; boxes with a
 * half-width below 3 on some axis therefore take
 *   sf_local_direct  two passes over each voxel's clipped box (the mean, then
 *                the squared deviations from it) with compensated sums: no
 *                cancellation, O(box) work per voxel.
 */
#include <cuda_runtime.h>

#include <cstdlib>

namespace {

typedef long long i64;

constexpr int kDirect = 2;       /* half-widths up to this: direct sums per output */
constexpr int kXThreads = 128;
constexpr int kXSeg = 128;       /* x planes per re-anchored segment */

/* ---- y-z box sums ---- */
constexpr int kMZ = 128;         /* output columns per CTA */
constexpr int kMT = 256;         /* threads: two per column (one per sum) */
constexpr int kRB = 16;          /* rows per step */
constexpr int kBS = 16;          /* z block and segment length */
constexpr int kRS = kMZ + 4;     /* ring row stride: 33 quads (odd) */
constexpr int kYRows = 256;      /* output rows per CTA at most */
/* a running sum of squares carries a rounding error within 2 ulps of the
 * total of its values along the chain; when that total exceeds kBudget times
 * the current value (large values entered and left), the output is summed
 * directly and the chain restarts from it, so the error stays within
 * 2 * kBudget ulps of the value */
constexpr float kBudget = 64.f;

/* staged row stride: columns up to 131 + 2 sz are read, in float4 quads; an
 * odd number of quads keeps eight rows' quads in distinct banks */
__host__ __device__ inline int yz_sw(int sz)
{
    int w = (132 + 2 * sz + 3) & ~3;
    if (((w >> 2) & 1) == 0) w += 4;
    return w;
}
/* 16-column block sums per row: the anchors of segments 0..7 span blocks
 * 0 .. 7 + nf - 1 */
__host__ __device__ inline int yz_nbk(int sz)
{
    const int nf = (2 * sz + 1) / kBS;
    return sz <= kDirect || nf == 0 ? 0 : kMZ / kBS - 1 + nf;
}
__host__ __device__ inline int yz_ring(int sy) { return 2 * sy + 1 + kRB; }
/* the Q ring starts 16 banks after the P ring, so that a warp reading one row
 * of P (lanes 0-15) and of Q (lanes 16-31) hits 32 distinct banks */
__host__ __device__ inline int yz_qpad(int sy) { return (16 - (yz_ring(sy) * kRS) % 32 + 32) % 32; }
__host__ __device__ inline size_t yz_smem_floats(int sy, int sz)
{
    return (size_t)kRB * yz_sw(sz) + 2 * (size_t)yz_nbk(sz) * kRB + 2 * (size_t)yz_ring(sy) * kRS + yz_qpad(sy);
}

__device__ __forceinline__ i64 clipped(i64 v, int h, i64 n)
{
    const i64 lo = v - h < 0 ? 0 : v - h, hi = v + h >= n ? n - 1 : v + h;
    return hi - lo + 1;
}
__device__ __forceinline__ int clipped32(int v, int h, int n) { return min(v + h, n - 1) - max(v - h, 0) + 1; }

__device__ __forceinline__ void ld4(const float *p, float *v)
{
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
}
__device__ __forceinline__ void st4(float *p, const float *v)
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

/* term of the sums: SQ 0 -> d, 1 -> d^2, added to acc */
template <int SQ>
__device__ __forceinline__ float yz_add(float acc, float d)
{
    return SQ ? fmaf(d, d, acc) : acc + d;
}

/* one z sum (SQ 0: of c - s, 1: of (c - s)^2) of one staged row for outputs
 * j0 .. j0+15 into the ring row.  SH = (2 sz + 1) mod 4 places the entering
 * columns j + 2 sz inside the float4 quads loaded from the aligned column
 * j0 + 2 sz + 1 - SH. */
template <bool SHIFTED, int SH, int SQ>
__device__ __forceinline__ void yz_segment(const float *__restrict__ u, const float2 *__restrict__ bs, float *ring,
                                           int j0, int nf, int rem, int sz, float s)
{
    const float s0 = SHIFTED ? 0.f : s;
    float acc = 0.f;
    for (int k = 0; k < nf; ++k) {
        const float2 b = bs[k * kRB];
        acc += SQ ? b.y : b.x;
    }
    /* the box's last rem columns after the full blocks (rem odd, <= 15) */
    const float *rp = u + j0 + kBS * nf;
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
        if (4 * ch < rem) {
            float v[4];
            ld4(rp + 4 * ch, v);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (4 * ch + i < rem) acc = yz_add<SQ>(acc, v[i] - s0);
        }
    }
    float L[16], E[20];
#pragma unroll
    for (int i = 0; i < 4; ++i) ld4(u + j0 + 4 * i, L + 4 * i);
    const float *ep = u + j0 + (2 * sz + 1 - SH);
#pragma unroll
    for (int i = 0; i < 5; ++i) ld4(ep + 4 * i, E + 4 * i);
    float o4[4];
    o4[0] = acc;
    float tot = acc;   /* the total of the chain's sums of squares since its start */
    unsigned int redo = 0u;   /* outputs whose chain total exceeds kBudget times them */
#pragma unroll
    for (int i = 1; i < 16; ++i) {
        const float vin = E[SH - 1 + i] - s0, vout = L[i - 1] - s0;
        if (SQ) {
            acc = fmaf(-vout, vout, fmaf(vin, vin, acc));
            tot += fabsf(acc);
            redo |= (acc * kBudget < tot ? 1u : 0u) << i;
        } else {
            acc += vin - vout;
        }
        o4[i & 3] = acc;
        if ((i & 3) == 3) st4(ring + j0 + i - 3, o4);
    }
    if (SQ && redo) {
        /* large values entered and left: the rounding they left would
         * dominate, so these outputs are summed directly */
        for (int i = 1; i < 16; ++i)
            if (redo >> i & 1u) {
                float q = 0.f;
                for (int o = 0; o <= 2 * sz; ++o) {
                    const float d = u[j0 + i + o] - s0;
                    q = fmaf(d, d, q);
                }
                ring[j0 + i] = q;
            }
    }
}

/* short boxes (sz <= kDirect): a direct sum for every output */
template <bool SHIFTED, int SQ>
__device__ __forceinline__ void yz_segment_direct(const float *__restrict__ u, float *ring, int j0, int sz, float s)
{
    const float s0 = SHIFTED ? 0.f : s;
    float v[20];
#pragma unroll
    for (int i = 0; i < 5; ++i) ld4(u + j0 + 4 * i, v + 4 * i);
    float o4[4];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        float acc = 0.f;
#pragma unroll
        for (int o = 0; o <= 2 * kDirect; ++o)
            if (o <= 2 * sz) acc = yz_add<SQ>(acc, v[i + o] - s0);
        o4[i & 3] = acc;
        if ((i & 3) == 3) st4(ring + j0 + i - 3, o4);
    }
}

template <bool SHIFTED, int SQ>
__device__ __forceinline__ void yz_task(const float *u, const float2 *bs, float *ring, int j0, int nf, int rem,
                                        int sz, int sh, float s)
{
    if (sz <= kDirect) yz_segment_direct<SHIFTED, SQ>(u, ring, j0, sz, s);
    else if (sh == 1) yz_segment<SHIFTED, 1, SQ>(u, bs, ring, j0, nf, rem, sz, s);
    else yz_segment<SHIFTED, 3, SQ>(u, bs, ring, j0, nf, rem, sz, s);
}

struct YzGeom {
    const float *c;
    i64 plane0;          /* offset of plane x */
    int ny, nz;          /* extents (the launcher checks they fit 31 bits) */
    int sy, sz, SW, NBK, RING, nf, rem, sh;
    int ys, zst, zt0;    /* first output row, first staged column, first output column */
    int nout, NR;        /* output rows, staged rows (nout + 2 sy) */
};

/* stage rows rr0 .. rr0+15 of the segment (y = ys - sy + rr) into U:
 * CH-element cp.async chunks, zero-filled past the cube's z range (EDGE
 * tiles only); rows outside the cube are left as they are (their ring rows
 * are set to 0) */
template <int CH, bool EDGE>
__device__ __forceinline__ void yz_stage(float *U, const YzGeom &g, int rr0)
{
    const int lane = threadIdx.x & 31;
    const unsigned int ub = (unsigned int)__cvta_generic_to_shared(U);
    for (int r = threadIdx.x >> 5; r < kRB; r += kMT / 32) {
        const int rr = rr0 + r;
        const int y = g.ys - g.sy + rr;
        if (rr >= g.NR || y < 0 || y >= g.ny) continue;
        const float *row = g.c + g.plane0 + (i64)y * g.nz + g.zst;   /* staged column 0 */
        for (int ch = lane; ch < g.SW / CH; ch += 32) {
            const int q = ch * CH;
            unsigned int bytes = 4u * CH;
            const float *src = row + q;
            if (EDGE) {
                const int z = g.zst + q, left = g.nz - z;
                bytes = z >= 0 && left > 0 ? 4u * (unsigned int)(left < CH ? left : CH) : 0u;
                if (!bytes) src = g.c;
            }
            const unsigned int dst = ub + 4u * (unsigned int)(r * g.SW + q);
            if constexpr (CH == 4)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes)
                             : "memory");
            else
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(bytes)
                             : "memory");
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

/* after the copies landed: subtract s from the staged values inside the cube
 * (each thread the chunks its own copies wrote); zeros stay zeros */
template <int CH>
__device__ __forceinline__ void yz_shift(float *U, const YzGeom &g, int rr0, float s)
{
    const int lane = threadIdx.x & 31;
    for (int r = threadIdx.x >> 5; r < kRB; r += kMT / 32) {
        const int rr = rr0 + r;
        const int y = g.ys - g.sy + rr;
        if (rr >= g.NR || y < 0 || y >= g.ny) continue;
        for (int ch = lane; ch < g.SW / CH; ch += 32) {
            const int z = g.zst + ch * CH;
#pragma unroll
            for (int e = 0; e < CH; ++e)
                if (z + e >= 0 && z + e < g.nz) U[r * g.SW + ch * CH + e] -= s;
        }
    }
}

/* one output row of the y march: the second-moment lane (sq) takes p from
 * its partner lane; rn = 1 / (box count) */
__device__ __forceinline__ void yz_emit(float acc, int lane, int sq, bool zok, float rn, float s, float *op)
{
    const float p = __shfl_sync(0xffffffffu, acc, lane & 15);
    const float da = p * rn;
    /* a rounded product (no contraction into an fma): for a one-voxel box q
     * and p*p round alike and M is exactly 0 */
    const float v = sq ? fmaxf(acc - __fmul_rn(p, da), 0.f) : s + da;
    if (zok) *op = v;
}

/* EDGE: some staged columns lie outside the cube; the staged values are then
 * shifted in place, otherwise s is subtracted as they are read */
template <int CH, bool EDGE>
__device__ __forceinline__ void yz_body(float *__restrict__ A, float *__restrict__ M, const YzGeom &g, float s,
                                        float *sm)
{
    float *U = sm;                                              /* [kRB][SW] staged rows */
    float2 *Bs = reinterpret_cast<float2 *>(U + kRB * g.SW);    /* [NBK][kRB] block sums */
    float *P = U + kRB * g.SW + 2 * g.NBK * kRB;                /* [RING][kRS] z sums of c - s */
    float *Q = P + g.RING * kRS + yz_qpad(g.sy);                /* [RING][kRS] z sums of (c - s)^2 */
    const int t = threadIdx.x, lane = t & 31;
    const bool direct_y = g.sy <= kDirect;
    /* y march: lanes 0-15 of warp w carry the sum of c - s, lanes 16-31 the
     * sum of (c - s)^2, of column 16 w + (lane & 15) */
    const int col = 16 * (t >> 5) + (lane & 15), sq = lane >> 4;
    const float *ring = sq ? Q : P;
    const int z = g.zt0 + col;
    const bool zok = z >= 0 && z < g.nz;
    const float rcz = zok ? __frcp_rn((float)clipped32(z, g.sz, g.nz)) : 1.f;
    const int cy_full = 2 * g.sy + 1;
    const float rn_full = rcz * __frcp_rn((float)cy_full);
    float *out = (sq ? M : A) + g.plane0 + (i64)g.ys * g.nz + z;
    const int nsteps = (g.NR + kRB - 1) / kRB;
    float acc = 0.f;   /* this lane's y box sum of the current output row */
    float tot = 0.f;   /* the total of its values since the chain's start (sums of squares) */
    if (EDGE) {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        yz_shift<CH>(U, g, 0, s);
    }
    for (int b = 0; b < nsteps; ++b) {
        const int rr0 = b * kRB;
        __syncthreads();   /* U holds this step's rows; the ring reads of the last step are done */
        if (g.NBK > 0) {
            const float s0 = EDGE ? 0.f : s;
            for (int task = t; task < g.NBK * kRB; task += kMT) {
                const int k = task >> 4, r = task & 15;
                const float *u = U + r * g.SW + kBS * k;
                float pa2[2] = {0.f, 0.f}, qa2[2] = {0.f, 0.f};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float v[4];
                    ld4(u + 4 * i, v);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float d = v[e] - s0;
                        pa2[e & 1] += d;
                        qa2[e & 1] = fmaf(d, d, qa2[e & 1]);
                    }
                }
                Bs[task] = make_float2(pa2[0] + pa2[1], qa2[0] + qa2[1]);
            }
        }
        __syncthreads();
        {
            /* z sums: task (row r, segment gi), warps 0-3 the sums of c - s and
             * warps 4-7 those of (c - s)^2; the eight lanes of a float4 phase
             * hold eight rows of one segment */
            const int task = t & 127, r = task & 15, gi = task >> 4, j0 = kBS * gi;
            const int rr = rr0 + r;
            const int y = g.ys - g.sy + rr;
            int slot = rr0 % g.RING + r;
            if (slot >= g.RING) slot -= g.RING;
            const bool qsum = t >= 128;
            float *rw = (qsum ? Q : P) + slot * kRS;
            if (rr >= g.NR || y < 0 || y >= g.ny) {
                const float zero[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int i = 0; i < 4; ++i) st4(rw + j0 + 4 * i, zero);
            } else {
                const float *u = U + r * g.SW;
                const float2 *bs = Bs + gi * kRB + r;
                if (qsum) yz_task<EDGE, 1>(u, bs, rw, j0, g.nf, g.rem, g.sz, g.sh, s);
                else yz_task<EDGE, 0>(u, bs, rw, j0, g.nf, g.rem, g.sz, g.sh, s);
            }
        }
        __syncthreads();   /* U is free; the ring holds this step's rows */
        if (b + 1 < nsteps) yz_stage<CH, EDGE>(U, g, rr0 + kRB);
        /* y sums down the ring for the outputs whose last box row arrived:
         * the step's first output is a direct sum over its box rows, the
         * others run from it (at most 16 outputs per chain) in stretches
         * where neither ring pointer wraps */
        const int rend = min(kRB, g.NR - rr0);
        const int o0 = max(0, rr0 - 2 * g.sy), o1 = rr0 + rend - 2 * g.sy;   /* outputs [o0, o1) */
        if (o1 > o0) {
            int si = rr0 % g.RING + (o0 + 2 * g.sy - rr0);   /* slot of row o0 + 2 sy */
            if (si >= g.RING) si -= g.RING;
            int so = si + kRB + 1;                             /* slot of row o0 */
            if (so >= g.RING) so -= g.RING;
            /* full y boxes for every output of the step: one reciprocal */
            const bool yfull = g.ys + o0 - g.sy >= 0 && g.ys + o1 - 1 + g.sy < g.ny;
            float *op = out + (i64)o0 * g.nz;
            for (int o = o0; o < o1;) {
                /* direct sum of rows o .. o + 2 sy */
                {
                    int sl = so + (o - o0);
                    if (sl >= g.RING) sl -= g.RING;
                    const int n1 = min(cy_full, g.RING - sl);
                    acc = 0.f;
                    for (int i = 0; i < n1; ++i) acc += ring[(sl + i) * kRS + col];
                    for (int i = 0; i < cy_full - n1; ++i) acc += ring[i * kRS + col];
                }
                tot = fabsf(acc);
                {
                    float rn = rn_full;
                    if (!yfull) rn = rcz * __frcp_rn((float)clipped32(g.ys + o, g.sy, g.ny));
                    yz_emit(acc, lane, sq, zok, rn, s, op);
                }
                op += g.nz;
                ++o;
                if (direct_y) continue;
                /* rows o + 2 sy in (slot a), o - 1 out (slot c) */
                int a = si + (o - o0), c = so + (o - 1 - o0);
                if (a >= g.RING) a -= g.RING;
                if (c >= g.RING) c -= g.RING;
                while (o < o1) {
                    const int m = min(o1 - o, min(g.RING - a, g.RING - c));
                    const float *pin = ring + a * kRS + col, *pout = ring + c * kRS + col;
                    unsigned int redo = 0u;   /* outputs of this stretch to sum directly */
                    float *op0 = op;
                    if (yfull) {
                        for (int i = 0; i < m; ++i) {
                            acc += pin[i * kRS] - pout[i * kRS];
                            tot += fabsf(acc);
                            redo |= (sq && acc * kBudget < tot ? 1u : 0u) << i;
                            yz_emit(acc, lane, sq, zok, rn_full, s, op);
                            op += g.nz;
                        }
                    } else {
                        for (int i = 0; i < m; ++i) {
                            acc += pin[i * kRS] - pout[i * kRS];
                            tot += fabsf(acc);
                            redo |= (sq && acc * kBudget < tot ? 1u : 0u) << i;
                            yz_emit(acc, lane, sq, zok,
                                    rcz * __frcp_rn((float)clipped32(g.ys + o + i, g.sy, g.ny)), s, op);
                            op += g.nz;
                        }
                    }
                    /* large values entered and left the sum of squares (see
                     * kBudget): both sums of those outputs are summed directly
                     * over rows o+i .. o+i+2 sy and written again, the warp
                     * visiting the union of its columns' outputs in order; the
                     * chain continues from the last output */
                    redo = __shfl_sync(0xffffffffu, redo, (lane & 15) + 16);
                    unsigned int todo = __reduce_or_sync(0xffffffffu, redo);
                    while (todo) {
                        const int i = __ffs(todo) - 1;
                        todo &= todo - 1u;
                        const bool mine = (redo >> i) & 1u;
                        int sl = c + i + 1;   /* slot of row o + i */
                        if (sl >= g.RING) sl -= g.RING;
                        const int n1 = min(cy_full, g.RING - sl);
                        float d = 0.f;
                        for (int r = 0; r < n1; ++r) d += ring[(sl + r) * kRS + col];
                        for (int r = 0; r < cy_full - n1; ++r) d += ring[r * kRS + col];
                        float rn = rn_full;
                        if (!yfull) rn = rcz * __frcp_rn((float)clipped32(g.ys + o + i, g.sy, g.ny));
                        yz_emit(d, lane, sq, zok && mine, rn, s, op0 + (i64)i * g.nz);
                        if (mine && i == m - 1) {
                            acc = d;
                            tot = fabsf(d);
                        }
                    }
                    o += m;
                    a += m;
                    c += m;
                    if (a == g.RING) a = 0;
                    if (c == g.RING) c = 0;
                }
            }
        }
        if (b + 1 < nsteps) {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            if (EDGE) yz_shift<CH>(U, g, rr0 + kRB, s);
        }
    }
}

template <int CH>
__global__ void __launch_bounds__(kMT, 3) sf_local_yz(const float *__restrict__ c, float *__restrict__ A,
                                                   float *__restrict__ M, i64 ny, i64 nz, int sy, int sz, int yrows)
{
    extern __shared__ __align__(16) float sm[];
    YzGeom g;
    g.c = c;
    g.ny = (int)ny;
    g.nz = (int)nz;
    g.plane0 = (i64)blockIdx.z * ny * nz;
    g.sy = sy;
    g.sz = sz;
    g.SW = yz_sw(sz);
    g.NBK = yz_nbk(sz);
    g.RING = yz_ring(sy);
    g.nf = (2 * sz + 1) / kBS;
    g.rem = 2 * sz + 1 - kBS * g.nf;
    g.sh = (2 * sz + 1) & 3;
    const int hz = (sz + 3) & ~3;
    g.ys = (int)blockIdx.y * yrows;
    g.nout = min(g.ny - g.ys, yrows);
    if (g.nout <= 0) return;   /* whole CTA: before any barrier */
    g.NR = g.nout + 2 * sy;
    g.zst = (int)blockIdx.x * kMZ - hz;      /* 16-byte aligned first staged column */
    g.zt0 = g.zst + sz;                      /* first output column */
    /* the segment's shift: the mean of the tile's columns on its centre row,
     * so that the shifted sums stay near the local means and the second
     * moments do not cancel */
    __shared__ float sred[2 * (kMT / 32)];
    float s;
    {
        const int yc = g.ys + g.nout / 2;
        const int zq = g.zt0 + (int)(threadIdx.x & (kMZ - 1));
        const bool in = threadIdx.x < kMZ && zq >= 0 && zq < g.nz;
        float v = in ? c[g.plane0 + (i64)yc * g.nz + zq] : 0.f, n = in ? 1.f : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            v += __shfl_xor_sync(0xffffffffu, v, off);
            n += __shfl_xor_sync(0xffffffffu, n, off);
        }
        if ((threadIdx.x & 31) == 0) {
            sred[threadIdx.x >> 5] = v;
            sred[kMT / 32 + (threadIdx.x >> 5)] = n;
        }
        __syncthreads();
        float sv = 0.f, sn = 0.f;
#pragma unroll
        for (int w = 0; w < kMT / 32; ++w) {
            sv += sred[w];
            sn += sred[kMT / 32 + w];
        }
        s = sn > 0.f ? sv / sn : 0.f;
    }
    if (g.zst >= 0 && g.zst + g.SW <= g.nz) {
        /* interior tile: every staged value is data; subtract s on the fly */
        yz_stage<CH, false>(sm, g, 0);
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        yz_body<CH, false>(A, M, g, s, sm);
    } else {
        yz_stage<CH, true>(sm, g, 0);
        yz_body<CH, true>(A, M, g, s, sm);
    }
}

/* compensated running sum */
/* compensated running sum (Neumaier): each addition's rounding error is
 * recovered exactly by the branch-free two-sum and accumulated in comp, so a
 * large term that enters and later leaves a small sum leaves no residue
 * (Kahan's form assumes the sum outweighs the term and does not) */
struct CompSum {
    float s = 0.f, comp = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        const float t = s + v;
        const float bp = t - s;
        comp += (s - (t - bp)) + (v - bp);
        s = t;
    }
    __device__ __forceinline__ float value() const { return s + comp; }
};


__device__ __forceinline__ void ldv(const float *p, float *v, int V)
{
    if (V == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    } else if (V == 2) {
        const float2 q = *reinterpret_cast<const float2 *>(p);
        v[0] = q.x;
        v[1] = q.y;
    } else {
        v[0] = *p;
    }
}

/* bit i of the low 32/V bits of x moved to bit V*i (V = 2: the low 16 bits
 * to the even positions; V = 4: the low 8 bits to every fourth) */
template <int V>
__device__ __forceinline__ unsigned int spread_bits(unsigned int x)
{
    if (V == 2) {
        x &= 0xffffu;
        x = (x | (x << 8)) & 0x00ff00ffu;
        x = (x | (x << 4)) & 0x0f0f0f0fu;
        x = (x | (x << 2)) & 0x33333333u;
        x = (x | (x << 1)) & 0x55555555u;
    } else if (V == 4) {
        x &= 0xffu;
        x = (x | (x << 12)) & 0x000f000fu;
        x = (x | (x << 6)) & 0x03030303u;
        x = (x | (x << 3)) & 0x11111111u;
    }
    return x;
}

/* MODE 0: mean / std cubes; 1: mask words set; 2: mask words OR-ed;
 * 3: z-score cube (c - mean) / std, 0 where std = 0, into `mean`.
 * V consecutive z per thread (V-element loads; a warp covers 32 V z and V
 * mask words).  Each step's loads are issued one step ahead. */
template <int MODE, int V>
__global__ void __launch_bounds__(kXThreads, V == 4 ? 4 : 8)
    sf_local_x(const float *__restrict__ c, const float *__restrict__ A, const float *__restrict__ M, i64 nx,
               i64 ny, i64 nz, i64 nw32, int sx, int sy, int sz, int ddof, float k, float *__restrict__ mean,
               float *__restrict__ stdv, unsigned int *__restrict__ mask)
{
    /* lanes per row: 32 / V per mask word, whole warps per row */
    const i64 words_pad = (nw32 + V - 1) / V * V;
    const i64 per_row = words_pad * (32 / V);
    const i64 lane = (i64)blockIdx.x * kXThreads + threadIdx.x;
    const i64 y = lane / per_row;
    if (y >= ny) return;   /* whole warps */
    const i64 lr = lane - y * per_row;
    const i64 z = lr * V;
    const int wl = threadIdx.x & 31;
    bool valid[V];
    float nyz[V], rnyz[V];
    for (int e = 0; e < V; ++e) {
        valid[e] = z + e < nz;
        nyz[e] = (float)(clipped(y, sy, ny) * (valid[e] ? clipped(z + e, sz, nz) : 1));
        rnyz[e] = __frcp_rn(nyz[e]);
    }
    const i64 plane = ny * nz;
    const i64 off = y * nz + (valid[0] ? z : 0);
    const float *pa = A + off, *pm = M + off, *pc = c + off;
    const int nxi = (int)nx;
    const int x0 = (int)blockIdx.y * kXSeg;
    const int x1 = min(x0 + kXSeg, nxi);
    const int Xfull = 2 * sx + 1;
    const float rXfull = __frcp_rn((float)Xfull);
    /* segment blockIdx.y of kXSeg planes: the sums start from a direct sum
     * over the box of the segment's first plane, shifted by that plane's A,
     * so the running updates neither drift nor cancel */
    float s[V];
    ldv(pa + (i64)x0 * plane, s, V);
    CompSum sa[V], sb[V], sm[V];   /* sums over the x box of A - s, (A - s)^2, M */
    {
        const int lo = max(x0 - sx, 0), hi = min(x0 + sx, nxi - 1);
        for (int xi = lo; xi <= hi; ++xi) {
            float a[V], m[V];
            ldv(pa + (i64)xi * plane, a, V);
            ldv(pm + (i64)xi * plane, m, V);
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const float d = a[e] - s[e];
                sa[e].add(d);
                sb[e].add(d * d);
                sm[e].add(m[e]);
            }
        }
    }
    /* the loads of step x: planes entering (x + sx) and leaving (x - sx - 1)
     * the box (plane 0 where there is none), and plane x */
    auto load = [&](int x, float *ain, float *min_, float *aout, float *mout, float *cv) {
        const bool hin = x > x0 && x + sx < nxi, hout = x > x0 && x - sx - 1 >= 0;
        const i64 pin = hin ? (i64)(x + sx) * plane : 0, pout = hout ? (i64)(x - sx - 1) * plane : 0;
        ldv(pa + pin, ain, V);
        ldv(pm + pin, min_, V);
        ldv(pa + pout, aout, V);
        ldv(pm + pout, mout, V);
        if (MODE != 0) ldv(pc + (i64)x * plane, cv, V);
    };
    float ain[V], min_[V], aout[V], mout[V], cv[V] = {};
    load(x0, ain, min_, aout, mout, cv);
    for (int x = x0; x < x1; ++x) {
        float nain[V], nmin[V], naout[V], nmout[V], ncv[V] = {};
        load(min(x + 1, x1 - 1), nain, nmin, naout, nmout, ncv);
        const bool hin = x > x0 && x + sx < nxi, hout = x > x0 && x - sx - 1 >= 0;
        const int X = min(x + sx, nxi - 1) - max(x - sx, 0) + 1;
        const float rX = X == Xfull ? rXfull : __frcp_rn((float)X);
        float mu[V], sd[V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
            if (hin) {
                const float d = ain[e] - s[e];
                sa[e].add(d);
                sb[e].add(d * d);
                sm[e].add(min_[e]);
            }
            if (hout) {
                const float d = aout[e] - s[e];
                sa[e].add(-d);
                sb[e].add(-(d * d));
                sm[e].add(-mout[e]);
            }
            float m2;
            if (sx == 0) {
                /* the x box is the plane itself */
                float a1[V], m1[V];
                ldv(pa + (i64)x * plane, a1, V);
                ldv(pm + (i64)x * plane, m1, V);
                mu[e] = a1[e];
                m2 = m1[e];
            } else {
                const float Sa = sa[e].value(), Sb = sb[e].value(), Sm = sm[e].value();
                const float da = Sa * rX;
                mu[e] = s[e] + da;
                /* a rounded product (no contraction into an fma) */
                m2 = Sm + nyz[e] * fmaxf(Sb - __fmul_rn(Sa, da), 0.f);
            }
            if (ddof == 0) {
                sd[e] = sqrtf(m2 * rX * rnyz[e]);
            } else {
                /* sample std: over n - 1 */
                const float nn = (float)X * nyz[e] - 1.f;
                sd[e] = nn > 0.f ? sqrtf(m2 / nn) : 0.f;
            }
        }
        if (MODE == 0) {
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (valid[e]) {
                    mean[(i64)x * plane + off + e] = mu[e];
                    stdv[(i64)x * plane + off + e] = sd[e];
                }
        } else if (MODE == 3) {
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (valid[e]) mean[(i64)x * plane + off + e] = sd[e] > 0.f ? (cv[e] - mu[e]) / sd[e] : 0.f;
        } else {
            unsigned int bits[V];
#pragma unroll
            for (int e = 0; e < V; ++e)
                bits[e] = __ballot_sync(0xffffffffu, valid[e] && cv[e] > fmaf(k, sd[e], mu[e]));
            unsigned int word = bits[0];
            i64 wi = lr >> 5;   /* V == 1: word of this warp */
            if (V > 1) {
                /* lanes 0 .. V-1 assemble the warp's V words: word h holds
                 * lanes (32/V) h .. (32/V)(h+1) - 1, V bits each */
                const int h = wl & (V - 1);
                word = 0;
#pragma unroll
                for (int e = 0; e < V; ++e) word |= spread_bits<V>(bits[e] >> ((32 / V) * h)) << e;
                wi = (lr >> 5) * V + h;
            }
            if (wl < V && wi < nw32) {
                unsigned int *w = mask + ((i64)x * ny + y) * nw32 + wi;
                if (MODE == 2) {
                    if (word) atomicOr(w, word);   /* nothing waits on it */
                } else {
                    *w = word;
                }
            }
        }
#pragma unroll
        for (int e = 0; e < V; ++e) {
            ain[e] = nain[e];
            min_[e] = nmin[e];
            aout[e] = naout[e];
            mout[e] = nmout[e];
            cv[e] = ncv[e];
        }
    }
}

/* Boxes one, three or five voxels wide on some axis (a half-width below
 * kNarrow): the statistics of each voxel's clipped box in two passes over the box, the
 * mean first and then the sum of squared deviations from it, both with
 * compensated (Neumaier) sums.  Nothing cancels, at the cost of reading the
 * box once per pass for every voxel (O(box) work per voxel), which the thin
 * box keeps small.  One warp per (x, y, 32-z mask word): lane = z offset.
 * MODE as sf_local_x. */
constexpr int kNarrow = 3;
constexpr int kDThreads = 128;

template <int MODE>
__global__ void __launch_bounds__(kDThreads)
    sf_local_direct(const float *__restrict__ c, i64 nx, i64 ny, i64 nz, i64 nw32, int sx, int sy, int sz,
                    int ddof, float k, float *__restrict__ mean, float *__restrict__ stdv,
                    unsigned int *__restrict__ mask)
{
    const i64 wg = ((i64)blockIdx.x * kDThreads + threadIdx.x) >> 5;   /* warp: (x, y, word) */
    const int lane = threadIdx.x & 31;
    if (wg >= nx * ny * nw32) return;   /* whole warps */
    const i64 wi = wg % nw32, xy = wg / nw32;
    const i64 y = xy % ny, x = xy / ny;
    const i64 z = wi * 32 + lane;
    const bool valid = z < nz;
    const i64 zq = valid ? z : nz - 1;
    const i64 x0 = x - sx < 0 ? 0 : x - sx, x1 = x + sx >= nx ? nx - 1 : x + sx;
    const i64 y0 = y - sy < 0 ? 0 : y - sy, y1 = y + sy >= ny ? ny - 1 : y + sy;
    const i64 z0 = zq - sz < 0 ? 0 : zq - sz, z1 = zq + sz >= nz ? nz - 1 : zq + sz;
    const float n = (float)((x1 - x0 + 1) * (y1 - y0 + 1) * (z1 - z0 + 1));
    CompSum s1;
    for (i64 xi = x0; xi <= x1; ++xi)
        for (i64 yi = y0; yi <= y1; ++yi) {
            const float *row = c + (xi * ny + yi) * nz;
            for (i64 zi = z0; zi <= z1; ++zi) s1.add(__ldg(row + zi));
        }
    const float mu = s1.value() / n;
    CompSum s2;
    for (i64 xi = x0; xi <= x1; ++xi)
        for (i64 yi = y0; yi <= y1; ++yi) {
            const float *row = c + (xi * ny + yi) * nz;
            for (i64 zi = z0; zi <= z1; ++zi) {
                const float d = __ldg(row + zi) - mu;
                s2.add(d * d);
            }
        }
    const float q = fmaxf(s2.value(), 0.f);
    const float sd = ddof == 0 ? sqrtf(q / n) : (n > 1.f ? sqrtf(q / (n - 1.f)) : 0.f);
    const i64 v = (x * ny + y) * nz + zq;
    if (MODE == 0) {
        if (valid) {
            mean[v] = mu;
            stdv[v] = sd;
        }
    } else if (MODE == 3) {
        if (valid) mean[v] = sd > 0.f ? (c[v] - mu) / sd : 0.f;
    } else {
        const unsigned int word = __ballot_sync(0xffffffffu, valid && c[v] > fmaf(k, sd, mu));
        if (lane == 0) {
            unsigned int *w = mask + (x * ny + y) * nw32 + wi;
            if (MODE == 2) {
                if (word) atomicOr(w, word);
            } else {
                *w = word;
            }
        }
    }
}

}  // namespace

/* boxes with a half-width below kNarrow on some axis (and not the voxel
 * itself) take the two-pass direct kernel */
bool sf_local_is_narrow(int sx, int sy, int sz)
{
    const int lo = sx < sy ? (sx < sz ? sx : sz) : (sy < sz ? sy : sz);
    return lo < kNarrow && (sx | sy | sz) != 0;
}

cudaError_t sf_launch_local_direct(const float *c, long long nx, long long ny, long long nz, long long nw32,
                                   int sx, int sy, int sz, float k, float *mean, float *stdv, unsigned int *mask,
                                   int mode, int ddof, cudaStream_t st)
{
    const long long warps = nx * ny * nw32;
    const long long blocks = (warps * 32 + kDThreads - 1) / kDThreads;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
#define SF_LD(MODE) sf_local_direct<MODE><<<(unsigned)blocks, kDThreads, 0, st>>>(c, nx, ny, nz, nw32, sx, sy, sz, ddof, k, mean, stdv, mask)
    if (mode == 0) SF_LD(0);
    else if (mode == 1) SF_LD(1);
    else if (mode == 2) SF_LD(2);
    else SF_LD(3);
#undef SF_LD
    return cudaGetLastError();
}

/* shared memory of sf_local_yz for half-widths (sy, sz) */
size_t sf_local_yz_smem(int sy, int sz) { return sizeof(float) * yz_smem_floats(sy, sz); }

cudaError_t sf_launch_local_yz(const float *c, float *A, float *M, long long nx, long long ny, long long nz, int sy,
                               int sz, cudaStream_t st)
{
    if (ny > (1LL << 30) || nz > (1LL << 30)) return cudaErrorInvalidValue;
    if (sy == 0 && sz == 0) {
        /* the y-z box is the voxel: A = c and M = 0 exactly */
        const size_t bytes = (size_t)(nx * ny * nz) * sizeof(float);
        cudaError_t e = cudaMemcpyAsync(A, c, bytes, cudaMemcpyDeviceToDevice, st);
        return e == cudaSuccess ? cudaMemsetAsync(M, 0, bytes, st) : e;
    }
    const size_t smem = sf_local_yz_smem(sy, sz);
    /* y segments of at most kYRows rows, split evenly */
    const long long nseg = (ny + kYRows - 1) / kYRows;
    const int yrows = (int)((ny + nseg - 1) / nseg);
    const int hz = (sz + 3) & ~3;
    const dim3 grid((unsigned)((nz + hz - sz + kMZ - 1) / kMZ), (unsigned)nseg, (unsigned)nx);
    cudaError_t e;
    if (nz % 4 == 0) {
        e = cudaFuncSetAttribute(sf_local_yz<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        sf_local_yz<4><<<grid, kMT, smem, st>>>(c, A, M, ny, nz, sy, sz, yrows);
    } else {
        e = cudaFuncSetAttribute(sf_local_yz<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        sf_local_yz<1><<<grid, kMT, smem, st>>>(c, A, M, ny, nz, sy, sz, yrows);
    }
    return cudaGetLastError();
}

cudaError_t sf_launch_local_x(const float *c, const float *A, const float *M, long long nx, long long ny,
                              long long nz, long long nw32, int sx, int sy, int sz, float k, float *mean,
                              float *stdv, unsigned int *mask, int mode, int ddof, cudaStream_t st)
{
    if (nx > (1LL << 30)) return cudaErrorInvalidValue;
    /* z per thread: 2 when nz is even (8-byte loads), else 1; SF_LXV = 4
     * takes four where nz allows (16-byte loads, 120 registers: measured
     * slower with the compensated sums), SF_LXV = 1 one */
    int V = nz % 2 == 0 ? 2 : 1;
    if (const char *e = getenv("SF_LXV")) {
        const int want = atoi(e);
        if (want == 4 && nz % 4 == 0) V = 4;
        else if (want == 1) V = 1;
    }
    const long long lanes = ny * ((nw32 + V - 1) / V * V) * (32 / V);
    const dim3 grid((unsigned)((lanes + kXThreads - 1) / kXThreads), (unsigned)((nx + kXSeg - 1) / kXSeg));
#define SF_LX(MODE, VV) sf_local_x<MODE, VV><<<grid, kXThreads, 0, st>>>(c, A, M, nx, ny, nz, nw32, sx, sy, sz, ddof, k, mean, stdv, mask)
#define SF_LXV(VV)                     \
    if (mode == 0) SF_LX(0, VV);       \
    else if (mode == 1) SF_LX(1, VV);  \
    else if (mode == 2) SF_LX(2, VV);  \
    else SF_LX(3, VV);
    if (V == 4) {
        SF_LXV(4)
    } else if (V == 2) {
        SF_LXV(2)
    } else {
        SF_LXV(1)
    }
#undef SF_LXV
#undef SF_LX
    return cudaGetLastError();
}
