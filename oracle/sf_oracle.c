/*
 * FP64 CPU oracle for the Gaussian source-finder hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check in
 * __graft_entry__.py and the CPU-baseline leg of bench.py may load this code.
 * The CUDA library never links, calls or includes it, and it shares no code,
 * header, table or helper with the CUDA path.
 *
 * What it computes (Westerlund & Harris, "Performance Analysis of
 * GPU-Accelerated Filter-Based Source Finding for HI Spectral Line Image
 * Data"):
 *   - taps of a sampled, truncated, normalised 1D Gaussian per axis
 *     (Sec. 2.1: the finder applies several 3D Gaussian filters; Sec. 3.4:
 *     filter values are a small table of constants);
 *   - the unweighted 3D convolution of Eq. 2, with offsets o in [-R, R] per
 *     axis and the image taken as zero outside the cube, the 3D filter being
 *     the outer product of the three 1D tap vectors; evaluated either by three
 *     1D passes (x, then y, then z) or literally as the triple sum of Eq. 2;
 *   - the local mean and (population) standard deviation of the filtered cube
 *     over non-overlapping windows tiling the cube from the origin (Sec. 3.3);
 *   - the per-voxel threshold  c > mean + k * std  of the window holding the
 *     voxel (Sec. 3.3, "z-score" voxel selection), OR-ed over the filter bank
 *     and packed 32 consecutive z per uint32 word.
 *
 * Everything is plain loops in double precision, in the order the
 * definitions state them.  No blocking, fusion or reordering.
 *
 * Layout: cube[x][y][z], z contiguous (Sec. 3.1: X is the major axis and Z
 * the minor axis in memory).  Mask word index (x*ny + y)*ceil(nz/32) + z/32,
 * bit z%32.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Radius of a truncated Gaussian: R = ceil(truncation * sigma); sigma <= 0
 * means "no smoothing on this axis" (R = 0, a single unit tap). */
int or_radius(double sigma, double truncation)
{
    if (!(sigma > 0.0)) return 0;
    return (int)ceil(truncation * sigma);
}

/* Taps g[o + R] = exp(-o^2 / (2 sigma^2)) for o = -R..R, divided by their sum
 * so that they add up to one. */
void or_taps(double sigma, int R, double *g)
{
    if (R == 0) { g[0] = 1.0; return; }
    double sum = 0.0;
    for (int o = -R; o <= R; ++o) {
        g[o + R] = exp(-((double)o * (double)o) / (2.0 * sigma * sigma));
        sum += g[o + R];
    }
    for (int o = -R; o <= R; ++o) g[o + R] /= sum;
}

/* Image value with zero outside the cube. */
static double at(const float *d, int64_t nx, int64_t ny, int64_t nz,
                 int64_t x, int64_t y, int64_t z, int take_abs)
{
    if (x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz) return 0.0;
    double v = (double)d[(x * ny + y) * nz + z];
    return take_abs ? fabs(v) : v;
}

/*
 * Filtered values on the box [x0,x1) x [y0,y1) x [z0,z1) of the cube, by three
 * 1D passes: t1 = gx * d along x, t2 = gy * t1 along y, c = gz * t2 along z.
 * Each pass is evaluated on the part of the box (plus the halo the later
 * passes need) only.  take_abs != 0 filters |d| instead of d (the error scale
 * used by the tests).  out is [x1-x0][y1-y0][z1-z0], z fastest.
 * Returns 0, or -1 when memory runs out.
 */
int or_filter_box(const float *d, int64_t nx, int64_t ny, int64_t nz,
                  const double *gx, int rx, const double *gy, int ry,
                  const double *gz, int rz,
                  int64_t x0, int64_t x1, int64_t y0, int64_t y1,
                  int64_t z0, int64_t z1, int take_abs, double *out)
{
    const int64_t ex = x1 - x0, ey = y1 - y0, ez = z1 - z0;
    const int64_t eyh = ey + 2 * ry, ezh = ez + 2 * rz;
    double *t1 = (double *)malloc(sizeof(double) * (size_t)(ex * eyh * ezh));
    double *t2 = (double *)malloc(sizeof(double) * (size_t)(ex * ey * ezh));
    if (!t1 || !t2) { free(t1); free(t2); return -1; }

    /* x pass on [x0,x1) x [y0-ry, y1+ry) x [z0-rz, z1+rz) */
    for (int64_t i = 0; i < ex; ++i)
        for (int64_t j = 0; j < eyh; ++j)
            for (int64_t k = 0; k < ezh; ++k) {
                const int64_t x = x0 + i, y = y0 - ry + j, z = z0 - rz + k;
                double s = 0.0;
                for (int o = -rx; o <= rx; ++o)
                    s += gx[o + rx] * at(d, nx, ny, nz, x + o, y, z, take_abs);
                t1[(i * eyh + j) * ezh + k] = s;
            }
    /* y pass on [x0,x1) x [y0,y1) x [z0-rz, z1+rz) */
    for (int64_t i = 0; i < ex; ++i)
        for (int64_t j = 0; j < ey; ++j)
            for (int64_t k = 0; k < ezh; ++k) {
                double s = 0.0;
                for (int o = -ry; o <= ry; ++o)
                    s += gy[o + ry] * t1[(i * eyh + (j + ry + o)) * ezh + k];
                t2[(i * ey + j) * ezh + k] = s;
            }
    /* z pass on the box */
    for (int64_t i = 0; i < ex; ++i)
        for (int64_t j = 0; j < ey; ++j)
            for (int64_t k = 0; k < ez; ++k) {
                double s = 0.0;
                for (int o = -rz; o <= rz; ++o)
                    s += gz[o + rz] * t2[(i * ey + j) * ezh + (k + rz + o)];
                out[(i * ey + j) * ez + k] = s;
            }
    free(t1);
    free(t2);
    return 0;
}

/* Eq. 2 written out literally for one voxel: the triple sum over the filter
 * offsets of d[x+ox][y+oy][z+oz] * f[ox][oy][oz], f = gx (x) gy (x) gz. */
double or_filter_direct_voxel(const float *d, int64_t nx, int64_t ny, int64_t nz,
                              const double *gx, int rx, const double *gy, int ry,
                              const double *gz, int rz,
                              int64_t x, int64_t y, int64_t z)
{
    double s = 0.0;
    for (int ox = -rx; ox <= rx; ++ox)
        for (int oy = -ry; oy <= ry; ++oy)
            for (int oz = -rz; oz <= rz; ++oz) {
                const double f = gx[ox + rx] * gy[oy + ry] * gz[oz + rz];
                s += at(d, nx, ny, nz, x + ox, y + oy, z + oz, 0) * f;
            }
    return s;
}

/* Mean and standard deviation of n values, two passes: the squared
 * deviations divided by n - ddof (ddof 0: population, 1: sample; 0 when
 * n <= ddof). */
void or_moments(const double *c, int64_t n, int ddof, double *mean, double *stdv)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += c[i];
    const double m = s / (double)n;
    double q = 0.0;
    for (int64_t i = 0; i < n; ++i) q += (c[i] - m) * (c[i] - m);
    *mean = m;
    *stdv = n > ddof ? sqrt(q / (double)(n - ddof)) : 0.0;
}

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

/*
 * Window statistics of a whole filtered cube c (double, [x][y][z]).
 * Windows tile the cube from the origin: window (a,b,e) covers
 * [a*wx, min((a+1)*wx, nx)) x ... ; tail windows hold the voxels present.
 * mean/stdv are [nwx][nwy][nwz].
 */
int or_window_stats(const double *c, int64_t nx, int64_t ny, int64_t nz,
                    int wx, int wy, int wz, int ddof, double *mean, double *stdv)
{
    const int64_t nwx = ceil_div(nx, wx), nwy = ceil_div(ny, wy), nwz = ceil_div(nz, wz);
    double *buf = (double *)malloc(sizeof(double) * (size_t)wx * wy * wz);
    if (!buf) return -1;
    for (int64_t a = 0; a < nwx; ++a)
        for (int64_t b = 0; b < nwy; ++b)
            for (int64_t e = 0; e < nwz; ++e) {
                int64_t n = 0;
                for (int64_t x = a * wx; x < nx && x < (a + 1) * wx; ++x)
                    for (int64_t y = b * wy; y < ny && y < (b + 1) * wy; ++y)
                        for (int64_t z = e * wz; z < nz && z < (e + 1) * wz; ++z)
                            buf[n++] = c[(x * ny + y) * nz + z];
                const int64_t w = (a * nwy + b) * nwz + e;
                or_moments(buf, n, ddof, &mean[w], &stdv[w]);
            }
    free(buf);
    return 0;
}

/*
 * Threshold of one filtered cube against its window statistics:
 * voxel fires when c > mean + k*std (strict).  Fired voxels are OR-ed into
 * mask (packed words, caller zeroes it first).  When amb != NULL, voxels with
 * |c - T| < band_rel * std are OR-ed into amb (same packing): there the
 * decision depends on rounding.
 */
void or_threshold(const double *c, int64_t nx, int64_t ny, int64_t nz,
                  int wx, int wy, int wz, const double *mean, const double *stdv,
                  double k, double band_rel, uint32_t *mask, uint32_t *amb)
{
    const int64_t nwy = ceil_div(ny, wy), nwz = ceil_div(nz, wz);
    const int64_t nw32 = ceil_div(nz, 32);
    for (int64_t x = 0; x < nx; ++x)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t z = 0; z < nz; ++z) {
                const int64_t w = ((x / wx) * nwy + y / wy) * nwz + z / wz;
                const double T = mean[w] + k * stdv[w];
                const double v = c[(x * ny + y) * nz + z];
                const int64_t word = (x * ny + y) * nw32 + z / 32;
                const uint32_t bit = 1u << (z % 32);
                if (v > T) mask[word] |= bit;
                if (amb && fabs(v - T) < band_rel * stdv[w]) amb[word] |= bit;
            }
}

/*
 * One window of the whole method for a bank of nf filters: filter f uses the
 * spatial taps gxy_f on x and on y and the spectral taps gz_f on z.
 * Taps are concatenated: filter f's spatial taps start at sum_{g<f}(2 rxy[g]+1).
 *
 * Outputs for window (a,b,e):
 *   mean[f], stdv[f]                         window statistics per filter;
 *   fire[v]   (v over the window's voxels)   OR over filters of c_f > T_f;
 *   sure[v]   1 unless the OR could flip with rounding: some filter has
 *             |c_f - T_f| < band_rel*std_f and no filter fires by more
 *             than that band;
 *   cvals     (optional) [nf][window voxels] filtered values;
 *   thr       (optional) [nf] thresholds T_f.
 * Window voxels are ordered [x][y][z] over the window's extent.
 */
int or_detect_window(const float *d, int64_t nx, int64_t ny, int64_t nz,
                     int nf, const int *rxy, const double *gxy_all,
                     const int *rz, const double *gz_all,
                     int wx, int wy, int wz, int ddof, double k, double band_rel,
                     int64_t a, int64_t b, int64_t e,
                     double *mean, double *stdv, uint8_t *fire, uint8_t *sure,
                     double *cvals, double *thr)
{
    const int64_t x0 = a * wx, y0 = b * wy, z0 = e * wz;
    const int64_t x1 = (x0 + wx < nx) ? x0 + wx : nx;
    const int64_t y1 = (y0 + wy < ny) ? y0 + wy : ny;
    const int64_t z1 = (z0 + wz < nz) ? z0 + wz : nz;
    const int64_t n = (x1 - x0) * (y1 - y0) * (z1 - z0);
    double *c = (double *)malloc(sizeof(double) * (size_t)n);
    if (!c) return -1;
    uint8_t *amb = (uint8_t *)calloc((size_t)n, 1);
    uint8_t *big = (uint8_t *)calloc((size_t)n, 1);
    if (!amb || !big) { free(c); free(amb); free(big); return -1; }
    memset(fire, 0, (size_t)n);
    int64_t oxy = 0, oz = 0;
    for (int f = 0; f < nf; ++f) {
        const double *gxy = gxy_all + oxy, *gz = gz_all + oz;
        if (or_filter_box(d, nx, ny, nz, gxy, rxy[f], gxy, rxy[f], gz, rz[f],
                          x0, x1, y0, y1, z0, z1, 0, c) != 0) {
            free(c); free(amb); free(big); return -1;
        }
        or_moments(c, n, ddof, &mean[f], &stdv[f]);
        const double T = mean[f] + k * stdv[f];
        const double band = band_rel * stdv[f];
        if (thr) thr[f] = T;
        for (int64_t v = 0; v < n; ++v) {
            if (c[v] > T) fire[v] = 1;
            if (fabs(c[v] - T) < band) amb[v] = 1;
            else if (c[v] > T) big[v] = 1;
            if (cvals) cvals[(int64_t)f * n + v] = c[v];
        }
        oxy += 2 * rxy[f] + 1;
        oz += 2 * rz[f] + 1;
    }
    for (int64_t v = 0; v < n; ++v) sure[v] = (uint8_t)(big[v] || !amb[v]);
    free(c); free(amb); free(big);
    return 0;
}

/*
 * The whole cube: every window through or_detect_window, in parallel over
 * windows with nthreads OpenMP threads (<= 0: the runtime's default).
 * mask and sure are packed words (zeroed here); mean/stdv are
 * [nf][nwx][nwy][nwz].  Returns the number of threads used, or -1.
 */
int or_detect(const float *d, int64_t nx, int64_t ny, int64_t nz,
              int nf, const int *rxy, const double *gxy_all,
              const int *rz, const double *gz_all,
              int wx, int wy, int wz, int ddof, double k, double band_rel,
              uint32_t *mask, uint32_t *sure_words, double *mean, double *stdv,
              int nthreads)
{
    const int64_t nwx = ceil_div(nx, wx), nwy = ceil_div(ny, wy), nwz = ceil_div(nz, wz);
    const int64_t nwin = nwx * nwy * nwz, nw32 = ceil_div(nz, 32);
    memset(mask, 0, sizeof(uint32_t) * (size_t)(nx * ny * nw32));
    memset(sure_words, 0, sizeof(uint32_t) * (size_t)(nx * ny * nw32));
    int used = 1, failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#else
    (void)nthreads;
#endif
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t w = 0; w < nwin; ++w) {
        const int64_t a = w / (nwy * nwz), b = (w / nwz) % nwy, e = w % nwz;
        const size_t nvox = (size_t)wx * wy * wz;
        uint8_t *fire = (uint8_t *)malloc(nvox), *sure = (uint8_t *)malloc(nvox);
        double *m = (double *)malloc(sizeof(double) * (size_t)nf);
        double *s = (double *)malloc(sizeof(double) * (size_t)nf);
        if (!fire || !sure || !m || !s ||
            or_detect_window(d, nx, ny, nz, nf, rxy, gxy_all, rz, gz_all, wx, wy, wz,
                             ddof, k, band_rel, a, b, e, m, s, fire, sure, NULL, NULL) != 0) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            failed = 1;
        } else {
            for (int f = 0; f < nf; ++f) {
                mean[(int64_t)f * nwin + w] = m[f];
                stdv[(int64_t)f * nwin + w] = s[f];
            }
            const int64_t x0 = a * wx, y0 = b * wy, z0 = e * wz;
            const int64_t x1 = (x0 + wx < nx) ? x0 + wx : nx;
            const int64_t y1 = (y0 + wy < ny) ? y0 + wy : ny;
            const int64_t z1 = (z0 + wz < nz) ? z0 + wz : nz;
            int64_t v = 0;
            for (int64_t x = x0; x < x1; ++x)
                for (int64_t y = y0; y < y1; ++y)
                    for (int64_t z = z0; z < z1; ++z, ++v) {
                        const int64_t word = (x * ny + y) * nw32 + z / 32;
                        const uint32_t bit = 1u << (z % 32);
                        /* a word may hold voxels of two windows along z:
                         * update it atomically */
                        if (fire[v]) {
#ifdef _OPENMP
#pragma omp atomic update
#endif
                            mask[word] |= bit;
                        }
                        if (sure[v]) {
#ifdef _OPENMP
#pragma omp atomic update
#endif
                            sure_words[word] |= bit;
                        }
                    }
        }
        free(fire); free(sure); free(m); free(s);
    }
    return failed ? -1 : used;
}

/*
 * A listed subset of windows through or_detect_window, in parallel over the
 * list with nthreads OpenMP threads (<= 0: the runtime's default).  widx holds
 * n (a, b, e) triples; fired[i] receives the number of voxels of window i that
 * fire.  Used to time the oracle on a bounded sample of a large cube.
 * Returns the number of threads used, or -1.
 */
int or_detect_windows(const float *d, int64_t nx, int64_t ny, int64_t nz,
                      int nf, const int *rxy, const double *gxy_all,
                      const int *rz, const double *gz_all,
                      int wx, int wy, int wz, int ddof, double k, double band_rel,
                      int64_t n, const int64_t *widx, int64_t *fired, int nthreads)
{
    int used = 1, failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#else
    (void)nthreads;
#endif
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < n; ++i) {
        const size_t nvox = (size_t)wx * wy * wz;
        uint8_t *fire = (uint8_t *)malloc(nvox), *sure = (uint8_t *)malloc(nvox);
        double *m = (double *)malloc(sizeof(double) * (size_t)nf);
        double *s = (double *)malloc(sizeof(double) * (size_t)nf);
        int64_t cnt = -1;
        if (fire && sure && m && s &&
            or_detect_window(d, nx, ny, nz, nf, rxy, gxy_all, rz, gz_all, wx, wy, wz, ddof, k, band_rel,
                             widx[3 * i], widx[3 * i + 1], widx[3 * i + 2], m, s, fire, sure,
                             NULL, NULL) == 0) {
            const int64_t x0 = widx[3 * i] * wx, y0 = widx[3 * i + 1] * wy, z0 = widx[3 * i + 2] * wz;
            const int64_t ex = (x0 + wx < nx ? wx : nx - x0), ey = (y0 + wy < ny ? wy : ny - y0),
                          ez = (z0 + wz < nz ? wz : nz - z0);
            cnt = 0;
            for (int64_t v = 0; v < ex * ey * ez; ++v) cnt += fire[v];
        } else {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            failed = 1;
        }
        fired[i] = cnt;
        free(fire); free(sure); free(m); free(s);
    }
    return failed ? -1 : used;
}

/*
 * Local statistics per voxel (Sec. 3.3: the mean and standard deviation of
 * each voxel come from a user-specified range of the filtered data around it),
 * read as the box [x-sx, x+sx] x [y-sy, y+sy] x [z-sz, z+sz] clipped to the
 * cube, n = number of voxels in the clipped box, population statistics (two
 * passes: the mean, then the mean squared deviation).
 *
 * c: filtered cube [x][y][z] (double).  The voxels evaluated are the n_idx
 * flat indices in idx, or every voxel when idx is NULL; mean/stdv receive one
 * value per evaluated voxel, in that order.  Returns the OpenMP threads used.
 */
int or_local_stats(const double *c, int64_t nx, int64_t ny, int64_t nz, int sx, int sy, int sz,
                   int ddof, const int64_t *idx, int64_t n_idx, double *mean, double *stdv, int nthreads)
{
    const int64_t nv = idx ? n_idx : nx * ny * nz;
    int used = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#else
    (void)nthreads;
#endif
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t i = 0; i < nv; ++i) {
        const int64_t v = idx ? idx[i] : i;
        const int64_t x = v / (ny * nz), y = (v / nz) % ny, z = v % nz;
        const int64_t x0 = x - sx < 0 ? 0 : x - sx, x1 = x + sx >= nx ? nx - 1 : x + sx;
        const int64_t y0 = y - sy < 0 ? 0 : y - sy, y1 = y + sy >= ny ? ny - 1 : y + sy;
        const int64_t z0 = z - sz < 0 ? 0 : z - sz, z1 = z + sz >= nz ? nz - 1 : z + sz;
        double s = 0.0;
        int64_t n = 0;
        for (int64_t a = x0; a <= x1; ++a)
            for (int64_t b = y0; b <= y1; ++b)
                for (int64_t e = z0; e <= z1; ++e) {
                    s += c[(a * ny + b) * nz + e];
                    ++n;
                }
        const double m = s / (double)n;
        double q = 0.0;
        for (int64_t a = x0; a <= x1; ++a)
            for (int64_t b = y0; b <= y1; ++b)
                for (int64_t e = z0; e <= z1; ++e) {
                    const double d = c[(a * ny + b) * nz + e] - m;
                    q += d * d;
                }
        mean[i] = m;
        stdv[i] = n > ddof ? sqrt(q / (double)(n - ddof)) : 0.0;
    }
    return used;
}

/*
 * Eq. 1 (weighted convolution) on the box [x0,x1) x [y0,y1) x [z0,z1):
 *   c_w = sum_o d[i] f[o] w[i] / D,  i = v + o over the filter offsets,
 * with d and w zero outside the cube.  The denominator is read two ways (the
 * printed form sums w alone, which does not reduce to Eq. 2 for unit
 * weights):
 *   den_mode 0  D = sum_o f[o] w[i]   (normalised convolution; w = 1 gives
 *                                      Eq. 2 wherever the support is inside);
 *   den_mode 1  D = sum_o w[i]        (as printed).
 * Where D = 0 (no weight in the support) c_w = 0.  Both sums use the same
 * three 1D passes as or_filter_box (x, then y, then z), on the product d*w
 * and on w, in double precision.  out is [x1-x0][y1-y0][z1-z0].
 * Returns 0, or -1 when memory runs out.
 */
static void passes3(const double *src, int64_t ex, int64_t ey, int64_t ez, const double *gx, int rx,
                    const double *gy, int ry, const double *gz, int rz, double *t1, double *t2,
                    double *out)
{
    /* src covers [x0-rx, x1+rx) x [y0-ry, y1+ry) x [z0-rz, z1+rz) */
    const int64_t exh = ex + 2 * rx, eyh = ey + 2 * ry, ezh = ez + 2 * rz;
    for (int64_t i = 0; i < ex; ++i)
        for (int64_t j = 0; j < eyh; ++j)
            for (int64_t k = 0; k < ezh; ++k) {
                double s = 0.0;
                for (int o = -rx; o <= rx; ++o)
                    s += gx[o + rx] * src[((i + rx + o) * eyh + j) * ezh + k];
                t1[(i * eyh + j) * ezh + k] = s;
            }
    (void)exh;
    for (int64_t i = 0; i < ex; ++i)
        for (int64_t j = 0; j < ey; ++j)
            for (int64_t k = 0; k < ezh; ++k) {
                double s = 0.0;
                for (int o = -ry; o <= ry; ++o)
                    s += gy[o + ry] * t1[(i * eyh + (j + ry + o)) * ezh + k];
                t2[(i * ey + j) * ezh + k] = s;
            }
    for (int64_t i = 0; i < ex; ++i)
        for (int64_t j = 0; j < ey; ++j)
            for (int64_t k = 0; k < ez; ++k) {
                double s = 0.0;
                for (int o = -rz; o <= rz; ++o)
                    s += gz[o + rz] * t2[(i * ey + j) * ezh + (k + rz + o)];
                out[(i * ey + j) * ez + k] = s;
            }
}

int or_weighted_filter_box(const float *d, const float *w, int64_t nx, int64_t ny, int64_t nz,
                           const double *gx, int rx, const double *gy, int ry, const double *gz, int rz,
                           int den_mode, int64_t x0, int64_t x1, int64_t y0, int64_t y1, int64_t z0,
                           int64_t z1, double *out)
{
    const int64_t ex = x1 - x0, ey = y1 - y0, ez = z1 - z0;
    const int64_t exh = ex + 2 * rx, eyh = ey + 2 * ry, ezh = ez + 2 * rz;
    const size_t nh = (size_t)(exh * eyh * ezh), nb = (size_t)(ex * ey * ez);
    double *pw = (double *)malloc(sizeof(double) * nh), *ww = (double *)malloc(sizeof(double) * nh);
    double *t1 = (double *)malloc(sizeof(double) * (size_t)(ex * eyh * ezh));
    double *t2 = (double *)malloc(sizeof(double) * (size_t)(ex * ey * ezh));
    double *num = (double *)malloc(sizeof(double) * nb), *den = (double *)malloc(sizeof(double) * nb);
    double *ones = (double *)malloc(sizeof(double) * (size_t)(2 * (rx > ry ? (rx > rz ? rx : rz) : (ry > rz ? ry : rz)) + 1));
    if (!pw || !ww || !t1 || !t2 || !num || !den || !ones) {
        free(pw); free(ww); free(t1); free(t2); free(num); free(den); free(ones);
        return -1;
    }
    for (int64_t i = 0; i < exh; ++i)
        for (int64_t j = 0; j < eyh; ++j)
            for (int64_t k = 0; k < ezh; ++k) {
                const int64_t x = x0 - rx + i, y = y0 - ry + j, z = z0 - rz + k;
                const size_t q = (size_t)((i * eyh + j) * ezh + k);
                if (x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz) {
                    pw[q] = 0.0;
                    ww[q] = 0.0;
                } else {
                    const size_t v = (size_t)((x * ny + y) * nz + z);
                    pw[q] = (double)d[v] * (double)w[v];
                    ww[q] = (double)w[v];
                }
            }
    passes3(pw, ex, ey, ez, gx, rx, gy, ry, gz, rz, t1, t2, num);
    if (den_mode == 0) {
        passes3(ww, ex, ey, ez, gx, rx, gy, ry, gz, rz, t1, t2, den);
    } else {
        const int rm = rx > ry ? (rx > rz ? rx : rz) : (ry > rz ? ry : rz);
        for (int o = 0; o <= 2 * rm; ++o) ones[o] = 1.0;
        passes3(ww, ex, ey, ez, ones, rx, ones, ry, ones, rz, t1, t2, den);
    }
    for (size_t v = 0; v < nb; ++v) out[v] = den[v] != 0.0 ? num[v] / den[v] : 0.0;
    free(pw); free(ww); free(t1); free(t2); free(num); free(den); free(ones);
    return 0;
}

/* Eq. 1 written out literally for one voxel: the triple sums of the
 * numerator and of the denominator (den_mode as above). */
double or_weighted_direct_voxel(const float *d, const float *w, int64_t nx, int64_t ny, int64_t nz,
                                const double *gx, int rx, const double *gy, int ry, const double *gz,
                                int rz, int den_mode, int64_t x, int64_t y, int64_t z)
{
    double num = 0.0, den = 0.0;
    for (int ox = -rx; ox <= rx; ++ox)
        for (int oy = -ry; oy <= ry; ++oy)
            for (int oz = -rz; oz <= rz; ++oz) {
                const double f = gx[ox + rx] * gy[oy + ry] * gz[oz + rz];
                const double wv = at(w, nx, ny, nz, x + ox, y + oy, z + oz, 0);
                num += at(d, nx, ny, nz, x + ox, y + oy, z + oz, 0) * f * wv;
                den += den_mode == 0 ? f * wv : wv;
            }
    return den != 0.0 ? num / den : 0.0;
}
