/*
 * sf.h — C ABI of the GB300 Gaussian source-finder hot path.
 *
 * The library applies a bank of separable 3D Gaussian filters to an HI
 * spectral cube, computes the mean and standard deviation of every filtered
 * cube over windows, marks the voxels whose filtered value exceeds
 * mean + k * std of their window, and ORs the marks of all filters into one
 * bit-packed mask (Westerlund & Harris, Sec. 2.1 Eq. 2 for the filter,
 * Sec. 3.3 for the local statistics and the z-score voxel selection).
 *
 * Conventions shared by every entry point:
 *   - Cube layout is cube[x][y][z], z (frequency) contiguous, x the major
 *     axis (Sec. 3.1).  1 <= nx, ny, nz <= 2^31; an empty cube (a zero
 *     extent) is refused with SF_EINVAL before any device work.
 *   - Pointers prefixed d_ are device pointers, h_ host pointers.  The caller
 *     owns every buffer it passes and must keep it alive until the work
 *     enqueued on `stream` has finished.  Device pointers must be 16-byte
 *     aligned.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *     entry points only enqueue work and return; they do not synchronise.
 *   - The context owns the filter taps, the execution plan, the compiled
 *     kernels and its scratch buffers (the x-filtered cubes, one per distinct
 *     non-zero sigma_xy).  Calls on one context are not thread-safe and must
 *     not overlap on the GPU (use one context per concurrent stream).
 *   - Errors are return codes; sf_last_error() gives a message.  Arguments
 *     are validated on the host before anything is enqueued.  After a CUDA
 *     error the context returns SF_ESTATE until it is destroyed.
 *   - Mask layout: uint32 words, word (x*ny + y)*ceil(nz/32) + z/32 holds
 *     voxel (x, y, z) in bit z%32; bits beyond nz in the last word of a row
 *     are zero.
 *   - Windows tile the cube from the origin: window (a, b, e) covers
 *     [a*wx, min((a+1)*wx, nx)) x [b*wy, ...) x [e*wz, ...); tail windows
 *     hold the voxels present.  Statistics arrays are float32
 *     [n_filters][nwx][nwy][nwz] (sf_stats: [nwx][nwy][nwz]).
 */
#ifndef SF_H
#define SF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sf_ctx sf_ctx;

typedef enum sf_status {
    SF_OK = 0,
    SF_EINVAL = 1,    /* invalid argument or configuration */
    SF_ENOMEM = 2,    /* device or host allocation failed */
    SF_EBUDGET = 3,   /* request does not fit the memory budget (serving) */
    SF_ECUDA = 4,     /* CUDA runtime error */
    SF_ETIMEOUT = 5,  /* a bounded wait expired */
    SF_ESTATE = 6,    /* context unusable after an earlier CUDA error */
    SF_EJIT = 7,      /* run-time compilation of a kernel failed */
    SF_ECANCELED = 8  /* a served request was cancelled before admission */
} sf_status;

typedef enum sf_dtype {
    SF_F32 = 0,       /* float32 storage of the cube and intermediates */
    SF_F16 = 1,       /* IEEE half storage, float32 arithmetic */
    SF_BF16 = 2       /* bfloat16 storage, float32 arithmetic */
} sf_dtype;

/* One filter of the bank: Gaussian sigma along x and y (in pixels; 0 means
 * no spatial smoothing) and along z (in channels). */
typedef struct sf_filter_spec {
    float sigma_xy;
    float sigma_z;
} sf_filter_spec;

typedef struct sf_config {
    int64_t nx, ny, nz;            /* cube dimensions */
    int32_t n_filters;             /* 1 .. 64 */
    const sf_filter_spec *filters; /* copied by sf_create */
    float truncation;              /* radius R = ceil(truncation*sigma) per axis */
    int32_t wx, wy, wz;            /* statistics window (>= 1 each) */
    float k;                       /* threshold multiplier */
    int32_t storage;               /* sf_dtype of the cube and the x-filtered scratch */
    int32_t stats_fp64;            /* window statistics: 0 merges the per-thread FP32 partial
                                    * moments in FP32, 1 in FP64 (Chan's pairwise merge) */
    int32_t device;                /* CUDA device ordinal, -1 = current device */
    int32_t std_ddof;              /* standard deviation: squared deviations over n - std_ddof;
                                    * 0 population (the default), 1 sample; std = 0 when
                                    * n <= std_ddof.  Applies to every statistic. */
} sf_config;

/* Create a context: copies cfg, computes the taps (Sec. 2.1: sampled Gaussian
 * exp(-o^2/2sigma^2), o in [-R, R], normalised to sum 1; radius limit 64 per
 * axis), plans the kernels, compiles them for the device at run time and
 * allocates the scratch cubes: one per distinct non-zero sigma_xy, in the
 * storage dtype.  Where nz * element size is not a multiple of 16 bytes the
 * scratch rows are padded to 16 bytes and one more scratch cube holds a
 * padded copy of the input, written by the detect path's x pass, so that the
 * window kernels read every input with TMA (results are identical; the
 * environment variable SF_NO_PAD=1 at creation keeps the unpadded layout).
 * *out is NULL on failure. */
sf_status sf_create(const sf_config *cfg, sf_ctx **out);

/* Free the context after synchronising the device work it owns. NULL-safe. */
sf_status sf_destroy(sf_ctx *ctx);

const char *sf_status_str(sf_status s);
/* Message of the last failure on ctx (or of the last failed sf_create when
 * ctx is NULL); never NULL. */
const char *sf_last_error(const sf_ctx *ctx);

/* Host query of the float32 taps the device uses for filter `filter` along
 * axis 0 (x and y) or 2 (z): writes 2R+1 values (offset o at index o+R) into
 * out (capacity cap) and R into *radius.  Sec. 2.1 / Sec. 3.4. */
sf_status sf_taps(const sf_ctx *ctx, int32_t filter, int32_t axis, float *out, int32_t cap,
                  int32_t *radius);

/* Window grid size and mask size in uint32 words. */
sf_status sf_window_grid(const sf_ctx *ctx, int32_t *nwx, int32_t *nwy, int32_t *nwz);
sf_status sf_mask_words(const sf_ctx *ctx, int64_t *words);

/* Filtered cube of one filter (Eq. 2 with the 3D filter the product of the
 * three 1D tap vectors, image zero outside the cube, no renormalisation at
 * the edges).  d_cube: storage dtype, nx*ny*nz elements.  d_filtered: float32,
 * nx*ny*nz elements. */
sf_status sf_filter(sf_ctx *ctx, const void *d_cube, int32_t filter, float *d_filtered,
                    void *stream);

/* Window mean and population standard deviation of a float32 filtered cube
 * (Sec. 3.3).  d_mean, d_std: float32 [nwx][nwy][nwz]. */
sf_status sf_stats(sf_ctx *ctx, const float *d_filtered, float *d_mean, float *d_std,
                   void *stream);

/* Threshold of a float32 filtered cube against its window statistics
 * (Sec. 3.3 voxel selection): bit set where value > mean + k*std (strict).
 * accumulate = 0 overwrites d_mask, 1 ORs into it. */
sf_status sf_threshold(sf_ctx *ctx, const float *d_filtered, const float *d_mean,
                       const float *d_std, uint32_t *d_mask, int32_t accumulate, void *stream);

/* The whole hot path for every filter of the bank: filter, window statistics,
 * threshold, OR of the per-filter marks into d_mask (overwritten).  d_mean and
 * d_std, when not NULL, receive the statistics of every filter
 * ([n_filters][nwx][nwy][nwz]). */
sf_status sf_detect(sf_ctx *ctx, const void *d_cube, uint32_t *d_mask, float *d_mean,
                    float *d_std, void *stream);

/* sf_detect from host memory: copies h_cube (storage dtype) to a device
 * buffer the context owns, runs the hot path and copies the mask back into
 * h_mask; returns after the mask is on the host.  Pinned host buffers make
 * the copies asynchronous DMA; pageable ones work too. */
sf_status sf_detect_host(sf_ctx *ctx, const void *h_cube, uint32_t *h_mask, void *stream);

/* One x slab of a larger cube, for cubes split across devices along x
 * (Sec. 3.1: the paper's nodes and sections take x slabs whose x pass needs
 * the neighbours' planes).  The context is planned for the extended slab:
 * cfg.nx = halo + S + halo, where S is the slab's own planes and the `halo`
 * planes on each side are the neighbours' (zeros beyond the cube's edge).
 *   d_ext   the extended slab [nx][ny][nz] in the storage type (device);
 *   halo    >= the largest x radius of the bank, and nx - 2 halo >= 1;
 *   d_mask  mask words of the S slab planes, [S][ny][ceil(nz/32)];
 *   d_mean, d_std  NULL, or [n_filters][ceil(S/wx)][nwy][nwz] float32.
 * Statistics windows tile the slab from its first plane, so a slab that
 * starts at a multiple of wx of the cube has exactly the cube's windows and
 * its mask rows equal sf_detect's on the whole cube bit for bit.  Needs the
 * fused window kernel (wy % 8 == 0, wz % 32 == 0), else SF_EINVAL; not for
 * batched contexts. */
sf_status sf_detect_slab(sf_ctx *ctx, const void *d_ext, int64_t halo, uint32_t *d_mask, float *d_mean,
                         float *d_std, void *stream);

/* Sectioned form for cubes larger than device memory (Sec. 3.1: the cube is
 * split into sections that each fit the device, with a halo).  The cube stays
 * in host memory.  sf_detect_host on this context cuts it along x into
 * sections of `section` planes, a positive multiple of cfg->wx (SF_EINVAL
 * otherwise).  Each section goes to the device together with h halo planes
 * on each side, where h is the largest x radius of the bank rounded up to a
 * multiple of wx.  Halo planes outside the cube are zero.  The section's x
 * pass and statistics windows then equal the whole cube's: every window lies
 * in one section, since sections start on window boundaries.  The mask
 * equals sf_detect's bit for bit.
 *
 * Device memory holds two section buffers and the scratch of one context of
 * (section + 2h) planes, plus, when nx is not a multiple of wx, a second
 * context for the last section.  It does not depend on nx.  Copies in, the
 * section's detect and the copy back overlap on three streams.  Every other
 * entry point except sf_synchronize and sf_destroy returns SF_EINVAL on this
 * context. */
sf_status sf_create_sectioned(const sf_config *cfg, int64_t section, sf_ctx **out);

/* Batched form.  One context for n cubes of different shapes that share the
 * filter bank, window, threshold and storage of cfg (cfg->nx, ny, nz are
 * ignored; dims holds n triples nx, ny, nz).  The context plans one
 * persistent kernel for all cubes: a device work queue of x-pass items (lane
 * chunks of one cube) and window items (one statistics window), ordered so
 * that a cube's x items precede its windows; a window item waits, bounded in
 * time, for its cube's x pass.  The launch is captured once in a CUDA graph
 * (counter reset, the per-call cube tables copied from pinned staging, the
 * kernel) and replayed by sf_detect_batch.  Sec. 4.1 tunes block sizes by a
 * sweep and Sec. 6 proposes automatic configuration: see sf_tune. */
sf_status sf_create_batch(const sf_config *cfg, int32_t n, const int64_t *dims, sf_ctx **out);

/* sf_detect over every cube of a batched context.  d_cubes, d_masks: host
 * arrays of n device pointers (cube i in the storage dtype, mask i of
 * nx*ny*ceil(nz/32) words).  d_means/d_stds: NULL, or host arrays of n device
 * pointers (each [n_filters][nwin_i] float32).  A call waits on the host for
 * the previous call's tables to be consumed before it rewrites them. */
sf_status sf_detect_batch(sf_ctx *ctx, const void *const *d_cubes, uint32_t *const *d_masks,
                          float *const *d_means, float *const *d_stds, void *stream);

/* Autotuner (Sec. 6: automatic configuration of the thread topology).  Runs
 * sf_detect / sf_detect_batch on the given inputs for each candidate launch
 * shape (for a plain context: the two-kernel path and the persistent kernel
 * with several x-slab sizes and x-item sizes; for a batched context: the
 * persistent shapes), keeps the fastest and returns after synchronising.
 * For a plain context pass one cube and one mask.  sf_tune_report writes the
 * timings as JSON text into buf. */
sf_status sf_tune(sf_ctx *ctx, const void *const *d_cubes, uint32_t *const *d_masks, void *stream);
sf_status sf_tune_report(const sf_ctx *ctx, char *buf, int32_t cap);

/* Serving form: a continuous-batching request loop on one GPU.
 * Requests are cubes of any shape in host memory (storage dtype of proto;
 * pinned memory makes the copies DMA).  A request is admitted as soon as one
 * of max_inflight worker slots is free and its device footprint (cube, mask
 * and one x-filtered scratch cube per distinct non-zero sigma_xy) fits the
 * HBM budget; admitted requests run concurrently on their own CUDA streams.
 * Per-shape contexts stay resident after use and count against the budget;
 * idle ones are destroyed (least recently used first) when an admission
 * needs the room.  A request larger than the budget completes at once with
 * SF_EBUDGET.  proto->nx/ny/nz are ignored.  (Sec. 3.1 copies sections one
 * at a time; Sec. 6 proposes overlapping input with processing.) */
typedef struct sf_server sf_server;
sf_status sf_server_create(const sf_config *proto, int64_t budget_bytes, int32_t max_inflight,
                           sf_server **out);
/* Queue a request; h_cube and h_mask must stay valid until it completes.
 * *id receives the request id. */
sf_status sf_server_submit(sf_server *srv, const void *h_cube, int64_t nx, int64_t ny, int64_t nz,
                           uint32_t *h_mask, int64_t *id);
/* Cancel request `id` if it is still waiting for admission: it completes at
 * once with status SF_ECANCELED (reported by sf_server_poll) and its buffers
 * are not touched again.  SF_ESTATE if it was already admitted (it then runs
 * to its end), completed, or is unknown. */
sf_status sf_server_cancel(sf_server *srv, int64_t id);
/* Up to cap completed requests: id, status and latency (ns from submit to
 * the mask being on the host).  Waits at most timeout_ms for a first one. */
sf_status sf_server_poll(sf_server *srv, int64_t *ids, int32_t *statuses, int64_t *latency_ns,
                         int32_t cap, int32_t timeout_ms, int32_t *n);
/* Counters: submitted, admitted, completed, rejected, bytes in use, peak
 * bytes (in use + idle contexts), idle bytes, evictions, contexts created,
 * busy slots, queued requests, budget, cancelled (up to cap values). */
sf_status sf_server_stats(sf_server *srv, int64_t *out, int32_t cap);
/* Drain the queue, wait for the requests in flight, free everything. */
sf_status sf_server_destroy(sf_server *srv);

/* Filtered cube of one filter without allocating anything, for callers that
 * cannot call cudaMalloc (allocation-free loops, hosts that own every
 * allocation).  No context: the filter is (sigma_xy, sigma_z, truncation),
 * radius at most 32 per axis, and the two intermediate cubes live in a fixed
 * 64 MiB scratch array inside the library (held on every GPU that loads it),
 * so nx*ny*nz is limited to 8,388,608 voxels; larger cubes return SF_EINVAL
 * with the reason in sf_last_error(NULL).
 * d_cube and d_filtered are float32 device buffers of nx*ny*nz elements.
 * All calls share the scratch array: calls that overlap on the GPU race.
 * The first call on a device sets up the scratch address with
 * cudaGetSymbolAddress; make it before any stream capture.  The address is
 * kept for the life of the process: after cudaDeviceReset on that device it
 * is stale, so do not call this entry point after a device reset.  The paper
 * has no counterpart of this entry point. */
sf_status sf_filter_noalloc(const float *d_cube, int64_t nx, int64_t ny, int64_t nz,
                            float sigma_xy, float sigma_z, float truncation, float *d_filtered,
                            void *stream);

/* Per-voxel local statistics (Sec. 3.3: each voxel's mean and standard
 * deviation come from a user-specified range of the filtered data around it),
 * read as the box [x-sx, x+sx] x [y-sy, y+sy] x [z-sz, z+sz] clipped to the
 * cube, with n the number of voxels of the clipped box; population
 * statistics, float32 results.
 *   d_filtered  float32 [nx][ny][nz] of the context's shape (device);
 *   d_mean, d_std  float32 [nx][ny][nz] (device), written for every voxel.
 * sx, sy, sz >= 0; sy <= 64 and sz <= 128 (the y-z tile of the box sums
 * lives in shared memory); nx <= 65535.  The context keeps two float32
 * scratch cubes for the partial sums, allocated on first use (SF_ENOMEM if
 * that fails).  Not for batched contexts.
 * Accuracy against the exact statistics of the float32 input: boxes with a
 * half-width below 3 on some axis (and not all 0) are evaluated in two passes
 * over each voxel's box (O(box) work per voxel), within 1e-5 max(std, |mean|)
 * for mean and std; wider boxes take separable running sums about one shift
 * per tile, within 1e-5 max(std, |mean|) where the box mean is near the
 * shift and within 2e-5 next to bright sources at the cube's edges (the sums
 * of squares then carry the distance from the shift).  A box of half-widths
 * (0, 0, 0) is exact (mean = c, std = 0). */
sf_status sf_local_stats(sf_ctx *ctx, const float *d_filtered, int32_t sx, int32_t sy, int32_t sz,
                         float *d_mean, float *d_std, void *stream);

/* Per-voxel z-score over the same box: z = (c - mean) / std for every voxel
 * of d_filtered, z = 0 where std = 0 (a box of equal values), float32
 * [nx][ny][nz] into d_z (device).  The selection of sf_local_detect is
 * z > k.  Same limits and scratch as sf_local_stats. */
sf_status sf_local_zscore(sf_ctx *ctx, const float *d_filtered, int32_t sx, int32_t sy, int32_t sz,
                          float *d_z, void *stream);

/* The detect with per-voxel local statistics instead of windows: every
 * filter of the bank (Eq. 2), the local mean / std of each filtered cube over
 * the box above, c_f > mean_f + k std_f, OR over the bank, packed into d_mask
 * like sf_detect's (every word written).  Same limits as sf_local_stats; the
 * context keeps one more float32 scratch cube for the filtered values. */
sf_status sf_local_detect(sf_ctx *ctx, const void *d_cube, int32_t sx, int32_t sy, int32_t sz,
                          uint32_t *d_mask, void *stream);

/* Weighted convolution (Eq. 1): c_w = sum_o d[i] f[o] w[i] / D over the
 * filter's offsets, d and w zero outside the cube, with
 *   den = 0  D = sum_o f[o] w[i]  (normalised convolution: unit weights give
 *            Eq. 2 wherever the support lies inside the cube),
 *   den = 1  D = sum_o w[i]       (the denominator as the paper prints it);
 * c_w = 0 where D = 0.  d_cube and d_weights: float32 [nx][ny][nz] (device,
 * 16-byte aligned); float32 storage contexts only, not batched.  The context
 * keeps three float32 scratch cubes (product, numerator, denominator), and
 * for den = 1 a second plan with the bank's radii and unit taps, both created
 * on first use (SF_ENOMEM if that fails). */
sf_status sf_weighted_filter(sf_ctx *ctx, const float *d_cube, const float *d_weights, int32_t filter,
                             int32_t den, float *d_out, void *stream);

/* The detect with Eq. 1 filtering: every filter of the bank weighted by w,
 * window statistics, c > mean + k*std, OR over the bank into d_mask (every
 * word written).  d_mean / d_std: NULL, or float32 [n_filters][nwx*nwy*nwz]
 * like sf_detect's. */
sf_status sf_weighted_detect(sf_ctx *ctx, const float *d_cube, const float *d_weights, int32_t den,
                             uint32_t *d_mask, float *d_mean, float *d_std, void *stream);

/* Wait for the work enqueued on `stream`, then report kernel-side failures:
 * SF_ETIMEOUT when a kernel's bounded wait expired since the last call (the
 * flag is cleared): a wait on its own shared-memory loads, or, in the
 * persistent kernel, a window's wait for its cube's x pass done by other
 * CTAs.  The kernel that gave up has left; the context stays usable. */
sf_status sf_synchronize(sf_ctx *ctx, void *stream);

/* Limit, in nanoseconds of %globaltimer, of every bounded wait of the
 * context's kernels (the paper's GPU kernels were split to stay under the
 * display watchdog, Sec. 3.4; here each wait is bounded instead).  Default
 * 2 s; accepted range [1 us, 60 s], else SF_EINVAL.  Applies to later
 * launches; a batched context captures its graph again (allocates nothing
 * new).  Not to be called while work of the context is being captured. */
sf_status sf_set_wait_limit(sf_ctx *ctx, int64_t limit_ns);

/* Test hook for the bounded-wait path (no counterpart in the paper).  For a
 * batched context whose bank has an x pass: switches its plan to the
 * persistent kernel with the x pass as items of its queue (whole cubes,
 * 1024 lanes per item) and makes every window item wait for `extra` more x
 * items than its cube has, so with extra > 0 no such wait can complete: each
 * runs into the wait limit, its CTA records the expiry and leaves, and
 * sf_synchronize returns SF_ETIMEOUT.  extra = 0 keeps that plan with the
 * true count.  SF_EINVAL for other contexts or extra outside [0, 1e6]. */
sf_status sf_test_stall_batch(sf_ctx *ctx, int32_t extra);

/* Stage timing (tracing).  While enabled, every sf_detect records CUDA
 * events on its stream around each of its stages: stage 0 = the x pass
 * launches, stage 1 = the fused window kernel (or the composed per-filter
 * path).  sf_profile_read waits for the recorded events, returns per stage
 * the summed milliseconds and the number of kernel launches since the last
 * read, and clears the record.  ms and launches have n_stages entries. */
sf_status sf_profile_enable(sf_ctx *ctx, int32_t enable);
sf_status sf_profile_read(sf_ctx *ctx, double *ms, int64_t *launches, int32_t n_stages);

/* Measured FP32 arithmetic peak of `device` (TFLOP/s, 2 flops per lane-FMA):
 * the denominator of the ALU roofline of the fused window kernel, which runs
 * its filter taps, pair sums and moments on the FP32 FMA pipe.  A probe kernel
 * with eight independent fma chains per thread on 2048 threads per SM is
 * timed with CUDA events (best of three after a warm-up), once with scalar
 * fma.rn.f32 (*tflops_scalar) and once with packed fma.rn.f32x2
 * (*tflops_pair).  Synchronous; allocates and frees one small device buffer.
 * The paper has no counterpart: this measures the machine, not the method.
 * Errors: SF_EINVAL for null outputs, SF_ECUDA for a CUDA failure (message
 * from sf_fp32_peak_error()). */
sf_status sf_fp32_peak(int32_t device, double *tflops_scalar, double *tflops_pair);
const char *sf_fp32_peak_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SF_H */
