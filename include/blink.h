/*
 * blink.h -- C ABI of the GB300 (sm_103a) BLINK dirty-image library.
 *
 * The library turns batches of complex visibilities into dirty images, one
 * image per (time step, frequency channel) "layer" (Sokolowski et al.,
 * arXiv 2405.13478, Sec. 5.2.4).  For every layer it
 *   (1) computes each baseline's (u,v) in wavelengths from the antenna
 *       positions and the layer frequency, in FP64 (Sec. 5.2.1 step 1; the
 *       Fig. 7 listing; w is dropped for a coplanar zenith-phased array,
 *       Sec. 4.3 Eqs. 4-5);
 *   (2) assigns the grid cell k = round-half-away(u / delta_u), zero spatial
 *       frequency in the centre bin, keeping |k_u|,|k_v| <= N/2-1 (Sec. 4.4.1
 *       Eq. 9; Sec. 5.2.1 step 1);
 *   (3) grids V at k and conj(V) at -k (Sec. 5.2.1 steps 2-3);
 *   (4) applies natural or uniform (1/count) weighting (Sec. 4.4.2);
 *   (5) runs the inverse 2-D FFT with FFT shifts and real part (Sec. 4.3 Eq. 6,
 *       Sec. 5.2.2), unnormalised: a unit source at the phase centre gives a
 *       centre pixel equal to the summed weight.
 *
 * Conventions for every entry point:
 *   - Pointers prefixed d_ are device pointers on the context's device; h_
 *     pointers are host memory.  The caller owns all of them; the library
 *     never frees caller memory.
 *   - Complex numbers are interleaved float pairs (re, im) = complex64.
 *   - Baselines are the cross-correlation pairs (i < j) in lexicographic
 *     order, B = n_ant (n_ant - 1) / 2; baseline b of pair (i, j) has
 *     u = (x_j - x_i) / lambda.
 *   - Antenna positions are float64 [n_ant][3] metres (x east, y north, z up;
 *     z is ignored).
 *   - Images are float32 [N][N] row-major: row y <-> m (v axis), column x <->
 *     l (u axis), phase centre at pixel (N/2, N/2).  Grids are complex64
 *     [N][N] with the same orientation (row = k_v + N/2, column = k_u + N/2).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All work is enqueued asynchronously on it unless stated.
 *   - Every call returns a blink_status.  Invalid arguments are rejected on the
 *     host before anything is launched; blink_last_error() then describes the
 *     problem.  No C++ exception crosses this boundary.
 *   - A context is not thread safe: use one per host thread (or lock).
 */
#ifndef BLINK_H
#define BLINK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BLINK_ABI_VERSION 2

#if defined(__GNUC__)
#define BLINK_API __attribute__((visibility("default")))
#else
#define BLINK_API
#endif

typedef enum {
    BLINK_OK = 0,
    BLINK_ERR_INVALID = -1,     /* bad argument (caught on the host) */
    BLINK_ERR_UNSUPPORTED = -2, /* valid but not implemented (e.g. image size) */
    BLINK_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    BLINK_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
    BLINK_ERR_WORKSPACE = -5    /* device memory for the workspace ran out */
} blink_status;

typedef enum { BLINK_NATURAL = 0, BLINK_UNIFORM = 1 } blink_weighting;

/* Flags of blink_image_batch / blink_plan_image. */
#define BLINK_NORMALIZE 0x1u /* divide each image by its summed weight */
/* Transform of the second pass (along v).  Default: FP32 FFT.  The others
 * run it as a dense real GEMM on the tensor cores (image sizes that are a
 * multiple of 256; other sizes keep the FFT), FP32 accumulation:
 *   BF16 / FP16        one product of rounded operands,
 *   BF16X3 / FP16X3    split-precision recovery (hi*hi + hi*lo + lo*hi).
 * Error against the FP64 result is stated per mode in the tests. */
#define BLINK_TRANSFORM_MASK 0xF0u
#define BLINK_TRANSFORM_FFT 0x00u
#define BLINK_TRANSFORM_BF16 0x10u
#define BLINK_TRANSFORM_BF16X3 0x20u
#define BLINK_TRANSFORM_FP16 0x30u
#define BLINK_TRANSFORM_FP16X3 0x40u

/* One image ("layer", Sec. 5.2.4). */
typedef struct {
    int32_t n_px;       /* image side N: even, one of blink_supported_sizes() */
    int32_t weighting;  /* blink_weighting */
    double freq_hz;     /* channel frequency nu (> 0) */
    double delta_u;     /* cell size in wavelengths, 1 / (N dx) (Sec. 4.4.1 Eq. 9) (> 0) */
    int64_t vis_offset; /* complex64 element offset of this layer's B visibilities */
    int64_t out_offset; /* element offset of this layer's N*N output
                           (float32 for images, complex64 for grids) */
} blink_layer;

typedef struct blink_ctx blink_ctx;
typedef struct blink_plan blink_plan;

/* ---------------------------------------------------------------- context */
/* Version of this ABI (BLINK_ABI_VERSION). */
BLINK_API int blink_abi_version(void);

/* Writes up to `cap` supported image sizes N into `sizes`; returns how many
 * sizes exist (call with cap = 0 to count). */
BLINK_API int blink_supported_sizes(int32_t *sizes, int cap);

/* Creates a context on CUDA device `device` (makes it current for the call).
 * The context owns a device workspace that grows on demand and is freed by
 * blink_ctx_destroy, and an auxiliary stream: the adjoint runs half of each
 * wave of layers on it, forked from and joined back to the caller's stream
 * with events, so every call stays ordered on the caller's stream (and can
 * be captured in a CUDA graph).  *out is NULL on failure. */
BLINK_API int blink_ctx_create(blink_ctx **out, int device);
BLINK_API void blink_ctx_destroy(blink_ctx *ctx);

/* Text of the last error recorded on `ctx` ("" if none).  The string belongs
 * to the context and stays valid until its next call. */
BLINK_API const char *blink_last_error(const blink_ctx *ctx);

/* ------------------------------------------------- cell indices only */
/* Cell indices of every baseline of every layer, bit-exact FP64 rounding
 * (steps 1-2).  d_cells: int32 [n_layers][B][2] = (k_u, k_v) per baseline, or
 * (INT32_MIN, INT32_MIN) when the baseline falls outside |k| <= N/2-1 and is
 * not gridded.  vis_offset/out_offset of h_layers are ignored. */
BLINK_API int blink_cells(blink_ctx *ctx, const double *d_ant_xyz, int n_ant, const blink_layer *h_layers,
                int n_layers, int32_t *d_cells, void *stream);

/* ------------------------------------------------------------- grids */
/* Gridded, weighted visibilities of every layer (steps 1-4), Hermitian-complete:
 * d_grid + out_offset holds complex64 [N][N] with zero spatial frequency at
 * (N/2, N/2) (Sec. 5.2.1 step 1).  d_wsum (float32 [n_layers], may be NULL)
 * receives each layer's summed weight.  d_vis holds the complex64 visibilities
 * addressed by vis_offset.  Gridding runs in shared memory without global
 * atomics. */
BLINK_API int blink_grid(blink_ctx *ctx, const double *d_ant_xyz, int n_ant, const blink_layer *h_layers,
               int n_layers, const float *d_vis, float *d_grid, float *d_wsum, void *stream);

/* ------------------------------------------------------- dirty images */
/* Dirty images of every layer (steps 1-5): d_images + out_offset receives the
 * float32 [N][N] FFT-shifted real image, unnormalised unless flags has
 * BLINK_NORMALIZE.  d_wsum (float32 [n_layers], may be NULL) receives the
 * summed weights.  Layers of different sizes may be mixed.  Images are the
 * same bits on every call: every cell sums its visibilities in an order fixed
 * by the array geometry, without atomics (the fused small-image kernel by its
 * per-channel register schedule, the large-image row pass by its sorted row
 * buckets, or -- when a group's support fits 40 KB as a compact grid of rows
 * r < R and columns |k_u| <= kmax -- by one CTA per layer summing per-chunk
 * cell-sorted entries in shared memory).  Large images run as one persistent
 * launch per image size whose CTAs take row and column work items from a
 * device queue; groups with compact grids run the same row and column passes
 * as waves of two kernels after the compact gridding.
 * This call builds the per-channel tables on `stream` and synchronises that
 * stream once to size the image kernels; use a plan (below) to build the
 * tables once and image many batches asynchronously. */
BLINK_API int blink_image_batch(blink_ctx *ctx, const double *d_ant_xyz, int n_ant,
                      const blink_layer *h_layers, int n_layers, const float *d_vis,
                      float *d_images, float *d_wsum, uint32_t flags, void *stream);

/* --------------------------------------------------------------- adjoint */
/* The paper images only; these calls differentiate its image path.  The
 * dirty image is linear in the visibilities (Sec. 4.3 Eq. 6 with the gridding
 * of Sec. 5.2.1): I[p] = sum_b w_b 2 Re(V_b exp(+2 pi i k_b.(p - N/2) / N)).
 * Given d_dimage = dL/dI of a real loss L (float32 [N][N] at out_offset, same
 * layout and flags as the forward images), blink_degrid writes
 *     d_dvis[b] = dL/dRe V_b + i dL/dIm V_b = 2 w_b H[k_b]
 * (complex64 at vis_offset), H the forward 2-D DFT of dL/dI
 * (exp(-2 pi i k.(p - N/2) / N)); zero for baselines that are not gridded.
 * It recomputes from the layer description (no state of the forward pass is
 * kept).  With BLINK_NORMALIZE the forward scaling by 1/sum(w) is included. */
BLINK_API int blink_degrid(blink_ctx *ctx, const double *d_ant_xyz, int n_ant, const blink_layer *h_layers,
                           int n_layers, const float *d_dimage, float *d_dvis, uint32_t flags, void *stream);
BLINK_API int blink_plan_degrid(blink_plan *plan, const float *d_dimage, float *d_dvis, uint32_t flags,
                                void *stream);
/* blink_plan_degrid with the gradient of layer l (index into the plan's
 * layer array) multiplied by d_layer_scale[l] (float32 [n_layers], device
 * memory; NULL = 1).  For a loss f(s) of the per-layer sums of squares s_l of
 * blink_epilogue.d_sqnorm, dL/dI_l = 2 (df/ds_l) r_l with r_l the stored
 * output: pass the stored images as d_dimage and 2 df/ds_l as the scale, and
 * no image-sized gradient is formed. */
BLINK_API int blink_plan_degrid_scaled(blink_plan *plan, const float *d_dimage, const float *d_layer_scale,
                                       float *d_dvis, uint32_t flags, void *stream);
/* Bytes of the d_adjoint buffer of blink_epilogue for this plan. */
BLINK_API int blink_plan_adjoint_bytes(const blink_plan *plan, int64_t *bytes);
/* blink_plan_degrid_scaled(plan, images, d_layer_scale, ...) for the images
 * a blink_plan_image_ex call stored while it filled d_adjoint: the second
 * half of the adjoint (DFT along u of the kept rows, gather at each
 * baseline's cell) only.  Same results as that call, bit for bit. */
BLINK_API int blink_plan_degrid_adjoint(blink_plan *plan, const float *d_adjoint, const float *d_layer_scale,
                                        float *d_dvis, uint32_t flags, void *stream);

/* Per-antenna complex gains g (complex64 [n_ant]) on model visibilities
 * (antenna-level calibration, Sec. 4.2): d_vis[b] = g_i conj(g_j) d_model[b]
 * for baseline b = (i < j) of every layer (vis_offset addressing; other layer
 * fields ignored). */
BLINK_API int blink_apply_gains(blink_ctx *ctx, int n_ant, const blink_layer *h_layers, int n_layers,
                                const float *d_model, const float *d_gains, float *d_vis, void *stream);
/* Chain rule of blink_degrid's output to the gains, summed over all layers:
 * d_dgains[i] = sum_l [ sum_{j>i} d_dvis(ij) g_j conj(M_ij)
 *                     + sum_{k<i} conj(d_dvis(ki)) g_k M_ki ]
 * (dL/dRe g + i dL/dIm g), overwrites d_dgains.  Products in FP32; each
 * thread's sums compensated FP32 (Kahan), their reduction FP64, all in a
 * fixed order (the same bits from run to run); every baseline is read once,
 * row by row of the upper triangle.  At most 1024 antennas
 * (BLINK_ERR_UNSUPPORTED above). */
BLINK_API int blink_gain_grad(blink_ctx *ctx, int n_ant, const blink_layer *h_layers, int n_layers,
                              const float *d_dvis, const float *d_model, const float *d_gains, float *d_dgains,
                              void *stream);

/* -------------------------------------------------- host-resident buffers */
/* blink_image_batch for data in host memory: h_ant_xyz, h_vis and h_images
 * (and h_wsum, may be NULL) are host pointers addressed like their d_
 * counterparts.  The call builds the plan once, then streams the layers in
 * chunks through double-buffered device staging: the host-to-device copy of
 * chunk i+1 and the device-to-host copy of chunk i-1 overlap the kernels of
 * chunk i (the copy/compute overlap and pinned host memory suggested in the
 * paper's summary, Sec. 7).  Pinned host memory (cudaHostAlloc /
 * cudaHostRegister) gives full copy bandwidth; pageable memory works but
 * serialises the copies.  Returns after the images are in h_images. */
BLINK_API int blink_image_batch_host(blink_ctx *ctx, const double *h_ant_xyz, int n_ant,
                                     const blink_layer *h_layers, int n_layers, const float *h_vis,
                                     float *h_images, float *h_wsum, uint32_t flags, void *stream);

/* ------------------------------------------------------------------ plans */
/* A plan fixes the array and the layer descriptors, runs steps 1-2 and the
 * weighting tables once (on `stream`, which it synchronises once), and keeps
 * them on the device.  blink_plan_image then only launches the gridding and
 * FFT kernels: it is asynchronous and may be captured in a CUDA graph.  The
 * plan reads d_ant_xyz only during blink_plan_create. */
BLINK_API int blink_plan_create(blink_ctx *ctx, const double *d_ant_xyz, int n_ant,
                      const blink_layer *h_layers, int n_layers, blink_plan **out, void *stream);
BLINK_API int blink_plan_image(blink_plan *plan, const float *d_vis, float *d_images, float *d_wsum,
                     uint32_t flags, void *stream);

/* Fused epilogue of blink_plan_image_ex / blink_plan_capture (every field may
 * be NULL / 0; a NULL blink_epilogue pointer means none):
 *   d_gains      complex64 (re, im) antenna gains, device memory.  Layer l
 *                (index into the plan's layer array) uses the n_ant gains at
 *                d_gains + 2 * r * gain_stride floats, r = l mod gain_period
 *                (r = l when gain_period is 0); each visibility of the
 *                pair (i < j) is multiplied by g_i conj(g_j) as it is loaded
 *                for gridding (calibration applied after correlation,
 *                Sec. 4.2 step ii; pass reciprocal gains to remove a
 *                solution).  Needs n_ant < 65536.
 *   gain_stride  complex elements between consecutive gain rows; 0 = one
 *                row for every layer.  Must be >= 0.
 *   gain_period  0, or the number of gain rows that repeat over the layers:
 *                with time-major layers, gain_period = channels gives
 *                per-channel gains constant over time.  Must be >= 0.
 *   d_ref        float32 reference images, device memory, addressed like
 *                d_images (layer l at out_offset).  The output becomes the
 *                dirty image minus the reference, subtracted as the image is
 *                stored (Sec. 2 and Sec. 4.3 after Eq. 6: side-lobes of a
 *                transient search removed by subtracting a reference image of
 *                the same field).  With BLINK_NORMALIZE the dirty image is
 *                normalised first.  d_ref must not overlap the output
 *                extent (BLINK_ERR_INVALID).
 *   d_sqnorm     float64 [n_layers] in device memory, or NULL: layer l (index
 *                into the plan's layer array) gets the sum over its N x N
 *                output pixels of out^2, the output being what is stored
 *                (with d_ref, the squared norm of the residual image, a
 *                least-squares image loss).  Summed as the pixels are stored:
 *                each transform task's 2 N2 squares in FP32 (N = N1 N2 the
 *                four-step split), those sums in FP64, all in a fixed order
 *                (the same bits on every call).  Needs the FFT transform: with
 *                a tensor-core mode flag the call returns
 *                BLINK_ERR_UNSUPPORTED.  The first call allocates 8 bytes per
 *                layer and column item of the largest size (64 at 1024^2)
 *                from the context's pool.
 *   d_adjoint    device buffer of blink_plan_adjoint_bytes bytes (8-byte
 *                aligned), or NULL: receives the first half of blink_degrid
 *                applied to the stored output -- the forward DFT along v of
 *                every image column, rows k < R of the support -- so that
 *                blink_plan_degrid_adjoint can later finish the adjoint
 *                without reading the images again.  Where the column pass
 *                holds exactly one 16-column strip of the image per CTA
 *                (1024^2 on the FFT path) the strip is transformed in shared
 *                memory as it is stored; other sizes and the tensor-core
 *                modes transform the stored images after their launch.
 *                Layout: per size group in plan order, per layer of the
 *                group, r_alloc rows of N complex64 (FFT-order columns).
 *                With d_adjoint set, d_images may be NULL: no image is
 *                stored (sizes whose columns come from stored images image
 *                into an array of the plan's output extent that the plan
 *                allocates from the context's pool on first need and keeps
 *                until it is destroyed). */
typedef struct {
    const float *d_gains;
    int64_t gain_stride;
    int64_t gain_period;
    const float *d_ref;
    double *d_sqnorm;
    float *d_adjoint;
} blink_epilogue;

BLINK_API int blink_plan_image_ex(blink_plan *plan, const float *d_vis, float *d_images, float *d_wsum,
                                  uint32_t flags, const blink_epilogue *epi, void *stream);
BLINK_API void blink_plan_destroy(blink_plan *plan);

/* Autotuner: for every image size of the plan, times the candidate kernel
 * configurations on the given data (the atomic-free scheduled fused kernel,
 * the shared-atomic fused kernel, and the two-pass large-image path as one
 * persistent work-queue launch or as waves of two kernels, each with 12, 24
 * and 48 MB of row-transform scratch) and keeps the fastest for later calls.
 * Synchronises `stream`; writes images as a side effect.  blink_plan_tuning
 * reports the choice for size group `group` (groups are the plan's distinct
 * sizes in increasing order; path 1 scheduled fused, 2 atomic fused, 3
 * persistent queue, 4 waves). */
BLINK_API int blink_plan_autotune(blink_plan *plan, const float *d_vis, float *d_images, void *stream);
BLINK_API int blink_plan_tuning(const blink_plan *plan, int group, int *n_px, int *path, int64_t *wave_bytes);
/* Sets a size group's kernel choice by hand (e.g. a tuning kept from an
 * earlier run): path 0 default, 1 scheduled fused (sizes <= 256 whose
 * schedule fits), 2 atomic fused (sizes <= 256), 3 persistent work queue,
 * 4 waves of two kernels (3 and 4: any size); wave_bytes = row-transform
 * scratch in use (the ring of path 3, a wave of path 4), 0 = default.
 * BLINK_ERR_INVALID for a path the group cannot take; the plan is unchanged
 * then.  Path 2, and paths 3 and 4 on sizes whose full support always fits
 * the fused kernels (their channels get no row buckets), grid with
 * shared-memory atomics: equal within FP32 rounding, not the same bits from
 * call to call (the autotuner may keep such a choice). */
BLINK_API int blink_plan_set_tuning(blink_plan *plan, int group, int path, int64_t wave_bytes);

/* CUDA graph of the plan's image launches: blink_plan_capture runs
 * blink_plan_image_ex once on `stream` (allocating whatever it needs), then
 * records the same launches, bound to these pointers and flags, into a graph
 * owned by the plan (replacing any earlier one).  blink_plan_replay launches
 * the whole batch -- every image size -- as that one graph on `stream`. */
BLINK_API int blink_plan_capture(blink_plan *plan, const float *d_vis, float *d_images, float *d_wsum,
                                 uint32_t flags, const blink_epilogue *epi, void *stream);
BLINK_API int blink_plan_replay(blink_plan *plan, void *stream);

/* Limit, in nanoseconds, of the first barrier waits of the tensor-core
 * kernels of every later launch on `ctx` (< 0: the default, one second).
 * A wait that runs out records BLINK_ERR_TIMEOUT in the plan's status word
 * (read by blink_plan_check), lets its own copies and MMAs finish, frees its
 * tensor memory and returns without writing the image; the context stays
 * usable.  0 makes those waits give up after one poll, which is how the
 * timeout path is tested. */
BLINK_API int blink_ctx_set_wait_limit(blink_ctx *ctx, int64_t limit_ns);

/* Waits for `stream` and returns the plan's device status word: BLINK_OK, or
 * BLINK_ERR_TIMEOUT if a bounded device-side wait of an earlier launch gave
 * up (that launch's output is incomplete).  Clears the word. */
BLINK_API int blink_plan_check(blink_plan *plan, void *stream);

/* Summed weight and kept-baseline count of layer `layer` of a plan (host
 * copies; no device work). */
BLINK_API int blink_plan_layer_info(const blink_plan *plan, int layer, float *wsum, int64_t *n_kept);

/* ------------------------------------------------------------- measurement */
/* Not a step of the paper's method: measures the FMA rate of the CUDA cores
 * of `device` (bits = 32: FP32, 64: FP64) so roofline fractions of the
 * arithmetic-bound kernels (the transforms in FP32, the cell assignment in
 * FP64) are stated against a measured peak.  One full-occupancy launch of
 * eight independent FMA chains per thread; *tflops = 2 flops per FMA over its
 * CUDA-event time.  Synchronous (own stream); BLINK_ERR_INVALID for other
 * `bits`, BLINK_ERR_CUDA when the launch fails. */
BLINK_API int blink_probe_fma_peak(int device, int bits, double *tflops);

/* ------------------------------------------------- allocation-free variant */
/* The paper has no counterpart of this entry point; it serves callers that
 * must not allocate device memory while they run -- for example a real-time
 * telescope pipeline that reserves all GPU memory when an observation starts
 * and forbids allocation (and its unpredictable latency) afterwards, or a
 * host framework whose own allocator already owns the whole device.
 *
 * Same result as blink_image_batch (steps 1-5 on every layer), but it allocates
 * nothing: no cudaMalloc, no cudaFree, no memory pool, no context.  All of
 * its scratch -- channel tables, layer descriptors, the gridding schedule of
 * sizes up to 256, the row buckets of large sizes, the work queue and the
 * row-transform ring of large images -- lives in one static device array of
 * BLINK_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the library holds
 * until the process exits.  When all of that fits, the call runs the kernels
 * blink_image_batch runs and gives the same bits; a schedule or bucket set
 * that does not fit is left out for that call, and its images then come from
 * the shared-atomic gridding fallback (equal within FP32 rounding, not bit
 * for bit).  A 256-antenna station with 32 channels of 180^2 takes about
 * 31 MB of tables.
 *
 * Limits: all layers of a call share one n_px; at most
 * BLINK_NOALLOC_MAX_CHANNELS distinct (freq_hz, delta_u, weighting) channels;
 * the tables (4 bytes per baseline per channel, plus N*N/2 floats per
 * uniform-weighted or scheduled channel, plus 56 bytes per layer) and one
 * layer's row-transform buffer (large images only) must fit in the static
 * array.  A request beyond a limit returns BLINK_ERR_WORKSPACE (or
 * BLINK_ERR_INVALID for mixed sizes) before any launch, with a message in
 * err_msg.
 *
 * Runs on the calling thread's current device and on `stream`, which it
 * synchronises once (like blink_image_batch).  The first call on each device
 * looks up the device address of the static array (cudaGetSymbolAddress);
 * make that first call before any stream capture.  Every call reuses the same
 * array and clears what must start at zero; calls whose GPU work overlaps
 * (other streams or host threads at the same time) race on it, so serialise
 * them.  err_msg (may be NULL) receives a NUL-terminated description of a
 * failure, truncated to err_cap bytes. */
#define BLINK_NOALLOC_SCRATCH_BYTES (32u << 20)
#define BLINK_NOALLOC_MAX_CHANNELS 256
BLINK_API int blink_image_batch_noalloc(const double *d_ant_xyz, int n_ant,
                                        const blink_layer *h_layers, int n_layers,
                                        const float *d_vis, float *d_images, float *d_wsum,
                                        uint32_t flags, void *stream, char *err_msg,
                                        size_t err_cap);

#ifdef __cplusplus
}
#endif
#endif /* BLINK_H */
