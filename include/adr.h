/*
 * adr.h — C ABI of libadr.so, a GB300 (sm_103a) implementation of the
 * AdR-Gaussian rasterization path (Wang, Yi, Ma: "AdR-Gaussian: Accelerating
 * Gaussian Splatting with Adaptive Radius", SIGGRAPH Asia 2024, arXiv 2409.08669).
 *
 * The path is the paper's six-stage tile rasterizer (Sec. 3.2.1: Preprocess,
 * InclusiveSum, DuplicateWithKeys, SortPairs, IdentifyTileRanges, Render) with
 * the early culling of Gaussian-tile pairs whose splatting opacity cannot reach
 * alpha_low = 1/255: the adaptive radius (Sec. 4.2, Eq. 5-8) and the
 * axis-aligned bounding box (Sec. 4.3, Eq. 9-11).  Render also counts the
 * per-pixel load l_i (Sec. 4.4, Eq. 12) that the load-balancing loss uses.
 *
 * Conventions shared by every entry point:
 *   - Every array argument is caller-owned memory.  Unless an entry point says
 *     HOST, it is device memory on the context's device, C-contiguous float32
 *     (or the stated integer type), and it is only read/written during the
 *     stream-ordered work the call enqueues.  The library never frees it.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls enqueue asynchronously and return without waiting unless
 *     the entry point says it synchronises.
 *   - A context holds one frame's intermediates; calls that use the same
 *     context must be ordered on one stream (or externally synchronised).
 *   - Parameters are activated: positive scales, opacity in (0, 1), rotation
 *     quaternions (w, x, y, z) of any non-zero norm (normalised internally).
 *   - On failure an entry point returns a non-zero adr_status and
 *     adr_last_error() describes it (thread-local, valid until the next call
 *     on that thread).  Invalid arguments are rejected before any work is
 *     enqueued.
 */
#ifndef ADR_H
#define ADR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADR_TILE 16            /* tile edge in pixels (Sec. 3.2) */
#define ADR_CAMERA_FLOATS 24   /* view[16], fx, fy, cx, cy, near, cam_pos[3] */
#define ADR_GEOM_FLOATS 12     /* see adr_read_gaussians */

typedef enum adr_status {
    ADR_OK = 0,
    ADR_ERR_INVALID = 1,    /* bad argument (NULL, size out of range, bad mode) */
    ADR_ERR_CAPACITY = 2,   /* more pairs than pair_capacity; nothing written out of bounds */
    ADR_ERR_CUDA = 3,       /* a CUDA runtime call failed */
    ADR_ERR_TIMEOUT = 4,    /* a bounded device-side wait gave up: the frame's later stages
                               were skipped and its image holds only the background */
    ADR_PENDING = 5,        /* serving: request not finished yet */
    ADR_ERR_ADMISSION = 6   /* serving: request can never fit the memory budget */
} adr_status;

/* Pair-culling mode of Preprocess.
 *   ADR_PLAIN  : 3DGS tile range, square of radius r_o = ceil(3 sqrt(lambda'_max))
 *                (the "99% confidence" range the paper compares against, Sec. 4.2).
 *   ADR_CIRCLE : adaptive radius r = min(sqrt(2 lambda'_max ln(sigma/alpha_low)), r_o)
 *                (Eq. 7-8); no pairs when sigma < alpha_low.
 *   ADR_AABB   : r_x = min(sqrt(2 Sigma'_X ln(sigma/alpha_low)), r_o),
 *                r_y = min(sqrt(2 Sigma'_Y ln(sigma/alpha_low)), r_o) (Eq. 10-11).
 * All modes produce the same image (the culled pairs have alpha < alpha_low at
 * every pixel of the culled tile, Sec. 5.2 and 5.3). */
typedef enum adr_mode { ADR_PLAIN = 0, ADR_CIRCLE = 1, ADR_AABB = 2 } adr_mode;

/* Pinhole camera.  view: row-major world->camera matrix with OpenCV axes
 * (x right, y down, z forward).  A pixel (i, j) has its centre at integer
 * coordinates.  near_z (> 0, finite): Gaussians with view depth <= near_z
 * are culled.  fx, fy must be positive and finite; width, height within the
 * context's maximum (else ADR_ERR_INVALID). */
typedef struct adr_camera {
    float view[16];
    float fx, fy, cx, cy;
    float near_z;
    float cam_pos[3];
    int32_t width, height;
} adr_camera;

/* Tile-rectangle rule of Preprocess, for the half-widths (r_x, r_y) the
 * mode chose around the pixel centre (px, py).
 *   ADR_RECT_PIXEL : the tiles holding a pixel centre x in
 *                    [ceil(px - r_x), floor(px + r_x)] clipped to the image
 *                    (likewise y).  Lossless: no pixel within the half-widths
 *                    misses the Gaussian.  The default.
 *   ADR_RECT_3DGS  : the original 3DGS rasterizer's rounding, for comparison
 *                    with renders of that rasterizer: R = ceil(r_x), tiles
 *                    [floor((px - R)/16), floor((px + R + 15)/16)) clamped to
 *                    the tile grid (likewise y).  Not lossless: when
 *                    px + R lies in [16k, 16k+1) the tile k is dropped
 *                    although its pixel 16k is within the radius. */
typedef enum adr_rect_rule { ADR_RECT_PIXEL = 0, ADR_RECT_3DGS = 1 } adr_rect_rule;

/* How the per-pixel load l_i (Eq. 12, an integer count) passes a gradient to
 * the opacities alpha_k of the Gaussians blended into the pixel in
 * adr_render_backward; the paper does not say.
 *   ADR_LOAD_GRAD_STRAIGHT    : d l_i / d alpha_k = 1 (straight-through).  The
 *                               default.
 *   ADR_LOAD_GRAD_TERMINATION : the same for pixels that reached the end of
 *                               their list; for a pixel that stopped early
 *                               (transmittance below t_min),
 *                               d l_i / d alpha_k = -l_i / (-ln T_final) / (1 - alpha_k):
 *                               raising any alpha_k by d(-ln(1 - alpha_k))
 *                               brings the stop forward by that much optical
 *                               depth, -ln T_final / l_i per blended Gaussian
 *                               on average. */
typedef enum adr_load_grad { ADR_LOAD_GRAD_STRAIGHT = 0, ADR_LOAD_GRAD_TERMINATION = 1 } adr_load_grad;

/* Render settings.  alpha_low: minimum splatting opacity (paper: 1/255,
 * Sec. 5.1.2); t_min: blending stops before a Gaussian that would take the
 * transmittance below it; lowpass: added to the diagonal of Sigma';
 * jac_clamp: the projection Jacobian uses x/z, y/z clamped to
 * +-jac_clamp*tan(fov/2); bg: background colour; sh_degree: 0..3;
 * rect_rule: an adr_rect_rule; load_grad: an adr_load_grad. */
typedef struct adr_settings {
    int32_t mode;
    float alpha_low, t_min, lowpass, jac_clamp;
    float bg[3];
    int32_t sh_degree;
    int32_t rect_rule;
    int32_t load_grad;
} adr_settings;

typedef struct adr_ctx adr_ctx;

/* Create a context on `device` with workspace for up to `max_gaussians`
 * Gaussians (at most 2^29), `pair_capacity` Gaussian-tile pairs (at most
 * 2^30) and images up to max_width x max_height (at most 4096 per side).
 * All workspace is allocated here (cudaMalloc); no later call allocates,
 * except the first adr_render_host, which allocates its staging buffers.
 * Returns ADR_ERR_INVALID for sizes <= 0 or too large (checked before any
 * CUDA call), ADR_ERR_CUDA if allocation fails (nothing leaks). */
adr_status adr_create(adr_ctx **ctx, int64_t max_gaussians, int64_t pair_capacity,
                      int32_t max_width, int32_t max_height, int32_t device);

/* Synchronise the context's device and free its workspace.  NULL is a no-op. */
void adr_destroy(adr_ctx *ctx);

/* Stages 1-3 (Sec. 3.2.1): Preprocess each Gaussian (projection, EWA
 * covariance Sigma', conic, SH colour of degree sh_degree, early cull by
 * settings->mode), order the Gaussians by view depth, scan their tile counts
 * and emit one (tile, Gaussian) pair per overlapped tile.
 *   means [n,3], scales [n,3], rots [n,4] (w,x,y,z), opac [n], sh [n,16,3]
 *   (coefficient index l*l+l+m, channel last; only (sh_degree+1)^2 used).
 * 0 <= n <= max_gaussians; camera size within the context's maximum.
 * The pair count stays on the device (see adr_num_pairs).  If it exceeds
 * pair_capacity the excess pairs are dropped and a device flag is set; the
 * next adr_num_pairs / adr_sync_status returns ADR_ERR_CAPACITY. */
adr_status adr_preprocess(adr_ctx *ctx, const float *means, const float *scales,
                          const float *rots, const float *opac, const float *sh, int64_t n,
                          const adr_camera *camera, const adr_settings *settings, void *stream);

/* Depth slices of adr_sort / adr_render (see adr_sort): never, always, or
 * (the default) when the context's last sliced frame shows they pay.  The
 * images are the same in every mode; only the time differs. */
typedef enum adr_slice_mode {
    ADR_SLICES_NEVER = 0, ADR_SLICES_ALWAYS = 1, ADR_SLICES_ADAPTIVE = 2
} adr_slice_mode;
/* Sets the context's adr_slice_mode for the following frames.  ADR_ERR_INVALID
 * for an unknown mode. */
adr_status adr_set_depth_slices(adr_ctx *ctx, int32_t mode);

/* Heavy tiles across CTAs (the uneven load across tiles, Sec. 4.4): with
 * ADR_TILE_SPLIT_LAST_SLICE, the last depth slice renders every unfinished
 * tile as two CTAs of one pixel per thread (the tile's top and bottom 8
 * rows), so each tile runs on twice the warps; every pixel's arithmetic is
 * unchanged and the frames are bit-identical to ADR_TILE_SPLIT_OFF (the
 * default, faster on the measured workloads).  A tile's list is not split:
 * front-to-back blending stops at a transmittance that depends on the whole
 * prefix.  Applies to adr_render of this context from the next call;
 * ADR_ERR_INVALID for an unknown mode. */
typedef enum adr_tile_split {
    ADR_TILE_SPLIT_OFF = 0, ADR_TILE_SPLIT_LAST_SLICE = 1
} adr_tile_split;
adr_status adr_set_tile_split(adr_ctx *ctx, int32_t mode);

/* Stages 4-5: the tile lists, ordered by (tile, depth, index) (the Gaussians
 * are already in depth order).  The pairs are grouped by column of tiles:
 * each Gaussian contributes one run per tile column of its rectangle (its
 * rows in that column), stably sorted by column, with each column's
 * [start, end).  A tile's list is the runs of its column that cover its row,
 * in order; adr_render reads it from there, so the pairs are never written
 * out one by one.  The runs are built in two depth slices: adr_sort builds
 * those of the nearest Gaussians; adr_render renders them, then builds and
 * renders the runs of the farther Gaussians that touch a tile with a pixel
 * still blending (a pixel's blend stops once its transmittance falls below
 * t_min, so the others cannot change a pixel).  A context slices a frame when
 * the last sliced frame's two slices held fewer than half of all runs (read
 * back without waiting), and every 16th frame to measure again; otherwise it
 * builds every Gaussian's runs at once.  Either way the image is the same.
 * adr_render_backward, adr_read_pairs and adr_read_ranges first build every
 * Gaussian's runs and expand them into per-tile lists and ranges (a second,
 * stable pass by tile row), enqueued on their own stream. */
adr_status adr_sort(adr_ctx *ctx, void *stream);

/* Stage 6: per-tile front-to-back alpha blending (Eq. 2-3) of the sorted
 * Gaussians; pairs with alpha < alpha_low are skipped and a pixel stops
 * before the Gaussian that would take its transmittance below t_min.
 *   img [3,H,W] = sum_k c_k alpha_k T_k + T_final * bg
 *   t_final [H,W] final transmittance (may be NULL)
 *   load [H,W] int32 Gaussians blended per pixel, l_i of Eq. 12 (may be NULL). */
adr_status adr_render(adr_ctx *ctx, float *img, float *t_final, int32_t *load, void *stream);

/* Backward of the last adr_render (the differentiable path the paper trains
 * through, Sec. 4.4 total loss): given dL/dimg [3,H,W] and optionally
 * dL/dload [H,W] (may be NULL; it reaches the opacities through the reading
 * of d l_i / d alpha_ik that the frame's settings->load_grad selects, see
 * adr_load_grad), writes dL/d means [n,3], scales [n,3],
 * rots [n,4] (w,x,y,z; 16-byte aligned), opac [n] and sh [n,16,3] (16-byte aligned; coefficients
 * above sh_degree get 0).  The parameter arrays must be the ones passed to
 * adr_preprocess for this frame, unchanged.  Gradient buffers are overwritten.
 * Per tile, each pixel walks its blended Gaussians back to front recovering
 * T_k = T_{k+1}/(1-alpha_k); contributions are warp-reduced and then added to
 * per-Gaussian accumulators with atomics (summation order varies run to run). */
adr_status adr_render_backward(adr_ctx *ctx, const float *means, const float *scales,
                               const float *rots, const float *opac, const float *sh,
                               const float *dl_dimg, const float *dl_dload, float *g_means,
                               float *g_scales, float *g_rots, float *g_opac, float *g_sh,
                               void *stream);

/* Load-balancing loss (Sec. 4.4, Eq. 13): L_load = std over the hw pixels of
 * load (int32, population standard deviation).  Writes stats[0] = mean,
 * stats[1] = std (device doubles) and, if dl_dload is non-NULL, the gradient
 * weight * dL_load/dl_i = weight * (l_i - mean) / (hw * std) (0 if std = 0),
 * ready to pass to adr_render_backward. */
adr_status adr_load_loss(adr_ctx *ctx, const int32_t *load, int64_t hw, float weight,
                         double *stats, float *dl_dload, void *stream);

/* Image loss of the training objective (Sec. 4.4 total loss: the L1 and SSIM
 * terms beside L_load).  img and ref: [channels, height, width] device fp32
 * (the render and its target).  SSIM follows Wang et al. 2004: per channel,
 * local means, variances and covariance under the 11x11 Gaussian window of
 * standard deviation 1.5 (normalised), extended past the border with zeros so
 * the SSIM map has the image's size, with C1 = 0.01^2 and C2 = 0.03^2.
 * Writes stats[0] = mean |img - ref| and stats[1] = mean SSIM over every
 * element (device doubles).  If dl_dimg is non-NULL it is overwritten with the
 * gradient of  w_l1 * mean|img - ref| + w_ssim * (1 - mean SSIM)  with respect
 * to img (the L1 subgradient is 0 where img == ref); scratch must then hold
 * 3 * channels * height * width floats (device memory, contents clobbered).
 * Runs on the current CUDA device, which must own the pointers; enqueued on
 * `stream`.  ADR_ERR_INVALID for NULL pointers, non-positive sizes or more than
 * 2^31 elements, or a missing scratch. */
adr_status adr_image_loss(const float *img, const float *ref, int32_t channels, int32_t height,
                          int32_t width, float w_l1, float w_ssim, double *stats, float *dl_dimg,
                          float *scratch, void *stream);

/* Waits for the context's last stream and returns the pair count P (the sum
 * of tiles over Gaussians, which may exceed pair_capacity).  Returns
 * ADR_ERR_CAPACITY if P > pair_capacity, ADR_ERR_TIMEOUT if a bounded device
 * wait gave up (device flags are cleared).  SYNCHRONISES that stream. */
adr_status adr_num_pairs(adr_ctx *ctx, int64_t *num_pairs);

/* Inspection: sizes of the last rendered frame, first min(n, 7) of (HOST
 * int64 array): the pair count P, the Gaussians with tiles V, the column runs
 * of all of them C, whether the frame rendered in two depth slices (0/1), the
 * runs the tile sort built for slice 0 and for slice 1, and the Gaussians of
 * slice 1 (the last three 0 for an unsliced frame).  A sliced frame's tile
 * sort moves the runs of its two slices only.  SYNCHRONISES the context's
 * last stream.  ADR_ERR_INVALID before the first adr_render. */
adr_status adr_frame_counts(adr_ctx *ctx, int64_t *out, int32_t n);

/* Inspection (tests, debugging).  Copy the sorted pairs as 64-bit keys
 * (tile << 32) | bits(depth) and Gaussian indices into caller device buffers
 * of `capacity` entries (at most min(P, capacity) written).  Enqueued on
 * `stream` after adr_sort. */
adr_status adr_read_pairs(adr_ctx *ctx, uint64_t *keys, uint32_t *vals, int64_t capacity,
                          void *stream);

/* Inspection: per-Gaussian Preprocess results for the last adr_preprocess.
 *   geom [n, ADR_GEOM_FLOATS]: px, py, conic_a, conic_b, conic_c, opacity,
 *        r_x, r_y, red, green, blue, depth (for a Gaussian without tiles only
 *        r_x, r_y and depth; the other fields read 0).  After adr_render_host
 *        with mapped host buffers only the Gaussians the frame blended have
 *        their colour (see there; the others read 0)
 *   rect [n,4] int32 tile rectangle tx0, ty0, tx1, ty1 (exclusive ends)
 *   tiles [n] int32 number of tiles (0 = culled) */
adr_status adr_read_gaussians(adr_ctx *ctx, float *geom, int32_t *rect, int32_t *tiles,
                              void *stream);

/* Inspection: per-tile ranges [start, end) as uint32 pairs, tiles_x*tiles_y rows. */
adr_status adr_read_ranges(adr_ctx *ctx, uint32_t *ranges, void *stream);

/* Inspection: per-pixel statistics of the last adr_render, [H,W] int32 each
 * (either may be NULL).  last: 1-based position in the tile's sorted list of
 * the last Gaussian blended into the pixel (0 if none).  traversed: list
 * positions the pixel evaluated before it stopped or the list ended, i.e.
 * the pixel thread's serial load (Sec. 4.4). */
adr_status adr_read_pixel_stats(adr_ctx *ctx, int32_t *last, int32_t *traversed, void *stream);

/* Per-kernel timing (tracing).  While enabled, every kernel launch of the
 * context is bracketed by CUDA events recorded on the launching stream (a
 * few microseconds of host overhead per launch; the kernels themselves are
 * unchanged).  adr_profile_read waits for the recorded launches, reports for
 * each kernel that ran its id, summed device milliseconds and launch count
 * (at most max_kernels entries; *num_kernels = entries written), and resets
 * the record.  Names come from adr_profile_kernel_name.  Up to 8192 launches
 * are kept between reads; later ones are not timed. */
adr_status adr_profile_enable(adr_ctx *ctx, int32_t enable);
adr_status adr_profile_read(adr_ctx *ctx, int32_t max_kernels, int32_t *kernel_ids,
                            double *total_ms, int32_t *launches, int32_t *num_kernels);
const char *adr_profile_kernel_name(int32_t kernel_id);

/* Per-tile tracing of Render (scheduling and load balance across tiles, the
 * uneven load of Sec. 4.4).  While enabled (the first call allocates 32 bytes
 * per tile of the largest image; disabling synchronises the device and frees
 * them), every adr_render records for each tile the %globaltimer nanoseconds
 * (low 32 bits) at which its CTA started and ended, the SM it ran on and the
 * list positions it staged.  adr_read_tile_trace copies the last frame's
 * record into `out` (device memory, uint32 [2, tiles_y * tiles_x, 4]: the
 * first block for the whole list or depth slice 0, the second for depth slice
 * 1, whose tiles that finished in slice 0 stay zero), enqueued on `stream`.
 * ADR_ERR_INVALID if tracing is off or no frame was rendered. */
adr_status adr_trace_tiles(adr_ctx *ctx, int32_t enable);
adr_status adr_read_tile_trace(adr_ctx *ctx, uint32_t *out, void *stream);

/* Waits for the context's work and reports device-side flags as a status;
 * clears them.  SYNCHRONISES.  In order of precedence: ADR_ERR_TIMEOUT (a
 * bounded lookback wait of the run scan gave up; that frame's later stages
 * were skipped), ADR_ERR_CAPACITY (more pairs than pair_capacity), ADR_ERR_CUDA
 * (a device-side consistency check failed: a scatter index fell outside its
 * buffer and the write was skipped; not expected from valid inputs), else
 * ADR_OK. */
adr_status adr_sync_status(adr_ctx *ctx);

/* Testing hook for failure detection (the paper has no counterpart).  Every
 * device-side wait of the library is bounded: a decoupled-lookback wait of the
 * run-count scan (stage 2) that sees no progress for 2^22 polls gives up, flags
 * the frame and lets its kernels return, and the frame's later stages skip
 * their work; adr_sync_status, adr_render_frame_noalloc and adr_serve_poll then
 * return ADR_ERR_TIMEOUT.  This hook makes that happen on purpose, so tests can
 * drive the path without a fault: while withheld_chunk >= 0, the scan's chunk
 * `withheld_chunk` (4096 Gaussians with tiles per chunk, in depth order) never
 * publishes its prefix and every lookback wait gives up after spin_limit
 * (1..2^22) polls, so the next chunk's wait runs out (frames whose Gaussians
 * with tiles fill fewer than withheld_chunk + 2 chunks are unaffected).
 * withheld_chunk < 0 restores normal operation (spin_limit ignored).  The
 * setting is process-wide, applies to kernels launched after the call (a CUDA
 * graph captured meanwhile keeps it) and is not thread-safe with respect to
 * launches in flight on other threads.  ADR_ERR_INVALID for a spin_limit out
 * of range. */
adr_status adr_test_lookback_expiry(int32_t withheld_chunk, int32_t spin_limit);

/* End-to-end frame from HOST memory: the scene arrays and img [3,H,W] (and
 * t_final, load if non-NULL) are HOST pointers.  Runs preprocess, sort and
 * render and SYNCHRONISES `stream` before returning.
 * With ADR_HOST_READ_MAPPED (the default), if every one of those buffers is
 * pinned memory mapped into the device's address space (cudaHostAlloc /
 * cudaHostRegister, e.g. torch pin_memory; rots and sh 16-byte aligned),
 * Preprocess reads the scene in place over the host link (at most 44 bytes
 * of each Gaussian), the SH colours (192 bytes each) are read for the
 * Gaussians with tiles -- or, in a frame with depth slices, just before each
 * Render launch for the Gaussians it blends only, far fewer -- and Render
 * writes the outputs in place: nothing is copied.  Otherwise, and always with
 * ADR_HOST_READ_COPY, the arrays are copied into device staging buffers,
 * allocated by the first such call (max_gaussians * 236 bytes + image
 * buffers), and the outputs copied back.  The host buffers must not change
 * until the call returns. */
/* How adr_render_host reaches its HOST buffers (see there).  ADR_ERR_INVALID
 * for an unknown mode. */
typedef enum adr_host_read {
    ADR_HOST_READ_COPY = 0, ADR_HOST_READ_MAPPED = 1
} adr_host_read;
adr_status adr_set_host_reads(adr_ctx *ctx, int32_t mode);

adr_status adr_render_host(adr_ctx *ctx, const float *means, const float *scales,
                           const float *rots, const float *opac, const float *sh, int64_t n,
                           const adr_camera *camera, const adr_settings *settings,
                           float *img, float *t_final, int32_t *load, void *stream);

/* Allocation-free frame for small scenes.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc (or anything
 * that allocates) when they render -- e.g. an application whose device
 * memory belongs to its own allocator and forbids allocations after start-up,
 * or a real-time loop that cannot afford an allocation's implicit device
 * synchronisation -- and so cannot create an adr_ctx.
 * It runs the same stages as adr_preprocess + adr_sort + adr_render with all
 * intermediates in one static device array compiled into the library (about
 * 20 MB).  CUDA loads the array and the kernels it uses onto a device when they
 * are first used there (by default lazily, at the first call on that device);
 * from then on that device holds the array until the process exits.  That
 * first load is the driver's one-time allocation and may synchronise, so
 * callers that cannot take it make their first call on each device during
 * start-up, or set CUDA_MODULE_LOADING=EAGER.
 * Limits: n <= 32768 Gaussians, width and height <= 512, at most 1048576
 * Gaussian-tile pairs; larger sizes are rejected with ADR_ERR_INVALID, and a
 * frame that produces more pairs returns ADR_ERR_CAPACITY (image incomplete).
 * A bounded device wait that gave up returns ADR_ERR_TIMEOUT (checked first)
 * and a failed device-side consistency check ADR_ERR_CUDA.
 * Arguments are as for adr_preprocess and adr_render (device memory, the
 * caller's inputs and outputs; t_final and load may be NULL); the frame runs
 * on the current CUDA device.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  All calls on a device
 * share the one array: calls whose work overlaps on the GPU (different
 * streams or threads without ordering) race and corrupt each other.  Each
 * call clears what must start at zero, waits for its frame (SYNCHRONISES
 * `stream`) and reports device-side errors in its return value.  It calls no
 * cudaMalloc, cudaFree or allocating library routine. */
adr_status adr_render_frame_noalloc(const float *means, const float *scales, const float *rots,
                                    const float *opac, const float *sh, int64_t n,
                                    const adr_camera *camera, const adr_settings *settings,
                                    float *img, float *t_final, int32_t *load, void *stream);

/* ---- Serving: continuous batching of frames over resident scenes ---------
 * A server renders requests {scene, camera (any size up to max_width x
 * max_height)} -> image with the stages of adr_preprocess + adr_sort +
 * adr_render (Sec. 3, Fig. 2) on a device.  The paper renders one camera at a
 * time; the server's scheduler is this library's own.  A scheduler thread owns
 * max_slots execution slots, each a frame workspace (as adr_create's, for
 * slot_max_gaussians and slot_pair_capacity) with its own CUDA stream, so
 * frames in different slots overlap on the GPU.  Requests wait in a FIFO queue;
 * the head is admitted as soon as a slot is free and the predicted bytes of
 * everything in flight, plus its own, stay within mem_budget_bytes (a request
 * is always admitted when nothing is in flight).  Predicted bytes of a request
 * = 12 * pairs + 150 * n + 32 * W * H, with pairs = 1.25 * (the scene's learned
 * pairs per pixel) * W * H, or slot_pair_capacity while the scene has no
 * completed frame; each slot's buffers are allocated once, at creation, so the
 * budget bounds the working set in flight, not the allocation.  Batching: the
 * slots form max_slots / max_batch groups of max_batch; a free group takes the
 * queue head together with later queued requests on the same scene (up to
 * max_batch, each admitted only if the budget allows) and renders them as one
 * batched frame: one Preprocess launch over all their cameras (the scene is
 * read once), each camera's sort stages on its own stream, and one Render
 * launch per depth slice over all their tiles.  With max_batch = 1 each slot
 * renders one request at a time and frames of different requests only
 * overlap.  With use_graphs != 0 each (group, scene, batch size, image sizes)
 * frame is captured once into a CUDA graph and replayed after one-thread
 * kernels write the requests' cameras into the device copies the graph's
 * kernels read.  A request's result equals that of adr_preprocess + adr_sort +
 * adr_render on its own (bit-identical image), batched or not. */
typedef struct adr_server adr_server;

typedef struct adr_serve_config {
    int32_t max_slots;            /* 1..64 concurrent frames (a multiple of max_batch) */
    int64_t mem_budget_bytes;     /* admission budget, > 0 */
    int64_t slot_pair_capacity;   /* Gaussian-tile pairs per slot, 1..2^30 */
    int64_t slot_max_gaussians;   /* largest scene, 1..2^29 */
    int32_t max_width, max_height;/* largest image, <= 4096 each */
    int32_t use_graphs;           /* 0: plain launches; else graph replay */
    int32_t device;               /* CUDA device ordinal */
    int32_t max_batch;            /* 1..4 requests on one scene per batched frame */
} adr_serve_config;

/* Allocates every slot and starts the scheduler thread.  ADR_ERR_INVALID for
 * a configuration out of range (including max_batch outside 1..4 or not
 * dividing max_slots), ADR_ERR_CUDA if an allocation fails (nothing leaks). */
adr_status adr_serve_create(adr_server **server, const adr_serve_config *config);
/* Waits for frames in flight, stops the scheduler and frees everything.
 * Requests still queued are dropped.  NULL is a no-op. */
void adr_serve_destroy(adr_server *server);
/* Registers a resident scene (device pointers with the layout of
 * adr_preprocess; BORROWED: they must stay valid and unchanged while the
 * server lives) rendered with `settings`.  ADR_ERR_INVALID if n is outside
 * 1..slot_max_gaussians or a pointer is NULL or misaligned. */
adr_status adr_serve_add_scene(adr_server *server, const float *means, const float *scales,
                               const float *rots, const float *opac, const float *sh, int64_t n,
                               const adr_settings *settings, int32_t *scene_id);
/* Queues a request and returns at once with its ticket.  out_img: caller's
 * DEVICE buffer [3, H, W] fp32, written when the request completes; it must
 * stay valid until adr_serve_poll reports the ticket finished.  ADR_ERR_INVALID
 * for an unknown scene or a bad camera; ADR_ERR_ADMISSION (nothing queued) if
 * the request's minimum bytes (150 n + 32 W H + 49152) exceed the budget, so it
 * could never be admitted. */
adr_status adr_serve_submit(adr_server *server, int32_t scene_id, const adr_camera *camera,
                            float *out_img, uint64_t *ticket);
/* Waits up to timeout_us microseconds (0: do not wait) for a request.
 * Returns ADR_OK when its image is written (the ticket is then released),
 * ADR_PENDING if timeout_us == 0 and it is not finished, ADR_ERR_TIMEOUT if
 * the wait ran out (the ticket stays valid), or the request's own error
 * (ADR_ERR_CAPACITY: more pairs than slot_pair_capacity, image incomplete;
 * ADR_ERR_TIMEOUT: a bounded device wait gave up; ADR_ERR_CUDA), which also
 * releases the ticket.  ADR_ERR_INVALID for an unknown ticket or a negative
 * timeout_us (the ticket is left as it was). */
adr_status adr_serve_poll(adr_server *server, uint64_t ticket, int64_t timeout_us);
/* Statistics since creation, first min(n, 13) of: completed requests, p50
 * latency ms, p99 latency ms, mean latency ms (submit to completion seen by
 * the scheduler), the largest number of frames in flight at once, requests
 * admitted while another was in flight, requests rejected by admission,
 * completed frames per second (first submit to last completion), requests
 * that ended with ADR_ERR_CAPACITY, graph replays, batched frames launched,
 * the largest batch, mean requests per batched frame. */
adr_status adr_serve_stats(adr_server *server, double *out, int32_t n);
/* Restarts the statistics (requests in flight still complete into the new
 * window). */
adr_status adr_serve_reset_stats(adr_server *server);

/* Thread-local description of the last failure on this thread ("" if none). */
const char *adr_last_error(void);

/* Library version string. */
const char *adr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ADR_H */
