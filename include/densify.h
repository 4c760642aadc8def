/*
 * densify.h - C ABI of the GB300 LiDAR densification library (libdensify.so).
 *
 * The library implements the per-viewpoint hot path of Murasaki et al.,
 * "Real-Time LiDAR Point Cloud Densification for Low-Latency Spatial Data
 * Transmission":
 *
 *   1. merge the three staggered LiDAR scans of a viewpoint and project them
 *      into the camera view as one depth image (Sec. 2, System Overview),
 *      keeping the nearest depth per pixel;
 *   2. densify that sparse depth with the RGB-guided joint bilateral filter of
 *      Eq. (1)-(4) (Sec. 4.2; Algorithm 1 gives the same filter as a
 *      convolution / transpose-convolution pipeline), run in the two-stage
 *      form of Sec. 5: radius 4 on a depth map pooled to 1/3 resolution, then
 *      radius 2 at full resolution after restoring the first result;
 *   3. back-project the dense depth to coloured 3D points in the common frame
 *      (Sec. 2: coloured point clouds of all viewpoints are overlaid).
 *
 * Every step runs in hand-written CUDA kernels for sm_103a. The host side
 * admits frames against a device-memory budget, batches the frames waiting
 * for the GPU into one launch sequence (replayed as a CUDA graph), and hands
 * results back through tickets.
 *
 * Conventions
 *   - Matrices are row-major 4x4 rigid transforms in FP64 (*_to_world).
 *   - Camera frame: x right, y down, z forward; pixel (i, j) covers
 *     [i, i+1) x [j, j+1), so its centre is (i + 1/2, j + 1/2).
 *   - Depth is the camera z coordinate in the units of the point clouds.
 *   - RGB frames are H x W x 3 uint8, row pitch in bytes (>= 3 W, multiple
 *     of 16).
 *   - Unless a function says otherwise, pointers inside densify_frame are
 *     DEVICE pointers (memory = DENSIFY_MEM_DEVICE) owned by the caller; with
 *     memory = DENSIFY_MEM_HOST they are host pointers (page-locked for
 *     asynchronous copies) and the library copies inputs in and results out;
 *     page-locked point and count buffers are written by the GPU directly,
 *     at exact size, with no copy.
 *   - Every call returns a status; nothing throws across the ABI. Invalid
 *     point values (NaN, z <= 0 in the camera, outside the image) are not
 *     errors: such points are skipped.
 *   - A context is not thread-safe: use one context per host thread, or
 *     serialise the calls on it.
 */
#ifndef DENSIFY_H
#define DENSIFY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DENSIFY_API __attribute__((visibility("default")))
#else
#define DENSIFY_API
#endif

#define DENSIFY_ABI_VERSION 1
#define DENSIFY_MAX_SCANS 3     /* three LiDARs per viewpoint (Sec. 2) */
#define DENSIFY_MAX_BATCH 64    /* frames in one batched launch */

typedef struct densify_ctx densify_ctx; /* opaque */

typedef enum densify_status {
    DENSIFY_OK = 0,
    DENSIFY_PENDING = 1,      /* submitted, not finished yet */
    DENSIFY_E_INVALID = -1,   /* bad argument; see densify_last_error() */
    DENSIFY_E_NOMEM = -2,     /* can never fit the device-memory budget */
    DENSIFY_E_AGAIN = -3,     /* no free slot / budget now: poll, then retry */
    DENSIFY_E_CUDA = -4,      /* a CUDA call failed; context is unusable */
    DENSIFY_E_TIMEOUT = -5,   /* poll timed out; the frame is still pending */
    DENSIFY_E_TICKET = -6     /* unknown or already-collected ticket */
} densify_status;

typedef enum densify_precision {
    DENSIFY_FP32 = 0,         /* FP32 guide, weights and accumulation */
    DENSIFY_FP16 = 1          /* full-resolution filter stage: FP16 guide and weights, FP32
                                 numerator and weight sum (the pooled first stage stays FP32) */
} densify_precision;

typedef enum densify_memory {
    DENSIFY_MEM_DEVICE = 0,
    DENSIFY_MEM_HOST = 1
} densify_memory;

/* One joint bilateral filter stage (Eq. (1)-(4)): square window of
 * (2 radius + 1)^2 pixels (Algorithm 1: offsets a, b in [-r, r]), spatial
 * Gaussian sigma_p in the stage's own pixel units (Eq. (3)), colour Gaussian
 * sigma_c on the 0-255 RGB scale (Eq. (2)). */
typedef struct densify_stage {
    int32_t radius;
    float sigma_p;
    float sigma_c;
} densify_stage;

/* Context parameters. Fill with densify_default_params() and override.
 *   num_stages    1: one JBF at full resolution on the projected depth.
 *                 2: the two-stage filter of Sec. 5 (stage[0] on the map
 *                 pooled by `pool`, stage[1] at full resolution on the
 *                 restored result).
 *   stage         radii and sigmas. Supported radii: single stage 1-7,
 *                 coarse stage 1-7, full-resolution second stage 1-3.
 *   pool          pooling factor of the two-stage form (Sec. 5 uses 3).
 *   stage2_input  0: the second stage filters the restored first-stage result
 *                 only (the literal reading of Sec. 5); 1: pixels with a
 *                 LiDAR depth keep it instead of the restored value.
 *   precision     DENSIFY_FP32 or DENSIFY_FP16.
 *   emit_points   1: back-project to coloured points; 0: depth only.
 *   max_inflight  frames admitted at once (submitted and not yet collected).
 *   max_batch     frames per batched launch (<= DENSIFY_MAX_BATCH).
 *   batches_in_flight  launches allowed on the GPU at once; frames that
 *                 arrive while they run wait and go out together in the next
 *                 launch (continuous batching).
 *   hbm_budget_bytes   device memory the context may use for per-frame
 *                 scratch (z-buffers, coarse maps, staging of host frames);
 *                 admission fails with DENSIFY_E_AGAIN when it is full. In the
 *                 two-stage form with stage2_input 0 and no occlusion removal, a
 *                 quarter of it holds z-buffers that are kept empty between
 *                 frames (the pooling kernel empties the cells it read, so no
 *                 frame needs a clear), used by every frame that does not ask
 *                 for out_zbuf.
 *   use_graphs    1: replay each batch slot's launch sequence as a CUDA graph.
 *   timing        1: record CUDA events around every kernel of every batch and
 *                 accumulate per-kernel device time (densify_kernel_times);
 *                 each event is a node of the batch's graph and adds a small
 *                 gap between kernels. 2: events around the full-resolution
 *                 (last) filter kernel only. 0: none.
 *   launch_policy 0 (eager): a queued frame goes to the GPU as soon as a
 *                 launch slot is free; frames that arrive while every slot is
 *                 busy are launched together when one frees (continuous
 *                 batching). 1 (batch): frames wait until max_batch are
 *                 queued, or until densify_flush() / densify_poll().
 *   kernel_variant 0: filter kernels whose tiles are staged by TMA where the
 *                 stage has one (radius 1-3 second stage with pool 3 and
 *                 stage2_input 0; radius 2 or 4 first stage; radius 2, 4 or 7
 *                 single stage), the plain shared-memory kernels elsewhere.
 *                 In FP32 the TMA kernels take the expanded form (squared
 *                 colour distance as |c_p|^2 - 2 c_p.c_q + |c_q|^2 with colours
 *                 centred at 128; same sums, different rounding, within the
 *                 FP32 tolerance) where log2(e) / (2 sigma_c^2) * 3 * 128^2 +
 *                 log2(e) / (2 sigma_p^2) * 2 r^2 <= 100, else the difference
 *                 form; at radius 2 of a full-resolution stage also on pairs of
 *                 output columns in two-lane FP32 instructions, the colour
 *                 dot product taken exactly by dp4a on the colour bytes (one
 *                 rounding of the exponent instead of three, within the same
 *                 tolerance). For a single stage on the z-buffer the sparse
 *                 form runs first: a warp walks only the observed positions
 *                 of its 8 x 8 block's footprint and sums in registers (same
 *                 weights up to a per-pixel factor that cancels; in FP16, with
 *                 half2 weights and FP32 sums). 1: the plain
 *                 kernels everywhere (difference form, for comparison). 2: the
 *                 TMA kernels in the difference form only (the same bits as
 *                 1).
 *   autotune      1: on the first batch, time every kernel that can run each
 *                 filter stage (TMA-staged at each instantiated tile height,
 *                 and the plain kernel) on that batch and keep the fastest for
 *                 the context's lifetime; with DENSIFY_TUNE_CACHE=<file> in the
 *                 environment, choices are stored there and reused.
 * Preprocessing of the merged scans (Sec. 4.1) and post-filtering (Sec. 5);
 * each is off at 0 (the paper gives no values):
 *   occlusion_radius, occlusion_margin   occluded points: an observed pixel
 *                 deeper than the mean observed depth of its (2 r + 1)^2
 *                 window by more than the margin is removed before filtering
 *                 (radius 1-16).
 *   motion_threshold, motion_close_radius   afterimages: pixels whose RGB
 *                 distance to the previous frame (frame.prev_rgb) exceeds the
 *                 threshold, closed with a square element of this radius,
 *                 keep only the points of the most recent scan
 *                 (frame.newest_scan).
 *   contour_threshold   contours: a dense pixel with a 4-neighbour whose depth
 *                 differs by more than this fraction of its own depth is
 *                 dropped before back-projection.
 */
typedef struct densify_params {
    int32_t num_stages;
    densify_stage stage[2];
    int32_t pool;
    int32_t stage2_input;
    int32_t precision;
    int32_t emit_points;
    int32_t max_inflight;
    int32_t max_batch;
    int32_t batches_in_flight;
    int32_t use_graphs;
    uint64_t hbm_budget_bytes;
    int32_t timing;
    int32_t launch_policy;
    int32_t kernel_variant;
    int32_t autotune;
    int32_t occlusion_radius;
    float occlusion_margin;
    float motion_threshold;
    int32_t motion_close_radius;
    float contour_threshold;
    int32_t reserved[3];
} densify_params;

/* Pinhole intrinsics of the camera (Sec. 2: calibrated in advance). */
typedef struct densify_intrinsics {
    int32_t width, height;
    float fx, fy, cx, cy;
} densify_intrinsics;

/* One LiDAR scan: `count` points of float32 (x, y, z) in the LiDAR frame,
 * `stride_bytes` apart (12: packed xyz, 16: xyzw). The base address must be
 * 16-byte aligned. lidar_to_world is the scan's calibrated extrinsic. */
typedef struct densify_scan {
    const float *xyz;
    int64_t count;
    int32_t stride_bytes;
    int32_t reserved;
    double lidar_to_world[16];
} densify_scan;

/* One frame of one viewpoint.
 * Inputs: intrinsics, camera pose, 0..3 scans, the RGB frame.
 * Outputs (caller-owned, written when the frame completes):
 *   out_depth  H x W float, densified depth, 0 where invalid (may be NULL)
 *   out_valid  H x W uint8, 1 where the filter window held an observation
 *   out_points up to out_points_cap points of 4 floats
 *              (x, y, z in the world frame, then the colour packed as
 *              r | g << 8 | b << 16 | 255 << 24 in the bits of the 4th float),
 *              in row-major pixel order of the valid pixels;
 *   out_points_n  one int64: the number of valid pixels. Points past the
 *              capacity are dropped, so n > cap means the buffer was short.
 * Optional debug outputs (NULL to skip; device memory like the rest):
 *   out_zbuf     H x W uint32: the nearest-depth z-buffer (bit patterns of
 *                FP32 depths, 0x7F800000 where empty)
 *   out_coarse   ceil(H/pool) x ceil(W/pool) float: first-stage depth
 *   out_coarse_valid  same size, uint8: first-stage validity
 * Afterimage removal (params.motion_threshold > 0):
 *   prev_rgb     the viewpoint's previous RGB frame (same size; NULL: skip)
 *   newest_scan  index of the most recent scan; the others lose their points
 *                inside the motion mask
 *   out_motion   optional H x W uint8 copy of the closed motion mask
 * memory says whether every pointer above is a device or a host pointer. */
typedef struct densify_frame {
    densify_intrinsics K;
    double cam_to_world[16];
    int32_t num_scans;
    int32_t memory;
    densify_scan scans[DENSIFY_MAX_SCANS];
    const uint8_t *rgb;
    int64_t rgb_pitch;
    float *out_depth;
    uint8_t *out_valid;
    float *out_points;
    int64_t out_points_cap;
    int64_t *out_points_n;
    uint32_t *out_zbuf;
    float *out_coarse;
    uint8_t *out_coarse_valid;
    const uint8_t *prev_rgb;
    int64_t prev_rgb_pitch;
    int32_t newest_scan;
    int32_t reserved_f;
    uint8_t *out_motion;
} densify_frame;

/* Fill *p with the paper's two-stage configuration (Sec. 5: pool 3, radius 4
 * then radius 2; sigma_p = 5 px and sigma_c = 20 in both stages, since the
 * paper sets the sigmas empirically without printing them), FP32, points on,
 * 16 frames in flight, batches of up to 16, one batch on the GPU at a time,
 * a 2 GiB budget and CUDA graphs on. */
DENSIFY_API void densify_default_params(densify_params *p);

/* Sets up the per-viewpoint path of Sec. 2 (merge and projection of the
 * scans, the joint bilateral filter of Eq. (1)-(4) in the two-stage schedule
 * of Sec. 5, back-projection to coloured points) on one GPU.
 * Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL: the context creates its own non-blocking stream).
 * Allocates the scratch arena (hbm_budget_bytes) and per-batch descriptors
 * up front; nothing is allocated per frame afterwards.
 * Errors: E_INVALID (bad params), E_NOMEM, E_CUDA. *out is NULL on error. */
DENSIFY_API densify_status densify_create(const densify_params *params, int device, void *cuda_stream,
                              densify_ctx **out);

/* One frame of one viewpoint: its camera image and the (up to three) LiDAR
 * scans staggered in time that Sec. 2 merges into one depth image.
 * Admit one frame (non-blocking). Validates it, reserves its scratch in the
 * arena and queues it; the frame goes to the GPU at once if a launch slot
 * is free, else with the next batch. The caller keeps every buffer alive and
 * unmodified until densify_poll() returns DENSIFY_OK (or an error) for the
 * ticket. Errors: E_INVALID (bad frame), E_AGAIN (max_inflight frames
 * admitted or no scratch free right now: collect results, then retry),
 * E_NOMEM (the frame can never fit the budget), E_CUDA. */
DENSIFY_API densify_status densify_submit(densify_ctx *ctx, const densify_frame *frame, uint64_t *ticket);

/* Runs the queued frames' path (Sec. 2: projection and densification, done
 * independently per viewpoint, here many viewpoints in one batched launch).
 * Send every queued frame to the GPU now, waiting (bounded by timeout_ns,
 * <0: no bound) for a launch slot if all are busy. */
DENSIFY_API densify_status densify_flush(densify_ctx *ctx, int64_t timeout_ns);

/* Collects one frame's results: the dense depth and validity of Eq. (1)
 * (after the two stages of Sec. 5) and its coloured points (Sec. 2).
 * Wait up to timeout_ns (0: just check; <0: no bound) for a ticket.
 * Returns OK (results written; the ticket is collected and its scratch
 * freed), PENDING (timeout_ns == 0 and not done), E_TIMEOUT, E_TICKET or
 * E_CUDA. Polling also launches frames that were waiting for a slot. */
DENSIFY_API densify_status densify_poll(densify_ctx *ctx, uint64_t ticket, int64_t timeout_ns);

/* Ends the per-viewpoint path of Sec. 2 set up by densify_create.
 * Wait (bounded: at most timeout_ns per outstanding batch, 10 s if <0) for
 * in-flight work, then free every resource of the context. */
DENSIFY_API densify_status densify_destroy(densify_ctx *ctx);

/* Static string naming a status. (No counterpart in the paper: Sec. 2
 * describes no error reporting; the codes are this library's.) */
DENSIFY_API const char *densify_status_str(densify_status s);

/* (No counterpart in the paper: error detail of this library's calls.)
 * The last error message of a context (empty if none). Valid until the next
 * call on the context. ctx may be NULL: the last error of a failed create. */
DENSIFY_API const char *densify_last_error(const densify_ctx *ctx);

/* Device bytes one frame of this shape reserves from the arena: the z-buffer
 * (D and B of Algorithm 1), the pooled maps and first-stage result of the
 * two-stage filter (Sec. 5) and the compaction counts. */
DENSIFY_API uint64_t densify_frame_scratch_bytes(const densify_params *params, const densify_frame *frame);

/* (No counterpart in the paper: Table 1 reports only a per-frame total.)
 * Per-kernel device time accumulated since the last reset, when the context
 * was created with timing = 1: for each kernel, its static name, the summed
 * CUDA-event duration in microseconds over all completed batches and the
 * number of launches. Times are read when batches are collected, so call
 * after the tickets of interest returned OK. Returns the number of kernels
 * written (<= cap). */
DENSIFY_API int32_t densify_kernel_times(densify_ctx *ctx, const char **names, double *total_us,
                             int64_t *launches, int32_t cap);

/* Zero the accumulated kernel times and the kernel launch count. (No
 * counterpart in the paper.) */
DENSIFY_API void densify_reset_kernel_times(densify_ctx *ctx);

/* (No counterpart in the paper: launch accounting of this library.)
 * Number of CUDA kernels launched by the context's completed batches since
 * creation or the last densify_reset_kernel_times (a replayed graph counts each
 * of its kernels; the autotuner's trial launches are not counted). With
 * timing = 1 or 0 alike. */
DENSIFY_API int64_t densify_kernel_launches(densify_ctx *ctx);

/* (No counterpart in the paper: a test hook for this library's error path.)
 * Makes the next batch launched on the context report what its kernels report
 * when a bounded wait on tile copies gives up: the host sets bit 0 of the
 * batch's device status word on the batch's stream, after its kernels and
 * before the status is read back (no wait on the GPU actually runs out).
 * Collecting that batch's tickets then returns DENSIFY_E_CUDA with the
 * bounded-wait message in densify_last_error(), and the context stays
 * unusable (every later call returns DENSIFY_E_CUDA), as after a real
 * timeout. Errors: E_INVALID (ctx NULL), E_CUDA (context already failed). */
DENSIFY_API densify_status densify_inject_wait_failure(densify_ctx *ctx);

/* The kernels that run the filter stages of Sec. 5 (Eq. (1)-(4) each).
 * JSON text describing the filter kernels the context runs: per filter stage the
 * chosen kernel (TMA-staged or plain, rows per thread, tile, grid) and, after
 * autotuning, every candidate's measured time; then the number of batches
 * launched and the most batches in flight at once (launched, not yet
 * complete). Writes at most cap bytes
 * (NUL-terminated); returns the length of the full text. */
DENSIFY_API int32_t densify_describe(densify_ctx *ctx, char *buf, int32_t cap);

/* Densify one frame without allocating any device memory. (The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc, for example a
 * real-time loop whose device-memory footprint is frozen after start-up, or a
 * plug-in hosted by an application whose allocator owns the GPU's memory.)
 *
 * Runs the same steps as a context (calibration, projection, the filter stages
 * of *params, back-projection) on `cuda_stream` (a cudaStream_t, NULL: the
 * default stream) and returns once the work is enqueued; the results are in
 * the frame's output buffers when the stream reaches that point. Every frame
 * pointer must be a device pointer (memory = DENSIFY_MEM_DEVICE); out_depth
 * and out_valid are required; out_points / out_points_n as for a context when
 * params->emit_points is set; out_zbuf, out_coarse, out_coarse_valid optional.
 * The filter runs in the plain shared-memory kernels (no TMA staging).
 *
 * Scratch (descriptor, z-buffer, pooled maps, first-stage result, compaction
 * counts) is one fixed 16 MiB array in device memory that every GPU loading
 * the library holds until the process exits: one 1920x1080 two-stage frame
 * fits; a frame needing more returns DENSIFY_E_INVALID with the byte count.
 * Every call reuses the same array and leaves its contents behind: all of it
 * is rewritten or cleared before it is read, but calls whose work overlaps on
 * the GPU (two streams, or two host threads) race on it; serialise them.
 * The first call on a device looks up the array's device address and the SM
 * count (once per device, with that device current); make that first call
 * before any stream capture, and before the device-memory footprint is
 * frozen: like the first launch of any kernel under lazy module loading, it
 * may load the library's kernel code into device memory. Later calls leave the
 * device's free memory unchanged. No cudaMalloc, cudaFree or other allocating call
 * is made. Errors: E_INVALID (bad argument or too large), E_CUDA (a launch
 * failed); the message is in densify_last_error(NULL). */
DENSIFY_API densify_status densify_frame_noalloc(const densify_params *params, const densify_frame *frame,
                                                 void *cuda_stream);

/* Gradient of the depth error with respect to the filter's sigmas (Sec. 4:
 * when dense ground truth exists, the Gaussian variances can be optimised by
 * backpropagation). Runs the context's path on one device frame (calibration,
 * projection, pooling, the filter stages with their sigma derivatives,
 * chained through the restore of the two-stage form) and returns
 *   *loss      mean over pixels with a filtered depth and gt_depth > 0 of
 *              (depth - gt)^2,
 *   grad[4]    d loss / d (stage[0].sigma_p, stage[0].sigma_c,
 *              stage[1].sigma_p, stage[1].sigma_c) (the last two 0 for a
 *              single stage),
 *   *n_pixels  the number of pixels in the mean.
 * gt_depth is a device H x W float map. Synchronous: waits for in-flight
 * batches, uses arena scratch, returns when the numbers are on the host.
 * Preprocessing and contour removal are not part of it. Errors: E_INVALID,
 * E_AGAIN (scratch full), E_CUDA. */
DENSIFY_API densify_status densify_sigma_grad(densify_ctx *ctx, const densify_frame *frame, const float *gt_depth,
                                              double *loss, double *grad, int64_t *n_pixels);

/* ABI version of the loaded library (DENSIFY_ABI_VERSION). (No counterpart
 * in the paper.) */
DENSIFY_API int32_t densify_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DENSIFY_H */
