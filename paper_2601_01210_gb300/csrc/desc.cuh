// Device-side descriptors shared by the host runtime and the kernels.
//
// One batched launch processes up to kMaxBatch frames (viewpoints) of uneven
// resolution and point count. The host writes a BatchDev table into a fixed
// device buffer per batch slot; every kernel is a persistent grid-stride loop
// over work items (point chunks, z-buffer chunks, coarse pixels, filter
// tiles, compaction chunks) whose per-frame prefix sums sit in the table, so
// the launch sequence of a slot never changes and can be replayed as a CUDA
// graph.
#pragma once

#include <cstdint>
#include <cuda.h>          // CUtensorMap (type only; maps are encoded through the runtime's driver entry point)
#include <cuda_runtime.h>

namespace dz {

constexpr int kMaxBatch = 64;
constexpr int kMaxScans = 3;
constexpr uint32_t kEmpty = 0x7F800000u;   // z-buffer cell with no depth (+inf)

// Work-item granularity of the non-filter kernels.
constexpr int kThreads = 256;
constexpr int kPtsPerThread = 4;
constexpr int kPtsPerChunk = kThreads * kPtsPerThread;        // 1024 points
constexpr int kZbWordsPerChunk = 8192;                        // z-buffer clear: 8 uint4 stores a thread
constexpr int kPoolPerChunk = kThreads;                       // coarse pixels (one coarse row segment)
constexpr int kBpChunk = 4096;                                // compaction: 8 warps x 512 px
constexpr int kBpWarps = kThreads / 32;                       // parts of a chunk, one per warp
constexpr int kBpPart = kBpChunk / kBpWarps;                  // 512 pixels
constexpr int kPxChunk = 1024;                                // per-pixel kernels: 256 threads x 4 px
constexpr int kMarkBand = 16;                                 // tile marks: rows of a warp's band

struct ScanDev {
    const float *xyz;
    int64_t count;
    int32_t stride_floats;   // 3 or 4
    int32_t pad;
    double l2w[16];          // lidar_to_world, row-major
    float M[12];             // camera <- LiDAR, composed on the GPU in FP64
};

// Tensor maps of a frame (TMA descriptors, encoded on the host per batch).
enum { TM_RGB = 0, TM_S1 = 1, TM_CGUIDE = 2, TM_CSSUM = 3, TM_ZBUF = 4, TM_COUNT = 5 };

struct alignas(64) FrameDev {
    CUtensorMap tm[TM_COUNT];
    int32_t W, H, Wc, Hc;    // full and coarse (ceil(H/pool) x ceil(W/pool)) grids
    int32_t cpitch;          // row pitch of the coarse arrays in elements (multiple of 4)
    int32_t zpitch;          // row pitch of the z-buffer in elements (multiple of 4)
    int32_t pad0;
    int32_t tma;             // tensor maps valid
    float fx, fy, cx, cy;
    double c2w[16];          // cam_to_world, row-major
    float c2w32[12];         // written by the prep kernel (FP64 -> FP32 once)
    int32_t num_scans;
    int32_t n_bp_chunks;
    ScanDev scans[kMaxScans];
    const uint8_t *rgb;      // H x W x 3, rgb_pitch bytes per row
    int64_t rgb_pitch;
    // scratch (context arena)
    uint32_t *zbuf;          // H x zpitch nearest-depth bit patterns
    float4 *cguide;          // Hc x cpitch: pooled mean r, g, b and observation count
    float *cssum;            // Hc x cpitch: pooled depth sum
    float2 *s1;              // Hc x cpitch: first-stage depth and validity (0/1)
    float2 *g1;              // Hc x cpitch: first-stage depth derivatives (sigma gradient only)
    uint32_t *chunk_cnt;     // n_bp_chunks * kBpWarps valid-pixel counts of 512-pixel parts
    // preprocessing (Sec. 4.1) and post-filtering (Sec. 5); NULL / 0 when off
    const uint8_t *prev_rgb;     // previous RGB frame (afterimage removal)
    int64_t prev_pitch;
    uint8_t *motion;             // H x W motion mask after the closing
    uint8_t *motion_tmp;         // the raw mask, then its dilation, bit-packed (rows of ceil(W / 32) words)
    uint32_t *zbuf_raw;          // projection target when occluded points are removed into zbuf
    int32_t newest_scan;         // scan kept inside the motion mask
    int32_t n_px_chunks;         // ceil(W H / kPxChunk)
    // filter outputs (== out_* unless contour removal rewrites them)
    float *flt_depth;
    uint8_t *flt_valid;
    // outputs (caller memory, or arena staging for host frames)
    float *out_depth;
    uint8_t *out_valid;
    float4 *out_points;
    int64_t points_cap;
    int64_t *points_n;
    float *out_coarse;       // optional first-stage depth copy
    uint8_t *out_coarse_valid;
    // TMA filters (index 0: first or only filter, 1: second): one flag per tile of the stage,
    // row-major over the frame's tiles, nonzero when some observation reaches the tile; both
    // stages' flags are one block of ntflags words of the frame's scratch, zeroed by the batch's
    // first kernel and set by the kernel in front of the filter (the pooling kernel for the first
    // of two stages, the first filter for the second, tile_mark_kernel for a single stage)
    int32_t *tflags[2];
    int32_t ntflags;
    // z-buffer upkeep: zclear = the batch's first kernel clears it; zrestore = it comes from the
    // context's pool of clean z-buffers and the pooling kernel, its last reader, writes the empty
    // pattern back into the cells it finds observed
    uint8_t zclear;
    uint8_t zrestore;
    uint8_t pad1[2];
};

struct BatchDev {
    int32_t n_frames;
    int32_t pad;
    int32_t *status;                               // device word: nonzero after a bounded wait gave up
    int32_t zb_pre[kMaxBatch + 1];                 // z-buffer clear chunks
    int32_t pt_pre[kMaxBatch * kMaxScans + 1];     // point chunks per (frame, scan)
    int32_t pool_pre[kMaxBatch + 1];               // pooling chunks
    int32_t t1_pre[kMaxBatch + 1];                 // tiles of the first (or only) filter
    int32_t t2_pre[kMaxBatch + 1];                 // tiles of the full-resolution second filter
    int32_t bp_pre[kMaxBatch + 1];                 // compaction chunks
    int32_t px_pre[kMaxBatch + 1];                 // pixel chunks of the motion / contour kernels
    int32_t oc_pre[kMaxBatch + 1];                 // tiles of the occlusion kernel
    int32_t mk_pre[kMaxBatch + 1];                 // 32-pixel row segments of the observation grid
    // TMA filters (index 0: first or only filter, 1: second); the tile flags are per frame
    // (FrameDev::tflags)
    int32_t tl_on;                                 // some stage runs a TMA filter: frames carry tile flags
    int32_t tl_pad;
    int32_t tl_next[2];                            // the filter's tile counter (reset by the prep kernel; by the
                                                   // mark kernel or a memset before a filter launched on its own)
    int32_t tl_tw[2];                              // tile width of a TMA filter stage (32 or 64)
    int32_t tl_th[2];                              // tile height of a TMA filter stage (0: no tile flags)
    int32_t tl_r[2];                               // its radius
    FrameDev f[kMaxBatch];
};

// Per-context filter constants for one stage (by value in kernel parameters,
// so the per-tap spatial terms are constant-bank operands).
constexpr int kMaxR = 7;
struct StageArgs {
    float kc;                // log2(e) / (2 sigma_c^2)
    float kp;                // log2(e) / (2 sigma_p^2)
    int32_t pool;            // restore factor of the second stage
    int32_t override_sparse; // second stage: LiDAR depths replace the restored value
    float sp[(2 * kMaxR + 1) * (2 * kMaxR + 1)];   // -(dx^2 + dy^2) kp, row-major over (dy, dx)
    // FP16 form (pairs of vertically adjacent output pixels, see jbf_tma.cuh):
    uint32_t kc2;            // half2 bits of (-kc, -kc)
    // half2 bits of (sp[d][dx], sp[d-1][dx]) for d = 0 .. 2R+1, row-major over (d, dx);
    // a term outside 0..2R is -inf (its weight is 0)
    uint32_t sp2[(2 * kMaxR + 2) * (2 * kMaxR + 1)];
    // Expanded FP32 form (see jbf_tma.cuh): the spatial weight of offset
    // (dx - R, dy - R) split into a column factor ex_sx[dx] = 2^(-(dx-R)^2 kp)
    // and a row exponent ex_sy[dy] = -(dy-R)^2 kp (0 beyond 2R)
    float ex_sx[2 * kMaxR + 1];
    float ex_sy[2 * kMaxR + 1];
};

// Flag the filter tiles (tw x th output pixels, tw a power of two, row-major per frame) that an
// observation range reaches: columns [ox0, ox1] and rows [oy0, oy1] of a grid f times coarser
// than the gw x gh output grid, grown by the radius r. The lanes of one warp share the stores,
// plain stores of the same value (no read first: the caller does not wait on a load).
__device__ __forceinline__ void mark_reach(int32_t *flags, int tw, int th, int r, int f, int gw, int gh, int ox0,
                                           int ox1, int oy0, int oy1, int lane) {
    const int xlo = max(0, f * ox0 - r), xhi = min(gw - 1, f * ox1 + f - 1 + r);
    const int ylo = max(0, f * oy0 - r), yhi = min(gh - 1, f * oy1 + f - 1 + r);
    if (xlo > xhi || ylo > yhi) return;
    const int sw = __ffs(tw) - 1;   // tile widths are powers of two
    const int tiles_x = (gw + tw - 1) >> sw;
    const int tx0 = xlo >> sw, tx1 = xhi >> sw;
    const int sh = __ffs(th) - 1;   // tile heights mostly are
    const bool pow2 = th == 1 << sh;
    const int ty0 = pow2 ? ylo >> sh : ylo / th, ty1 = pow2 ? yhi >> sh : yhi / th;
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0 + lane; tx <= tx1; tx += 32) flags[ty * tiles_x + tx] = 1;
}

// Largest i with pre[i] <= item (pre is non-decreasing, pre[0] = 0).
__device__ __forceinline__ int find_segment(const int32_t *pre, int n, int item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Kernel launchers. Grids are persistent: a multiple of the SM count.
enum KernelId {
    K_PREP = 0, K_MOTION, K_DILATE, K_ERODE, K_PROJECT, K_OCCLUSION, K_POOL, K_JBF1, K_JBF2, K_CONTOUR,
    K_BP_COUNT, K_BP_WRITE, K_MARK1, K_COUNT
};

// Preprocessing / post-filtering (k_prepost.cu).
struct PrepostArgs {
    float motion_t2;      // squared RGB distance threshold (FP32)
    int32_t close_radius; // closing structuring element radius
    int32_t occ_radius;   // averaging window radius
    float occ_margin;     // depth margin behind the window average
    float contour_t;      // relative depth step threshold
};
cudaError_t launch_motion(const BatchDev *b, const PrepostArgs &a, int grid, cudaStream_t s);
cudaError_t launch_morph(const BatchDev *b, const PrepostArgs &a, bool dilate, int grid, cudaStream_t s);
cudaError_t launch_occlusion(const BatchDev *b, const PrepostArgs &a, int grid, cudaStream_t s);
cudaError_t launch_contour(const BatchDev *b, const PrepostArgs &a, int grid, cudaStream_t s);
int occupancy_prepost(KernelId k);
constexpr int kOccTile = 32;   // occlusion kernel output tile (32 x 32)

cudaError_t launch_prep(const BatchDev *b, int grid, cudaStream_t s);
// every word of [p, p + n) set to the empty z-buffer cell
cudaError_t launch_fill_empty(uint32_t *p, uint64_t n, cudaStream_t s);
cudaError_t launch_project(const BatchDev *b, int grid, cudaStream_t s);
cudaError_t launch_pool(const BatchDev *b, int pool, int grid, cudaStream_t s);
cudaError_t launch_bp_count(const BatchDev *b, int grid, cudaStream_t s);
cudaError_t launch_bp_write(const BatchDev *b, int grid, cudaStream_t s);
int occupancy_points(KernelId k);
int occupancy_pool_bp(KernelId k);

// Joint bilateral filter, one entry per stage kind:
//   single: full resolution, z-buffer input (radii 1-7)
//   coarse: pooled grid, first of the two stages (radii 1-7)
//   up:     full resolution on the restored first-stage result (radii 1-3)
// Tiles are 32 x (8 * kp) output pixels.
cudaError_t launch_jbf_single(int radius, const BatchDev *b, const StageArgs &a, int grid, cudaStream_t s);
cudaError_t launch_jbf_coarse(int radius, const BatchDev *b, const StageArgs &a, int grid, cudaStream_t s);
cudaError_t launch_jbf_up(int radius, const BatchDev *b, const StageArgs &a, int grid, cudaStream_t s);
int occupancy_jbf_single(int radius);
int occupancy_jbf_coarse(int radius);
int occupancy_jbf_up(int radius);
int kp_jbf_single(int radius);
int kp_jbf_coarse(int radius);
int kp_jbf_up(int radius);

}  // namespace dz
