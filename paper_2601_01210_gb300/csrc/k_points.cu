// Calibration compose, z-buffer clear and LiDAR projection (Sec. 2: the three
// scans of a viewpoint are merged and projected into the camera view to form
// one depth image; the depth image D and mask B of Algorithm 1).
//
// Arithmetic contract (bit-exact z-buffer):
//   * M_s = inverse(cam_to_world) * lidar_to_world in FP64 with the rigid
//     inverse [R^T, -R^T t]; each entry summed left to right over k = 0..2,
//     translation added last; rounded once to FP32.
//   * per point, FP32 with every product, sum and quotient rounded on its own
//     (no contraction): xc = ((m00 x + m01 y) + m02 z) + m03 (likewise yc, zc),
//     u = fx (xc / zc) + cx, v = fy (yc / zc) + cy;
//   * kept iff zc > 0 and finite, 0 <= u < W, 0 <= v < H; pixel (floor u,
//     floor v); the z-buffer keeps the smallest zc as its FP32 bit pattern
//     (atomicMin on uint32 is order-preserving for positive floats).
#include "desc.cuh"

namespace dz {

// ---------------------------------------------------------------------------
// prep: one work item per z-buffer chunk; the first chunk of each frame also
// composes the frame's calibration (the only FP64 arithmetic on the GPU).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double compose_entry(const double *c2w, const double *l2w, int i, int j) {
    // Rinv[i][k] = R[k][i]
    const double r0 = c2w[0 * 4 + i], r1 = c2w[1 * 4 + i], r2 = c2w[2 * 4 + i];
    double s = __dmul_rn(r0, l2w[0 * 4 + j]);
    s = __dadd_rn(s, __dmul_rn(r1, l2w[1 * 4 + j]));
    s = __dadd_rn(s, __dmul_rn(r2, l2w[2 * 4 + j]));
    if (j == 3) {
        double t = __dmul_rn(r0, c2w[0 * 4 + 3]);
        t = __dadd_rn(t, __dmul_rn(r1, c2w[1 * 4 + 3]));
        t = __dadd_rn(t, __dmul_rn(r2, c2w[2 * 4 + 3]));
        s = __dadd_rn(s, -t);
    }
    return s;
}

// The batch's first kernel: calibration compose, tile flags and counters, z-buffer clear.
__global__ void __launch_bounds__(kThreads) prep_kernel(BatchDev *__restrict__ B) {
    // the batch's clear prefix, each frame's z-buffer and tile-flag block in shared memory, all read
    // at once: the stores below then wait on no chain of dependent global loads (a store through a
    // pointer read from the descriptor could alias the descriptor, which would order the next read
    // after it)
    __shared__ int32_t s_pre[kMaxBatch + 1];
    __shared__ uint32_t *s_z[kMaxBatch];
    __shared__ int64_t s_n[kMaxBatch];
    __shared__ int32_t *s_fl[kMaxBatch];
    __shared__ int32_t s_nfl[kMaxBatch];
    __shared__ int32_t s_tl_on;
    const int nf = B->n_frames;
    if (threadIdx.x == 0) s_tl_on = B->tl_on;
    for (int i = threadIdx.x; i <= nf; i += kThreads) s_pre[i] = B->zb_pre[i];
    for (int i = threadIdx.x; i < nf; i += kThreads) {
        s_z[i] = B->f[i].zbuf_raw;
        s_n[i] = (int64_t)B->f[i].zpitch * B->f[i].H;
        s_fl[i] = B->f[i].tflags[0];
        s_nfl[i] = B->f[i].ntflags;
    }
    __syncthreads();
    // the TMA filters' tile flags (each frame's block of both stages) and tile counters start the
    // batch cleared; the producers (pooling, first filter) and the mark kernel set the flags
    if (s_tl_on) {
        if (blockIdx.x == 0 && threadIdx.x == 0) B->tl_next[0] = B->tl_next[1] = 0;   // the filters' tile counters
        for (int f = 0; f < nf; ++f) {
            int32_t *const fl = s_fl[f];
            const int n = s_nfl[f];
            for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) fl[i] = 0;
        }
    }
    // calibration compose: block f takes frame f
    for (int f = blockIdx.x; f < nf; f += gridDim.x) {
        FrameDev &F = B->f[f];
        const int t = threadIdx.x;
        if (t < F.num_scans * 12) {
            const int s = t / 12, e = t % 12;
            F.scans[s].M[e] = __double2float_rn(compose_entry(F.c2w, F.scans[s].l2w, e / 4, e % 4));
        } else if (t >= 64 && t < 76) {
            const int e = t - 64;
            F.c2w32[e] = __double2float_rn(F.c2w[(e / 4) * 4 + (e % 4)]);
        }
    }
    // z-buffer clear: the chunks of the frames that clear (a frame from the clean pool has none)
    const int total = s_pre[nf];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int f = find_segment(s_pre, nf, item);
        const int c = item - s_pre[f];
        const int64_t n = s_n[f];
        const int64_t w0 = (int64_t)c * kZbWordsPerChunk;
        const int64_t w1 = min(n, w0 + kZbWordsPerChunk);
        uint32_t *z = s_z[f];
        // arena buffers are 256-byte aligned and w0 is a multiple of 4; every thread's stores of the
        // chunk are issued together
        const int64_t v1 = w0 + ((w1 - w0) & ~int64_t(3));
        const uint4 e4 = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
#pragma unroll
        for (int k = 0; k < kZbWordsPerChunk / (4 * kThreads); ++k) {
            const int64_t w = w0 + 4 * (threadIdx.x + k * kThreads);
            if (w < v1) *reinterpret_cast<uint4 *>(z + w) = e4;
        }
        for (int64_t w = v1 + threadIdx.x; w < w1; w += kThreads) z[w] = kEmpty;
    }
}

// ---------------------------------------------------------------------------
// project: one work item = kPtsPerChunk consecutive points of one (frame, scan);
// each thread takes kPtsPerThread points with 16-byte vector loads.
// ---------------------------------------------------------------------------
// A (frame, scan) of the batch as the projection reads it. Every block copies the batch's table
// into shared memory once, all entries at once, so that a work item starts its point loads
// without first waiting on the descriptor (an atomic on the z-buffer could alias the descriptor,
// so the compiler would reload it from global memory after every atomic).
struct ProjSeg {
    float M[12];
    float fx, fy, cx, cy, w, h;
    const float *xyz;
    uint32_t *zbuf;
    const uint8_t *motion;   // NULL unless afterimage removal applies to this scan
    int64_t count;
    int64_t zpitch;
    int32_t W;
    int32_t stride_floats;
};

__device__ __forceinline__ void project_one(const ProjSeg &C, float x, float y, float z) {
    const float *M = C.M;
    const float xc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(M[0], x), __fmul_rn(M[1], y)), __fmul_rn(M[2], z)), M[3]);
    const float yc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(M[4], x), __fmul_rn(M[5], y)), __fmul_rn(M[6], z)), M[7]);
    const float zc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(M[8], x), __fmul_rn(M[9], y)), __fmul_rn(M[10], z)), M[11]);
    if (!(zc > 0.0f) || !(zc < __int_as_float(0x7F800000))) return;
    const float u = __fadd_rn(__fmul_rn(C.fx, __fdiv_rn(xc, zc)), C.cx);
    const float v = __fadd_rn(__fmul_rn(C.fy, __fdiv_rn(yc, zc)), C.cy);
    if (!(u >= 0.0f && u < C.w && v >= 0.0f && v < C.h)) return;
    const int i = __float2int_rz(u);   // u >= 0: truncation is floor
    const int j = __float2int_rz(v);
    // afterimage removal: points of older scans are dropped where the scene moved
    if (C.motion && C.motion[(int64_t)j * C.W + i]) return;
    atomicMin(C.zbuf + (int64_t)j * C.zpitch + i, __float_as_uint(zc));
}

__global__ void __launch_bounds__(kThreads) project_kernel(const BatchDev *__restrict__ B) {
    __shared__ int32_t s_pre[kMaxBatch * kMaxScans + 1];   // point-chunk prefix, searched per work item
    __shared__ ProjSeg s_seg[kMaxBatch * kMaxScans];
    const int nseg = B->n_frames * kMaxScans;
    for (int i = threadIdx.x; i <= nseg; i += kThreads) s_pre[i] = B->pt_pre[i];
    for (int i = threadIdx.x; i < nseg; i += kThreads) {
        // a scan slot past the frame's num_scans has no chunks and is never read
        const FrameDev &F = B->f[i / kMaxScans];
        const int sc = i % kMaxScans;
        const ScanDev &S = F.scans[sc];
        ProjSeg &D = s_seg[i];
#pragma unroll
        for (int e = 0; e < 12; ++e) D.M[e] = S.M[e];
        D.fx = F.fx;
        D.fy = F.fy;
        D.cx = F.cx;
        D.cy = F.cy;
        D.w = (float)F.W;
        D.h = (float)F.H;
        D.xyz = S.xyz;
        D.zbuf = F.zbuf_raw;
        D.motion = sc != F.newest_scan ? F.motion : nullptr;
        D.count = S.count;
        D.zpitch = F.zpitch;
        D.W = F.W;
        D.stride_floats = S.stride_floats;
    }
    __syncthreads();
    const int total = s_pre[nseg];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int seg = find_segment(s_pre, nseg, item);
        const ProjSeg &C = s_seg[seg];
        const int64_t p0 = (int64_t)(item - s_pre[seg]) * kPtsPerChunk + (int64_t)threadIdx.x * kPtsPerThread;
        const int64_t count = C.count;
        if (p0 >= count) continue;
        if (C.stride_floats == 3) {
            if (p0 + kPtsPerThread <= count) {
                // kPtsPerThread packed points = 3 kPtsPerThread / 4 aligned float4 (base 16-byte
                // aligned, p0 % 4 == 0), all loaded before any is used
                const float4 *q = reinterpret_cast<const float4 *>(C.xyz + p0 * 3);
                float v[3 * kPtsPerThread];
#pragma unroll
                for (int k = 0; k < 3 * kPtsPerThread / 4; ++k) {
                    const float4 a = __ldg(q + k);
                    v[4 * k] = a.x; v[4 * k + 1] = a.y; v[4 * k + 2] = a.z; v[4 * k + 3] = a.w;
                }
#pragma unroll
                for (int k = 0; k < kPtsPerThread; ++k) project_one(C, v[3 * k], v[3 * k + 1], v[3 * k + 2]);
            } else {
                const float *xyz = C.xyz;
                for (int64_t p = p0; p < count; ++p)
                    project_one(C, __ldg(xyz + 3 * p), __ldg(xyz + 3 * p + 1), __ldg(xyz + 3 * p + 2));
            }
        } else {
            const float4 *q = reinterpret_cast<const float4 *>(C.xyz) + p0;
            const int n = (int)(count - p0 < kPtsPerThread ? count - p0 : kPtsPerThread);
            float4 a[kPtsPerThread];
#pragma unroll
            for (int k = 0; k < kPtsPerThread; ++k)
                if (k < n) a[k] = __ldg(q + k);
#pragma unroll
            for (int k = 0; k < kPtsPerThread; ++k)
                if (k < n) project_one(C, a[k].x, a[k].y, a[k].z);
        }
    }
}

__global__ void fill_empty_kernel(uint32_t *__restrict__ p, uint64_t n) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = kEmpty;
}

cudaError_t launch_fill_empty(uint32_t *p, uint64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = (n + kThreads - 1) / kThreads;
    fill_empty_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), kThreads, 0, s>>>(p, n);
    return cudaGetLastError();
}

cudaError_t launch_prep(const BatchDev *b, int grid, cudaStream_t s) {
    prep_kernel<<<grid, kThreads, 0, s>>>(const_cast<BatchDev *>(b));
    return cudaGetLastError();
}

cudaError_t launch_project(const BatchDev *b, int grid, cudaStream_t s) {
    project_kernel<<<grid, kThreads, 0, s>>>(b);
    return cudaGetLastError();
}

int occupancy_points(KernelId k) {
    int n = 0;
    if (k == K_PREP) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, prep_kernel, kThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, project_kernel, kThreads, 0);
    return n > 0 ? n : 1;
}

}  // namespace dz
