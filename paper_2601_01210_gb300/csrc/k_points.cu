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
    // the batch's clear prefix and each frame's z-buffer in shared memory: a work item then starts
    // its stores without a chain of dependent global loads
    __shared__ int32_t s_pre[kMaxBatch + 1];
    __shared__ uint32_t *s_z[kMaxBatch];
    __shared__ int64_t s_n[kMaxBatch];
    const int nf = B->n_frames;
    for (int i = threadIdx.x; i <= nf; i += kThreads) s_pre[i] = B->zb_pre[i];
    for (int i = threadIdx.x; i < nf; i += kThreads) {
        s_z[i] = B->f[i].zbuf_raw;
        s_n[i] = (int64_t)B->f[i].zpitch * B->f[i].H;
    }
    // the TMA filters' tile flags (each frame's block of both stages) and tile counters start the
    // batch cleared; the producers (pooling, first filter) and the mark kernel set the flags
    if (B->tl_on) {
        if (blockIdx.x == 0 && threadIdx.x == 0) B->tl_next[0] = B->tl_next[1] = 0;   // the filters' tile counters
        for (int f = 0; f < nf; ++f) {
            int32_t *const fl = B->f[f].tflags[0];
            const int n = B->f[f].ntflags;
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
    __syncthreads();
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
// The camera of a frame in registers: read once per work item (an atomic on the z-buffer could
// alias the frame descriptor, so reading it per point would mean a reload after every atomic).
struct ProjCam {
    float fx, fy, cx, cy, w, h;
    int W;
    int64_t zpitch;
    const uint8_t *motion;   // NULL unless afterimage removal applies to this scan
};

__device__ __forceinline__ void project_one(const float (&M)[12], float x, float y, float z, const ProjCam &C,
                                            uint32_t *zbuf) {
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
    atomicMin(zbuf + (int64_t)j * C.zpitch + i, __float_as_uint(zc));
}

__global__ void __launch_bounds__(kThreads) project_kernel(const BatchDev *__restrict__ B) {
    __shared__ int32_t s_pre[kMaxBatch * kMaxScans + 1];   // point-chunk prefix, searched per work item
    const int nseg = B->n_frames * kMaxScans;
    for (int i = threadIdx.x; i <= nseg; i += kThreads) s_pre[i] = B->pt_pre[i];
    __syncthreads();
    const int total = s_pre[nseg];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int seg = find_segment(s_pre, nseg, item);
        const FrameDev &F = B->f[seg / kMaxScans];
        const ScanDev &S = F.scans[seg % kMaxScans];
        float M[12];
#pragma unroll
        for (int e = 0; e < 12; ++e) M[e] = S.M[e];
        const int64_t p0 = (int64_t)(item - s_pre[seg]) * kPtsPerChunk + (int64_t)threadIdx.x * kPtsPerThread;
        if (p0 >= S.count) continue;
        uint32_t *zbuf = F.zbuf_raw;
        const bool old_scan = (seg % kMaxScans) != F.newest_scan;
        const ProjCam C{F.fx, F.fy, F.cx, F.cy, (float)F.W, (float)F.H, F.W, F.zpitch, old_scan ? F.motion : nullptr};
        const int64_t count = S.count;
        if (S.stride_floats == 3) {
            if (p0 + kPtsPerThread <= S.count) {
                // kPtsPerThread packed points = 3 kPtsPerThread / 4 aligned float4 (base 16-byte
                // aligned, p0 % 4 == 0), all loaded before any is used
                const float4 *q = reinterpret_cast<const float4 *>(S.xyz + p0 * 3);
                float v[3 * kPtsPerThread];
#pragma unroll
                for (int k = 0; k < 3 * kPtsPerThread / 4; ++k) {
                    const float4 a = __ldg(q + k);
                    v[4 * k] = a.x; v[4 * k + 1] = a.y; v[4 * k + 2] = a.z; v[4 * k + 3] = a.w;
                }
#pragma unroll
                for (int k = 0; k < kPtsPerThread; ++k) project_one(M, v[3 * k], v[3 * k + 1], v[3 * k + 2], C, zbuf);
            } else {
                const float *xyz = S.xyz;
                for (int64_t p = p0; p < count; ++p)
                    project_one(M, __ldg(xyz + 3 * p), __ldg(xyz + 3 * p + 1), __ldg(xyz + 3 * p + 2), C, zbuf);
            }
        } else {
            const float4 *q = reinterpret_cast<const float4 *>(S.xyz) + p0;
            const int n = (int)(count - p0 < kPtsPerThread ? count - p0 : kPtsPerThread);
            float4 a[kPtsPerThread];
#pragma unroll
            for (int k = 0; k < kPtsPerThread; ++k)
                if (k < n) a[k] = __ldg(q + k);
#pragma unroll
            for (int k = 0; k < kPtsPerThread; ++k)
                if (k < n) project_one(M, a[k].x, a[k].y, a[k].z, C, zbuf);
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
