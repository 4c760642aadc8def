// Pooling to the coarse grid of the two-stage filter (Sec. 5) and
// back-projection of the dense depth to coloured points with a deterministic
// row-major compaction (Sec. 2: coloured point clouds in a common frame).
#include "desc.cuh"

namespace dz {

// ---------------------------------------------------------------------------
// pool: coarse pixel (I, J) covers the full-resolution block
// [fI, fI+f) x [fJ, fJ+f) clipped to the image. It gets the sum and count of
// the observed depths (average pooling of D*B and B, with the common divisor
// dropped because it cancels in the filter's ratio) and the mean RGB of the
// block's in-image pixels as the coarse guide. Sums run in row-major order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) pool_kernel(const BatchDev *__restrict__ B, int f) {
    const int nf = B->n_frames;
    const int total = B->pool_pre[nf];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int fi = find_segment(B->pool_pre, nf, item);
        const FrameDev &F = B->f[fi];
        const int idx = (item - B->pool_pre[fi]) * kPoolPerChunk + threadIdx.x;
        if (idx >= F.Wc * F.Hc) continue;
        const int I = idx % F.Wc, J = idx / F.Wc;
        const int x0 = I * f, y0 = J * f;
        const int x1 = min(x0 + f, F.W), y1 = min(y0 + f, F.H);
        float s = 0.0f, cnt = 0.0f, r = 0.0f, g = 0.0f, b = 0.0f;
        for (int y = y0; y < y1; ++y) {
            const uint32_t *zr = F.zbuf + (int64_t)y * F.zpitch;
            const uint8_t *cr = F.rgb + (int64_t)y * F.rgb_pitch;
            for (int x = x0; x < x1; ++x) {
                const uint32_t z = zr[x];
                if (z != kEmpty) {
                    s = __fadd_rn(s, __uint_as_float(z));
                    cnt += 1.0f;
                }
                r += (float)cr[3 * x];
                g += (float)cr[3 * x + 1];
                b += (float)cr[3 * x + 2];
            }
        }
        const float npx = (float)((x1 - x0) * (y1 - y0));
        const int64_t o = (int64_t)J * F.cpitch + I;
        F.cguide[o] = make_float4(__fdiv_rn(r, npx), __fdiv_rn(g, npx), __fdiv_rn(b, npx), cnt);
        F.cssum[o] = s;
    }
}

cudaError_t launch_pool(const BatchDev *b, int pool, int grid, cudaStream_t s) {
    pool_kernel<<<grid, kThreads, 0, s>>>(b, pool);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// back-projection with deterministic compaction.
// A chunk is 4096 consecutive pixels in row-major order; warp w of the block
// owns pixels [512 w, 512 w + 512) of it, 128 per step, 4 per lane.
// bp_count writes each chunk's valid count; bp_write sums the counts of the
// preceding chunks of its frame, scans inside the chunk and writes
//   (x, y, z) = cam_to_world * ((u + 1/2 - cx) Z / fx, (v + 1/2 - cy) Z / fy, Z)
// with the pixel colour packed r | g << 8 | b << 16 | 255 << 24.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t valid4(const uint8_t *valid, int64_t p, int64_t n) {
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (p + k < n && valid[p + k]) m |= 1u << k;
    return m;
}

__global__ void __launch_bounds__(kThreads) bp_count_kernel(const BatchDev *__restrict__ B) {
    __shared__ uint32_t wsum[kThreads / 32];
    const int nf = B->n_frames;
    const int total = B->bp_pre[nf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int fi = find_segment(B->bp_pre, nf, item);
        const FrameDev &F = B->f[fi];
        const int c = item - B->bp_pre[fi];
        const int64_t n = (int64_t)F.W * F.H;
        const int64_t base = (int64_t)c * kBpChunk + warp * 512;
        uint32_t cnt = 0;
#pragma unroll
        for (int it = 0; it < 4; ++it) cnt += __popc(valid4(F.out_valid, base + it * 128 + lane * 4, n));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        __syncthreads();
        if (lane == 0) wsum[warp] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < kThreads / 32; ++w) t += wsum[w];
            F.chunk_cnt[c] = t;
        }
    }
}

__global__ void __launch_bounds__(kThreads) bp_write_kernel(const BatchDev *__restrict__ B) {
    __shared__ uint32_t wsum[kThreads / 32];
    __shared__ int64_t red[kThreads / 32];
    __shared__ int64_t chunk_base;
    const int nf = B->n_frames;
    const int total = B->bp_pre[nf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int fi = find_segment(B->bp_pre, nf, item);
        const FrameDev &F = B->f[fi];
        const int c = item - B->bp_pre[fi];
        const int64_t n = (int64_t)F.W * F.H;
        // exclusive prefix over the frame's earlier chunks
        int64_t part = 0;
        for (int k = threadIdx.x; k < c; k += kThreads) part += F.chunk_cnt[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        __syncthreads();
        if (lane == 0) red[warp] = part;
        // per-warp counts of this chunk
        const int64_t base = (int64_t)c * kBpChunk + warp * 512;
        uint32_t m[4], wc = 0;
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            m[it] = valid4(F.out_valid, base + it * 128 + lane * 4, n);
            wc += __popc(m[it]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wc += __shfl_xor_sync(0xffffffffu, wc, o);
        if (lane == 0) wsum[warp] = wc;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t t = 0;
            for (int w = 0; w < kThreads / 32; ++w) t += red[w];
            chunk_base = t;
            int64_t all = 0;
            for (int w = 0; w < kThreads / 32; ++w) all += wsum[w];
            if (c == F.n_bp_chunks - 1) *F.points_n = t + all;
        }
        __syncthreads();
        int64_t off = chunk_base;
        for (int w = 0; w < warp; ++w) off += wsum[w];
        const float *c2w = F.c2w32;
        const float r00 = c2w[0], r01 = c2w[1], r02 = c2w[2], t0 = c2w[3];
        const float r10 = c2w[4], r11 = c2w[5], r12 = c2w[6], t1 = c2w[7];
        const float r20 = c2w[8], r21 = c2w[9], r22 = c2w[10], t2 = c2w[11];
        const float ifx = 1.0f / F.fx, ify = 1.0f / F.fy;
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            const uint32_t cnt = __popc(m[it]);
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            int64_t pos = off + (incl - cnt);
            const int64_t p0 = base + it * 128 + lane * 4;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (m[it] & (1u << k)) {
                    const int64_t p = p0 + k;
                    const int y = (int)(p / F.W), x = (int)(p - (int64_t)y * F.W);
                    const float Z = F.out_depth[p];
                    const float X = ((float)x + 0.5f - F.cx) * Z * ifx;
                    const float Y = ((float)y + 0.5f - F.cy) * Z * ify;
                    const uint8_t *col = F.rgb + (int64_t)y * F.rgb_pitch + 3 * x;
                    const uint32_t rgba = (uint32_t)col[0] | ((uint32_t)col[1] << 8) | ((uint32_t)col[2] << 16) | 0xFF000000u;
                    if (pos < F.points_cap)
                        F.out_points[pos] = make_float4(fmaf(r00, X, fmaf(r01, Y, fmaf(r02, Z, t0))),
                                                        fmaf(r10, X, fmaf(r11, Y, fmaf(r12, Z, t1))),
                                                        fmaf(r20, X, fmaf(r21, Y, fmaf(r22, Z, t2))),
                                                        __uint_as_float(rgba));
                    ++pos;
                }
            }
            off += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

cudaError_t launch_bp_count(const BatchDev *b, int grid, cudaStream_t s) {
    bp_count_kernel<<<grid, kThreads, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_bp_write(const BatchDev *b, int grid, cudaStream_t s) {
    bp_write_kernel<<<grid, kThreads, 0, s>>>(b);
    return cudaGetLastError();
}

int occupancy_pool_bp(KernelId k) {
    int n = 0;
    if (k == K_POOL) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pool_kernel, kThreads, 0);
    else if (k == K_BP_COUNT) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bp_count_kernel, kThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bp_write_kernel, kThreads, 0);
    return n > 0 ? n : 1;
}

}  // namespace dz
