// Preprocessing of the merged scans (Sec. 4.1) and post-filtering of the dense
// depth (Sec. 5), each off unless its parameter is set:
//
//   motion_kernel   afterimages: pixels whose RGB moved between consecutive
//                   frames (squared distance above tau^2, integers against
//                   the FP32 tau^2)
//   morph_kernel    closing of that mask: dilation, then erosion, with a
//                   square (2c+1)^2 element (outside the image: no motion for
//                   the dilation, motion for the erosion); the projection then
//                   drops points of older scans inside the mask
//   occlusion_kernel  occluded points: an observed pixel deeper than the mean
//                   observed depth of its (2 rho + 1)^2 window by more than a
//                   margin is removed. The sum is fixed to FP32 row sums over
//                   dx, added over dy, divided by the count (correctly rounded
//                   FP32 throughout), so the decision is bit-reproducible.
//   contour_kernel  contours: a valid pixel with a valid 4-neighbour whose
//                   depth differs by more than t times its own depth is dropped
//                   (FP32 on the filtered map).
#include "desc.cuh"

namespace dz {

namespace {

template <typename F>
__device__ __forceinline__ void for_px(const BatchDev *B, F &&body) {
    const int nf = B->n_frames;
    const int total = B->px_pre[nf];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int fi = find_segment(B->px_pre, nf, item);
        const FrameDev &Fr = B->f[fi];
        const int64_t n = (int64_t)Fr.W * Fr.H;
        const int64_t p0 = (int64_t)(item - B->px_pre[fi]) * kPxChunk + threadIdx.x;
#pragma unroll
        for (int k = 0; k < kPxChunk / kThreads; ++k) {
            const int64_t p = p0 + k * kThreads;
            if (p < n) body(Fr, p);
        }
    }
}

}  // namespace

__global__ void __launch_bounds__(kThreads) motion_kernel(const BatchDev *__restrict__ B, const PrepostArgs a) {
    for_px(B, [&](const FrameDev &F, int64_t p) {
        if (!F.motion) return;
        const int y = (int)(p / F.W), x = (int)(p - (int64_t)y * F.W);
        const uint8_t *c = F.rgb + (int64_t)y * F.rgb_pitch + 3 * x;
        const uint8_t *q = F.prev_rgb + (int64_t)y * F.prev_pitch + 3 * x;
        int d2 = 0;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const int d = (int)c[ch] - (int)q[ch];
            d2 += d * d;
        }
        F.motion[p] = (float)d2 > a.motion_t2;
    });
}

__global__ void __launch_bounds__(kThreads) morph_kernel(const BatchDev *__restrict__ B, const PrepostArgs a,
                                                         int dilate) {
    const int c = a.close_radius;
    for_px(B, [&](const FrameDev &F, int64_t p) {
        if (!F.motion) return;
        const uint8_t *src = dilate ? F.motion : F.motion_tmp;
        uint8_t *dst = dilate ? F.motion_tmp : F.motion;
        const int y = (int)(p / F.W), x = (int)(p - (int64_t)y * F.W);
        uint8_t m = dilate ? 0 : 1;
        for (int dy = -c; dy <= c; ++dy) {
            const int qy = y + dy;
            if (qy < 0 || qy >= F.H) continue;
            for (int dx = -c; dx <= c; ++dx) {
                const int qx = x + dx;
                if (qx < 0 || qx >= F.W) continue;
                const uint8_t v = src[(int64_t)qy * F.W + qx];
                if (dilate) m |= v;
                else m &= v;
            }
        }
        dst[p] = m;
    });
}

// Tiles of 32 x 32 output pixels; the tile plus a rho halo is staged as depth
// (0 where empty) and an observation flag, then row sums and column sums.
constexpr int kMaxOccR = 16;
__global__ void __launch_bounds__(kThreads) occlusion_kernel(const BatchDev *__restrict__ B, const PrepostArgs a) {
    constexpr int T = kOccTile, S = T + 2 * kMaxOccR;
    __shared__ float sd[S * S];
    __shared__ uint8_t sc[S * S];
    __shared__ float hs[S * T];
    __shared__ int16_t hc[S * T];
    const int rho = a.occ_radius, sw = T + 2 * rho;
    const int nf = B->n_frames;
    const int total = B->oc_pre[nf];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int fi = find_segment(B->oc_pre, nf, item);
        const FrameDev &F = B->f[fi];
        const int tiles_x = (F.W + T - 1) / T;
        const int t = item - B->oc_pre[fi];
        const int x0 = (t % tiles_x) * T, y0 = (t / tiles_x) * T;
        __syncthreads();
        for (int i = threadIdx.x; i < sw * sw; i += kThreads) {
            const int sy = i / sw, sx = i - sy * sw;
            const int gx = x0 - rho + sx, gy = y0 - rho + sy;
            uint32_t z = kEmpty;
            if (gx >= 0 && gx < F.W && gy >= 0 && gy < F.H) z = F.zbuf_raw[(int64_t)gy * F.zpitch + gx];
            sd[i] = z != kEmpty ? __uint_as_float(z) : 0.0f;
            sc[i] = z != kEmpty;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < sw * T; i += kThreads) {
            const int r = i / T, x = i - r * T;
            float s = 0.0f;
            int n = 0;
            for (int dx = 0; dx <= 2 * rho; ++dx) {
                s = __fadd_rn(s, sd[r * sw + x + dx]);   // adding 0 for an empty cell changes nothing
                n += sc[r * sw + x + dx];
            }
            hs[i] = s;
            hc[i] = (int16_t)n;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < T * T; i += kThreads) {
            const int y = i / T, x = i - y * T;
            const int gx = x0 + x, gy = y0 + y;
            if (gx >= F.W || gy >= F.H) continue;
            const uint32_t z = F.zbuf_raw[(int64_t)gy * F.zpitch + gx];
            uint32_t out = z;
            if (z != kEmpty) {
                float s = 0.0f;
                int n = 0;
                for (int dy = 0; dy <= 2 * rho; ++dy) {
                    s = __fadd_rn(s, hs[(y + dy) * T + x]);
                    n += hc[(y + dy) * T + x];
                }
                const float avg = __fdiv_rn(s, (float)n);
                if (__uint_as_float(z) > __fadd_rn(avg, a.occ_margin)) out = kEmpty;
            }
            F.zbuf[(int64_t)gy * F.zpitch + gx] = out;
        }
    }
}

__global__ void __launch_bounds__(kThreads) contour_kernel(const BatchDev *__restrict__ B, const PrepostArgs a) {
    for_px(B, [&](const FrameDev &F, int64_t p) {
        const int y = (int)(p / F.W), x = (int)(p - (int64_t)y * F.W);
        const uint8_t v = F.flt_valid[p];
        const float d = F.flt_depth[p];
        bool drop = false;
        if (v) {
            const float lim = __fmul_rn(a.contour_t, d);
            const int qx[4] = {x - 1, x + 1, x, x}, qy[4] = {y, y, y - 1, y + 1};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (qx[k] < 0 || qx[k] >= F.W || qy[k] < 0 || qy[k] >= F.H) continue;
                const int64_t q = (int64_t)qy[k] * F.W + qx[k];
                if (F.flt_valid[q] && fabsf(__fadd_rn(F.flt_depth[q], -d)) > lim) drop = true;
            }
        }
        F.out_valid[p] = v && !drop;
        F.out_depth[p] = drop ? 0.0f : d;
    });
}

cudaError_t launch_motion(const BatchDev *b, const PrepostArgs &a, int grid, cudaStream_t s) {
    motion_kernel<<<grid, kThreads, 0, s>>>(b, a);
    return cudaGetLastError();
}

cudaError_t launch_morph(const BatchDev *b, const PrepostArgs &a, bool dilate, int grid, cudaStream_t s) {
    morph_kernel<<<grid, kThreads, 0, s>>>(b, a, dilate ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_occlusion(const BatchDev *b, const PrepostArgs &a, int grid, cudaStream_t s) {
    if (a.occ_radius < 1 || a.occ_radius > kMaxOccR) return cudaErrorInvalidValue;
    occlusion_kernel<<<grid, kThreads, 0, s>>>(b, a);
    return cudaGetLastError();
}

cudaError_t launch_contour(const BatchDev *b, const PrepostArgs &a, int grid, cudaStream_t s) {
    contour_kernel<<<grid, kThreads, 0, s>>>(b, a);
    return cudaGetLastError();
}

int occupancy_prepost(KernelId k) {
    int n = 0;
    if (k == K_MOTION) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, motion_kernel, kThreads, 0);
    else if (k == K_DILATE || k == K_ERODE) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, morph_kernel, kThreads, 0);
    else if (k == K_OCCLUSION) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, occlusion_kernel, kThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, contour_kernel, kThreads, 0);
    return n > 0 ? n : 1;
}

}  // namespace dz
