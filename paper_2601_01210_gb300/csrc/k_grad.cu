// Gradient of the mean squared depth error with respect to the filter's
// sigmas (Sec. 4: when dense ground truth exists, the Gaussian variances can
// be optimised by backpropagation).
//
// For one stage, with e = ||dI||^2 / (2 sc^2) + ||dx||^2 / (2 sp^2) and
// w = exp(-e): dw/dsc = w ||dI||^2 / sc^3 and dw/dsp = w ||dx||^2 / sp^3, and
// for out = sum w beta_d / sum w beta,
//   d out / d theta = (sum dw/dtheta beta_d - out sum dw/dtheta beta) / sum w beta.
// In the two-stage form the second stage's input depth is the restored
// first-stage result, so d out2 / d theta1 = sum w2 beta2 d out1(c(q)) / d theta1
// / sum w2 beta2 with c(q) the pooled pixel under q. Every pixel's window is
// evaluated with exponents shifted by their maximum (the factor cancels).
// Everything on the device is FP32: per-pixel terms, each thread's running
// sums, a pairwise (shuffle-tree) sum per warp and per block; every block
// writes one row of partial sums, which the host adds in FP64.
#include "desc.cuh"
#include "grad.h"

namespace dz {

namespace {

__device__ __forceinline__ float ex2f(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct Acc {
    float N = 0, Wt = 0, Np = 0, Wp = 0, Nc = 0, Wc = 0, Q0 = 0, Q1 = 0;
};

// One output pixel. fetch(q, beta, beta_d, dq0, dq1, r, g, b) -> observed.
template <typename Fetch>
__device__ __forceinline__ bool grad_pixel(int px, int py, int gw, int gh, int R, float cr, float cg, float cb,
                                           const GradStage &s, Fetch fetch, float &out, float dd[4]) {
    const float kc = s.kc, kp = s.kp;   // log2(e) / (2 sigma^2)
    float amax = -__int_as_float(0x7F800000);
    bool any = false;
    for (int qy = py - R; qy <= py + R; ++qy) {
        if (qy < 0 || qy >= gh) continue;
        for (int qx = px - R; qx <= px + R; ++qx) {
            if (qx < 0 || qx >= gw) continue;
            float be, bd, d0, d1, r, g, b;
            if (!fetch(qx, qy, be, bd, d0, d1, r, g, b)) continue;
            const float n2 = (r - cr) * (r - cr) + (g - cg) * (g - cg) + (b - cb) * (b - cb);
            const float s2 = (float)((qx - px) * (qx - px) + (qy - py) * (qy - py));
            amax = fmaxf(amax, -(n2 * kc + s2 * kp));
            any = true;
        }
    }
    if (!any) return false;
    Acc a;
    for (int qy = py - R; qy <= py + R; ++qy) {
        if (qy < 0 || qy >= gh) continue;
        for (int qx = px - R; qx <= px + R; ++qx) {
            if (qx < 0 || qx >= gw) continue;
            float be, bd, d0, d1, r, g, b;
            if (!fetch(qx, qy, be, bd, d0, d1, r, g, b)) continue;
            const float n2 = (r - cr) * (r - cr) + (g - cg) * (g - cg) + (b - cb) * (b - cb);
            const float s2 = (float)((qx - px) * (qx - px) + (qy - py) * (qy - py));
            const float w = ex2f(-(n2 * kc + s2 * kp) - amax);
            const float wp = w * s2 * s.inv_sp3, wc = w * n2 * s.inv_sc3;
            a.N = fmaf(w, bd, a.N);
            a.Wt = fmaf(w, be, a.Wt);
            a.Np = fmaf(wp, bd, a.Np);
            a.Wp = fmaf(wp, be, a.Wp);
            a.Nc = fmaf(wc, bd, a.Nc);
            a.Wc = fmaf(wc, be, a.Wc);
            a.Q0 = fmaf(w, d0, a.Q0);
            a.Q1 = fmaf(w, d1, a.Q1);
        }
    }
    out = a.N / a.Wt;
    dd[0] = (a.Np - out * a.Wp) / a.Wt;
    dd[1] = (a.Nc - out * a.Wc) / a.Wt;
    dd[2] = a.Q0 / a.Wt;
    dd[3] = a.Q1 / a.Wt;
    return true;
}

}  // namespace

// First of two stages: one thread per pooled pixel; writes s1 (depth, valid)
// and g1 (d depth / d sp1, d depth / d sc1).
__global__ void __launch_bounds__(kThreads) grad_coarse_kernel(const BatchDev *__restrict__ B, const GradArgs ga) {
    const int nf = B->n_frames;
    const int total = B->pool_pre[nf];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int fi = find_segment(B->pool_pre, nf, item);
        const FrameDev &F = B->f[fi];
        const int idx = (item - B->pool_pre[fi]) * kPoolPerChunk + threadIdx.x;
        if (idx >= F.Wc * F.Hc) continue;
        const int x = idx % F.Wc, y = idx / F.Wc;
        const float4 c = F.cguide[(int64_t)y * F.cpitch + x];
        auto fetch = [&](int qx, int qy, float &be, float &bd, float &d0, float &d1, float &r, float &g, float &b) {
            const int64_t o = (int64_t)qy * F.cpitch + qx;
            const float4 q = F.cguide[o];
            be = q.w;
            bd = F.cssum[o];
            d0 = d1 = 0.0f;
            r = q.x; g = q.y; b = q.z;
            return be > 0.0f;
        };
        float out = 0.0f, dd[4] = {0, 0, 0, 0};
        const bool v = grad_pixel(x, y, F.Wc, F.Hc, ga.s[0].radius, c.x, c.y, c.z, ga.s[0], fetch, out, dd);
        F.s1[(int64_t)y * F.cpitch + x] = make_float2(v ? out : 0.0f, v ? 1.0f : 0.0f);
        F.g1[(int64_t)y * F.cpitch + x] = make_float2(v ? dd[0] : 0.0f, v ? dd[1] : 0.0f);
    }
}

// Full-resolution stage (the second of two, or the only one): per pixel with
// ground truth, the squared error and its gradient; per-block partial sums.
__global__ void __launch_bounds__(kThreads) grad_full_kernel(const BatchDev *__restrict__ B, const GradArgs ga,
                                                             const float *__restrict__ gt, float *__restrict__ part) {
    __shared__ float red[kThreads / 32][6];
    float acc[6] = {0, 0, 0, 0, 0, 0};   // loss, n, d/d(sp1, sc1, sp2, sc2) -- or (sp, sc, 0, 0) single
    const int nf = B->n_frames;
    const int total = B->px_pre[nf];
    const GradStage &S = ga.s[ga.two_stage ? 1 : 0];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int fi = find_segment(B->px_pre, nf, item);
        const FrameDev &F = B->f[fi];
        const int64_t n = (int64_t)F.W * F.H;
        const int64_t p0 = (int64_t)(item - B->px_pre[fi]) * kPxChunk + threadIdx.x;
        for (int k = 0; k < kPxChunk / kThreads; ++k) {
            const int64_t p = p0 + k * kThreads;
            if (p >= n) continue;
            const float t = gt[p];
            if (!(t > 0.0f)) continue;
            const int y = (int)(p / F.W), x = (int)(p - (int64_t)y * F.W);
            const uint8_t *cp = F.rgb + (int64_t)y * F.rgb_pitch + 3 * x;
            float out = 0.0f, dd[4] = {0, 0, 0, 0};
            bool v;
            if (ga.two_stage) {
                auto fetch = [&](int qx, int qy, float &be, float &bd, float &d0, float &d1, float &r, float &g,
                                 float &b) {
                    const int64_t c = (int64_t)(qy / ga.pool) * F.cpitch + qx / ga.pool;
                    const float2 s1 = F.s1[c];
                    if (!(s1.y > 0.0f)) return false;
                    const float2 g1 = F.g1[c];
                    const uint8_t *q = F.rgb + (int64_t)qy * F.rgb_pitch + 3 * qx;
                    be = 1.0f;
                    bd = s1.x;
                    d0 = g1.x;
                    d1 = g1.y;
                    r = (float)q[0]; g = (float)q[1]; b = (float)q[2];
                    return true;
                };
                v = grad_pixel(x, y, F.W, F.H, S.radius, (float)cp[0], (float)cp[1], (float)cp[2], S, fetch, out, dd);
            } else {
                auto fetch = [&](int qx, int qy, float &be, float &bd, float &d0, float &d1, float &r, float &g,
                                 float &b) {
                    const uint32_t z = F.zbuf[(int64_t)qy * F.zpitch + qx];
                    if (z == kEmpty) return false;
                    const uint8_t *q = F.rgb + (int64_t)qy * F.rgb_pitch + 3 * qx;
                    be = 1.0f;
                    bd = __uint_as_float(z);
                    d0 = d1 = 0.0f;
                    r = (float)q[0]; g = (float)q[1]; b = (float)q[2];
                    return true;
                };
                v = grad_pixel(x, y, F.W, F.H, S.radius, (float)cp[0], (float)cp[1], (float)cp[2], S, fetch, out, dd);
            }
            if (!v) continue;
            const float e = out - t;
            acc[0] = fmaf(e, e, acc[0]);
            acc[1] += 1.0f;
            if (ga.two_stage) {   // (sp1, sc1) come through the input, (sp2, sc2) from this stage
                acc[2] = fmaf(2.0f * e, dd[2], acc[2]);
                acc[3] = fmaf(2.0f * e, dd[3], acc[3]);
                acc[4] = fmaf(2.0f * e, dd[0], acc[4]);
                acc[5] = fmaf(2.0f * e, dd[1], acc[5]);
            } else {
                acc[2] = fmaf(2.0f * e, dd[0], acc[2]);
                acc[3] = fmaf(2.0f * e, dd[1], acc[3]);
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 6; ++j)
        for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
    if (lane == 0)
        for (int j = 0; j < 6; ++j) red[warp][j] = acc[j];
    __syncthreads();
    if (threadIdx.x < 6) {   // pairwise over the block's warps
        float v[kThreads / 32];
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) v[w] = red[w][threadIdx.x];
#pragma unroll
        for (int h = kThreads / 64; h > 0; h >>= 1)
#pragma unroll
            for (int w = 0; w < h; ++w) v[w] += v[w + h];
        part[(int64_t)blockIdx.x * 6 + threadIdx.x] = v[0];
    }
}

cudaError_t launch_grad(const BatchDev *b, const GradArgs &ga, const float *gt, float *part, int grid,
                        cudaStream_t s) {
    if (ga.two_stage) {
        grad_coarse_kernel<<<grid, kThreads, 0, s>>>(b, ga);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    grad_full_kernel<<<grid, kThreads, 0, s>>>(b, ga, gt, part);
    return cudaGetLastError();
}

}  // namespace dz
