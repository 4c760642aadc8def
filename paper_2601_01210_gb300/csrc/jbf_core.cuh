// Joint bilateral filter kernel (Eq. (1)-(4)), gather form, FP32.
//
// For output pixel p and every in-image neighbour q with
// max(|qx - px|, |qy - py|) <= R (the square window of Algorithm 1):
//   arg(p, q) = -log2(e) (||I(q) - I(p)||^2 / (2 sigma_c^2) + |q - p|^2 / (2 sigma_p^2))
//   out(p)    = sum_q beta_d(q) 2^arg / sum_q beta(q) 2^arg
// where beta is the observation weight of q (mask, or block count after
// pooling) and beta_d the matching depth sum. Algorithm 1 computes the same
// sums by scattering each source's weighted depth to its neighbours (the
// weights are symmetric in p and q), which on a GPU means atomics or a
// materialised (2R+1)^2 weight tensor; the gather form needs neither.
//
// Layout: a CTA owns a TW x TH output tile (TW = 32 = one warp across, TH =
// 8 warps x KP rows). The tile plus an R-pixel halo is staged in shared
// memory as float4 (r, g, b, beta) plus float beta_d. Thread (lane, warp)
// owns the KP pixels of column lane, rows warp*KP .. warp*KP+KP-1, and walks
// the KP + 2R staged rows once: each staged neighbour is loaded once per
// column offset and reused by all KP pixels whose window holds it, so shared
// memory traffic is (KP + 2R)(2R + 1) loads for KP (2R + 1)^2 taps.
//
// Range: the plain 2^arg underflows in FP32 when every observed neighbour is
// far in colour (arg < -126). Pixels whose weight sum falls below 2^-60 are
// recomputed with every exponent shifted by the largest arg of the window,
// which is the same quotient (the common factor cancels) with a weight sum
// >= 1. The validity of p (some neighbour observed) is an integer decision
// made from the staged beta, independent of the weights.
#pragma once

#include "desc.cuh"

namespace dz {

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

enum { JBF_SINGLE = 0, JBF_COARSE = 1, JBF_UP = 2 };

template <int STAGE>
__device__ __forceinline__ void grid_size(const FrameDev &F, int &gw, int &gh) {
    if (STAGE == JBF_COARSE) { gw = F.Wc; gh = F.Hc; }
    else { gw = F.W; gh = F.H; }
}

// Stage input at grid pixel (gx, gy), inside the grid.
template <int STAGE>
__device__ __forceinline__ void load_src(const FrameDev &F, const StageArgs &a, int gx, int gy, float4 &g, float &bd) {
    if (STAGE == JBF_COARSE) {
        const int64_t o = (int64_t)gy * F.cpitch + gx;
        g = F.cguide[o];                      // mean r, g, b and count
        bd = F.cssum[o];
    } else {
        const uint8_t *c = F.rgb + (int64_t)gy * F.rgb_pitch + 3 * gx;
        g.x = (float)c[0]; g.y = (float)c[1]; g.z = (float)c[2];
        if (STAGE == JBF_SINGLE) {
            const uint32_t z = F.zbuf[(int64_t)gy * F.zpitch + gx];
            g.w = z != kEmpty ? 1.0f : 0.0f;
            bd = z != kEmpty ? __uint_as_float(z) : 0.0f;
        } else {
            const float2 s = F.s1[(int64_t)(gy / a.pool) * F.cpitch + gx / a.pool];
            g.w = s.y;
            bd = s.y > 0.0f ? s.x : 0.0f;
            if (a.override_sparse) {
                const uint32_t z = F.zbuf[(int64_t)gy * F.zpitch + gx];
                if (z != kEmpty) { g.w = 1.0f; bd = __uint_as_float(z); }
            }
        }
    }
}

// Shifted recomputation of one pixel (rare: all observed neighbours far in colour).
template <int R, int SW>
__device__ __noinline__ float jbf_shifted(const float4 *sG, const float *sD, int row0, int col0, float cr, float cg,
                                          float cb, float kc, float kp) {
    float amax = -__int_as_float(0x7F800000);
    for (int dy = 0; dy <= 2 * R; ++dy)
        for (int dx = 0; dx <= 2 * R; ++dx) {
            const float4 q = sG[(row0 + dy) * SW + col0 + dx];
            if (q.w > 0.0f) {
                const float dr = q.x - cr, dg = q.y - cg, db = q.z - cb;
                const float n2 = fmaf(dr, dr, fmaf(dg, dg, db * db));
                const float s2 = (float)((dx - R) * (dx - R) + (dy - R) * (dy - R));
                amax = fmaxf(amax, fmaf(n2, -kc, -s2 * kp));
            }
        }
    float num = 0.0f, den = 0.0f;
    for (int dy = 0; dy <= 2 * R; ++dy)
        for (int dx = 0; dx <= 2 * R; ++dx) {
            const int o = (row0 + dy) * SW + col0 + dx;
            const float4 q = sG[o];
            if (q.w > 0.0f) {
                const float dr = q.x - cr, dg = q.y - cg, db = q.z - cb;
                const float n2 = fmaf(dr, dr, fmaf(dg, dg, db * db));
                const float s2 = (float)((dx - R) * (dx - R) + (dy - R) * (dy - R));
                const float w = ex2_approx(fmaf(n2, -kc, -s2 * kp) - amax);
                num = fmaf(w, sD[o], num);
                den = fmaf(w, q.w, den);
            }
        }
    return num / den;
}

template <int STAGE, int R, int KP>
__global__ void __launch_bounds__(256) jbf_kernel(const BatchDev *__restrict__ B, const StageArgs a) {
    constexpr int TW = 32, NW = 8, TH = NW * KP;
    constexpr int SW = TW + 2 * R, SH = TH + 2 * R;
    constexpr int T = 2 * R + 1;
    __shared__ float4 sG[SH * SW];
    __shared__ float sD[SH * SW];
    __shared__ uint8_t sH[SH * TW];

    const int32_t *pre = STAGE == JBF_UP ? B->t2_pre : B->t1_pre;
    const int nf = B->n_frames;
    const int total = pre[nf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int fi = find_segment(pre, nf, item);
        const FrameDev &F = B->f[fi];
        int gw, gh;
        grid_size<STAGE>(F, gw, gh);
        const int tiles_x = (gw + TW - 1) / TW;
        const int t = item - pre[fi];
        const int x0 = (t % tiles_x) * TW, y0 = (t / tiles_x) * TH;

        __syncthreads();   // the previous tile's readers are done
        for (int i = threadIdx.x; i < SH * SW; i += 256) {
            const int sy = i / SW, sx = i - sy * SW;
            const int gx = x0 - R + sx, gy = y0 - R + sy;
            float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
            float bd = 0.0f;
            if (gx >= 0 && gx < gw && gy >= 0 && gy < gh) load_src<STAGE>(F, a, gx, gy, g, bd);
            sG[i] = g;
            sD[i] = bd;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < SH * TW; i += 256) {
            const int sy = i / TW, sx = i - sy * TW;
            bool any = false;
#pragma unroll
            for (int dx = 0; dx < T; ++dx) any |= sG[sy * SW + sx + dx].w > 0.0f;
            sH[i] = any;
        }
        __syncthreads();

        const int rbase = warp * KP;        // staged row of the first output's window top
        float cr[KP], cg[KP], cb[KP], num[KP], den[KP];
        bool val[KP];
        bool any_val = false;
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const float4 c = sG[(rbase + k + R) * SW + lane + R];
            cr[k] = c.x; cg[k] = c.y; cb[k] = c.z;
            num[k] = 0.0f; den[k] = 0.0f;
            bool v = false;
#pragma unroll
            for (int dy = 0; dy < T; ++dy) v |= sH[(rbase + k + dy) * TW + lane] != 0;
            val[k] = v;
            any_val |= v;
        }
        if (__any_sync(0xffffffffu, any_val)) {
            const float kc = a.kc;
#pragma unroll
            for (int iy = 0; iy < KP + 2 * R; ++iy) {
#pragma unroll
                for (int dx = 0; dx < T; ++dx) {
                    const int o = (rbase + iy) * SW + lane + dx;
                    const float4 q = sG[o];
                    const float qd = sD[o];
#pragma unroll
                    for (int k = 0; k < KP; ++k) {
                        const int dy = iy - k;
                        if (dy >= 0 && dy < T) {
                            const float dr = q.x - cr[k], dg = q.y - cg[k], db = q.z - cb[k];
                            const float n2 = fmaf(dr, dr, fmaf(dg, dg, db * db));
                            const float w = ex2_approx(fmaf(n2, -kc, a.sp[dy * (2 * kMaxR + 1) + dx]));
                            num[k] = fmaf(w, qd, num[k]);
                            den[k] = fmaf(w, q.w, den[k]);
                        }
                    }
                }
            }
        }
        const int x = x0 + lane;
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const int y = y0 + rbase + k;
            float out = 0.0f;
            if (val[k]) {
                if (den[k] >= 0x1p-60f) out = __fdividef(num[k], den[k]);
                else out = jbf_shifted<R, SW>(sG, sD, rbase + k, lane, cr[k], cg[k], cb[k], a.kc, a.kp);
            }
            if (x < gw && y < gh) {
                const int64_t o = (int64_t)y * gw + x;
                if (STAGE == JBF_COARSE) {
                    F.s1[(int64_t)y * F.cpitch + x] = make_float2(out, val[k] ? 1.0f : 0.0f);
                    if (F.out_coarse) F.out_coarse[o] = out;
                    if (F.out_coarse_valid) F.out_coarse_valid[o] = val[k];
                } else {
                    F.flt_depth[o] = out;
                    F.flt_valid[o] = val[k];
                }
            }
        }
        if (STAGE == JBF_COARSE && B->tl_th[1] > 0) {   // flag the second-stage tiles the valid pixels reach
            uint32_t cols = 0u;
            int kf = KP, kl = -1;
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const uint32_t m = __ballot_sync(0xffffffffu, val[k] && x < gw && y0 + rbase + k < gh);
                cols |= m;
                if (m) {
                    kf = min(kf, k);
                    kl = k;
                }
            }
            if (cols)
                mark_reach(F.tflags[1], B->tl_tw[1], B->tl_th[1], B->tl_r[1], a.pool, F.W, F.H,
                           x0 + __ffs(cols) - 1, x0 + 31 - __clz(cols), y0 + rbase + kf, y0 + rbase + kl, lane);
        }
    }
}

}  // namespace dz
