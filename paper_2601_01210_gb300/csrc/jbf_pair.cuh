// One tile of the joint bilateral filter (Eq. (1)-(4)) in the expanded FP32
// form, on pairs of output columns in packed two-lane FP32 arithmetic. Called
// by the TMA-staged kernel (jbf_tma.cuh) once the tile's raw boxes are in
// shared memory; the full-resolution stages only (restored first-stage result
// or z-buffer as depth, RGB bytes as guide).
//
// Expanded form (same arithmetic as the scalar one in jbf_tma.cuh): with the
// centred colours c' = c - 128 (exact in FP32), the colour term of a tap is
//   -kc |c'_p - c'_q|^2 = 2 kc c'_p . c'_q - kc |c'_p|^2 - kc |c'_q|^2,
// so the weight of neighbour q at offset (dx - R, dy - R) is
//   2^(2 kc c'_p . c'_q - kc |c'_p|^2 + ex_sy[dy]) * F_q * ex_sx[dx],
// F_q = 2^(-kc |c'_q|^2) computed once per staged neighbour (0 when q holds no
// observation), and the depth enters as G_q = F_q * depth_q. Per tap: three
// FMAs for the exponent, one ex2, one FMA each into numerator and weight sum.
//
// Column pairs: a thread owns output columns x0 + lane and x0 + 32 + lane of a
// 64-column tile, rows rbase .. rbase + KP - 1. Staged slot s of a row holds
// the records of staged columns s and s + 32 side by side, so the neighbour at
// tap dx of both pixels sits in one slot (lane + dx) and every arithmetic step
// above runs once for the two pixels as a two-lane FP32 instruction
// (__ffma2_rn / __fmul2_rn / __fadd2_rn, each lane rounded as its scalar
// counterpart): slot records are
//   sc = {r', r'', g', g''},  sb = {b', b'', F', F''},  sg = {G', G''}
// (' for the first staged column of the slot, '' for the second).
#pragma once

#include <type_traits>

#include "jbf_core.cuh"
#include "tma_common.cuh"

namespace dz {

__device__ __forceinline__ float2 f2(float lo, float hi) { return make_float2(lo, hi); }

// after_conversion() runs right after the barrier that publishes the staged records
// (the kernel's thread 0 advances its tile queue there); the caller ends the tile with
// a barrier before the staged records or the raw boxes are rewritten.
template <int SRC, int R, int KP, int NW, class AfterConversion>
__device__ __forceinline__ void pair_tile(const FrameDev &F, const StageArgs &a, int x0, int y0, int gw, int gh,
                                          const uint8_t *rgbraw, const uint8_t *rawb, uint8_t *smem,
                                          AfterConversion &&after_conversion) {
    using G = TmaGeom<SRC, R, KP, NW, FORM_EXP_PAIRS>;
    static_assert(SRC != SRC_COARSE, "paired form: full-resolution stages");
    constexpr int SP = G::SP, SH = G::SH, T = 2 * R + 1, NT = G::NT, NCONV = G::NCONV;
    constexpr uint32_t TMASK = (1u << T) - 1u;
    float4 *sc = reinterpret_cast<float4 *>(smem + G::OFF_STAGED);
    float4 *sb = sc + SH * SP;
    float2 *sg = reinterpret_cast<float2 *>(smem + G::OFF_G);
    uint32_t *obs0 = reinterpret_cast<uint32_t *>(smem + G::OFF_OBS);   // first column of each slot
    uint32_t *obs1 = obs0 + G::OBS_ONE / 4;                              // second column
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // staged position (sy, sx) <-> image pixel (x0 - R + sx, y0 - R + sy): colour bytes in the
    // raw RGB box, depth and observation in the raw first-stage box (restored by x / 3, y / 3)
    // or the raw z-buffer box
    const int cx0 = floor_div3(x0 - R) & ~1, cy0 = floor_div3(y0 - R);
    const float2 *craw = reinterpret_cast<const float2 *>(rawb);
    const uint32_t *zraw = reinterpret_cast<const uint32_t *>(rawb);
    auto rgb_at = [&](int sy, int sx) { return rgbraw + sy * G::RGB_BX + 3 * sx - 3 * R + G::RGB_LEAD; };
    // a tile whose halo lies inside the image needs no bounds checks on its staged positions
    const bool interior = x0 >= R && x0 + G::TW + R <= gw && y0 >= R && y0 + G::TH + R <= gh;
    auto depth_of = [&](int sy, int sx, float &d, auto inside) -> bool {
        const int gx = x0 - R + sx, gy = y0 - R + sy;
        if (!decltype(inside)::value && (gx < 0 || gx >= gw || gy < 0 || gy >= gh)) return false;
        if (SRC == SRC_UP) {
            const float2 c = craw[((int)((unsigned)gy / 3u) - cy0) * G::C_BX + ((int)((unsigned)gx / 3u) - cx0)];
            d = c.x;
            return c.y > 0.0f;
        }
        const uint32_t z = zraw[sy * G::Z_BX + sx - R + G::Z_LEAD];
        d = __uint_as_float(z);
        return z != kEmpty;
    };

    // ---- conversion: every thread takes slots threadIdx.x + j * NT, all raw loads first,
    // then the records; one ballot per half gives a word of each observation bitmap
    uint32_t om0 = 0u, om1 = 0u;   // bit j: first / second column of slot j observed
    float d0[NCONV], d1[NCONV];
    uint32_t r0[NCONV], g0[NCONV], b0[NCONV], r1[NCONV], g1[NCONV], b1[NCONV];
    auto load_slots = [&](auto inside) {
#pragma unroll
        for (int j = 0; j < NCONV; ++j) {
            const int i = threadIdx.x + j * NT;
            d0[j] = d1[j] = 0.0f;
            r0[j] = g0[j] = b0[j] = r1[j] = g1[j] = b1[j] = 0u;
            if (i < SH * SP) {
                const int sy = i / SP, s = i - sy * SP;
                float d = 0.0f;
                if (depth_of(sy, s, d, inside)) om0 |= 1u << j;
                d0[j] = d;
                d = 0.0f;
                if (depth_of(sy, s + 32, d, inside)) om1 |= 1u << j;
                d1[j] = d;
                const uint8_t *p = rgb_at(sy, s), *q = p + 96;
                r0[j] = p[0]; g0[j] = p[1]; b0[j] = p[2];
                r1[j] = q[0]; g1[j] = q[1]; b1[j] = q[2];
            }
        }
    };
    if (interior) load_slots(std::true_type{});
    else load_slots(std::false_type{});
    // bytes b, b' as exact floats minus 128: 2^23 + b has b in its low mantissa bits
    auto bytes2 = [](uint32_t b, uint32_t b2) {
        return __fadd2_rn(f2(__uint_as_float(0x4B000000u | b), __uint_as_float(0x4B000000u | b2)),
                          f2(-8388736.0f, -8388736.0f));
    };
    const float kc = a.kc;
#pragma unroll
    for (int j = 0; j < NCONV; ++j) {
        const int i = threadIdx.x + j * NT;
        const bool o0 = (om0 >> j) & 1u, o1 = (om1 >> j) & 1u;
        if (i < SH * SP) {
            // centred colours (exact); an unobserved record keeps its colour with F = G = 0
            const float2 r = bytes2(r0[j], r1[j]), g = bytes2(g0[j], g1[j]), b = bytes2(b0[j], b1[j]);
            const float2 e = __fmul2_rn(f2(-kc, -kc), __ffma2_rn(r, r, __ffma2_rn(g, g, __fmul2_rn(b, b))));
            const float f0 = o0 ? ex2_approx(e.x) : 0.0f, f1 = o1 ? ex2_approx(e.y) : 0.0f;
            const float2 fd = __fmul2_rn(f2(f0, f1), f2(d0[j], d1[j]));
            sc[i] = make_float4(r.x, r.y, g.x, g.y);
            sb[i] = make_float4(b.x, b.y, f0, f1);
            sg[i] = f2(o0 ? fd.x : 0.0f, o1 ? fd.y : 0.0f);   // an empty z-buffer cell holds +inf
        }
        const uint32_t w0 = __ballot_sync(0xffffffffu, o0), w1 = __ballot_sync(0xffffffffu, o1);
        if (lane == 0) {
            obs0[(threadIdx.x + j * NT) >> 5] = w0;
            obs1[(threadIdx.x + j * NT) >> 5] = w1;
        }
    }
    __syncthreads();
    after_conversion();

    // ---- validity: an output pixel is valid when its window holds an observation
    const int rbase = warp * KP;
    bool val0[KP], val1[KP];
    bool any_val = false;
    uint32_t rows_warp;   // bit iy: some lane of the warp has an observation in its window of staged row rbase + iy
    {
        uint32_t rows0 = 0u, rows1 = 0u;   // bit iy: an observation in staged row rbase + iy, slots lane .. lane + 2R
#pragma unroll
        for (int iy = 0; iy < KP + 2 * R; ++iy) {
            const int bit = (rbase + iy) * SP + lane;   // the window never leaves its row
            const uint32_t w0 = __funnelshift_r(obs0[bit >> 5], obs0[(bit >> 5) + 1], bit & 31);
            const uint32_t w1 = __funnelshift_r(obs1[bit >> 5], obs1[(bit >> 5) + 1], bit & 31);
            rows0 |= ((w0 & TMASK) != 0 ? 1u : 0u) << iy;
            rows1 |= ((w1 & TMASK) != 0 ? 1u : 0u) << iy;
        }
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            val0[k] = ((rows0 >> k) & TMASK) != 0;
            val1[k] = ((rows1 >> k) & TMASK) != 0;
            any_val |= val0[k] || val1[k];
        }
        rows_warp = __reduce_or_sync(0xffffffffu, rows0 | rows1);
    }

    // ---- taps
    float2 num[KP], den[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) num[k] = den[k] = f2(0.0f, 0.0f);
    if (__any_sync(0xffffffffu, any_val)) {
        const float kc2 = 2.0f * kc;
        float2 ar[KP], ag[KP], ab[KP], cp[KP];   // 2 kc c'_p per channel, -kc |c'_p|^2
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const int o = (rbase + k + R) * SP + lane + R;
            const float4 c = sc[o], b = sb[o];
            ar[k] = f2(kc2 * c.x, kc2 * c.y);
            ag[k] = f2(kc2 * c.z, kc2 * c.w);
            ab[k] = f2(kc2 * b.x, kc2 * b.y);
            cp[k] = f2(-kc * fmaf(c.x, c.x, fmaf(c.z, c.z, b.x * b.x)), -kc * fmaf(c.y, c.y, fmaf(c.w, c.w, b.y * b.y)));
        }
#pragma unroll
        for (int iy = 0; iy < KP + 2 * R; ++iy) {
            // a staged row no lane's window observes adds exact zeros (F = G = 0): skip it
            if (!((rows_warp >> iy) & 1u)) continue;
            float2 dd[KP];
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const int dy = iy - k;
                dd[k] = (dy >= 0 && dy < T) ? __fadd2_rn(cp[k], f2(a.ex_sy[dy], a.ex_sy[dy])) : f2(0.0f, 0.0f);
            }
#pragma unroll
            for (int dx = 0; dx < T; ++dx) {
                const int o = (rbase + iy) * SP + lane + dx;
                const float4 qc = sc[o], qb = sb[o];
                const float2 qg = sg[o];
                const float2 ex = f2(a.ex_sx[dx], a.ex_sx[dx]);
                const float2 fx = __fmul2_rn(f2(qb.z, qb.w), ex), gx = __fmul2_rn(qg, ex);
#pragma unroll
                for (int k = 0; k < KP; ++k) {
                    const int dy = iy - k;
                    if (dy >= 0 && dy < T) {
                        const float2 e = __ffma2_rn(
                            ar[k], f2(qc.x, qc.y),
                            __ffma2_rn(ag[k], f2(qc.z, qc.w), __ffma2_rn(ab[k], f2(qb.x, qb.y), dd[k])));
                        const float2 w = f2(ex2_approx(e.x), ex2_approx(e.y));
                        num[k] = __ffma2_rn(w, gx, num[k]);
                        den[k] = __ffma2_rn(w, fx, den[k]);
                    }
                }
            }
        }
    }

    // ---- outputs; a valid pixel whose weight sum is too small for the plain form (dominant
    // weight near the bottom of the FP32 range) is recomputed with shifted exponents
    // the output pointers in registers: a store through them could alias the frame descriptor,
    // which would make the compiler reload them after every store
    float *const out_depth = F.flt_depth;
    uint8_t *const out_valid = F.flt_valid;
    auto store = [&](int x, int y, float out, bool v) {
        if (x < gw && y < gh) {
            const int64_t o = (int64_t)y * gw + x;
            out_depth[o] = out;
            out_valid[o] = v;
        }
    };
    uint32_t slow = 0u;   // bit 2k + h: pixel (k, half h)
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const int y = y0 + rbase + k;
        if (val0[k] && !(den[k].x >= 0x1p-60f)) slow |= 1u << (2 * k);
        else store(x0 + lane, y, val0[k] ? __fdividef(num[k].x, den[k].x) : 0.0f, val0[k]);
        if (val1[k] && !(den[k].y >= 0x1p-60f)) slow |= 2u << (2 * k);
        else store(x0 + 32 + lane, y, val1[k] ? __fdividef(num[k].y, den[k].y) : 0.0f, val1[k]);
    }
    while (slow) {   // rare: from the raw boxes, largest exponent of the window first
        const int bit = __ffs(slow) - 1;
        slow &= slow - 1u;
        const int k = bit >> 1, cx = lane + 32 * (bit & 1);   // staged column of the pixel, minus R
        const uint8_t *pc = rgb_at(rbase + k + R, cx + R);
        const float cr0 = (float)pc[0], cg0 = (float)pc[1], cb0 = (float)pc[2];
        auto tap = [&](int dy, int dx, float &arg, float &wd) -> bool {
            const int sy = rbase + k + dy, sx = cx + dx;
            const uint8_t *p = rgb_at(sy, sx);
            const float dr = (float)p[0] - cr0, dg = (float)p[1] - cg0, db = (float)p[2] - cb0;
            wd = 0.0f;
            const bool seen = depth_of(sy, sx, wd, std::false_type{});
            const float n2 = fmaf(dr, dr, fmaf(dg, dg, db * db));
            const float s2 = (float)((dx - R) * (dx - R) + (dy - R) * (dy - R));
            arg = fmaf(n2, -a.kc, -s2 * a.kp);
            return seen;
        };
        float amax = -__int_as_float(0x7F800000);
#pragma unroll 1
        for (int dy = 0; dy < T; ++dy)
#pragma unroll 1
            for (int dx = 0; dx < T; ++dx) {
                float arg, wd;
                if (tap(dy, dx, arg, wd)) amax = fmaxf(amax, arg);
            }
        float nn = 0.0f, dn = 0.0f;
#pragma unroll 1
        for (int dy = 0; dy < T; ++dy)
#pragma unroll 1
            for (int dx = 0; dx < T; ++dx) {
                float arg, wd;
                if (tap(dy, dx, arg, wd)) {
                    const float w = ex2_approx(arg - amax);
                    nn = fmaf(w, wd, nn);
                    dn += w;
                }
            }
        store(x0 + cx, y0 + rbase + k, nn / dn, true);
    }
}

}  // namespace dz
