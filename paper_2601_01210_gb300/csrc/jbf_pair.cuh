// One tile of the joint bilateral filter (Eq. (1)-(4)) in the expanded FP32
// form, on pairs of output columns in packed two-lane FP32 arithmetic. Called
// by the TMA-staged kernel (jbf_tma.cuh) once the tile's raw boxes are in
// shared memory; the full-resolution stages only (restored first-stage result
// or z-buffer as depth, RGB bytes as guide).
//
// Expanded form: with the centred colours c' = c - 128 (one signed byte per
// channel), the colour term of a tap is
//   -kc |c'_p - c'_q|^2 = 2 kc c'_p . c'_q - kc |c'_p|^2 - kc |c'_q|^2,
// so the weight of neighbour q at offset (dx - R, dy - R) is
//   2^(2 kc c'_p . c'_q - kc |c'_p|^2) * F_q * S(dx) * S(dy),
// with F_q = 2^(-kc |c'_q|^2) computed once per staged neighbour (0 when q
// holds no observation), S(d) = 2^(-kp (d - R)^2) the separable spatial
// factor, and the depth entering as G_q = F_q * depth_q.
//
// The dot product c'_p . c'_q is one dp4a of the packed signed bytes, exact in
// integers. Started from the bit pattern of 1.5 * 2^23, the dp4a result read
// as a float is exactly 1.5 * 2^23 + c'_p . c'_q, and one FMA gives the
// exponent: f * 2kc + C_p, C_p = -kc |c'_p|^2 - 2kc * 1.5 * 2^23 rounded once.
// The FMA cancels the large terms exactly; the rounding of C_p moves every
// exponent of pixel p by the same amount, which cancels in Eq. (1)'s quotient.
// The row factor S(dy) scales each staged row's partial sums. A tap costs one
// dp4a, one FMA, one ex2 and one FMA each into the numerator and weight sum.
//
// Column pairs: a thread owns output columns x0 + lane and x0 + 32 + lane of a
// 64-column tile, rows rbase .. rbase + KP - 1. Staged slot s of a row holds
// the records of staged columns s and s + 32 side by side, so the neighbour at
// tap dx of both pixels sits in one slot (lane + dx) and every floating-point
// step runs once for the two pixels as a two-lane FP32 instruction
// (__ffma2_rn / __fmul2_rn / __fadd2_rn, each lane rounded as its scalar
// counterpart). A slot's records (24 bytes):
//   sc = (colour word of column s, colour word of column s + 32), each the
//        packed signed bytes (r', g', b', 0);
//   fg = (F of column s, F of column s + 32, G of column s, G of column s + 32).
//
// A tile takes two steps: pair_convert writes the slot records and
// observation bitmaps from the raw boxes (every thread of the CTA), then
// pair_filter computes the outputs of KP rows of the tile from those records
// (one warp per KP rows).
#pragma once

#include <type_traits>

#include "jbf_core.cuh"
#include "tma_common.cuh"

namespace dz {

__device__ __forceinline__ float2 f2(float lo, float hi) { return make_float2(lo, hi); }

// Bit pattern of 1.5 * 2^23: a float whose last mantissa bit weighs 1, with 2^22 of room on either side.
constexpr int kDotBias = 0x4B400000;
constexpr float kDotBiasF = 12582912.0f;

// Colour bytes r, g, b (0..255) as the packed signed bytes of c - 128 (byte b xor 0x80 = b - 128).
__device__ __forceinline__ uint32_t pack_centred(uint32_t r, uint32_t g, uint32_t b) {
    return (r | (g << 8) | (b << 16)) ^ 0x00808080u;
}

// One set of slot records and observation bitmaps in shared memory (bit i of
// obs0 / obs1: the first / second staged column of slot i holds an observation;
// each bitmap ends in a zero guard word).
struct PairRecords {
    float4 *fg;
    uint2 *sc;
    uint32_t *obs0, *obs1;
};

// Staged position (sy, sx) <-> image pixel (x0 - R + sx, y0 - R + sy): depth and
// observation in the raw first-stage box (restored by x / 3, y / 3) or the raw
// z-buffer box. G gives the boxes' geometry.
template <int SRC, int R, class G, bool INSIDE>
__device__ __forceinline__ bool pair_raw_depth(const uint8_t *rawb, int x0, int y0, int gw, int gh, int sy, int sx,
                                               float &d) {
    const int gx = x0 - R + sx, gy = y0 - R + sy;
    if (!INSIDE && (gx < 0 || gx >= gw || gy < 0 || gy >= gh)) return false;
    if (SRC == SRC_UP) {
        const int cx0 = floor_div3(x0 - R) & ~1, cy0 = floor_div3(y0 - R);
        const float2 c = reinterpret_cast<const float2 *>(
            rawb)[((int)((unsigned)gy / 3u) - cy0) * G::C_BX + ((int)((unsigned)gx / 3u) - cx0)];
        d = c.x;
        return c.y > 0.0f;
    }
    const uint32_t z = reinterpret_cast<const uint32_t *>(rawb)[sy * G::Z_BX + sx - R + G::Z_LEAD];
    d = __uint_as_float(z);
    return z != kEmpty;
}

// Slot records of a tile: the NCT converting threads take slots t, t + NCT, ... (t their index
// among them, consecutive within each warp), in groups of up to 8 per thread: all raw loads of a
// group first, then its records; one ballot per half gives a word of each observation bitmap.
template <int SRC, int R, class G, int NCT>
__device__ __forceinline__ void pair_convert(const StageArgs &a, int x0, int y0, int gw, int gh, const uint8_t *rgbraw,
                                             const uint8_t *rawb, const PairRecords st, int t) {
    static_assert(SRC != SRC_COARSE, "paired form: full-resolution stages");
    constexpr int SP = G::SP, SH = G::SH, NCONV = (SH * SP + NCT - 1) / NCT;
    constexpr int CH = NCONV <= 8 ? NCONV : 4;   // slots of a thread per group
    const int lane = t & 31;
    auto rgb_at = [&](int sy, int sx) { return rgbraw + sy * G::RGB_BX + 3 * sx - 3 * R + G::RGB_LEAD; };
    // a tile whose halo lies inside the image needs no bounds checks on its staged positions
    const bool interior = x0 >= R && x0 + G::TW + R <= gw && y0 >= R && y0 + G::TH + R <= gh;
    const float kc = a.kc;
#pragma unroll 1
    for (int j0 = 0; j0 < NCONV; j0 += CH) {
        uint32_t om0 = 0u, om1 = 0u;   // bit j: first / second column of slot j of the group observed
        float d0[CH], d1[CH];
        uint32_t r0[CH], g0[CH], b0[CH], r1[CH], g1[CH], b1[CH];
        auto load_slots = [&](auto inside) {
            constexpr bool IN = decltype(inside)::value;
#pragma unroll
            for (int j = 0; j < CH; ++j) {
                const int i = t + (j0 + j) * NCT;
                d0[j] = d1[j] = 0.0f;
                r0[j] = g0[j] = b0[j] = r1[j] = g1[j] = b1[j] = 0u;
                if (j0 + j < NCONV && i < SH * SP) {
                    const int sy = i / SP, s = i - sy * SP;
                    float d = 0.0f;
                    if (pair_raw_depth<SRC, R, G, IN>(rawb, x0, y0, gw, gh, sy, s, d)) om0 |= 1u << j;
                    d0[j] = d;
                    d = 0.0f;
                    if (pair_raw_depth<SRC, R, G, IN>(rawb, x0, y0, gw, gh, sy, s + 32, d)) om1 |= 1u << j;
                    d1[j] = d;
                    const uint8_t *p = rgb_at(sy, s), *q = p + 96;
                    r0[j] = p[0]; g0[j] = p[1]; b0[j] = p[2];
                    r1[j] = q[0]; g1[j] = q[1]; b1[j] = q[2];
                }
            }
        };
        if (interior) load_slots(std::true_type{});
        else load_slots(std::false_type{});
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            if (j0 + j >= NCONV) break;
            const int i = t + (j0 + j) * NCT;
            const bool o0 = (om0 >> j) & 1u, o1 = (om1 >> j) & 1u;
            if (i < SH * SP) {
                // centred colours; |c'|^2 by dp4a (exact integer below 2^16, read as a float from
                // 2^23 + n); an unobserved record keeps its colour with F = G = 0
                const uint32_t c0 = pack_centred(r0[j], g0[j], b0[j]), c1 = pack_centred(r1[j], g1[j], b1[j]);
                const float2 n2 = __fadd2_rn(f2(__int_as_float(__dp4a((int)c0, (int)c0, 0x4B000000)),
                                                __int_as_float(__dp4a((int)c1, (int)c1, 0x4B000000))),
                                             f2(-8388608.0f, -8388608.0f));
                const float2 e = __fmul2_rn(f2(-kc, -kc), n2);
                const float f0 = o0 ? ex2_approx(e.x) : 0.0f, f1 = o1 ? ex2_approx(e.y) : 0.0f;
                const float2 fd = __fmul2_rn(f2(f0, f1), f2(d0[j], d1[j]));
                st.sc[i] = make_uint2(c0, c1);
                // an empty z-buffer cell holds +inf: G = 0 where unobserved
                st.fg[i] = make_float4(f0, f1, o0 ? fd.x : 0.0f, o1 ? fd.y : 0.0f);
            }
            const uint32_t w0 = __ballot_sync(0xffffffffu, o0), w1 = __ballot_sync(0xffffffffu, o1);
            if (lane == 0) {
                st.obs0[i >> 5] = w0;
                st.obs1[i >> 5] = w1;
            }
        }
    }
}

// Outputs of tile rows rbase .. rbase + KP - 1 (one warp) from the tile's slot records.
// raw_at(sy, sx, r, g, b, d) gives the colour bytes and the depth of staged position (sy, sx)
// and whether it holds an observation, for the shifted recomputation of a valid pixel whose
// weight sum is too small for the plain form (dominant weight near the bottom of the FP32 range).
template <int SRC, int R, int KP, class G, class RawAt>
__device__ __forceinline__ void pair_filter(float *out_depth, uint8_t *out_valid, const StageArgs &a, int x0, int y0,
                                            int gw, int gh, const PairRecords st, int rbase, int lane,
                                            RawAt &&raw_at) {
    constexpr int SP = G::SP, T = 2 * R + 1;
    constexpr uint32_t TMASK = (1u << T) - 1u;
    const float kc = a.kc;

    // ---- validity: an output pixel is valid when its window holds an observation
    bool val0[KP], val1[KP];
    bool any_val = false;
    uint32_t rows_warp;   // bit iy: some lane of the warp has an observation in its window of staged row rbase + iy
    {
        uint32_t rows0 = 0u, rows1 = 0u;   // bit iy: an observation in staged row rbase + iy, slots lane .. lane + 2R
#pragma unroll
        for (int iy = 0; iy < KP + 2 * R; ++iy) {
            const int bit = (rbase + iy) * SP + lane;   // the window never leaves its row
            const uint32_t w0 = __funnelshift_r(st.obs0[bit >> 5], st.obs0[(bit >> 5) + 1], bit & 31);
            const uint32_t w1 = __funnelshift_r(st.obs1[bit >> 5], st.obs1[(bit >> 5) + 1], bit & 31);
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
        const float kc2 = 2.0f * kc, bias = -kc2 * kDotBiasF;
        uint2 cq[KP];     // packed centred colours of the thread's two pixels in row k
        float2 cp[KP];    // C_p of both: -kc |c'_p|^2 + bias (one rounding, the same for every tap of p)
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            cq[k] = st.sc[(rbase + k + R) * SP + lane + R];
            cp[k] = f2(fmaf(-kc, (float)__dp4a((int)cq[k].x, (int)cq[k].x, 0), bias),
                       fmaf(-kc, (float)__dp4a((int)cq[k].y, (int)cq[k].y, 0), bias));
        }
#pragma unroll
        for (int iy = 0; iy < KP + 2 * R; ++iy) {
            // a staged row no lane's window observes adds exact zeros (F = G = 0): skip it
            if (!((rows_warp >> iy) & 1u)) continue;
            float2 rn[KP], rd[KP];   // the row's partial sums of pixel k, before its factor S(dy)
#pragma unroll
            for (int dx = 0; dx < T; ++dx) {
                const int o = (rbase + iy) * SP + lane + dx;
                const uint2 qc = st.sc[o];
                const float4 q = st.fg[o];
                const float2 ex = f2(a.ex_sx[dx], a.ex_sx[dx]);
                const float2 fx = __fmul2_rn(f2(q.x, q.y), ex), gx = __fmul2_rn(f2(q.z, q.w), ex);
#pragma unroll
                for (int k = 0; k < KP; ++k) {
                    const int dy = iy - k;
                    if (dy >= 0 && dy < T) {
                        const float2 f = f2(__int_as_float(__dp4a((int)cq[k].x, (int)qc.x, kDotBias)),
                                            __int_as_float(__dp4a((int)cq[k].y, (int)qc.y, kDotBias)));
                        const float2 e = __ffma2_rn(f, f2(kc2, kc2), cp[k]);
                        const float2 w = f2(ex2_approx(e.x), ex2_approx(e.y));
                        if (dx == 0) {
                            rn[k] = __fmul2_rn(w, gx);
                            rd[k] = __fmul2_rn(w, fx);
                        } else {
                            rn[k] = __ffma2_rn(w, gx, rn[k]);
                            rd[k] = __ffma2_rn(w, fx, rd[k]);
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const int dy = iy - k;
                if (dy >= 0 && dy < T) {
                    const float2 ey = f2(a.ex_sx[dy], a.ex_sx[dy]);   // S(dy): the factor is symmetric
                    num[k] = __ffma2_rn(ey, rn[k], num[k]);
                    den[k] = __ffma2_rn(ey, rd[k], den[k]);
                }
            }
        }
    }

    // ---- outputs, through one pair of pointers for the warp's rows (row k at k * gw); columns
    // and rows outside the grid are left alone
    auto store = [&](int x, int y, float out, bool v) {
        if (x < gw && y < gh) {
            const int64_t o = (int64_t)y * gw + x;
            out_depth[o] = out;
            out_valid[o] = v;
        }
    };
    uint32_t slow = 0u;   // bit 2k + h: pixel (k, half h)
    {
        const int64_t o0 = (int64_t)(y0 + rbase) * gw + x0 + lane;
        float *const dp = out_depth + o0;
        uint8_t *const vp = out_valid + o0;
        const bool in0 = x0 + lane < gw, in1 = x0 + 32 + lane < gw;
        const int rows_in = gh - (y0 + rbase);
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            if (k >= rows_in) break;
            const int64_t ok = (int64_t)k * gw;
            if (val0[k] && !(den[k].x >= 0x1p-60f)) {
                slow |= 1u << (2 * k);
            } else if (in0) {
                dp[ok] = val0[k] ? __fdividef(num[k].x, den[k].x) : 0.0f;
                vp[ok] = val0[k];
            }
            if (val1[k] && !(den[k].y >= 0x1p-60f)) {
                slow |= 2u << (2 * k);
            } else if (in1) {
                dp[ok + 32] = val1[k] ? __fdividef(num[k].y, den[k].y) : 0.0f;
                vp[ok + 32] = val1[k];
            }
        }
    }
    while (slow) {   // rare: largest exponent of the window first
        const int bit = __ffs(slow) - 1;
        slow &= slow - 1u;
        const int k = bit >> 1, cx = lane + 32 * (bit & 1);   // staged column of the pixel, minus R
        float cr0, cg0, cb0, cd;
        raw_at(rbase + k + R, cx + R, cr0, cg0, cb0, cd);
        auto tap = [&](int dy, int dx, float &arg, float &wd) -> bool {
            float r, g, b;
            wd = 0.0f;
            const bool seen = raw_at(rbase + k + dy, cx + dx, r, g, b, wd);
            const float dr = r - cr0, dg = g - cg0, db = b - cb0;
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

// One tile with all NW warps of the CTA: conversion, a barrier, then each warp's KP rows.
// A warp with bad set (its copies did not land) skips the conversion; the barrier ORs the
// flag and the function then returns true at once, for the caller to leave. Otherwise
// after_conversion() runs right after the barrier that publishes the slot records (the
// kernel's thread 0 advances its tile queue there) and the function returns false; the
// caller ends the tile with a barrier before the records or the raw boxes are rewritten.
template <int SRC, int R, int KP, int NW, class AfterConversion>
__device__ __forceinline__ bool pair_tile(float *out_depth, uint8_t *out_valid, const StageArgs &a, int x0, int y0,
                                          int gw, int gh,
                                          const uint8_t *rgbraw, const uint8_t *rawb, uint8_t *smem, bool bad,
                                          AfterConversion &&after_conversion) {
    using G = TmaGeom<SRC, R, KP, NW, FORM_EXP_PAIRS>;
    PairRecords st;
    st.fg = reinterpret_cast<float4 *>(smem + G::OFF_STAGED);
    st.sc = reinterpret_cast<uint2 *>(smem + G::OFF_G);
    st.obs0 = reinterpret_cast<uint32_t *>(smem + G::OFF_OBS);
    st.obs1 = st.obs0 + G::OBS_ONE / 4;
    if (!bad) pair_convert<SRC, R, G, G::NT>(a, x0, y0, gw, gh, rgbraw, rawb, st, threadIdx.x);
    if (__syncthreads_or(bad)) return true;
    after_conversion();
    // the shifted recomputation reads the raw boxes, which stay in place until the tile ends
    auto raw_at = [&](int sy, int sx, float &r, float &g, float &b, float &d) -> bool {
        const uint8_t *p = rgbraw + sy * G::RGB_BX + 3 * sx - 3 * R + G::RGB_LEAD;
        r = (float)p[0];
        g = (float)p[1];
        b = (float)p[2];
        return pair_raw_depth<SRC, R, G, false>(rawb, x0, y0, gw, gh, sy, sx, d);
    };
    pair_filter<SRC, R, KP, G>(out_depth, out_valid, a, x0, y0, gw, gh, st, (threadIdx.x >> 5) * KP, threadIdx.x & 31,
                               raw_at);
    return false;
}

}  // namespace dz
