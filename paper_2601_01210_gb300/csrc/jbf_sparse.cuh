// One tile of the joint bilateral filter (Eq. (1)-(4)) for a sparse input:
// the single stage on the z-buffer, where a few percent of the pixels hold an
// observation. Called by the TMA-staged kernel (jbf_tma.cuh) once the tile's
// raw boxes (colour bytes, z-buffer words) are in shared memory.
//
// A dense gather evaluates every position of every pixel's window; here each
// warp owns an 8 x 8 block of output pixels (two per lane, rows ly and ly + 4
// of column lx) and walks only the observed positions of the block's footprint
// (the block grown by the radius), in a loop that every lane of the warp runs
// together: for each observed position q the lanes evaluate the taps (p, q) of
// their pixels that fall inside the window and accumulate numerator and weight
// sum in registers. The work per block follows the observations in its
// footprint, not the window area.
//
// The observed positions of the tile and its halo are found once per tile (one
// 64-bit mask per staged row) and each gets a record:
//   A = (2 kc c'_q, -kc |c'_q|^2),  B = (x_q, y_q, depth_q)
// with colours centred at 128 (exact) and tile-relative coordinates. The weight
// of q at pixel p is then
//   2^(2 kc c'_p . c'_q - kc |c'_q|^2 - kp |p - q|^2)
// = Eq. (2)-(3)'s weight times 2^(kc |c'_p|^2), a factor shared by every tap of
// p that cancels in Eq. (1)'s quotient; the exponent is at most kc 3 128^2 (the
// host keeps that within range). Validity is an observed position inside the
// window, the same integer decision as the other forms. A valid pixel whose
// weight sum falls below 2^-60 is recomputed with the largest exponent of its
// window shifted to 0.
//
// FP16 form (HALF): the guide and the weights in half precision, the sums in
// FP32 (the precision of the FP16 form in jbf_tma.cuh, on the same error
// bound). A record holds the colour bytes as half2 pairs (exact) and the
// depth; per observed position the lane forms both pixels' colour differences,
// squared distance and exponent -kc |c_p - c_q|^2 - kp |p - q|^2 as half2 and
// takes both weights with one ex2.approx.f16x2. A valid pixel whose weight sum
// is below 2^-6, or whose weighted depth spread could carry the FP16 weight
// error past half of the 1e-3 relative bar, is recomputed in FP32 (its
// window's largest exponent shifted to 0).
#pragma once

#include <cstdint>

#include "jbf_core.cuh"
#include "tma_common.cuh"

namespace dz {

// store(x, y, depth, valid) takes tile-relative pixel coordinates. A warp with bad set (its copies
// did not land) skips the records; the barrier after them ORs the flag and the function then
// returns true at once, for the caller to leave (false once the tile is done).
template <int R, int KP, int NW, bool HALF, class AfterRecords, class Store>
__device__ __forceinline__ bool sparse_tile(const StageArgs &a, int x0, int y0, int gw, int gh, const uint8_t *rgbraw,
                                            const uint8_t *rawb, uint8_t *smem, bool bad,
                                            AfterRecords &&after_records, Store &&store) {
    using G = TmaGeom<SRC_ZBUF, R, KP, NW, HALF ? FORM_SPARSE_FP16 : FORM_SPARSE>;
    constexpr int TW = G::TW, TH = G::TH, SW = G::SW, SH = G::SH, RPW = G::RPW;
    constexpr int FW = 8 + 2 * R;                      // footprint of a block: columns bx .. bx + FW - 1 staged
    constexpr uint64_t FMASK = (uint64_t(1) << FW) - 1u;
    constexpr int BLOCKS = (TW / 8) * (TH / 8);
    static_assert(TW == 32 && TH % 8 == 0 && SW <= 64 && FW <= 32 + 2 * R, "sparse form: 32-column tiles");
    float4 *rec_a = reinterpret_cast<float4 *>(smem + G::OFF_STAGED);   // per staged position (observed only)
    uint4 *rec_h = reinterpret_cast<uint4 *>(rec_a);                    // FP16 form: the same 16 bytes
    float4 *rec_b = rec_a + SH * SW;
    uint64_t *rowmask = reinterpret_cast<uint64_t *>(smem + G::OFF_ROWS);
    const uint32_t *zraw = reinterpret_cast<const uint32_t *>(rawb);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float kc = a.kc, kc2 = 2.0f * a.kc, kp = a.kp;
    auto rgb_at = [&](int sy, int sx) { return rgbraw + sy * G::RGB_BX + 3 * sx - 3 * R + G::RGB_LEAD; };
    auto bytef = [](uint32_t b) { return __uint_as_float(0x4B000000u | b) - 8388736.0f; };   // b - 128, exact

    // ---- records of the observed positions; warp w scans staged rows w, w + NW, ...
#pragma unroll 1
    for (int i = 0; i < (bad ? 0 : RPW); ++i) {
        const int sy = warp + NW * i;
        if (sy >= SH) break;
        uint64_t mask = 0;
#pragma unroll
        for (int c0 = 0; c0 < SW; c0 += 32) {
            const int sx = c0 + lane;
            bool o = false;
            uint32_t z = kEmpty;
            if (sx < SW) {
                const int gx = x0 - R + sx, gy = y0 - R + sy;
                z = zraw[sy * G::Z_BX + sx - R + G::Z_LEAD];
                o = gx >= 0 && gx < gw && gy >= 0 && gy < gh && z != kEmpty;
            }
            if (o) {
                const uint8_t *p = rgb_at(sy, sx);
                if (HALF) {   // colour bytes as half2 pairs (exact), depth bits
                    rec_h[sy * SW + sx] = make_uint4(h2u(__float2half2_rn((float)p[0])), h2u(__float2half2_rn((float)p[1])),
                                                     h2u(__float2half2_rn((float)p[2])), z);
                } else {
                    const float r = bytef(p[0]), g = bytef(p[1]), b = bytef(p[2]);
                    rec_a[sy * SW + sx] = make_float4(kc2 * r, kc2 * g, kc2 * b, -kc * fmaf(r, r, fmaf(g, g, b * b)));
                }
                rec_b[sy * SW + sx] = make_float4((float)(sx - R), (float)(sy - R), __uint_as_float(z), 0.0f);
            }
            mask |= (uint64_t)__ballot_sync(0xffffffffu, o) << c0;
        }
        if (lane == 0) rowmask[sy] = mask;
    }
    if (__syncthreads_or(bad)) return true;
    after_records();

    // ---- blocks of 8 x 8 pixels: lane (lx, ly) owns pixels (bx + lx, by + ly) and (bx + lx, by + ly + 4)
    const int lx = lane & 7, ly = lane >> 3;
    const float rr = (float)R;
#pragma unroll 1
    for (int blk = warp; blk < BLOCKS; blk += NW) {
        const int bx = (blk % (TW / 8)) * 8, by = (blk / (TW / 8)) * 8;
        const int px = bx + lx;
        const float pxf = (float)px;
        float cr[2], cg[2], cb[2], pyf[2], num[2], den[2], sq[2];
        bool hit[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int py = by + ly + 4 * k;
            const uint8_t *p = rgb_at(py + R, px + R);
            cr[k] = bytef(p[0]);
            cg[k] = bytef(p[1]);
            cb[k] = bytef(p[2]);
            pyf[k] = (float)py;
            num[k] = den[k] = sq[k] = 0.0f;
            hit[k] = false;
        }
        // FP16 form: the two pixels' colour bytes as half2 (exact), -kc as half2
        const __half2 hr = __floats2half2_rn(cr[0] + 128.0f, cr[1] + 128.0f),
                      hg = __floats2half2_rn(cg[0] + 128.0f, cg[1] + 128.0f),
                      hb = __floats2half2_rn(cb[0] + 128.0f, cb[1] + 128.0f), nkc = __float2half2_rn(-kc);
        // footprint: staged rows by .. by + 7 + 2R, columns bx .. bx + FW - 1 (the same in every lane)
#pragma unroll 1
        for (int sy = by; sy < by + 8 + 2 * R; ++sy) {
            uint64_t m = (rowmask[sy] >> bx) & FMASK;
            while (m) {
                const int sx = bx + __ffsll((long long)m) - 1;
                m &= m - 1;
                const float4 qb = rec_b[sy * SW + sx];
                const float dx = qb.x - pxf, adx = fabsf(dx), dx2 = dx * dx;
                if (HALF) {
                    const uint4 qh = rec_h[sy * SW + sx];
                    const float dy0 = qb.y - pyf[0], dy1 = qb.y - pyf[1];
                    const bool in0 = fmaxf(adx, fabsf(dy0)) <= rr, in1 = fmaxf(adx, fabsf(dy1)) <= rr;
                    const __half2 sp = __floats2half2_rn(-kp * fmaf(dy0, dy0, dx2), -kp * fmaf(dy1, dy1, dx2));
                    const __half2 dr = __hsub2(h2bits(qh.x), hr), dg = __hsub2(h2bits(qh.y), hg),
                                  db = __hsub2(h2bits(qh.z), hb);
                    const __half2 n2 = __hfma2(dr, dr, __hfma2(dg, dg, __hmul2(db, db)));
                    const float2 w = __half22float2(h2exp2_approx(__hfma2(n2, nkc, sp)));
                    const float d = qb.z, wd0 = w.x * d, wd1 = w.y * d;
                    if (in0) {
                        num[0] += wd0;
                        den[0] += w.x;
                        sq[0] = fmaf(wd0, d, sq[0]);
                        hit[0] = true;
                    }
                    if (in1) {
                        num[1] += wd1;
                        den[1] += w.y;
                        sq[1] = fmaf(wd1, d, sq[1]);
                        hit[1] = true;
                    }
                } else {
                    const float4 qa = rec_a[sy * SW + sx];
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const float dy = qb.y - pyf[k];
                        const bool in = fmaxf(adx, fabsf(dy)) <= rr;
                        const float s2 = fmaf(dy, dy, dx2);
                        const float e = fmaf(qa.x, cr[k], fmaf(qa.y, cg[k], fmaf(qa.z, cb[k], fmaf(s2, -kp, qa.w))));
                        const float w = ex2_approx(e);
                        if (in) {
                            num[k] = fmaf(w, qb.z, num[k]);
                            den[k] += w;
                            hit[k] = true;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int py = by + ly + 4 * k;
            float out = 0.0f;
            if (hit[k]) {
                bool plain = den[k] >= (HALF ? 0x1p-6f : 0x1p-60f);
                if (plain) {
                    out = __fdividef(num[k], den[k]);
                    if (HALF) {
                        // the FP16 weights' error bound (see kHalfWeightErr): the depth error is at most
                        // kHalfWeightErr times the weighted standard deviation of the window's depths
                        const float var = __fdividef(sq[k], den[k]) - out * out, lim = kHalfStdFrac * out;
                        plain = !(var > lim * lim);
                    }
                }
                if (!plain) {   // rare: in FP32, the window's largest exponent shifted to 0
                    float amax = -__int_as_float(0x7F800000), nn = 0.0f, dd = 0.0f;
                    for (int pass = 0; pass < 2; ++pass)
                        for (int sy = py; sy <= py + 2 * R; ++sy) {
                            uint64_t mm = (rowmask[sy] >> px) & ((uint64_t(1) << (2 * R + 1)) - 1u);
                            while (mm) {
                                const int sx = px + __ffsll((long long)mm) - 1;
                                mm &= mm - 1;
                                const float4 qb = rec_b[sy * SW + sx];
                                const float dx = qb.x - pxf, dy = qb.y - pyf[k];
                                float e;
                                if (HALF) {   // the difference form from the exact colour bytes
                                    const uint4 qh = rec_h[sy * SW + sx];
                                    const float dr = __low2float(h2bits(qh.x)) - 128.0f - cr[k],
                                                dg = __low2float(h2bits(qh.y)) - 128.0f - cg[k],
                                                db = __low2float(h2bits(qh.z)) - 128.0f - cb[k];
                                    e = fmaf(fmaf(dr, dr, fmaf(dg, dg, db * db)), -kc, -kp * fmaf(dy, dy, dx * dx));
                                } else {
                                    const float4 qa = rec_a[sy * SW + sx];
                                    e = fmaf(qa.x, cr[k], fmaf(qa.y, cg[k], fmaf(qa.z, cb[k],
                                             fmaf(fmaf(dy, dy, dx * dx), -kp, qa.w))));
                                }
                                if (pass == 0) {
                                    amax = fmaxf(amax, e);
                                } else {
                                    const float w = ex2_approx(e - amax);
                                    nn = fmaf(w, qb.z, nn);
                                    dd += w;
                                }
                            }
                        }
                    out = nn / dd;
                }
            }
            store(px, py, out, hit[k]);
        }
    }
    return false;
}

}  // namespace dz
