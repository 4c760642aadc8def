// One tile of the joint bilateral filter (Eq. (1)-(4)) in the scatter form of
// Algorithm 1: every observed neighbour q of the tile and its halo adds its
// weighted depth and its weight into the numerator and weight-sum accumulators
// of the output pixels its window reaches (Algorithm 1's transpose
// convolution), so the work follows the observed taps instead of the window
// area. Called by the TMA-staged kernel (jbf_tma.cuh) for the single stage on
// the z-buffer, whose input is sparse. (On the pooled first stage, about a third
// observed, it measured four times slower than the register-blocked gather: the
// per-tap shared-memory adds and their addresses cost more than the unobserved
// taps the gather evaluates.)
//
// Weight of neighbour q at output pixel p, with colours centred at 128 (exact):
//   2^(2 kc c'_p . c'_q - kc |c'_q|^2 + sp(p - q))
// which is Eq. (2)-(3)'s weight 2^(-kc |c'_p - c'_q|^2 + sp(p - q)) times
// 2^(kc |c'_p|^2), a factor shared by every tap of p that cancels in Eq. (1)'s
// quotient. The exponent is at most kc |c'_p|^2 <= kc 3 128^2, which the host
// keeps within range (the same condition as the expanded gather form).
// Per tap: one load of c'_p, three FMAs and one add for the exponent, one ex2,
// and two shared-memory adds (numerator: weight times the neighbour's depth,
// or its pooled depth sum; weight sum: weight times 1, or the pooled count).
//
// Races and order: warp w lists the observed positions of the staged rows w,
// w + NW, w + 2 NW, ... (in row-major order). The scatter runs in 2R + 1
// phases, one per row offset oy, separated by block barriers. In phase oy the
// targets of warp w lie in rows (its source rows + oy), which no other warp
// reaches in that phase; within one instruction the lanes' sources differ, so
// do their targets. Every accumulator therefore receives its adds from one warp
// per phase, in instruction order, and the sums are the same on every run.
//
// Validity (an observation in the window) comes from a 64-bit observation mask
// per staged row, exactly as the gather forms decide it. A valid pixel whose
// weight sum falls below 2^-60 is recomputed by a gather with shifted exponents.
#pragma once

#include <cstdint>

#include "jbf_core.cuh"
#include "tma_common.cuh"

namespace dz {

// FP32 add into shared memory, no return value (the address is a shared-window offset, so the
// add takes the shared-memory path whatever the compiler infers about a generic pointer)
__device__ __forceinline__ void red_shared_add(uint32_t addr, float v) {
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// Epilogue sink of one output pixel: store(k, depth, valid) for row k of the thread.
template <int SRC, int R, int KP, int NW, class AfterLists, class Store, class MarkRows>
__device__ __forceinline__ void scatter_tile(const FrameDev &F, const StageArgs &a, int x0, int y0, int gw, int gh,
                                             const uint8_t *rawa, const uint8_t *rawb, uint8_t *smem,
                                             AfterLists &&after_lists, Store &&store, MarkRows &&mark_rows) {
    using G = TmaGeom<SRC, R, KP, NW, FORM_SCATTER>;
    constexpr int TW = G::TW, TH = G::TH, SW = G::SW, SH = G::SH, T = 2 * R + 1, NT = G::NT, RPW = G::RPW;
    constexpr int TWP = G::TWP;   // row pitch of the target and accumulator arrays
    constexpr uint32_t TMASK = (1u << T) - 1u;
    static_assert(TW == 32 && SW <= 64, "scatter form: 32-column tiles, row masks of 64 bits");
    float4 *tgt = reinterpret_cast<float4 *>(smem + G::OFF_TGT);           // c'_p of the tile's pixels
    float *acc_n = reinterpret_cast<float *>(smem + G::OFF_ACC);           // numerators
    float *acc_d = acc_n + TH * TWP;                                       // weight sums
    // source lists, two arrays of float4 (structure of arrays: consecutive sources, consecutive words)
    float4 *list_a = reinterpret_cast<float4 *>(smem + G::OFF_STAGED);
    float4 *list_v = list_a + NW * RPW * SW;
    uint64_t *rowmask = reinterpret_cast<uint64_t *>(smem + G::OFF_ROWS);  // observed staged positions
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float kc = a.kc, kc2 = 2.0f * a.kc;

    // raw boxes: SRC_COARSE pooled guide (float4 r, g, b, count; staged column sx at 4 sx) and pooled
    // depth sums; SRC_ZBUF colour bytes and z-buffer words
    const float4 *cg = reinterpret_cast<const float4 *>(rawa);
    const float *cs = reinterpret_cast<const float *>(rawb);
    const uint32_t *zraw = reinterpret_cast<const uint32_t *>(rawb);
    auto rgb_at = [&](int sy, int sx) { return rawa + sy * G::RGB_BX + 3 * sx - 3 * R + G::RGB_LEAD; };
    auto bytef = [](uint32_t b) { return __uint_as_float(0x4B000000u | b) - 8388736.0f; };   // b - 128, exact
    // centred colour of staged position (sy, sx)
    auto colour = [&](int sy, int sx, float &r, float &g, float &b) {
        if (SRC == SRC_COARSE) {
            const float4 q = cg[sy * SW + sx];
            r = q.x - 128.0f; g = q.y - 128.0f; b = q.z - 128.0f;
        } else {
            const uint8_t *p = rgb_at(sy, sx);
            r = bytef(p[0]); g = bytef(p[1]); b = bytef(p[2]);
        }
    };

    // ---- target colours and zeroed accumulators (flat over the tile's pixels)
#pragma unroll 1
    for (int i = threadIdx.x; i < TW * TH; i += NT) {
        const int tx = i & (TW - 1), ty = i / TW;
        float r, g, b;
        colour(ty + R, tx + R, r, g, b);
        tgt[ty * TWP + tx] = make_float4(r, g, b, 0.0f);
        acc_n[ty * TWP + tx] = 0.0f;
        acc_d[ty * TWP + tx] = 0.0f;
    }

    // ---- this warp's source list: observed positions of staged rows warp, warp + NW, ...
    float4 *mine_a = list_a + warp * RPW * SW, *mine_v = list_v + warp * RPW * SW;
    int n = 0;   // the same in every lane
#pragma unroll 1
    for (int i = 0; i < RPW; ++i) {
        const int sy = warp + NW * i;
        if (sy >= SH) break;
        uint64_t mask = 0;
#pragma unroll
        for (int c0 = 0; c0 < SW; c0 += 32) {
            const int sx = c0 + lane;
            bool o = false;
            float val = 0.0f, base = 1.0f;
            if (sx < SW) {
                const int gx = x0 - R + sx, gy = y0 - R + sy;
                if (SRC == SRC_COARSE) {
                    base = cg[sy * SW + sx].w;   // the box's fill outside the grid is 0: no observation
                    val = cs[sy * G::S_BX + sx - R + G::S_LEAD];
                    o = base > 0.0f;
                } else {
                    const uint32_t z = zraw[sy * G::Z_BX + sx - R + G::Z_LEAD];
                    o = gx >= 0 && gx < gw && gy >= 0 && gy < gh && z != kEmpty;
                    val = __uint_as_float(z);
                }
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, o);
            if (o) {
                float r, g, b;
                colour(sy, sx, r, g, b);
                const int at = n + __popc(bal & ((1u << lane) - 1u));
                mine_a[at] = make_float4(kc2 * r, kc2 * g, kc2 * b, -kc * fmaf(r, r, fmaf(g, g, b * b)));
                mine_v[at] = make_float4(val, base, __int_as_float(sx | (sy << 16)), 0.0f);
            }
            n += __popc(bal);
            mask |= (uint64_t)bal << c0;
        }
        if (lane == 0) rowmask[sy] = mask;
    }
    __syncthreads();
    after_lists();

    // ---- scatter, one phase per row offset
    const uint32_t an0 = smem_u32(acc_n), ad0 = smem_u32(acc_d);
#pragma unroll
    for (int oy = -R; oy <= R; ++oy) {
#pragma unroll 1
        for (int b0 = 0; b0 < n; b0 += 32) {
            const int j = b0 + lane;
            float4 A = make_float4(0.0f, 0.0f, 0.0f, 0.0f), V = A;
            if (j < n) {
                A = mine_a[j];
                V = mine_v[j];
            }
            const int pos = __float_as_int(V.z);
            const int sx = pos & 0xffff, sy = pos >> 16;
            const int ty = sy - R + oy;
            const bool row_ok = j < n && (unsigned)ty < (unsigned)TH;
            const int rowbase = ty * TWP + sx - R;   // target index of offset ox: rowbase + ox
            float w[T];
#pragma unroll
            for (int ox = -R; ox <= R; ++ox) {
                const bool ok = row_ok && (unsigned)(sx - R + ox) < (unsigned)TW;
                w[ox + R] = 0.0f;
                if (ok) {
                    const float4 t = tgt[rowbase + ox];
                    const float e = fmaf(A.x, t.x, fmaf(A.y, t.y, fmaf(A.z, t.z,
                                         A.w + a.sp[(oy + R) * (2 * kMaxR + 1) + ox + R])));
                    w[ox + R] = ex2_approx(e);
                }
            }
#pragma unroll
            for (int ox = -R; ox <= R; ++ox) {
                const bool ok = row_ok && (unsigned)(sx - R + ox) < (unsigned)TW;
                if (ok) {
                    red_shared_add(an0 + 4u * (uint32_t)(rowbase + ox), w[ox + R] * V.x);
                    red_shared_add(ad0 + 4u * (uint32_t)(rowbase + ox), SRC == SRC_COARSE ? w[ox + R] * V.y : w[ox + R]);
                }
            }
        }
        __syncthreads();
    }

    // ---- outputs: thread (lane, warp) owns column lane, rows warp * KP .. + KP - 1
    const int rbase = warp * KP;
    bool val[KP];
    float out[KP];
    uint32_t slow = 0u;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const int ty = rbase + k;
        uint32_t any = 0u;
#pragma unroll
        for (int sy = 0; sy < T; ++sy) any |= (uint32_t)(rowmask[ty + sy] >> lane) & TMASK;
        val[k] = any != 0u;
        const float num = acc_n[ty * TWP + lane], den = acc_d[ty * TWP + lane];
        out[k] = 0.0f;
        if (val[k]) {
            if (den >= 0x1p-60f) out[k] = __fdividef(num, den);
            else slow |= 1u << k;
        }
    }
    mark_rows(val, rbase);
    // rare: a valid pixel whose weight sum is too small, by a gather with the largest exponent of
    // its window shifted to 0 (Eq. (1) in the plain difference form)
    while (slow) {
        const int k = __ffs(slow) - 1;
        slow &= slow - 1u;
        float cr0, cg0, cb0;
        colour(rbase + k + R, lane + R, cr0, cg0, cb0);
        auto tap = [&](int dy, int dx, float &arg, float &wd, float &wb) -> bool {
            const int sy = rbase + k + dy, sx = lane + dx;
            if (!((rowmask[sy] >> sx) & 1u)) return false;
            float r, g, b;
            colour(sy, sx, r, g, b);
            if (SRC == SRC_COARSE) {
                wd = cs[sy * G::S_BX + sx - R + G::S_LEAD];
                wb = cg[sy * SW + sx].w;
            } else {
                wd = __uint_as_float(zraw[sy * G::Z_BX + sx - R + G::Z_LEAD]);
                wb = 1.0f;
            }
            const float dr = r - cr0, dg = g - cg0, db = b - cb0;
            const float n2 = fmaf(dr, dr, fmaf(dg, dg, db * db));
            arg = fmaf(n2, -kc, a.sp[dy * (2 * kMaxR + 1) + dx]);
            return true;
        };
        float amax = -__int_as_float(0x7F800000);
#pragma unroll 1
        for (int dy = 0; dy < T; ++dy)
#pragma unroll 1
            for (int dx = 0; dx < T; ++dx) {
                float arg, wd, wb;
                if (tap(dy, dx, arg, wd, wb)) amax = fmaxf(amax, arg);
            }
        float nn = 0.0f, dd = 0.0f;
#pragma unroll 1
        for (int dy = 0; dy < T; ++dy)
#pragma unroll 1
            for (int dx = 0; dx < T; ++dx) {
                float arg, wd, wb;
                if (tap(dy, dx, arg, wd, wb)) {
                    const float wt = ex2_approx(arg - amax);
                    nn = fmaf(wt, wd, nn);
                    dd = fmaf(wt, wb, dd);
                }
            }
        out[k] = nn / dd;
    }
#pragma unroll
    for (int k = 0; k < KP; ++k) store(k, out[k], val[k]);
}

}  // namespace dz
