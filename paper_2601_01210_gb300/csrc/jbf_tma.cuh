// Joint bilateral filter (Eq. (1)-(4)), gather form, with the input tiles
// staged by TMA.
//
// Same arithmetic as jbf_core.cuh; what changes is how a tile reaches shared
// memory. The kernel is persistent (a multiple of the SM count of CTAs, each
// walking tiles t = blockIdx.x + i * gridDim.x across all frames of the
// batch). Thread 0 issues the 2-D bulk tensor copies (cp.async.bulk.tensor,
// no multicast) of tile i+1 into the second of two raw buffers while the CTA
// filters tile i, so global-memory latency is hidden behind the ALU work.
//
// Sources:
//   SRC_UP     second stage: raw RGB bytes of the full-resolution tile + halo,
//              and the first-stage result (float2 depth, validity) on the
//              coarse grid; restored by nearest-neighbour indexing (x / 3).
//   SRC_ZBUF   single stage: raw RGB bytes and the z-buffer tile.
//   SRC_COARSE first stage: pooled guide (float4 r, g, b, count) and pooled
//              depth sums (float); used in place, no conversion.
// For SRC_UP / SRC_ZBUF a conversion pass writes each staged neighbour as one
// float4 (r, g, b, depth); an unobserved neighbour gets the colour 1e18, so
// its weight 2^(-kc * 1e36 ...) is exactly 0 and the weight sum needs no mask
// multiply. The centre colour of each output pixel is read from the raw bytes.
//
// Bounded waits: every mbarrier wait gives up after kWaitCycles SM clocks
// (about 2 s); the CTA then sets bit 0 of the batch status word, waits (again
// bounded) for its own copies in flight and leaves. The host reports the
// status as a CUDA error of the batch.
//
// FP16 form (HALF = true; second stage and single stage): the staged neighbour
// keeps its colour as three half2 (r, r), (g, g), (b, b) and its depth as
// float. Each thread pairs output rows (2j, 2j+1) of its column: one staged
// neighbour at row iy is tap (iy - 2j, dx) of the first pixel and tap
// (iy - 2j - 1, dx) of the second, so colour difference, squared distance,
// exponent and ex2 run once in half2 for both; the spatial term of a half whose
// row offset falls outside the window is -inf (weight exactly 0). The weights
// are widened to FP32 and the numerator and weight sum accumulate in FP32.
// Unobserved neighbours carry the half colour 65504: the squared difference
// overflows to +inf and the weight is exactly 0. Pixels whose weight sum is
// below 2^-6 (dominant weight in the half subnormal range) are recomputed in
// FP32 with shifted exponents.
//
// Expanded FP32 forms: FORM_EXP expands the squared colour distance into a dot
// product (per-neighbour factors staged once, see the tap loop); FORM_EXP_PAIRS
// runs the same arithmetic on 64-column tiles, two output columns per thread in
// packed two-lane FP32 instructions (pair_tile, jbf_pair.cuh). The scheduling,
// copies and waits below are shared by all forms.
#pragma once

#include <cuda_fp16.h>

#include "jbf_core.cuh"
#include "jbf_pair.cuh"
#include "jbf_sparse.cuh"
#include "tma_common.cuh"

namespace dz {

// FP16 staged record -> FP32 colour and depth (sentinel colour: unobserved).
__device__ __forceinline__ bool half_record(const uint4 &q, float &r, float &g, float &b, float &d) {
    r = __low2float(*reinterpret_cast<const __half2 *>(&q.x));
    g = __low2float(*reinterpret_cast<const __half2 *>(&q.y));
    b = __low2float(*reinterpret_cast<const __half2 *>(&q.z));
    d = __uint_as_float(q.w);
    return r < 65000.0f;
}

// Resident CTAs per SM the compiler is asked to fit (registers): 16 warps per SM; 32 for the
// paired form at two rows per thread, whose state fits 64 registers; 24 for the scalar expanded
// form at two rows per thread, whose state fits 80 (the pooled first stage's 32 x 16 tiles: three
// CTAs of 8 warps ran 70 us against 75 us at two CTAs on 8 1080p frames); 8 for the paired form
// at eight rows per thread, whose state needs more than 128.
constexpr int tma_min_ctas(int form, int kp, int nw) {
    return (form == FORM_EXP_PAIRS && kp == 2   ? 32
            : form == FORM_EXP && kp == 2       ? 24
            : form == FORM_EXP_PAIRS && kp == 8 ? 8
                                                : 16) /
           nw;
}


// A frame's outputs as the filter writes them, copied into shared memory once per CTA: the outputs
// of a tile then wait on no read of the frame descriptor.
struct TileOut {
    float *depth;      // full-resolution output depth and validity
    uint8_t *valid;
    float2 *s1;        // first of two stages: pooled result and validity, and its optional copies
    float *cdepth;
    uint8_t *cvalid;
    int32_t *flags2;   // first of two stages: the second stage's tile flags
    int64_t cpitch;
    int32_t gw, gh;    // the stage's grid
    int32_t W, H;      // full resolution
};

template <int SRC, int R, int KP, int FORM = FORM_FP32, int NW = 8>
__global__ void __launch_bounds__(NW * 32, tma_min_ctas(FORM, KP, NW)) jbf_tma_kernel(const BatchDev *__restrict__ B,
                                                                           const StageArgs a) {
    constexpr bool HALF = FORM == FORM_FP16, EXP = FORM == FORM_EXP;
    using G = TmaGeom<SRC, R, KP, NW, FORM>;
    constexpr int TW = G::TW, TH = G::TH, SW = G::SW, SH = G::SH, T = 2 * R + 1;
    constexpr int NT = NW * 32;   // threads
    static_assert(!HALF || (SRC != SRC_COARSE && KP % 2 == 0), "FP16 form: full-resolution stages, row pairs");
    extern __shared__ __align__(128) uint8_t smem[];
    // raw buffer b: A part at smem + b * (RAW_A + RAW_B), B part right after it
    auto rawA = [&](int b) { return smem + G::OFF_RAW + b * (G::RAW_A + G::RAW_B); };
    auto rawB = [&](int b) { return smem + G::OFF_RAW + b * (G::RAW_A + G::RAW_B) + G::RAW_A; };
    float4 *staged = reinterpret_cast<float4 *>(smem + G::OFF_STAGED);
    uint4 *staged_h = reinterpret_cast<uint4 *>(smem + G::OFF_STAGED);   // FP16 records, same 16 bytes
    float *staged_g = reinterpret_cast<float *>(smem + G::OFF_G);         // expanded form: F_q times depth
    uint32_t *obsw = reinterpret_cast<uint32_t *>(smem + G::OFF_OBS);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + G::OFF_BAR);

    // every tile of the stage; tile_mark_kernel flagged those that some observation reaches
    const int stage = SRC == SRC_UP ? 1 : 0;
    const int32_t *pre = stage ? B->t2_pre : B->t1_pre;
    const int nf = B->n_frames;
    const int total = pre[nf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // Tiles are handed out dynamically: a CTA starts with tile blockIdx.x and takes every further
    // tile from the stage's counter (gridDim.x + atomicAdd), so CTAs stay balanced however the
    // tiles without observations are placed. Thread 0 issues the copies of the CTA's next tile
    // while the CTA works on the current one: it takes the tile and reads its flag one tile ahead,
    // acquires each frame's tensor maps once, and leaves the tile's (frame, x0, y0, copies issued,
    // tile index or -1 when there is none) in s_tile[buffer] for the other threads, so the start of
    // a tile waits on no global load. A tile no observation reaches gets no copies.
    __shared__ int s_tile[2][5];
    // The stage's tile prefix and each frame's tiles per row and tile flags, read into shared
    // memory once: locating a tile then waits on no global load. A wait in thread 0's queue work
    // would hold up warp 0, and with it every warp of the CTA at the tile's closing barrier.
    // The same holds for each frame's outputs and the second stage's tile geometry (s_mk: width,
    // height, radius; height 0: no flags to set).
    __shared__ int32_t s_pre[kMaxBatch + 1];
    __shared__ int32_t s_tx[kMaxBatch];
    __shared__ const int32_t *s_fl[kMaxBatch];
    __shared__ TileOut s_out[kMaxBatch];
    __shared__ int32_t s_mk[3];
    for (int i = threadIdx.x; i <= nf; i += NT) s_pre[i] = pre[i];
    for (int i = threadIdx.x; i < nf; i += NT) {
        const FrameDev &F = B->f[i];
        const int gw = SRC == SRC_COARSE ? F.Wc : F.W, gh = SRC == SRC_COARSE ? F.Hc : F.H;
        s_tx[i] = (gw + TW - 1) / TW;
        s_fl[i] = F.tflags[stage];
        TileOut &O = s_out[i];
        O.depth = F.flt_depth;
        O.valid = F.flt_valid;
        O.s1 = F.s1;
        O.cdepth = F.out_coarse;
        O.cvalid = F.out_coarse_valid;
        O.flags2 = F.tflags[1];
        O.cpitch = F.cpitch;
        O.gw = gw;
        O.gh = gh;
        O.W = F.W;
        O.H = F.H;
    }
    if (threadIdx.x == 0) {
        s_mk[0] = B->tl_tw[1];
        s_mk[1] = SRC == SRC_COARSE ? B->tl_th[1] : 0;
        s_mk[2] = B->tl_r[1];
    }
    __syncthreads();
    auto locate = [&](int item, int &fi, int &x0, int &y0) {
        fi = find_segment(s_pre, nf, item);
        const int tiles_x = s_tx[fi];
        const int t = item - s_pre[fi];
        x0 = (t % tiles_x) * TW;
        y0 = (t / tiles_x) * TH;
    };
    // the tile's coordinates (fi, x0, y0) were located beforehand
    auto issue = [&](int item, int flag, int fi, int x0, int y0, int buf) {
        s_tile[buf][4] = item < total ? item : -1;
        if (item >= total) return;
        s_tile[buf][0] = fi;
        s_tile[buf][1] = x0;
        s_tile[buf][2] = y0;
        s_tile[buf][3] = flag != 0;
        if (!flag) return;
        const FrameDev &F = B->f[fi];
        mbar_expect_tx(&bar[buf], G::TX_BYTES);
        if (SRC == SRC_COARSE) {
            tma_load_2d(rawA(buf), &F.tm[TM_CGUIDE], 4 * (x0 - R), y0 - R, &bar[buf]);
            tma_load_2d(rawB(buf), &F.tm[TM_CSSUM], x0 - G::S_LEAD, y0 - R, &bar[buf]);
        } else {
            tma_load_2d(rawA(buf), &F.tm[TM_RGB], 3 * x0 - G::RGB_LEAD, y0 - R, &bar[buf]);
            if (SRC == SRC_UP)
                tma_load_2d(rawB(buf), &F.tm[TM_S1], floor_div3(x0 - R) & ~1, floor_div3(y0 - R), &bar[buf]);
            else
                tma_load_2d(rawB(buf), &F.tm[TM_ZBUF], x0 - G::Z_LEAD, y0 - R, &bar[buf]);
        }
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
        obsw[G::OBS_WORDS - 1] = 0u;   // guard words, never rewritten
        if (G::PAIRS) obsw[G::OBS_ONE / 4 + G::OBS_WORDS - 1] = 0u;
        // the tensor maps of every frame of the batch, acquired once before thread 0 has any memory
        // operation outstanding (a fence later in the loop would wait for its stores and atomics)
        for (int f = 0; f < nf; ++f) {
            const FrameDev &F = B->f[f];
            if (SRC == SRC_COARSE) {
                tmap_acquire(&F.tm[TM_CGUIDE]);
                tmap_acquire(&F.tm[TM_CSSUM]);
            } else {
                tmap_acquire(&F.tm[TM_RGB]);
                tmap_acquire(SRC == SRC_UP ? &F.tm[TM_S1] : &F.tm[TM_ZBUF]);
            }
        }
    }
    __syncthreads();
    uint32_t inflight = 0u;   // bit b: thread 0 issued copies into buffer b not yet consumed
    uint32_t phase = 0u;      // bit b: parity of buffer b's barrier
    // Thread 0 keeps the next tile n1 ready (its flag f1 requested and its coordinates located)
    // and the counter's reply for the tile after it (n2raw) requested. At the top of a tile it
    // only issues n1's copies; the queue advances after the conversion barrier, while the CTA
    // filters, and every global result is used one tile after it was requested: the flag load
    // and the counter's reply land in registers (a store of either to shared memory would wait
    // for it), so the issuing thread never waits on a load or on the counter, which a whole grid
    // of CTAs shares. The counter is only ever touched atomically (the descriptor's other fields
    // are read-only here).
    __shared__ int s_q[4];   // thread 0's queue state, kept out of every thread's registers
    int &n1 = s_q[0], &l1f = s_q[1], &l1x = s_q[2], &l1y = s_q[3];
    int f1 = 0, n2raw = 0;
    if (threadIdx.x == 0) {
        n1 = total;
        l1f = l1x = l1y = 0;
    }
    auto request = [&]() { return atomicAdd(const_cast<int32_t *>(&B->tl_next[stage]), 1); };
    auto advance = [&]() {   // thread 0: n1 <- the counter's last reply; request the next one
        n1 = (int)gridDim.x + n2raw;
        if (n1 < total) {
            locate(n1, l1f, l1x, l1y);
            f1 = load_issue(s_fl[l1f] + (n1 - s_pre[l1f]));
            n2raw = request();
        }
    };
    if (threadIdx.x == 0) {
        const int t0 = blockIdx.x;
        if (t0 < total) {
            int fi, x0, y0;
            locate(t0, fi, x0, y0);
            const int f0 = s_fl[fi][t0 - s_pre[fi]];
            issue(t0, f0, fi, x0, y0, 0);
            if (f0) inflight |= 1u;
            n2raw = request();
            advance();
        } else {
            s_tile[0][4] = -1;
        }
    }
    __syncthreads();          // s_tile[0]
    for (int it = 0;; ++it) {
        const int buf = it & 1;
        if (s_tile[buf][4] < 0) break;   // the same for every thread of the CTA
        if (threadIdx.x == 0) {   // the other buffer was released by the last barrier
            issue(n1, f1, l1f, l1x, l1y, buf ^ 1);
            if (n1 < total && f1) inflight |= 1u << (buf ^ 1);
        }
        const bool copied = s_tile[buf][3] != 0;   // the same for every thread of the CTA
        // A wait that gives up makes its warp skip the conversion; the barrier that publishes the
        // staged records ORs the warps' failures, and on a failure the CTA leaves there (leave()).
        // No barrier sits between the tiles' copies and the conversion.
        bool bad = false;
        if (copied) {
            const bool ok = mbar_wait_bounded(&bar[buf], (phase >> buf) & 1u);
            bad = !__all_sync(0xffffffffu, ok);
            if (ok) {
                phase ^= 1u << buf;
                inflight &= ~(1u << buf);
            }
        }
        // after a failed wait: record it and let the CTA's own copies land before it returns
        auto leave = [&]() {
            if (threadIdx.x == 0) {
                atomicOr(B->status, 1);
                for (int b = 0; b < 2; ++b)
                    if ((inflight >> b) & 1u) mbar_wait_bounded(&bar[b], (phase >> b) & 1u);
            }
        };

        const int fi = s_tile[buf][0], x0 = s_tile[buf][1], y0 = s_tile[buf][2];
        const TileOut &O = s_out[fi];
        const int gw = O.gw, gh = O.gh;
        if (!copied) {   // no observation reaches the tile: every output is (0, invalid)
            if (threadIdx.x == 0 && n1 < total) advance();
            for (int i = threadIdx.x; i < TW * TH; i += NT) {
                const int x = x0 + i % TW, y = y0 + i / TW;
                if (x >= gw || y >= gh) continue;
                const int64_t o = (int64_t)y * gw + x;
                if (SRC == SRC_COARSE) {
                    O.s1[(int64_t)y * O.cpitch + x] = make_float2(0.0f, 0.0f);
                    if (O.cdepth) O.cdepth[o] = 0.0f;
                    if (O.cvalid) O.cvalid[o] = 0;
                } else {
                    O.depth[o] = 0.0f;
                    O.valid[o] = 0;
                }
            }
            __syncthreads();   // s_tile[buf] is rewritten for the tile after next
            continue;
        }
        if constexpr (G::PAIRS) {
            if (pair_tile<SRC, R, KP, NW>(O.depth, O.valid, a, x0, y0, gw, gh, rawA(buf), rawB(buf), smem, bad, [&]() {
                    if (threadIdx.x == 0 && n1 < total) advance();   // off the path of the CTA's barriers
                })) {
                leave();
                return;
            }
            __syncthreads();   // staged records / raw[buf] are reused by the next tile
            continue;
        }
        if constexpr (G::SPARSE) {
            static_assert(SRC == SRC_ZBUF, "sparse form: the single stage on the z-buffer");
            float *const out_depth = O.depth;
            uint8_t *const out_valid = O.valid;
            auto store = [&](int tx, int ty, float out, bool v) {
                const int x = x0 + tx, y = y0 + ty;
                if (x < gw && y < gh) {
                    const int64_t o = (int64_t)y * gw + x;
                    out_depth[o] = out;
                    out_valid[o] = v;
                }
            };
            if (sparse_tile<R, KP, NW, FORM == FORM_SPARSE_FP16>(a, x0, y0, gw, gh, rawA(buf), rawB(buf), smem, bad, [&]() {
                    if (threadIdx.x == 0 && n1 < total) advance();   // off the path of the CTA's barriers
                }, store)) {
                leave();
                return;
            }
            __syncthreads();   // records and raw[buf] are reused by the next tile
            continue;
        }
        const uint8_t *rgbraw = rawA(buf);
        const float4 *cg = reinterpret_cast<const float4 *>(rawA(buf));
        const float *cs = reinterpret_cast<const float *>(rawB(buf));

        // ---- conversion and observation map
        // staged position (sy, sx): colour bytes in the raw RGB box, depth and observation
        // from the raw first-stage box (SRC_UP) or z-buffer box (SRC_ZBUF)
        const int cx0 = floor_div3(x0 - R) & ~1, cy0 = floor_div3(y0 - R);
        const float2 *craw = reinterpret_cast<const float2 *>(rawB(buf));
        const uint32_t *zraw = reinterpret_cast<const uint32_t *>(rawB(buf));
        auto rgb_at = [&](int sy, int sx) { return rgbraw + sy * G::RGB_BX + 3 * sx - 3 * R + G::RGB_LEAD; };
        auto depth_of = [&](int sy, int sx, float &d) -> bool {
            const int gx = x0 - R + sx, gy = y0 - R + sy;
            if (gx < 0 || gx >= gw || gy < 0 || gy >= gh) return false;
            if (SRC == SRC_UP) {
                const float2 c = craw[((int)((unsigned)gy / 3u) - cy0) * G::C_BX + ((int)((unsigned)gx / 3u) - cx0)];
                d = c.x;
                return c.y > 0.0f;
            }
            const uint32_t z = zraw[sy * G::Z_BX + sx - R + G::Z_LEAD];
            d = __uint_as_float(z);
            return z != kEmpty;
        };
        // Every thread converts positions threadIdx.x + j * NT in two unrolled passes: first every
        // load of its positions (raw boxes; shared-memory stores in between would keep the compiler
        // from overlapping them), then the records; a warp's ballot gives one word of the
        // observation bitmap.
        if (!bad) {   // (a warp whose copies did not land skips its conversion)
            uint32_t omask = 0u;                     // bit j: position j observed
            float dq[G::NCONV];                      // depth (SRC_UP / SRC_ZBUF) or depth sum (SRC_COARSE)
            uint32_t c0[G::NCONV], c1[G::NCONV], c2[G::NCONV];   // colour bytes, or guide bits (SRC_COARSE)
            float cw[G::NCONV];                      // pooled count (SRC_COARSE)
    #pragma unroll
            for (int j = 0; j < G::NCONV; ++j) {
                const int i = threadIdx.x + j * NT;
                dq[j] = 0.0f;
                c0[j] = c1[j] = c2[j] = 0u;
                cw[j] = 0.0f;
                if (i < SH * SW) {
                    const int sy = i / SW, sx = i - sy * SW;
                    if (SRC != SRC_COARSE) {
                        float d = 0.0f;
                        if (depth_of(sy, sx, d)) omask |= 1u << j;
                        dq[j] = d;
                        const uint8_t *p = rgb_at(sy, sx);
                        c0[j] = p[0];
                        c1[j] = p[1];
                        c2[j] = p[2];
                    } else {
                        const float4 q = cg[i];
                        c0[j] = __float_as_uint(q.x);
                        c1[j] = __float_as_uint(q.y);
                        c2[j] = __float_as_uint(q.z);
                        cw[j] = q.w;
                        if (q.w > 0.0f) omask |= 1u << j;
                        if (EXP) dq[j] = cs[sy * G::S_BX + sx - R + G::S_LEAD];
                    }
                }
            }
            // byte b as an exact float minus bias: 2^23 + b has b in its low mantissa bits
            auto bytef = [](uint32_t b, float bias) { return __uint_as_float(0x4B000000u | b) - (8388608.0f + bias); };
    #pragma unroll
            for (int j = 0; j < G::NCONV; ++j) {
                const int i = threadIdx.x + j * NT;
                const bool o = (omask >> j) & 1u;
                if (i < SH * SW) {
                    if (SRC != SRC_COARSE) {
                        const float d = dq[j];
                        if (HALF) {
                            staged_h[i] = o ? make_uint4(h2u(__float2half2_rn(bytef(c0[j], 0.0f))),
                                                         h2u(__float2half2_rn(bytef(c1[j], 0.0f))),
                                                         h2u(__float2half2_rn(bytef(c2[j], 0.0f))), __float_as_uint(d))
                                            : make_uint4(h2u(__float2half2_rn(65504.0f)), 0u, 0u, 0u);
                        } else if (EXP) {
                            // centred colour (exact), F_q = 2^(-kc |c'_q|^2); unobserved: F_q = 0
                            const float rr = bytef(c0[j], 128.0f), gg = bytef(c1[j], 128.0f), bb = bytef(c2[j], 128.0f);
                            const float f = o ? ex2_approx(-a.kc * fmaf(rr, rr, fmaf(gg, gg, bb * bb))) : 0.0f;
                            staged[i] = o ? make_float4(rr, gg, bb, f) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                            staged_g[i] = o ? f * d : 0.0f;   // an empty z-buffer cell holds +inf
                        } else {
                            staged[i] = o ? make_float4(bytef(c0[j], 0.0f), bytef(c1[j], 0.0f), bytef(c2[j], 0.0f), d)
                                          : make_float4(kSentinel, 0.0f, 0.0f, 0.0f);
                        }
                    } else if (EXP) {   // pooled guide: F_q times the count and times the depth sum (count 0: weight 0)
                        const float rr = __uint_as_float(c0[j]) - 128.0f, gg = __uint_as_float(c1[j]) - 128.0f,
                                    bb = __uint_as_float(c2[j]) - 128.0f;
                        const float f = ex2_approx(-a.kc * fmaf(rr, rr, fmaf(gg, gg, bb * bb)));
                        staged[i] = make_float4(rr, gg, bb, f * cw[j]);
                        staged_g[i] = f * dq[j];
                    }
                }
                const uint32_t bits = __ballot_sync(0xffffffffu, o);
                if (lane == 0) obsw[(threadIdx.x + j * NT) >> 5] = bits;
            }
        }
        if (__syncthreads_or(bad)) {
            leave();
            return;
        }

        if (threadIdx.x == 0 && n1 < total) advance();   // off the path of the CTA's barriers

        // ---- filter: thread owns column lane, rows rbase .. rbase + KP - 1 of the tile
        const int rbase = warp * KP;
        float cr[KP], cgr[KP], cb[KP], num[KP], den[KP];
        float sq[HALF ? KP : 1];   // FP16 form: weighted sum of squared depths (the error bound below)
        bool val[KP];
        bool any_val = false;
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            if (SRC == SRC_COARSE) {
                const float4 c = cg[(rbase + k + R) * SW + lane + R];
                cr[k] = c.x; cgr[k] = c.y; cb[k] = c.z;
            } else if (!HALF) {
                const uint8_t *p = rgbraw + (rbase + k + R) * G::RGB_BX + 3 * lane + G::RGB_LEAD;
                cr[k] = (float)p[0]; cgr[k] = (float)p[1]; cb[k] = (float)p[2];
            }
            num[k] = 0.0f;
            den[k] = 0.0f;
            if (HALF) sq[k] = 0.0f;
        }
        uint32_t rows_warp;   // bit iy: some lane's window of staged row rbase + iy holds an observation
        {
            uint32_t rows = 0;   // bit iy: an observation in staged row rbase + iy, columns lane .. lane + 2R
#pragma unroll
            for (int iy = 0; iy < KP + 2 * R; ++iy) {
                const int bit = (rbase + iy) * SW + lane;   // the window never leaves its row
                const uint32_t win = __funnelshift_r(obsw[bit >> 5], obsw[(bit >> 5) + 1], bit & 31);
                rows |= ((win & ((1u << T) - 1u)) != 0 ? 1u : 0u) << iy;
            }
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                val[k] = ((rows >> k) & ((1u << T) - 1u)) != 0;
                any_val |= val[k];
            }
            rows_warp = __reduce_or_sync(0xffffffffu, rows);
        }
        if (HALF && __any_sync(0xffffffffu, any_val)) {
            // centre colours of row pairs (2j, 2j+1) as half2
            __half2 cr2[KP / 2], cg2[KP / 2], cb2[KP / 2];
#pragma unroll
            for (int j = 0; j < KP / 2; ++j) {
                const uint8_t *p0 = rgbraw + (rbase + 2 * j + R) * G::RGB_BX + 3 * lane + G::RGB_LEAD;
                const uint8_t *p1 = p0 + G::RGB_BX;
                cr2[j] = __floats2half2_rn((float)p0[0], (float)p1[0]);
                cg2[j] = __floats2half2_rn((float)p0[1], (float)p1[1]);
                cb2[j] = __floats2half2_rn((float)p0[2], (float)p1[2]);
            }
            const __half2 kc2 = h2bits(a.kc2);
#pragma unroll
            for (int iy = 0; iy < KP + 2 * R; ++iy) {
#pragma unroll
                for (int dx = 0; dx < T; ++dx) {
                    const uint4 q = staged_h[(rbase + iy) * SW + lane + dx];
                    const __half2 qr = h2bits(q.x), qg = h2bits(q.y), qb = h2bits(q.z);
                    const float qd = __uint_as_float(q.w), qd2 = qd * qd;
#pragma unroll
                    for (int j = 0; j < KP / 2; ++j) {
                        const int d = iy - 2 * j;   // row offset of the pair's first pixel
                        if (d >= 0 && d <= T) {
                            const __half2 dr = __hsub2(qr, cr2[j]), dg = __hsub2(qg, cg2[j]), db = __hsub2(qb, cb2[j]);
                            const __half2 n2 = __hfma2(dr, dr, __hfma2(dg, dg, __hmul2(db, db)));
                            const __half2 w2 = h2exp2_approx(__hfma2(n2, kc2, h2bits(a.sp2[d * (2 * kMaxR + 1) + dx])));
                            const float2 w = __half22float2(w2);
                            num[2 * j] = fmaf(w.x, qd, num[2 * j]);
                            den[2 * j] += w.x;
                            sq[2 * j] = fmaf(w.x, qd2, sq[2 * j]);
                            num[2 * j + 1] = fmaf(w.y, qd, num[2 * j + 1]);
                            den[2 * j + 1] += w.y;
                            sq[2 * j + 1] = fmaf(w.y, qd2, sq[2 * j + 1]);
                        }
                    }
                }
            }
        } else if (EXP && __any_sync(0xffffffffu, any_val)) {
            // exponent 2 kc c'_p . c'_q - kc |c'_p|^2 + ex_sy[dy]; weight times F_q ex_sx[dx]
            const float kc = a.kc, kc2 = 2.0f * a.kc;
            float ar[KP], ag[KP], ab[KP], cp[KP];
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const float rr = cr[k] - 128.0f, gg = cgr[k] - 128.0f, bb = cb[k] - 128.0f;
                ar[k] = kc2 * rr;
                ag[k] = kc2 * gg;
                ab[k] = kc2 * bb;
                cp[k] = -kc * fmaf(rr, rr, fmaf(gg, gg, bb * bb));
            }
#pragma unroll
            for (int iy = 0; iy < KP + 2 * R; ++iy) {
                // a staged row no lane's window observes adds exact zeros (F q = 0): skip it
                if (!((rows_warp >> iy) & 1u)) continue;
                float dd[KP];
#pragma unroll
                for (int k = 0; k < KP; ++k) {
                    const int dy = iy - k;
                    dd[k] = (dy >= 0 && dy < T) ? cp[k] + a.ex_sy[dy] : 0.0f;
                }
#pragma unroll
                for (int dx = 0; dx < T; ++dx) {
                    const int o = (rbase + iy) * SW + lane + dx;
                    const float4 q = staged[o];
                    const float fx = q.w * a.ex_sx[dx], gx = staged_g[o] * a.ex_sx[dx];
#pragma unroll
                    for (int k = 0; k < KP; ++k) {
                        const int dy = iy - k;
                        if (dy >= 0 && dy < T) {
                            const float w = ex2_approx(fmaf(ar[k], q.x, fmaf(ag[k], q.y, fmaf(ab[k], q.z, dd[k]))));
                            num[k] = fmaf(w, gx, num[k]);
                            den[k] = fmaf(w, fx, den[k]);
                        }
                    }
                }
            }
        } else if (!HALF && !EXP && __any_sync(0xffffffffu, any_val)) {
            const float kc = a.kc;
#pragma unroll
            for (int iy = 0; iy < KP + 2 * R; ++iy) {
#pragma unroll
                for (int dx = 0; dx < T; ++dx) {
                    float4 q;
                    float qs = 0.0f;
                    if (SRC == SRC_COARSE) {
                        q = cg[(rbase + iy) * SW + lane + dx];
                        qs = cs[(rbase + iy) * G::S_BX + lane + dx - R + G::S_LEAD];
                    } else {
                        q = staged[(rbase + iy) * SW + lane + dx];
                    }
#pragma unroll
                    for (int k = 0; k < KP; ++k) {
                        const int dy = iy - k;
                        if (dy >= 0 && dy < T) {
                            const float dr = q.x - cr[k], dg = q.y - cgr[k], db = q.z - cb[k];
                            const float n2 = fmaf(dr, dr, fmaf(dg, dg, db * db));
                            const float w = ex2_approx(fmaf(n2, -kc, a.sp[dy * (2 * kMaxR + 1) + dx]));
                            if (SRC == SRC_COARSE) {
                                num[k] = fmaf(w, qs, num[k]);
                                den[k] = fmaf(w, q.w, den[k]);
                            } else {
                                num[k] = fmaf(w, q.w, num[k]);
                                den[k] += w;
                            }
                        }
                    }
                }
            }
        }
        const int x = x0 + lane;
        float2 *const out_s1 = O.s1;
        const int64_t cpitch = O.cpitch;
        float *const out_coarse = O.cdepth, *const out_depth = O.depth;
        uint8_t *const out_coarse_valid = O.cvalid, *const out_valid = O.valid;
        auto store = [&](int k, float out, bool v) {
            const int y = y0 + rbase + k;
            if (x < gw && y < gh) {
                const int64_t o = (int64_t)y * gw + x;
                if (SRC == SRC_COARSE) {
                    out_s1[(int64_t)y * cpitch + x] = make_float2(out, v ? 1.0f : 0.0f);
                    if (out_coarse) out_coarse[o] = out;
                    if (out_coarse_valid) out_coarse_valid[o] = v;
                } else {
                    out_depth[o] = out;
                    out_valid[o] = v;
                }
            }
        };
        if (SRC == SRC_COARSE && s_mk[1] > 0) {   // flag the second-stage tiles the valid pixels reach
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
                mark_reach(O.flags2, s_mk[0], s_mk[1], s_mk[2], a.pool, O.W, O.H, x0 + __ffs(cols) - 1,
                           x0 + 31 - __clz(cols), y0 + rbase + kf, y0 + rbase + kl, lane);
        }
        uint32_t slow = 0u;   // bit k: valid pixel whose weight sum is too small for the plain form
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            if (val[k] && !(den[k] >= (HALF ? 0x1p-6f : 0x1p-60f))) {
                slow |= 1u << k;
                continue;
            }
            const float out = val[k] ? __fdividef(num[k], den[k]) : 0.0f;
            if (HALF && val[k]) {
                // FP16 weights carry a relative error of at most kHalfWeightErr (exponents rounded in
                // half precision); the depth error is then at most kHalfWeightErr times the weighted
                // standard deviation of the window's depths (Cauchy-Schwarz over the weights). Where that
                // bound could exceed half of 1e-3 of the depth, the pixel is recomputed in FP32.
                const float var = __fdividef(sq[k], den[k]) - out * out;
                const float lim = kHalfStdFrac * out;
                if (var > lim * lim) {
                    slow |= 1u << k;
                    continue;
                }
            }
            store(k, out, val[k]);
        }
        // shifted recomputation in FP32 (rare): largest exponent of the window first
        while (slow) {
            const int k = __ffs(slow) - 1;
            slow &= slow - 1u;
            float cr0, cg0, cb0;
            if (SRC == SRC_COARSE) {
                const float4 c = cg[(rbase + k + R) * SW + lane + R];
                cr0 = c.x; cg0 = c.y; cb0 = c.z;
            } else {
                const uint8_t *p = rgbraw + (rbase + k + R) * G::RGB_BX + 3 * lane + G::RGB_LEAD;
                cr0 = (float)p[0]; cg0 = (float)p[1]; cb0 = (float)p[2];
            }
            auto tap = [&](int dy, int dx, float &arg, float &wd, float &wb) -> bool {
                const int o = (rbase + k + dy) * SW + lane + dx;
                float r, g, b;
                bool seen;
                if (SRC == SRC_COARSE) {
                    const float4 q = cg[o];
                    r = q.x; g = q.y; b = q.z;
                    seen = q.w > 0.0f;
                    wd = cs[(rbase + k + dy) * G::S_BX + lane + dx - R + G::S_LEAD];
                    wb = q.w;
                } else if (HALF) {
                    seen = half_record(staged_h[o], r, g, b, wd);
                    wb = 1.0f;
                } else if (EXP) {   // from the raw boxes
                    const int sy = rbase + k + dy, sx = lane + dx;
                    const uint8_t *p = rgb_at(sy, sx);
                    r = (float)p[0]; g = (float)p[1]; b = (float)p[2];
                    wd = 0.0f;
                    seen = depth_of(sy, sx, wd);
                    wb = 1.0f;
                } else {
                    const float4 q = staged[o];
                    r = q.x; g = q.y; b = q.z;
                    seen = q.x < 1.0e17f;
                    wd = q.w;
                    wb = 1.0f;
                }
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
                        const float w = ex2_approx(arg - amax);
                        nn = fmaf(w, wd, nn);
                        dd = fmaf(w, wb, dd);
                    }
                }
            store(k, nn / dd, true);
        }
        __syncthreads();   // staged / raw[buf] / hor are reused by the next tile
    }
}

// Tile marks for the TMA filters. One warp per band of 32 columns x kMarkRows
// rows of the observation grid (the pooled grid for SRC_UP and SRC_COARSE, the
// image for SRC_ZBUF); every lane reads its column's kMarkRows observation flags
// (in flight together). The output pixels the band's observations reach (grown
// by the radius; a pooled pixel covers a 3 x 3 block at full resolution for
// SRC_UP) span a range of the stage's tiles (tw x th, row-major per frame), whose
// flags the warp sets. The range spans the band's first to last observed column
// and row, a superset: a flagged tile that no observation reaches is filtered to
// all-invalid outputs, as it should be. The first block also resets the
// filter's tile counter.
constexpr int kMarkThreads = 256, kMarkRows = kMarkBand;
template <int SRC>
__global__ void __launch_bounds__(kMarkThreads) tile_mark_kernel(BatchDev *__restrict__ B, int stage, int th, int r) {
    constexpr int kWarps = kMarkThreads / 32;
    if (blockIdx.x == 0 && threadIdx.x == 0) B->tl_next[stage] = 0;
    const int32_t *mpre = B->mk_pre;
    const int nf = B->n_frames;
    const int total = mpre[nf];
    const int lane = threadIdx.x & 31;
    for (int item = blockIdx.x * kWarps + (threadIdx.x >> 5); item < total; item += gridDim.x * kWarps) {
        const int fi = find_segment(mpre, nf, item);
        const FrameDev &F = B->f[fi];
        const int ow = SRC == SRC_ZBUF ? F.W : F.Wc, oh = SRC == SRC_ZBUF ? F.H : F.Hc;
        const int segs = (ow + 31) / 32;
        const int t = item - mpre[fi];
        const int band = t / segs, sx0 = (t - band * segs) * 32, ox = sx0 + lane, oy0 = band * kMarkRows;
        uint32_t w[kMarkRows];
#pragma unroll
        for (int k = 0; k < kMarkRows; ++k) {
            const int oy = oy0 + k;
            w[k] = SRC == SRC_ZBUF ? kEmpty : 0u;
            if (ox < ow && oy < oh) {
                if (SRC == SRC_UP) w[k] = __float_as_uint(F.s1[(int64_t)oy * F.cpitch + ox].y);
                else if (SRC == SRC_COARSE) w[k] = __float_as_uint(F.cguide[(int64_t)oy * F.cpitch + ox].w);
                else w[k] = F.zbuf[(int64_t)oy * F.zpitch + ox];
            }
        }
        uint32_t rows = 0u;   // bit k: this lane's column is observed in row oy0 + k
#pragma unroll
        for (int k = 0; k < kMarkRows; ++k)
            if (SRC == SRC_ZBUF ? w[k] != kEmpty : __uint_as_float(w[k]) > 0.0f) rows |= 1u << k;
        const uint32_t cols = __ballot_sync(0xffffffffu, rows != 0);
        const uint32_t all = __reduce_or_sync(0xffffffffu, rows);
        if (!cols) continue;
        const int gw = SRC == SRC_COARSE ? F.Wc : F.W, gh = SRC == SRC_COARSE ? F.Hc : F.H;
        const int ox0 = sx0 + __ffs(cols) - 1, ox1 = sx0 + 31 - __clz(cols);
        const int oy1 = oy0 + 31 - __clz(all), oyf = oy0 + __ffs(all) - 1;
        const int f = SRC == SRC_UP ? 3 : 1;   // output pixels per observation pixel and axis
        mark_reach(F.tflags[stage], B->tl_tw[stage], th, r, f, gw, gh, ox0, ox1, oyf, oy1, lane);
    }
}

}  // namespace dz
