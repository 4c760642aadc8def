// Pieces shared by the TMA-staged filter kernels (jbf_tma.cuh, jbf_pair.cuh):
// mbarrier and bulk-tensor-copy wrappers (inline PTX), the bounded wait, and
// the tile geometry that the kernels and the host's tensor-map boxes agree on.
#pragma once

#include <cuda_fp16.h>

#include <cstdint>

#include "desc.cuh"

namespace dz {

constexpr long long kWaitCycles = 4000000000LL;
constexpr float kSentinel = 1.0e18f;

enum { SRC_UP = 0, SRC_ZBUF = 1, SRC_COARSE = 2 };

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Relaxed: the issuing thread's earlier global stores need not be performed first (a release
// arrive waits for them). Nothing is published through this arrive: tile coordinates reach the
// CTA through a barrier, and copies into a buffer are issued only after the barrier that frees it.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.relaxed.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

// A global load issued here and waited for only where its value is first used (the compiler may
// not move a volatile asm, so the load is not sunk to its use).
__device__ __forceinline__ int load_issue(const int32_t *p) {
    int v;
    asm volatile("ld.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void tmap_acquire(const CUtensorMap *m) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)m) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *m, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"((uint64_t)m), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ int floor_div3(int a) { return a >= 0 ? a / 3 : -((2 - a) / 3); }

// half2 <-> its 32 bits, and ex2.approx.f16x2 (the FP16 forms' weights)
__device__ __forceinline__ __half2 h2bits(uint32_t u) { return *reinterpret_cast<const __half2 *>(&u); }
__device__ __forceinline__ uint32_t h2u(__half2 h) { return *reinterpret_cast<const uint32_t *>(&h); }

__device__ __forceinline__ __half2 h2exp2_approx(__half2 x) {
    uint32_t y;
    asm("ex2.approx.f16x2 %0, %1;" : "=r"(y) : "r"(h2u(x)));
    return h2bits(y);
}

// FP16 form: bound on the relative error of a weight (2^(e) with e = -kc |dc|^2 + spatial term
// evaluated in half precision: roundings of kc, of the squared distance and of e, about 2^-10.4 of
// |e| each, for |e| <= 24, plus the ex2.approx.f16 error), and the weighted standard deviation of a
// window's depths, as a fraction of the pixel's depth, above which the pixel is recomputed in FP32
// (kHalfWeightErr * kHalfStdFrac = 5e-4, half the 1e-3 relative bar).
constexpr float kHalfWeightErr = 0.02f;
constexpr float kHalfStdFrac = 5e-4f / kHalfWeightErr;


constexpr int ceil_to(int x, int m) { return (x + m - 1) / m * m; }

// Tile geometry shared by the kernel and the host (tensor-map boxes).
// Arithmetic forms of the kernels (the host's TMA_FORM_* values).
enum { FORM_FP32 = 0, FORM_FP16 = 1, FORM_EXP = 2, FORM_EXP_PAIRS = 3, FORM_SPARSE = 4, FORM_SPARSE_FP16 = 5 };

// Tile geometry shared by the kernels and the host (tensor-map boxes). The
// paired form filters 64-column tiles, a thread taking columns c and c + 32;
// its staged records are slots of SP = 32 + 2R per staged row, slot s holding
// staged columns s and s + 32 side by side. The sparse forms (jbf_sparse.cuh,
// FP32 and FP16 weights) keep a 32-byte record per staged position (written for
// the observed ones)
// and one 64-bit observation mask per staged row.
template <int SRC, int R, int KP, int NW_ = 8, int FORM = FORM_FP32>
struct TmaGeom {
    static constexpr bool EXP = FORM == FORM_EXP, PAIRS = FORM == FORM_EXP_PAIRS;
    static constexpr bool SPARSE = FORM == FORM_SPARSE || FORM == FORM_SPARSE_FP16;
    static constexpr int TW = PAIRS ? 64 : 32, NW = NW_, TH = NW * KP, SW = TW + 2 * R, SH = TH + 2 * R;
    static constexpr int SP = PAIRS ? 32 + 2 * R : SW;   // staged records per staged row
    // RGB bytes: box starts at byte 3*x0 - RGB_LEAD (x0 is a multiple of 32, so 3*x0 of 16)
    static constexpr int RGB_LEAD = ceil_to(3 * R, 16);
    static constexpr int RGB_BX = ceil_to(3 * TW + 3 * R + RGB_LEAD, 16);
    static constexpr int RGB_BY = SH;
    // first-stage result (float2) on the pooled grid, pool 3: rows floor((y0-R)/3) ..
    // floor((y0+TH-1+R)/3); columns from floor((x0-R)/3) rounded down to even
    static constexpr int C_BX = ceil_to(2 + (SW + 1) / 3, 2);
    static constexpr int C_BY = 1 + (SH + 1) / 3;
    // z-buffer (uint32): box starts at x0 - Z_LEAD
    static constexpr int Z_LEAD = ceil_to(R, 4);
    static constexpr int Z_BX = ceil_to(TW + R + Z_LEAD, 4);
    static constexpr int Z_BY = SH;
    // pooled guide (float4, as 4 floats per element) and pooled sums (float, starts at x0 - S_LEAD)
    static constexpr int G_BX = 4 * SW;
    static constexpr int G_BY = SH;
    static constexpr int S_LEAD = ceil_to(R, 4);
    static constexpr int S_BX = ceil_to(TW + R + S_LEAD, 4);
    static constexpr int S_BY = SH;

    // raw buffer bytes (each rounded to 128 for TMA destination alignment)
    static constexpr int RAW_A = SRC == SRC_COARSE ? ceil_to(G_BX * G_BY * 4, 128) : ceil_to(RGB_BX * RGB_BY, 128);
    static constexpr int RAW_B = SRC == SRC_UP     ? ceil_to(C_BX * C_BY * 8, 128)
                                 : SRC == SRC_ZBUF ? ceil_to(Z_BX * Z_BY * 4, 128)
                                                   : ceil_to(S_BX * S_BY * 4, 128);
    static constexpr int TX_BYTES = SRC == SRC_COARSE ? G_BX * G_BY * 4 + S_BX * S_BY * 4
                                    : SRC == SRC_UP   ? RGB_BX * RGB_BY + C_BX * C_BY * 8
                                                      : RGB_BX * RGB_BY + Z_BX * Z_BY * 4;
    // sparse form: staged rows per warp in the record pass (warp w scans rows w, w + NW, ...)
    static constexpr int RPW = (SH + NW - 1) / NW;
    // staged records: float4 per position (per slot in the paired form: F and G of both columns;
    // two per position in the sparse form)
    static constexpr int STAGED = SPARSE ? 2 * SH * SW * 16
                                  : PAIRS ? SH * SP * 16
                                  : SRC == SRC_COARSE && !EXP ? 0 : SH * SW * 16;
    // scalar expanded form: F_q times depth (float per position); paired form: both columns'
    // packed colour words (uint2 per slot)
    static constexpr int STAGED_G = PAIRS ? SH * SP * 8 : EXP ? ceil_to(SH * SW * 4, 16) : 0;
    // sparse form: one observation mask (uint64) per staged row
    static constexpr int ROWS = SPARSE ? ceil_to(SH * 8, 16) : 0;
    // observation bitmap: bit i = staged record i observed; one word per 32 records for every
    // record the conversion loop visits, plus a zero guard word (the paired form keeps one
    // bitmap per half of its slots)
    static constexpr int NT = NW * 32, NCONV = (SH * SP + NT - 1) / NT;
    static constexpr int OBS_WORDS = NCONV * NT / 32 + 1;
    static constexpr int OBS_ONE = ceil_to(OBS_WORDS * 4, 16);
    static constexpr int OBS = OBS_ONE * (PAIRS ? 2 : 1);
    static constexpr int HOR = 0;
    static constexpr int OFF_RAW = 0;
    static constexpr int OFF_STAGED = OFF_RAW + 2 * (RAW_A + RAW_B);
    static constexpr int OFF_G = OFF_STAGED + STAGED;
    static constexpr int OFF_ROWS = OFF_G + STAGED_G;
    static constexpr int OFF_OBS = OFF_ROWS + ROWS;
    static constexpr int OFF_HOR = OFF_OBS + OBS;
    static constexpr int OFF_BAR = ceil_to(OFF_HOR + HOR, 16);
    static constexpr int SMEM = OFF_BAR + 16;
};

}  // namespace dz
