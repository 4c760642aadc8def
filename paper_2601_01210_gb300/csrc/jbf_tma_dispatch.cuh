// Host-side helpers shared by the translation units that instantiate the
// TMA-staged filter: tile description, shared-memory opt-in, launch and
// occupancy of one instantiation (source, radius, rows per thread, form, warps).
#pragma once

#include "jbf_tma.cuh"
#include "tma_info.h"

namespace dz {
namespace tma_detail {

template <int SRC, int R, int KP, int FORM, int NW>
using Geom = TmaGeom<SRC, R, KP, NW, FORM>;

template <int SRC, int R, int KP, int FORM, int NW>
void fill_info(TmaKernelInfo *o) {
    using G = Geom<SRC, R, KP, FORM, NW>;
    o->supported = 1;
    o->kp = KP;
    o->threads = NW * 32;
    o->tile_w = G::TW;
    o->tile_h = G::TH;
    o->smem = G::SMEM;
    o->rgb_box[0] = G::RGB_BX; o->rgb_box[1] = G::RGB_BY;
    o->s1_box[0] = G::C_BX;    o->s1_box[1] = G::C_BY;
    o->zbuf_box[0] = G::Z_BX;  o->zbuf_box[1] = G::Z_BY;
    o->cguide_box[0] = G::G_BX; o->cguide_box[1] = G::G_BY;
    o->cssum_box[0] = G::S_BX; o->cssum_box[1] = G::S_BY;
}

template <int SRC, int R, int KP, int FORM, int NW>
cudaError_t prep() {
    return cudaFuncSetAttribute(jbf_tma_kernel<SRC, R, KP, FORM, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Geom<SRC, R, KP, FORM, NW>::SMEM);
}

template <int SRC, int R, int KP, int FORM, int NW>
cudaError_t go(const BatchDev *b, const StageArgs &a, int grid, cudaStream_t s) {
    jbf_tma_kernel<SRC, R, KP, FORM, NW><<<grid, NW * 32, Geom<SRC, R, KP, FORM, NW>::SMEM, s>>>(b, a);
    return cudaGetLastError();
}

template <int SRC, int R, int KP, int FORM, int NW>
int occ() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, jbf_tma_kernel<SRC, R, KP, FORM, NW>, NW * 32,
                                                  Geom<SRC, R, KP, FORM, NW>::SMEM);
    return n > 0 ? n : 1;
}

}  // namespace tma_detail
}  // namespace dz

// Defines the five lookups of one translation unit's instantiation list
// CASES(X), X(source, radius, rows per thread, form, warps), under the names
// PREFIX_variants / _info / _prepare / _launch / _occupancy.
#define DZ_TMA_LOOKUPS(CASES, PREFIX)                                                                              \
    int PREFIX##_variants(int src, int r, int form, TmaVariant *out, int cap) {                                   \
        int n = 0;                                                                                                 \
        CASES(DZ_TMA_X_VARIANT)                                                                                    \
        return n;                                                                                                  \
    }                                                                                                              \
    bool PREFIX##_info(int src, int r, TmaVariant v, int form, TmaKernelInfo *out) {                              \
        CASES(DZ_TMA_X_INFO)                                                                                       \
        return false;                                                                                              \
    }                                                                                                              \
    cudaError_t PREFIX##_prepare(int src, int r, TmaVariant v, int form) {                                        \
        CASES(DZ_TMA_X_PREPARE)                                                                                    \
        return cudaErrorInvalidValue;                                                                              \
    }                                                                                                              \
    cudaError_t PREFIX##_launch(int src, int r, TmaVariant v, int form, const BatchDev *b, const StageArgs &a,    \
                                int grid, cudaStream_t s) {                                                        \
        CASES(DZ_TMA_X_LAUNCH)                                                                                     \
        return cudaErrorInvalidValue;                                                                              \
    }                                                                                                              \
    int PREFIX##_occupancy(int src, int r, TmaVariant v, int form) {                                              \
        CASES(DZ_TMA_X_OCC)                                                                                        \
        return 0;                                                                                                  \
    }

#define DZ_TMA_MATCH(S, RR, K, F, NW) (src == S && r == RR && v.kp == K && v.nw == NW && form == F)
#define DZ_TMA_X_VARIANT(S, RR, K, F, NW) \
    if (src == S && r == RR && form == F && n < cap) out[n++] = TmaVariant{K, NW};
#define DZ_TMA_X_INFO(S, RR, K, F, NW) \
    if (DZ_TMA_MATCH(S, RR, K, F, NW)) { tma_detail::fill_info<S, RR, K, F, NW>(out); return true; }
#define DZ_TMA_X_PREPARE(S, RR, K, F, NW) \
    if (DZ_TMA_MATCH(S, RR, K, F, NW)) return tma_detail::prep<S, RR, K, F, NW>();
#define DZ_TMA_X_LAUNCH(S, RR, K, F, NW) \
    if (DZ_TMA_MATCH(S, RR, K, F, NW)) return tma_detail::go<S, RR, K, F, NW>(b, a, grid, s);
#define DZ_TMA_X_OCC(S, RR, K, F, NW) \
    if (DZ_TMA_MATCH(S, RR, K, F, NW)) return tma_detail::occ<S, RR, K, F, NW>();
