// Instantiations of the TMA-staged joint bilateral filter and the host-side
// description of their tiles (tensor-map boxes, shared memory, rows per tile).
#include "jbf_tma.cuh"
#include "tma_info.h"

namespace dz {

namespace {

template <int SRC, int R, int KP, int NW>
void fill_info(TmaKernelInfo *o) {
    using G = TmaGeom<SRC, R, KP, NW>;
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

template <int SRC, int R, int KP, bool H, int NW>
cudaError_t prep() {
    return cudaFuncSetAttribute(jbf_tma_kernel<SRC, R, KP, H, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TmaGeom<SRC, R, KP, NW>::SMEM);
}

template <int SRC, int R, int KP, bool H, int NW>
cudaError_t go(const BatchDev *b, const StageArgs &a, int grid, cudaStream_t s) {
    jbf_tma_kernel<SRC, R, KP, H, NW><<<grid, NW * 32, TmaGeom<SRC, R, KP, NW>::SMEM, s>>>(b, a);
    return cudaGetLastError();
}

template <int SRC, int R, int KP, bool H, int NW>
int occ() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, jbf_tma_kernel<SRC, R, KP, H, NW>, NW * 32,
                                                  TmaGeom<SRC, R, KP, NW>::SMEM);
    return n > 0 ? n : 1;
}

// (source, radius, rows per thread, FP16 form, warps per CTA); the first listed
// variant of a (source, radius, form) is the default before autotuning
#define DZ_TMA_CASES(X)               \
    X(SRC_UP, 1, 8, false, 8)         \
    X(SRC_UP, 2, 8, false, 8)         \
    X(SRC_UP, 2, 8, false, 16)        \
    X(SRC_UP, 2, 4, false, 8)         \
    X(SRC_UP, 3, 4, false, 8)         \
    X(SRC_COARSE, 2, 4, false, 8)     \
    X(SRC_COARSE, 4, 4, false, 8)     \
    X(SRC_COARSE, 4, 2, false, 8)     \
    X(SRC_ZBUF, 2, 8, false, 8)       \
    X(SRC_ZBUF, 4, 8, false, 8)       \
    X(SRC_ZBUF, 4, 4, false, 8)       \
    X(SRC_ZBUF, 7, 4, false, 8)       \
    X(SRC_UP, 1, 8, true, 8)          \
    X(SRC_UP, 2, 8, true, 8)          \
    X(SRC_UP, 2, 8, true, 16)         \
    X(SRC_UP, 2, 4, true, 8)          \
    X(SRC_UP, 3, 4, true, 8)          \
    X(SRC_ZBUF, 2, 8, true, 8)        \
    X(SRC_ZBUF, 4, 8, true, 8)        \
    X(SRC_ZBUF, 4, 4, true, 8)        \
    X(SRC_ZBUF, 7, 4, true, 8)

}  // namespace

int jbf_tma_variants(int src, int r, bool half, TmaVariant *out, int cap) {
    int n = 0;
#define X(S, RR, K, H, NW) if (src == S && r == RR && half == H && n < cap) out[n++] = TmaVariant{K, NW};
    DZ_TMA_CASES(X)
#undef X
    return n;
}

bool jbf_tma_info(int src, int r, TmaVariant v, bool half, TmaKernelInfo *out) {
    *out = TmaKernelInfo{};
#define X(S, RR, K, H, NW) \
    if (src == S && r == RR && v.kp == K && v.nw == NW && half == H) { fill_info<S, RR, K, NW>(out); return true; }
    DZ_TMA_CASES(X)
#undef X
    return false;
}

cudaError_t jbf_tma_prepare(int src, int r, TmaVariant v, bool half) {
#define X(S, RR, K, H, NW) if (src == S && r == RR && v.kp == K && v.nw == NW && half == H) return prep<S, RR, K, H, NW>();
    DZ_TMA_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_jbf_tma(int src, int r, TmaVariant v, bool half, const BatchDev *b, const StageArgs &a, int grid,
                           cudaStream_t s) {
#define X(S, RR, K, H, NW) \
    if (src == S && r == RR && v.kp == K && v.nw == NW && half == H) return go<S, RR, K, H, NW>(b, a, grid, s);
    DZ_TMA_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

int occupancy_jbf_tma(int src, int r, TmaVariant v, bool half) {
#define X(S, RR, K, H, NW) if (src == S && r == RR && v.kp == K && v.nw == NW && half == H) return occ<S, RR, K, H, NW>();
    DZ_TMA_CASES(X)
#undef X
    return 1;
}


}  // namespace dz
