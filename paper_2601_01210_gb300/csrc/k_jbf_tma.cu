// Instantiations of the TMA-staged joint bilateral filter in the FP32
// difference form and the FP16 form, and the public lookups over all forms
// (the expanded FP32 form is instantiated in k_jbf_tma_exp.cu).
#include "jbf_tma_dispatch.cuh"

namespace dz {

namespace {

// (source, radius, rows per thread, form, warps per CTA); the first listed
// variant of a (source, radius, form) is the default before autotuning
#define DZ_TMA_CASES(X)                   \
    X(SRC_UP, 1, 8, FORM_FP32, 8)         \
    X(SRC_UP, 2, 8, FORM_FP32, 8)         \
    X(SRC_UP, 2, 8, FORM_FP32, 16)        \
    X(SRC_UP, 2, 4, FORM_FP32, 8)         \
    X(SRC_UP, 3, 4, FORM_FP32, 8)         \
    X(SRC_COARSE, 2, 4, FORM_FP32, 8)     \
    X(SRC_COARSE, 4, 4, FORM_FP32, 8)     \
    X(SRC_COARSE, 4, 2, FORM_FP32, 8)     \
    X(SRC_ZBUF, 2, 8, FORM_FP32, 8)       \
    X(SRC_ZBUF, 4, 8, FORM_FP32, 8)       \
    X(SRC_ZBUF, 4, 4, FORM_FP32, 8)       \
    X(SRC_ZBUF, 7, 4, FORM_FP32, 8)       \
    X(SRC_UP, 1, 8, FORM_FP16, 8)         \
    X(SRC_UP, 2, 8, FORM_FP16, 8)         \
    X(SRC_UP, 2, 8, FORM_FP16, 16)        \
    X(SRC_UP, 2, 4, FORM_FP16, 8)         \
    X(SRC_UP, 3, 4, FORM_FP16, 8)         \
    X(SRC_ZBUF, 2, 8, FORM_FP16, 8)       \
    X(SRC_ZBUF, 4, 8, FORM_FP16, 8)       \
    X(SRC_ZBUF, 4, 4, FORM_FP16, 8)       \
    X(SRC_ZBUF, 7, 4, FORM_FP16, 8)

DZ_TMA_LOOKUPS(DZ_TMA_CASES, base)

}  // namespace

int jbf_tma_variants(int src, int r, int form, TmaVariant *out, int cap) {
    int n = base_variants(src, r, form, out, cap);
    n += jbf_tma_exp_variants(src, r, form, out + n, cap - n);
    return n + jbf_tma_sp_variants(src, r, form, out + n, cap - n);
}

bool jbf_tma_info(int src, int r, TmaVariant v, int form, TmaKernelInfo *out) {
    *out = TmaKernelInfo{};
    return base_info(src, r, v, form, out) || jbf_tma_exp_info(src, r, v, form, out) ||
           jbf_tma_sp_info(src, r, v, form, out);
}

cudaError_t jbf_tma_prepare(int src, int r, TmaVariant v, int form) {
    return form >= TMA_FORM_SPARSE ? jbf_tma_sp_prepare(src, r, v, form)
           : form >= TMA_FORM_EXP   ? jbf_tma_exp_prepare(src, r, v, form)
                                    : base_prepare(src, r, v, form);
}

cudaError_t launch_jbf_tma(int src, int r, TmaVariant v, int form, const BatchDev *b, const StageArgs &a, int grid,
                           cudaStream_t s) {
    return form >= TMA_FORM_SPARSE ? jbf_tma_sp_launch(src, r, v, form, b, a, grid, s)
           : form >= TMA_FORM_EXP   ? jbf_tma_exp_launch(src, r, v, form, b, a, grid, s)
                                    : base_launch(src, r, v, form, b, a, grid, s);
}

cudaError_t launch_tile_mark(int src, const BatchDev *b, int stage, int th, int r, int grid, cudaStream_t s) {
    BatchDev *bb = const_cast<BatchDev *>(b);
    if (src == TMA_SRC_UP) tile_mark_kernel<SRC_UP><<<grid, kMarkThreads, 0, s>>>(bb, stage, th, r);
    else if (src == TMA_SRC_COARSE) tile_mark_kernel<SRC_COARSE><<<grid, kMarkThreads, 0, s>>>(bb, stage, th, r);
    else tile_mark_kernel<SRC_ZBUF><<<grid, kMarkThreads, 0, s>>>(bb, stage, th, r);
    return cudaGetLastError();
}

int occupancy_jbf_tma(int src, int r, TmaVariant v, int form) {
    const int n = form >= TMA_FORM_SPARSE ? jbf_tma_sp_occupancy(src, r, v, form)
                  : form >= TMA_FORM_EXP   ? jbf_tma_exp_occupancy(src, r, v, form)
                                           : base_occupancy(src, r, v, form);
    return n > 0 ? n : 1;
}

}  // namespace dz
