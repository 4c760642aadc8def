// Instantiations of the TMA-staged joint bilateral filter in the sparse forms
// (jbf_sparse.cuh; FP32, and FP16 guide and weights): the single stage on the
// z-buffer, whose input holds an observation at a few percent of the pixels.
#include "jbf_tma_dispatch.cuh"

namespace dz {

// (source, radius, rows per thread, form, warps per CTA); 32-column tiles of
// rows per thread x warps rows, worked in 8 x 8 blocks
#define DZ_TMA_SP_CASES(X)              \
    X(SRC_ZBUF, 4, 4, FORM_SPARSE, 8)   \
    X(SRC_ZBUF, 4, 2, FORM_SPARSE, 8)   \
    X(SRC_ZBUF, 2, 4, FORM_SPARSE, 8)   \
    X(SRC_ZBUF, 7, 4, FORM_SPARSE, 8)   \
    X(SRC_ZBUF, 7, 2, FORM_SPARSE, 8)   \
    X(SRC_ZBUF, 4, 4, FORM_SPARSE_FP16, 8) \
    X(SRC_ZBUF, 2, 4, FORM_SPARSE_FP16, 8) \
    X(SRC_ZBUF, 7, 4, FORM_SPARSE_FP16, 8)

DZ_TMA_LOOKUPS(DZ_TMA_SP_CASES, jbf_tma_sp)

}  // namespace dz
