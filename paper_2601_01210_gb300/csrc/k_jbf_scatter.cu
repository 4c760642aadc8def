// Instantiations of the TMA-staged joint bilateral filter in Algorithm 1's
// scatter form (jbf_scatter.cuh) for the single stage on the z-buffer, whose
// input is sparse (a few percent of the pixels observed).
#include "jbf_tma_dispatch.cuh"

namespace dz {

// (source, radius, rows per thread, form, warps per CTA); 32-column tiles of
// rows per thread x warps rows
#define DZ_TMA_SC_CASES(X)                 \
    X(SRC_ZBUF, 4, 4, FORM_SCATTER, 8)     \
    X(SRC_ZBUF, 4, 2, FORM_SCATTER, 16)    \
    X(SRC_ZBUF, 2, 4, FORM_SCATTER, 8)     \
    X(SRC_ZBUF, 7, 4, FORM_SCATTER, 8)

DZ_TMA_LOOKUPS(DZ_TMA_SC_CASES, jbf_tma_sc)

}  // namespace dz
