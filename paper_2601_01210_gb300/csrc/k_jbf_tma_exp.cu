// Instantiations of the TMA-staged joint bilateral filter in the expanded
// FP32 forms (squared colour distance expanded into a dot product; scalar, see
// jbf_tma.cuh, and on column pairs, see jbf_pair.cuh), in a translation unit of
// their own so that the library's sources compile in parallel.
#include "jbf_tma_dispatch.cuh"

namespace dz {

// (source, radius, rows per thread, form, warps per CTA); the first listed
// variant of a (source, radius) is the default before autotuning
#define DZ_TMA_EXP_CASES(X)              \
    X(SRC_UP, 2, 6, FORM_EXP_PAIRS, 8)   \
    X(SRC_UP, 2, 4, FORM_EXP_PAIRS, 8)   \
    X(SRC_UP, 2, 6, FORM_EXP_PAIRS, 4)   \
    X(SRC_UP, 2, 4, FORM_EXP_PAIRS, 4)   \
    X(SRC_UP, 2, 8, FORM_EXP_PAIRS, 4)   \
    X(SRC_UP, 2, 8, FORM_EXP, 16)        \
    X(SRC_UP, 2, 8, FORM_EXP, 8)         \
    X(SRC_UP, 2, 4, FORM_EXP, 8)         \
    X(SRC_UP, 1, 8, FORM_EXP, 8)         \
    X(SRC_UP, 3, 4, FORM_EXP, 8)         \
    X(SRC_COARSE, 4, 2, FORM_EXP, 8)     \
    X(SRC_COARSE, 4, 4, FORM_EXP, 8)     \
    X(SRC_COARSE, 4, 2, FORM_EXP, 4)     \
    X(SRC_COARSE, 2, 4, FORM_EXP, 8)     \
    X(SRC_ZBUF, 2, 4, FORM_EXP_PAIRS, 4) \
    X(SRC_ZBUF, 2, 8, FORM_EXP, 8)       \
    X(SRC_ZBUF, 4, 4, FORM_EXP, 8)       \
    X(SRC_ZBUF, 7, 4, FORM_EXP, 8)

DZ_TMA_LOOKUPS(DZ_TMA_EXP_CASES, jbf_tma_exp)

}  // namespace dz
