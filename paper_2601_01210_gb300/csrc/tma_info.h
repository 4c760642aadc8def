// Host-side description of the TMA-staged filter kernels.
#pragma once

#include <cuda_runtime.h>

#include "desc.cuh"

namespace dz {

enum { TMA_SRC_UP = 0, TMA_SRC_ZBUF = 1, TMA_SRC_COARSE = 2 };

struct TmaVariant {
    int kp;                 // output rows per thread
    int nw;                 // warps per CTA
};

struct TmaKernelInfo {
    int supported;
    int kp;                 // output rows per thread
    int threads;            // threads per CTA
    int tile_w, tile_h;     // output tile
    int smem;               // dynamic shared memory bytes
    int rgb_box[2];         // boxes in elements of each tensor map
    int s1_box[2];
    int zbuf_box[2];
    int cguide_box[2];      // in floats (4 per pooled pixel)
    int cssum_box[2];
};

// Instantiated variants: (source, radius, rows per thread kp, FP16 form). half: guide and
// weights in FP16 with FP32 sums (full-resolution stages only).
int jbf_tma_variants(int src, int r, bool half, TmaVariant *out, int cap);   // instantiated variants
bool jbf_tma_info(int src, int r, TmaVariant v, bool half, TmaKernelInfo *out);
cudaError_t jbf_tma_prepare(int src, int r, TmaVariant v, bool half);
cudaError_t launch_jbf_tma(int src, int r, TmaVariant v, bool half, const BatchDev *b, const StageArgs &a, int grid,
                           cudaStream_t s);
int occupancy_jbf_tma(int src, int r, TmaVariant v, bool half);

}  // namespace dz
