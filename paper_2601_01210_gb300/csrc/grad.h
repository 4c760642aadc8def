// Sigma-gradient kernels (k_grad.cu).
#pragma once

#include "desc.cuh"

namespace dz {

struct GradStage {
    int32_t radius;
    float kc, kp;            // log2(e) / (2 sigma_c^2), log2(e) / (2 sigma_p^2)
    float inv_sc3, inv_sp3;  // 1 / sigma_c^3, 1 / sigma_p^3
};

struct GradArgs {
    GradStage s[2];
    int32_t two_stage;
    int32_t pool;
};

// grid: persistent CTAs; part: grid x 6 floats, one row per block (squared-error
// sum, pixel count, gradient sums for sp1, sc1, sp2, sc2), added by the caller.
cudaError_t launch_grad(const BatchDev *b, const GradArgs &ga, const float *gt, float *part, int grid,
                        cudaStream_t s);

}  // namespace dz
