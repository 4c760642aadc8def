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

// Arithmetic forms of the filter kernels: FP32 with colour differences, FP16
// guide and weights with FP32 sums (full-resolution stages only), FP32 with the
// squared colour distance expanded into a dot product (weights kept in range
// only while kc * 3 * 128^2 + kp * 2 R^2 <= kExpRange, see jbf_tma.cuh), the
// expanded form on pairs of output columns in packed two-lane FP32 arithmetic
// (64-column tiles, see jbf_pair.cuh), and the sparse forms (a warp walks only the
// observed positions of its block's footprint; the single stage on the z-buffer, see
// jbf_sparse.cuh) with the expanded FP32 weights or with FP16 guide and weights.
enum { TMA_FORM_FP32 = 0, TMA_FORM_FP16 = 1, TMA_FORM_EXP = 2, TMA_FORM_EXP_PAIRS = 3, TMA_FORM_SPARSE = 4,
       TMA_FORM_SPARSE_FP16 = 5 };
constexpr double kExpRange = 100.0;

// Instantiated variants of (source, radius, form).
int jbf_tma_variants(int src, int r, int form, TmaVariant *out, int cap);
bool jbf_tma_info(int src, int r, TmaVariant v, int form, TmaKernelInfo *out);
cudaError_t jbf_tma_prepare(int src, int r, TmaVariant v, int form);
cudaError_t launch_jbf_tma(int src, int r, TmaVariant v, int form, const BatchDev *b, const StageArgs &a, int grid,
                           cudaStream_t s);
int occupancy_jbf_tma(int src, int r, TmaVariant v, int form);
// Flag the tiles of the stage's grid (tw x th) that some observation within radius r
// reaches (the flags were zeroed by the batch's first kernel).
cudaError_t launch_tile_mark(int src, const BatchDev *b, int stage, int th, int r, int grid, cudaStream_t s);

// the expanded form's instantiations (k_jbf_tma_exp.cu)
int jbf_tma_exp_variants(int src, int r, int form, TmaVariant *out, int cap);
bool jbf_tma_exp_info(int src, int r, TmaVariant v, int form, TmaKernelInfo *out);
cudaError_t jbf_tma_exp_prepare(int src, int r, TmaVariant v, int form);
cudaError_t jbf_tma_exp_launch(int src, int r, TmaVariant v, int form, const BatchDev *b, const StageArgs &a,
                               int grid, cudaStream_t s);
int jbf_tma_exp_occupancy(int src, int r, TmaVariant v, int form);

// the sparse form's instantiations (k_jbf_sparse.cu)
int jbf_tma_sp_variants(int src, int r, int form, TmaVariant *out, int cap);
bool jbf_tma_sp_info(int src, int r, TmaVariant v, int form, TmaKernelInfo *out);
cudaError_t jbf_tma_sp_prepare(int src, int r, TmaVariant v, int form);
cudaError_t jbf_tma_sp_launch(int src, int r, TmaVariant v, int form, const BatchDev *b, const StageArgs &a,
                              int grid, cudaStream_t s);
int jbf_tma_sp_occupancy(int src, int r, TmaVariant v, int form);

}  // namespace dz
