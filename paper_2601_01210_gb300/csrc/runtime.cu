// Host runtime behind the C ABI (include/densify.h).
//
// * Admission: every frame reserves its scratch (z-buffer, coarse maps,
//   compaction counts, staging of host frames) from one device arena that is
//   allocated when the context is created; a frame that does not fit now
//   gets DENSIFY_E_AGAIN, one that never fits DENSIFY_E_NOMEM. Nothing is
//   allocated per frame.
// * Batching: admitted frames queue on the host. A batch slot takes up to
//   max_batch of them, writes their descriptors into its device table and
//   runs the fixed kernel sequence (prep, project, [pool, coarse filter],
//   filter, compaction count, compaction write) on the context stream,
//   replayed from a CUDA graph captured the first time the slot is used.
//   Frames that arrive while every slot is busy go out together as soon as a
//   slot frees (continuous batching).
// * Completion: each slot records an event; densify_poll() queries events
//   (bounded waits only), finishes host-frame copies, frees scratch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include "../../include/densify.h"
#include "desc.cuh"
#include "grad.h"
#include "runtime_internal.h"
#include "tma_info.h"

using namespace dz;

namespace {

const char *const kKernelNames[K_COUNT] = {"prep_compose_clear", "motion_mask", "motion_dilate", "motion_erode",
                                           "project_zbuf",       "occlusion",   "pool3",         "jbf_stage1",
                                           "jbf_stage2",         "contour",     "bp_count",      "bp_write",
                                           "tile_mark1"};

constexpr uint64_t kAlign = 256;
uint64_t align_up(uint64_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

thread_local std::string g_create_error;

// First-fit allocator over offsets of the device arena.
class Arena {
public:
    void init(uint64_t size) {
        size_ = size;
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(uint64_t n, uint64_t *off) {
        n = align_up(n ? n : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const uint64_t rest = it->second - n;
                const uint64_t at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t n) {
        n = align_up(n ? n : 1);
        auto it = free_.emplace(off, n).first;
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
                it = prev;
            }
        }
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
    }
    uint64_t size() const { return size_; }

private:
    uint64_t size_ = 0;
    std::map<uint64_t, uint64_t> free_;
};

// Scratch layout of one frame inside its arena block.
struct Layout {
    uint64_t zbuf = 0, cguide = 0, cssum = 0, s1 = 0, chunk = 0, depth = 0, valid = 0;
    uint64_t zbuf_raw = 0, motion = 0, motion_tmp = 0, prev = 0, depth_f = 0, valid_f = 0;
    bool has_motion = false;
    uint64_t pts[kMaxScans] = {0, 0, 0}, rgb = 0, points = 0, npts = 0, coarse = 0, coarse_valid = 0;
    int64_t rgb_pitch = 0;   // pitch of the staged RGB copy (0: the caller's frame is used in place)
    float4 *points_direct = nullptr;    // device view of a page-locked host point buffer
    int64_t *count_direct = nullptr;    // device view of a page-locked host count
    uint64_t tflags = 0;                // tile flags of the TMA filters (both stages)
    bool zpooled = false;               // z-buffer from the context's pool of clean z-buffers
    uint64_t zbytes = 0;                // its size (not part of total)
    uint64_t total = 0;
    bool own_depth = false, own_valid = false;
};

struct FrameRec {
    densify_frame fr;
    Layout L;
    uint64_t off = 0;
    uint64_t zoff = 0;       // offset of a pooled z-buffer
    int state = 0;   // 0 queued, 1 on the GPU, 2 finished
    int slot = -1;
    FrameDev dev;
    int64_t host_npts = 0;   // points count copied back for host frames
};

struct Slot {
    cudaStream_t stream = nullptr;   // the context stream, or the slot's own when the context owns its streams
    bool own_stream = false;
    BatchDev *d = nullptr;       // device table
    BatchDev *h = nullptr;       // pinned host mirror
    int32_t *d_status = nullptr; // device status word (bounded waits that gave up)
    int32_t *h_status = nullptr; // pinned copy, written at the end of every batch
    cudaEvent_t done = nullptr;
    cudaEvent_t kev[K_COUNT + 1] = {};
    int kord[K_COUNT] = {};      // timed steps in launch order: step j lies between kev[j] and kev[j + 1]
    int ntimed = 0;
    cudaGraphExec_t exec = nullptr;
    bool busy = false;
    std::vector<uint64_t> tickets;
    int nkern = 0;               // CUDA kernels one batch of this slot launches
};

// One filter launch: which kernel runs it and its tile height.
struct FilterSel {
    int kind = 0;        // 0 single, 1 coarse, 2 restored full resolution
    int radius = 0;
    bool tma = false;
    bool half = false;   // FP16 form
    int form = 0;        // arithmetic form of a TMA kernel (TMA_FORM_*)
    int src = 0;         // TMA source kind
    int kp = 0;          // output rows per thread
    int nw = 8;          // warps per CTA (tile height = kp * nw)
    int tile_w = 32;     // output tile (tile_w x tile_h pixels)
    int tile_h = 0;
    int occ = 1;         // resident CTAs per SM
    TmaKernelInfo info{};
    float tuned_us = -1.0f;   // measured by the autotuner (-1: not tuned)
};

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool tensor_map_encoder() {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        cudaGetLastError();
    });
    return g_encode != nullptr;
}

bool encode2d(CUtensorMap *m, CUtensorMapDataType dt, const void *base, uint64_t d0, uint64_t d1, uint64_t stride,
              int b0, int b1) {
    const cuuint64_t dims[2] = {d0, d1};
    const cuuint64_t strides[1] = {stride};
    const cuuint32_t box[2] = {(cuuint32_t)b0, (cuuint32_t)b1};
    const cuuint32_t es[2] = {1, 1};
    return g_encode(m, dt, 2, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

}  // namespace

struct densify_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;   // private stream for graph capture
    cudaStream_t d2h_stream = nullptr;   // exact-size point copies of host frames
    densify_params p{};
    StageArgs sa[2]{};
    PrepostArgs pp{};
    void *arena_base = nullptr;
    Arena arena;
    // clean z-buffers (two-stage contexts whose pooling kernel is the z-buffer's last reader): a free
    // region of this pool is all empty cells, so a frame's z-buffer needs no clear
    void *zpool_base = nullptr;
    Arena zpool;
    std::vector<Slot> slots;
    std::deque<uint64_t> queue;
    std::map<uint64_t, FrameRec> frames;
    uint64_t next_ticket = 1;
    int admitted = 0;
    int grid[K_COUNT] = {};
    FilterSel sel[2];                    // first (or only) and second filter
    std::vector<FilterSel> cands[2];     // kernels able to run each filter stage
    int sms = 0;
    bool tuned = true;                   // false until the autotuner ran (params.autotune)
    std::string err;
    bool dead = false;
    double t_us[K_COUNT] = {};
    int64_t t_n[K_COUNT] = {};
    int64_t kernel_launches = 0;   // CUDA kernels of completed batches
    bool inject_wait_failure = false;   // densify_inject_wait_failure: armed for the next batch
    int64_t batches = 0;                // batches launched
    int max_busy = 0;                   // most batches on the GPU at once
    bool grids_fixed = false;           // the kernel grids were settled by the first batch
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

densify_status fail(densify_ctx *c, densify_status s, const std::string &msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return s;
}

densify_status cuda_fail(densify_ctx *c, cudaError_t e, const char *what) {
    c->dead = true;
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return DENSIFY_E_CUDA;
}

#define CU(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

bool stage_supported(int kind, int r) {
    if (r < 1) return false;
    if (kind == 2) return r <= 3;
    return r <= kMaxR;
}

// Kernels that can run one filter stage: the TMA-staged kernel at each
// instantiated tile height (rows per thread), then the plain kernel. The first
// entry is the default; the autotuner times them all on the first batch.
std::vector<FilterSel> filter_candidates(const densify_params &p, int kind, int r) {
    std::vector<FilterSel> out;
    const int src = kind == 0 ? TMA_SRC_ZBUF : kind == 1 ? TMA_SRC_COARSE : TMA_SRC_UP;
    const bool allowed = p.kernel_variant != 1 && (kind != 2 || (p.pool == 3 && p.stage2_input == 0));
    // FP16: the full-resolution stage (the pooled first stage stays FP32)
    const bool half = p.precision == DENSIFY_FP16 && kind != 1;
    auto add_tma = [&](int form) {
        TmaVariant vs[16];
        const int n = jbf_tma_variants(src, r, form, vs, 16);
        for (int i = 0; i < n; ++i) {
            FilterSel s;
            s.kind = kind;
            s.radius = r;
            s.tma = true;
            s.half = form == TMA_FORM_FP16 || form == TMA_FORM_SPARSE_FP16;
            s.form = form;
            s.src = src;
            s.kp = vs[i].kp;
            s.nw = vs[i].nw;
            jbf_tma_info(src, r, vs[i], form, &s.info);
            s.tile_w = s.info.tile_w;
            s.tile_h = s.info.tile_h;
            out.push_back(s);
        }
    };
    if (allowed) {
        if (half) {
            // the single stage on the z-buffer: the sparse form first, as in FP32
            if (kind == 0) add_tma(TMA_FORM_SPARSE_FP16);
            add_tma(TMA_FORM_FP16);
        } else {
            // expanded FP32 form first where its weights stay in range (colours centred at 128)
            const densify_stage &st = p.stage[kind == 2 ? 1 : 0];
            const double log2e = 1.4426950408889634;
            const double kc = log2e / (2.0 * (double)st.sigma_c * (double)st.sigma_c);
            const double kp = log2e / (2.0 * (double)st.sigma_p * (double)st.sigma_p);
            if (p.kernel_variant == 0 && kc * 3.0 * 128.0 * 128.0 + kp * 2.0 * r * r <= kExpRange) {
                // the single stage on the z-buffer (a few percent of the pixels observed): the sparse
                // form first, whose work follows the observations; then the gather forms
                if (kind == 0) add_tma(TMA_FORM_SPARSE);
                add_tma(TMA_FORM_EXP_PAIRS);
                add_tma(TMA_FORM_EXP);
            }
            add_tma(TMA_FORM_FP32);
        }
    }
    if (!half) {
        FilterSel s;
        s.kind = kind;
        s.radius = r;
        s.kp = kind == 0 ? kp_jbf_single(r) : kind == 1 ? kp_jbf_coarse(r) : kp_jbf_up(r);
        s.tile_h = 8 * s.kp;
        out.push_back(s);
    }
    return out;
}

void fill_stage(StageArgs &a, const densify_stage &st, int pool, int override_sparse) {
    const double log2e = 1.4426950408889634;
    a.kc = (float)(log2e / (2.0 * (double)st.sigma_c * (double)st.sigma_c));
    a.kp = (float)(log2e / (2.0 * (double)st.sigma_p * (double)st.sigma_p));
    a.pool = pool;
    a.override_sparse = override_sparse;
    const int R = st.radius;
    for (int dy = 0; dy < 2 * kMaxR + 1; ++dy)
        for (int dx = 0; dx < 2 * kMaxR + 1; ++dx) {
            const double d2 = (double)((dx - R) * (dx - R) + (dy - R) * (dy - R));
            a.sp[dy * (2 * kMaxR + 1) + dx] = (float)(-d2 * log2e / (2.0 * (double)st.sigma_p * (double)st.sigma_p));
        }
    // FP16 form: (-kc, -kc) and per row offset d of a pixel pair (sp[d][dx], sp[d-1][dx]), -inf outside 0..2R
    auto h2 = [](float lo, float hi) {
        const __half2 v = __floats2half2_rn(lo, hi);
        uint32_t u;
        std::memcpy(&u, &v, 4);
        return u;
    };
    const float ninf = -INFINITY;
    a.kc2 = h2(-a.kc, -a.kc);
    const int T = 2 * R + 1;
    for (int d = 0; d < 2 * kMaxR + 2; ++d)
        for (int dx = 0; dx < 2 * kMaxR + 1; ++dx) {
            const float first = (d < T && dx < T) ? a.sp[d * (2 * kMaxR + 1) + dx] : ninf;
            const float second = (d >= 1 && d - 1 < T && dx < T) ? a.sp[(d - 1) * (2 * kMaxR + 1) + dx] : ninf;
            a.sp2[d * (2 * kMaxR + 1) + dx] = h2(first, second);
        }
    const double kp = log2e / (2.0 * (double)st.sigma_p * (double)st.sigma_p);
    for (int i = 0; i < 2 * kMaxR + 1; ++i) {
        const double o2 = (double)((i - R) * (i - R));
        a.ex_sx[i] = i < T ? (float)std::exp2(-o2 * kp) : 0.0f;
        a.ex_sy[i] = i < T ? (float)(-o2 * kp) : 0.0f;
    }
}

std::string validate_params(const densify_params &p) {
    if (p.num_stages != 1 && p.num_stages != 2) return "num_stages must be 1 or 2";
    for (int s = 0; s < p.num_stages; ++s) {
        const int kind = p.num_stages == 1 ? 0 : (s == 0 ? 1 : 2);
        if (!stage_supported(kind, p.stage[s].radius)) return "unsupported radius for stage " + std::to_string(s);
        if (!(p.stage[s].sigma_p > 0.0f) || !(p.stage[s].sigma_c > 0.0f) || !std::isfinite(p.stage[s].sigma_p) ||
            !std::isfinite(p.stage[s].sigma_c))
            return "sigmas must be positive and finite";
    }
    if (p.num_stages == 2 && (p.pool < 1 || p.pool > 8)) return "pool must be in 1..8";
    if (p.precision != DENSIFY_FP32 && p.precision != DENSIFY_FP16) return "precision must be FP32 or FP16";
    if (p.precision == DENSIFY_FP16) {
        if (p.kernel_variant != 0) return "the FP16 form runs in the TMA kernels (kernel_variant 0)";
        const int full = p.num_stages == 2 ? 1 : 0;   // the full-resolution stage
        const int kind = p.num_stages == 2 ? 2 : 0;
        TmaVariant vs[8];
        if (jbf_tma_variants(kind == 2 ? TMA_SRC_UP : TMA_SRC_ZBUF, p.stage[full].radius, TMA_FORM_FP16, vs, 8) == 0 ||
            (kind == 2 && (p.pool != 3 || p.stage2_input != 0)))
            return "FP16 form available for the full-resolution stage with radius 1-3 (pool 3, stage2_input 0) "
                   "after a first stage, or radius 2, 4, 7 as the only stage";
    }
    if (p.max_inflight < 1) return "max_inflight must be >= 1";
    if (p.max_batch < 1 || p.max_batch > kMaxBatch) return "max_batch must be in 1..64";
    if (p.batches_in_flight < 1 || p.batches_in_flight > 8) return "batches_in_flight must be in 1..8";
    if (p.hbm_budget_bytes < (1u << 20)) return "hbm_budget_bytes must be >= 1 MiB";
    if (p.launch_policy != 0 && p.launch_policy != 1) return "launch_policy must be 0 or 1";
    if (p.timing < 0 || p.timing > 2) return "timing must be 0, 1 or 2";
    if (p.kernel_variant < 0 || p.kernel_variant > 2) return "kernel_variant must be 0, 1 or 2";
    if (p.autotune != 0 && p.autotune != 1) return "autotune must be 0 or 1";
    if (p.occlusion_radius < 0 || p.occlusion_radius > 16) return "occlusion_radius must be in 0..16";
    if (!std::isfinite(p.occlusion_margin) || p.occlusion_margin < 0.0f) return "occlusion_margin must be >= 0";
    if (!std::isfinite(p.motion_threshold) || p.motion_threshold < 0.0f) return "motion_threshold must be >= 0";
    if (p.motion_close_radius < 0 || p.motion_close_radius > 16) return "motion_close_radius must be in 0..16";
    if (!std::isfinite(p.contour_threshold) || p.contour_threshold < 0.0f) return "contour_threshold must be >= 0";
    return "";
}

std::string validate_frame(const densify_ctx *c, const densify_frame *f) {
    if (!f) return "frame is NULL";
    const int W = f->K.width, H = f->K.height;
    if (W < 1 || H < 1 || W > 16384 || H > 16384) return "image size must be in 1..16384";
    if (!std::isfinite(f->K.fx) || !std::isfinite(f->K.fy) || f->K.fx == 0.0f || f->K.fy == 0.0f ||
        !std::isfinite(f->K.cx) || !std::isfinite(f->K.cy))
        return "intrinsics must be finite with nonzero focal lengths";
    if (f->num_scans < 0 || f->num_scans > kMaxScans) return "num_scans must be in 0..3";
    if (f->memory != DENSIFY_MEM_DEVICE && f->memory != DENSIFY_MEM_HOST) return "memory must be DEVICE or HOST";
    for (int s = 0; s < f->num_scans; ++s) {
        const densify_scan &S = f->scans[s];
        if (S.count < 0 || S.count > (int64_t)1 << 30) return "scan count must be in 0..2^30";
        if (S.stride_bytes != 12 && S.stride_bytes != 16) return "scan stride_bytes must be 12 or 16";
        if (S.count > 0 && !S.xyz) return "scan xyz is NULL";
        if (S.count > 0 && f->memory == DENSIFY_MEM_DEVICE && ((uintptr_t)S.xyz & 15u))
            return "scan xyz must be 16-byte aligned";
    }
    if (!f->rgb) return "rgb is NULL";
    if (f->prev_rgb && f->prev_rgb_pitch < 3 * (int64_t)W) return "prev_rgb_pitch must be >= 3 * width";
    if (c->p.motion_threshold > 0.0f && f->prev_rgb && f->num_scans > 0 &&
        (f->newest_scan < 0 || f->newest_scan >= f->num_scans))
        return "newest_scan must index one of the scans";
    if (f->rgb_pitch < 3 * (int64_t)W) return "rgb_pitch must be >= 3 * width";
    if (c->p.emit_points) {
        if (!f->out_points_n) return "out_points_n is NULL while points are on";
        if (f->out_points_cap < 0) return "out_points_cap must be >= 0";
        if (f->out_points_cap > 0 && !f->out_points) return "out_points is NULL with a nonzero capacity";
        if (f->out_points && ((uintptr_t)f->out_points & 15u)) return "out_points must be 16-byte aligned";
    }
    return "";
}

// Device address of page-locked host memory (unified addressing), or NULL.
template <typename T>
T *mapped_host(void *p) {
    if (!p) return nullptr;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost && at.devicePointer ? static_cast<T *>(at.devicePointer) : nullptr;
}

// Tile flags one frame needs (both stages): the most any TMA candidate of a stage needs, so that
// the frame's reservation holds whichever kernel the autotuner picks; 0 without a TMA stage.
int64_t tile_flag_words(const densify_params &p, int64_t W, int64_t H) {
    int64_t words = 0;
    for (int i = 0; i < p.num_stages; ++i) {
        const int kind = p.num_stages == 1 ? 0 : (i == 0 ? 1 : 2);
        const int64_t gw = kind == 1 ? (W + p.pool - 1) / p.pool : W, gh = kind == 1 ? (H + p.pool - 1) / p.pool : H;
        int64_t most = 0;
        for (const FilterSel &s : filter_candidates(p, kind, p.stage[i].radius))
            if (s.tma) most = std::max<int64_t>(most, ((gw + s.tile_w - 1) / s.tile_w) * ((gh + s.tile_h - 1) / s.tile_h));
        words += most;
    }
    return words;
}

// The pooling kernel is the last reader of the z-buffer: two stages with the restored first stage
// as the second stage's only input, no occluded-point removal (which rewrites the z-buffer).
bool zpool_applies(const densify_params &p) {
    return p.num_stages == 2 && p.stage2_input == 0 && p.occlusion_radius <= 0;
}

// allow_zpool: the frame may take its z-buffer from the context's clean pool (not when the caller
// wants the z-buffer itself, which is copied out after the pooling kernel has emptied it).
Layout layout_of(const densify_params &p, const densify_frame *f, bool allow_zpool = true) {
    Layout L;
    const int64_t W = f->K.width, H = f->K.height, npx = W * H;
    const bool host = f->memory == DENSIFY_MEM_HOST;
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) {
        const uint64_t at = o;
        o += align_up(bytes ? bytes : 1);
        return at;
    };
    const int64_t zp = (W + 3) & ~int64_t(3);
    L.zpooled = allow_zpool && zpool_applies(p) && !f->out_zbuf;
    if (L.zpooled) L.zbytes = align_up((uint64_t)zp * H * 4);
    else L.zbuf = take(zp * H * 4);
    if (p.occlusion_radius > 0) L.zbuf_raw = take(zp * H * 4);
    L.has_motion = p.motion_threshold > 0.0f && f->prev_rgb;
    if (L.has_motion) {
        L.motion = take(npx);
        // two bit-packed masks (32 pixels a word, rows of ceil(W / 32) words): the raw and the dilated one
        L.motion_tmp = take(std::max<int64_t>(npx, 2 * 4 * ((W + 31) / 32) * H));
        if (host) L.prev = take((uint64_t)npx * 3);
    }
    if (p.contour_threshold > 0.0f) {
        L.depth_f = take(npx * 4);
        L.valid_f = take(npx);
    }
    if (p.num_stages == 2) {
        const int64_t Wc = (W + p.pool - 1) / p.pool, Hc = (H + p.pool - 1) / p.pool;
        const int64_t cp = (Wc + 3) & ~int64_t(3);
        L.cguide = take(cp * Hc * 16);
        L.cssum = take(cp * Hc * 4);
        L.s1 = take(cp * Hc * 8);
        if (host && f->out_coarse) L.coarse = take(Wc * Hc * 4);
        if (host && f->out_coarse_valid) L.coarse_valid = take(Wc * Hc);
    }
    L.chunk = take(((npx + kBpChunk - 1) / kBpChunk) * kBpWarps * 4);
    if (const int64_t tw = tile_flag_words(p, W, H)) L.tflags = take((uint64_t)tw * 4);
    L.own_depth = host || !f->out_depth;
    L.own_valid = host || !f->out_valid;
    if (L.own_depth) L.depth = take(npx * 4);
    if (L.own_valid) L.valid = take(npx);
    if (host) {
        for (int s = 0; s < f->num_scans; ++s) L.pts[s] = take((uint64_t)f->scans[s].count * f->scans[s].stride_bytes);
        if (p.emit_points) {
            // points go straight from the compaction kernel into page-locked host memory, at exact size
            L.points_direct = mapped_host<float4>(f->out_points);
            L.count_direct = mapped_host<int64_t>(f->out_points_n);
            if (!L.points_direct) L.points = take((uint64_t)f->out_points_cap * 16);
            if (!L.count_direct) L.npts = take(8);
        }
    } else if (p.emit_points) {
        L.npts = 0;
    }
    // RGB goes to the kernels through TMA, which needs a 16-byte aligned base and
    // pitch: host frames and unaligned device frames are staged with pitch ceil16(3W)
    if (host || ((uintptr_t)f->rgb & 15u) || (f->rgb_pitch & 15)) {
        L.rgb_pitch = (3 * W + 15) & ~int64_t(15);
        L.rgb = take((uint64_t)L.rgb_pitch * H);
    }
    L.total = o;
    return L;
}

void build_frame_dev(densify_ctx *c, FrameRec &r) {
    const densify_frame *f = &r.fr;
    const Layout &L = r.L;
    char *base = (char *)c->arena_base + r.off;
    const bool host = f->memory == DENSIFY_MEM_HOST;
    FrameDev &d = r.dev;
    std::memset(&d, 0, sizeof(d));
    d.W = f->K.width;
    d.H = f->K.height;
    const int pool = c->p.num_stages == 2 ? c->p.pool : 1;
    d.Wc = (d.W + pool - 1) / pool;
    d.Hc = (d.H + pool - 1) / pool;
    d.cpitch = (d.Wc + 3) & ~3;
    d.fx = f->K.fx; d.fy = f->K.fy; d.cx = f->K.cx; d.cy = f->K.cy;
    std::memcpy(d.c2w, f->cam_to_world, sizeof(d.c2w));
    d.num_scans = f->num_scans;
    d.n_bp_chunks = ceil_div((int64_t)d.W * d.H, kBpChunk);
    for (int s = 0; s < kMaxScans; ++s) {
        ScanDev &S = d.scans[s];
        if (s < f->num_scans) {
            S.xyz = host ? (const float *)(base + L.pts[s]) : f->scans[s].xyz;
            S.count = f->scans[s].count;
            S.stride_floats = f->scans[s].stride_bytes / 4;
            std::memcpy(S.l2w, f->scans[s].lidar_to_world, sizeof(S.l2w));
        } else {
            S.count = 0;
            S.stride_floats = 3;
        }
    }
    d.rgb = L.rgb_pitch ? (const uint8_t *)(base + L.rgb) : f->rgb;
    d.rgb_pitch = L.rgb_pitch ? L.rgb_pitch : f->rgb_pitch;
    d.zpitch = (d.W + 3) & ~3;
    d.zbuf = L.zpooled ? (uint32_t *)((char *)c->zpool_base + r.zoff) : (uint32_t *)(base + L.zbuf);
    d.zclear = !L.zpooled;
    d.zrestore = L.zpooled;
    d.zbuf_raw = c->p.occlusion_radius > 0 ? (uint32_t *)(base + L.zbuf_raw) : d.zbuf;
    d.newest_scan = f->newest_scan;
    d.n_px_chunks = ceil_div((int64_t)d.W * d.H, kPxChunk);
    if (L.has_motion) {
        d.motion = (uint8_t *)(base + L.motion);
        d.motion_tmp = (uint8_t *)(base + L.motion_tmp);
        d.prev_rgb = host ? (const uint8_t *)(base + L.prev) : f->prev_rgb;
        d.prev_pitch = host ? (int64_t)d.W * 3 : f->prev_rgb_pitch;
    }
    if (c->p.num_stages == 2) {
        d.cguide = (float4 *)(base + L.cguide);
        d.cssum = (float *)(base + L.cssum);
        d.s1 = (float2 *)(base + L.s1);
        d.out_coarse = host ? (f->out_coarse ? (float *)(base + L.coarse) : nullptr) : f->out_coarse;
        d.out_coarse_valid =
            host ? (f->out_coarse_valid ? (uint8_t *)(base + L.coarse_valid) : nullptr) : f->out_coarse_valid;
    }
    d.chunk_cnt = (uint32_t *)(base + L.chunk);
    if (L.tflags) {   // the chosen kernels' tile counts (at most what the layout reserved)
        int64_t n[2] = {0, 0};
        for (int i = 0; i < c->p.num_stages; ++i) {
            const FilterSel &s = c->sel[i];
            if (!s.tma) continue;
            const int gw = s.kind == 1 ? d.Wc : d.W, gh = s.kind == 1 ? d.Hc : d.H;
            n[i] = (int64_t)ceil_div(gw, s.tile_w) * ceil_div(gh, s.tile_h);
        }
        d.tflags[0] = (int32_t *)(base + L.tflags);
        d.tflags[1] = d.tflags[0] + n[0];
        d.ntflags = (int32_t)(n[0] + n[1]);
    }
    d.out_depth = L.own_depth ? (float *)(base + L.depth) : f->out_depth;
    d.out_valid = L.own_valid ? (uint8_t *)(base + L.valid) : f->out_valid;
    const bool contour = c->p.contour_threshold > 0.0f;
    d.flt_depth = contour ? (float *)(base + L.depth_f) : d.out_depth;
    d.flt_valid = contour ? (uint8_t *)(base + L.valid_f) : d.out_valid;
    if (c->p.emit_points) {
        d.out_points = host ? (L.points_direct ? L.points_direct : (float4 *)(base + L.points)) : (float4 *)f->out_points;
        d.points_cap = f->out_points_cap;
        d.points_n = host ? (L.count_direct ? L.count_direct : (int64_t *)(base + L.npts)) : f->out_points_n;
    }
}

void fill_batch(densify_ctx *c, Slot &sl, const std::vector<uint64_t> &tk) {
    BatchDev &b = *sl.h;
    const int n = (int)tk.size();
    b.n_frames = n;
    b.status = sl.d_status;
    b.zb_pre[0] = b.pt_pre[0] = b.pool_pre[0] = b.t1_pre[0] = b.t2_pre[0] = b.bp_pre[0] = 0;
    b.px_pre[0] = b.oc_pre[0] = b.mk_pre[0] = 0;
    const int nst = c->p.num_stages;
    const int r1 = c->p.stage[0].radius, r2 = nst == 2 ? c->p.stage[1].radius : 0;
    (void)r1;
    (void)r2;
    const int tw1 = c->sel[0].tile_w, th1 = c->sel[0].tile_h;
    const int tw2 = nst == 2 ? c->sel[1].tile_w : 32, th2 = nst == 2 ? c->sel[1].tile_h : 1;
    for (int i = 0; i < n; ++i) {
        FrameRec &r = c->frames[tk[i]];
        const FrameDev &d = r.dev;
        b.f[i] = d;
        b.zb_pre[i + 1] = b.zb_pre[i] + (d.zclear ? ceil_div((int64_t)d.zpitch * d.H, kZbWordsPerChunk) : 0);
        for (int s = 0; s < kMaxScans; ++s) {
            const int k = i * kMaxScans + s;
            b.pt_pre[k + 1] = b.pt_pre[k] + ceil_div(d.scans[s].count, kPtsPerChunk);
        }
        b.pool_pre[i + 1] = b.pool_pre[i] + (nst == 2 ? ceil_div(d.Wc, kPoolPerChunk) * d.Hc : 0);
        const int g1w = nst == 2 ? d.Wc : d.W, g1h = nst == 2 ? d.Hc : d.H;
        b.t1_pre[i + 1] = b.t1_pre[i] + ceil_div(g1w, tw1) * ceil_div(g1h, th1);
        b.t2_pre[i + 1] = b.t2_pre[i] + (nst == 2 ? ceil_div(d.W, tw2) * ceil_div(d.H, th2) : 0);
        b.bp_pre[i + 1] = b.bp_pre[i] + (c->p.emit_points ? d.n_bp_chunks : 0);
        b.px_pre[i + 1] = b.px_pre[i] + d.n_px_chunks;
        b.oc_pre[i + 1] = b.oc_pre[i] + ceil_div(d.W, kOccTile) * ceil_div(d.H, kOccTile);
        b.mk_pre[i + 1] = b.mk_pre[i] + (nst == 2 ? ceil_div(d.Hc, kMarkBand) * ceil_div(d.Wc, 32)
                                                  : ceil_div(d.H, kMarkBand) * ceil_div(d.W, 32));
    }
}

void set_filter(densify_ctx *c, int i, const FilterSel &f) {
    c->sel[i] = f;
    c->grid[i == 0 ? K_JBF1 : K_JBF2] = c->sms * f.occ;
}

cudaError_t launch_filter(densify_ctx *c, int i, const BatchDev *b, cudaStream_t s);
void fill_batch(densify_ctx *c, Slot &sl, const std::vector<uint64_t> &tk);
densify_status prepare_tile_lists(densify_ctx *c, Slot &sl);
std::string encode_maps(densify_ctx *c, FrameDev &d);

// Autotuner: on the context's first batch, time every candidate kernel of each
// filter stage (3 launches after one warm-up, CUDA events) on that batch's real
// inputs and keep the fastest; stage 2 is tuned after stage 1's choice is made.
// Choices are remembered per (stage kind, radius, precision, batch pixel class)
// in the file named by DENSIFY_TUNE_CACHE, when set, and reused from it.
std::string tune_key(const densify_ctx *c, int i, int64_t px) {
    int cls = 0;
    while ((int64_t(1) << (cls + 1)) <= px) ++cls;
    const FilterSel &f = c->cands[i][0];
    return "kind=" + std::to_string(f.kind) + ",r=" + std::to_string(f.radius) + ",half=" + std::to_string(f.half) +
           ",px=2^" + std::to_string(cls);
}

bool cache_lookup(const std::string &key, std::string *val) {
    const char *path = std::getenv("DENSIFY_TUNE_CACHE");
    if (!path) return false;
    FILE *fp = std::fopen(path, "r");
    if (!fp) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof line, fp)) {
        std::string l(line);
        while (!l.empty() && (l.back() == '\n' || l.back() == '\r')) l.pop_back();
        const size_t sp = l.find(' ');
        if (sp != std::string::npos && l.substr(0, sp) == key) {
            *val = l.substr(sp + 1);
            found = true;
        }
    }
    std::fclose(fp);
    return found;
}

void cache_store(const std::string &key, const std::string &val) {
    const char *path = std::getenv("DENSIFY_TUNE_CACHE");
    if (!path) return;
    if (FILE *fp = std::fopen(path, "a")) {
        std::fprintf(fp, "%s %s\n", key.c_str(), val.c_str());
        std::fclose(fp);
    }
}

std::string cand_name(const FilterSel &f) {
    static const char *forms[] = {"fp32", "fp16", "exp", "exp_pairs", "sparse", "sparse_fp16"};
    return std::string(f.tma ? "tma" : "plain") + ":kp" + std::to_string(f.kp) + ":nw" + std::to_string(f.nw) +
           (f.tma ? std::string(":") + forms[f.form] : std::string());
}

densify_status autotune(densify_ctx *c, Slot &sl, const std::vector<uint64_t> &tk) {
    int64_t px = 0;
    for (uint64_t t : tk) px += (int64_t)c->frames[t].fr.K.width * c->frames[t].fr.K.height;   // the frames themselves (their descriptors are built later)
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CU(cudaEventCreate(&e0), "tuner event");
    CU(cudaEventCreate(&e1), "tuner event");
    densify_status st = DENSIFY_OK;
    for (int i = 0; i < c->p.num_stages && st == DENSIFY_OK; ++i) {
        const std::string key = tune_key(c, i, px);
        std::string cached;
        int best = 0;
        float best_us = -1.0f;
        bool from_cache = false;
        if (cache_lookup(key, &cached)) {
            for (size_t j = 0; j < c->cands[i].size(); ++j)
                if (cand_name(c->cands[i][j]) == cached) { best = (int)j; from_cache = true; }
        }
        if (!from_cache && c->cands[i].size() > 1) {
            for (size_t j = 0; j < c->cands[i].size() && st == DENSIFY_OK; ++j) {
                set_filter(c, i, c->cands[i][j]);
                for (uint64_t t : tk) {   // tensor-map boxes follow the candidate's tile
                    build_frame_dev(c, c->frames[t]);
                    const std::string me = encode_maps(c, c->frames[t].dev);
                    if (!me.empty()) {
                        c->dead = true;
                        c->err = me;
                        st = DENSIFY_E_CUDA;
                    }
                }
                if (st != DENSIFY_OK) break;
                fill_batch(c, sl, tk);
                if ((st = prepare_tile_lists(c, sl)) != DENSIFY_OK) break;
                const size_t bytes = offsetof(BatchDev, f) + sizeof(FrameDev) * tk.size();
                cudaError_t e = cudaMemcpyAsync(sl.d, sl.h, bytes, cudaMemcpyHostToDevice, sl.stream);
                // inputs of this stage
                if (e == cudaSuccess) e = launch_prep(sl.d, c->grid[K_PREP], sl.stream);
                if (e == cudaSuccess && c->p.motion_threshold > 0.0f) {
                    e = launch_motion(sl.d, c->pp, c->grid[K_MOTION], sl.stream);
                    if (e == cudaSuccess) e = launch_morph(sl.d, c->pp, true, c->grid[K_DILATE], sl.stream);
                    if (e == cudaSuccess) e = launch_morph(sl.d, c->pp, false, c->grid[K_ERODE], sl.stream);
                }
                if (e == cudaSuccess) e = launch_project(sl.d, c->grid[K_PROJECT], sl.stream);
                if (e == cudaSuccess && c->p.occlusion_radius > 0)
                    e = launch_occlusion(sl.d, c->pp, c->grid[K_OCCLUSION], sl.stream);
                if (e == cudaSuccess && c->p.num_stages == 2) e = launch_pool(sl.d, c->p.pool, c->grid[K_POOL], sl.stream);
                if (e == cudaSuccess && i == 1) e = launch_filter(c, 0, sl.d, sl.stream);
                if (e == cudaSuccess) e = launch_filter(c, i, sl.d, sl.stream);   // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(e0, sl.stream);
                for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) e = launch_filter(c, i, sl.d, sl.stream);
                if (e == cudaSuccess) e = cudaEventRecord(e1, sl.stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.0f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    st = cuda_fail(c, e, "autotune");
                    break;
                }
                const float us = 1000.0f * ms / 3.0f;
                c->cands[i][j].tuned_us = us;
                if (best_us < 0.0f || us < best_us) {
                    best_us = us;
                    best = (int)j;
                }
            }
            if (st == DENSIFY_OK) cache_store(key, cand_name(c->cands[i][best]));
        }
        set_filter(c, i, c->cands[i][best]);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tuned = true;
    return st;
}

// Tile geometry of the batch's TMA filters. The flags (one word per tile of both stages) are part
// of each frame's scratch, reserved at admission, so a batch allocates nothing.
densify_status prepare_tile_lists(densify_ctx *c, Slot &sl) {
    BatchDev &b = *sl.h;
    // the flags themselves live in each frame's scratch (FrameDev::tflags); tile geometry of the TMA stages: on the two-stage path the pooling kernel flags the first
    // stage's tiles and the first filter's epilogue the second's; a single stage's are flagged by
    // the mark kernel
    for (int i = 0; i < 2; ++i) {
        const bool on = i < c->p.num_stages && c->sel[i].tma;
        b.tl_tw[i] = on ? c->sel[i].tile_w : 32;
        b.tl_th[i] = on ? c->sel[i].tile_h : 0;
        b.tl_r[i] = on ? c->sel[i].radius : 0;
    }
    b.tl_on = b.tl_th[0] > 0 || b.tl_th[1] > 0;
    return DENSIFY_OK;
}

// The tiles of a TMA filter are flagged by the kernel in front of it: the pooling kernel for the
// first of two stages, the first filter for the second; a single stage has a mark kernel of its own.
bool tiles_marked_by_mark_kernel(const densify_ctx *c, int i) { return c->sel[i].tma && c->p.num_stages == 1; }

// CUDA kernels of one filter launch (a single TMA stage: tile marks + filter).
int filter_kernels(const densify_ctx *c, int i) { return tiles_marked_by_mark_kernel(c, i) ? 2 : 1; }

// In front of a TMA filter launched on its own (the autotuner's trials): the tile mark kernel,
// which also resets the tile counter (single stage), or the counter reset alone (two-stage path,
// whose batches reset both counters in the prep kernel). Nothing for the plain kernels.
cudaError_t launch_filter_scan(densify_ctx *c, int i, const BatchDev *b, cudaStream_t s) {
    const FilterSel &f = c->sel[i];
    if (!f.tma) return cudaSuccess;
    if (!tiles_marked_by_mark_kernel(c, i))
        return cudaMemsetAsync(const_cast<int32_t *>(&b->tl_next[i]), 0, sizeof(int32_t), s);
    return launch_tile_mark(f.src, b, i, f.tile_h, f.radius, c->sms * 8, s);
}

cudaError_t launch_filter_kernel(densify_ctx *c, int i, const BatchDev *b, cudaStream_t s) {
    const FilterSel &f = c->sel[i];
    const int k = i == 0 ? K_JBF1 : K_JBF2;
    if (f.tma) return launch_jbf_tma(f.src, f.radius, TmaVariant{f.kp, f.nw}, f.form, b, c->sa[i], c->grid[k], s);
    if (f.kind == 0) return launch_jbf_single(f.radius, b, c->sa[i], c->grid[k], s);
    if (f.kind == 1) return launch_jbf_coarse(f.radius, b, c->sa[i], c->grid[k], s);
    return launch_jbf_up(f.radius, b, c->sa[i], c->grid[k], s);
}

cudaError_t launch_filter(densify_ctx *c, int i, const BatchDev *b, cudaStream_t s) {
    cudaError_t e = launch_filter_scan(c, i, b, s);
    return e != cudaSuccess ? e : launch_filter_kernel(c, i, b, s);
}

// Tensor maps of one frame for the TMA filter kernels of the context.
std::string encode_maps(densify_ctx *c, FrameDev &d) {
    d.tma = 0;
    bool need = false;
    for (int i = 0; i < c->p.num_stages; ++i) need |= c->sel[i].tma;
    if (!need) return "";
    if (!tensor_map_encoder()) return "cuTensorMapEncodeTiled is not available";
    for (int i = 0; i < c->p.num_stages; ++i) {
        const FilterSel &f = c->sel[i];
        if (!f.tma) continue;
        const TmaKernelInfo &I = f.info;
        bool ok = true;
        if (f.src == TMA_SRC_UP || f.src == TMA_SRC_ZBUF)
            ok &= encode2d(&d.tm[TM_RGB], CU_TENSOR_MAP_DATA_TYPE_UINT8, d.rgb, (uint64_t)d.W * 3, d.H,
                           (uint64_t)d.rgb_pitch, I.rgb_box[0], I.rgb_box[1]);
        if (f.src == TMA_SRC_UP)
            ok &= encode2d(&d.tm[TM_S1], CU_TENSOR_MAP_DATA_TYPE_UINT64, d.s1, d.Wc, d.Hc, (uint64_t)d.cpitch * 8,
                           I.s1_box[0], I.s1_box[1]);
        if (f.src == TMA_SRC_ZBUF)
            ok &= encode2d(&d.tm[TM_ZBUF], CU_TENSOR_MAP_DATA_TYPE_UINT32, d.zbuf, d.W, d.H, (uint64_t)d.zpitch * 4,
                           I.zbuf_box[0], I.zbuf_box[1]);
        if (f.src == TMA_SRC_COARSE) {
            ok &= encode2d(&d.tm[TM_CGUIDE], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, d.cguide, (uint64_t)d.Wc * 4, d.Hc,
                           (uint64_t)d.cpitch * 16, I.cguide_box[0], I.cguide_box[1]);
            ok &= encode2d(&d.tm[TM_CSSUM], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, d.cssum, d.Wc, d.Hc,
                           (uint64_t)d.cpitch * 4, I.cssum_box[0], I.cssum_box[1]);
        }
        if (!ok) return "tensor map encoding failed";
    }
    d.tma = 1;
    return "";
}

// The fixed kernel sequence of one batch (captured into a graph or issued directly).
densify_status issue_kernels(densify_ctx *c, Slot &sl, cudaStream_t s, bool record_events) {
    const BatchDev *b = sl.d;
    const int nst = c->p.num_stages;
    int ev = 0;
    // timing 1: an event after every kernel (and one in front); timing 2: events around the
    // last filter kernel only (the full-resolution stage), which adds two graph nodes a batch
    const int last = nst == 2 ? K_JBF2 : K_JBF1;
    const bool all = c->p.timing == 1;
    auto record = [&]() -> cudaError_t {
        return cudaEventRecordWithFlags(sl.kev[ev++], s, s == c->cap_stream ? cudaEventRecordExternal : 0);
    };
    auto mark = [&](int k) -> cudaError_t {
        if (!record_events || (!all && k != last)) return cudaSuccess;
        if (k >= 0) sl.kord[sl.ntimed++] = k;
        return record();
    };
    auto start_last = [&]() -> cudaError_t {   // timing 2: the event in front of the last filter kernel
        return record_events && !all ? record() : cudaSuccess;
    };
    sl.ntimed = 0;
    int nk = 1 + (c->p.motion_threshold > 0.0f ? 3 : 0) + 1 + (c->p.occlusion_radius > 0 ? 1 : 0) +
             (nst == 2 ? 1 + filter_kernels(c, 0) + filter_kernels(c, 1) : filter_kernels(c, 0)) +
             (c->p.contour_threshold > 0.0f ? 1 : 0) + (c->p.emit_points ? 3 : 0);
    sl.nkern = nk;   // prep, motion (3), project, occlusion, pool, filters, contour, compaction (3)
    if (all) CU(mark(-1), "event");
    CU(launch_prep(b, c->grid[K_PREP], s), "prep launch");
    CU(mark(K_PREP), "event");
    if (c->p.motion_threshold > 0.0f) {
        CU(launch_motion(b, c->pp, c->grid[K_MOTION], s), "motion launch");
        CU(mark(K_MOTION), "event");
        CU(launch_morph(b, c->pp, true, c->grid[K_DILATE], s), "dilate launch");
        CU(mark(K_DILATE), "event");
        CU(launch_morph(b, c->pp, false, c->grid[K_ERODE], s), "erode launch");
        CU(mark(K_ERODE), "event");
    }
    CU(launch_project(b, c->grid[K_PROJECT], s), "project launch");
    CU(mark(K_PROJECT), "event");
    if (c->p.occlusion_radius > 0) {
        CU(launch_occlusion(b, c->pp, c->grid[K_OCCLUSION], s), "occlusion launch");
        CU(mark(K_OCCLUSION), "event");
    }
    if (nst == 2) {
        // the prep kernel reset both tile counters; pooling flags the first filter's tiles, the
        // first filter the second's
        CU(launch_pool(b, c->p.pool, c->grid[K_POOL], s), "pool launch");
        CU(mark(K_POOL), "event");
        CU(launch_filter_kernel(c, 0, b, s), "stage-1 filter launch");
        CU(mark(K_JBF1), "event");
        CU(start_last(), "event");
        CU(launch_filter_kernel(c, 1, b, s), "stage-2 filter launch");
        CU(mark(K_JBF2), "event");
    } else {
        if (c->sel[0].tma) {
            CU(launch_filter_scan(c, 0, b, s), "tile mark launch");
            CU(mark(K_MARK1), "event");
        }
        CU(start_last(), "event");
        CU(launch_filter_kernel(c, 0, b, s), "filter launch");
        CU(mark(K_JBF1), "event");
    }
    if (c->p.contour_threshold > 0.0f) {
        CU(launch_contour(b, c->pp, c->grid[K_CONTOUR], s), "contour launch");
        CU(mark(K_CONTOUR), "event");
    }
    if (c->p.emit_points) {
        CU(launch_bp_count(b, c->grid[K_BP_COUNT], s), "compaction count launch");
        CU(mark(K_BP_COUNT), "event");
        CU(launch_bp_write(b, c->grid[K_BP_WRITE], s), "compaction write launch");   // see settle_grids
        CU(mark(K_BP_WRITE), "event");
    }
    return DENSIFY_OK;
}

// The first batch settles the kernel grids (they are part of every slot's graph). A compaction
// write whose points go straight into page-locked host memory runs at the host link's rate, about
// a millisecond for eight 1080p frames; with the persistent grid on every SM it would hold them all
// that long, and the next batch's kernels (on another slot's stream) could not start. When every
// frame of the first batch writes its points that way, the compaction write gets an eighth of its
// persistent grid (one block on every second SM), which still keeps the link busy, and the rest run
// the next batch (measured on eight 1080p frames, three batches in flight: 6.6k frames/s end to end
// at an eighth, 6.3k at a quarter, 6.1k at a half, 6.2k at a sixteenth).
void settle_grids(densify_ctx *c, const std::vector<uint64_t> &tk) {
    if (c->grids_fixed) return;
    c->grids_fixed = true;
    // (only a context with its own streams overlaps its slots' batches)
    bool host_points = c->p.emit_points && c->own_stream && c->slots.size() > 1 && !tk.empty();
    for (uint64_t t : tk) host_points &= c->frames[t].L.points_direct != nullptr;
    if (host_points) c->grid[K_BP_WRITE] = std::max(1, c->grid[K_BP_WRITE] / 8);
}

// Capture a slot's kernel sequence (its own device descriptor) into a graph, instantiate it and
// upload it to the device ahead of its first launch.
densify_status capture_slot(densify_ctx *c, Slot &sl) {
    CU(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    densify_status st = issue_kernels(c, sl, c->cap_stream, c->p.timing != 0);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (st != DENSIFY_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
    e = cudaGraphInstantiate(&sl.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
    CU(cudaGraphUpload(sl.exec, sl.stream), "graph upload");
    return DENSIFY_OK;
}

densify_status launch_batch(densify_ctx *c, int si) {
    Slot &sl = c->slots[si];
    std::vector<uint64_t> tk;
    while (!c->queue.empty() && (int)tk.size() < c->p.max_batch) {
        tk.push_back(c->queue.front());
        c->queue.pop_front();
    }
    if (tk.empty()) return DENSIFY_OK;
    if (!c->tuned) {   // first batch: pick the filter kernels
        densify_status st = autotune(c, sl, tk);
        if (st != DENSIFY_OK) return st;
    }
    settle_grids(c, tk);
    for (uint64_t t : tk) {
        build_frame_dev(c, c->frames[t]);
        const std::string e = encode_maps(c, c->frames[t].dev);
        if (!e.empty()) {
            c->dead = true;
            c->err = e;
            return DENSIFY_E_CUDA;
        }
    }
    fill_batch(c, sl, tk);
    {
        densify_status st = prepare_tile_lists(c, sl);
        if (st != DENSIFY_OK) return st;
    }
    const size_t bytes = offsetof(BatchDev, f) + sizeof(FrameDev) * tk.size();
    CU(cudaMemcpyAsync(sl.d, sl.h, bytes, cudaMemcpyHostToDevice, sl.stream), "descriptor upload");
    // host frames: inputs in
    for (uint64_t t : tk) {
        FrameRec &r = c->frames[t];
        if (r.fr.memory != DENSIFY_MEM_HOST) continue;
        for (int s = 0; s < r.fr.num_scans; ++s)
            if (r.fr.scans[s].count > 0)
                CU(cudaMemcpyAsync((void *)r.dev.scans[s].xyz, r.fr.scans[s].xyz,
                                   (size_t)r.fr.scans[s].count * r.fr.scans[s].stride_bytes, cudaMemcpyHostToDevice,
                                   sl.stream),
                   "points upload");
    }
    // previous frame of host frames (afterimage removal)
    for (uint64_t t : tk) {
        FrameRec &r = c->frames[t];
        if (!r.L.has_motion || r.fr.memory != DENSIFY_MEM_HOST) continue;
        CU(cudaMemcpy2DAsync((void *)r.dev.prev_rgb, (size_t)r.dev.prev_pitch, r.fr.prev_rgb, (size_t)r.fr.prev_rgb_pitch,
                             (size_t)r.fr.K.width * 3, (size_t)r.fr.K.height, cudaMemcpyHostToDevice, sl.stream),
           "previous frame upload");
    }
    // RGB staging (host frames, and device frames whose base or pitch is not 16-byte aligned)
    for (uint64_t t : tk) {
        FrameRec &r = c->frames[t];
        if (!r.L.rgb_pitch) continue;
        CU(cudaMemcpy2DAsync((void *)r.dev.rgb, (size_t)r.dev.rgb_pitch, r.fr.rgb, (size_t)r.fr.rgb_pitch,
                             (size_t)r.fr.K.width * 3, (size_t)r.fr.K.height,
                             r.fr.memory == DENSIFY_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                             sl.stream),
           "rgb staging");
    }
    if (c->p.use_graphs) {
        // the first batch captures, instantiates and uploads every slot's graph (the kernel sequence
        // is fixed once the filter kernels are chosen), so no later batch pays for a capture
        for (auto &other : c->slots) {
            if (other.exec) continue;
            densify_status st = capture_slot(c, other);
            if (st != DENSIFY_OK) return st;
        }
        CU(cudaGraphLaunch(sl.exec, sl.stream), "graph launch");
    } else {
        densify_status st = issue_kernels(c, sl, sl.stream, c->p.timing != 0);
        if (st != DENSIFY_OK) return st;
    }
    // debug motion mask out, both memory kinds
    for (uint64_t t : tk) {
        FrameRec &r = c->frames[t];
        if (!r.fr.out_motion || !r.L.has_motion) continue;
        CU(cudaMemcpyAsync(r.fr.out_motion, r.dev.motion, (size_t)r.fr.K.width * r.fr.K.height,
                           r.fr.memory == DENSIFY_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                           sl.stream),
           "motion copy");
    }
    // debug z-buffer out (row pitch W), both memory kinds
    for (uint64_t t : tk) {
        FrameRec &r = c->frames[t];
        if (!r.fr.out_zbuf) continue;
        CU(cudaMemcpy2DAsync(r.fr.out_zbuf, (size_t)r.fr.K.width * 4, r.dev.zbuf, (size_t)r.dev.zpitch * 4,
                             (size_t)r.fr.K.width * 4, (size_t)r.fr.K.height,
                             r.fr.memory == DENSIFY_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                             sl.stream),
           "zbuf copy");
    }
    // host frames: results out (points are copied at poll time, exactly n of them)
    for (uint64_t t : tk) {
        FrameRec &r = c->frames[t];
        if (r.fr.memory != DENSIFY_MEM_HOST) continue;
        const size_t npx = (size_t)r.fr.K.width * r.fr.K.height;
        if (r.fr.out_depth)
            CU(cudaMemcpyAsync(r.fr.out_depth, r.dev.out_depth, npx * 4, cudaMemcpyDeviceToHost, sl.stream), "depth copy");
        if (r.fr.out_valid)
            CU(cudaMemcpyAsync(r.fr.out_valid, r.dev.out_valid, npx, cudaMemcpyDeviceToHost, sl.stream), "valid copy");
        if (c->p.num_stages == 2) {
            const size_t nc = (size_t)r.dev.Wc * r.dev.Hc;
            if (r.fr.out_coarse)
                CU(cudaMemcpyAsync(r.fr.out_coarse, r.dev.out_coarse, nc * 4, cudaMemcpyDeviceToHost, sl.stream),
                   "coarse copy");
            if (r.fr.out_coarse_valid)
                CU(cudaMemcpyAsync(r.fr.out_coarse_valid, r.dev.out_coarse_valid, nc, cudaMemcpyDeviceToHost,
                                   sl.stream),
                   "coarse valid copy");
        }
        if (c->p.emit_points && !r.L.count_direct)
            CU(cudaMemcpyAsync(r.fr.out_points_n, r.dev.points_n, 8, cudaMemcpyDeviceToHost, sl.stream), "count copy");
    }
    if (c->inject_wait_failure) {   // test hook: the status a kernel sets when a bounded wait gives up (bit 0)
        CU(cudaMemsetAsync(sl.d_status, 1, 1, sl.stream), "status injection");
        c->inject_wait_failure = false;
    }
    CU(cudaMemcpyAsync(sl.h_status, sl.d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, sl.stream), "status copy");
    CU(cudaEventRecord(sl.done, sl.stream), "event record");
    for (uint64_t t : tk) {
        FrameRec &r = c->frames[t];
        r.state = 1;
        r.slot = si;
    }
    sl.tickets = tk;
    sl.busy = true;
    ++c->batches;
    int busy = 0;
    for (const auto &other : c->slots) busy += other.busy;
    c->max_busy = std::max(c->max_busy, busy);
    return DENSIFY_OK;
}

densify_status complete_slot(densify_ctx *c, Slot &sl) {
    if (*sl.h_status != 0) {
        c->dead = true;
        c->err = "a kernel's bounded wait on its tile copies gave up (status " + std::to_string(*sl.h_status) + ")";
        return DENSIFY_E_CUDA;
    }
    if (c->p.timing) {
        for (int j = 0; j < sl.ntimed; ++j) {
            const int k = sl.kord[j];
            float ms = 0.0f;
            CU(cudaEventElapsedTime(&ms, sl.kev[j], sl.kev[j + 1]), "elapsed time");
            c->t_us[k] += 1000.0 * ms;
            c->t_n[k] += 1;
        }
    }
    c->kernel_launches += sl.nkern;
    for (uint64_t t : sl.tickets) {
        auto it = c->frames.find(t);
        if (it != c->frames.end()) it->second.state = 2;
    }
    sl.tickets.clear();
    sl.busy = false;
    return DENSIFY_OK;
}

densify_status progress(densify_ctx *c, bool launch) {
    if (c->dead) return DENSIFY_E_CUDA;
    for (auto &sl : c->slots) {
        if (!sl.busy) continue;
        cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaSuccess) {
            densify_status st = complete_slot(c, sl);
            if (st != DENSIFY_OK) return st;
        } else if (q != cudaErrorNotReady) {
            return cuda_fail(c, q, "batch failed");
        }
    }
    if (launch) {
        for (int si = 0; si < (int)c->slots.size() && !c->queue.empty(); ++si) {
            if (c->slots[si].busy) continue;
            densify_status st = launch_batch(c, si);
            if (st != DENSIFY_OK) return st;
        }
    }
    return DENSIFY_OK;
}

bool any_busy(const densify_ctx *c) {
    for (const auto &sl : c->slots)
        if (sl.busy) return true;
    return false;
}

// Bounded wait for some busy slot to finish: spin on the event with a yield.
densify_status wait_some(densify_ctx *c, int64_t deadline_ns) {
    while (true) {
        for (auto &sl : c->slots) {
            if (!sl.busy) continue;
            cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaSuccess) return DENSIFY_OK;
            if (q != cudaErrorNotReady) return cuda_fail(c, q, "batch failed");
        }
        if (deadline_ns >= 0 && now_ns() >= deadline_ns) return DENSIFY_E_TIMEOUT;
        std::this_thread::yield();
    }
}

densify_status finalize(densify_ctx *c, FrameRec &r) {
    if (r.fr.memory == DENSIFY_MEM_HOST && c->p.emit_points && r.fr.out_points && r.fr.out_points_cap > 0 &&
        !r.L.points_direct) {
        const int64_t n = std::min<int64_t>(*r.fr.out_points_n, r.fr.out_points_cap);
        if (n > 0) {
            CU(cudaMemcpyAsync(r.fr.out_points, r.dev.out_points, (size_t)n * 16, cudaMemcpyDeviceToHost,
                               c->d2h_stream),
               "points copy");
            CU(cudaStreamSynchronize(c->d2h_stream), "points copy sync");
        }
    }
    return DENSIFY_OK;
}

void destroy_resources(densify_ctx *c) {
    for (auto &sl : c->slots) {
        if (sl.exec) cudaGraphExecDestroy(sl.exec);
        if (sl.done) cudaEventDestroy(sl.done);
        for (auto &e : sl.kev)
            if (e) cudaEventDestroy(e);
        if (sl.own_stream && sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.d) cudaFree(sl.d);
        if (sl.h) cudaFreeHost(sl.h);
        if (sl.d_status) cudaFree(sl.d_status);
        if (sl.h_status) cudaFreeHost(sl.h_status);
    }
    c->slots.clear();
    if (c->arena_base) cudaFree(c->arena_base);
    c->arena_base = nullptr;
    if (c->zpool_base) cudaFree(c->zpool_base);
    c->zpool_base = nullptr;
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->d2h_stream) cudaStreamDestroy(c->d2h_stream);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int32_t densify_abi_version(void) { return DENSIFY_ABI_VERSION; }

const char *densify_status_str(densify_status s) {
    switch (s) {
    case DENSIFY_OK: return "DENSIFY_OK";
    case DENSIFY_PENDING: return "DENSIFY_PENDING";
    case DENSIFY_E_INVALID: return "DENSIFY_E_INVALID";
    case DENSIFY_E_NOMEM: return "DENSIFY_E_NOMEM";
    case DENSIFY_E_AGAIN: return "DENSIFY_E_AGAIN";
    case DENSIFY_E_CUDA: return "DENSIFY_E_CUDA";
    case DENSIFY_E_TIMEOUT: return "DENSIFY_E_TIMEOUT";
    case DENSIFY_E_TICKET: return "DENSIFY_E_TICKET";
    }
    return "DENSIFY_UNKNOWN";
}

const char *densify_last_error(const densify_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

void densify_default_params(densify_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->num_stages = 2;
    p->stage[0] = densify_stage{4, 5.0f, 20.0f};
    p->stage[1] = densify_stage{2, 5.0f, 20.0f};
    p->pool = 3;
    p->stage2_input = 0;
    p->precision = DENSIFY_FP32;
    p->emit_points = 1;
    p->max_inflight = 16;
    p->max_batch = 16;
    p->batches_in_flight = 1;
    p->use_graphs = 1;
    p->hbm_budget_bytes = (uint64_t)2 << 30;
    p->timing = 0;
    p->launch_policy = 0;
    p->kernel_variant = 0;
    p->autotune = 0;
}

uint64_t densify_frame_scratch_bytes(const densify_params *params, const densify_frame *frame) {
    if (!params || !frame) return 0;
    const Layout L = layout_of(*params, frame);
    return L.total + L.zbytes;
}

densify_status densify_create(const densify_params *params, int device, void *cuda_stream, densify_ctx **out) {
    if (!out) return fail(nullptr, DENSIFY_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!params) return fail(nullptr, DENSIFY_E_INVALID, "params is NULL");
    const std::string perr = validate_params(*params);
    if (!perr.empty()) return fail(nullptr, DENSIFY_E_INVALID, perr);
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return fail(nullptr, DENSIFY_E_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    if (device < 0 || device >= ndev) return fail(nullptr, DENSIFY_E_INVALID, "device out of range");
    DeviceGuard guard(device);
    densify_ctx *c = new densify_ctx();
    c->device = device;
    c->p = *params;
    auto bail = [&](densify_status s, const std::string &m) {
        g_create_error = m + (c->err.empty() ? "" : (": " + c->err));
        destroy_resources(c);
        delete c;
        return s;
    };
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(DENSIFY_E_CUDA, std::string("stream: ") + cudaGetErrorString(e));
        c->own_stream = true;
    }
    if ((e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&c->d2h_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(DENSIFY_E_CUDA, std::string("stream: ") + cudaGetErrorString(e));
    // a quarter of the budget holds the clean z-buffers where they apply (a 1080p frame's z-buffer is
    // about a quarter of its scratch), the rest the other scratch
    const uint64_t zpool_bytes = zpool_applies(*params) ? (params->hbm_budget_bytes / 4) & ~(kAlign - 1) : 0;
    const uint64_t arena_bytes = params->hbm_budget_bytes - zpool_bytes;
    if ((e = cudaMalloc(&c->arena_base, arena_bytes)) != cudaSuccess) {
        cudaGetLastError();
        return bail(DENSIFY_E_NOMEM, std::string("arena: ") + cudaGetErrorString(e));
    }
    c->arena.init(arena_bytes);
    if (zpool_bytes) {
        if ((e = cudaMalloc(&c->zpool_base, zpool_bytes)) != cudaSuccess) {
            cudaGetLastError();
            return bail(DENSIFY_E_NOMEM, std::string("z-buffer pool: ") + cudaGetErrorString(e));
        }
        if ((e = launch_fill_empty((uint32_t *)c->zpool_base, zpool_bytes / 4, c->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
            return bail(DENSIFY_E_CUDA, std::string("z-buffer pool: ") + cudaGetErrorString(e));
        c->zpool.init(zpool_bytes);
    }
    c->slots.resize(params->batches_in_flight);
    for (auto &sl : c->slots) {
        // a context that owns its streams gives every slot its own, so that one batch's host copies
        // overlap another batch's kernels; with a caller stream every batch is ordered on it
        if (c->own_stream && c->slots.size() > 1) {
            if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess)
                return bail(DENSIFY_E_CUDA, std::string("slot stream: ") + cudaGetErrorString(e));
            sl.own_stream = true;
        } else {
            sl.stream = c->stream;
        }
        if ((e = cudaMalloc(&sl.d, sizeof(BatchDev))) != cudaSuccess ||
            (e = cudaMallocHost(&sl.h, sizeof(BatchDev))) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaMalloc(&sl.d_status, 256)) != cudaSuccess ||
            (e = cudaMallocHost(&sl.h_status, sizeof(int32_t))) != cudaSuccess ||
            (e = cudaMemset(sl.d_status, 0, 256)) != cudaSuccess)
            return bail(DENSIFY_E_CUDA, std::string("slot: ") + cudaGetErrorString(e));
        *sl.h_status = 0;
        if (params->timing)
            for (auto &ev : sl.kev)
                if ((e = cudaEventCreate(&ev)) != cudaSuccess)
                    return bail(DENSIFY_E_CUDA, std::string("event: ") + cudaGetErrorString(e));
    }
    // stage constants
    if (params->num_stages == 1) {
        fill_stage(c->sa[0], params->stage[0], 1, 0);
    } else {
        fill_stage(c->sa[0], params->stage[0], params->pool, 0);
        fill_stage(c->sa[1], params->stage[1], params->pool, params->stage2_input);
    }
    // persistent grids: SM count x resident blocks
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
        return bail(DENSIFY_E_CUDA, std::string("attribute: ") + cudaGetErrorString(e));
    c->grid[K_PREP] = sms * occupancy_points(K_PREP);
    c->grid[K_PROJECT] = sms * occupancy_points(K_PROJECT);
    c->grid[K_POOL] = sms * occupancy_pool_bp(K_POOL);
    c->grid[K_BP_COUNT] = sms * occupancy_pool_bp(K_BP_COUNT);
    c->grid[K_BP_WRITE] = sms * occupancy_pool_bp(K_BP_WRITE);
    for (KernelId k : {K_MOTION, K_DILATE, K_ERODE, K_OCCLUSION, K_CONTOUR}) c->grid[k] = sms * occupancy_prepost(k);
    c->pp.motion_t2 = params->motion_threshold * params->motion_threshold;
    c->pp.close_radius = params->motion_close_radius;
    c->pp.occ_radius = params->occlusion_radius;
    c->pp.occ_margin = params->occlusion_margin;
    c->pp.contour_t = params->contour_threshold;
    c->sms = sms;
    for (int i = 0; i < params->num_stages; ++i) {
        const int kind = params->num_stages == 1 ? 0 : (i == 0 ? 1 : 2);
        c->cands[i] = filter_candidates(*params, kind, params->stage[i].radius);
        if (c->cands[i].empty()) return bail(DENSIFY_E_INVALID, "no kernel for filter stage " + std::to_string(i));
        for (FilterSel &f : c->cands[i]) {
            if (f.tma) {
                if ((e = jbf_tma_prepare(f.src, f.radius, TmaVariant{f.kp, f.nw}, f.form)) != cudaSuccess)
                    return bail(DENSIFY_E_CUDA, std::string("filter setup: ") + cudaGetErrorString(e));
                f.occ = occupancy_jbf_tma(f.src, f.radius, TmaVariant{f.kp, f.nw}, f.form);
            } else {
                f.occ = kind == 0 ? occupancy_jbf_single(f.radius) : kind == 1 ? occupancy_jbf_coarse(f.radius)
                                                                              : occupancy_jbf_up(f.radius);
            }
        }
        set_filter(c, i, c->cands[i][0]);
    }
    c->tuned = !params->autotune;
    if ((e = cudaGetLastError()) != cudaSuccess)
        return bail(DENSIFY_E_CUDA, std::string("setup: ") + cudaGetErrorString(e));
    *out = c;
    return DENSIFY_OK;
}

densify_status densify_submit(densify_ctx *c, const densify_frame *frame, uint64_t *ticket) {
    if (!c) return fail(nullptr, DENSIFY_E_INVALID, "ctx is NULL");
    if (!ticket) return fail(c, DENSIFY_E_INVALID, "ticket is NULL");
    *ticket = 0;
    if (c->dead) return DENSIFY_E_CUDA;
    const std::string ferr = validate_frame(c, frame);
    if (!ferr.empty()) return fail(c, DENSIFY_E_INVALID, ferr);
    DeviceGuard guard(c->device);
    densify_status st = progress(c, false);
    if (st != DENSIFY_OK) return st;
    if (c->admitted >= c->p.max_inflight) return fail(c, DENSIFY_E_AGAIN, "max_inflight frames admitted");
    FrameRec r;
    r.fr = *frame;
    r.L = layout_of(c->p, frame);
    if (r.L.total > c->arena.size() || r.L.zbytes > c->zpool.size())
        return fail(c, DENSIFY_E_NOMEM, "frame scratch exceeds hbm_budget_bytes");
    if (!c->arena.alloc(r.L.total, &r.off)) return fail(c, DENSIFY_E_AGAIN, "scratch arena full");
    if (r.L.zpooled && !c->zpool.alloc(r.L.zbytes, &r.zoff)) {
        c->arena.release(r.off, r.L.total);
        return fail(c, DENSIFY_E_AGAIN, "z-buffer pool full");
    }
    const uint64_t t = c->next_ticket++;
    c->frames.emplace(t, r);
    c->queue.push_back(t);
    c->admitted++;
    *ticket = t;
    const bool eager = c->p.launch_policy == 0;
    if (eager || (int)c->queue.size() >= c->p.max_batch) return progress(c, true);
    return DENSIFY_OK;
}

densify_status densify_flush(densify_ctx *c, int64_t timeout_ns) {
    if (!c) return fail(nullptr, DENSIFY_E_INVALID, "ctx is NULL");
    DeviceGuard guard(c->device);
    const int64_t deadline = timeout_ns < 0 ? -1 : now_ns() + timeout_ns;
    while (true) {
        densify_status st = progress(c, true);
        if (st != DENSIFY_OK) return st;
        if (c->queue.empty()) return DENSIFY_OK;
        if (timeout_ns == 0) return DENSIFY_PENDING;
        st = wait_some(c, deadline);
        if (st != DENSIFY_OK) return st;
    }
}

densify_status densify_poll(densify_ctx *c, uint64_t ticket, int64_t timeout_ns) {
    if (!c) return fail(nullptr, DENSIFY_E_INVALID, "ctx is NULL");
    auto it = c->frames.find(ticket);
    if (it == c->frames.end()) return fail(c, DENSIFY_E_TICKET, "unknown ticket");
    DeviceGuard guard(c->device);
    const int64_t deadline = timeout_ns < 0 ? -1 : now_ns() + timeout_ns;
    while (true) {
        densify_status st = progress(c, true);
        if (st != DENSIFY_OK) return st;
        FrameRec &r = c->frames[ticket];
        if (r.state == 2) {
            st = finalize(c, r);
            c->arena.release(r.off, r.L.total);
            if (r.L.zpooled) c->zpool.release(r.zoff, r.L.zbytes);
            c->frames.erase(ticket);
            c->admitted--;
            return st;
        }
        if (timeout_ns == 0) return DENSIFY_PENDING;
        if (deadline >= 0 && now_ns() >= deadline) return fail(c, DENSIFY_E_TIMEOUT, "poll timed out");
        if (r.state == 1 && timeout_ns < 0) {
            cudaError_t e = cudaEventSynchronize(c->slots[r.slot].done);
            if (e != cudaSuccess) return cuda_fail(c, e, "batch failed");
            continue;
        }
        if (!any_busy(c) && r.state == 0) continue;   // a slot is free: the next progress launches it
        st = wait_some(c, deadline);
        if (st == DENSIFY_E_TIMEOUT) return fail(c, st, "poll timed out");
        if (st != DENSIFY_OK) return st;
    }
}

densify_status densify_destroy(densify_ctx *c) {
    if (!c) return DENSIFY_E_INVALID;
    densify_status ret = DENSIFY_OK;
    {
        DeviceGuard guard(c->device);
        const int64_t per = 10ll * 1000 * 1000 * 1000;
        for (auto &sl : c->slots) {
            if (!sl.busy) continue;
            const int64_t deadline = now_ns() + per;
            while (true) {
                cudaError_t q = cudaEventQuery(sl.done);
                if (q == cudaSuccess) break;
                if (q != cudaErrorNotReady) { ret = DENSIFY_E_CUDA; break; }
                if (now_ns() >= deadline) { ret = DENSIFY_E_TIMEOUT; break; }
                std::this_thread::yield();
            }
        }
        if (ret == DENSIFY_OK) destroy_resources(c);
    }
    if (ret == DENSIFY_OK) delete c;
    return ret;
}

int32_t densify_kernel_times(densify_ctx *c, const char **names, double *total_us, int64_t *launches, int32_t cap) {
    if (!c) return 0;
    DeviceGuard guard(c->device);
    progress(c, false);
    int32_t n = 0;
    for (int k = 0; k < K_COUNT && n < cap; ++k) {
        if (c->t_n[k] == 0) continue;
        if (names) names[n] = kKernelNames[k];
        if (total_us) total_us[n] = c->t_us[k];
        if (launches) launches[n] = c->t_n[k];
        ++n;
    }
    return n;
}

densify_status densify_sigma_grad(densify_ctx *c, const densify_frame *frame, const float *gt, double *loss,
                                  double *grad, int64_t *n_pixels) {
    if (!c) return fail(nullptr, DENSIFY_E_INVALID, "ctx is NULL");
    if (!gt || !loss || !grad) return fail(c, DENSIFY_E_INVALID, "gt_depth, loss and grad must not be NULL");
    if (c->dead) return DENSIFY_E_CUDA;
    const std::string ferr = validate_frame(c, frame);
    if (!ferr.empty()) return fail(c, DENSIFY_E_INVALID, ferr);
    if (frame->memory != DENSIFY_MEM_DEVICE) return fail(c, DENSIFY_E_INVALID, "the sigma gradient takes device frames");
    DeviceGuard guard(c->device);
    // in-flight batches first (bounded: 10 s each)
    while (any_busy(c)) {
        densify_status st = wait_some(c, now_ns() + 10ll * 1000 * 1000 * 1000);
        if (st != DENSIFY_OK) return st == DENSIFY_E_TIMEOUT ? fail(c, st, "waiting for in-flight batches") : st;
        if ((st = progress(c, false)) != DENSIFY_OK) return st;
    }
    densify_params p = c->p;
    p.emit_points = 0;
    FrameRec r;
    r.fr = *frame;
    r.fr.out_zbuf = nullptr;
    r.L = layout_of(p, &r.fr, false);   // its z-buffer in the main arena, cleared by the prep kernel
    const int grid = c->sms * 4;
    const int pool = p.num_stages == 2 ? p.pool : 1;
    const int64_t Wc = (frame->K.width + pool - 1) / pool, Hc = (frame->K.height + pool - 1) / pool;
    const uint64_t off_g1 = r.L.total;
    const uint64_t off_part = off_g1 + align_up((uint64_t)((Wc + 3) & ~3) * Hc * 8);
    const uint64_t hdr = offsetof(BatchDev, f) + sizeof(FrameDev);
    const uint64_t off_batch = off_part + align_up((uint64_t)grid * 6 * 4);
    const uint64_t total = off_batch + align_up(hdr);
    if (total > c->arena.size()) return fail(c, DENSIFY_E_NOMEM, "frame scratch exceeds hbm_budget_bytes");
    if (!c->arena.alloc(total, &r.off)) return fail(c, DENSIFY_E_AGAIN, "scratch arena full");
    char *base = (char *)c->arena_base + r.off;
    build_frame_dev(c, r);
    FrameDev &d = r.dev;
    d.zbuf_raw = d.zbuf;       // no preprocessing in the gradient
    d.motion = nullptr;
    d.g1 = (float2 *)(base + off_g1);
    std::unique_ptr<BatchDev> hbuf(new BatchDev());   // zeroed, correctly aligned
    BatchDev *hb = hbuf.get();
    hb->n_frames = 1;
    hb->zb_pre[1] = ceil_div((int64_t)d.zpitch * d.H, kZbWordsPerChunk);
    for (int s = 0; s < kMaxScans; ++s) hb->pt_pre[s + 1] = hb->pt_pre[s] + ceil_div(d.scans[s].count, kPtsPerChunk);
    hb->pool_pre[1] = p.num_stages == 2 ? ceil_div(d.Wc, kPoolPerChunk) * d.Hc : 0;
    hb->px_pre[1] = d.n_px_chunks;
    std::memcpy(&hb->f[0], &d, sizeof(FrameDev));
    GradArgs ga{};
    ga.two_stage = p.num_stages == 2;
    ga.pool = pool;
    for (int i = 0; i < p.num_stages; ++i) {
        const double log2e = 1.4426950408889634, sp = p.stage[i].sigma_p, sc = p.stage[i].sigma_c;
        ga.s[i].radius = p.stage[i].radius;
        ga.s[i].kc = (float)(log2e / (2.0 * sc * sc));
        ga.s[i].kp = (float)(log2e / (2.0 * sp * sp));
        ga.s[i].inv_sc3 = (float)(1.0 / (sc * sc * sc));
        ga.s[i].inv_sp3 = (float)(1.0 / (sp * sp * sp));
    }
    cudaStream_t s = c->slots[0].stream;
    BatchDev *bd = (BatchDev *)(base + off_batch);
    std::vector<float> host_part((size_t)grid * 6);
    cudaError_t e = cudaMemcpyAsync(bd, hb, hdr, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_prep(bd, c->grid[K_PREP], s);
    if (e == cudaSuccess) e = launch_project(bd, c->grid[K_PROJECT], s);
    if (e == cudaSuccess && ga.two_stage) e = launch_pool(bd, pool, c->grid[K_POOL], s);
    if (e == cudaSuccess) e = launch_grad(bd, ga, gt, (float *)(base + off_part), grid, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_part.data(), base + off_part, host_part.size() * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    c->arena.release(r.off, total);
    if (e != cudaSuccess) return cuda_fail(c, e, "sigma gradient");
    double host_out[6] = {0, 0, 0, 0, 0, 0};   // the blocks' FP32 partial sums, added on the host in FP64
    for (int b = 0; b < grid; ++b)
        for (int k = 0; k < 6; ++k) host_out[k] += (double)host_part[(size_t)b * 6 + k];
    const double n = host_out[1];
    *loss = n > 0 ? host_out[0] / n : 0.0;
    for (int k = 0; k < 4; ++k) grad[k] = n > 0 ? host_out[2 + k] / n : 0.0;
    if (n_pixels) *n_pixels = (int64_t)n;
    return DENSIFY_OK;
}

int32_t densify_describe(densify_ctx *c, char *buf, int32_t cap) {
    if (!c) return 0;
    auto one = [&](const FilterSel &f) {
        char tmp[256];
        std::snprintf(tmp, sizeof tmp,
                      "{\"kernel\": \"%s\", \"kp\": %d, \"warps\": %d, \"tile\": [%d, %d], \"fp16\": %s, "
                      "\"form\": \"%s\", \"ctas_per_sm\": %d%s",
                      f.tma ? "tma" : "plain", f.kp, f.nw, f.tile_w, f.tile_h, f.half ? "true" : "false",
                      f.form == TMA_FORM_SPARSE_FP16 ? "fp16_sparse"
                      : f.half                        ? "fp16"
                      : f.form == TMA_FORM_SPARSE    ? "fp32_sparse"
                      : f.form == TMA_FORM_EXP_PAIRS ? "fp32_expanded_pairs"
                      : f.form == TMA_FORM_EXP        ? "fp32_expanded"
                                                      : "fp32",
                      f.occ,
                      f.tuned_us >= 0.0f ? "" : "}");
        std::string s(tmp);
        if (f.tuned_us >= 0.0f) {
            std::snprintf(tmp, sizeof tmp, ", \"tuned_us\": %.3f}", f.tuned_us);
            s += tmp;
        }
        return s;
    };
    std::string out = "{\"tuned\": " + std::string(c->tuned && c->p.autotune ? "true" : "false") + ", \"stages\": [";
    for (int i = 0; i < c->p.num_stages; ++i) {
        if (i) out += ", ";
        out += "{\"chosen\": " + one(c->sel[i]) + ", \"candidates\": [";
        for (size_t j = 0; j < c->cands[i].size(); ++j) {
            if (j) out += ", ";
            out += one(c->cands[i][j]);
        }
        out += "]}";
    }
    out += "], \"batches\": {\"launched\": " + std::to_string(c->batches) +
           ", \"max_in_flight\": " + std::to_string(c->max_busy) + "}}";
    if (buf && cap > 0) {
        const size_t n = std::min<size_t>(out.size(), (size_t)cap - 1);
        std::memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return (int32_t)out.size();
}

void densify_reset_kernel_times(densify_ctx *c) {
    if (!c) return;
    for (int k = 0; k < K_COUNT; ++k) {
        c->t_us[k] = 0.0;
        c->t_n[k] = 0;
    }
    c->kernel_launches = 0;
}

densify_status densify_inject_wait_failure(densify_ctx *c) {
    if (!c) return fail(nullptr, DENSIFY_E_INVALID, "ctx is NULL");
    if (c->dead) return DENSIFY_E_CUDA;
    c->inject_wait_failure = true;
    return DENSIFY_OK;
}

int64_t densify_kernel_launches(densify_ctx *c) {
    if (!c) return 0;
    DeviceGuard guard(c->device);
    progress(c, false);
    return c->kernel_launches;
}

}  // extern "C"

namespace dz {

void fill_stage_args(StageArgs &a, const densify_stage &st, int pool, int override_sparse) {
    fill_stage(a, st, pool, override_sparse);
}

std::string check_params(const densify_params &p) { return validate_params(p); }

void set_thread_error(const std::string &m) { g_create_error = m; }

}  // namespace dz
