// densify_frame_noalloc: the whole path for one frame without any device
// allocation, for callers that cannot call cudaMalloc (for example code that
// runs inside a real-time loop with a frozen memory footprint, or a host that
// shares the GPU under an allocator it does not own).
//
// The scratch the kernels need (batch descriptor, status word, z-buffer,
// pooled maps, first-stage result, compaction counts) lives in one file-scope
// __device__ array of kNoallocScratchBytes per device. Host code cannot use
// the array's name as a device address, so at set-up (once per device, on the
// first call made with that device current) the entry point asks the runtime
// for the array's device address with cudaGetSymbolAddress and passes that
// pointer to the kernels. Everything the kernels read is rewritten or cleared
// on every call: the descriptor and status by a one-block init kernel, the
// z-buffer by the clear kernel, the other maps before they are read.
#include <cstring>
#include <mutex>
#include <string>

#include "runtime_internal.h"

namespace dz {

namespace {

constexpr size_t kNoallocScratchBytes = size_t(16) << 20;   // enough for one 1920x1080 two-stage frame
constexpr int kMaxDevices = 64;

}  // namespace

// The scratch itself: one copy per device that loads the library, kept until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {

struct DeviceSetup {
    bool ready = false;
    unsigned char *scratch = nullptr;   // device address of g_noalloc_scratch
    int sms = 0;
};

std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

// Frame descriptor passed by value as raw words (its tensor-map members are
// 64-byte aligned, which kernel parameters do not guarantee).
struct FrameWords {
    uint32_t w[sizeof(FrameDev) / 4];
};
static_assert(sizeof(FrameDev) % 4 == 0, "FrameDev is a whole number of words");

struct Prefix {
    int32_t zb, pt[kMaxScans], pool, t1, t2, bp;
};

__global__ void noalloc_init_kernel(BatchDev *b, FrameWords f, Prefix p, int32_t *status) {
    uint32_t *dst = reinterpret_cast<uint32_t *>(&b->f[0]);
    for (int i = threadIdx.x; i < (int)(sizeof(FrameDev) / 4); i += blockDim.x) dst[i] = f.w[i];
    if (threadIdx.x == 0) {
        b->n_frames = 1;
        b->status = status;
        *status = 0;
        b->zb_pre[0] = 0;
        b->zb_pre[1] = p.zb;
        b->pt_pre[0] = 0;
        for (int s = 0; s < kMaxScans; ++s) b->pt_pre[s + 1] = b->pt_pre[s] + p.pt[s];
        b->pool_pre[0] = 0;
        b->pool_pre[1] = p.pool;
        b->t1_pre[0] = 0;
        b->t1_pre[1] = p.t1;
        b->t2_pre[0] = 0;
        b->t2_pre[1] = p.t2;
        b->bp_pre[0] = 0;
        b->bp_pre[1] = p.bp;
        b->mk_pre[0] = b->mk_pre[1] = 0;
        b->tl_on = 0;   // plain filter kernels only: no tile flags
        b->tl_th[0] = b->tl_th[1] = 0;
        b->tl_tw[0] = b->tl_tw[1] = 32;
    }
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }
int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

densify_status fail(densify_status s, const std::string &m) {
    set_thread_error(m);
    return s;
}

}  // namespace

}  // namespace dz

using namespace dz;

extern "C" DENSIFY_API densify_status densify_frame_noalloc(const densify_params *params, const densify_frame *f,
                                                            void *cuda_stream) {
    if (!params || !f) return fail(DENSIFY_E_INVALID, "params and frame must not be NULL");
    const std::string perr = check_params(*params);
    if (!perr.empty()) return fail(DENSIFY_E_INVALID, perr);
    if (f->memory != DENSIFY_MEM_DEVICE) return fail(DENSIFY_E_INVALID, "the no-allocation entry takes device frames");
    if (params->occlusion_radius > 0 || params->motion_threshold > 0.0f || params->contour_threshold > 0.0f)
        return fail(DENSIFY_E_INVALID, "the no-allocation entry runs without occlusion, afterimage or contour removal");
    const int W = f->K.width, H = f->K.height;
    if (W < 1 || H < 1 || W > 16384 || H > 16384) return fail(DENSIFY_E_INVALID, "image size must be in 1..16384");
    if (f->num_scans < 0 || f->num_scans > kMaxScans) return fail(DENSIFY_E_INVALID, "num_scans must be in 0..3");
    for (int s = 0; s < f->num_scans; ++s) {
        const densify_scan &S = f->scans[s];
        if (S.count < 0 || S.count > (int64_t)1 << 30) return fail(DENSIFY_E_INVALID, "scan count out of range");
        if (S.stride_bytes != 12 && S.stride_bytes != 16) return fail(DENSIFY_E_INVALID, "stride_bytes must be 12 or 16");
        if (S.count > 0 && (!S.xyz || ((uintptr_t)S.xyz & 15u)))
            return fail(DENSIFY_E_INVALID, "scan xyz must be a 16-byte aligned device pointer");
    }
    if (!f->rgb || f->rgb_pitch < 3 * (int64_t)W) return fail(DENSIFY_E_INVALID, "rgb missing or pitch < 3 * width");
    if (!f->out_depth || !f->out_valid)
        return fail(DENSIFY_E_INVALID, "the no-allocation entry needs out_depth and out_valid");
    if (params->emit_points && (!f->out_points_n || (f->out_points_cap > 0 && !f->out_points) ||
                                ((uintptr_t)f->out_points & 15u)))
        return fail(DENSIFY_E_INVALID, "points on: out_points_n needed, out_points 16-byte aligned");

    // scratch layout
    const int pool = params->num_stages == 2 ? params->pool : 1;
    const int Wc = (W + pool - 1) / pool, Hc = (H + pool - 1) / pool;
    const int zpitch = (W + 3) & ~3, cpitch = (Wc + 3) & ~3;
    const int64_t npx = (int64_t)W * H;
    const int n_bp = cdiv(npx, kBpChunk);
    size_t o = 0;
    const size_t off_batch = o;
    o += up256(offsetof(BatchDev, f) + sizeof(FrameDev));
    const size_t off_status = o;
    o += 256;
    const size_t off_zbuf = o;
    o += up256((size_t)zpitch * H * 4);
    size_t off_cg = 0, off_cs = 0, off_s1 = 0;
    if (params->num_stages == 2) {
        off_cg = o;
        o += up256((size_t)cpitch * Hc * 16);
        off_cs = o;
        o += up256((size_t)cpitch * Hc * 4);
        off_s1 = o;
        o += up256((size_t)cpitch * Hc * 8);
    }
    const size_t off_cnt = o;
    o += up256((size_t)n_bp * kBpWarps * 4);
    if (o > kNoallocScratchBytes)
        return fail(DENSIFY_E_INVALID, "frame needs " + std::to_string(o) + " bytes of scratch; the no-allocation "
                                       "entry holds " + std::to_string(kNoallocScratchBytes) +
                                       " (one 1920x1080 two-stage frame fits)");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(DENSIFY_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(DENSIFY_E_INVALID, "device index too large");
    DeviceSetup setup;
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        DeviceSetup &S = g_setup[dev];
        if (!S.ready) {
            void *p = nullptr;
            if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess)
                return fail(DENSIFY_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            if ((e = cudaDeviceGetAttribute(&S.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
                return fail(DENSIFY_E_CUDA, std::string("device attribute: ") + cudaGetErrorString(e));
            S.scratch = static_cast<unsigned char *>(p);
            S.ready = true;
        }
        setup = S;
    }
    unsigned char *base = setup.scratch;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // frame descriptor
    FrameDev d;
    std::memset(&d, 0, sizeof(d));
    d.W = W; d.H = H; d.Wc = Wc; d.Hc = Hc; d.cpitch = cpitch; d.zpitch = zpitch;
    d.fx = f->K.fx; d.fy = f->K.fy; d.cx = f->K.cx; d.cy = f->K.cy;
    std::memcpy(d.c2w, f->cam_to_world, sizeof(d.c2w));
    d.num_scans = f->num_scans;
    d.n_bp_chunks = n_bp;
    for (int k = 0; k < kMaxScans; ++k) {
        if (k < f->num_scans) {
            d.scans[k].xyz = f->scans[k].xyz;
            d.scans[k].count = f->scans[k].count;
            d.scans[k].stride_floats = f->scans[k].stride_bytes / 4;
            std::memcpy(d.scans[k].l2w, f->scans[k].lidar_to_world, sizeof(d.scans[k].l2w));
        } else {
            d.scans[k].stride_floats = 3;
        }
    }
    d.rgb = f->rgb;
    d.rgb_pitch = f->rgb_pitch;
    d.zbuf = reinterpret_cast<uint32_t *>(base + off_zbuf);
    d.zbuf_raw = d.zbuf;
    d.zclear = 1;   // the static scratch holds whatever the last call left: cleared every call
    d.newest_scan = -1;
    if (params->num_stages == 2) {
        d.cguide = reinterpret_cast<float4 *>(base + off_cg);
        d.cssum = reinterpret_cast<float *>(base + off_cs);
        d.s1 = reinterpret_cast<float2 *>(base + off_s1);
        d.out_coarse = f->out_coarse;
        d.out_coarse_valid = f->out_coarse_valid;
    }
    d.chunk_cnt = reinterpret_cast<uint32_t *>(base + off_cnt);
    d.out_depth = f->out_depth;
    d.out_valid = f->out_valid;
    d.flt_depth = f->out_depth;
    d.flt_valid = f->out_valid;
    if (params->emit_points) {
        d.out_points = reinterpret_cast<float4 *>(f->out_points);
        d.points_cap = f->out_points_cap;
        d.points_n = f->out_points_n;
    }
    FrameWords fw;
    std::memcpy(fw.w, &d, sizeof(d));
    Prefix pre{};
    pre.zb = cdiv((int64_t)zpitch * H, kZbWordsPerChunk);
    for (int k = 0; k < kMaxScans; ++k) pre.pt[k] = cdiv(d.scans[k].count, kPtsPerChunk);
    const int r1 = params->stage[0].radius, r2 = params->num_stages == 2 ? params->stage[1].radius : 0;
    if (params->num_stages == 2) {
        pre.pool = cdiv(Wc, kPoolPerChunk) * Hc;
        pre.t1 = cdiv(Wc, 32) * cdiv(Hc, 8 * kp_jbf_coarse(r1));
        pre.t2 = cdiv(W, 32) * cdiv(H, 8 * kp_jbf_up(r2));
    } else {
        pre.t1 = cdiv(W, 32) * cdiv(H, 8 * kp_jbf_single(r1));
    }
    pre.bp = params->emit_points ? n_bp : 0;

    StageArgs sa[2];
    if (params->num_stages == 1) {
        fill_stage_args(sa[0], params->stage[0], 1, 0);
    } else {
        fill_stage_args(sa[0], params->stage[0], params->pool, 0);
        fill_stage_args(sa[1], params->stage[1], params->pool, params->stage2_input);
    }

    BatchDev *b = reinterpret_cast<BatchDev *>(base + off_batch);
    int32_t *status = reinterpret_cast<int32_t *>(base + off_status);
    const int sms = setup.sms;
    noalloc_init_kernel<<<1, 128, 0, s>>>(b, fw, pre, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(DENSIFY_E_CUDA, cudaGetErrorString(e));
#define NA_TRY(x)                                                             \
    do {                                                                      \
        if ((e = (x)) != cudaSuccess) return fail(DENSIFY_E_CUDA, cudaGetErrorString(e)); \
    } while (0)
    NA_TRY(launch_prep(b, sms * occupancy_points(K_PREP), s));
    NA_TRY(launch_project(b, sms * occupancy_points(K_PROJECT), s));
    if (params->num_stages == 2) {
        NA_TRY(launch_pool(b, params->pool, sms * occupancy_pool_bp(K_POOL), s));
        NA_TRY(launch_jbf_coarse(r1, b, sa[0], sms * occupancy_jbf_coarse(r1), s));
        NA_TRY(launch_jbf_up(r2, b, sa[1], sms * occupancy_jbf_up(r2), s));
    } else {
        NA_TRY(launch_jbf_single(r1, b, sa[0], sms * occupancy_jbf_single(r1), s));
    }
    if (params->emit_points) {
        NA_TRY(launch_bp_count(b, sms * occupancy_pool_bp(K_BP_COUNT), s));
        NA_TRY(launch_bp_write(b, sms * occupancy_pool_bp(K_BP_WRITE), s));
    }
    if (f->out_zbuf)
        NA_TRY(cudaMemcpy2DAsync(f->out_zbuf, (size_t)W * 4, d.zbuf, (size_t)zpitch * 4, (size_t)W * 4, (size_t)H,
                                 cudaMemcpyDeviceToDevice, s));
#undef NA_TRY
    return DENSIFY_OK;
}
