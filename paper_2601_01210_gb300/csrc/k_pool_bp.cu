// Pooling to the coarse grid of the two-stage filter (Sec. 5) and
// back-projection of the dense depth to coloured points with a deterministic
// row-major compaction (Sec. 2: coloured point clouds in a common frame).
#include "desc.cuh"
#include "tma_common.cuh"

namespace dz {

// ---------------------------------------------------------------------------
// pool: coarse pixel (I, J) covers the full-resolution block
// [fI, fI+f) x [fJ, fJ+f) clipped to the image. It gets the sum and count of
// the observed depths (average pooling of D*B and B, with the common divisor
// dropped because it cancels in the filter's ratio) and the mean RGB of the
// block's in-image pixels as the coarse guide. Sums run in row-major order.
// ---------------------------------------------------------------------------
// A work item is one coarse row J and a segment of 256 coarse pixels; one
// thread per coarse pixel. For f = 3 the thread reads 18 words of its block:
// per row the 3 z-buffer words and the 3 aligned words covering the row's 9
// colour bytes (byte offset 9I, rounded down to a word), from the item's rows
// staged in shared memory by bulk copies (pool_kernel), or from global memory
// (all 18 loads issued first) for items at a ragged edge. The colour bytes are
// shifted into place, each channel's 3 bytes gathered by a byte permute and
// summed by dp4a: integer sums, exactly the FP32 sums of the bytes. Blocks at
// the image border, other factors and layouts use plain loads.
// A frame as the pooling kernel reads it. Every block copies the batch's frames into shared
// memory once, all at once, so that a work item starts its loads without first waiting on the
// frame descriptor (a store could alias the descriptor, so the compiler would otherwise reload
// its fields from global memory after every store).
struct PoolFrame {
    uint32_t *zbuf;
    const uint8_t *rgb;
    float4 *cguide;
    float *cssum;
    int32_t *tflags;
    int64_t rgb_pitch, zpitch, cpitch;
    int32_t W, H, Wc, Hc, segs;
    int32_t zrestore;
    int32_t bulk_ok;   // z-buffer and colour rows start on 16-byte boundaries (bulk-copy path)
};

__device__ __forceinline__ bool pool_words_ok(const PoolFrame &F) {
    return ((((uintptr_t)F.zbuf) | ((uintptr_t)F.rgb)) & 3u) == 0 && (F.rgb_pitch & 3) == 0;
}

// The guide is the colour sum times the reciprocal of the block's pixel count (within one rounding
// of the quotient; the filter's tolerance covers it).
__device__ __forceinline__ void pool_store(const PoolFrame &F, int I, int J, float rr, float gg, float bb, float cnt,
                                           float s, float inv_npx) {
    const int64_t o = (int64_t)J * F.cpitch + I;
    F.cguide[o] = make_float4(rr * inv_npx, gg * inv_npx, bb * inv_npx, cnt);
    F.cssum[o] = s;
}

// Pooled pixel (I, J): its guide and sums; cnt_out = its observation count.
__device__ __forceinline__ void pool_one(const PoolFrame &F, int I, int J, int f, float &cnt_out) {
    const int x0 = I * f, y0 = J * f;
    const int o = (9 * I) & 3;                            // first colour byte inside its word
    const int64_t wb = 9 * (int64_t)I - o;                // byte offset of the first covering word
    if (f == 3 && x0 + 3 <= F.W && y0 + 3 <= F.H && wb + 12 <= 3 * (int64_t)F.W && pool_words_ok(F)) {
        uint32_t z[3][3], c[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const uint32_t *zr = F.zbuf + (int64_t)(y0 + r) * F.zpitch + x0;
            const uint32_t *cw = reinterpret_cast<const uint32_t *>(F.rgb + (int64_t)(y0 + r) * F.rgb_pitch + wb);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                z[r][j] = zr[j];
                c[r][j] = cw[j];
            }
        }
        float s = 0.0f, cnt = 0.0f;
        uint32_t rs = 0u, gs = 0u, bs = 0u;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (z[r][j] != kEmpty) {
                    s = __fadd_rn(s, __uint_as_float(z[r][j]));
                    cnt += 1.0f;
                    if (F.zrestore) F.zbuf[(int64_t)(y0 + r) * F.zpitch + x0 + j] = kEmpty;   // the clean pool's invariant
                }
            }
            // bytes c0 .. c8 of the row (r, g, b of 3 pixels) into a0 = c0..c3, a1 = c4..c7, a2 = c8..
            const uint32_t a0 = __funnelshift_r(c[r][0], c[r][1], 8 * o);
            const uint32_t a1 = __funnelshift_r(c[r][1], c[r][2], 8 * o);
            const uint32_t a2 = c[r][2] >> (8 * o);
            rs = __dp4a(__byte_perm(a0, a1, 0x0630), 0x00010101u, rs);   // c0 + c3 + c6
            gs = __dp4a(__byte_perm(a0, a1, 0x0741), 0x00010101u, gs);   // c1 + c4 + c7
            bs = __dp4a(__byte_perm(a0, a1, 0x0052), 0x00000101u, bs) + (a2 & 0xFFu);   // c2 + c5 + c8
        }
        pool_store(F, I, J, (float)rs, (float)gs, (float)bs, cnt, s, 1.0f / 9.0f);
        cnt_out = cnt;
    } else {
        const int x1 = min(x0 + f, F.W), y1 = min(y0 + f, F.H);
        float s = 0.0f, cnt = 0.0f, r = 0.0f, g = 0.0f, b = 0.0f;
        for (int y = y0; y < y1; ++y) {
            uint32_t *zr = F.zbuf + (int64_t)y * F.zpitch;
            const uint8_t *cr = F.rgb + (int64_t)y * F.rgb_pitch;
            for (int x = x0; x < x1; ++x) {
                const uint32_t zz = zr[x];
                if (zz != kEmpty) {
                    s = __fadd_rn(s, __uint_as_float(zz));
                    cnt += 1.0f;
                    if (F.zrestore) zr[x] = kEmpty;
                }
                r += (float)cr[3 * x];
                g += (float)cr[3 * x + 1];
                b += (float)cr[3 * x + 2];
            }
        }
        pool_store(F, I, J, r, g, b, cnt, s, 1.0f / (float)((x1 - x0) * (y1 - y0)));
        cnt_out = cnt;
    }
}

// Pooled pixel (I, J), f = 3, from a work item's rows staged in shared memory: zs holds the three
// rows' z-buffer words and cs their colour bytes (row strides kPoolSegPx words and 3 kPoolSegPx
// bytes), both starting at full-resolution column 3 (I - i); i is the pixel's index in the item.
// The same sums in the same order as pool_one.
constexpr int kPoolSegPx = 3 * kPoolPerChunk;                      // full-resolution columns of an item
constexpr int kPoolZBytes = 3 * kPoolSegPx * 4;                    // three rows of z-buffer words
constexpr int kPoolCBytes = 3 * kPoolSegPx * 3 + 16;               // three rows of colour bytes, read 2 past
constexpr int kPoolBuf = kPoolZBytes + kPoolCBytes;               // one buffer (a multiple of 16 bytes)
static_assert(kPoolZBytes % 16 == 0 && kPoolBuf % 16 == 0 && (3 * kPoolSegPx) % 16 == 0, "bulk copy alignment");

__device__ __forceinline__ void pool_staged(const PoolFrame &F, int I, int J, int i, const uint32_t *zs,
                                            const uint8_t *cs, float &cnt_out) {
    const int x0 = I * 3, y0 = J * 3;
    const int o = (9 * i) & 3;          // first colour byte inside its word (9 I and 9 i agree mod 4)
    const int wb = 9 * i - o;
    uint32_t z[3][3], c[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const uint32_t *cw = reinterpret_cast<const uint32_t *>(cs + r * 3 * kPoolSegPx + wb);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            z[r][j] = zs[r * kPoolSegPx + 3 * i + j];
            c[r][j] = cw[j];
        }
    }
    float s = 0.0f, cnt = 0.0f;
    uint32_t rs = 0u, gs = 0u, bs = 0u;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (z[r][j] != kEmpty) {
                s = __fadd_rn(s, __uint_as_float(z[r][j]));
                cnt += 1.0f;
                if (F.zrestore) F.zbuf[(int64_t)(y0 + r) * F.zpitch + x0 + j] = kEmpty;   // the clean pool's invariant
            }
        }
        const uint32_t a0 = __funnelshift_r(c[r][0], c[r][1], 8 * o);
        const uint32_t a1 = __funnelshift_r(c[r][1], c[r][2], 8 * o);
        const uint32_t a2 = c[r][2] >> (8 * o);
        rs = __dp4a(__byte_perm(a0, a1, 0x0630), 0x00010101u, rs);   // c0 + c3 + c6
        gs = __dp4a(__byte_perm(a0, a1, 0x0741), 0x00010101u, gs);   // c1 + c4 + c7
        bs = __dp4a(__byte_perm(a0, a1, 0x0052), 0x00000101u, bs) + (a2 & 0xFFu);   // c2 + c5 + c8
    }
    pool_store(F, I, J, (float)rs, (float)gs, (float)bs, cnt, s, 1.0f / 9.0f);
    cnt_out = cnt;
}

__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// With a TMA first-stage filter (tl_th[0] > 0) every warp also flags the first-stage tiles that
// its observed pooled pixels reach (one ballot; a row segment of 32 pooled pixels grown by the
// radius spans at most two tiles across and two down), so no mark kernel runs before that filter.
//
// For f = 3 a work item's three full-resolution rows reach shared memory by 1-D bulk copies
// (cp.async.bulk, one per row for the z-buffer words and one for the colour bytes), issued by
// thread 0 one item ahead into the other of two buffers: the next item's copies run while the
// block pools the current one from shared memory. An item is staged when its rows lie inside the
// image, its pooled pixels are whole 3 x 3 blocks, its row segments are a multiple of 16 columns
// and its frame's rows start on 16-byte boundaries; other items take the per-thread loads of
// pool_one. A wait that gives up (about 2 s) sets bit 0 of the batch status word; the block then
// waits (bounded) for its own copies in flight and leaves.
__global__ void __launch_bounds__(kThreads) pool_kernel(const BatchDev *__restrict__ B, int f) {
    __shared__ int32_t s_pre[kMaxBatch + 1];   // pooling chunk prefix, searched per work item
    __shared__ PoolFrame s_f[kMaxBatch];
    __shared__ int32_t s_geo[3];               // the first filter's tile width, height and radius
    __shared__ __align__(128) uint8_t s_buf[2][kPoolBuf];
    __shared__ __align__(8) uint64_t s_bar[2];
    const int nf = B->n_frames;
    for (int i = threadIdx.x; i <= nf; i += kThreads) s_pre[i] = B->pool_pre[i];
    for (int i = threadIdx.x; i < nf; i += kThreads) {
        const FrameDev &F = B->f[i];
        PoolFrame &P = s_f[i];
        P.zbuf = F.zbuf;
        P.rgb = F.rgb;
        P.cguide = F.cguide;
        P.cssum = F.cssum;
        P.tflags = F.tflags[0];
        P.rgb_pitch = F.rgb_pitch;
        P.zpitch = F.zpitch;
        P.cpitch = F.cpitch;
        P.W = F.W;
        P.H = F.H;
        P.Wc = F.Wc;
        P.Hc = F.Hc;
        P.segs = (F.Wc + kPoolPerChunk - 1) / kPoolPerChunk;
        P.zrestore = F.zrestore;
        P.bulk_ok = ((((uintptr_t)F.zbuf) | ((uintptr_t)F.rgb)) & 15u) == 0 && (F.zpitch & 3) == 0 &&
                    (F.rgb_pitch & 15) == 0;
    }
    if (threadIdx.x == 0) {
        s_geo[0] = B->tl_tw[0];
        s_geo[1] = B->tl_th[0];
        s_geo[2] = B->tl_r[0];
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const int total = s_pre[nf];
    const int lane = threadIdx.x & 31;
    const int mtw = s_geo[0], mth = s_geo[1], mr = s_geo[2];
    const bool marks = mth > 0;

    // item -> frame, coarse row J, first pooled pixel I0, pooled pixels m, and whether it is staged
    auto locate = [&](int item, int &fi, int &J, int &I0, int &m) -> bool {
        fi = find_segment(s_pre, nf, item);
        const PoolFrame &F = s_f[fi];
        const int t = item - s_pre[fi];
        J = t / F.segs;
        I0 = (t - J * F.segs) * kPoolPerChunk;
        m = min(kPoolPerChunk, F.Wc - I0);
        const int n = min(kPoolSegPx, F.W - 3 * I0);   // full-resolution columns of the segment
        return f == 3 && F.bulk_ok && 3 * J + 3 <= F.H && n == 3 * m && (n & 15) == 0;
    };
    // thread 0: the copies of a staged item into buffer b (rows y0 .. y0 + 2, columns 3 I0 .. + n)
    auto issue = [&](int fi, int J, int I0, int m, int b) {
        const PoolFrame &F = s_f[fi];
        const int n = 3 * m, x0 = 3 * I0;
        uint32_t *zs = reinterpret_cast<uint32_t *>(s_buf[b]);
        uint8_t *cs = s_buf[b] + kPoolZBytes;
        mbar_expect_tx(&s_bar[b], (uint32_t)(3 * 7 * n));
        for (int r = 0; r < 3; ++r) {
            const int64_t y = 3 * J + r;
            bulk_copy(zs + r * kPoolSegPx, F.zbuf + y * F.zpitch + x0, (uint32_t)(4 * n), &s_bar[b]);
            bulk_copy(cs + r * 3 * kPoolSegPx, F.rgb + y * F.rgb_pitch + 3 * (int64_t)x0, (uint32_t)(3 * n), &s_bar[b]);
        }
    };
    uint32_t phase = 0u, inflight = 0u;   // per buffer: wait parity; copies issued and not yet waited for
    int fi, J, I0, m;
    if (threadIdx.x == 0 && (int)blockIdx.x < total && locate(blockIdx.x, fi, J, I0, m)) {
        issue(fi, J, I0, m, 0);
        inflight |= 1u;
    }
    int b = 0;
    for (int item = blockIdx.x; item < total; item += gridDim.x, b ^= 1) {
        const int next = item + gridDim.x;
        if (threadIdx.x == 0 && next < total) {   // buffer b ^ 1 was freed by the previous item's barrier
            int nfi, nJ, nI0, nm;
            if (locate(next, nfi, nJ, nI0, nm)) {
                issue(nfi, nJ, nI0, nm, b ^ 1);
                inflight |= 1u << (b ^ 1);
            }
        }
        const bool staged = locate(item, fi, J, I0, m);
        const PoolFrame &F = s_f[fi];
        const int I = I0 + threadIdx.x;
        float cnt = 0.0f;
        bool ok = true;
        if (staged) {
            ok = mbar_wait_bounded(&s_bar[b], (phase >> b) & 1u);
            if (ok) {
                phase ^= 1u << b;
                inflight &= ~(1u << b);
                if ((int)threadIdx.x < m)
                    pool_staged(F, I, J, threadIdx.x, reinterpret_cast<const uint32_t *>(s_buf[b]),
                                s_buf[b] + kPoolZBytes, cnt);
            }
        } else if (I < F.Wc) {
            pool_one(F, I, J, f, cnt);
        }
        if (marks) {
            const uint32_t mk = __ballot_sync(0xffffffffu, cnt > 0.0f);
            const int Ib = I - lane;
            if (mk)
                mark_reach(F.tflags, mtw, mth, mr, 1, F.Wc, F.Hc, Ib + __ffs(mk) - 1, Ib + 31 - __clz(mk), J, J, lane);
        }
        if (__syncthreads_or(!ok)) {   // buffer b is free again once every thread is past this barrier
            if (threadIdx.x == 0) {
                atomicOr(B->status, 1);
                for (int bb = 0; bb < 2; ++bb)
                    if ((inflight >> bb) & 1u) mbar_wait_bounded(&s_bar[bb], (phase >> bb) & 1u);
            }
            return;
        }
    }
}


cudaError_t launch_pool(const BatchDev *b, int pool, int grid, cudaStream_t s) {
    pool_kernel<<<grid, kThreads, 0, s>>>(b, pool);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// back-projection with deterministic compaction.
// A chunk is 4096 consecutive pixels in row-major order, a part its 512-pixel
// eighth. bp_count writes each part's number of valid pixels and bp_scan turns
// them into each frame's exclusive prefix. In bp_write, warp w of the block
// owns part w of the chunk in 4 steps of 128 pixels (4 per lane): the warp's
// output offset is its part's prefix, so warps never wait for one another;
// inside a step an inclusive warp scan of the lanes' counts places every point. Points are built in shared memory and leave in
// coalesced 16-byte stores. Each point is
//   (x, y, z) = cam_to_world * ((u + 1/2 - cx) Z / fx, (v + 1/2 - cy) Z / fy, Z)
// with the pixel colour packed r | g << 8 | b << 16 | 255 << 24.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t valid_bits4(const uint8_t *v, int64_t p, int64_t n, bool vec) {
    if (vec && p + 4 <= n) {
        const uint32_t w = *reinterpret_cast<const uint32_t *>(v + p);   // bytes are 0 or 1
        return (w & 1u) | ((w >> 7) & 2u) | ((w >> 14) & 4u) | ((w >> 21) & 8u);
    }
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (p + k < n && v[p + k]) m |= 1u << k;
    return m;
}

// Valid pixels of 512-pixel parts: a warp takes kCountParts consecutive parts of a chunk, 16
// pixels of each per lane, with all its loads in flight before any is used.
constexpr int kCountParts = 4;
__global__ void __launch_bounds__(kThreads) bp_count_kernel(const BatchDev *__restrict__ B) {
    constexpr int kGroups = kBpWarps / kCountParts;   // part groups of a chunk
    // the chunk prefix and each frame's validity map, pixel count and part counts, read at once:
    // a work item then starts its loads without first waiting on the frame descriptor
    __shared__ int32_t s_pre[kMaxBatch + 1];
    __shared__ const uint8_t *s_valid[kMaxBatch];
    __shared__ uint32_t *s_cnt[kMaxBatch];
    __shared__ int64_t s_n[kMaxBatch];
    const int nf = B->n_frames;
    for (int i = threadIdx.x; i <= nf; i += kThreads) s_pre[i] = B->bp_pre[i];
    for (int i = threadIdx.x; i < nf; i += kThreads) {
        s_valid[i] = B->f[i].out_valid;
        s_cnt[i] = B->f[i].chunk_cnt;
        s_n[i] = (int64_t)B->f[i].W * B->f[i].H;
    }
    __syncthreads();
    const int total = s_pre[nf] * kGroups;
    const int lane = threadIdx.x & 31;
    for (int wi = blockIdx.x * kBpWarps + (threadIdx.x >> 5); wi < total; wi += gridDim.x * kBpWarps) {
        const int item = wi / kGroups;
        const int fi = find_segment(s_pre, nf, item);
        const uint8_t *const valid = s_valid[fi];
        const int sub0 = (item - s_pre[fi]) * kBpWarps + (wi % kGroups) * kCountParts;   // the frame's first part
        const int64_t n = s_n[fi];
        const bool vec = (((uintptr_t)valid) & 15u) == 0;
        uint4 w[kCountParts];
#pragma unroll
        for (int j = 0; j < kCountParts; ++j) {
            const int64_t p = (int64_t)(sub0 + j) * kBpPart + lane * 16;
            w[j] = make_uint4(0u, 0u, 0u, 0u);
            if (vec && p + 16 <= n) w[j] = *reinterpret_cast<const uint4 *>(valid + p);   // bytes are 0 or 1
        }
#pragma unroll
        for (int j = 0; j < kCountParts; ++j) {
            const int64_t p = (int64_t)(sub0 + j) * kBpPart + lane * 16;
            uint32_t cnt = __popc(w[j].x) + __popc(w[j].y) + __popc(w[j].z) + __popc(w[j].w);
            if (!(vec && p + 16 <= n)) {
                cnt = 0;
                for (int k = 0; k < 16; ++k) cnt += (p + k < n && valid[p + k]) ? 1u : 0u;
            }
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            if (lane == 0) s_cnt[fi][sub0 + j] = cnt;
        }
    }
}

// Exclusive prefix of the part counts of every frame, in place, and the
// frame's point count. One block of kScanBlock threads per frame: thread t
// takes the contiguous run of E = ceil(parts / kScanBlock) counts starting at
// t * E, sums it, the block scans the run sums (warp scans, then the warp
// totals) and each thread writes its run's exclusive prefixes.
constexpr int kScanBlock = 1024;
__global__ void __launch_bounds__(kScanBlock) bp_scan_kernel(const BatchDev *__restrict__ B) {
    __shared__ uint32_t wsum[kScanBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int fi = blockIdx.x; fi < B->n_frames; fi += gridDim.x) {
        const FrameDev &F = B->f[fi];
        // the frame's fields in registers before any store (a store through them could alias the
        // descriptor, which would make every later access reload them)
        uint32_t *const cnt = F.chunk_cnt;
        int64_t *const total = F.points_n;
        const int nparts = F.n_bp_chunks * kBpWarps;
        if (nparts == 0 || !total) continue;
        const int E = (nparts + kScanBlock - 1) / kScanBlock;
        const int c0 = threadIdx.x * E, c1 = min(nparts, c0 + E);
        uint32_t run = 0;
#pragma unroll 4
        for (int c = c0; c < c1; ++c) run += cnt[c];
        uint32_t incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t v = wsum[lane];
            uint32_t w = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += u;
            }
            wsum[lane] = w - v;                                  // exclusive over warps
            if (lane == 31 && threadIdx.x == 31) *total = (int64_t)w;   // the frame's total
        }
        __syncthreads();
        uint32_t before = wsum[warp] + incl - run;
#pragma unroll 4
        for (int c = c0; c < c1; ++c) {
            const uint32_t v = cnt[c];
            cnt[c] = before;
            before += v;
        }
        __syncthreads();                                         // wsum is reused by the next frame
    }
}

// (row, column) of pixel p of a row-major image of width W: a float estimate of
// p / W corrected by integer steps (exact for every p; one step at most while
// p < 2^24)
__device__ __forceinline__ void row_col(int64_t p, int W, float inv_w, int &y, int &x) {
    int64_t q = (int64_t)((float)p * inv_w);
    int64_t r = p - q * W;
    while (r < 0) { --q; r += W; }
    while (r >= W) { ++q; r -= W; }
    y = (int)q;
    x = (int)r;
}

// A frame as the compaction write reads it (copied into shared memory once per block, all frames
// at once, for the same reason as PoolFrame).
struct BpFrame {
    const uint8_t *valid;
    const float *depth;
    const uint8_t *rgb;
    const uint32_t *cnt;
    float4 *points;
    int64_t rgb_pitch, cap;
    float c2w[12];
    float ifx, ify, cx, cy, iw;
    int32_t W, H;
};

__global__ void __launch_bounds__(kThreads, 4) bp_write_kernel(const BatchDev *__restrict__ B) {
    __shared__ float4 stage[kThreads / 32][128];
    __shared__ int32_t s_pre[kMaxBatch + 1];          // chunk prefix, searched per work item
    __shared__ BpFrame s_f[kMaxBatch];
    const int nf = B->n_frames;
    for (int i = threadIdx.x; i <= nf; i += kThreads) s_pre[i] = B->bp_pre[i];
    for (int i = threadIdx.x; i < nf; i += kThreads) {
        const FrameDev &F = B->f[i];
        BpFrame &P = s_f[i];
        P.valid = F.out_valid;
        P.depth = F.out_depth;
        P.rgb = F.rgb;
        P.cnt = F.chunk_cnt;
        P.points = F.out_points;
        P.rgb_pitch = F.rgb_pitch;
        P.cap = F.points_cap;
#pragma unroll
        for (int e = 0; e < 12; ++e) P.c2w[e] = F.c2w32[e];
        P.ifx = 1.0f / F.fx;
        P.ify = 1.0f / F.fy;
        P.cx = F.cx;
        P.cy = F.cy;
        P.iw = 1.0f / (float)F.W;
        P.W = F.W;
        P.H = F.H;
    }
    __syncthreads();
    const int total = s_pre[nf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int fi = find_segment(s_pre, nf, item);
        const BpFrame &F = s_f[fi];
        const int c = item - s_pre[fi];
        const int W = F.W;
        const int64_t n = (int64_t)W * F.H;
        const bool vvalid = (((uintptr_t)F.valid) & 3u) == 0;
        const bool vdepth = (((uintptr_t)F.depth) & 15u) == 0;
        const bool rows4 = (W & 3) == 0 && (F.rgb_pitch & 3) == 0 && (((uintptr_t)F.rgb) & 3u) == 0;
        const int64_t wbase = (int64_t)c * kBpChunk + warp * 512;
        const float *c2w = F.c2w;
        const float r00 = c2w[0], r01 = c2w[1], r02 = c2w[2], t0 = c2w[3];
        const float r10 = c2w[4], r11 = c2w[5], r12 = c2w[6], t1 = c2w[7];
        const float r20 = c2w[8], r21 = c2w[9], r22 = c2w[10], t2 = c2w[11];
        const float ifx = F.ifx, ify = F.ify, iw = F.iw;
        float4 *st = stage[warp];
        // staged point j sits at j ^ ((j >> 2) & 7): a lane's four consecutive points and the read-back's
        // eight consecutive points of a quarter warp then fall on distinct 16-byte bank groups
        auto sw = [](uint32_t j) { return j ^ ((j >> 2) & 7u); };
        // all loads of the four steps (validity, depth, colour) are issued before any is used:
        // one memory round trip per chunk; depth and colour lines are mostly needed anyway
        uint32_t m[4];
        float4 zq[4];
        uint32_t cw[4][3];
        int ys[4], xs[4];   // row and column of each step's first pixel (128 pixels apart)
        row_col(wbase + lane * 4, W, iw, ys[0], xs[0]);
#pragma unroll
        for (int it = 1; it < 4; ++it) {
            ys[it] = ys[it - 1];
            xs[it] = xs[it - 1] + 128;
            while (xs[it] >= W) {
                xs[it] -= W;
                ++ys[it];
            }
        }
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            const int64_t p0 = wbase + it * 128 + lane * 4;
            m[it] = valid_bits4(F.valid, p0, n, vvalid);
            zq[it] = make_float4(0.f, 0.f, 0.f, 0.f);
            cw[it][0] = cw[it][1] = cw[it][2] = 0u;
            if (vdepth && rows4 && p0 + 4 <= n) {
                zq[it] = *reinterpret_cast<const float4 *>(F.depth + p0);
                const uint32_t *cp =
                    reinterpret_cast<const uint32_t *>(F.rgb + (int64_t)ys[it] * F.rgb_pitch + 3 * xs[it]);
                cw[it][0] = cp[0];
                cw[it][1] = cp[1];
                cw[it][2] = cp[2];
            }
        }
        int64_t off = F.cnt[c * kBpWarps + warp];   // exclusive prefix of the part counts (bp_scan_kernel)
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            const uint32_t cnt = __popc(m[it]);
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
            if (m[it]) {
                const int64_t p0 = wbase + it * 128 + lane * 4;
                uint32_t j = incl - cnt;
                if (vdepth && rows4 && p0 + 4 <= n) {
                    // the 4 pixels share a row; colour bytes were loaded as 3 words. The point is
                    // Z (R (u, v, 1)) + t with the ray (u, v) = ((x + 1/2 - cx) / fx, (y + 1/2 - cy) / fy),
                    // so each pixel takes 3 fma for R's ray column and 3 for the point.
                    const float z[4] = {zq[it].x, zq[it].y, zq[it].z, zq[it].w};
                    const uint32_t w0 = cw[it][0], w1 = cw[it][1], w2 = cw[it][2];
                    const uint32_t col[4] = {w0 & 0xFFFFFFu, (w0 >> 24) | ((w1 & 0xFFFFu) << 8),
                                             (w1 >> 16) | ((w2 & 0xFFu) << 16), w2 >> 8};
                    const float v = ((float)ys[it] + 0.5f - F.cy) * ify;
                    const float u0 = ((float)xs[it] + 0.5f - F.cx) * ifx;
                    const float b0 = fmaf(r01, v, r02), b1 = fmaf(r11, v, r12), b2 = fmaf(r21, v, r22);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (m[it] >> k & 1u) {
                            const float Z = z[k];
                            const float u = fmaf((float)k, ifx, u0);
                            st[sw(j++)] = make_float4(fmaf(fmaf(r00, u, b0), Z, t0), fmaf(fmaf(r10, u, b1), Z, t1),
                                                      fmaf(fmaf(r20, u, b2), Z, t2), __uint_as_float(col[k] | 0xFF000000u));
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (m[it] >> k & 1u) {
                            const int64_t p = p0 + k;
                            int y, x;
                            row_col(p, W, iw, y, x);
                            const uint8_t *cb = F.rgb + (int64_t)y * F.rgb_pitch + 3 * x;
                            const uint32_t rgba = (uint32_t)cb[0] | ((uint32_t)cb[1] << 8) | ((uint32_t)cb[2] << 16) |
                                                  0xFF000000u;
                            const float Z = F.depth[p];
                            const float X = ((float)x + 0.5f - F.cx) * Z * ifx;
                            const float Yz = ((float)y + 0.5f - F.cy) * ify * Z;
                            st[sw(j++)] = make_float4(fmaf(r00, X, fmaf(r01, Yz, fmaf(r02, Z, t0))),
                                                  fmaf(r10, X, fmaf(r11, Yz, fmaf(r12, Z, t1))),
                                                  fmaf(r20, X, fmaf(r21, Yz, fmaf(r22, Z, t2))),
                                                  __uint_as_float(rgba));
                        }
                    }
                }
            }
            __syncwarp();
            // the part's points from off on, as far as the caller's capacity goes
            const uint32_t fit = (uint32_t)max((int64_t)0, min((int64_t)tot, F.cap - off));
            float4 *dst = F.points + off;
            for (uint32_t i = lane; i < fit; i += 32) dst[i] = st[sw(i)];
            __syncwarp();
            off += tot;
        }
    }
}

cudaError_t launch_bp_count(const BatchDev *b, int grid, cudaStream_t s) {
    bp_count_kernel<<<grid, kThreads, 0, s>>>(b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bp_scan_kernel<<<kMaxBatch, kScanBlock, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_bp_write(const BatchDev *b, int grid, cudaStream_t s) {
    bp_write_kernel<<<grid, kThreads, 0, s>>>(b);
    return cudaGetLastError();
}

int occupancy_pool_bp(KernelId k) {
    int n = 0;
    if (k == K_POOL) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pool_kernel, kThreads, 0);
    else if (k == K_BP_COUNT) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bp_count_kernel, kThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bp_write_kernel, kThreads, 0);
    return n > 0 ? n : 1;
}

}  // namespace dz
