// Preprocessing of the merged scans (Sec. 4.1) and post-filtering of the dense
// depth (Sec. 5), each off unless its parameter is set:
//
//   motion_kernel   afterimages: pixels whose RGB moved between consecutive
//                   frames (squared distance above tau^2, integers against
//                   the FP32 tau^2)
//   morph_kernel    closing of that mask: dilation, then erosion, with a
//                   square (2c+1)^2 element (outside the image: no motion for
//                   the dilation, motion for the erosion); the projection then
//                   drops points of older scans inside the mask
//   occlusion_kernel  occluded points: an observed pixel deeper than the mean
//                   observed depth of its (2 rho + 1)^2 window by more than a
//                   margin is removed. The sum is fixed to FP32 row sums over
//                   dx, added over dy, divided by the count (correctly rounded
//                   FP32 throughout), so the decision is bit-reproducible.
//   contour_kernel  contours: a valid pixel with a valid 4-neighbour whose
//                   depth differs by more than t times its own depth is dropped
//                   (FP32 on the filtered map).
//
// Every kernel copies the fields it needs of each frame into shared memory once
// per block, so that no work item waits on a read of the frame descriptor (a
// store through a pointer read from the descriptor could alias it, which would
// make the compiler read the descriptor again after every store). The motion mask
// and its closing work on bit-packed rows, a warp per 32 x 32 tile; the occlusion
// window on 32 x 32 tiles staged in shared memory, one pass along the rows and
// one along the columns; the contour test takes 4 consecutive pixels a thread.
#include "desc.cuh"

namespace dz {

namespace {

constexpr int kPxPerThread = kPxChunk / kThreads;   // 4 consecutive pixels
static_assert(kPxPerThread == 4, "per-pixel kernels: 4 consecutive pixels a thread");

// (row, column) of pixel p of a W-wide image (p < 2^28)
__device__ __forceinline__ void px_row_col(int p, int W, int &y, int &x) {
    y = p / W;
    x = p - y * W;
}

// The 3 colour bytes of pixel k (0..3) of 4 consecutive pixels whose 12 bytes are the words w0..w2,
// as the low three bytes r, g, b of one word (the top byte is not specified).
__device__ __forceinline__ uint32_t rgb_of(uint32_t w0, uint32_t w1, uint32_t w2, int k) {
    switch (k) {
        case 0: return __byte_perm(w0, 0u, 0x0210);
        case 1: return __byte_perm(w0, w1, 0x0543);
        case 2: return __byte_perm(w1, w2, 0x0432);
        default: return __byte_perm(w2, 0u, 0x0321);
    }
}

// Stage count elements into shared memory: each thread loads up to kStagePer of them (i = threadIdx.x,
// threadIdx.x + kThreads, ...) before storing any, so that its global loads are in flight together.
constexpr int kStagePer = 8;
template <typename T, typename Load, typename Store>
__device__ __forceinline__ void stage(int count, Load &&load, Store &&store) {
    for (int base = threadIdx.x; base < count; base += kStagePer * kThreads) {
        T v[kStagePer];
#pragma unroll
        for (int j = 0; j < kStagePer; ++j) {
            const int i = base + j * kThreads;
            if (i < count) v[j] = load(i);
        }
#pragma unroll
        for (int j = 0; j < kStagePer; ++j) {
            const int i = base + j * kThreads;
            if (i < count) store(i, v[j]);
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// The motion mask and its closing work on bit-packed rows: bit i of word j of row y is pixel
// (32 j + i, y), a row of Wp = ceil(W / 32) words, the bits past W zero. One warp takes a 32 x 32
// tile (the occlusion tiles): 32 rows of one word each.
constexpr int kMaxCloseR = 16;
constexpr int kPPWarps = kThreads / 32;
struct MotionFrame {
    const uint8_t *rgb, *prev;
    uint32_t *raw;     // the raw mask, bit-packed; NULL: afterimage removal is off for the frame
    uint32_t *dil;     // its dilation, bit-packed
    uint8_t *mask;     // the closing, one byte a pixel
    int64_t pitch, ppitch;
    int32_t W, H, Wp;
};

__device__ __forceinline__ void motion_frames(const BatchDev *B, int32_t *s_pre, MotionFrame *s_f) {
    const int nf = B->n_frames;
    for (int i = threadIdx.x; i <= nf; i += kThreads) s_pre[i] = B->oc_pre[i];
    for (int i = threadIdx.x; i < nf; i += kThreads) {
        const FrameDev &F = B->f[i];
        const int Wp = (F.W + 31) / 32;
        uint32_t *raw = reinterpret_cast<uint32_t *>(F.motion_tmp);
        s_f[i] = MotionFrame{F.rgb, F.prev_rgb, raw, raw ? raw + (int64_t)Wp * F.H : nullptr, F.motion,
                             F.rgb_pitch, F.prev_pitch, F.W, F.H, Wp};
    }
}

__global__ void __launch_bounds__(kThreads) motion_kernel(const BatchDev *__restrict__ B, const PrepostArgs a) {
    __shared__ int32_t s_pre[kMaxBatch + 1];
    __shared__ MotionFrame s_f[kMaxBatch];
    motion_frames(B, s_pre, s_f);
    __syncthreads();
    const int nf = B->n_frames;
    const int total = s_pre[nf];
    const int lane = threadIdx.x & 31;
    for (int item = blockIdx.x * kPPWarps + (threadIdx.x >> 5); item < total; item += gridDim.x * kPPWarps) {
        const int fi = find_segment(s_pre, nf, item);
        const MotionFrame &F = s_f[fi];
        if (!F.raw) continue;   // the same for every lane of the warp
        const int t = item - s_pre[fi];
        const int tx = t % F.Wp, y0 = (t / F.Wp) * 32;
        // lane = 4 consecutive columns (group g = lane & 7) of one of 4 rows (lane >> 3); 8 steps of 4
        // rows. A group inside the image on word-aligned rows reads 3 words of each frame; the 8
        // groups' nibbles of a row meet in one word by 3 shuffles.
        const int g = lane & 7, rr = lane >> 3;
        const int x = 32 * tx + 4 * g;
        const bool words = x + 4 <= F.W && ((((uintptr_t)F.rgb) | ((uintptr_t)F.prev) | F.pitch | F.ppitch) & 3) == 0;
#pragma unroll 4
        for (int step = 0; step < 8; ++step) {
            const int y = y0 + 4 * step + rr;
            uint32_t bits = 0u;   // bit k: pixel x + k moved
            if (y < F.H && x < F.W) {
                if (words) {   // 12 bytes at 3 x, a multiple of 4
                    const uint32_t *c = reinterpret_cast<const uint32_t *>(F.rgb + (int64_t)y * F.pitch + 3 * x);
                    const uint32_t *q = reinterpret_cast<const uint32_t *>(F.prev + (int64_t)y * F.ppitch + 3 * x);
                    const uint32_t c0 = c[0], c1 = c[1], c2 = c[2], q0 = q[0], q1 = q[1], q2 = q[2];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t d = __vabsdiffu4(rgb_of(c0, c1, c2, k), rgb_of(q0, q1, q2, k));
                        const uint32_t d2 = __dp4a(d, d & 0x00FFFFFFu, 0u);   // squared RGB distance, exact
                        if ((float)d2 > a.motion_t2) bits |= 1u << k;
                    }
                } else {
                    for (int k = 0; k < 4 && x + k < F.W; ++k) {
                        const uint8_t *c = F.rgb + (int64_t)y * F.pitch + 3 * (x + k);
                        const uint8_t *q = F.prev + (int64_t)y * F.ppitch + 3 * (x + k);
                        int d2 = 0;
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) {
                            const int d = (int)c[ch] - (int)q[ch];
                            d2 += d * d;
                        }
                        if ((float)d2 > a.motion_t2) bits |= 1u << k;
                    }
                }
            }
            uint32_t word = bits << (4 * g);
            word |= __shfl_xor_sync(0xffffffffu, word, 1);
            word |= __shfl_xor_sync(0xffffffffu, word, 2);
            word |= __shfl_xor_sync(0xffffffffu, word, 4);
            if (g == 0 && y < F.H) F.raw[(int64_t)y * F.Wp + tx] = word;
        }
    }
}

// Dilation (src: the raw mask, out: its packed dilation) or erosion (src: the dilation, out: the byte
// mask) with a square (2c+1)^2 element. Lane r of a warp takes row y0 + r of the tile's word column tx:
// the rows y0 - c .. y0 + 31 + c are first dilated (eroded) along the row, 2c funnel shifts a word with
// its neighbour words, then the lane combines the 2c + 1 rows of its window. Outside the image the
// dilation sees no motion and the erosion motion (the bits past W of the erosion's input are set).
__global__ void __launch_bounds__(kThreads) morph_kernel(const BatchDev *__restrict__ B, const PrepostArgs a,
                                                         int dilate) {
    __shared__ int32_t s_pre[kMaxBatch + 1];
    __shared__ MotionFrame s_f[kMaxBatch];
    __shared__ uint32_t s_h[kPPWarps][32 + 2 * kMaxCloseR];
    motion_frames(B, s_pre, s_f);
    __syncthreads();
    const int c = a.close_radius;
    const uint32_t fill = dilate ? 0u : ~0u;
    const int nf = B->n_frames;
    const int total = s_pre[nf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *const h = s_h[warp];
    for (int item = blockIdx.x * kPPWarps + warp; item < total; item += gridDim.x * kPPWarps) {
        const int fi = find_segment(s_pre, nf, item);
        const MotionFrame &F = s_f[fi];
        if (!F.raw) continue;   // the same for every lane of the warp
        const int t = item - s_pre[fi];
        const int tx = t % F.Wp, y0 = (t / F.Wp) * 32;
        const uint32_t *src = dilate ? F.raw : F.dil;
        // the erosion's input has the bits past W set (outside: motion)
        const int tailbits = F.W - 32 * (F.Wp - 1);
        const uint32_t tail = dilate || tailbits == 32 ? 0u : ~0u << tailbits;
        auto word = [&](int y, int j) -> uint32_t {
            if (y < 0 || y >= F.H || j < 0 || j >= F.Wp) return fill;
            const uint32_t v = src[(int64_t)y * F.Wp + j];
            return j == F.Wp - 1 ? (v | tail) : v;
        };
        for (int k = lane; k < 32 + 2 * c; k += 32) {   // rows y0 - c + k
            const int y = y0 - c + k;
            const uint32_t w = word(y, tx), l = word(y, tx - 1), r = word(y, tx + 1);
            uint32_t v = w;
            for (int s = 1; s <= c; ++s) {
                const uint32_t lo = __funnelshift_l(l, w, s), hi = __funnelshift_r(w, r, s);   // pixels x - s, x + s
                v = dilate ? (v | lo | hi) : (v & lo & hi);
            }
            h[k] = v;
        }
        __syncwarp();
        const int y = y0 + lane;
        uint32_t v = h[lane];
        for (int s = 1; s <= 2 * c; ++s) v = dilate ? (v | h[lane + s]) : (v & h[lane + s]);
        __syncwarp();   // h is rewritten by the warp's next tile
        if (y >= F.H) continue;
        if (dilate) {
            F.dil[(int64_t)y * F.Wp + tx] = v;
        } else {
            const int x0 = 32 * tx, n = min(32, F.W - x0);
            uint8_t *row = F.mask + (int64_t)y * F.W + x0;
            if ((((uintptr_t)row) & 3) == 0) {
                int i = 0;
                for (; i + 4 <= n; i += 4) {
                    const uint32_t nib = (v >> i) & 0xFu;
                    *reinterpret_cast<uint32_t *>(row + i) =
                        (nib & 1u) | ((nib & 2u) << 7) | ((nib & 4u) << 14) | ((nib & 8u) << 21);
                }
                for (; i < n; ++i) row[i] = (v >> i) & 1u;
            } else {
                for (int i = 0; i < n; ++i) row[i] = (v >> i) & 1u;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Tiles of 32 x 32 output pixels; the tile plus a rho halo is staged as depth
// (0 where empty) and an observation flag, then row sums and column sums.
constexpr int kMaxOccR = 16;
struct OccFrame {
    const uint32_t *src;   // merged z-buffer
    uint32_t *dst;         // kept z-buffer
    int64_t zpitch;
    int32_t W, H, tiles_x;
};

// RHO > 0: the window radius fixed at compile time (the sliding sums unrolled); 0: a.occ_radius.
template <int RHO>
__global__ void __launch_bounds__(kThreads) occlusion_kernel(const BatchDev *__restrict__ B, const PrepostArgs a) {
    constexpr int T = kOccTile, RMAX = RHO > 0 ? RHO : kMaxOccR;
    constexpr int S = T + 2 * RMAX;                  // staged rows
    constexpr int SW = T + 2 * ((RMAX + 3) / 4 * 4);   // staged row stride (columns from x0 - lead)
    __shared__ float sd[S * SW];
    __shared__ uint8_t sc[S * SW];
    __shared__ float hs[S * T];
    __shared__ int16_t hc[S * T];
    __shared__ int32_t s_pre[kMaxBatch + 1];
    __shared__ OccFrame s_f[kMaxBatch];
    const int rho = RHO > 0 ? RHO : a.occ_radius, sw = T + 2 * rho;
    const int lead = (rho + 3) & ~3, off = lead - rho, gpr = (T + 2 * lead) / 4;   // groups of 4 words a row
    const int nf = B->n_frames;
    for (int i = threadIdx.x; i <= nf; i += kThreads) s_pre[i] = B->oc_pre[i];
    for (int i = threadIdx.x; i < nf; i += kThreads) {
        const FrameDev &F = B->f[i];
        s_f[i] = OccFrame{F.zbuf_raw, F.zbuf, F.zpitch, F.W, F.H, (F.W + T - 1) / T};
    }
    __syncthreads();
    const int total = s_pre[nf];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int fi = find_segment(s_pre, nf, item);
        const OccFrame &F = s_f[fi];
        const int t = item - s_pre[fi];
        const int x0 = (t % F.tiles_x) * T, y0 = (t / F.tiles_x) * T;
        // rows y0 - rho .. y0 + 31 + rho, columns x0 - lead .. x0 + 31 + lead (lead = rho rounded up
        // to 4) in aligned groups of 4 words: one 16-byte load a group; a group lies either inside
        // the row's zpitch words (the cells past W hold the empty pattern) or outside it
        stage<uint4>(sw * gpr, [&](int i) -> uint4 {
            const int sy = i / gpr, gx = x0 - lead + 4 * (i - sy * gpr), gy = y0 - rho + sy;
            if (gy < 0 || gy >= F.H || gx < 0 || gx >= F.zpitch) return make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
            return *reinterpret_cast<const uint4 *>(F.src + (int64_t)gy * F.zpitch + gx);
        }, [&](int i, uint4 z) {
            const int sy = i / gpr, c = 4 * (i - sy * gpr);
            const uint32_t w[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                sd[sy * SW + c + k] = w[k] != kEmpty ? __uint_as_float(w[k]) : 0.0f;
                sc[sy * SW + c + k] = w[k] != kEmpty;
            }
        });
        __syncthreads();
        // row sums: a thread takes 4 consecutive columns of a staged row, its 4 window sums (over dx
        // in order) fed from a window of 4 staged values that slides along the row
        for (int i = threadIdx.x; i < sw * (T / 4); i += kThreads) {
            const int r = i / (T / 4), x = 4 * (i - r * (T / 4));
            const float *d = sd + r * SW + off + x;
            const uint8_t *cc = sc + r * SW + off + x;
            float v0 = d[0], v1 = d[1], v2 = d[2], v3 = d[3];
            int c0 = cc[0], c1 = cc[1], c2 = cc[2], c3 = cc[3];
            float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;   // adding 0 for an empty cell changes nothing
            int n0 = 0, n1 = 0, n2 = 0, n3 = 0;
#pragma unroll
            for (int dx = 0; dx <= 2 * rho; ++dx) {
                s0 = __fadd_rn(s0, v0); s1 = __fadd_rn(s1, v1); s2 = __fadd_rn(s2, v2); s3 = __fadd_rn(s3, v3);
                n0 += c0; n1 += c1; n2 += c2; n3 += c3;
                v0 = v1; v1 = v2; v2 = v3;
                c0 = c1; c1 = c2; c2 = c3;
                if (dx < 2 * rho) {
                    v3 = d[dx + 4];
                    c3 = cc[dx + 4];
                }
            }
            float *hrow = hs + r * T + x;
            int16_t *crow = hc + r * T + x;
            hrow[0] = s0; hrow[1] = s1; hrow[2] = s2; hrow[3] = s3;
            crow[0] = (int16_t)n0; crow[1] = (int16_t)n1; crow[2] = (int16_t)n2; crow[3] = (int16_t)n3;
        }
        __syncthreads();
        // column sums (over dy in order) of the row sums and the decision: a thread takes 4
        // consecutive rows of a column, likewise with a sliding window of 4 row sums
        for (int i = threadIdx.x; i < T * (T / 4); i += kThreads) {
            const int x = i % T, y = 4 * (i / T);
            const float *hcol = hs + y * T + x;
            const int16_t *ccol = hc + y * T + x;
            float v0 = hcol[0], v1 = hcol[T], v2 = hcol[2 * T], v3 = hcol[3 * T];
            int c0 = ccol[0], c1 = ccol[T], c2 = ccol[2 * T], c3 = ccol[3 * T];
            float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
            int n0 = 0, n1 = 0, n2 = 0, n3 = 0;
#pragma unroll
            for (int dy = 0; dy <= 2 * rho; ++dy) {
                s0 = __fadd_rn(s0, v0); s1 = __fadd_rn(s1, v1); s2 = __fadd_rn(s2, v2); s3 = __fadd_rn(s3, v3);
                n0 += c0; n1 += c1; n2 += c2; n3 += c3;
                v0 = v1; v1 = v2; v2 = v3;
                c0 = c1; c1 = c2; c2 = c3;
                if (dy < 2 * rho) {
                    v3 = hcol[(dy + 4) * T];
                    c3 = ccol[(dy + 4) * T];
                }
            }
            const float sum[4] = {s0, s1, s2, s3};
            const int cnt[4] = {n0, n1, n2, n3};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int gx = x0 + x, gy = y0 + y + k;
                if (gx >= F.W || gy >= F.H) continue;
                const int o = (y + k + rho) * SW + off + x + rho;   // the pixel's own staged cell
                uint32_t out = kEmpty;
                if (sc[o]) {
                    const float z = sd[o];
                    const float avg = __fdiv_rn(sum[k], (float)cnt[k]);
                    out = z > __fadd_rn(avg, a.occ_margin) ? kEmpty : __float_as_uint(z);
                }
                F.dst[(int64_t)gy * F.zpitch + gx] = out;
            }
        }
        __syncthreads();   // the staged tile and sums are rewritten by the next tile
    }
}

// ---------------------------------------------------------------------------
struct ContourFrame {
    const float *depth;
    const uint8_t *valid;
    float *out_depth;
    uint8_t *out_valid;
    int32_t W, H;
};

__global__ void __launch_bounds__(kThreads) contour_kernel(const BatchDev *__restrict__ B, const PrepostArgs a) {
    __shared__ int32_t s_pre[kMaxBatch + 1];
    __shared__ ContourFrame s_f[kMaxBatch];
    const int nf = B->n_frames;
    for (int i = threadIdx.x; i <= nf; i += kThreads) s_pre[i] = B->px_pre[i];
    for (int i = threadIdx.x; i < nf; i += kThreads) {
        const FrameDev &F = B->f[i];
        s_f[i] = ContourFrame{F.flt_depth, F.flt_valid, F.out_depth, F.out_valid, F.W, F.H};
    }
    __syncthreads();
    const int total = s_pre[nf];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int fi = find_segment(s_pre, nf, item);
        const ContourFrame &F = s_f[fi];
        const int n = F.W * F.H;
        const int p0 = (item - s_pre[fi]) * kPxChunk + threadIdx.x * kPxPerThread;
        if (p0 >= n) continue;
        int y, x;
        px_row_col(p0, F.W, y, x);
        // 4 pixels of one row, rows of a width divisible by 4 and aligned arrays: the 4 pixels and the
        // rows above and below by 16- and 4-byte loads, the left and right neighbours by single loads
        const bool vec = (F.W & 3) == 0 && x + 4 <= F.W &&
                         ((((uintptr_t)F.depth) | ((uintptr_t)F.out_depth)) & 15) == 0 &&
                         ((((uintptr_t)F.valid) | ((uintptr_t)F.out_valid)) & 3) == 0;
        if (vec) {
            const float4 dc = *reinterpret_cast<const float4 *>(F.depth + p0);
            const uint32_t vc = *reinterpret_cast<const uint32_t *>(F.valid + p0);
            float4 du = make_float4(0.f, 0.f, 0.f, 0.f), dd = du;
            uint32_t vu = 0u, vd = 0u;
            if (y > 0) {
                du = *reinterpret_cast<const float4 *>(F.depth + p0 - F.W);
                vu = *reinterpret_cast<const uint32_t *>(F.valid + p0 - F.W);
            }
            if (y + 1 < F.H) {
                dd = *reinterpret_cast<const float4 *>(F.depth + p0 + F.W);
                vd = *reinterpret_cast<const uint32_t *>(F.valid + p0 + F.W);
            }
            float dl = 0.0f, dr = 0.0f;
            uint8_t vl = 0, vr = 0;
            if (x > 0) {
                dl = F.depth[p0 - 1];
                vl = F.valid[p0 - 1];
            }
            if (x + 4 < F.W) {
                dr = F.depth[p0 + 4];
                vr = F.valid[p0 + 4];
            }
            const float d[6] = {dl, dc.x, dc.y, dc.z, dc.w, dr};   // the row, with the left and right neighbour
            const uint8_t v[6] = {vl, (uint8_t)(vc & 1u), (uint8_t)((vc >> 8) & 1u), (uint8_t)((vc >> 16) & 1u),
                                  (uint8_t)((vc >> 24) & 1u), vr};
            const float up[4] = {du.x, du.y, du.z, du.w}, dn[4] = {dd.x, dd.y, dd.z, dd.w};
            float od[4];
            uint32_t ov = 0u;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float c = d[k + 1];
                bool keep = v[k + 1] != 0;
                if (keep) {
                    const float lim = __fmul_rn(a.contour_t, c);
                    // left, right, above, below (the order of the per-pixel form; any step drops)
                    if (v[k] && fabsf(__fadd_rn(d[k], -c)) > lim) keep = false;
                    if (v[k + 2] && fabsf(__fadd_rn(d[k + 2], -c)) > lim) keep = false;
                    if (((vu >> (8 * k)) & 1u) && fabsf(__fadd_rn(up[k], -c)) > lim) keep = false;
                    if (((vd >> (8 * k)) & 1u) && fabsf(__fadd_rn(dn[k], -c)) > lim) keep = false;
                }
                const bool drop = v[k + 1] && !keep;
                od[k] = drop ? 0.0f : c;
                ov |= (uint32_t)(v[k + 1] && keep) << (8 * k);
            }
            *reinterpret_cast<float4 *>(F.out_depth + p0) = make_float4(od[0], od[1], od[2], od[3]);
            *reinterpret_cast<uint32_t *>(F.out_valid + p0) = ov;
            continue;
        }
        // every load of the 4 pixels and their neighbours first
        float d[kPxPerThread], nd[kPxPerThread][4];
        uint8_t v[kPxPerThread], nv[kPxPerThread][4];
        int yk = y, xk = x;
#pragma unroll
        for (int k = 0; k < kPxPerThread; ++k) {
            const int p = p0 + k;
            v[k] = 0;
            d[k] = 0.0f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                nv[k][j] = 0;
                nd[k][j] = 0.0f;
            }
            if (p < n) {
                v[k] = F.valid[p];
                d[k] = F.depth[p];
                const int qx[4] = {xk - 1, xk + 1, xk, xk}, qy[4] = {yk, yk, yk - 1, yk + 1};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (qx[j] >= 0 && qx[j] < F.W && qy[j] >= 0 && qy[j] < F.H) {
                        const int q = qy[j] * F.W + qx[j];
                        nv[k][j] = F.valid[q];
                        nd[k][j] = F.depth[q];
                    }
            }
            if (++xk == F.W) {
                xk = 0;
                ++yk;
            }
        }
#pragma unroll
        for (int k = 0; k < kPxPerThread; ++k) {
            const int p = p0 + k;
            if (p >= n) break;
            bool drop = false;
            if (v[k]) {
                const float lim = __fmul_rn(a.contour_t, d[k]);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (nv[k][j] && fabsf(__fadd_rn(nd[k][j], -d[k])) > lim) drop = true;
            }
            F.out_valid[p] = v[k] && !drop;
            F.out_depth[p] = drop ? 0.0f : d[k];
        }
    }
}

cudaError_t launch_motion(const BatchDev *b, const PrepostArgs &a, int grid, cudaStream_t s) {
    motion_kernel<<<grid, kThreads, 0, s>>>(b, a);
    return cudaGetLastError();
}

cudaError_t launch_morph(const BatchDev *b, const PrepostArgs &a, bool dilate, int grid, cudaStream_t s) {
    if (a.close_radius < 0 || a.close_radius > kMaxCloseR) return cudaErrorInvalidValue;
    morph_kernel<<<grid, kThreads, 0, s>>>(b, a, dilate ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_occlusion(const BatchDev *b, const PrepostArgs &a, int grid, cudaStream_t s) {
    if (a.occ_radius < 1 || a.occ_radius > kMaxOccR) return cudaErrorInvalidValue;
    switch (a.occ_radius) {
        case 1: occlusion_kernel<1><<<grid, kThreads, 0, s>>>(b, a); break;
        case 2: occlusion_kernel<2><<<grid, kThreads, 0, s>>>(b, a); break;
        case 3: occlusion_kernel<3><<<grid, kThreads, 0, s>>>(b, a); break;
        case 4: occlusion_kernel<4><<<grid, kThreads, 0, s>>>(b, a); break;
        case 5: occlusion_kernel<5><<<grid, kThreads, 0, s>>>(b, a); break;
        case 6: occlusion_kernel<6><<<grid, kThreads, 0, s>>>(b, a); break;
        case 7: occlusion_kernel<7><<<grid, kThreads, 0, s>>>(b, a); break;
        case 8: occlusion_kernel<8><<<grid, kThreads, 0, s>>>(b, a); break;
        default: occlusion_kernel<0><<<grid, kThreads, 0, s>>>(b, a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_contour(const BatchDev *b, const PrepostArgs &a, int grid, cudaStream_t s) {
    contour_kernel<<<grid, kThreads, 0, s>>>(b, a);
    return cudaGetLastError();
}

int occupancy_prepost(KernelId k) {
    int n = 0;
    if (k == K_MOTION) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, motion_kernel, kThreads, 0);
    else if (k == K_DILATE || k == K_ERODE) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, morph_kernel, kThreads, 0);
    else if (k == K_OCCLUSION) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, occlusion_kernel<0>, kThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, contour_kernel, kThreads, 0);
    return n > 0 ? n : 1;
}

}  // namespace dz
