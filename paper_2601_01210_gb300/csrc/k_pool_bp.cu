// Pooling to the coarse grid of the two-stage filter (Sec. 5) and
// back-projection of the dense depth to coloured points with a deterministic
// row-major compaction (Sec. 2: coloured point clouds in a common frame).
#include "desc.cuh"

namespace dz {

// ---------------------------------------------------------------------------
// pool: coarse pixel (I, J) covers the full-resolution block
// [fI, fI+f) x [fJ, fJ+f) clipped to the image. It gets the sum and count of
// the observed depths (average pooling of D*B and B, with the common divisor
// dropped because it cancels in the filter's ratio) and the mean RGB of the
// block's in-image pixels as the coarse guide. Sums run in row-major order.
// ---------------------------------------------------------------------------
// Warp-cooperative form: one warp pools 32 consecutive coarse pixels of a
// coarse row. The 3 full-resolution rows under them are read with coalesced
// word loads into shared memory (z-buffer: 96 words a row; RGB: 288 bytes a
// row when the row start is word aligned), then each lane sums its block.
constexpr int kPoolWarps = kThreads / 32;
__global__ void __launch_bounds__(kThreads) pool_kernel(const BatchDev *__restrict__ B, int f) {
    __shared__ uint32_t sz[kPoolWarps][3][96];
    __shared__ uint32_t sc[kPoolWarps][3][72];
    const int nf = B->n_frames;
    const int total = B->pool_pre[nf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int fi = find_segment(B->pool_pre, nf, item);
        const FrameDev &F = B->f[fi];
        const int segs = (F.Wc + 255) / 256;                 // 256 coarse pixels per block item
        const int t = item - B->pool_pre[fi];
        const int J = t / segs;
        const int I0 = (t - J * segs) * 256 + warp * 32;     // this warp's first coarse pixel
        if (I0 >= F.Wc) continue;
        const int I = I0 + lane;
        const int y0 = J * f;
        if (f == 3) {
            const int x0 = 3 * I0;                            // first full-resolution column
            const bool words = ((F.rgb_pitch & 3) == 0) && ((((uintptr_t)F.rgb) & 3u) == 0);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int y = y0 + r;
                if (y >= F.H) break;
                const uint32_t *zr = F.zbuf + (int64_t)y * F.zpitch;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int x = x0 + lane + 32 * k;
                    sz[warp][r][lane + 32 * k] = x < F.W ? zr[x] : kEmpty;
                }
                const uint8_t *cr = F.rgb + (int64_t)y * F.rgb_pitch + 3 * x0;
                const int nbytes = 3 * min(96, F.W - x0);
                if (words) {
                    const uint32_t *cw = reinterpret_cast<const uint32_t *>(cr);
                    for (int k = lane; k < 72; k += 32) sc[warp][r][k] = 4 * k < nbytes ? cw[k] : 0u;
                } else {
                    uint8_t *sb = reinterpret_cast<uint8_t *>(sc[warp][r]);
                    for (int k = lane; k < 288; k += 32) sb[k] = k < nbytes ? cr[k] : 0;
                }
            }
            __syncwarp();
            if (I < F.Wc) {
                const int xa = 3 * I, xb = min(xa + 3, F.W), yb = min(y0 + 3, F.H);
                float s = 0.0f, cnt = 0.0f, rr = 0.0f, gg = 0.0f, bb = 0.0f;
                for (int y = y0; y < yb; ++y) {
                    const int r = y - y0;
                    const uint8_t *sb = reinterpret_cast<const uint8_t *>(sc[warp][r]);
                    for (int x = xa; x < xb; ++x) {
                        const uint32_t z = sz[warp][r][x - x0];
                        if (z != kEmpty) {
                            s = __fadd_rn(s, __uint_as_float(z));
                            cnt += 1.0f;
                        }
                        const int o = 3 * (x - x0);
                        rr += (float)sb[o];
                        gg += (float)sb[o + 1];
                        bb += (float)sb[o + 2];
                    }
                }
                const float npx = (float)((xb - xa) * (yb - y0));
                const int64_t o = (int64_t)J * F.cpitch + I;
                F.cguide[o] = make_float4(__fdiv_rn(rr, npx), __fdiv_rn(gg, npx), __fdiv_rn(bb, npx), cnt);
                F.cssum[o] = s;
            }
            __syncwarp();
        } else if (I < F.Wc) {   // other pooling factors: direct loads
            const int x0 = I * f;
            const int x1 = min(x0 + f, F.W), y1 = min(y0 + f, F.H);
            float s = 0.0f, cnt = 0.0f, r = 0.0f, g = 0.0f, b = 0.0f;
            for (int y = y0; y < y1; ++y) {
                const uint32_t *zr = F.zbuf + (int64_t)y * F.zpitch;
                const uint8_t *cr = F.rgb + (int64_t)y * F.rgb_pitch;
                for (int x = x0; x < x1; ++x) {
                    const uint32_t z = zr[x];
                    if (z != kEmpty) {
                        s = __fadd_rn(s, __uint_as_float(z));
                        cnt += 1.0f;
                    }
                    r += (float)cr[3 * x];
                    g += (float)cr[3 * x + 1];
                    b += (float)cr[3 * x + 2];
                }
            }
            const float npx = (float)((x1 - x0) * (y1 - y0));
            const int64_t o = (int64_t)J * F.cpitch + I;
            F.cguide[o] = make_float4(__fdiv_rn(r, npx), __fdiv_rn(g, npx), __fdiv_rn(b, npx), cnt);
            F.cssum[o] = s;
        }
    }
}

cudaError_t launch_pool(const BatchDev *b, int pool, int grid, cudaStream_t s) {
    pool_kernel<<<grid, kThreads, 0, s>>>(b, pool);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// back-projection with deterministic compaction.
// A chunk is 4096 consecutive pixels in row-major order. bp_count writes each
// chunk's number of valid pixels. In bp_write, warp w of the block owns pixels
// [512 w, 512 w + 512) of the chunk in 4 steps of 128 (4 per lane): the warp's
// output offset is the sum of the frame's earlier chunks plus the earlier
// warps of the chunk; inside a step an inclusive warp scan of the lanes'
// counts places every point. Points are built in shared memory and leave in
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

__global__ void __launch_bounds__(kThreads) bp_count_kernel(const BatchDev *__restrict__ B) {
    __shared__ uint32_t wsum[kThreads / 32];
    const int nf = B->n_frames;
    const int total = B->bp_pre[nf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int fi = find_segment(B->bp_pre, nf, item);
        const FrameDev &F = B->f[fi];
        const int c = item - B->bp_pre[fi];
        const int64_t n = (int64_t)F.W * F.H;
        const int64_t p = (int64_t)c * kBpChunk + threadIdx.x * 16;
        uint32_t cnt = 0;
        if ((((uintptr_t)F.out_valid) & 15u) == 0 && p + 16 <= n) {
            const uint4 w = *reinterpret_cast<const uint4 *>(F.out_valid + p);
            cnt = __popc(w.x) + __popc(w.y) + __popc(w.z) + __popc(w.w);
        } else {
            for (int k = 0; k < 16; ++k) cnt += (p + k < n && F.out_valid[p + k]) ? 1u : 0u;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        __syncthreads();
        if (lane == 0) wsum[warp] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < kThreads / 32; ++w) t += wsum[w];
            F.chunk_cnt[c] = t;
        }
    }
}

// Exclusive prefix of the chunk counts of every frame, in place, and the
// frame's point count. One block per frame.
__global__ void __launch_bounds__(kThreads) bp_scan_kernel(const BatchDev *__restrict__ B) {
    __shared__ uint32_t wsum[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int fi = blockIdx.x; fi < B->n_frames; fi += gridDim.x) {
        const FrameDev &F = B->f[fi];
        if (F.n_bp_chunks == 0 || !F.points_n) continue;
        uint32_t carry = 0;
        for (int c0 = 0; c0 < F.n_bp_chunks; c0 += kThreads) {
            const int c = c0 + threadIdx.x;
            const uint32_t v = c < F.n_bp_chunks ? F.chunk_cnt[c] : 0u;
            uint32_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            __syncthreads();
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();
            uint32_t before = carry, all = carry;
            for (int w = 0; w < kThreads / 32; ++w) {
                if (w < warp) before += wsum[w];
                all += wsum[w];
            }
            if (c < F.n_bp_chunks) F.chunk_cnt[c] = before + incl - v;
            carry = all;
        }
        if (threadIdx.x == 0) *F.points_n = (int64_t)carry;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) bp_write_kernel(const BatchDev *__restrict__ B) {
    __shared__ float4 stage[kThreads / 32][128];
    __shared__ uint32_t wtot[kThreads / 32];
    const int nf = B->n_frames;
    const int total = B->bp_pre[nf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int fi = find_segment(B->bp_pre, nf, item);
        const FrameDev &F = B->f[fi];
        const int c = item - B->bp_pre[fi];
        const int W = F.W;
        const int64_t n = (int64_t)W * F.H;
        const bool vvalid = (((uintptr_t)F.out_valid) & 3u) == 0;
        const bool vdepth = (((uintptr_t)F.out_depth) & 15u) == 0;
        const bool rows4 = (W & 3) == 0 && (F.rgb_pitch & 3) == 0 && (((uintptr_t)F.rgb) & 3u) == 0;
        const int64_t wbase = (int64_t)c * kBpChunk + warp * 512;
        uint32_t m[4], wc = 0;
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            m[it] = valid_bits4(F.out_valid, wbase + it * 128 + lane * 4, n, vvalid);
            wc += __popc(m[it]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wc += __shfl_xor_sync(0xffffffffu, wc, o);
        __syncthreads();   // the previous chunk is done with wtot
        if (lane == 0) wtot[warp] = wc;
        __syncthreads();
        int64_t off = F.chunk_cnt[c];   // exclusive prefix of the chunk counts (bp_scan_kernel)
        for (int w = 0; w < warp; ++w) off += wtot[w];

        const float *c2w = F.c2w32;
        const float r00 = c2w[0], r01 = c2w[1], r02 = c2w[2], t0 = c2w[3];
        const float r10 = c2w[4], r11 = c2w[5], r12 = c2w[6], t1 = c2w[7];
        const float r20 = c2w[8], r21 = c2w[9], r22 = c2w[10], t2 = c2w[11];
        const float ifx = 1.0f / F.fx, ify = 1.0f / F.fy;
        float4 *st = stage[warp];
        // issue the loads of all four steps before using any of them (memory-level parallelism)
        float4 zq[4];
        uint32_t cw[4][3];
        int yq[4], xq[4];
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            const int64_t p0 = wbase + it * 128 + lane * 4;
            zq[it] = make_float4(0.f, 0.f, 0.f, 0.f);
            cw[it][0] = cw[it][1] = cw[it][2] = 0u;
            yq[it] = 0;
            xq[it] = 0;
            if (m[it] && vdepth && rows4 && p0 + 4 <= n) {
                zq[it] = *reinterpret_cast<const float4 *>(F.out_depth + p0);
                yq[it] = (int)(p0 / W);
                xq[it] = (int)(p0 - (int64_t)yq[it] * W);
                const uint32_t *cp =
                    reinterpret_cast<const uint32_t *>(F.rgb + (int64_t)yq[it] * F.rgb_pitch + 3 * xq[it]);
                cw[it][0] = cp[0];
                cw[it][1] = cp[1];
                cw[it][2] = cp[2];
            }
        }
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
                    // the 4 pixels share a row; colour bytes were loaded as 3 words
                    const float z[4] = {zq[it].x, zq[it].y, zq[it].z, zq[it].w};
                    const uint32_t w0 = cw[it][0], w1 = cw[it][1], w2 = cw[it][2];
                    const uint32_t col[4] = {w0 & 0xFFFFFFu, (w0 >> 24) | ((w1 & 0xFFFFu) << 8),
                                             (w1 >> 16) | ((w2 & 0xFFu) << 16), w2 >> 8};
                    const int y = yq[it], x0 = xq[it];
                    const float Y = ((float)y + 0.5f - F.cy) * ify;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (m[it] >> k & 1u) {
                            const float Z = z[k];
                            const float X = ((float)(x0 + k) + 0.5f - F.cx) * Z * ifx;
                            const float Yz = Y * Z;
                            st[j++] = make_float4(fmaf(r00, X, fmaf(r01, Yz, fmaf(r02, Z, t0))),
                                                  fmaf(r10, X, fmaf(r11, Yz, fmaf(r12, Z, t1))),
                                                  fmaf(r20, X, fmaf(r21, Yz, fmaf(r22, Z, t2))),
                                                  __uint_as_float(col[k] | 0xFF000000u));
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (m[it] >> k & 1u) {
                            const int64_t p = p0 + k;
                            const int y = (int)(p / W), x = (int)(p - (int64_t)y * W);
                            const uint8_t *cb = F.rgb + (int64_t)y * F.rgb_pitch + 3 * x;
                            const uint32_t rgba = (uint32_t)cb[0] | ((uint32_t)cb[1] << 8) | ((uint32_t)cb[2] << 16) |
                                                  0xFF000000u;
                            const float Z = F.out_depth[p];
                            const float X = ((float)x + 0.5f - F.cx) * Z * ifx;
                            const float Yz = ((float)y + 0.5f - F.cy) * ify * Z;
                            st[j++] = make_float4(fmaf(r00, X, fmaf(r01, Yz, fmaf(r02, Z, t0))),
                                                  fmaf(r10, X, fmaf(r11, Yz, fmaf(r12, Z, t1))),
                                                  fmaf(r20, X, fmaf(r21, Yz, fmaf(r22, Z, t2))),
                                                  __uint_as_float(rgba));
                        }
                    }
                }
            }
            __syncwarp();
            for (uint32_t i = lane; i < tot; i += 32) {
                const int64_t pos = off + i;
                if (pos < F.points_cap) F.out_points[pos] = st[i];
            }
            __syncwarp();
            off += tot;
        }
    }
}

cudaError_t launch_bp_count(const BatchDev *b, int grid, cudaStream_t s) {
    bp_count_kernel<<<grid, kThreads, 0, s>>>(b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bp_scan_kernel<<<kMaxBatch, kThreads, 0, s>>>(b);
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
