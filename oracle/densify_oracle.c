/*
 * densify_oracle.c - plain, slow FP64 CPU oracle of the LiDAR densification
 * path (Murasaki et al., "Real-Time LiDAR Point Cloud Densification for
 * Low-Latency Spatial Data Transmission").
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code. The product path (the CUDA
 * library) never calls it, and it shares no code, header, table or constant
 * with the CUDA path.
 *
 * Every function is the definition written out as loops, in FP64, with no
 * blocking, fusion or reordering beyond what the definition states:
 *
 *   oracle_compose        calibration: world<-camera inverse times LiDAR pose
 *                         (Sec. 2, "calibrated in advance")
 *   oracle_project        merged scans -> nearest-depth z-buffer (Sec. 2;
 *                         the depth image D and mask B of Algorithm 1).
 *                         The pixel index and stored depth are decided in the
 *                         kernel's precision (FP32), emulated exactly here.
 *   oracle_project_fp64   the same projection in pure FP64 (compared with the
 *                         FP32 contract: how many pixels it assigns differently)
 *   oracle_pool           1/3 pooling of depth, mask and guide (Sec. 5,
 *                         two-stage filtering)
 *   oracle_jbf_gather     Eq. (1)-(4), gather form, plain or shifted exponent
 *   oracle_jbf_scatter    Algorithm 1 (colour weights, Gaussian, Hadamard
 *                         with the spatial Gaussian, transpose-convolution
 *                         scatter, normalisation)
 *   oracle_upsample       restore of the stage-1 result to full resolution
 *                         (Sec. 5, two-stage filtering)
 *   oracle_backproject    dense depth -> coloured 3D points (Sec. 2, Sec. 5)
 *
 * Parity pins: all functions above are pinned by the CPU tests (closed forms,
 * brute force, invariants). The exact pooling / restore semantics of the
 * two-stage filter are a documented reading of Sec. 5, which only says
 * "pooling" and "restoring".
 *
 * Build with -ffp-contract=off: the FP32 emulation relies on every product
 * and sum being rounded separately.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* FP32 emulation: an FP64 operation on two FP32 values, rounded once to FP32,
 * equals the correctly rounded FP32 operation (53 >= 2*24 + 2). */
static float r32(double x) { return (float)x; }
static float mul32(float a, float b) { return r32((double)a * (double)b); }
static float add32(float a, float b) { return r32((double)a + (double)b); }
static float div32(float a, float b) { return r32((double)a / (double)b); }

static uint32_t f32_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float bits_f32(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

#define ZBUF_EMPTY 0x7F800000u /* bit pattern of +inf */

/* ------------------------------------------------------------------------ */
/* Calibration (Sec. 2). M = inverse(cam_to_world) * lidar_to_world, with the
 * rigid inverse [R^T, -R^T t]. Inputs are row-major 4x4 rigid transforms;
 * the output is the top 3x4 block, row-major, in FP64 and rounded once to
 * FP32. The operation order is fixed: every dot product is summed left to
 * right over k = 0, 1, 2 and the translation is added last. */
void oracle_compose(const double cam_to_world[16], const double lidar_to_world[16],
                    double out64[12], float out32[12])
{
    double Rinv[3][3], tinv[3];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k)
            Rinv[i][k] = cam_to_world[k * 4 + i];          /* R^T */
    for (int i = 0; i < 3; ++i) {
        double s = Rinv[i][0] * cam_to_world[0 * 4 + 3];
        s = s + Rinv[i][1] * cam_to_world[1 * 4 + 3];
        s = s + Rinv[i][2] * cam_to_world[2 * 4 + 3];
        tinv[i] = -s;                                       /* -R^T t */
    }
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 4; ++j) {
            double s = Rinv[i][0] * lidar_to_world[0 * 4 + j];
            s = s + Rinv[i][1] * lidar_to_world[1 * 4 + j];
            s = s + Rinv[i][2] * lidar_to_world[2 * 4 + j];
            if (j == 3) s = s + tinv[i];
            out64[i * 4 + j] = s;
            out32[i * 4 + j] = (float)s;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Projection and nearest-depth z-buffer (Sec. 2: "merged and projected into
 * the camera view to form a single depth image"; Algorithm 1 input D, B).
 *
 * For each point p = (x, y, z) of a scan with FP32 matrix M (3x4):
 *   xc = ((m00 x + m01 y) + m02 z) + m03, likewise yc, zc   (FP32, each op rounded)
 *   u  = fx (xc / zc) + cx,  v = fy (yc / zc) + cy           (FP32, each op rounded)
 * The point is kept iff zc > 0, zc finite, 0 <= u < W and 0 <= v < H; it
 * lands on pixel (floor u, floor v). The z-buffer keeps the smallest camera
 * depth zc, stored as its FP32 bit pattern (order-preserving for positive
 * values); an empty pixel holds the bit pattern of +inf.
 *
 * zbuf must be cleared to ZBUF_EMPTY by the caller (scans are merged into
 * one buffer). Points are read with a stride of stride_floats floats.
 * Returns the number of points that landed inside the image. */
int64_t oracle_project(const float M[12], const float *xyz, int64_t n, int64_t stride_floats,
                       int W, int H, float fx, float fy, float cx, float cy, uint32_t *zbuf)
{
    int64_t kept = 0;
    for (int64_t k = 0; k < n; ++k) {
        const float x = xyz[k * stride_floats + 0];
        const float y = xyz[k * stride_floats + 1];
        const float z = xyz[k * stride_floats + 2];
        float c[3];
        for (int i = 0; i < 3; ++i) {
            float s = mul32(M[i * 4 + 0], x);
            s = add32(s, mul32(M[i * 4 + 1], y));
            s = add32(s, mul32(M[i * 4 + 2], z));
            s = add32(s, M[i * 4 + 3]);
            c[i] = s;
        }
        if (!(c[2] > 0.0f) || !(c[2] < INFINITY)) continue;
        const float u = add32(mul32(fx, div32(c[0], c[2])), cx);
        const float v = add32(mul32(fy, div32(c[1], c[2])), cy);
        if (!(u >= 0.0f && u < (float)W && v >= 0.0f && v < (float)H)) continue;
        const int i = (int)floor((double)u);
        const int j = (int)floor((double)v);
        const uint32_t b = f32_bits(c[2]);
        uint32_t *cell = &zbuf[(int64_t)j * W + i];
        if (b < *cell) *cell = b;
        ++kept;
    }
    return kept;
}

/* Pure FP64 projection of the same points (informational: it shows how many
 * pixels an FP64 pipeline would assign differently). depth must be cleared to
 * +inf by the caller; it keeps the nearest FP64 camera depth per pixel. */
int64_t oracle_project_fp64(const double M[12], const float *xyz, int64_t n, int64_t stride_floats,
                            int W, int H, double fx, double fy, double cx, double cy, double *depth)
{
    int64_t kept = 0;
    for (int64_t k = 0; k < n; ++k) {
        const double p[3] = {xyz[k * stride_floats], xyz[k * stride_floats + 1], xyz[k * stride_floats + 2]};
        double c[3];
        for (int i = 0; i < 3; ++i)
            c[i] = M[i * 4] * p[0] + M[i * 4 + 1] * p[1] + M[i * 4 + 2] * p[2] + M[i * 4 + 3];
        if (!(c[2] > 0.0) || !isfinite(c[2])) continue;
        const double u = fx * (c[0] / c[2]) + cx, v = fy * (c[1] / c[2]) + cy;
        if (!(u >= 0.0 && u < W && v >= 0.0 && v < H)) continue;
        double *cell = &depth[(int64_t)floor(v) * W + (int64_t)floor(u)];
        if (c[2] < *cell) *cell = c[2];
        ++kept;
    }
    return kept;
}

/* Depth image D and mask B from the z-buffer (Algorithm 1 input). */
void oracle_zbuf_to_depth(const uint32_t *zbuf, int64_t npix, double *D, double *B)
{
    for (int64_t k = 0; k < npix; ++k) {
        if (zbuf[k] != ZBUF_EMPTY) { D[k] = (double)bits_f32(zbuf[k]); B[k] = 1.0; }
        else { D[k] = 0.0; B[k] = 0.0; }
    }
}

/* ------------------------------------------------------------------------ */
/* Pooling to 1/f resolution (Sec. 5, first stage: "reduced to 1/3 ... using
 * pooling"). Coarse pixel (I, J) covers the full-resolution block
 * [fI, fI+f) x [fJ, fJ+f) clipped to the image (ceil mode). Reading: average
 * pooling of D*B and of B as in a CNN; the uniform divisor cancels in the
 * filter's ratio, so the outputs are the block sums
 *   ssum(I,J) = sum of D over observed pixels,  cnt(I,J) = number observed,
 * and the coarse guide is the mean RGB over the block's in-image pixels.
 * guide is Hc x Wc x 3 (channel fastest); Hc = ceil(H/f), Wc = ceil(W/f). */
void oracle_pool(const uint32_t *zbuf, const uint8_t *rgb, int64_t rgb_pitch, int W, int H, int f,
                 double *ssum, double *cnt, double *guide)
{
    const int Wc = (W + f - 1) / f, Hc = (H + f - 1) / f;
    for (int J = 0; J < Hc; ++J) {
        for (int I = 0; I < Wc; ++I) {
            double s = 0.0, c = 0.0, g[3] = {0.0, 0.0, 0.0}, npx = 0.0;
            for (int y = J * f; y < J * f + f && y < H; ++y) {
                for (int x = I * f; x < I * f + f && x < W; ++x) {
                    const uint32_t z = zbuf[(int64_t)y * W + x];
                    if (z != ZBUF_EMPTY) { s += (double)bits_f32(z); c += 1.0; }
                    for (int ch = 0; ch < 3; ++ch) g[ch] += rgb[(int64_t)y * rgb_pitch + 3 * x + ch];
                    npx += 1.0;
                }
            }
            const int64_t o = (int64_t)J * Wc + I;
            ssum[o] = s;
            cnt[o] = c;
            for (int ch = 0; ch < 3; ++ch) guide[o * 3 + ch] = g[ch] / npx;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Joint bilateral filter, Eq. (1)-(4), gather form.
 *
 * For output pixel p and every in-image pixel q with max(|qx-px|,|qy-py|) <= r:
 *   e(p,q) = ||I(q) - I(p)||^2 / (2 sigma_c^2) + ((qx-px)^2 + (qy-py)^2) / (2 sigma_p^2)
 *   out(p) = sum_q beta_d(q) exp(-e) / sum_q beta(q) exp(-e)
 * beta(q) is the observation weight (the mask B at a single stage, the block
 * count after pooling) and beta_d(q) the matching depth sum (B*D, or the
 * block depth sum). Only q with beta(q) > 0 are in the neighbour set eps(x)
 * of Eq. (1). valid(p) = 1 iff that set is non-empty; an invalid output is 0.
 *
 * guide is H x W x 3 (channel fastest), on the 0-255 scale.
 * shifted = 0: the plain form. shifted = 1: exp(-(e - e_min)) with e_min the
 * smallest e over the neighbour set; the common factor exp(-e_min) cancels,
 * so both forms are the same number up to rounding. */
void oracle_jbf_gather(const double *guide, const double *beta, const double *beta_d,
                       int W, int H, int r, double sigma_p, double sigma_c, int shifted,
                       double *out, uint8_t *valid)
{
    const double kc = 1.0 / (2.0 * sigma_c * sigma_c);
    const double kp = 1.0 / (2.0 * sigma_p * sigma_p);
    for (int py = 0; py < H; ++py) {
        for (int px = 0; px < W; ++px) {
            const double *Ip = &guide[((int64_t)py * W + px) * 3];
            double emin = INFINITY;
            int any = 0;
            if (shifted) {
                for (int qy = py - r; qy <= py + r; ++qy) {
                    for (int qx = px - r; qx <= px + r; ++qx) {
                        if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
                        const int64_t q = (int64_t)qy * W + qx;
                        if (!(beta[q] > 0.0)) continue;
                        const double *Iq = &guide[q * 3];
                        const double dc = (Iq[0] - Ip[0]) * (Iq[0] - Ip[0]) + (Iq[1] - Ip[1]) * (Iq[1] - Ip[1]) +
                                          (Iq[2] - Ip[2]) * (Iq[2] - Ip[2]);
                        const double ds = (double)(qx - px) * (qx - px) + (double)(qy - py) * (qy - py);
                        const double e = dc * kc + ds * kp;
                        if (e < emin) emin = e;
                    }
                }
            } else {
                emin = 0.0;
            }
            double num = 0.0, den = 0.0;
            for (int qy = py - r; qy <= py + r; ++qy) {
                for (int qx = px - r; qx <= px + r; ++qx) {
                    if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
                    const int64_t q = (int64_t)qy * W + qx;
                    if (!(beta[q] > 0.0)) continue;
                    const double *Iq = &guide[q * 3];
                    const double dc = (Iq[0] - Ip[0]) * (Iq[0] - Ip[0]) + (Iq[1] - Ip[1]) * (Iq[1] - Ip[1]) +
                                      (Iq[2] - Ip[2]) * (Iq[2] - Ip[2]);
                    const double ds = (double)(qx - px) * (qx - px) + (double)(qy - py) * (qy - py);
                    const double w = exp(-(dc * kc + ds * kp - emin));  /* w_c * w_p, Eq. (2), (3) */
                    num += beta_d[q] * w;                                  /* Eq. (1) numerator */
                    den += beta[q] * w;                                    /* Eq. (4) */
                    any = 1;
                }
            }
            const int64_t o = (int64_t)py * W + px;
            valid[o] = (uint8_t)any;
            out[o] = any ? num / den : 0.0;
        }
    }
}

/* Joint bilateral filter as Algorithm 1 (scatter form).
 * Step 1-3: for every source pixel (x, y) and offset (a, b) in [-r, r]^2, the
 *   weight w = exp(-||I(x,y) - I(x+a,y+b)||^2 / (2 sigma_c^2))
 *            * exp(-(a^2 + b^2) / (2 sigma_p^2)).
 * Step 4: spread beta_d(x,y) w into num(x+a, y+b) and beta(x,y) w into
 *   den(x+a, y+b) (transpose convolution; targets outside the image drop).
 * Step 5: out = num / den where den > 0; valid = (den > 0).
 * num and den are caller-provided scratch arrays of H x W doubles. */
void oracle_jbf_scatter(const double *guide, const double *beta, const double *beta_d,
                        int W, int H, int r, double sigma_p, double sigma_c,
                        double *num, double *den, double *out, uint8_t *valid)
{
    const int64_t npix = (int64_t)W * H;
    for (int64_t k = 0; k < npix; ++k) { num[k] = 0.0; den[k] = 0.0; }
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            const int64_t s = (int64_t)y * W + x;
            if (!(beta[s] > 0.0)) continue;      /* D = B = 0 adds nothing */
            const double *Is = &guide[s * 3];
            for (int a = -r; a <= r; ++a) {          /* a along x, b along y */
                for (int b = -r; b <= r; ++b) {
                    const int tx = x + a, ty = y + b;
                    if (tx < 0 || tx >= W || ty < 0 || ty >= H) continue;
                    const int64_t t = (int64_t)ty * W + tx;
                    const double *It = &guide[t * 3];
                    double d2 = 0.0;
                    for (int ch = 0; ch < 3; ++ch) d2 += (Is[ch] - It[ch]) * (Is[ch] - It[ch]);
                    double w = exp(-d2 / (2.0 * sigma_c * sigma_c));                    /* step 2 */
                    w = w * exp(-((double)a * a + (double)b * b) / (2.0 * sigma_p * sigma_p)); /* step 3 */
                    num[t] += beta_d[s] * w;                                           /* step 4 */
                    den[t] += beta[s] * w;
                }
            }
        }
    }
    for (int64_t k = 0; k < npix; ++k) {                                               /* step 5 */
        valid[k] = den[k] > 0.0;
        out[k] = den[k] > 0.0 ? num[k] / den[k] : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* Restore to full resolution (Sec. 5, second stage: "the depth map after
 * restoring it to the original resolution"). Nearest restore: full pixel
 * (x, y) takes coarse pixel (x / f, y / f). Literal reading (override = 0):
 * the stage-2 input is the restored stage-1 result, beta = restored valid,
 * beta_d = restored depth. With override = 1, pixels observed in the full
 * z-buffer keep their own depth instead (an alternative reading). */
void oracle_upsample(const double *d1, const uint8_t *v1, int Wc, int Hc, int f, int W, int H,
                     const uint32_t *zbuf, int override, double *beta, double *beta_d)
{
    (void)Hc;
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            const int64_t o = (int64_t)y * W + x;
            const int64_t c = (int64_t)(y / f) * Wc + (x / f);
            if (override && zbuf && zbuf[o] != ZBUF_EMPTY) {
                beta[o] = 1.0;
                beta_d[o] = (double)bits_f32(zbuf[o]);
            } else {
                beta[o] = v1[c] ? 1.0 : 0.0;
                beta_d[o] = v1[c] ? d1[c] : 0.0;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Back-projection to coloured points (Sec. 2: coloured point clouds in a
 * common frame). For every valid pixel (x, y) in row-major order:
 *   Z = depth, X = (x + 1/2 - cx) Z / fx, Y = (y + 1/2 - cy) Z / fy,
 *   world = R (X, Y, Z) + t from cam_to_world, colour = RGB(x, y).
 * out_xyz receives n x 3 doubles, out_rgba n packed colours
 * (r | g << 8 | b << 16 | 255 << 24). Returns n. */
int64_t oracle_backproject(const double *depth, const uint8_t *valid, const uint8_t *rgb, int64_t rgb_pitch,
                           int W, int H, double fx, double fy, double cx, double cy,
                           const double cam_to_world[16], double *out_xyz, uint32_t *out_rgba)
{
    int64_t n = 0;
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            const int64_t o = (int64_t)y * W + x;
            if (!valid[o]) continue;
            const double Z = depth[o];
            const double X = ((double)x + 0.5 - cx) * Z / fx;
            const double Y = ((double)y + 0.5 - cy) * Z / fy;
            for (int i = 0; i < 3; ++i)
                out_xyz[n * 3 + i] = cam_to_world[i * 4 + 0] * X + cam_to_world[i * 4 + 1] * Y +
                                     cam_to_world[i * 4 + 2] * Z + cam_to_world[i * 4 + 3];
            const uint8_t *c = &rgb[(int64_t)y * rgb_pitch + 3 * x];
            out_rgba[n] = (uint32_t)c[0] | ((uint32_t)c[1] << 8) | ((uint32_t)c[2] << 16) | (255u << 24);
            ++n;
        }
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Occluded-point removal (Sec. 4.1: an averaging filter on the merged depth
 * map; points significantly behind the average are removed). Reading: for an
 * observed pixel p, the window average is the mean of the observed depths in
 * the (2 rho + 1)^2 square around p (p included), summed in FP32 as row sums
 * (dx ascending) added up over rows (dy ascending), divided by their count in
 * FP32; p is removed iff D(p) > average + margin (FP32). The sums are
 * evaluated in FP64 and rounded to FP32 after every operation, which is the
 * FP32 result exactly. zin and zout are H x W bit patterns (empty 0x7F800000);
 * returns the number of removed points. */
int64_t oracle_occlusion(const uint32_t *zin, int W, int H, int rho, float margin, uint32_t *zout)
{
    int64_t removed = 0;
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            const int64_t o = (int64_t)y * W + x;
            zout[o] = zin[o];
            if (zin[o] == ZBUF_EMPTY) continue;
            float sum = 0.0f;
            int cnt = 0;
            for (int dy = -rho; dy <= rho; ++dy) {
                float row = 0.0f;
                for (int dx = -rho; dx <= rho; ++dx) {
                    const int qx = x + dx, qy = y + dy;
                    if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
                    const uint32_t z = zin[(int64_t)qy * W + qx];
                    if (z == ZBUF_EMPTY) continue;
                    row = add32(row, bits_f32(z));
                    ++cnt;
                }
                sum = add32(sum, row);
            }
            const float avg = div32(sum, (float)cnt);
            if (bits_f32(zin[o]) > add32(avg, margin)) {
                zout[o] = ZBUF_EMPTY;
                ++removed;
            }
        }
    }
    return removed;
}

/* Afterimage removal, motion mask (Sec. 4.1: Euclidean RGB distance between
 * consecutive frames above tau_m marks motion; a morphological closing fills
 * the mask). Motion at p iff (dr^2 + dg^2 + db^2) > tau^2 (integers against
 * the FP32 square of tau). Closing = dilation then erosion with the square
 * (2c + 1)^2 structuring element; outside the image counts as no motion for
 * the dilation and as motion for the erosion (so the closing never shrinks
 * the mask at the border). mask is H x W (1 = motion). */
void oracle_motion_mask(const uint8_t *rgb, int64_t pitch, const uint8_t *prev, int64_t prev_pitch, int W, int H,
                        float tau, int c, uint8_t *tmp, uint8_t *mask)
{
    const float t2 = mul32(tau, tau);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int d2 = 0;
            for (int ch = 0; ch < 3; ++ch) {
                const int d = (int)rgb[(int64_t)y * pitch + 3 * x + ch] - (int)prev[(int64_t)y * prev_pitch + 3 * x + ch];
                d2 += d * d;
            }
            mask[(int64_t)y * W + x] = (float)d2 > t2;
        }
    /* dilation */
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            uint8_t m = 0;
            for (int dy = -c; dy <= c; ++dy)
                for (int dx = -c; dx <= c; ++dx) {
                    const int qx = x + dx, qy = y + dy;
                    if (qx >= 0 && qx < W && qy >= 0 && qy < H && mask[(int64_t)qy * W + qx]) m = 1;
                }
            tmp[(int64_t)y * W + x] = m;
        }
    /* erosion */
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            uint8_t m = 1;
            for (int dy = -c; dy <= c; ++dy)
                for (int dx = -c; dx <= c; ++dx) {
                    const int qx = x + dx, qy = y + dy;
                    if (qx >= 0 && qx < W && qy >= 0 && qy < H && !tmp[(int64_t)qy * W + qx]) m = 0;
                }
            mask[(int64_t)y * W + x] = m;
        }
}

/* Projection with afterimage removal: as oracle_project, but a point of a scan
 * that is not the most recent one is dropped where the motion mask is set.
 * newest = 1 marks the most recent scan. */
int64_t oracle_project_masked(const float M[12], const float *xyz, int64_t n, int64_t stride_floats, int W, int H,
                              float fx, float fy, float cx, float cy, const uint8_t *mask, int newest, uint32_t *zbuf)
{
    int64_t kept = 0;
    for (int64_t k = 0; k < n; ++k) {
        const float x = xyz[k * stride_floats + 0];
        const float y = xyz[k * stride_floats + 1];
        const float z = xyz[k * stride_floats + 2];
        float c[3];
        for (int i = 0; i < 3; ++i) {
            float s = mul32(M[i * 4 + 0], x);
            s = add32(s, mul32(M[i * 4 + 1], y));
            s = add32(s, mul32(M[i * 4 + 2], z));
            s = add32(s, M[i * 4 + 3]);
            c[i] = s;
        }
        if (!(c[2] > 0.0f) || !(c[2] < INFINITY)) continue;
        const float u = add32(mul32(fx, div32(c[0], c[2])), cx);
        const float v = add32(mul32(fy, div32(c[1], c[2])), cy);
        if (!(u >= 0.0f && u < (float)W && v >= 0.0f && v < (float)H)) continue;
        const int i = (int)floor((double)u);
        const int j = (int)floor((double)v);
        if (!newest && mask && mask[(int64_t)j * W + i]) continue;
        const uint32_t b = f32_bits(c[2]);
        uint32_t *cell = &zbuf[(int64_t)j * W + i];
        if (b < *cell) *cell = b;
        ++kept;
    }
    return kept;
}

/* Contour removal (Sec. 5: unreliable depths near contours are removed by a
 * threshold on the gradient of the depth map). Reading: a valid pixel p is
 * dropped iff some valid 4-neighbour q has |D(q) - D(p)| > t * D(p) (FP32, the
 * step relative to the pixel's depth). depth is FP32 here: the decision is
 * taken on the map the filter produced, in its precision. Outputs: valid_out
 * and depth_out (0 where dropped). */
int64_t oracle_contour(const float *depth, const uint8_t *valid, int W, int H, float t, float *depth_out,
                       uint8_t *valid_out)
{
    int64_t dropped = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const int64_t o = (int64_t)y * W + x;
            depth_out[o] = depth[o];
            valid_out[o] = valid[o];
            if (!valid[o]) continue;
            const float d = depth[o];
            const float lim = mul32(t, d);
            const int qx[4] = {x - 1, x + 1, x, x}, qy[4] = {y, y, y - 1, y + 1};
            int drop = 0;
            for (int k = 0; k < 4; ++k) {
                if (qx[k] < 0 || qx[k] >= W || qy[k] < 0 || qy[k] >= H) continue;
                const int64_t q = (int64_t)qy[k] * W + qx[k];
                if (!valid[q]) continue;
                if (fabsf(add32(depth[q], -d)) > lim) drop = 1;
            }
            if (drop) {
                valid_out[o] = 0;
                depth_out[o] = 0.0f;
                ++dropped;
            }
        }
    return dropped;
}

/* ------------------------------------------------------------------------ */
/* Gradient of the joint bilateral filter with respect to its sigmas (Sec. 4:
 * the Gaussian variances can be optimised by backpropagation when dense
 * ground truth exists). With e = ||dI||^2 / (2 sc^2) + ||dx||^2 / (2 sp^2) and
 * w = exp(-e): dw/dsc = w ||dI||^2 / sc^3, dw/dsp = w ||dx||^2 / sp^3. For
 * out = N / Wt (N = sum w beta_d, Wt = sum w beta):
 *   d out / d theta = (sum dw/dtheta beta_d - out sum dw/dtheta beta) / Wt.
 * dbeta_d (2 channels per pixel, or NULL) is the derivative of beta_d with
 * respect to an earlier stage's (sp, sc); it passes through the weights:
 *   d out / d theta_prev = sum w dbeta_d / Wt.
 * dout receives 4 channels per pixel: d/dsp, d/dsc, d/dsp_prev, d/dsc_prev. */
void oracle_jbf_grad(const double *guide, const double *beta, const double *beta_d, const double *dbeta_d,
                     int W, int H, int r, double sp, double sc, double *out, uint8_t *valid, double *dout)
{
    for (int py = 0; py < H; ++py) {
        for (int px = 0; px < W; ++px) {
            const double *Ip = &guide[((int64_t)py * W + px) * 3];
            double N = 0, Wt = 0, Np = 0, Wp = 0, Nc = 0, Wc = 0, Q0 = 0, Q1 = 0;
            int any = 0;
            for (int qy = py - r; qy <= py + r; ++qy) {
                for (int qx = px - r; qx <= px + r; ++qx) {
                    if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
                    const int64_t q = (int64_t)qy * W + qx;
                    if (!(beta[q] > 0.0)) continue;
                    const double *Iq = &guide[q * 3];
                    const double dc = (Iq[0] - Ip[0]) * (Iq[0] - Ip[0]) + (Iq[1] - Ip[1]) * (Iq[1] - Ip[1]) +
                                      (Iq[2] - Ip[2]) * (Iq[2] - Ip[2]);
                    const double ds = (double)(qx - px) * (qx - px) + (double)(qy - py) * (qy - py);
                    const double w = exp(-(dc / (2.0 * sc * sc) + ds / (2.0 * sp * sp)));
                    const double wp = w * ds / (sp * sp * sp), wc = w * dc / (sc * sc * sc);
                    N += w * beta_d[q];
                    Wt += w * beta[q];
                    Np += wp * beta_d[q];
                    Wp += wp * beta[q];
                    Nc += wc * beta_d[q];
                    Wc += wc * beta[q];
                    if (dbeta_d) {
                        Q0 += w * dbeta_d[q * 2];
                        Q1 += w * dbeta_d[q * 2 + 1];
                    }
                    any = 1;
                }
            }
            const int64_t o = (int64_t)py * W + px;
            valid[o] = (uint8_t)any;
            if (!any) {
                out[o] = 0.0;
                dout[o * 4] = dout[o * 4 + 1] = dout[o * 4 + 2] = dout[o * 4 + 3] = 0.0;
                continue;
            }
            const double D = N / Wt;
            out[o] = D;
            dout[o * 4 + 0] = (Np - D * Wp) / Wt;
            dout[o * 4 + 1] = (Nc - D * Wc) / Wt;
            dout[o * 4 + 2] = Q0 / Wt;
            dout[o * 4 + 3] = Q1 / Wt;
        }
    }
}
