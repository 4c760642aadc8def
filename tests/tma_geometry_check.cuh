// Host-side model check of the TMA filter tiles' geometry (test code, compiled by
// tests/test_tma_geometry.py with nvcc as a host-only program; no GPU).
//
// For one instantiation TmaGeom<SRC, R, KP, NW, FORM> it checks, with the constants the
// kernels are compiled with:
//  * every tensor-map box within the hardware's 256 elements per dimension, with an inner
//    extent that is a multiple of 16 bytes;
//  * the shared-memory layout: 128-byte raw buffers, 16-byte staged arrays, the whole
//    within the 227 KB a CTA may use;
//  * on a set of grid sizes, every tile: the x coordinate of each bulk tensor copy on a
//    16-byte boundary, and every raw-box index the conversion and the slow path compute
//    (colour bytes, restored depth, z-buffer word, pooled guide and sums) inside its box,
//    every staged-record and bitmap index the tap and validity loops compute inside its
//    array.
// It returns the number of violations and prints the first few.
#pragma once

#include <cstdio>

#include "../paper_2601_01210_gb300/csrc/tma_common.cuh"

namespace geomcheck {

inline int fdiv3(int a) { return a >= 0 ? a / 3 : -((2 - a) / 3); }   // floor(a / 3)

struct Report {
    const char *name;
    int bad = 0;
    void fail(const char *what, int a, int b, int c) {
        if (bad++ < 5) std::printf("%s: %s (%d, %d, %d)\n", name, what, a, b, c);
    }
};

template <int SRC, int R, int KP, int NW, int FORM>
int check(const char *name) {
    using namespace dz;
    using G = TmaGeom<SRC, R, KP, NW, FORM>;
    Report rep{name};
    constexpr bool PAIRS = G::PAIRS;
    constexpr int T = 2 * R + 1;
    // ---- boxes and layout
    const int boxes[5][3] = {{G::RGB_BX, G::RGB_BY, 1}, {G::C_BX, G::C_BY, 8}, {G::Z_BX, G::Z_BY, 4},
                             {G::G_BX, G::G_BY, 4},     {G::S_BX, G::S_BY, 4}};
    const bool used[5] = {SRC != SRC_COARSE, SRC == SRC_UP, SRC == SRC_ZBUF, SRC == SRC_COARSE, SRC == SRC_COARSE};
    for (int b = 0; b < 5; ++b) {
        if (!used[b]) continue;
        if (boxes[b][0] < 1 || boxes[b][0] > 256 || boxes[b][1] < 1 || boxes[b][1] > 256) rep.fail("box size", b, boxes[b][0], boxes[b][1]);
        if ((boxes[b][0] * boxes[b][2]) % 16) rep.fail("box inner bytes", b, boxes[b][0], boxes[b][2]);
    }
    if (G::RAW_A % 128 || G::RAW_B % 128) rep.fail("raw buffer alignment", G::RAW_A, G::RAW_B, 0);
    if (G::OFF_STAGED % 16 || G::OFF_G % 16 || G::OFF_OBS % 4 || G::OFF_BAR % 8) rep.fail("layout alignment", G::OFF_STAGED, G::OFF_G, G::OFF_OBS);
    if (G::SMEM > 232448) rep.fail("shared memory", G::SMEM, 232448, 0);
    if (G::NCONV * G::NT < G::SH * G::SP) rep.fail("conversion coverage", G::NCONV, G::NT, G::SH * G::SP);
    if (PAIRS && (G::STAGED < G::SH * G::SP * 16 || G::STAGED_G < G::SH * G::SP * 8))
        rep.fail("paired records", G::STAGED, G::STAGED_G, G::SH * G::SP);
    if (G::SPARSE) {
        constexpr int FW = 8 + 2 * R;
        if (G::TW != 32 || G::TH % 8 || G::SW > 64) rep.fail("sparse tile / row mask", G::TW, G::TH, G::SW);
        if (G::NW * G::RPW < G::SH) rep.fail("sparse record rows", G::NW, G::RPW, G::SH);
        if (G::STAGED < 2 * G::SH * G::SW * 16) rep.fail("sparse records", G::STAGED, G::SH, G::SW);
        if (G::OFF_ROWS % 16 || G::ROWS < G::SH * 8) rep.fail("sparse row masks", G::OFF_ROWS, G::ROWS, G::SH);
        // every block's footprint: staged rows and the bits of its row masks
        for (int by = 0; by < G::TH; by += 8)
            for (int bx = 0; bx < G::TW; bx += 8) {
                if (by + 7 + 2 * R >= G::SH) rep.fail("sparse footprint rows", bx, by, R);
                if (bx + FW > G::SW || bx + FW > 64) rep.fail("sparse footprint columns", bx, by, R);
                for (int ly = 0; ly < 8; ++ly)
                    for (int lx = 0; lx < 8; ++lx) {   // a pixel's window for the shifted recomputation
                        const int px = bx + lx, py = by + ly;
                        if (py + 2 * R >= G::SH || px + 2 * R >= G::SW) rep.fail("sparse window", px, py, R);
                    }
            }
    }
    // ---- taps, validity words and centres of every thread (the same for every tile)
    for (int warp = 0; warp < NW; ++warp)
        for (int lane = 0; lane < 32; ++lane) {
            const int rbase = warp * KP;
            for (int iy = 0; iy < KP + 2 * R; ++iy) {
                const int bit = (rbase + iy) * G::SP + lane;
                if ((bit >> 5) + 1 >= G::OBS_WORDS) rep.fail("bitmap word", warp, lane, iy);
                if (lane + T - 1 >= G::SP) rep.fail("window leaves its row", warp, lane, iy);
                for (int dx = 0; dx < T; ++dx)
                    if ((rbase + iy) * G::SP + lane + dx >= G::SH * G::SP) rep.fail("staged record", warp, lane, iy);
            }
            for (int k = 0; k < KP; ++k)
                for (int h = 0; h < (PAIRS ? 2 : 1); ++h) {
                    const int cx = lane + 32 * h;   // staged column of the pixel, minus R
                    if (rbase + k + 2 * R >= G::SH || cx + 2 * R >= G::SW) rep.fail("window of a pixel", warp, lane, k);
                }
        }
    // ---- every tile of a set of grids (for SRC_COARSE the pooled grid)
    const int sizes[][2] = {{1920, 1080}, {1281, 721}, {640, 360}, {427, 241}, {97, 250}, {33, 17}, {1, 1}};
    for (const auto &sz : sizes) {
        const int gw = sz[0], gh = sz[1];
        for (int y0 = 0; y0 < gh; y0 += G::TH)
            for (int x0 = 0; x0 < gw; x0 += G::TW) {
                // bulk tensor copy x coordinates (bytes on a 16-byte boundary)
                if (SRC != SRC_COARSE && (3 * x0 - G::RGB_LEAD) % 16) rep.fail("rgb box x", x0, y0, 0);
                if (SRC == SRC_UP && ((fdiv3(x0 - R) & ~1) * 8) % 16) rep.fail("s1 box x", x0, y0, 0);
                if (SRC == SRC_ZBUF && ((x0 - G::Z_LEAD) * 4) % 16) rep.fail("z box x", x0, y0, 0);
                if (SRC == SRC_COARSE && ((4 * (x0 - R)) * 4 % 16 || ((x0 - G::S_LEAD) * 4) % 16)) rep.fail("pooled box x", x0, y0, 0);
                const int cx0 = fdiv3(x0 - R) & ~1, cy0 = fdiv3(y0 - R);
                for (int sy = 0; sy < G::SH; ++sy)
                    for (int sx = 0; sx < G::SW; ++sx) {
                        const int gx = x0 - R + sx, gy = y0 - R + sy;
                        if (SRC != SRC_COARSE) {
                            const int o = 3 * sx - 3 * R + G::RGB_LEAD;   // colour bytes of the position
                            if (o < 0 || o + 2 >= G::RGB_BX) rep.fail("rgb byte", x0, sy, sx);
                        }
                        const bool in = gx >= 0 && gx < gw && gy >= 0 && gy < gh;
                        if (SRC == SRC_UP && in) {
                            const int ci = gy / 3 - cy0, cj = gx / 3 - cx0;
                            if (ci < 0 || ci >= G::C_BY || cj < 0 || cj >= G::C_BX) rep.fail("restored depth", x0, y0, sx);
                        }
                        if (SRC == SRC_ZBUF) {
                            const int zi = sx - R + G::Z_LEAD;
                            if (zi < 0 || zi >= G::Z_BX) rep.fail("z word", x0, sy, sx);
                        }
                        if (SRC == SRC_COARSE) {
                            const int si = sx - R + G::S_LEAD;
                            if (si < 0 || si >= G::S_BX) rep.fail("pooled sum", x0, sy, sx);
                            if (4 * sx + 3 >= G::G_BX) rep.fail("pooled guide", x0, sy, sx);
                        }
                    }
            }
    }
    return rep.bad;
}

}  // namespace geomcheck
