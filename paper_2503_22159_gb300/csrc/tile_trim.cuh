// tile_trim.cuh -- per-column trims of a Gaussian's tile rectangle: the tiles
// of each of the rectangle's first kTrimCols columns that its alpha >= 1/255
// ellipse actually reaches.  The binning keeps only those (plus every tile of
// the columns beyond), which removes the rectangle's empty corners from the
// pair lists of the sort and the blend.  Self-contained and usable from host
// code (compiled with -ffp-contract=off), so its conservativeness can be
// checked on the CPU against the blend's per-pixel exponent.
#pragma once
#include <cmath>
#include <cstdint>

#ifdef __CUDACC__
#define D4DGS_TT __host__ __device__ __forceinline__
#else
#define D4DGS_TT inline
#endif

namespace d4dgs {

constexpr int kTrimCols = 8;                 // leading rectangle columns that carry trims
constexpr int kTrimMax = 15;                 // rows trimmed at most at a column's top and bottom
constexpr float kTrimMarginPx = 1.0f / 64.0f;

namespace trim_ops {
#ifdef __CUDA_ARCH__
D4DGS_TT float mul(float a, float b) { return __fmul_rn(a, b); }
D4DGS_TT float add(float a, float b) { return __fadd_rn(a, b); }
D4DGS_TT float sub(float a, float b) { return __fsub_rn(a, b); }
D4DGS_TT float dvd(float a, float b) { return __fdiv_rn(a, b); }
D4DGS_TT float sqr(float a) { return __fsqrt_rn(a); }
#else
D4DGS_TT float mul(float a, float b) { return a * b; }
D4DGS_TT float add(float a, float b) { return a + b; }
D4DGS_TT float sub(float a, float b) { return a - b; }
D4DGS_TT float dvd(float a, float b) { return a / b; }
D4DGS_TT float sqr(float a) { return std::sqrt(a); }
#endif
}  // namespace trim_ops

// Byte j of a trim word belongs to rectangle column x0 + j: low nibble the
// rows cut at the top, high nibble the rows cut at the bottom.  Columns from
// kTrimCols on are never trimmed.
D4DGS_TT uint32_t trim_byte(uint64_t w, int j) {
    const uint32_t half = j < 4 ? (uint32_t)w : (uint32_t)(w >> 32);
    return j < kTrimCols ? (half >> (8 * (j & 3))) & 0xFFu : 0u;
}
D4DGS_TT int trim_top(uint64_t w, int j) { return (int)(trim_byte(w, j) & 15u); }
D4DGS_TT int trim_bot(uint64_t w, int j) { return (int)(trim_byte(w, j) >> 4); }
// tiles kept in column j of a rectangle h rows tall
D4DGS_TT int trim_count(uint64_t w, int j, int h) {
    const uint32_t b = trim_byte(w, j);
    const int k = h - (int)(b & 15u) - (int)(b >> 4);
    return k > 0 ? k : 0;
}

// Trim word of one Gaussian: 2D mean (u, v), covariance (s00, s01, s11)
// with det = s00 s11 - s01^2 > 0, ellipse d^T Sigma^-1 d <= k2 (the binning
// ellipse, margins included) with half-extents ex = sqrt(k2 s00),
// ey = sqrt(k2 s11), inclusive tile rectangle [x0, x1] x [y0, y1], tile size
// and image width in pixels.
//
// For a column whose pixel centres span dx in [xa, xb] (dx = x - u) the
// ellipse's rows at dx are dy = (s01 dx -+ sqrt(det (k2 s00 - dx^2))) / s00;
// the upper branch is convex with its minimum at dx = -s01 ey / s11 (the
// ellipse's top point), the lower concave with its maximum at +s01 ey / s11,
// so clamping those abscissae to [max(xa, -ex), min(xb, ex)] gives the
// column's exact row extent (the divisions by s00 done as products with one
// rounded reciprocal 1/s00).  Widened by 1/64 px, it is compared with the
// pixel-centre rows [r T + 0.5, r T + T - 0.5] of every tile row: rows that
// miss it are cut (at most kTrimMax at either end; a column that misses the
// ellipse keeps min(h, 2 kTrimMax) rows cut).  T is a power of two, so
// products with 1/T are exact divisions.  Every operation is a single
// correctly rounded FP32 operation in this order, so other IEEE machines
// reproduce the word bit for bit.
D4DGS_TT uint64_t tile_trims(float u, float v, float s00, float s01, float s11, float det, float k2, float ex,
                             float ey, int x0, int x1, int y0, int y1, float tilef, float widthf) {
    using namespace trim_ops;
    const int h = y1 - y0 + 1;
    const int nc = x1 - x0 + 1 < kTrimCols ? x1 - x0 + 1 : kTrimCols;
    const float q = mul(k2, s00);
    const float dxb = dvd(mul(s01, ey), s11);
    const float is00 = dvd(1.0f, s00), itile = dvd(1.0f, tilef);
    const float tlast = sub(tilef, 0.5f), xlast = sub(widthf, 0.5f);
    uint64_t w = 0;
    for (int j = 0; j < nc; j++) {
        const float cx = mul((float)(x0 + j), tilef);
        const float da = fmaxf(sub(add(cx, 0.5f), u), -ex);
        const float db = fminf(sub(fminf(add(cx, tlast), xlast), u), ex);
        int top, bot;
        if (!(da <= db)) {   // the column's pixel centres miss the ellipse
            top = h < kTrimMax ? h : kTrimMax;
            bot = h - top < kTrimMax ? h - top : kTrimMax;
        } else {
            const float dT = fminf(fmaxf(-dxb, da), db), dB = fminf(fmaxf(dxb, da), db);
            const float st = sqr(fmaxf(0.0f, mul(det, sub(q, mul(dT, dT)))));
            const float sb = sqr(fmaxf(0.0f, mul(det, sub(q, mul(dB, dB)))));
            const float lo = sub(sub(add(v, mul(sub(mul(s01, dT), st), is00)), kTrimMarginPx), tlast);
            const float hi = sub(add(add(v, mul(add(mul(s01, dB), sb), is00)), kTrimMarginPx), 0.5f);
            const float r0 = ceilf(mul(lo, itile)), r1 = floorf(mul(hi, itile));
            top = (int)fminf(fmaxf(sub(r0, (float)y0), 0.0f), (float)kTrimMax);
            bot = (int)fminf(fmaxf(sub((float)y1, r1), 0.0f), (float)kTrimMax);
        }
        w |= (uint64_t)(uint32_t)(top | (bot << 4)) << (8 * j);
    }
    return w;
}

}  // namespace d4dgs
