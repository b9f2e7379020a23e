// Conservativeness and tightness check of the binning's column cuts
// (tile_trim.cuh), host build of the same header: for random 2D Gaussians
// (rotated, elongated, tiny and huge, opacity down to the 1/255 cut, centres
// on and off the image) with the preprocess's FP32 rectangle, every pixel of
// a cut tile must fail the blend's alpha test, both as the kernel evaluates
// the exponent in FP32 and in FP64 with a margin.  Prints "tile rect_tiles
// kept_tiles needed_tiles failures" per tile size; exit status 1 on any
// failure.
#include "tile_trim.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <random>

namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLog2AlphaMin = -7.9943534368588578f;

struct Counts {
    long rect = 0, kept = 0, needed = 0, failures = 0;
};

void run(int TS, std::mt19937_64 &rng, int trials, Counts &cnt) {
    const int W = 1352, H = 1014;
    const int tiles_x = (W + TS - 1) / TS, tiles_y = (H + TS - 1) / TS;
    const float tilef = (float)TS;
    std::uniform_real_distribution<double> U(0.0, 1.0);
    for (int it = 0; it < trials; it++) {
        const double th = U(rng) * M_PI;
        const int kind = it % 4;
        const double s_lo = kind == 0 ? 0.05 : 0.5, s_hi = kind == 1 ? 400.0 : 60.0;
        const double s1 = s_lo * std::pow(s_hi / s_lo, U(rng)), s2 = s_lo * std::pow(s_hi / s_lo, U(rng));
        const double ct = std::cos(th), st = std::sin(th);
        const float s00 = (float)(ct * ct * s1 * s1 + st * st * s2 * s2 + 0.3);
        const float s11 = (float)(st * st * s1 * s1 + ct * ct * s2 * s2 + 0.3);
        const float s01 = (float)(ct * st * (s1 * s1 - s2 * s2));
        const float det = s00 * s11 - s01 * s01;
        if (!(det > 0.0f)) continue;
        float oh;
        if (kind == 3 && (it & 4)) oh = 1.0f / 255.0f * (1.0f + (float)(U(rng) * 1e-3));
        else oh = (float)(std::pow(255.0, -U(rng)) * 0.99 + 1.0 / 255.0 * 0.01);
        if (oh < 1.0f / 255.0f) oh = 1.0f / 255.0f;
        const float u = (float)(-200.0 + U(rng) * (W + 400.0)), v = (float)(-200.0 + U(rng) * (H + 400.0));
        // the preprocess's FP32 rectangle
        const float k2 = ((2.0f * std::log(255.0f * oh)) * 1.0008f) + 0.0008f;
        const float ex = std::sqrt(k2 * s00), ey = std::sqrt(k2 * s11);
        const float rx = std::ceil(ex), ry = std::ceil(ey);
        const float fx0 = std::floor((u - rx) / tilef), fx1 = std::floor((u + rx) / tilef);
        const float fy0 = std::floor((v - ry) / tilef), fy1 = std::floor((v + ry) / tilef);
        if (!(fx1 >= 0.0f) || !(fx0 <= (float)(tiles_x - 1)) || !(fy1 >= 0.0f) || !(fy0 <= (float)(tiles_y - 1)))
            continue;
        const int x0 = (int)std::max(fx0, 0.0f), x1 = (int)std::min(fx1, (float)(tiles_x - 1));
        const int y0 = (int)std::max(fy0, 0.0f), y1 = (int)std::min(fy1, (float)(tiles_y - 1));
        const uint64_t tw = d4dgs::tile_trims(u, v, s00, s01, s11, det, k2, ex, ey, x0, x1, y0, y1, tilef, (float)W);
        // the blend's staged conic (record, then the base-2 scaling of the staging)
        const float inv_det = 1.0f / det;
        const float a = s11 * inv_det, b = -s01 * inv_det, c = s00 * inv_det;
        const float A = -0.5f * kLog2e * a, B = -kLog2e * b, C = -0.5f * kLog2e * c, L = std::log2(oh);
        const int h = y1 - y0 + 1;
        for (int tx = x0; tx <= x1; tx++)
            for (int ty = y0; ty <= y1; ty++) {
                const int j = tx - x0;
                const bool kept = ty - y0 >= d4dgs::trim_top(tw, j) && y1 - ty >= d4dgs::trim_bot(tw, j);
                bool any32 = false, near64 = false;
                for (int py = ty * TS; py < std::min(ty * TS + TS, H); py++)
                    for (int px = tx * TS; px < std::min(tx * TS + TS, W); px++) {
                        const float dx = u - ((float)px + 0.5f), dy = v - ((float)py + 0.5f);
                        const float p = std::fma(std::fma(C, dy, B * dx), dy, A * dx * dx);
                        if (p <= 0.0f && p + L >= kLog2AlphaMin) any32 = true;
                        const double dxd = (double)u - (px + 0.5), dyd = (double)v - (py + 0.5);
                        const double q64 = (double)A * dxd * dxd + (double)B * dxd * dyd + (double)C * dyd * dyd + L;
                        if (q64 >= (double)kLog2AlphaMin - 1e-4) near64 = true;
                    }
                cnt.rect++;
                cnt.kept += kept;
                cnt.needed += any32;
                if (!kept && (any32 || near64)) {
                    if (cnt.failures < 5)
                        std::printf("FAIL TS=%d u=%.9g v=%.9g s=(%.9g %.9g %.9g) oh=%.9g tile=(%d,%d) rect=[%d,%d]x[%d,%d] h=%d\n",
                                    TS, u, v, s00, s01, s11, oh, tx, ty, x0, x1, y0, y1, h);
                    cnt.failures++;
                }
            }
        // the count the preprocess records equals the kept tiles
        long k = 0;
        for (int j = 0; j <= x1 - x0; j++) k += d4dgs::trim_count(tw, j, h);
        long direct = 0;
        for (int tx = x0; tx <= x1; tx++)
            for (int ty = y0; ty <= y1; ty++)
                direct += ty - y0 >= d4dgs::trim_top(tw, tx - x0) && y1 - ty >= d4dgs::trim_bot(tw, tx - x0);
        if (k != direct) {
            if (cnt.failures < 5) std::printf("COUNT TS=%d %ld != %ld\n", TS, k, direct);
            cnt.failures++;
        }
    }
}

}  // namespace

int main(int argc, char **argv) {
    const int trials = argc > 1 ? std::atoi(argv[1]) : 3000;
    std::mt19937_64 rng(2503);
    const int ts[3] = {8, 16, 32};
    long fails = 0;
    for (int i = 0; i < 3; i++) {
        Counts c;
        run(ts[i], rng, trials, c);
        std::printf("%d %ld %ld %ld %ld\n", ts[i], c.rect, c.kept, c.needed, c.failures);
        fails += c.failures;
    }
    return fails ? 1 : 0;
}
