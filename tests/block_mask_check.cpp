// Conservativeness check of the blend's 8 x BH block mask (blend_mask.cuh):
// for random 2D Gaussians (rotated, elongated, tiny and huge, opacity down to
// the 1/255 cut), tiles of 8, 16 and 32 pixels and blocks 8 or 16 pixels
// tall, every pixel of every block
// whose bit is clear must fail the blend's alpha test, both as the kernel
// evaluates the exponent in FP32 and in FP64 with a margin.  Prints
// "tile block_height blocks set needed failures" per case; exit status 1 on
// any failure.
#include "blend_mask.cuh"

#include <cmath>
#include <cstdio>
#include <random>

namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLog2AlphaMin = -7.9943534368588578f;

struct Counts {
    long blocks = 0, set = 0, needed = 0, failures = 0;
};

template <int TS, int BH>
void run(std::mt19937_64 &rng, int trials, Counts &c) {
    constexpr int BX = TS / 8, BY = TS / BH;
    std::uniform_real_distribution<double> U(0.0, 1.0);
    for (int it = 0; it < trials; it++) {
        // covariance: random angle, log-uniform sigmas, +0.3 px^2 dilation
        const double th = U(rng) * M_PI;
        const int kind = it % 4;
        const double s_lo = kind == 0 ? 0.05 : 0.5, s_hi = kind == 1 ? 3000.0 : 60.0;
        const double s1 = s_lo * std::pow(s_hi / s_lo, U(rng)), s2 = s_lo * std::pow(s_hi / s_lo, U(rng));
        const double ct = std::cos(th), st = std::sin(th);
        const double c00 = ct * ct * s1 * s1 + st * st * s2 * s2 + 0.3;
        const double c11 = st * st * s1 * s1 + ct * ct * s2 * s2 + 0.3;
        const double c01 = ct * st * (s1 * s1 - s2 * s2);
        const double det = c00 * c11 - c01 * c01;
        const float a = (float)(c11 / det), b = (float)(-c01 / det), cc = (float)(c00 / det);
        float o;
        if (kind == 3 && (it & 4)) o = 1.0f / 255.0f * (1.0f + (float)(U(rng) * 1e-3));   // at the cut
        else o = (float)(std::pow(255.0, -U(rng)) * 0.99 + 1.0 / 255.0 * 0.01);
        if (o < 1.0f / 255.0f) o = 1.0f / 255.0f;
        // the same expressions as the blend's staging
        const float A = -0.5f * kLog2e * a, B = -kLog2e * b, C = -0.5f * kLog2e * cc, L = std::log2(o);
        const double ext = 3.5 * std::sqrt(std::max(c00, c11));
        const int x0 = 8 * (int)(U(rng) * 40), y0 = 8 * (int)(U(rng) * 40);
        const float u = (float)(x0 + TS * 0.5 + (U(rng) - 0.5) * (TS + 2.0 * ext));
        const float v = (float)(y0 + TS * 0.5 + (U(rng) - 0.5) * (TS + 2.0 * ext));
        const uint32_t m = d4dgs::block_mask<TS, BH>(u, v, A, B, C, L, x0, y0);
        for (int r = 0; r < BY; r++)
            for (int q = 0; q < BX; q++) {
                bool any32 = false, near64 = false;
                for (int yy = 0; yy < BH; yy++)
                    for (int xx = 0; xx < 8; xx++) {
                        const float pxf = (float)(x0 + 8 * q + xx) + 0.5f, pyf = (float)(y0 + BH * r + yy) + 0.5f;
                        const float dx = u - pxf, dy = v - pyf;
                        const float axx = A * dx * dx, bx = B * dx;
                        const float p = std::fma(std::fma(C, dy, bx), dy, axx);
                        const float qq = p + L;
                        if (p <= 0.0f && qq >= kLog2AlphaMin) any32 = true;
                        const double dxd = (double)u - pxf, dyd = (double)v - pyf;
                        const double q64 = (double)A * dxd * dxd + (double)B * dxd * dyd + (double)C * dyd * dyd + L;
                        if (q64 >= (double)kLog2AlphaMin - 1e-4) near64 = true;
                    }
                const bool bit = (m >> (r * BX + q)) & 1u;
                c.blocks++;
                c.set += bit;
                c.needed += any32;
                if (!bit && (any32 || near64)) {
                    if (c.failures < 5)
                        std::printf("FAIL TS=%d BH=%d u=%.6g v=%.6g A=%.9g B=%.9g C=%.9g L=%.9g tile=(%d,%d) block=(%d,%d)\n",
                                    TS, BH, u, v, A, B, C, L, x0, y0, q, r);
                    c.failures++;
                }
            }
    }
}

}  // namespace

int main(int argc, char **argv) {
    const int trials = argc > 1 ? std::atoi(argv[1]) : 20000;
    std::mt19937_64 rng(12345);
    Counts c[5];
    run<8, 8>(rng, trials, c[0]);
    run<16, 8>(rng, trials, c[1]);
    run<32, 8>(rng, trials, c[2]);
    run<16, 16>(rng, trials, c[3]);
    run<32, 16>(rng, trials, c[4]);
    const int ts[5] = {8, 16, 32, 16, 32}, bh[5] = {8, 8, 8, 16, 16};
    long fails = 0;
    for (int i = 0; i < 5; i++) {
        std::printf("%d %d %ld %ld %ld %ld\n", ts[i], bh[i], c[i].blocks, c[i].set, c[i].needed, c[i].failures);
        fails += c[i].failures;
    }
    return fails ? 1 : 0;
}
