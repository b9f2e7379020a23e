// blend_mask.cuh -- which 8 x BH pixel blocks of a tile one Gaussian's
// alpha >= 1/255 region reaches (used by the blend to let each warp skip the
// Gaussians of its tile list that cannot touch its block).  Self-contained
// and usable from host code, so its conservativeness can be checked on the
// CPU against the per-pixel exponent.
#pragma once
#include <cmath>
#include <cstdint>

#ifdef __CUDACC__
#define D4DGS_HD __host__ __device__ __forceinline__
#else
#define D4DGS_HD inline
#endif

namespace d4dgs {

constexpr float kLog2_255 = 7.9943534368588578f;   // -log2(1/255)
constexpr float kBlockMarginRel = 1e-3f;           // margins of the test (see block_mask)
constexpr float kBlockMarginAbs = 1e-3f;
constexpr float kBlockMarginPx = 1.0f / 64.0f;

// Bit set of the 8 x BH pixel blocks (8 wide, BH tall) of a TS x TS tile
// (row-major, bit r * (TS/8) + c) that the ellipse {q >= log2(1/255)} of one
// Gaussian reaches.
// With dx = u - x, dy = v - y the ellipse is al dx^2 + be dx dy + ga dy^2 <= K
// (al = -A, be = -B, ga = -C, K = L + log2 255).  For a band of pixel rows
// the reachable dx form one interval: for fixed dy they are centred at
// -be dy / (2 al) with half-width sqrt((K - D dy^2) / al), D = det / (4 al);
// the right end is concave in dy and largest at the dy of the ellipse's
// rightmost point, dy_R = -be e_x / (2 ga), the left end convex and smallest
// at -dy_R, so clamping those to the band gives the interval exactly.  Blocks
// whose pixel-centre columns miss it get no bit.  K is inflated (relative and
// absolute margins) and the interval widened by 1/64 px, far above the FP32
// rounding of both this test and the per-pixel exponent, so no pixel whose q
// passes in the blend loop lies in an unmarked block.  Every multiply-add is
// written as fmaf, so host and device builds compute the same bits.
template <int TS, int BH>
D4DGS_HD uint32_t block_mask(float u, float v, float A, float B, float C, float L, int x0, int y0) {
    constexpr int BX = TS / 8, BY = TS / BH;
    static_assert(BX >= 1 && BY >= 1 && BX * BY <= 16 && BY * BH == TS, "tile of 8, 16 or 32 pixels");
    constexpr uint32_t kAll = (1u << (BX * BY)) - 1u;
    const float al = -A, be = -B, ga = -C;
    float K = L + kLog2_255;
    if (!(K >= 0.0f)) return 0u;   // o_hat < 1/255: no pixel passes
    K = fmaf(K, 1.0f + kBlockMarginRel, kBlockMarginAbs);
    const float det4 = fmaf(4.0f * al, ga, -(be * be));
    if (!(det4 > 0.0f) || !(al > 0.0f) || !(ga > 0.0f)) return kAll;   // not positive definite in FP32
    const float ex = sqrtf(4.0f * ga * K / det4), ey = sqrtf(4.0f * al * K / det4);
    const float ia = 1.0f / al, cs = -0.5f * be * ia, D = 0.25f * det4 * ia;
    const float dyR = -0.5f * be * ex / ga;
    uint32_t m = 0u;
#pragma unroll 1
    for (int r = 0; r < BY; r++) {
        const float ylo = (float)(y0 + BH * r) + 0.5f, yhi = ylo + (float)(BH - 1);
        const float d0 = fmaxf(v - yhi, -ey), d1 = fminf(v - ylo, ey);
        if (d0 > d1) continue;   // the band is outside the ellipse's rows
        const float dA = fminf(fmaxf(dyR, d0), d1), dB = fminf(fmaxf(-dyR, d0), d1);
        const float dxmax = fmaf(cs, dA, sqrtf(fmaxf(0.0f, fmaf(-(D * dA), dA, K) * ia)));
        const float dxmin = fmaf(cs, dB, -sqrtf(fmaxf(0.0f, fmaf(-(D * dB), dB, K) * ia)));
        const float xlo_reach = u - dxmax - kBlockMarginPx, xhi_reach = u - dxmin + kBlockMarginPx;
#pragma unroll
        for (int c = 0; c < BX; c++) {
            const float xlo = (float)(x0 + 8 * c) + 0.5f, xhi = xlo + 7.0f;
            if (xlo_reach <= xhi && xhi_reach >= xlo) m |= 1u << (r * BX + c);
        }
    }
    return m;
}

}  // namespace d4dgs
