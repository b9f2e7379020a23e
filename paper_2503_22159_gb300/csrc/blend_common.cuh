// blend_common.cuh -- pieces shared by the blend (blend.cu) and its backward
// replay (backward.cu): packed FP32x2 arithmetic, the pixel layout of a tile
// and the fast-body conditions.  Both kernels evaluate a pair's exponent with
// the same operations, so the backward recovers the forward's alphas bit for
// bit.
#pragma once
#include "d4dgs_internal.cuh"

namespace d4dgs {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLog2AlphaMin = -7.9943534368588578f;   // log2(1/255)

// Packed FP32x2 arithmetic (sm_100 family): both lanes rounded to nearest,
// no flush to zero, exactly as the scalar operations.
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// A Gaussian takes the fast compositing body when neither the 0.99 clamp nor
// the p > 0 test can fire for it, so both can be left out with the same bits:
//  * L = log2(o_hat) <= log2(0.98): q <= L, and ex2.approx is within a few
//    ulp, so 2^q < 0.99;
//  * 4 al ga - be^2 > 2^-12 (al + ga)^2: the FP32 exponent p (two products
//    and two FMAs) is off by at most ~8 u (al + ga) r^2 (u = 2^-24, r the
//    pixel's distance to the mean) while -p >= lambda_min r^2 with
//    lambda_min >= det4 / (4 (al + ga)), so the computed p is never > 0
//    (margin 2^7).
// Every other Gaussian takes the general body.
constexpr float kLog2FastOpacity = -0.029146346f;    // log2(0.98)
constexpr float kInf = __builtin_huge_valf();
constexpr float kFastConditioning = 1.0f / 4096.0f;
constexpr uint32_t kSlowBit = 1u << 31;             // in the staged block mask

template <bool B>
struct BoolC {
    static constexpr bool value = B;
};

template <int TS>
struct BlendShape {
    static constexpr int PX = TS == 8 ? 2 : 4;   // pixels per thread (a column)
    static constexpr int NP = PX / 2;            // pixel pairs
    static constexpr int BH = 4 * PX;            // warp block: 8 wide, BH tall
    static constexpr int NT = TS * TS / PX;      // threads per CTA
    static constexpr int BX = TS / 8, BY = TS / BH;
    static_assert(NT / 32 == BX * BY, "one warp per block");
};

}  // namespace d4dgs
