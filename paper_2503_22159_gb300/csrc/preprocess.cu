// preprocess.cu -- K1: one thread per Gaussian, the per-frame preprocess of
// Algorithm 1 fused into one pass over the scene (HBM-bound: 64 B of
// geometry + up to 192 B of SH read per Gaussian, 64 B written).
//
//   tau = t - mu_t;  mu(t) = mu + tau V3D                      (Eq. 7)
//   X = R_cam mu(t) + T_cam  (= P_view + tau V_view)           (Eq. 9-11, 15)
//   o_hat = sigmoid(logit) * exp(-tau^2 / (2 s_t^2))           (Eq. 6-7)
//   (u, v) = (fx X/Z + cx, fy Y/Z + cy)                         (Eq. 12)
//   J at the time-shifted mean, x/z and y/z clamped             (Eq. 14)
//   Sigma' = (J W M)(J W M)^T + 0.3 I,  M = R(q) diag(s)        (Eq. 16; Sigma3D = M M^T)
//   radius = ceil(3.33 sqrt(lambda_max)); tile rectangle = bounding box of the
//   alpha >= 1/255 ellipse (half-extents ceil(k sqrt(Sigma'_00)), ceil(k sqrt(Sigma'_11)),
//   k^2 = 2 ln(255 o_hat) with a small margin); depth key = bits(Z)
//   colour = max(0, SH . Y(normalize(mu(t) - campos)) + 0.5)
//
// The quantities that decide binning (Z, u, v, o_hat, Sigma', lambda_max,
// radius, rectangle) use explicitly rounded single-precision operations in a
// fixed order (__fmul_rn/__fadd_rn/__fdiv_rn/__fsqrt_rn are never contracted
// into FMAs; the FMAs that are there are explicit), and exp and log are the
// explicit methods below rather than a math library's, so a CPU evaluation of
// the same steps reproduces every binning decision, and the tile lists, bit
// for bit.
#include "d4dgs_internal.cuh"
#include "tile_trim.cuh"

namespace d4dgs {

namespace {

__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float dvd(float a, float b) { return __fdiv_rn(a, b); }

// exp and log of the binning arithmetic, each a published method in explicitly
// rounded steps (within ~1 ulp of the exact function):
//   bexp(x): Cody-Waite reduction x = n ln2 + r with n = rint(x log2 e) and ln2
//            split into a 16-bit head (n ln2_hi is exact for |n| < 256) and a
//            tail; e^r by its Taylor series to r^7/7! in Horner form with fused
//            multiply-adds (|r| <= ln2/2, truncation below 0.1 ulp); times 2^n
//            (exact); x < -87 gives 0 and x > 88.5 gives +inf.
//   blog(x): x = m 2^e with m in [sqrt(1/2), sqrt(2)), s = (m-1)/(m+1),
//            log m = 2 atanh s = 2 (s + s^3/3 + s^5/5 + s^7/7 + s^9/9)
//            (|s| <= 0.172, truncation below 1e-9 relative), plus e ln2.
constexpr float kLn2Hi = 0.693145751953125f;   // ln 2 rounded to 16 significant bits
constexpr float kLn2Lo = 1.42860682e-06f;      // float(ln 2 - kLn2Hi)
constexpr float kLog2eF = 1.44269502f;         // float(1 / ln 2)
constexpr float kSqrt2F = 1.41421354f;         // float(sqrt 2)

__device__ __forceinline__ float bexp(float x) {
    if (x != x) return x;
    if (x < -87.0f) return 0.0f;
    if (x > 88.5f) return __int_as_float(0x7F800000);
    const float n = rintf(mul(x, kLog2eF));
    float r = __fmaf_rn(-n, kLn2Hi, x);
    r = __fmaf_rn(-n, kLn2Lo, r);
    float p = 1.98412701e-04f;              // 1/7!
    p = __fmaf_rn(p, r, 1.38888892e-03f);   // 1/6!
    p = __fmaf_rn(p, r, 8.33333377e-03f);   // 1/5!
    p = __fmaf_rn(p, r, 4.16666679e-02f);   // 1/4!
    p = __fmaf_rn(p, r, 1.66666672e-01f);   // 1/3!
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    int k = (int)n;
    if (k > 127) {
        p = mul(p, 2.0f);
        k -= 1;
    }
    return mul(p, __uint_as_float((uint32_t)(k + 127) << 23));
}

__device__ __forceinline__ float blog(float x) {
    if (!(x > 0.0f)) return x == 0.0f ? __int_as_float(0xFF800000) : __int_as_float(0x7FC00000);
    if (x == __int_as_float(0x7F800000)) return x;
    int e = 0;
    if (x < 1.17549435e-38f) {   // subnormal: times 2^23
        x = mul(x, 8388608.0f);
        e = -23;
    }
    uint32_t b = __float_as_uint(x);
    e += (int)(b >> 23) - 127;
    float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
    if (m > kSqrt2F) {
        m = mul(m, 0.5f);
        e += 1;
    }
    const float s = dvd(sub(m, 1.0f), add(m, 1.0f));
    const float z = mul(s, s);
    float p = 1.11111112e-01f;              // 1/9
    p = __fmaf_rn(p, z, 1.42857149e-01f);   // 1/7
    p = __fmaf_rn(p, z, 2.00000003e-01f);   // 1/5
    p = __fmaf_rn(p, z, 3.33333343e-01f);   // 1/3
    const float lm = __fmaf_rn(mul(s, z), p, s);   // atanh s
    const float ef = (float)e;
    return __fmaf_rn(ef, kLn2Hi, __fmaf_rn(ef, kLn2Lo, mul(2.0f, lm)));
}

// Real SH basis (Condon-Shortley phase; coefficient k = l^2 + l + m), constants
// from their closed forms.
constexpr float kC0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kC1 = 0.48860251190291992f;   // sqrt(3/(4 pi))
constexpr float kC2a = 1.0925484305920792f;   // sqrt(15/pi)/2
constexpr float kC2b = 0.31539156525252005f;  // sqrt(5/pi)/4
constexpr float kC2c = 0.54627421529603959f;  // sqrt(15/pi)/4
constexpr float kC3e = 0.59004358992664352f;  // sqrt(35/(2 pi))/4
constexpr float kC3f = 2.8906114426405538f;   // sqrt(105/pi)/2
constexpr float kC3g = 0.45704579946446577f;  // sqrt(21/(2 pi))/4
constexpr float kC3h = 0.3731763325901154f;   // sqrt(7/pi)/4
constexpr float kC3k = 1.4453057213202769f;   // sqrt(105/pi)/4

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y) {
    Y[0] = kC0;
    if (DEG >= 1) {
        Y[1] = -kC1 * y;
        Y[2] = kC1 * z;
        Y[3] = -kC1 * x;
    }
    if (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kC2a * x * y;
        Y[5] = -kC2a * y * z;
        Y[6] = kC2b * (2.0f * zz - xx - yy);
        Y[7] = -kC2a * x * z;
        Y[8] = kC2c * (xx - yy);
        if (DEG >= 3) {
            Y[9] = -kC3e * y * (3.0f * xx - yy);
            Y[10] = kC3f * x * y * z;
            Y[11] = -kC3g * y * (4.0f * zz - xx - yy);
            Y[12] = kC3h * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
            Y[13] = -kC3g * x * (4.0f * zz - xx - yy);
            Y[14] = kC3k * z * (xx - yy);
            Y[15] = -kC3e * x * (xx - 3.0f * yy);
        }
    }
}

// 2D footprint of one Gaussian at the view's time, before the shared tail.
struct Footprint {
    float m0, m1, m2;     // world-space mean at t (SH view direction)
    float Z, u, v, oh;    // camera depth, pixel mean, opacity at t
    float s00, s01, s11;  // Sigma' (with the 0.3 px^2 dilation)
    float fu, fv;         // screen flow (flow frames only)
};

// Screen flow of a Gaussian (Eq. 13 in pixels): the ray-space velocity of the
// mean, (fx V_x / Z, fy V_y / Z), V the camera-frame velocity.
__device__ __forceinline__ void screen_flow(const CamArgs &c, float v0, float v1, float v2, float Z, Footprint &f) {
    const float *R = c.R;
    const float Vx = R[0] * v0 + R[1] * v1 + R[2] * v2, Vy = R[3] * v0 + R[4] * v1 + R[5] * v2;
    f.fu = c.fx * Vx / Z;
    f.fv = c.fy * Vy / Z;
}

// Disentangled form (Algorithm 1): the deferred temporal slice of the mean
// and opacity, then the projection of the static 3D covariance R S S^T R^T.
// FP32 in the documented binning operation order.  False: not drawn.
__device__ __forceinline__ bool footprint_disentangled(const View &vw, int i, Footprint &f) {
    const CamArgs &c = vw.cam;
    const float t = vw.t;
    const float limx = c.limx, limy = c.limy;
    // every geometric parameter is loaded before the first cull test, so a Gaussian
    // costs one DRAM round trip instead of one per test
    const float p_tm = __ldg(vw.t_mean + i);
    const float p_m0 = __ldg(vw.means + 3 * i + 0), p_m1 = __ldg(vw.means + 3 * i + 1), p_m2 = __ldg(vw.means + 3 * i + 2);
    const float p_v0 = __ldg(vw.velocity + 3 * i + 0), p_v1 = __ldg(vw.velocity + 3 * i + 1);
    const float p_v2 = __ldg(vw.velocity + 3 * i + 2);
    const float p_lg = __ldg(vw.opacity_logit + i), p_lt = __ldg(vw.log_t_scale + i);
    const float4 q = __ldg(reinterpret_cast<const float4 *>(vw.quats) + i);
    const float p_s0 = __ldg(vw.log_scales + 3 * i + 0), p_s1 = __ldg(vw.log_scales + 3 * i + 1);
    const float p_s2 = __ldg(vw.log_scales + 3 * i + 2);
    do {
        // ---- deferred temporal slice and camera transform (binning order)
        const float tau = sub(t, p_tm);
        const float m0 = add(p_m0, mul(tau, p_v0));
        const float m1 = add(p_m1, mul(tau, p_v1));
        const float m2 = add(p_m2, mul(tau, p_v2));
        const float *R = c.R;
        const float X = add(add(add(mul(R[0], m0), mul(R[1], m1)), mul(R[2], m2)), c.T[0]);
        const float Y = add(add(add(mul(R[3], m0), mul(R[4], m1)), mul(R[5], m2)), c.T[1]);
        const float Z = add(add(add(mul(R[6], m0), mul(R[7], m1)), mul(R[8], m2)), c.T[2]);
        if (!(Z > c.near)) break;
        // ---- temporal opacity
        const float o = dvd(1.0f, add(1.0f, bexp(-p_lg)));
        const float st = bexp(p_lt);
        const float oh = mul(o, bexp(dvd(mul(-0.5f, mul(tau, tau)), mul(st, st))));
        if (!(oh >= kAlphaMin)) break;
        // ---- projection of the mean and the Jacobian at the shifted mean
        const float xz = dvd(X, Z), yz = dvd(Y, Z);
        const float u = add(mul(c.fx, xz), c.cx), v = add(mul(c.fy, yz), c.cy);
        const float xzc = fminf(limx, fmaxf(-limx, xz)), yzc = fminf(limy, fmaxf(-limy, yz));
        const float J00 = dvd(c.fx, Z), J02 = dvd(-mul(c.fx, xzc), Z);
        const float J11 = dvd(c.fy, Z), J12 = dvd(-mul(c.fy, yzc), Z);
        // ---- 3D covariance factor M = R(q) diag(s)
        const float qn = __fsqrt_rn(add(add(add(mul(q.x, q.x), mul(q.y, q.y)), mul(q.z, q.z)), mul(q.w, q.w)));
        const float qw = dvd(q.x, qn), qx = dvd(q.y, qn), qy = dvd(q.z, qn), qz = dvd(q.w, qn);
        float Rq[9];
        Rq[0] = sub(1.0f, mul(2.0f, add(mul(qy, qy), mul(qz, qz))));
        Rq[1] = mul(2.0f, sub(mul(qx, qy), mul(qw, qz)));
        Rq[2] = mul(2.0f, add(mul(qx, qz), mul(qw, qy)));
        Rq[3] = mul(2.0f, add(mul(qx, qy), mul(qw, qz)));
        Rq[4] = sub(1.0f, mul(2.0f, add(mul(qx, qx), mul(qz, qz))));
        Rq[5] = mul(2.0f, sub(mul(qy, qz), mul(qw, qx)));
        Rq[6] = mul(2.0f, sub(mul(qx, qz), mul(qw, qy)));
        Rq[7] = mul(2.0f, add(mul(qy, qz), mul(qw, qx)));
        Rq[8] = sub(1.0f, mul(2.0f, add(mul(qx, qx), mul(qy, qy))));
        const float sc[3] = {bexp(p_s0), bexp(p_s1), bexp(p_s2)};
        float M[9];
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int k = 0; k < 3; k++) M[3 * r + k] = mul(Rq[3 * r + k], sc[k]);
        // ---- T = J W (2x3), TM = T M, Sigma' = TM TM^T + 0.3 I
        float Tm[6];
#pragma unroll
        for (int j = 0; j < 3; j++) {
            Tm[j] = add(mul(J00, R[j]), mul(J02, R[6 + j]));
            Tm[3 + j] = add(mul(J11, R[3 + j]), mul(J12, R[6 + j]));
        }
        float TM[6];
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
            for (int k = 0; k < 3; k++)
                TM[3 * r + k] = add(add(mul(Tm[3 * r + 0], M[k]), mul(Tm[3 * r + 1], M[3 + k])), mul(Tm[3 * r + 2], M[6 + k]));
        const float s00 = add(add(add(mul(TM[0], TM[0]), mul(TM[1], TM[1])), mul(TM[2], TM[2])), kDilation);
        const float s01 = add(add(mul(TM[0], TM[3]), mul(TM[1], TM[4])), mul(TM[2], TM[5]));
        const float s11 = add(add(add(mul(TM[3], TM[3]), mul(TM[4], TM[4])), mul(TM[5], TM[5])), kDilation);
        f.m0 = m0; f.m1 = m1; f.m2 = m2;
        f.Z = Z; f.u = u; f.v = v; f.oh = oh;
        f.s00 = s00; f.s01 = s01; f.s11 = s11;
        if (vw.out_flow) screen_flow(c, p_v0, p_v1, p_v2, Z, f);
        return true;
    } while (0);
    return false;
}

// Slicing-first form (Eq. 5-7, the comparison baseline): every frame builds
// the 4D rotation from its quaternion pair (p -> q_l p q_r on p = t + x i +
// y j + z k), Sigma4D = R4 S4^2 R4^T = [[U, V], [V^T, W]], and slices it at t:
// Sigma3D = U - V V^T / W, mean mu + (t - mu_t) V / W, opacity times
// exp(-(t - mu_t)^2 / (2 W)); then the same projection.  Same arithmetic
// rules as the disentangled form (separately rounded products and sums,
// IEEE division and square root, full-precision exp), so the two are timed
// like for like.
__device__ __forceinline__ bool footprint_slicing(const View &vw, int i, Footprint &f) {
    const CamArgs &c = vw.cam;
    const float limx = c.limx, limy = c.limy;
    const float4 m4 = __ldg(reinterpret_cast<const float4 *>(vw.means4) + i);
    const float4 l4 = __ldg(reinterpret_cast<const float4 *>(vw.log_scales4) + i);
    float4 a = __ldg(reinterpret_cast<const float4 *>(vw.quat_l) + i);
    float4 b = __ldg(reinterpret_cast<const float4 *>(vw.quat_r) + i);
    const float na = __fsqrt_rn(add(add(add(mul(a.x, a.x), mul(a.y, a.y)), mul(a.z, a.z)), mul(a.w, a.w)));
    const float nb = __fsqrt_rn(add(add(add(mul(b.x, b.x), mul(b.y, b.y)), mul(b.z, b.z)), mul(b.w, b.w)));
    a = make_float4(dvd(a.x, na), dvd(a.y, na), dvd(a.z, na), dvd(a.w, na));
    b = make_float4(dvd(b.x, nb), dvd(b.y, nb), dvd(b.z, nb), dvd(b.w, nb));
    // left- and right-multiplication matrices in the quaternion basis (1, i, j, k)
    const float La[16] = {a.x, -a.y, -a.z, -a.w, a.y, a.x, -a.w, a.z, a.z, a.w, a.x, -a.y, a.w, -a.z, a.y, a.x};
    const float Rb[16] = {b.x, -b.y, -b.z, -b.w, b.y, b.x, b.w, -b.z, b.z, -b.w, b.x, b.y, b.w, b.z, -b.y, b.x};
    // R4 in (x, y, z, t) order: quaternion components (i, j, k, 1) = indices (1, 2, 3, 0)
    const int perm[4] = {1, 2, 3, 0};
    const float s4[4] = {expf(l4.x), expf(l4.y), expf(l4.z), expf(l4.w)};
    float M[16];   // M = R4 diag(s4)
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int pr = perm[r], pk = perm[k];
            const float acc = add(add(add(mul(La[4 * pr], Rb[pk]), mul(La[4 * pr + 1], Rb[4 + pk])),
                                      mul(La[4 * pr + 2], Rb[8 + pk])), mul(La[4 * pr + 3], Rb[12 + pk]));
            M[4 * r + k] = mul(acc, s4[k]);
        }
    auto sig = [&](int r, int q) {
        return add(add(add(mul(M[4 * r], M[4 * q]), mul(M[4 * r + 1], M[4 * q + 1])), mul(M[4 * r + 2], M[4 * q + 2])),
                   mul(M[4 * r + 3], M[4 * q + 3]));
    };
    const float W = sig(3, 3);
    const float V0 = sig(0, 3), V1 = sig(1, 3), V2 = sig(2, 3);
    const float v0 = dvd(V0, W), v1 = dvd(V1, W), v2 = dvd(V2, W);   // V / W
    const float S00 = sub(sig(0, 0), mul(V0, v0)), S01 = sub(sig(0, 1), mul(V0, v1)), S02 = sub(sig(0, 2), mul(V0, v2));
    const float S11 = sub(sig(1, 1), mul(V1, v1)), S12 = sub(sig(1, 2), mul(V1, v2)), S22 = sub(sig(2, 2), mul(V2, v2));
    const float tau = sub(vw.t, m4.w);
    const float m0 = add(m4.x, mul(tau, v0)), m1 = add(m4.y, mul(tau, v1)), m2 = add(m4.z, mul(tau, v2));
    const float *R = c.R;
    const float X = add(add(add(mul(R[0], m0), mul(R[1], m1)), mul(R[2], m2)), c.T[0]);
    const float Y = add(add(add(mul(R[3], m0), mul(R[4], m1)), mul(R[5], m2)), c.T[1]);
    const float Z = add(add(add(mul(R[6], m0), mul(R[7], m1)), mul(R[8], m2)), c.T[2]);
    if (!(Z > c.near)) return false;
    const float o = dvd(1.0f, add(1.0f, expf(-__ldg(vw.opacity_logit + i))));
    const float oh = mul(o, expf(dvd(mul(-0.5f, mul(tau, tau)), W)));
    if (!(oh >= kAlphaMin)) return false;
    const float xz = dvd(X, Z), yz = dvd(Y, Z);
    const float xzc = fminf(limx, fmaxf(-limx, xz)), yzc = fminf(limy, fmaxf(-limy, yz));
    const float J00 = dvd(c.fx, Z), J02 = dvd(-mul(c.fx, xzc), Z);
    const float J11 = dvd(c.fy, Z), J12 = dvd(-mul(c.fy, yzc), Z);
    float Tm[6];   // J W (2 x 3)
#pragma unroll
    for (int j = 0; j < 3; j++) {
        Tm[j] = add(mul(J00, R[j]), mul(J02, R[6 + j]));
        Tm[3 + j] = add(mul(J11, R[3 + j]), mul(J12, R[6 + j]));
    }
    const float S3[9] = {S00, S01, S02, S01, S11, S12, S02, S12, S22};
    float TS[6];   // (J W) Sigma3D
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
        for (int k = 0; k < 3; k++)
            TS[3 * r + k] = add(add(mul(Tm[3 * r], S3[k]), mul(Tm[3 * r + 1], S3[3 + k])), mul(Tm[3 * r + 2], S3[6 + k]));
    f.m0 = m0; f.m1 = m1; f.m2 = m2;
    f.Z = Z; f.u = add(mul(c.fx, xz), c.cx); f.v = add(mul(c.fy, yz), c.cy); f.oh = oh;
    f.s00 = add(add(add(mul(TS[0], Tm[0]), mul(TS[1], Tm[1])), mul(TS[2], Tm[2])), kDilation);
    f.s01 = add(add(mul(TS[0], Tm[3]), mul(TS[1], Tm[4])), mul(TS[2], Tm[5]));
    f.s11 = add(add(add(mul(TS[3], Tm[3]), mul(TS[4], Tm[4])), mul(TS[5], Tm[5])), kDilation);
    if (vw.out_flow) screen_flow(c, v0, v1, v2, Z, f);
    return true;
}

// One Gaussian of view v: writes its 2D record, depth key, tile count,
// rectangle and (config trim) column cuts, adds its tiles to the view's
// difference grid (2D differences of the rectangle, or per-column
// differences of the cut columns), and counts it in the shared depth-digit
// histogram.
// CACHE (config colour_cache): cc holds the Gaussian's colour once a view of its time group has
// evaluated it (towards the static mean, the same for every view of the group) for the group's next views.
template <int DEG, int KIND, bool CACHE>
__device__ __forceinline__ void preprocess_one(const View &vw, int i, uint32_t *hist, uint32_t &nvis, int *sgrid,
                                               float4 &cc) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const CamArgs &c = vw.cam;
    const float tilef = (float)c.tile;
    {
        uint32_t key = 0xFFFFFFFFu, tiles = 0;
        ushort4 rc = make_ushort4(0, 0, 0, 0);
        uint64_t tw = 0;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
        float flu = 0.0f, flv = 0.0f;
        do {
            Footprint f;
            if (!(KIND == 0 ? footprint_disentangled(vw, i, f) : footprint_slicing(vw, i, f))) break;
            const float m0 = f.m0, m1 = f.m1, m2 = f.m2, Z = f.Z, u = f.u, v = f.v, oh = f.oh;
            const float s00 = f.s00, s01 = f.s01, s11 = f.s11;
            if (vw.out_flow) {
                flu = f.fu;
                flv = f.fv;
            }
            const float det = sub(mul(s00, s11), mul(s01, s01));
            if (!(det > 0.0f)) break;
            const float mid = mul(0.5f, add(s00, s11));
            const float lam = add(mid, __fsqrt_rn(fmaxf(0.1f, sub(mul(mid, mid), det))));
            const float rf = ceilf(mul(kRadiusK, __fsqrt_rn(lam)));
            // ---- tile rectangle (inclusive tile indices): the bounding box of the
            // ellipse d^T Sigma'^-1 d <= k^2, k^2 = 2 ln(255 o_hat) (+ margin), outside
            // which alpha = o_hat e^p < 1/255; half-extents k sqrt(Sigma'_00), k sqrt(Sigma'_11)
            if (!(isfinite(u) && isfinite(v))) break;
            const float k2 = add(mul(mul(2.0f, blog(mul(255.0f, oh))), kK2Scale), kK2Pad);
            const float ex = __fsqrt_rn(mul(k2, s00)), ey = __fsqrt_rn(mul(k2, s11));
            const float rx = ceilf(ex), ry = ceilf(ey);
            // division by the tile size (a power of two) as the exact product with its reciprocal
            const float itile = 1.0f / tilef;
            const float fx0 = floorf(mul(sub(u, rx), itile)), fx1 = floorf(mul(add(u, rx), itile));
            const float fy0 = floorf(mul(sub(v, ry), itile)), fy1 = floorf(mul(add(v, ry), itile));
            if (!(fx1 >= 0.0f) || !(fx0 <= (float)(c.tiles_x - 1))) break;
            if (!(fy1 >= 0.0f) || !(fy0 <= (float)(c.tiles_y - 1))) break;
            const int x0 = (int)fmaxf(fx0, 0.0f), x1 = (int)fminf(fx1, (float)(c.tiles_x - 1));
            const int y0 = (int)fmaxf(fy0, 0.0f), y1 = (int)fminf(fy1, (float)(c.tiles_y - 1));
            const int gw = c.tiles_x + 1;
            int *g = sgrid ? sgrid : vw.grid;   // shared-memory copy when the grid is small
            if (vw.trim_on) {
                // ---- the rectangle's leading columns cut to the rows the ellipse reaches
                tw = tile_trims(u, v, s00, s01, s11, det, k2, ex, ey, x0, x1, y0, y1, tilef, (float)c.width);
                const int h = y1 - y0 + 1;
                for (int j = 0; j <= x1 - x0; j++) tiles += (uint32_t)trim_count(tw, j, h);
                if (tiles == 0) {   // no pixel centre within reach: culled
                    tw = 0;
                    break;
                }
                // per-tile pair counts as per-column differences on the ((tiles_x+1) x (tiles_y+1))
                // grid: +1 at a column's first kept row, -1 below its last
                for (int j = 0; j <= x1 - x0; j++) {
                    const int ra = y0 + trim_top(tw, j), rb = y1 - trim_bot(tw, j);
                    if (ra > rb) continue;
                    atomicAdd(g + ra * gw + x0 + j, 1);
                    atomicAdd(g + (rb + 1) * gw + x0 + j, -1);
                }
            } else {
                // whole rectangle: per-tile pair counts as a 2D difference grid
                tiles = (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
                atomicAdd(g + y0 * gw + x0, 1);
                atomicAdd(g + y0 * gw + x1 + 1, -1);
                atomicAdd(g + (y1 + 1) * gw + x0, -1);
                atomicAdd(g + (y1 + 1) * gw + x1 + 1, 1);
            }
            rc = make_ushort4((unsigned short)x0, (unsigned short)x1, (unsigned short)y0, (unsigned short)y1);
            key = __float_as_uint(Z);
            nvis++;
            // ---- conic (rendering only; ordinary arithmetic from here on): the inverse of
            // Sigma' through a determinant with one compensation step (Kahan's 2x2 determinant:
            // w = s01^2 rounded, its exact rounding error by an FMA, then s00 s11 - w by an FMA;
            // within 2 ulp however close s00 s11 and s01^2 are), so a thin splat's conic carries
            // only the rounding of Sigma' itself, not the cancellation of its determinant
            const float w01 = __fmul_rn(s01, s01);
            const float det_c = __fadd_rn(__fmaf_rn(s00, s11, -w01), __fmaf_rn(-s01, s01, w01));
            const float inv_det = 1.0f / det_c;
            // ---- view-dependent colour in the direction of the shifted mean (colour cache: of the
            // static mean, evaluated once per time group)
            constexpr bool cache = KIND == 0 && CACHE;
            float col[3] = {0.5f, 0.5f, 0.5f};
            if (cache && cc.w != 0.0f) {
                col[0] = cc.x; col[1] = cc.y; col[2] = cc.z;
            } else {
            float dx, dy, dz;
            if (cache) {
                dx = __ldg(vw.means + 3 * i) - c.campos[0];
                dy = __ldg(vw.means + 3 * i + 1) - c.campos[1];
                dz = __ldg(vw.means + 3 * i + 2) - c.campos[2];
            } else {
                dx = m0 - c.campos[0]; dy = m1 - c.campos[1]; dz = m2 - c.campos[2];
            }
            const float inv_n = rsqrtf(dx * dx + dy * dy + dz * dz);
            dx *= inv_n; dy *= inv_n; dz *= inv_n;
            float Yb[16];
            sh_basis<DEG>(dx, dy, dz, Yb);
            const float *shp = vw.sh + (size_t)i * (3 * K);
            if constexpr ((3 * K) % 4 == 0) {
                // 16-byte aligned rows (degree 1 and 3): vector loads
                const float4 *sh4 = reinterpret_cast<const float4 *>(shp);
                float buf[3 * K];
#pragma unroll
                for (int j = 0; j < (3 * K) / 4; j++) {
                    const float4 w4 = __ldg(sh4 + j);
                    buf[4 * j] = w4.x; buf[4 * j + 1] = w4.y; buf[4 * j + 2] = w4.z; buf[4 * j + 3] = w4.w;
                }
#pragma unroll
                for (int k = 0; k < K; k++) {
                    col[0] = fmaf(buf[3 * k + 0], Yb[k], col[0]);
                    col[1] = fmaf(buf[3 * k + 1], Yb[k], col[1]);
                    col[2] = fmaf(buf[3 * k + 2], Yb[k], col[2]);
                }
            } else {
#pragma unroll
                for (int k = 0; k < K; k++) {
                    col[0] = fmaf(__ldg(shp + 3 * k + 0), Yb[k], col[0]);
                    col[1] = fmaf(__ldg(shp + 3 * k + 1), Yb[k], col[1]);
                    col[2] = fmaf(__ldg(shp + 3 * k + 2), Yb[k], col[2]);
                }
            }
            if (cache) cc = make_float4(col[0], col[1], col[2], 1.0f);
            }
            r0 = make_float4(u, v, s11 * inv_det, -s01 * inv_det);
            r1 = make_float4(s00 * inv_det, oh, Z, rf);
            r2 = make_float4(fmaxf(col[0], 0.0f), fmaxf(col[1], 0.0f), fmaxf(col[2], 0.0f), log2f(oh));
        } while (0);
        vw.rec[3 * (size_t)i + 0] = r0;
        vw.rec[3 * (size_t)i + 1] = r1;
        vw.rec[3 * (size_t)i + 2] = r2;
        if (vw.out_flow) vw.flow2d[i] = key == 0xFFFFFFFFu ? make_float2(0.0f, 0.0f) : make_float2(flu, flv);
        vw.dkeys[0][i] = key;
        vw.tiles_touched[i] = tiles;
        vw.rect[i] = rc;
        vw.trim[i] = tw;
#pragma unroll
        for (int p = 0; p < 4; p++) atomicAdd(&hist[p * kRadix + ((key >> (8 * p)) & 0xFFu)], 1u);
    }
}

// Cells of the view's difference grid, and whether a CTA keeps its share of
// the grid in shared memory (small grids, where the corner atomics of all
// Gaussians would otherwise pile onto few addresses).
__device__ __forceinline__ int grid_cells(const View &v) { return (v.cam.tiles_x + 1) * (v.cam.tiles_y + 1); }

// Flush a CTA's depth-digit histogram, visible count and shared grid into view v.
__device__ __forceinline__ void flush_view(const View &v, uint32_t *hist, uint32_t &nvis, int *sgrid) {
    __syncthreads();
    const uint32_t w = __reduce_add_sync(0xFFFFFFFFu, nvis);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(v.ctl + kCtlNumVisible, w);
    nvis = 0;
    for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) {
        if (hist[i]) atomicAdd(v.ctl + kCtlDepthHist + i, hist[i]);
        hist[i] = 0;
    }
    if (sgrid) {
        const int cells = grid_cells(v);
        for (int i = threadIdx.x; i < cells; i += blockDim.x) {
            if (sgrid[i]) atomicAdd(v.grid + i, sgrid[i]);
            sgrid[i] = 0;
        }
    }
    __syncthreads();
}

// Persistent: CTAs take 256-Gaussian chunks of the time groups' flattened
// Gaussians.  For a chunk of a group of B views (one scene and camera, B
// times) each thread takes its Gaussian through the B views in turn, so its
// parameters come from DRAM once and from cache for the other views; every
// view keeps its own shared-memory depth histogram, visible count and, when B
// of them fit, tile-count grid.  The per-view arithmetic is the same as for a
// view alone, so a grouped view's outputs equal the ungrouped ones bit for bit.
// KIND: 0 disentangled, 1 slicing-first (every view of a launch has the same kind).
// CACHE: config colour_cache (shared by every view of a launch).
// PARAM: a launch of one view whose descriptor also travels as the kernel
// parameter v0, read from the constant bank instead of the batch table.
template <int KIND, bool CACHE, bool PARAM>
__global__ void __launch_bounds__(256, 4)
preprocess_kernel(const char *__restrict__ ba, int smem_cells, const __grid_constant__ View v0) {
    __shared__ uint32_t hist[kMaxGroup][4 * kRadix];
    __shared__ int32_t s_chunk;
    extern __shared__ int s_grid[];
    grid_dependency_wait();
    for (int i = threadIdx.x; i < smem_cells; i += blockDim.x) s_grid[i] = 0;
    const uint32_t *bw = reinterpret_cast<const uint32_t *>(ba);
    const int nviews = (int)bw[kBaNViews];
    const int total = (int)bw[kBaTotalChunks];
    uint32_t *counter = const_cast<uint32_t *>(bw) + kBaChunk;
    for (int i = threadIdx.x; i < kMaxGroup * 4 * kRadix; i += blockDim.x) (&hist[0][0])[i] = 0;
    uint32_t nvis[kMaxGroup];
#pragma unroll
    for (int b = 0; b < kMaxGroup; b++) nvis[b] = 0;
    auto view = [&](int u) -> const View & {
        if constexpr (PARAM) return v0;
        else return view_of(ba, u);
    };
    int cur = -1;   // first view of the group whose sums the CTA holds
    // shared-memory grid of slot b of group `lead` (null: the group's grids go to global memory)
    auto slot_grid = [&](int lead, int b) -> int * {
        const View &l = view(lead);
        const int cells = grid_cells(l);
        return cells * l.group_size <= smem_cells ? s_grid + b * cells : nullptr;
    };
    auto flush_group = [&](int lead) {
        const int gs = view(lead).group_size;
        for (int b = 0; b < gs; b++) flush_view(view(lead + b), hist[b], nvis[b], slot_grid(lead, b));
    };
    for (;;) {
        if (threadIdx.x == 0) s_chunk = (int32_t)atomicAdd(counter, 1u);
        __syncthreads();
        const int chunk = s_chunk;
        __syncthreads();
        if (chunk >= total) break;
        int lead = 0;
        for (int u = 1; u < (PARAM ? 1 : nviews); u++) {
            const View &w = view(u);
            if (w.group_size > 0 && w.chunk_base <= chunk) lead = u;
        }
        if (lead != cur) {
            if (cur >= 0) flush_group(cur);
            cur = lead;
        }
        const View &l = view(lead);
        const int i = (chunk - l.chunk_base) * kPreChunk + (int)threadIdx.x;
        const int gs = l.group_size;
        float4 cc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);   // colour cache of this Gaussian (w = 1: valid)
        for (int b = 0; b < gs; b++) {
            const View &v = view(lead + b);
            int *sg = slot_grid(lead, b);
            if (i < v.n) {
                switch (v.sh_degree) {
                    case 0: preprocess_one<0, KIND, CACHE>(v, i, hist[b], nvis[b], sg, cc); break;
                    case 1: preprocess_one<1, KIND, CACHE>(v, i, hist[b], nvis[b], sg, cc); break;
                    case 2: preprocess_one<2, KIND, CACHE>(v, i, hist[b], nvis[b], sg, cc); break;
                    default: preprocess_one<3, KIND, CACHE>(v, i, hist[b], nvis[b], sg, cc); break;
                }
            }
        }
    }
    if (cur >= 0) flush_group(cur);
}

// First kernel of a frame or batch: installs the descriptor table (from the
// by-value parameter, or from args_dev when given), the launch totals, zeroed
// work counters, and clears every view's per-frame region.
__global__ void __launch_bounds__(256)
clear_kernel(const __grid_constant__ BatchArgs args, const BatchArgs *args_dev, char *__restrict__ ba) {
    grid_dependency_wait();
    const BatchArgs *A = args_dev ? args_dev : &args;
    const int nviews = A->nviews;
    if (blockIdx.x == 0) {
        uint32_t *bw = reinterpret_cast<uint32_t *>(ba);
        for (int i = threadIdx.x; i < kBaWords; i += blockDim.x) bw[i] = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            bw[kBaNViews] = (uint32_t)nviews;
            bw[kBaTotalChunks] = (uint32_t)A->total_chunks;
            bw[kBaTotalDepthParts] = (uint32_t)A->total_depth_parts;
            bw[kBaTotalDupParts] = (uint32_t)A->total_dup_parts;
            bw[kBaTotalTiles] = (uint32_t)A->total_tiles;
            bw[kBaTotalDirParts] = (uint32_t)A->total_dir_parts;
            bw[kBaTotalBands] = (uint32_t)A->total_bands;
            bw[kBaTotalRankParts] = (uint32_t)A->total_rank_parts;
        }
        const uint32_t *src = reinterpret_cast<const uint32_t *>(A->v);
        uint32_t *dst = reinterpret_cast<uint32_t *>(ba + kBatchTableOffset);
        const int words = nviews * (int)(sizeof(View) / 4);
        for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    }
    for (int vi = 0; vi < nviews; vi++) {
        uint4 *z = reinterpret_cast<uint4 *>(A->v[vi].zero_base);
        const int64_t words = A->v[vi].zero_bytes / 16;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x)
            z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
}

}  // namespace

CamArgs make_cam_args(const d4dgs_camera *cam, int32_t tile, float near) {
    CamArgs a;
    a.near = near;
    for (int i = 0; i < 9; i++) a.R[i] = cam->R[i];
    for (int i = 0; i < 3; i++) a.T[i] = cam->T[i];
    a.fx = cam->fx; a.fy = cam->fy; a.cx = cam->cx; a.cy = cam->cy;
    for (int j = 0; j < 3; j++) {
        double p = -((double)cam->R[0 + j] * cam->T[0] + (double)cam->R[3 + j] * cam->T[1] + (double)cam->R[6 + j] * cam->T[2]);
        a.campos[j] = (float)p;
    }
    a.width = cam->width; a.height = cam->height; a.tile = tile;
    {   // one IEEE single-precision product, quotient and product each, as the kernels would round them
        const float hw = 0.5f * (float)cam->width, hh = 0.5f * (float)cam->height;
        const float qx = hw / cam->fx, qy = hh / cam->fy;
        a.limx = kJacClamp * qx;
        a.limy = kJacClamp * qy;
    }
    a.tiles_x = (cam->width + tile - 1) / tile;
    a.tiles_y = (cam->height + tile - 1) / tile;
    return a;
}

cudaError_t launch_clear(const BatchArgs &args, const void *args_dev, char *batch_area, cudaStream_t st,
                         int num_sms) {
    const cudaError_t e = launch_chained(clear_kernel, num_sms * 2, 256, 0, st, args,
                                         static_cast<const BatchArgs *>(args_dev), batch_area);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_preprocess(const BatchArgs &args, const char *batch_area, cudaStream_t st, int num_sms,
                              bool host_views) {
    if (args.total_chunks == 0) return cudaSuccess;
    // persistent grid of the CTAs that are resident at once (a CTA beyond them would only start
    // once the chunks are gone, and still clear and flush its shared sums); grids of up to
    // 6144 cells (e.g. 1352x1014 at 32-px tiles) are aggregated in shared memory
    constexpr int kSmemCells = 6144;
    constexpr size_t kSmem = kSmemCells * sizeof(int);
    static int occ[6] = {0, 0, 0, 0, 0, 0};   // by variant, queried once
    auto go = [&](auto fn, int which) {
        if (!occ[which] && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[which], (const void *)fn, 256, kSmem) !=
                                cudaSuccess ||
                            occ[which] < 1))
            occ[which] = 1;
        return launch_chained(fn, occ[which] * num_sms, 256, kSmem, st, (const char *)batch_area, kSmemCells,
                              args.v[0]);
    };
    // one view whose descriptor the host holds: the descriptor as a kernel parameter
    const bool param = host_views && args.nviews == 1;
    const int kind = args.v[0].kind == 1 ? 0 : args.v[0].colour_cache ? 1 : 2;
    cudaError_t e;
    if (param)
        e = kind == 0 ? go(preprocess_kernel<1, false, true>, 3)
            : kind == 1 ? go(preprocess_kernel<0, true, true>, 4)
                        : go(preprocess_kernel<0, false, true>, 5);
    else
        e = kind == 0 ? go(preprocess_kernel<1, false, false>, 0)
            : kind == 1 ? go(preprocess_kernel<0, true, false>, 1)
                        : go(preprocess_kernel<0, false, false>, 2);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace d4dgs
