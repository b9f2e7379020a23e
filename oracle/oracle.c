/*
 * oracle.c -- plain, slow CPU reference for rendering one frame of a
 * disentangled 4D Gaussian scene at time t (Disentangled 4D Gaussian
 * Splatting, arXiv 2503.22159).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code with the CUDA path.
 *
 * Contents
 *   orc_preprocess      FP64: activations, deferred temporal slice, camera
 *                       transform, projection to a 2D Gaussian, SH colour.
 *   orc_render_pixels   FP64: per-pixel brute force over *all* drawn
 *                       Gaussians, depth sort, front-to-back compositing
 *                       (Eq. 4), plus an error budget ("slack") per pixel for
 *                       decisions that sit within FP32 reach of a threshold.
 *   orc_bin_f32         FP32 mirror of the binning arithmetic in a fixed,
 *                       documented operation order (no FMA contraction; the
 *                       file is compiled with -ffp-contract=off) giving depth
 *                       key bits, radius, tile rectangle and tile count, with
 *                       flags on decisions that pass through expf within
 *                       3e-6 relative of a threshold.
 *   orc_backward        FP64 adjoint (reverse mode) of the whole frame with
 *                       respect to the raw per-Gaussian parameters.
 *
 * Readings of the paper (where it is silent, garbled or inconsistent):
 *   - Time shift: Eq. 7's mu(t) = mu + (t - mu_t) V (the definition the
 *     disentangled velocity V3D = V/W comes from, Sec. III-B-1); Eq. 15 and
 *     Algorithm 1 print the opposite sign (mu_t - t), which equals V -> -V.
 *   - Temporal factor: exp(-1/2 (t - mu_t)^2 / s_t^2) with s_t = sqrt(W) and
 *     lambda = 1/W (Eq. 6-7; Eq. 6 misprints x for t).  It multiplies the
 *     3DGS opacity.
 *   - The 2D mean is the exact perspective projection of the time-shifted
 *     camera-space mean P_view + tau V_view (Eq. 12, 15); Eq. 13's ray-space
 *     velocity is not used to render.
 *   - Depth for sorting is camera-space z (3DGS convention).
 *   - SH colour is evaluated in the direction of the time-shifted mean.
 *   - 3DGS constants (the paper defers to 3DGS for rasterisation): near plane
 *     0.2 unless the camera sets another,
 *     +0.3 px^2 dilation, Jacobian clamp 1.3 x half-FoV, alpha <= 0.99, skip
 *     alpha < 1/255, stop before blending when T(1-alpha) < 1e-4, black
 *     background; tile radius 3.33 sqrt(lambda_max) (3.33^2 > 2 ln 255, so
 *     every pixel with alpha >= 1/255 lies inside the square).
 *   - Compositing product runs over j = 1..i-1 (Eq. 4 misprints j = i).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_DILATION 0.3
#define ORC_ALPHA_MAX 0.99
#define ORC_ALPHA_MIN (1.0 / 255.0)
#define ORC_T_MIN 1e-4
#define ORC_RADIUS_K 3.33
#define ORC_JAC_CLAMP 1.3

typedef struct {
    int32_t n, sh_degree;
    const double *means;         /* N x 3 */
    const double *t_mean;        /* N */
    const double *velocity;      /* N x 3 */
    const double *log_scales;    /* N x 3 */
    const double *log_t_scale;   /* N */
    const double *quats;         /* N x 4, (w,x,y,z), not necessarily unit */
    const double *opacity_logit; /* N */
    const double *sh;            /* N x (deg+1)^2 x 3 */
    const double *cov3d;         /* optional N x 6 (xx,xy,xz,yy,yz,zz): replaces scales+quats */
    const double *in_err;        /* optional N x 10, with cov3d: bounds on the FP32 error of the inputs an
                                    FP32 evaluation starts from (see fp32_bounds) */
    int32_t colour_static;       /* 1: SH colour in the direction of the static mean mu (the per-camera
                                    colour cache, an approximation); 0: of the time-shifted mean mu(t) */
} orc_scene;

typedef struct {
    double R[9], T[3];           /* world -> camera, row-major */
    double fx, fy, cx, cy;
    int32_t width, height;
    double near;                 /* near plane on camera z (0.2, the 3DGS plane, unless set) */
} orc_camera;

typedef struct {                 /* per-Gaussian FP64 2D Gaussian, all arrays length N */
    int32_t *drawn;
    double *u, *v, *depth;
    double *conic;               /* N x 3 (a, b, c): inverse of the 2D covariance */
    double *cov2d;               /* N x 3 (xx, xy, yy) including the dilation */
    double *opacity_t;           /* sigmoid(logit) * temporal factor */
    double *rgb;                 /* N x 3 */
    double *lambda_max;
    double *err;                 /* optional N x 8: FP32 error bounds of the projection (fp32_bounds) */
} orc_g2d;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * Real spherical harmonics up to degree 3, coefficient k = l^2 + l + m, in the
 * convention Y_lm = sqrt2 Im Y_l^|m| (m<0), Y_l^0 (m=0), sqrt2 Re Y_l^m (m>0)
 * of the complex harmonics *with* the Condon-Shortley phase (the basis the
 * 3DGS colour model uses).  Constants from their closed forms.
 * ------------------------------------------------------------------------- */
void orc_sh_basis(const double d[3], int degree, double *Y) {
    const double pi = 3.14159265358979323846;
    double x = d[0], y = d[1], z = d[2];
    Y[0] = 0.5 * sqrt(1.0 / pi);
    if (degree < 1) return;
    double c1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    if (degree < 2) return;
    double xx = x * x, yy = y * y, zz = z * z;
    double a = 0.5 * sqrt(15.0 / pi), b = 0.25 * sqrt(5.0 / pi), c = 0.25 * sqrt(15.0 / pi);
    Y[4] = a * x * y;
    Y[5] = -a * y * z;
    Y[6] = b * (2.0 * zz - xx - yy);
    Y[7] = -a * x * z;
    Y[8] = c * (xx - yy);
    if (degree < 3) return;
    double e = 0.25 * sqrt(35.0 / (2.0 * pi)), f = 0.5 * sqrt(105.0 / pi);
    double g = 0.25 * sqrt(21.0 / (2.0 * pi)), h = 0.25 * sqrt(7.0 / pi);
    double k = 0.25 * sqrt(105.0 / pi);
    Y[9] = -e * y * (3.0 * xx - yy);
    Y[10] = f * x * y * z;
    Y[11] = -g * y * (4.0 * zz - xx - yy);
    Y[12] = h * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
    Y[13] = -g * x * (4.0 * zz - xx - yy);
    Y[14] = k * z * (xx - yy);
    Y[15] = -e * x * (xx - 3.0 * yy);
}

/* Rotation matrix of the unit quaternion (w,x,y,z), row-major. */
void orc_quat_to_rot(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

static void matmul3(const double *A, const double *B, double *C) { /* C = A B, 3x3 */
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}
static void transpose3(const double *A, double *At) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) At[3 * j + i] = A[3 * i + j];
}

/* 3D covariance of Gaussian i: Sigma3D = R S S^T R^T (Algorithm 1, "calculate
 * 3D covariance"), or the covariance supplied directly. */
static void cov3d_of(const orc_scene *sc, int i, double S3[9]) {
    if (sc->cov3d) {
        const double *c = sc->cov3d + 6 * (size_t)i;
        S3[0] = c[0]; S3[1] = c[1]; S3[2] = c[2];
        S3[3] = c[1]; S3[4] = c[3]; S3[5] = c[4];
        S3[6] = c[2]; S3[7] = c[4]; S3[8] = c[5];
        return;
    }
    const double *q = sc->quats + 4 * (size_t)i;
    double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double qn[4] = {q[0] / nq, q[1] / nq, q[2] / nq, q[3] / nq};
    double R[9], M[9], Mt[9];
    orc_quat_to_rot(qn, R);
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) M[3 * r + c] = R[3 * r + c] * exp(sc->log_scales[3 * (size_t)i + c]);
    transpose3(M, Mt);
    matmul3(M, Mt, S3);
}

static void cam_position(const orc_camera *cam, double p[3]) { /* -R^T T */
    for (int j = 0; j < 3; j++)
        p[j] = -(cam->R[0 * 3 + j] * cam->T[0] + cam->R[1 * 3 + j] * cam->T[1] + cam->R[2 * 3 + j] * cam->T[2]);
}

/* ---------------------------------------------------------------------------
 * Binary32 evaluation of the projection, in the fixed operation order the
 * GPU preprocess follows (the binning contract).  Every product, sum,
 * quotient and square root is a separately rounded IEEE single operation
 * evaluated left to right as parenthesised (this file is compiled with
 * -ffp-contract=off), so any IEEE machine gives the same bits.  exp and log
 * are not left to a math library (libraries differ by an ulp or two): both
 * sides evaluate the same published method in explicitly rounded steps,
 *   exp(x): Cody-Waite reduction x = n ln2 + r, n = rint(x log2 e), ln2 split
 *           into a 16-bit head (n ln2_hi exact) and a tail; e^r by its Taylor
 *           series to r^7/7! in Horner form with fused multiply-adds
 *           (|r| <= ln2/2: truncation below 0.1 ulp); times 2^n (exact);
 *           x < -87 gives 0, x > 88.5 gives +inf;
 *   log(x): x = m 2^e with m in [sqrt(1/2), sqrt(2)), s = (m-1)/(m+1),
 *           log m = 2 atanh s = 2 (s + s^3/3 + s^5/5 + s^7/7 + s^9/9)
 *           (|s| <= 0.172: truncation below 1e-9 relative), plus e ln2;
 * each within ~1 ulp of the exact function.  fmaf is the correctly rounded
 * fused multiply-add of C99.
 * ------------------------------------------------------------------------- */
#define ORC_LN2_HI 0.693145751953125f       /* ln 2 rounded to 16 significant bits */
#define ORC_LN2_LO 1.42860682e-06f          /* float(ln 2 - ORC_LN2_HI) */
#define ORC_LOG2E_F 1.44269502f             /* float(1 / ln 2) */
#define ORC_SQRT2_F 1.41421354f             /* float(sqrt 2) */

float orc_expf(float x) {
    if (x != x) return x;
    if (x < -87.0f) return 0.0f;
    if (x > 88.5f) return INFINITY;
    const float n = rintf(x * ORC_LOG2E_F);
    float r = fmaf(-n, ORC_LN2_HI, x);
    r = fmaf(-n, ORC_LN2_LO, r);
    float p = 1.98412701e-04f;                      /* 1/7! */
    p = fmaf(p, r, 1.38888892e-03f);                /* 1/6! */
    p = fmaf(p, r, 8.33333377e-03f);                /* 1/5! */
    p = fmaf(p, r, 4.16666679e-02f);                /* 1/4! */
    p = fmaf(p, r, 1.66666672e-01f);                /* 1/3! */
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int k = (int)n;
    if (k > 127) { p = p * 2.0f; k -= 1; }
    uint32_t b = (uint32_t)(k + 127) << 23;
    float scale;
    memcpy(&scale, &b, 4);
    return p * scale;
}

float orc_logf(float x) {
    if (!(x > 0.0f)) return x == 0.0f ? -INFINITY : NAN;
    if (x == INFINITY) return x;
    int e = 0;
    if (x < 1.17549435e-38f) { x = x * 8388608.0f; e = -23; }   /* subnormal: times 2^23 */
    uint32_t b;
    memcpy(&b, &x, 4);
    e += (int)(b >> 23) - 127;
    b = (b & 0x007FFFFFu) | 0x3F800000u;
    float m;
    memcpy(&m, &b, 4);
    if (m > ORC_SQRT2_F) { m = m * 0.5f; e += 1; }
    const float s = (m - 1.0f) / (m + 1.0f);
    const float z = s * s;
    float p = 1.11111112e-01f;                      /* 1/9 */
    p = fmaf(p, z, 1.42857149e-01f);                /* 1/7 */
    p = fmaf(p, z, 2.00000003e-01f);                /* 1/5 */
    p = fmaf(p, z, 3.33333343e-01f);                /* 1/3 */
    const float lm = fmaf(s * z, p, s);             /* atanh s */
    const float ef = (float)e;
    return fmaf(ef, ORC_LN2_HI, fmaf(ef, ORC_LN2_LO, 2.0f * lm));
}

typedef struct { float mu[3], tm, vel[3], ls[3], lt, q[4], lg; } orc_param_f32;
typedef struct { float R[9], T[3], fx, fy, cx, cy; int32_t width, height; float near; } orc_camera_f32;
typedef struct { float X, Y, Z, oh, u, v, s00, s01, s11, det; } orc_fp32;

/* The 2D footprint of one Gaussian in binary32 (order above):
 *   tau = t - mu_t;  m_j = mu_j + tau*v_j
 *   X_r = ((R_r0*m_0 + R_r1*m_1) + R_r2*m_2) + T_r;   cull !(Z > 0.2)
 *   o = 1/(1 + exp(-logit)); st = exp(lst); o_hat = o * exp((-0.5*(tau*tau))/(st*st)); cull !(o_hat >= 1/255)
 *   xz = X/Z, yz = Y/Z; u = fx*xz + cx; v = fy*yz + cy
 *   limx = 1.3*((0.5*W)/fx); xzc = min(limx, max(-limx, xz)) (same for y)
 *   J00 = fx/Z, J02 = -(fx*xzc)/Z, J11 = fy/Z, J12 = -(fy*yzc)/Z
 *   qn = q / sqrtf(((w*w + x*x) + y*y) + z*z); R(qn) as in orc_quat_to_rot
 *   with 1 - 2*(a*a + b*b) and 2*(a*b -/+ c*d); M_ij = R_ij * exp(ls_j)
 *   Tm_j = J00*W_0j + J02*W_2j; Tm_(3+j) = J11*W_1j + J12*W_2j   (T = J W)
 *   TM_ij = (Tm_i0*M_0j + Tm_i1*M_1j) + Tm_i2*M_2j            (TM = J W M)
 *   s00 = ((TM00^2 + TM01^2) + TM02^2) + 0.3; s11 likewise;
 *   s01 = (TM00*TM10 + TM01*TM11) + TM02*TM12
 *   det = s00*s11 - s01*s01; cull !(det > 0)
 * Returns 0 (near plane), 1 (temporal opacity), 2 (det) or 3 (projected);
 * the fields computed up to the cull are filled. */
static int project_f32(const orc_param_f32 *P, const orc_camera_f32 *cam, float t, orc_fp32 *f) {
    const float limx = 1.3f * ((0.5f * (float)cam->width) / cam->fx);
    const float limy = 1.3f * ((0.5f * (float)cam->height) / cam->fy);
    const float tau = t - P->tm;
    const float m0 = P->mu[0] + tau * P->vel[0], m1 = P->mu[1] + tau * P->vel[1], m2 = P->mu[2] + tau * P->vel[2];
    const float *R = cam->R;
    f->X = ((R[0] * m0 + R[1] * m1) + R[2] * m2) + cam->T[0];
    f->Y = ((R[3] * m0 + R[4] * m1) + R[5] * m2) + cam->T[1];
    f->Z = ((R[6] * m0 + R[7] * m1) + R[8] * m2) + cam->T[2];
    const float X = f->X, Y = f->Y, Z = f->Z;
    if (!(Z > cam->near)) return 0;
    const float o = 1.0f / (1.0f + orc_expf(-P->lg));
    const float st = orc_expf(P->lt);
    f->oh = o * orc_expf((-0.5f * (tau * tau)) / (st * st));
    if (!(f->oh >= (float)(1.0 / 255.0))) return 1;
    const float xz = X / Z, yz = Y / Z;
    f->u = cam->fx * xz + cam->cx;
    f->v = cam->fy * yz + cam->cy;
    const float xzc = fminf(limx, fmaxf(-limx, xz)), yzc = fminf(limy, fmaxf(-limy, yz));
    const float J00 = cam->fx / Z, J02 = -(cam->fx * xzc) / Z;
    const float J11 = cam->fy / Z, J12 = -(cam->fy * yzc) / Z;
    const float *q = P->q;
    const float qn = sqrtf(((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3]);
    const float w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
    float Rq[9];
    Rq[0] = 1.0f - 2.0f * (y * y + z * z); Rq[1] = 2.0f * (x * y - w * z);       Rq[2] = 2.0f * (x * z + w * y);
    Rq[3] = 2.0f * (x * y + w * z);       Rq[4] = 1.0f - 2.0f * (x * x + z * z); Rq[5] = 2.0f * (y * z - w * x);
    Rq[6] = 2.0f * (x * z - w * y);       Rq[7] = 2.0f * (y * z + w * x);       Rq[8] = 1.0f - 2.0f * (x * x + y * y);
    const float sc[3] = {orc_expf(P->ls[0]), orc_expf(P->ls[1]), orc_expf(P->ls[2])};
    float M[9];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) M[3 * r + c] = Rq[3 * r + c] * sc[c];
    float Tm[6];
    for (int j = 0; j < 3; j++) {
        Tm[j] = J00 * R[j] + J02 * R[6 + j];
        Tm[3 + j] = J11 * R[3 + j] + J12 * R[6 + j];
    }
    float TM[6];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++)
            TM[3 * r + c] = (Tm[3 * r + 0] * M[0 * 3 + c] + Tm[3 * r + 1] * M[1 * 3 + c]) + Tm[3 * r + 2] * M[2 * 3 + c];
    f->s00 = ((TM[0] * TM[0] + TM[1] * TM[1]) + TM[2] * TM[2]) + 0.3f;
    f->s01 = (TM[0] * TM[3] + TM[1] * TM[4]) + TM[2] * TM[5];
    f->s11 = ((TM[3] * TM[3] + TM[4] * TM[4]) + TM[5] * TM[5]) + 0.3f;
    f->det = f->s00 * f->s11 - f->s01 * f->s01;
    if (!(f->det > 0.0f)) return 2;
    return 3;
}

/* ---------------------------------------------------------------------------
 * fp32_bounds: first-order bounds on how far a binary32 evaluation of one
 * Gaussian's projection (the expression tree of orc_preprocess, sums in any
 * grouping) can land from the exact values.  They size the per-pixel slack of
 * orc_render_pixels and nothing else.
 *
 * Model: every float operation is correctly rounded, fl(a op b) = (a op b)(1+d)
 * with |d| <= u = 2^-24; a sum of k terms (each a product or an input) has an
 * error of at most k u times the sum of their magnitudes; exp, log and log2 are
 * within ORC_FN_REL relative.  Inputs (scene parameters, camera) are binary32
 * values, so they carry no error of their own, except in cov3d mode where the
 * caller passes bounds on the mean at t, the opacity at t and Sigma3D (the
 * slicing-first form, Eq. 5-7, computes them in FP32 before this tree starts).
 *
 *   tau = t - mu_t:                  |d tau| <= u |tau|
 *   m_j = mu_j + tau v_j:            |d m_j| <= 2u |tau v_j| + u |m_j|
 *   X_r = sum_j R_rj m_j + T_r:      |d X_r| <= sum_j |R_rj| |d m_j| + 4u (sum_j |R_rj m_j| + |T_r|)
 *   x/z:                             |d xz| <= (|d X| + |xz| |d Z|) / Z + u |xz|
 *   u_px = fx xz + cx:               |d u| <= fx |d xz| + 2u |fx xz| + u |cx|
 *   o_hat = sigmoid(lg) e^x, x = -tau^2 / (2 s_t^2):
 *                                    rel <= 2E + 3u + |x| (5u + 2E)
 *   J: the x/z clamp limit 1.3 (W/2)/fx carries 3u; J00 = fx/Z, J02 = -fx xzc / Z
 *   q_hat = q/|q| (4u rel per component) -> R(q_hat) entries within 24u
 *   M = R(q_hat) diag(e^ls):         |d M_rk| <= (24u + (E + u) |R_rk|) s_k
 *   Tm = J W, TM = Tm M, Sigma' = TM TM^T + 0.3 I (products and sums as above);
 *   cov3d mode: TS = Tm Sigma3D, Sigma' = TS Tm^T + 0.3 I.
 * err = {|d u|, |d v|, |d Z|, rel d o_hat, |d Sigma'_00|, |d Sigma'_01|, |d Sigma'_11|}.
 * orc_preprocess uses these a-priori bounds in cov3d mode only; for scenes in
 * the disentangled form it evaluates the binary32 footprint itself
 * (project_f32), whose error is then known exactly.
 * ------------------------------------------------------------------------- */
#define ORC_U (1.0 / 16777216.0)
#define ORC_FN_REL (4.0 * ORC_U)

static void fp32_bounds(const orc_scene *sc, const orc_camera *cam, int i, double tau, const double m[3],
                        const double X[3], double limx, double limy, double st, double err[7]) {
    const double u = ORC_U, E = ORC_FN_REL;
    const double *R = cam->R, *T = cam->T;
    const double *ie = sc->in_err ? sc->in_err + 10 * (size_t)i : NULL;
    double dm[3], dop;
    if (ie) {
        dm[0] = ie[0]; dm[1] = ie[1]; dm[2] = ie[2];
        dop = ie[3];
    } else {
        const double *v = sc->velocity + 3 * (size_t)i;
        for (int j = 0; j < 3; j++) dm[j] = 2.0 * u * fabs(tau * v[j]) + u * fabs(m[j]);
        const double x = 0.5 * tau * tau / (st * st);
        dop = 2.0 * E + 3.0 * u + x * (5.0 * u + 2.0 * E);
    }
    double dX[3];
    for (int r = 0; r < 3; r++) {
        double prop = 0.0, mag = fabs(T[r]);
        for (int j = 0; j < 3; j++) {
            prop += fabs(R[3 * r + j]) * dm[j];
            mag += fabs(R[3 * r + j] * m[j]);
        }
        dX[r] = prop + 4.0 * u * mag;
    }
    const double Z = X[2], dZ = dX[2];
    const double xz = X[0] / Z, yz = X[1] / Z;
    const double dxz = (dX[0] + fabs(xz) * dZ) / Z + u * fabs(xz);
    const double dyz = (dX[1] + fabs(yz) * dZ) / Z + u * fabs(yz);
    err[0] = cam->fx * dxz + 2.0 * u * fabs(cam->fx * xz) + u * fabs(cam->cx);
    err[1] = cam->fy * dyz + 2.0 * u * fabs(cam->fy * yz) + u * fabs(cam->cy);
    err[2] = dZ;
    err[3] = dop;
    /* Jacobian and T = J W (2 x 3) */
    const double xzc = fmin(limx, fmax(-limx, xz)), yzc = fmin(limy, fmax(-limy, yz));
    const double dxzc = dxz + 3.0 * u * limx, dyzc = dyz + 3.0 * u * limy;
    const double J00 = cam->fx / Z, J02 = -cam->fx * xzc / Z, J11 = cam->fy / Z, J12 = -cam->fy * yzc / Z;
    const double dJ00 = fabs(J00) * (u + dZ / Z), dJ11 = fabs(J11) * (u + dZ / Z);
    const double dJ02 = cam->fx / Z * (dxzc + 2.0 * u * fabs(xzc)) + fabs(J02) * dZ / Z;
    const double dJ12 = cam->fy / Z * (dyzc + 2.0 * u * fabs(yzc)) + fabs(J12) * dZ / Z;
    double Tm[6], dTm[6];
    for (int j = 0; j < 3; j++) {
        Tm[j] = J00 * R[j] + J02 * R[6 + j];
        dTm[j] = dJ00 * fabs(R[j]) + dJ02 * fabs(R[6 + j]) + 2.0 * u * (fabs(J00 * R[j]) + fabs(J02 * R[6 + j]));
        Tm[3 + j] = J11 * R[3 + j] + J12 * R[6 + j];
        dTm[3 + j] = dJ11 * fabs(R[3 + j]) + dJ12 * fabs(R[6 + j]) + 2.0 * u * (fabs(J11 * R[3 + j]) + fabs(J12 * R[6 + j]));
    }
    /* F = (the factor Sigma' is built from) and its bound: TM = Tm M, or TS = Tm Sigma3D */
    double F[6], dF[6], G[6], dG[6];   /* Sigma'_rq - 0.3 d_rq = sum_k F_rk G_qk */
    if (sc->cov3d) {
        const double *c = sc->cov3d + 6 * (size_t)i;
        const double S3[9] = {c[0], c[1], c[2], c[1], c[3], c[4], c[2], c[4], c[5]};
        double dS3[9];
        if (ie) {
            const double *d = ie + 4;
            const double t9[9] = {d[0], d[1], d[2], d[1], d[3], d[4], d[2], d[4], d[5]};
            memcpy(dS3, t9, sizeof t9);
        } else {
            for (int k = 0; k < 9; k++) dS3[k] = u * fabs(S3[k]);
        }
        for (int r = 0; r < 2; r++)
            for (int k = 0; k < 3; k++) {
                double v = 0.0, dv = 0.0, mag = 0.0;
                for (int j = 0; j < 3; j++) {
                    v += Tm[3 * r + j] * S3[3 * j + k];
                    dv += dTm[3 * r + j] * fabs(S3[3 * j + k]) + fabs(Tm[3 * r + j]) * dS3[3 * j + k];
                    mag += fabs(Tm[3 * r + j] * S3[3 * j + k]);
                }
                F[3 * r + k] = v;
                dF[3 * r + k] = dv + 3.0 * u * mag;
            }
        memcpy(G, Tm, sizeof G);
        memcpy(dG, dTm, sizeof dG);
    } else {
        const double *q = sc->quats + 4 * (size_t)i;
        const double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        const double qn[4] = {q[0] / nq, q[1] / nq, q[2] / nq, q[3] / nq};
        double Rq[9], M[9], dM[9];
        orc_quat_to_rot(qn, Rq);
        for (int r = 0; r < 3; r++)
            for (int k = 0; k < 3; k++) {
                const double s = exp(sc->log_scales[3 * (size_t)i + k]);
                M[3 * r + k] = Rq[3 * r + k] * s;
                dM[3 * r + k] = (24.0 * u + (E + u) * fabs(Rq[3 * r + k])) * s;
            }
        for (int r = 0; r < 2; r++)
            for (int k = 0; k < 3; k++) {
                double v = 0.0, dv = 0.0, mag = 0.0;
                for (int j = 0; j < 3; j++) {
                    v += Tm[3 * r + j] * M[3 * j + k];
                    dv += dTm[3 * r + j] * fabs(M[3 * j + k]) + fabs(Tm[3 * r + j]) * dM[3 * j + k];
                    mag += fabs(Tm[3 * r + j] * M[3 * j + k]);
                }
                F[3 * r + k] = v;
                dF[3 * r + k] = dv + 3.0 * u * mag;
            }
        memcpy(G, F, sizeof G);
        memcpy(dG, dF, sizeof dG);
    }
    const int rr[3] = {0, 0, 1}, qq[3] = {0, 1, 1};
    for (int e = 0; e < 3; e++) {
        const int r = rr[e], q2 = qq[e];
        double dv = 0.0, mag = (r == q2) ? ORC_DILATION : 0.0;
        for (int k = 0; k < 3; k++) {
            dv += dF[3 * r + k] * fabs(G[3 * q2 + k]) + fabs(F[3 * r + k]) * dG[3 * q2 + k];
            mag += fabs(F[3 * r + k] * G[3 * q2 + k]);
        }
        err[4 + e] = dv + 4.0 * u * mag;
    }
}

/* ---------------------------------------------------------------------------
 * orc_preprocess: per Gaussian, the dynamic 2D Gaussian at time t.
 *   tau = t - mu_t;  mu(t) = mu + tau V3D                       (Eq. 7)
 *   o_hat = sigmoid(logit) exp(-tau^2 / (2 s_t^2)), s_t = e^{log s_t}   (Eq. 6-7)
 *   X = R_cam mu(t) + T_cam = P_view + tau V_view               (Eq. 9-11, 15)
 *   (u, v) = (fx X/Z + cx, fy Y/Z + cy)                          (Eq. 12)
 *   J = d(u,v)/dX at X (x/z, y/z clamped)                       (Eq. 14)
 *   Sigma' = J R_cam Sigma3D R_cam^T J^T + 0.3 I                (Eq. 16)
 *   conic = Sigma'^{-1}; colour = max(0, SH . Y(dir) + 0.5)
 * temporal_cull: also drop o_hat < 1/255 (lossless: alpha < 1/255 everywhere).
 *
 * With out->err (N x 16) it also records, per Gaussian, what an FP32
 * evaluation makes of it, for the slack of orc_render_pixels:
 *   [0..3]  u, v, Z, o_hat of the binary32 footprint (project_f32 on the
 *           binary32 inputs), [4..6] the exact inverse (a, b, c) of its
 *           binary32 Sigma', [7] mode: 0 both draw it, 1 the definition draws
 *           it and binary32 culls it (near plane, temporal opacity), 2 binary32
 *           draws it and the definition does not (drawn stays 0, but the
 *           FP64 2D Gaussian is filled in so the renderer can see its pairs);
 *   [8..14] a-priori bounds (fp32_bounds) -- cov3d mode only, where no
 *           binary32 footprint is evaluated ([0..6] then repeat the FP64
 *           values); zero otherwise;  [15] 1 if [0..6] come from binary32.
 * ------------------------------------------------------------------------- */
void orc_preprocess(const orc_scene *sc, const orc_camera *cam, double t, int temporal_cull, orc_g2d *out) {
    const int n = sc->n, ncoef = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    double campos[3];
    cam_position(cam, campos);
    const double limx = ORC_JAC_CLAMP * (0.5 * cam->width) / cam->fx;
    const double limy = ORC_JAC_CLAMP * (0.5 * cam->height) / cam->fy;
    orc_camera_f32 cam32;
    for (int k = 0; k < 9; k++) cam32.R[k] = (float)cam->R[k];
    for (int k = 0; k < 3; k++) cam32.T[k] = (float)cam->T[k];
    cam32.fx = (float)cam->fx; cam32.fy = (float)cam->fy; cam32.cx = (float)cam->cx; cam32.cy = (float)cam->cy;
    cam32.width = cam->width; cam32.height = cam->height;
    cam32.near = (float)cam->near;
    const int with_f32 = out->err != NULL && sc->cov3d == NULL;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        out->drawn[i] = 0;
        double *err = out->err ? out->err + 16 * (size_t)i : NULL;
        if (err) memset(err, 0, 16 * sizeof(double));
        double tau = t - sc->t_mean[i];
        double m[3], X[3];
        for (int j = 0; j < 3; j++) m[j] = sc->means[3 * (size_t)i + j] + tau * sc->velocity[3 * (size_t)i + j];
        for (int r = 0; r < 3; r++)
            X[r] = cam->R[3 * r + 0] * m[0] + cam->R[3 * r + 1] * m[1] + cam->R[3 * r + 2] * m[2] + cam->T[r];
        double o = 1.0 / (1.0 + exp(-sc->opacity_logit[i]));
        double st = exp(sc->log_t_scale[i]);
        double oh = o * exp(-0.5 * tau * tau / (st * st));
        out->opacity_t[i] = oh;
        out->depth[i] = X[2];
        int f32_draws = -1, mode = 0;
        orc_fp32 f;
        if (with_f32) {
            orc_param_f32 P;
            for (int j = 0; j < 3; j++) {
                P.mu[j] = (float)sc->means[3 * (size_t)i + j];
                P.vel[j] = (float)sc->velocity[3 * (size_t)i + j];
                P.ls[j] = (float)sc->log_scales[3 * (size_t)i + j];
            }
            for (int j = 0; j < 4; j++) P.q[j] = (float)sc->quats[4 * (size_t)i + j];
            P.tm = (float)sc->t_mean[i];
            P.lt = (float)sc->log_t_scale[i];
            P.lg = (float)sc->opacity_logit[i];
            f32_draws = project_f32(&P, &cam32, (float)t, &f) == 3 && isfinite(f.u) && isfinite(f.v);
        }
        const int def_draws = X[2] > cam->near && (!temporal_cull || oh >= ORC_ALPHA_MIN);
        if (!def_draws) {
            /* binary32 draws what the definition culls: only within its reach of the thresholds */
            if (f32_draws != 1 || !(X[2] > 0.5 * cam->near)) continue;
            mode = 2;
        } else if (f32_draws == 0) {
            mode = 1;
        }
        double Z = X[2];
        double xz = X[0] / Z, yz = X[1] / Z;
        double xzc = fmin(limx, fmax(-limx, xz)), yzc = fmin(limy, fmax(-limy, yz));
        double J[6] = {cam->fx / Z, 0.0, -cam->fx * xzc / Z, 0.0, cam->fy / Z, -cam->fy * yzc / Z};
        double S3[9], Wt[9], A[9], Sc[9];
        cov3d_of(sc, i, S3);
        matmul3(cam->R, S3, A);
        transpose3(cam->R, Wt);
        matmul3(A, Wt, Sc); /* Sigma_cam = W Sigma3D W^T */
        double JS[6];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 3; c++) JS[3 * r + c] = J[3 * r] * Sc[c] + J[3 * r + 1] * Sc[3 + c] + J[3 * r + 2] * Sc[6 + c];
        double c00 = JS[0] * J[0] + JS[1] * J[1] + JS[2] * J[2] + ORC_DILATION;
        double c01 = JS[0] * J[3] + JS[1] * J[4] + JS[2] * J[5];
        double c11 = JS[3] * J[3] + JS[4] * J[4] + JS[5] * J[5] + ORC_DILATION;
        double det = c00 * c11 - c01 * c01;
        if (!(det > 0.0)) continue;
        out->cov2d[3 * (size_t)i + 0] = c00;
        out->cov2d[3 * (size_t)i + 1] = c01;
        out->cov2d[3 * (size_t)i + 2] = c11;
        out->conic[3 * (size_t)i + 0] = c11 / det;
        out->conic[3 * (size_t)i + 1] = -c01 / det;
        out->conic[3 * (size_t)i + 2] = c00 / det;
        double mid = 0.5 * (c00 + c11);
        out->lambda_max[i] = mid + sqrt(fmax(0.1, mid * mid - det));
        out->u[i] = cam->fx * xz + cam->cx;
        out->v[i] = cam->fy * yz + cam->cy;
        /* view direction of the colour: the time-shifted mean, or (colour cache) the static one */
        const double *cm = sc->colour_static ? sc->means + 3 * (size_t)i : m;
        double d[3] = {cm[0] - campos[0], cm[1] - campos[1], cm[2] - campos[2]};
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        d[0] /= dn; d[1] /= dn; d[2] /= dn;
        double Y[16];
        orc_sh_basis(d, sc->sh_degree, Y);
        for (int ch = 0; ch < 3; ch++) {
            double s = 0.0;
            for (int k = 0; k < ncoef; k++) s += sc->sh[((size_t)i * ncoef + k) * 3 + ch] * Y[k];
            out->rgb[3 * (size_t)i + ch] = fmax(0.0, s + 0.5);
        }
        if (err) {
            if (f32_draws == 1) {
                const double s00 = f.s00, s01 = f.s01, s11 = f.s11;
                const double dt = s00 * s11 - s01 * s01;
                err[0] = f.u; err[1] = f.v; err[2] = f.Z; err[3] = f.oh;
                err[4] = s11 / dt; err[5] = -s01 / dt; err[6] = s00 / dt;
                err[15] = 1.0;
            } else {
                err[0] = out->u[i]; err[1] = out->v[i]; err[2] = Z; err[3] = oh;
                err[4] = out->conic[3 * (size_t)i]; err[5] = out->conic[3 * (size_t)i + 1];
                err[6] = out->conic[3 * (size_t)i + 2];
                if (!with_f32) fp32_bounds(sc, cam, i, tau, m, X, limx, limy, st, err + 8);
            }
            err[7] = mode;
        }
        out->drawn[i] = mode == 2 ? 0 : 1;
    }
}

/* ---------------------------------------------------------------------------
 * orc_render_pixels: per pixel (centre x+0.5, y+0.5), brute force over every
 * drawn Gaussian (Eq. 1 evaluated with the 2D conic, Eq. 4 compositing):
 *   p = -1/2 (a dx^2 + c dy^2) - b dx dy; skip p > 0;
 *   alpha = min(0.99, o_hat e^p); skip alpha < 1/255;
 *   sort the kept by (depth, index); T = 1;
 *   for each: stop if T (1 - alpha) < 1e-4; C += alpha T c; T *= 1 - alpha.
 *   out = C + T bg.
 * Besides the colour it returns T, the number of blended Gaussians, a per-pixel
 * slack and Tw.  The slack is the most an FP32 renderer of the same definition
 * may move the colour because one of its discrete decisions goes the other way;
 * it is 0 on a pixel where no decision can.  An FP32 renderer starts from the
 * binary32 footprint of each Gaussian (g->err, see orc_preprocess), and its
 * blend adds only its own rounding (pair_window); so a decision is near when
 *   alpha vs 1/255:  the FP64 alpha and the binary32 footprint's alpha widened
 *                    by the window lie on different sides of 1/255 (or the
 *                    footprint is culled on one side only: mode 1 / 2);
 *   stop T (1 - alpha) vs 1e-4: the same with T of the footprint's alphas,
 *                    widened by the windows accumulated along the pixel (Tw);
 *   p vs 0:          |p| within the evaluation part of the window;
 *   depth order:     the binary32 depth keys (with the index as tie-break, the
 *                    order of the tile lists) order the pixel's kept Gaussians
 *                    differently from FP64 depth: the pixel is re-composited in
 *                    key order and the difference is added; in cov3d mode
 *                    (a-priori bounds) |z_i - z_j| <= ORC_SAFETY (dz_i + dz_j)
 *                    for consecutive blended ones instead.
 * Each near alpha decision adds 2 alpha T max c (1 + window), each near stop
 * T alpha max c + 2e-4 max c, each possibly swapped pair in cov3d mode
 * 2 alpha_1 alpha_2 max c T -- the size of the jump its flip causes (Eq. 4).
 * Tw bounds |T_fp32 / T - 1| on a pixel without near decisions.  Needs g->err.
 * ------------------------------------------------------------------------- */
#define ORC_SAFETY 1.25
#define ORC_LN2 0.69314718055994531
#define ORC_LOG2E 1.4426950408889634

/* Relative window of an FP32 blend's alpha around the alpha of Gaussian i's binary32 footprint
 * at pixel offset (dx, dy) = (u - x, v - y) (footprint values), p the footprint's exponent:
 *   the conic from the binary32 Sigma' (accurate 2x2 determinant, one division, one
 *   product: 4u relative), scaled by log2(e)/2 (3u) and the quadratic form (offsets
 *   rounded; two products and three FMAs or products and sums: 6u) on
 *   Q = 1/2 (|a| dx^2 + |c| dy^2) + |b dx dy|;
 *   q = log2(e) p + log2(o_hat) (u |q|; log2 within ORC_FN_REL |L|); 2^q within 16u;
 *   in cov3d mode also the a-priori bounds [8..14]: the mean within (du, dv),
 *   Sigma' within (ds00, ds01, ds11) (dp = 1/2 y^T dSigma' y, y = Sigma'^-1 d) and o_hat.
 * *w_nonpos: the part that can make an FP32 p positive (the evaluation and, in cov3d mode,
 * Sigma'; a displaced mean cannot: p is a negative definite form of the offset). */
static double pair_window(const double *e, double dx, double dy, double p, double *w_nonpos) {
    const double u = ORC_U;
    const double a = e[4], b = e[5], c = e[6];
    const double Q = 0.5 * (fabs(a) * dx * dx + fabs(c) * dy * dy) + fabs(b * dx * dy);
    const double dp_eval = 13.0 * u * Q + u * fabs(p);
    const double gx = a * dx + b * dy, gy = b * dx + c * dy;
    const double dp_pos = fabs(gx) * e[8] + fabs(gy) * e[9];
    const double dp_cov = 0.5 * (gx * gx * e[12] + 2.0 * fabs(gx * gy) * e[13] + gy * gy * e[14]);
    const double L = log2(e[3]);
    const double q = ORC_LOG2E * p + L;
    const double w = dp_eval + dp_pos + dp_cov + ORC_LN2 * (u * fabs(q) + ORC_FN_REL * fabs(L)) + e[11] + 16.0 * u;
    if (w_nonpos) *w_nonpos = ORC_SAFETY * (dp_eval + dp_cov);
    return ORC_SAFETY * w;
}

typedef struct {
    double depth, key;       /* FP64 depth; binary32 depth key */
    int32_t idx;
    double alpha;            /* FP64 alpha, negative when the definition skips the pair */
    double alpha_f;          /* the binary32 footprint's alpha (0 when binary32 culls the Gaussian) */
    double w;
    int near_alpha;
} orc_cand;

static int cand_cmp(const void *pa, const void *pb) {
    const orc_cand *a = (const orc_cand *)pa, *b = (const orc_cand *)pb;
    if (a->depth < b->depth) return -1;
    if (a->depth > b->depth) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

static int cand_key_cmp(const void *pa, const void *pb) {
    const orc_cand *a = (const orc_cand *)pa, *b = (const orc_cand *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* Eq. 4 over the kept candidates in the given order (stop rule included): colour and T. */
static double composite(const orc_g2d *g, const orc_cand *c, size_t nc, double C[3]) {
    double T = 1.0;
    C[0] = C[1] = C[2] = 0.0;
    for (size_t k = 0; k < nc; k++) {
        const double alpha = c[k].alpha;
        if (alpha < 0.0) continue;
        const double test = T * (1.0 - alpha);
        if (test < ORC_T_MIN) break;
        const double *col = g->rgb + 3 * (size_t)c[k].idx;
        for (int ch = 0; ch < 3; ch++) C[ch] += alpha * T * col[ch];
        T = test;
    }
    return T;
}

/* The candidates of the pixel at (x, y): every drawn (or binary32-drawn) Gaussian whose FP64
 * alpha passes, or whose decision is near (see orc_render_pixels), sorted by (depth, index).
 * *cand / *alt grow as needed (alt is scratch of the same capacity). */
static size_t pixel_candidates(const orc_g2d *g, const int32_t *ids, int nd, double x, double y,
                               orc_cand **cand, orc_cand **alt, size_t *cap) {
    size_t nc = 0;
    for (int k = 0; k < nd; k++) {
        const int i = ids[k];
        const double *e = g->err + 16 * (size_t)i;
        const double dx = g->u[i] - x, dy = g->v[i] - y;
        const double a = g->conic[3 * (size_t)i], b = g->conic[3 * (size_t)i + 1], c = g->conic[3 * (size_t)i + 2];
        const double p = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
        const double raw = g->opacity_t[i] * exp(fmin(p, 0.0));
        if (raw < 0.25 * ORC_ALPHA_MIN) continue;   /* no window reaches a factor 4 */
        const int mode = (int)e[7];
        /* the binary32 footprint's alpha and the blend's window around it */
        const double fx = e[0] - x, fy = e[1] - y;
        const double pf = -0.5 * (e[4] * fx * fx + e[6] * fy * fy) - e[5] * fx * fy;
        double wnp;
        const double w = pair_window(e, fx, fy, pf, &wnp);
        const double af = mode == 1 ? 0.0 : fmin(ORC_ALPHA_MAX, e[3] * exp(fmin(pf, 0.0)));
        const double gpu_hi = af * (1.0 + w);
        const double gpu_lo = (mode == 1 || pf > -wnp) ? 0.0 : af * (1.0 - w);
        const double alpha = fmin(ORC_ALPHA_MAX, raw);
        const int pass = g->drawn[i] && p <= 0.0 && alpha >= ORC_ALPHA_MIN;
        const int near_alpha = pass ? (gpu_lo < ORC_ALPHA_MIN) : (gpu_hi >= ORC_ALPHA_MIN);
        if (!pass && !near_alpha) continue;
        if (nc == *cap) {
            *cap *= 2;
            *cand = (orc_cand *)realloc(*cand, sizeof(orc_cand) * *cap);
            *alt = (orc_cand *)realloc(*alt, sizeof(orc_cand) * *cap);
        }
        orc_cand *cd = *cand + nc;
        cd->depth = g->depth[i];
        cd->key = e[2];
        cd->idx = i;
        cd->alpha = pass ? alpha : -alpha;
        cd->alpha_f = af;
        cd->w = w;
        cd->near_alpha = near_alpha;
        nc++;
    }
    qsort(*cand, nc, sizeof(orc_cand), cand_cmp);
    return nc;
}

void orc_render_pixels(const orc_g2d *g, int n, const orc_camera *cam, const double bg[3],
                       int64_t npix, const int32_t *px, const int32_t *py,
                       double *out_rgb, double *out_T, int32_t *out_ncontrib, double *out_slack,
                       double *out_Tw) {
    /* compact list of the Gaussians the definition or binary32 draws */
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    int nd = 0;
    for (int i = 0; i < n; i++)
        if (g->drawn[i] || g->err[16 * (size_t)i + 7] == 2.0) ids[nd++] = i;
    const int64_t W = cam->width;
    if (npix < 0) npix = (int64_t)cam->width * cam->height;
#pragma omp parallel
    {
        size_t cap = 1024;
        orc_cand *cand = (orc_cand *)malloc(sizeof(orc_cand) * cap);
        orc_cand *alt = (orc_cand *)malloc(sizeof(orc_cand) * cap);
#pragma omp for schedule(dynamic, 8)
        for (int64_t q = 0; q < npix; q++) {
            double x = (px ? px[q] : (int32_t)(q % W)) + 0.5;
            double y = (py ? py[q] : (int32_t)(q / W)) + 0.5;
            double slack = 0.0;
            const size_t nc = pixel_candidates(g, ids, nd, x, y, &cand, &alt, &cap);
            double T = 1.0, Tf = 1.0, C[3] = {0, 0, 0}, wT = 0.0, cmax = 0.0;
            int32_t ncontrib = 0;
            for (size_t k = 0; k < nc; k++) {
                const double *c = g->rgb + 3 * (size_t)cand[k].idx;
                double cm = fmax(c[0], fmax(c[1], c[2]));
                if (cm > cmax) cmax = cm;
            }
            int32_t last = -1, all_f32 = 1;
            int64_t stop_at = (int64_t)nc;   /* position of the candidate that stops the pixel */
            double prev_depth = -1.0, prev_alpha = 0.0, prev_dz = 0.0;
            for (size_t k = 0; k < nc; k++) {
                const double *e = g->err + 16 * (size_t)cand[k].idx;
                const double alpha = cand[k].alpha, af = cand[k].alpha_f;
                if (e[15] == 0.0) all_f32 = 0;
                if (cand[k].near_alpha) slack += 2.0 * fmax(fabs(alpha), af) * (1.0 + cand[k].w) * cmax * T + 1e-7;
                if (alpha < 0.0) continue; /* not blended in FP64 */
                /* cov3d mode: nearly equal depths may swap */
                if (e[15] == 0.0 && last >= 0 &&
                    fabs(cand[k].depth - prev_depth) <= ORC_SAFETY * (e[10] + prev_dz))
                    slack += 2.0 * prev_alpha * alpha * cmax * (T / (1.0 - prev_alpha)) + 1e-7;
                const double test = T * (1.0 - alpha), test_f = Tf * (1.0 - af);
                /* accumulated FP32 relative error of T (two roundings per step), and the stop decision */
                const double wstop = wT + cand[k].w * af / (1.0 - af) + 2.0 * ORC_U;
                const int stop = test < ORC_T_MIN;
                const int near_stop = stop ? (test_f * (1.0 + wstop) >= ORC_T_MIN) : (test_f * (1.0 - wstop) < ORC_T_MIN);
                if (near_stop) slack += T * alpha * cmax + 2.0 * ORC_T_MIN * cmax;
                if (stop) {
                    stop_at = (int64_t)k;
                    break;
                }
                const double *c = g->rgb + 3 * (size_t)cand[k].idx;
                for (int ch = 0; ch < 3; ch++) C[ch] += alpha * T * c[ch];
                T = test;
                Tf = test_f;
                wT = wstop;
                ncontrib++;
                last = (int32_t)k;
                prev_depth = cand[k].depth;
                prev_alpha = alpha;
                prev_dz = e[10];
            }
            if (all_f32) {
                /* the order of the binary32 depth keys (the tile lists' order): the kept
                 * Gaussians up to the one that stops the pixel (stop_at) must come in key
                 * order, and every later one after them, else the key order composites a
                 * different sequence */
                int sorted = 1;
                double pk = -INFINITY;
                int32_t pi = -1;
                for (size_t k = 0; k < nc && sorted; k++) {
                    if (cand[k].alpha < 0.0) continue;
                    const int after = (int64_t)k > stop_at;
                    if (cand[k].key < pk || (cand[k].key == pk && cand[k].idx < pi)) sorted = 0;
                    if (!after) { pk = cand[k].key; pi = cand[k].idx; }
                }
                if (!sorted) {
                    double C2[3];
                    memcpy(alt, cand, nc * sizeof(orc_cand));
                    qsort(alt, nc, sizeof(orc_cand), cand_key_cmp);
                    composite(g, alt, nc, C2);
                    slack += fmax(fabs(C2[0] - C[0]), fmax(fabs(C2[1] - C[1]), fabs(C2[2] - C[2])));
                }
            }
            for (int ch = 0; ch < 3; ch++) out_rgb[3 * q + ch] = C[ch] + T * bg[ch];
            if (out_T) out_T[q] = T;
            if (out_ncontrib) out_ncontrib[q] = ncontrib;
            if (out_slack) out_slack[q] = slack;
            if (out_Tw) out_Tw[q] = wT + fabs(Tf - T) / T;
        }
        free(cand);
        free(alt);
    }
    free(ids);
}

/* The per-pair quantities of orc_render_pixels for m given (Gaussian, pixel) pairs:
 * out[5 k ..] = {p, alpha = o_hat e^min(p, 0) (FP64, unclamped), p and alpha of the binary32
 * footprint, the blend's relative window around the latter}. */
void orc_pair_windows(const orc_g2d *g, int64_t m, const int32_t *gid, const int32_t *px, const int32_t *py,
                      double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < m; k++) {
        const int i = gid[k];
        const double *e = g->err + 16 * (size_t)i;
        const double x = px[k] + 0.5, y = py[k] + 0.5;
        const double dx = g->u[i] - x, dy = g->v[i] - y;
        const double *cn = g->conic + 3 * (size_t)i;
        const double p = -0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy;
        const double fx = e[0] - x, fy = e[1] - y;
        const double pf = -0.5 * (e[4] * fx * fx + e[6] * fy * fy) - e[5] * fx * fy;
        out[5 * k + 0] = p;
        out[5 * k + 1] = g->opacity_t[i] * exp(fmin(p, 0.0));
        out[5 * k + 2] = pf;
        out[5 * k + 3] = e[3] * exp(fmin(pf, 0.0));
        out[5 * k + 4] = pair_window(e, fx, fy, pf, NULL);
    }
}

/* ---------------------------------------------------------------------------
 * orc_bin_f32: FP32 mirror of the binning (per Gaussian: depth key bits,
 * radius, tile rectangle, tile count) on top of project_f32, in the same
 * fixed operation order as the GPU preprocess, so that tile/key lists can be
 * compared bit for bit:
 *   mid = 0.5*(s00 + s11); lam = mid + sqrtf(max(0.1, mid*mid - det))
 *   r = (int) ceilf(3.33 * sqrtf(lam))   (the 2D Gaussian's radius)
 *   cull unless u, v finite
 *   k2 = ((2*log(255*o_hat))*1.0008) + 0.0008;  rx = ceilf(sqrtf(k2*s00)), ry = ceilf(sqrtf(k2*s11))
 *   (bounding box of d^T Sigma'^-1 d <= k2: outside it o_hat e^p < 1/255)
 *   x0 = floorf((u - rx)/tile), x1 = floorf((u + rx)/tile),
 *   cull if x1 < 0 or x0 > tiles_x - 1, then clamp to [0, tiles_x-1] (same in y with ry)
 *   column cuts (only when `trim` is set; otherwise every column keeps its h
 *   rows), for rectangle columns c = x0 + j, j < 8 (ex = sqrtf(k2*s00),
 *   ey = sqrtf(k2*s11), q2 = k2*s00, xl = (s01*ey)/s11, tl = tile - 0.5):
 *     a = max(((c*tile) + 0.5) - u, -ex);  b = min(min((c*tile) + tl, W - 0.5) - u, ex)
 *     a > b (the column's pixel centres miss the ellipse): cut_t = min(h, 15),
 *       cut_b = min(h - cut_t, 15)
 *     else xt = min(max(-xl, a), b), xb = min(max(xl, a), b), i00 = 1/s00
 *       lo = ((v + ((s01*xt) - sqrtf(max(0, det*(q2 - xt*xt))))*i00) - 1/64) - tl
 *       hi = ((v + ((s01*xb) + sqrtf(max(0, det*(q2 - xb*xb))))*i00) + 1/64) - 0.5
 *       cut_t = clamp(ceilf(lo/tile) - y0, 0, 15), cut_b = clamp(y1 - floorf(hi/tile), 0, 15)
 *     (xt, xb: abscissae of the ellipse's top and bottom points clamped to the
 *     column; the column keeps the tile rows whose pixel-centre rows meet
 *     [lo + tl, hi + 0.5]); trims byte j = cut_t | cut_b << 4
 *   tiles = sum over columns of max(0, h - cut_t - cut_b) (columns from the
 *   9th on keep all h rows); culled if 0; depth key = bits of Z
 * Every operation is correctly rounded (exp and log are the explicit methods
 * above), so every decision is the same on any IEEE machine and no Gaussian
 * needs excluding from the comparison.  A culled Gaussian has depth key
 * 0xFFFFFFFF and 0 tiles.
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t n, sh_degree;
    const float *means, *t_mean, *velocity, *log_scales, *log_t_scale, *quats, *opacity_logit;
} orc_scene_f32;

static void param_f32(const orc_scene_f32 *sc, int i, orc_param_f32 *P) {
    for (int j = 0; j < 3; j++) {
        P->mu[j] = sc->means[3 * (size_t)i + j];
        P->vel[j] = sc->velocity[3 * (size_t)i + j];
        P->ls[j] = sc->log_scales[3 * (size_t)i + j];
    }
    for (int j = 0; j < 4; j++) P->q[j] = sc->quats[4 * (size_t)i + j];
    P->tm = sc->t_mean[i];
    P->lt = sc->log_t_scale[i];
    P->lg = sc->opacity_logit[i];
}

void orc_bin_f32(const orc_scene_f32 *sc, const orc_camera_f32 *cam, float t, int32_t tile, int32_t trim,
                 uint32_t *depth_key, int32_t *radius, int32_t *rect /* N x 4: x0,x1,y0,y1 */,
                 uint32_t *tiles_touched, uint64_t *trims, float *uv /* N x 2, may be NULL */,
                 float *foot /* N x 4: o_hat, Sigma'_00, Sigma'_01, Sigma'_11; may be NULL */) {
    const int n = sc->n;
    const int32_t tiles_x = (cam->width + tile - 1) / tile, tiles_y = (cam->height + tile - 1) / tile;
    const float tilef = (float)tile;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        depth_key[i] = 0xFFFFFFFFu;
        radius[i] = 0;
        rect[4 * (size_t)i + 0] = rect[4 * (size_t)i + 1] = rect[4 * (size_t)i + 2] = rect[4 * (size_t)i + 3] = 0;
        tiles_touched[i] = 0;
        trims[i] = 0;
        if (uv) { uv[2 * (size_t)i] = 0.f; uv[2 * (size_t)i + 1] = 0.f; }
        if (foot) memset(foot + 4 * (size_t)i, 0, 4 * sizeof(float));
        orc_param_f32 P;
        orc_fp32 f;
        param_f32(sc, i, &P);
        if (project_f32(&P, cam, t, &f) != 3) continue;
        const float u = f.u, v = f.v, Z = f.Z, oh = f.oh, s00 = f.s00, s01 = f.s01, s11 = f.s11, det = f.det;
        float mid = 0.5f * (s00 + s11);
        float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
        float rf = ceilf(3.33f * sqrtf(lam));
        if (!(isfinite(u) && isfinite(v))) continue;
        float k2 = ((2.0f * orc_logf(255.0f * oh)) * 1.0008f) + 0.0008f;
        float ex = sqrtf(k2 * s00), ey = sqrtf(k2 * s11);
        float rx = ceilf(ex), ry = ceilf(ey);
        float fx0 = floorf((u - rx) / tilef), fx1 = floorf((u + rx) / tilef);
        float fy0 = floorf((v - ry) / tilef), fy1 = floorf((v + ry) / tilef);
        if (!(fx1 >= 0.0f) || !(fx0 <= (float)(tiles_x - 1))) continue;
        if (!(fy1 >= 0.0f) || !(fy0 <= (float)(tiles_y - 1))) continue;
        int32_t x0 = (int32_t)fmaxf(fx0, 0.0f), x1 = (int32_t)fminf(fx1, (float)(tiles_x - 1));
        int32_t y0 = (int32_t)fmaxf(fy0, 0.0f), y1 = (int32_t)fminf(fy1, (float)(tiles_y - 1));
        /* column cuts */
        const int32_t h = y1 - y0 + 1;
        const float q2 = k2 * s00, xl = (s01 * ey) / s11, i00 = 1.0f / s00;
        const float tl = tilef - 0.5f, wl = (float)cam->width - 0.5f;
        uint64_t tw = 0;
        int64_t kept = 0;
        for (int32_t c = x0; c <= x1; c++) {
            const int32_t j = c - x0;
            int32_t cut_t = 0, cut_b = 0;
            if (trim && j < 8) {
                const float left = ((float)c * tilef + 0.5f) - u;
                const float right = fminf((float)c * tilef + tl, wl) - u;
                const float a = fmaxf(left, -ex), b = fminf(right, ex);
                if (!(a <= b)) {
                    cut_t = h < 15 ? h : 15;
                    cut_b = h - cut_t < 15 ? h - cut_t : 15;
                } else {
                    const float xt = fminf(fmaxf(-xl, a), b), xb = fminf(fmaxf(xl, a), b);
                    const float lo = ((v + ((s01 * xt) - sqrtf(fmaxf(0.0f, det * (q2 - xt * xt)))) * i00) - 0.015625f) - tl;
                    const float hi = ((v + ((s01 * xb) + sqrtf(fmaxf(0.0f, det * (q2 - xb * xb)))) * i00) + 0.015625f) - 0.5f;
                    const float flo = lo / tilef, fhi = hi / tilef;
                    cut_t = (int32_t)fminf(fmaxf(ceilf(flo) - (float)y0, 0.0f), 15.0f);
                    cut_b = (int32_t)fminf(fmaxf((float)y1 - floorf(fhi), 0.0f), 15.0f);
                }
                tw |= (uint64_t)(uint32_t)(cut_t | (cut_b << 4)) << (8 * j);
            }
            if (h - cut_t - cut_b > 0) kept += h - cut_t - cut_b;
        }
        if (kept == 0) continue;
        uint32_t bits;
        memcpy(&bits, &Z, 4);
        depth_key[i] = bits;
        radius[i] = (int32_t)rf;
        rect[4 * (size_t)i + 0] = x0; rect[4 * (size_t)i + 1] = x1;
        rect[4 * (size_t)i + 2] = y0; rect[4 * (size_t)i + 3] = y1;
        tiles_touched[i] = (uint32_t)kept;
        trims[i] = tw;
        if (uv) { uv[2 * (size_t)i] = u; uv[2 * (size_t)i + 1] = v; }
        if (foot) {
            foot[4 * (size_t)i + 0] = oh;
            foot[4 * (size_t)i + 1] = s00;
            foot[4 * (size_t)i + 2] = s01;
            foot[4 * (size_t)i + 3] = s11;
        }
    }
}

/* Emit the unsorted (tile, depth_bits, id) triples of all binned Gaussians in
 * index order, tiles of one Gaussian row-major (the rectangle less the column
 * cuts of orc_bin_f32); returns the count written. */
int64_t orc_emit_keys(int32_t n, const uint32_t *depth_key, const int32_t *rect, const uint64_t *trims,
                      const uint32_t *tiles_touched, int32_t tiles_x, int64_t cap, uint32_t *tile_out,
                      uint32_t *depth_out, uint32_t *id_out) {
    int64_t k = 0;
    for (int32_t i = 0; i < n; i++) {
        if (!tiles_touched[i]) continue;
        for (int32_t ty = rect[4 * (size_t)i + 2]; ty <= rect[4 * (size_t)i + 3]; ty++)
            for (int32_t tx = rect[4 * (size_t)i + 0]; tx <= rect[4 * (size_t)i + 1]; tx++) {
                const int32_t j = tx - rect[4 * (size_t)i + 0];
                if (j < 8) {
                    const uint32_t byte = (uint32_t)(trims[i] >> (8 * j)) & 0xFFu;
                    if (ty < rect[4 * (size_t)i + 2] + (int32_t)(byte & 15u) ||
                        ty > rect[4 * (size_t)i + 3] - (int32_t)(byte >> 4))
                        continue;
                }
                if (k < cap) {
                    tile_out[k] = (uint32_t)(ty * tiles_x + tx);
                    depth_out[k] = depth_key[i];
                    id_out[k] = (uint32_t)i;
                }
                k++;
            }
    }
    return k;
}

/* ---------------------------------------------------------------------------
 * orc_backward: FP64 adjoint of orc_preprocess + orc_render_pixels (full
 * frame, temporal cull on) for the loss L = sum(dl_drgb * image).
 *
 * Compositing (Eq. 4), back to front over each pixel's blended list with
 * G = dL/dC, B = the colour behind (starting at bg, B <- alpha c + (1-alpha) B):
 *   dL/dc_i = alpha_i T_i G,   dL/dalpha_i = T_i G.(c_i - B_{i+1})
 *   alpha = min(0.99, o_hat e^p): dalpha/dp = alpha, dalpha/do_hat = e^p
 *   (zero when the 0.99 clamp is active); p = -1/2(a dx^2 + c dy^2) - b dx dy.
 * Then per Gaussian, the chain of orc_preprocess in reverse:
 *   conic = Sigma'^-1 -> Sigma' = TM TM^T + 0.3 I -> TM = J W M ->
 *   J(X) (with the x/z, y/z clamp) and M = R(q/|q|) diag(e^ls);
 *   (u, v)(X); X = R_cam mu(t) + T_cam; mu(t) = mu + tau V; tau = t - mu_t;
 *   o_hat = sigmoid(logit) exp(-tau^2 / (2 e^(2 lst)));
 *   colour = max(0, SH . Y(d) + 0.5), d = (mu(t) - campos)/|mu(t) - campos|.
 * ------------------------------------------------------------------------- */
typedef struct {
    double *means, *t_mean, *velocity, *log_scales, *log_t_scale, *quats, *opacity_logit, *sh;
} orc_scene_grad;

/* d Y_k / d(x, y, z) of orc_sh_basis, treating x, y, z as independent. */
static void sh_basis_grad(const double d[3], int degree, double dY[16][3]) {
    const double pi = 3.14159265358979323846;
    double x = d[0], y = d[1], z = d[2];
    memset(dY, 0, sizeof(double) * 16 * 3);
    if (degree < 1) return;
    double c1 = sqrt(3.0 / (4.0 * pi));
    dY[1][1] = -c1;
    dY[2][2] = c1;
    dY[3][0] = -c1;
    if (degree < 2) return;
    double xx = x * x, yy = y * y, zz = z * z;
    double a = 0.5 * sqrt(15.0 / pi), b = 0.25 * sqrt(5.0 / pi), c = 0.25 * sqrt(15.0 / pi);
    dY[4][0] = a * y; dY[4][1] = a * x;
    dY[5][1] = -a * z; dY[5][2] = -a * y;
    dY[6][0] = -2.0 * b * x; dY[6][1] = -2.0 * b * y; dY[6][2] = 4.0 * b * z;
    dY[7][0] = -a * z; dY[7][2] = -a * x;
    dY[8][0] = 2.0 * c * x; dY[8][1] = -2.0 * c * y;
    if (degree < 3) return;
    double e = 0.25 * sqrt(35.0 / (2.0 * pi)), f = 0.5 * sqrt(105.0 / pi);
    double g = 0.25 * sqrt(21.0 / (2.0 * pi)), h = 0.25 * sqrt(7.0 / pi);
    double k = 0.25 * sqrt(105.0 / pi);
    dY[9][0] = -6.0 * e * x * y; dY[9][1] = -e * (3.0 * xx - 3.0 * yy);
    dY[10][0] = f * y * z; dY[10][1] = f * x * z; dY[10][2] = f * x * y;
    dY[11][0] = 2.0 * g * x * y; dY[11][1] = -g * (4.0 * zz - xx - 3.0 * yy); dY[11][2] = -8.0 * g * y * z;
    dY[12][0] = -6.0 * h * x * z; dY[12][1] = -6.0 * h * y * z; dY[12][2] = h * (6.0 * zz - 3.0 * xx - 3.0 * yy);
    dY[13][0] = -g * (4.0 * zz - 3.0 * xx - yy); dY[13][1] = 2.0 * g * x * y; dY[13][2] = -8.0 * g * x * z;
    dY[14][0] = 2.0 * k * x * z; dY[14][1] = -2.0 * k * y * z; dY[14][2] = k * (xx - yy);
    dY[15][0] = -e * (3.0 * xx - 3.0 * yy); dY[15][1] = 6.0 * e * x * y;
}

/* dR/dq for R = orc_quat_to_rot(q): dL/dq from dL/dR (both row-major). */
static void quat_rot_backward(const double q[4], const double dR[9], double dq[4]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    dq[0] = 2.0 * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    dq[1] = 2.0 * (y * dR[1] + z * dR[2] + y * dR[3] - 2.0 * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] -
                   2.0 * x * dR[8]);
    dq[2] = 2.0 * (-2.0 * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] -
                   2.0 * y * dR[8]);
    dq[3] = 2.0 * (-2.0 * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.0 * z * dR[4] + y * dR[5] + x * dR[6] +
                   y * dR[7]);
}

typedef struct { int32_t idx; double alpha, raw_alpha, T; } orc_blended;

/* The blended list of one pixel from its candidates in the given order (Eq. 4, stop before
 * blending once T (1 - alpha) < 1e-4).  flip >= 0: the candidate at that position goes the
 * other way (one the definition skips is blended with alpha_alt = max(its binary32 alpha,
 * |alpha|, 1/255)); stop_flip >= 0: the stop decision at that position goes the other way.
 * Returns the count; *stop_pos receives the position of the candidate that stopped it (nc if
 * none). */
static size_t pixel_blend_list(const orc_g2d *g, const orc_cand *c, size_t nc, double x, double y, int64_t flip,
                               int64_t stop_flip, orc_blended *bl, int64_t *stop_pos) {
    double T = 1.0;
    size_t nb = 0;
    *stop_pos = (int64_t)nc;
    for (size_t k = 0; k < nc; k++) {
        double alpha = c[k].alpha;
        if ((int64_t)k == flip)
            alpha = alpha < 0.0 ? fmax(fmax(c[k].alpha_f, -alpha), ORC_ALPHA_MIN) : -alpha;
        if (alpha < 0.0) continue;
        const double test = T * (1.0 - alpha);
        const int stop = (test < ORC_T_MIN) != ((int64_t)k == stop_flip);
        if (stop) {
            *stop_pos = (int64_t)k;
            break;
        }
        const int i = c[k].idx;
        const double *cn = g->conic + 3 * (size_t)i;
        const double dx = g->u[i] - x, dy = g->v[i] - y;
        const double p = -0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy;
        bl[nb].idx = i;
        bl[nb].alpha = alpha;
        bl[nb].raw_alpha = g->opacity_t[i] * exp(fmin(p, 0.0));
        bl[nb].T = T;
        nb++;
        T = test;
    }
    return nb;
}

/* The pixel's share of dL/d(u, v, a, b, c, o_hat, r, g, b) for each blended Gaussian,
 * back to front over its list with G = dL/dC and B the colour behind (from bg,
 * B <- alpha c + (1 - alpha) B):
 *   dL/dc_i = alpha_i T_i G,   dL/dalpha_i = T_i G.(c_i - B_{i+1});
 *   alpha = min(0.99, o_hat e^p): dalpha/dp = alpha, dalpha/do_hat = e^p (zero when the
 *   0.99 clamp is active); p = -1/2(a dx^2 + c dy^2) - b dx dy.
 * out[9 k ..] for list position k (overwritten). */
static void pixel_grad2d(const orc_g2d *g, const orc_blended *bl, size_t nb, const double G[3], const double bg[3],
                         double x, double y, double *out) {
    double B[3] = {bg[0], bg[1], bg[2]};
    for (size_t kk = nb; kk-- > 0;) {
        const int i = bl[kk].idx;
        const double alpha = bl[kk].alpha, Ti = bl[kk].T;
        const double *c = g->rgb + 3 * (size_t)i;
        double *gi = out + 9 * kk;
        for (int j = 0; j < 9; j++) gi[j] = 0.0;
        double dalpha = 0.0;
        for (int ch = 0; ch < 3; ch++) {
            gi[6 + ch] = alpha * Ti * G[ch];
            dalpha += Ti * G[ch] * (c[ch] - B[ch]);
            B[ch] = alpha * c[ch] + (1.0 - alpha) * B[ch];
        }
        if (bl[kk].raw_alpha > ORC_ALPHA_MAX) continue;   /* clamped: no gradient through alpha */
        const double *cn = g->conic + 3 * (size_t)i;
        const double dx = g->u[i] - x, dy = g->v[i] - y;
        const double dp = dalpha * alpha;
        gi[5] = dalpha * alpha / g->opacity_t[i];
        gi[0] = -dp * (cn[0] * dx + cn[1] * dy);
        gi[1] = -dp * (cn[1] * dx + cn[2] * dy);
        gi[2] = -0.5 * dp * dx * dx;
        gi[3] = -dp * dx * dy;
        gi[4] = -0.5 * dp * dy * dy;
    }
}

/* |alternative - base| of the per-Gaussian 2D gradients of one pixel, added to slk (N x 9). */
static void add_grad2d_change(const orc_blended *b0, const double *g0, size_t n0, const orc_blended *b1,
                              const double *g1, size_t n1, double *slk) {
    for (size_t k = 0; k < n0; k++) {
        const double *other = NULL;
        for (size_t j = 0; j < n1; j++)
            if (b1[j].idx == b0[k].idx) { other = g1 + 9 * j; break; }
        double *s = slk + 9 * (size_t)b0[k].idx;
        for (int c = 0; c < 9; c++) s[c] += fabs(g0[9 * k + c] - (other ? other[c] : 0.0));
    }
    for (size_t j = 0; j < n1; j++) {
        int found = 0;
        for (size_t k = 0; k < n0 && !found; k++) found = b0[k].idx == b1[j].idx;
        if (found) continue;
        double *s = slk + 9 * (size_t)b1[j].idx;
        for (int c = 0; c < 9; c++) s[c] += fabs(g1[9 * j + c]);
    }
}

/* Raw-parameter layout of one Gaussian's gradient: means 3, t_mean 1, velocity 3, log_scales 3,
 * log_t_scale 1, quats 4, opacity_logit 1, sh 3K. */
#define ORC_RAW_FIXED 16

/* dL/d(raw parameters) of Gaussian i from its dL/d(u, v, a, b, c, o_hat, r, g, b) G2: the chain
 * of orc_preprocess in reverse:
 *   conic = Sigma'^-1 -> Sigma' = TM TM^T + 0.3 I -> TM = J W M ->
 *   J(X) (with the x/z, y/z clamp) and M = R(q/|q|) diag(e^ls);
 *   (u, v)(X); X = R_cam mu(t) + T_cam; mu(t) = mu + tau V; tau = t - mu_t;
 *   o_hat = sigmoid(logit) exp(-tau^2 / (2 e^(2 lst)));
 *   colour = max(0, SH . Y(d) + 0.5), d = (mu(t) - campos)/|mu(t) - campos|. */
static void chain_raw(const orc_scene *sc, const orc_camera *cam, double t, const orc_g2d *g, int i,
                      const double G2[9], double *r) {
    const int ncoef = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    const double limx = ORC_JAC_CLAMP * (0.5 * cam->width) / cam->fx;
    const double limy = ORC_JAC_CLAMP * (0.5 * cam->height) / cam->fy;
    double campos[3];
    cam_position(cam, campos);
    double *gm = r, *gtm = r + 3, *gv = r + 4, *gls = r + 7, *glt = r + 10, *gq = r + 11, *glg = r + 15;
    double *gsh = r + ORC_RAW_FIXED;
    for (int j = 0; j < ORC_RAW_FIXED + 3 * ncoef; j++) r[j] = 0.0;
    /* ---- forward quantities */
    double tau = t - sc->t_mean[i];
    double m[3], X[3];
    for (int j = 0; j < 3; j++) m[j] = sc->means[3 * (size_t)i + j] + tau * sc->velocity[3 * (size_t)i + j];
    for (int rr = 0; rr < 3; rr++)
        X[rr] = cam->R[3 * rr] * m[0] + cam->R[3 * rr + 1] * m[1] + cam->R[3 * rr + 2] * m[2] + cam->T[rr];
    double Z = X[2], xz = X[0] / Z, yz = X[1] / Z;
    int clx = xz < -limx || xz > limx, cly = yz < -limy || yz > limy;
    double xzc = fmin(limx, fmax(-limx, xz)), yzc = fmin(limy, fmax(-limy, yz));
    double J[6] = {cam->fx / Z, 0.0, -cam->fx * xzc / Z, 0.0, cam->fy / Z, -cam->fy * yzc / Z};
    const double *q = sc->quats + 4 * (size_t)i;
    double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double qn[4] = {q[0] / nq, q[1] / nq, q[2] / nq, q[3] / nq};
    double Rq[9], s[3], M[9];
    orc_quat_to_rot(qn, Rq);
    for (int j = 0; j < 3; j++) s[j] = exp(sc->log_scales[3 * (size_t)i + j]);
    for (int a = 0; a < 3; a++)
        for (int c = 0; c < 3; c++) M[3 * a + c] = Rq[3 * a + c] * s[c];
    double Tm[6], TM[6];
    for (int a = 0; a < 2; a++)
        for (int c = 0; c < 3; c++) Tm[3 * a + c] = J[3 * a] * cam->R[c] + J[3 * a + 1] * cam->R[3 + c] + J[3 * a + 2] * cam->R[6 + c];
    for (int a = 0; a < 2; a++)
        for (int c = 0; c < 3; c++) TM[3 * a + c] = Tm[3 * a] * M[c] + Tm[3 * a + 1] * M[3 + c] + Tm[3 * a + 2] * M[6 + c];
    const double *cv = g->cov2d + 3 * (size_t)i;
    double s00 = cv[0], s01 = cv[1], s11 = cv[2], det = s00 * s11 - s01 * s01, det2 = det * det;
    /* ---- conic -> Sigma' */
    double ga = G2[2], gb = G2[3], gc = G2[4];
    double d00 = ga * (-s11 * s11 / det2) + gb * (s01 * s11 / det2) + gc * (1.0 / det - s00 * s11 / det2);
    double d11 = ga * (1.0 / det - s11 * s00 / det2) + gb * (s01 * s00 / det2) + gc * (-s00 * s00 / det2);
    double d01 = ga * (2.0 * s11 * s01 / det2) + gb * (-1.0 / det - 2.0 * s01 * s01 / det2) + gc * (2.0 * s00 * s01 / det2);
    /* ---- Sigma' = TM TM^T + 0.3 I -> TM */
    double dTM[6];
    for (int k = 0; k < 3; k++) {
        dTM[k] = 2.0 * d00 * TM[k] + d01 * TM[3 + k];
        dTM[3 + k] = 2.0 * d11 * TM[3 + k] + d01 * TM[k];
    }
    /* ---- TM = Tm M -> Tm, M ; Tm = J W -> J */
    double dTm[6] = {0}, dM[9] = {0}, dJ[6] = {0};
    for (int a = 0; a < 2; a++)
        for (int k = 0; k < 3; k++)
            for (int c = 0; c < 3; c++) {
                dTm[3 * a + k] += dTM[3 * a + c] * M[3 * k + c];
                dM[3 * k + c] += Tm[3 * a + k] * dTM[3 * a + c];
            }
    for (int a = 0; a < 2; a++)
        for (int k = 0; k < 3; k++)
            for (int c = 0; c < 3; c++) dJ[3 * a + k] += dTm[3 * a + c] * cam->R[3 * k + c];
    /* ---- J(X) and (u, v)(X) -> X */
    double dX[3] = {0, 0, 0};
    double fx = cam->fx, fy = cam->fy;
    dX[2] += dJ[0] * (-fx / (Z * Z)) + dJ[4] * (-fy / (Z * Z));
    if (!clx) {
        dX[0] += dJ[2] * (-fx / (Z * Z));
        dX[2] += dJ[2] * (2.0 * fx * X[0] / (Z * Z * Z));
    } else {
        dX[2] += dJ[2] * (fx * xzc / (Z * Z));
    }
    if (!cly) {
        dX[1] += dJ[5] * (-fy / (Z * Z));
        dX[2] += dJ[5] * (2.0 * fy * X[1] / (Z * Z * Z));
    } else {
        dX[2] += dJ[5] * (fy * yzc / (Z * Z));
    }
    dX[0] += G2[0] * fx / Z;
    dX[2] += -G2[0] * fx * X[0] / (Z * Z);
    dX[1] += G2[1] * fy / Z;
    dX[2] += -G2[1] * fy * X[1] / (Z * Z);
    /* ---- M = R(qn) diag(s) -> qn, ls */
    double dRq[9];
    for (int a = 0; a < 3; a++)
        for (int c = 0; c < 3; c++) dRq[3 * a + c] = dM[3 * a + c] * s[c];
    for (int c = 0; c < 3; c++) {
        double ds = 0.0;
        for (int a = 0; a < 3; a++) ds += dM[3 * a + c] * Rq[3 * a + c];
        gls[c] = ds * s[c];
    }
    double dqn[4];
    quat_rot_backward(qn, dRq, dqn);
    double dot = dqn[0] * qn[0] + dqn[1] * qn[1] + dqn[2] * qn[2] + dqn[3] * qn[3];
    for (int j = 0; j < 4; j++) gq[j] = (dqn[j] - qn[j] * dot) / nq;
    /* ---- colour: clamp, SH coefficients, view direction */
    double dir[3] = {m[0] - campos[0], m[1] - campos[1], m[2] - campos[2]};
    double dn = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    double d[3] = {dir[0] / dn, dir[1] / dn, dir[2] / dn};
    double Y[16], dY[16][3];
    orc_sh_basis(d, sc->sh_degree, Y);
    sh_basis_grad(d, sc->sh_degree, dY);
    double dd[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ch++) {
        double raw = 0.5;
        for (int k = 0; k < ncoef; k++) raw += sc->sh[((size_t)i * ncoef + k) * 3 + ch] * Y[k];
        if (raw < 0.0) continue;   /* clamped at zero */
        double gcol = G2[6 + ch];
        for (int k = 0; k < ncoef; k++) {
            gsh[3 * k + ch] = gcol * Y[k];
            for (int j = 0; j < 3; j++) dd[j] += gcol * sc->sh[((size_t)i * ncoef + k) * 3 + ch] * dY[k][j];
        }
    }
    double ddot = dd[0] * d[0] + dd[1] * d[1] + dd[2] * d[2];
    double dm[3];
    for (int j = 0; j < 3; j++) dm[j] = (dd[j] - d[j] * ddot) / dn;
    /* ---- X = R_cam m + T_cam -> m */
    for (int j = 0; j < 3; j++) dm[j] += cam->R[j] * dX[0] + cam->R[3 + j] * dX[1] + cam->R[6 + j] * dX[2];
    /* ---- m = mu + tau V, o_hat(tau), tau = t - mu_t */
    double dtau = 0.0;
    for (int j = 0; j < 3; j++) {
        gm[j] = dm[j];
        gv[j] = tau * dm[j];
        dtau += sc->velocity[3 * (size_t)i + j] * dm[j];
    }
    double oh = g->opacity_t[i], st = exp(sc->log_t_scale[i]);
    double sig = 1.0 / (1.0 + exp(-sc->opacity_logit[i]));
    double goh = G2[5];
    *glg = goh * oh * (1.0 - sig);
    dtau += goh * oh * (-tau / (st * st));
    *glt = goh * oh * tau * tau / (st * st);
    *gtm = -dtau;
}

static void raw_store(const double *r, int i, int ncoef, orc_scene_grad *out, int accumulate_abs, const double *w) {
    /* out = r (accumulate_abs 0), or out += |r| w (accumulate_abs 1) */
    double *dst[8] = {out->means + 3 * (size_t)i, out->t_mean + i, out->velocity + 3 * (size_t)i,
                      out->log_scales + 3 * (size_t)i, out->log_t_scale + i, out->quats + 4 * (size_t)i,
                      out->opacity_logit + i, out->sh + (size_t)i * ncoef * 3};
    const int len[8] = {3, 1, 3, 3, 1, 4, 1, 3 * ncoef};
    int o = 0;
    for (int f = 0; f < 8; f++)
        for (int j = 0; j < len[f]; j++, o++) {
            if (accumulate_abs) dst[f][j] += fabs(r[o]) * *w;
            else dst[f][j] = r[o];
        }
}

/* ---------------------------------------------------------------------------
 * orc_backward: FP64 adjoint of orc_preprocess + orc_render_pixels (full
 * frame, temporal cull on) for the loss L = sum(dl_drgb * image): per pixel
 * pixel_grad2d over its blended list, then per Gaussian chain_raw.
 *
 * With `slack` (same shapes as the gradients) it also returns, per element,
 * how far an FP32 renderer's gradient may legitimately differ because a
 * discrete decision at some pixel goes the other way (the decisions the image
 * slack of orc_render_pixels counts: alpha against 1/255, the stop rule, the
 * binary32 depth-key order; the same binary32 footprint decides which are
 * near).  At each pixel with near decisions the list is re-walked with each
 * decision flipped in turn (and in key order); the change of every Gaussian's
 * 2D gradient is accumulated in absolute value, then carried to the raw
 * parameters through the absolute value of the chain's Jacobian.  It is 0 for
 * an element whose Gaussian has no near decision in any pixel it touches.
 * ------------------------------------------------------------------------- */
void orc_backward(const orc_scene *sc, const orc_camera *cam, double t, const double *dl_drgb, const double bg[3],
                  orc_scene_grad *out, orc_scene_grad *slack) {
    const int n = sc->n, ncoef = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    const int nraw = ORC_RAW_FIXED + 3 * ncoef;
    const int64_t npix = (int64_t)cam->width * cam->height;
    orc_g2d g;
    g.drawn = (int32_t *)calloc(n > 0 ? n : 1, sizeof(int32_t));
    double *buf = (double *)calloc((size_t)(n > 0 ? n : 1) * 15, sizeof(double));
    g.u = buf; g.v = buf + n; g.depth = buf + 2 * (size_t)n; g.conic = buf + 3 * (size_t)n;
    g.cov2d = buf + 6 * (size_t)n; g.opacity_t = buf + 9 * (size_t)n; g.rgb = buf + 10 * (size_t)n;
    g.lambda_max = buf + 13 * (size_t)n;
    g.err = (double *)calloc((size_t)(n > 0 ? n : 1) * 16, sizeof(double));
    orc_preprocess(sc, cam, t, 1, &g);
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    int nd = 0;
    for (int i = 0; i < n; i++)
        if (g.drawn[i] || g.err[16 * (size_t)i + 7] == 2.0) ids[nd++] = i;
    /* per-Gaussian gradients of the 2D quantities: u, v, a, b, c, o_hat, r, g, b (and their slack) */
    double *g2 = (double *)calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double));
    double *s2 = slack ? (double *)calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double)) : NULL;
#pragma omp parallel
    {
        double *loc = (double *)calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double));
        double *sloc = slack ? (double *)calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double)) : NULL;
        size_t cap = 1024;
        orc_cand *cand = (orc_cand *)malloc(sizeof(orc_cand) * cap);
        orc_cand *alt = (orc_cand *)malloc(sizeof(orc_cand) * cap);
        size_t bcap = 0;
        orc_blended *bl = NULL, *bl2 = NULL;
        double *c0 = NULL, *c1 = NULL;
        int64_t *near_pos = NULL;
#pragma omp for schedule(dynamic, 8)
        for (int64_t q = 0; q < npix; q++) {
            const double x = (double)(q % cam->width) + 0.5, y = (double)(q / cam->width) + 0.5;
            const size_t nc = pixel_candidates(&g, ids, nd, x, y, &cand, &alt, &cap);
            if (bcap < nc + 1) {
                bcap = 2 * (nc + 1);
                bl = (orc_blended *)realloc(bl, sizeof(orc_blended) * bcap);
                bl2 = (orc_blended *)realloc(bl2, sizeof(orc_blended) * bcap);
                c0 = (double *)realloc(c0, sizeof(double) * 9 * bcap);
                c1 = (double *)realloc(c1, sizeof(double) * 9 * bcap);
                near_pos = (int64_t *)realloc(near_pos, sizeof(int64_t) * 2 * bcap);
            }
            int64_t stop_pos;
            const size_t nb = pixel_blend_list(&g, cand, nc, x, y, -1, -1, bl, &stop_pos);
            const double *G = dl_drgb + 3 * q;
            pixel_grad2d(&g, bl, nb, G, bg, x, y, c0);
            for (size_t k = 0; k < nb; k++)
                for (int j = 0; j < 9; j++) loc[9 * (size_t)bl[k].idx + j] += c0[9 * k + j];
            if (!slack) continue;
            /* near decisions up to the stop: alpha flips and stop flips (as orc_render_pixels) */
            size_t nn = 0;
            double T = 1.0, Tf = 1.0, wT = 0.0;
            for (size_t k = 0; k < nc && (int64_t)k <= stop_pos; k++) {
                if (cand[k].near_alpha) near_pos[nn++] = (int64_t)k;
                const double alpha = cand[k].alpha, af = cand[k].alpha_f;
                if (alpha < 0.0) continue;
                const double test = T * (1.0 - alpha), test_f = Tf * (1.0 - af);
                const double wstop = wT + cand[k].w * af / (1.0 - af) + 2.0 * ORC_U;
                const int stop = test < ORC_T_MIN;
                const int near_stop = stop ? (test_f * (1.0 + wstop) >= ORC_T_MIN) : (test_f * (1.0 - wstop) < ORC_T_MIN);
                if (near_stop) near_pos[nn++] = -1 - (int64_t)k;   /* negative: a stop flip */
                if (stop) break;
                T = test;
                Tf = test_f;
                wT = wstop;
            }
            for (size_t j = 0; j < nn; j++) {
                int64_t sp;
                const size_t n1 = near_pos[j] >= 0 ? pixel_blend_list(&g, cand, nc, x, y, near_pos[j], -1, bl2, &sp)
                                                   : pixel_blend_list(&g, cand, nc, x, y, -1, -1 - near_pos[j], bl2, &sp);
                pixel_grad2d(&g, bl2, n1, G, bg, x, y, c1);
                add_grad2d_change(bl, c0, nb, bl2, c1, n1, sloc);
            }
            /* the binary32 depth-key order */
            int sorted = 1, all_f32 = 1;
            double pk = -INFINITY;
            int32_t pi = -1;
            for (size_t k = 0; k < nc; k++) {
                if (g.err[16 * (size_t)cand[k].idx + 15] == 0.0) all_f32 = 0;
                if (cand[k].alpha < 0.0) continue;
                if (cand[k].key < pk || (cand[k].key == pk && cand[k].idx < pi)) sorted = 0;
                if ((int64_t)k <= stop_pos) { pk = cand[k].key; pi = cand[k].idx; }
            }
            if (all_f32 && !sorted) {
                int64_t sp;
                memcpy(alt, cand, nc * sizeof(orc_cand));
                qsort(alt, nc, sizeof(orc_cand), cand_key_cmp);
                const size_t n1 = pixel_blend_list(&g, alt, nc, x, y, -1, -1, bl2, &sp);
                pixel_grad2d(&g, bl2, n1, G, bg, x, y, c1);
                add_grad2d_change(bl, c0, nb, bl2, c1, n1, sloc);
            }
        }
#pragma omp critical
        {
            for (size_t j = 0; j < (size_t)n * 9; j++) g2[j] += loc[j];
            if (slack)
                for (size_t j = 0; j < (size_t)n * 9; j++) s2[j] += sloc[j];
        }
        free(loc);
        free(sloc);
        free(cand);
        free(alt);
        free(bl);
        free(bl2);
        free(c0);
        free(c1);
        free(near_pos);
    }
    /* per Gaussian: chain rule back to the raw parameters (and the slack through |Jacobian|) */
#pragma omp parallel
    {
        double *r = (double *)malloc(sizeof(double) * (size_t)nraw);
#pragma omp for schedule(static)
        for (int i = 0; i < n; i++) {
            for (int j = 0; j < nraw; j++) r[j] = 0.0;
            if (slack) raw_store(r, i, ncoef, slack, 0, NULL);
            if (!g.drawn[i]) {
                raw_store(r, i, ncoef, out, 0, NULL);
                continue;
            }
            chain_raw(sc, cam, t, &g, i, g2 + 9 * (size_t)i, r);
            raw_store(r, i, ncoef, out, 0, NULL);
            if (!slack) continue;
            for (int k = 0; k < 9; k++) {
                const double w = s2[9 * (size_t)i + k];
                if (w == 0.0) continue;
                double e9[9] = {0};
                e9[k] = 1.0;
                chain_raw(sc, cam, t, &g, i, e9, r);
                raw_store(r, i, ncoef, slack, 1, &w);
            }
        }
        free(r);
    }
    free(g2);
    free(s2);
    free(ids);
    free(buf);
    free(g.err);
    free(g.drawn);
}

/* Per-pixel fingerprint of the blended contributor lists (for finite
 * differences: a parameter step that changes any pixel's list crosses a
 * discontinuity of the image). */
void orc_fingerprint(const orc_scene *sc, const orc_camera *cam, double t, uint64_t *out) {
    const int n = sc->n;
    const int64_t npix = (int64_t)cam->width * cam->height;
    orc_g2d g;
    g.drawn = (int32_t *)calloc(n > 0 ? n : 1, sizeof(int32_t));
    double *buf = (double *)calloc((size_t)(n > 0 ? n : 1) * 15, sizeof(double));
    g.u = buf; g.v = buf + n; g.depth = buf + 2 * (size_t)n; g.conic = buf + 3 * (size_t)n;
    g.cov2d = buf + 6 * (size_t)n; g.opacity_t = buf + 9 * (size_t)n; g.rgb = buf + 10 * (size_t)n;
    g.lambda_max = buf + 13 * (size_t)n;
    g.err = NULL;
    orc_preprocess(sc, cam, t, 1, &g);
#pragma omp parallel
    {
        size_t cap = 1024;
        orc_cand *cand = (orc_cand *)malloc(sizeof(orc_cand) * cap);
#pragma omp for schedule(dynamic, 8)
        for (int64_t q = 0; q < npix; q++) {
            double x = (double)(q % cam->width) + 0.5, y = (double)(q / cam->width) + 0.5;
            size_t nc = 0;
            for (int i = 0; i < n; i++) {
                if (!g.drawn[i]) continue;
                double dx = g.u[i] - x, dy = g.v[i] - y;
                const double *cn = g.conic + 3 * (size_t)i;
                double p = -0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy;
                if (p > 0.0) continue;
                double alpha = fmin(ORC_ALPHA_MAX, g.opacity_t[i] * exp(p));
                if (alpha < ORC_ALPHA_MIN) continue;
                if (nc == cap) { cap *= 2; cand = (orc_cand *)realloc(cand, sizeof(orc_cand) * cap); }
                cand[nc].depth = g.depth[i];
                cand[nc].idx = i;
                cand[nc].alpha = alpha;
                nc++;
            }
            qsort(cand, nc, sizeof(orc_cand), cand_cmp);
            double T = 1.0;
            uint64_t h = 1469598103934665603ull;
            for (size_t k = 0; k < nc; k++) {
                double test = T * (1.0 - cand[k].alpha);
                if (test < ORC_T_MIN) break;
                h = (h ^ (uint64_t)(cand[k].idx + 1)) * 1099511628211ull;
                h ^= (cand[k].alpha >= 0.99) ? 0x9E3779B97F4A7C15ull : 0ull;   /* alpha clamp active */
                T = test;
            }
            out[q] = h;
        }
        free(cand);
    }
    free(buf);
    free(g.drawn);
}
