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
 *   - 3DGS constants (the paper defers to 3DGS for rasterisation): near 0.2,
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

#define ORC_NEAR 0.2
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
} orc_scene;

typedef struct {
    double R[9], T[3];           /* world -> camera, row-major */
    double fx, fy, cx, cy;
    int32_t width, height;
} orc_camera;

typedef struct {                 /* per-Gaussian FP64 2D Gaussian, all arrays length N */
    int32_t *drawn;
    double *u, *v, *depth;
    double *conic;               /* N x 3 (a, b, c): inverse of the 2D covariance */
    double *cov2d;               /* N x 3 (xx, xy, yy) including the dilation */
    double *opacity_t;           /* sigmoid(logit) * temporal factor */
    double *rgb;                 /* N x 3 */
    double *lambda_max;
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
 * orc_preprocess: per Gaussian, the dynamic 2D Gaussian at time t.
 *   tau = t - mu_t;  mu(t) = mu + tau V3D                       (Eq. 7)
 *   o_hat = sigmoid(logit) exp(-tau^2 / (2 s_t^2)), s_t = e^{log s_t}   (Eq. 6-7)
 *   X = R_cam mu(t) + T_cam = P_view + tau V_view               (Eq. 9-11, 15)
 *   (u, v) = (fx X/Z + cx, fy Y/Z + cy)                          (Eq. 12)
 *   J = d(u,v)/dX at X (x/z, y/z clamped)                       (Eq. 14)
 *   Sigma' = J R_cam Sigma3D R_cam^T J^T + 0.3 I                (Eq. 16)
 *   conic = Sigma'^{-1}; colour = max(0, SH . Y(dir) + 0.5)
 * temporal_cull: also drop o_hat < 1/255 (lossless: alpha < 1/255 everywhere).
 * ------------------------------------------------------------------------- */
void orc_preprocess(const orc_scene *sc, const orc_camera *cam, double t, int temporal_cull, orc_g2d *out) {
    const int n = sc->n, ncoef = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    double campos[3];
    cam_position(cam, campos);
    const double limx = ORC_JAC_CLAMP * (0.5 * cam->width) / cam->fx;
    const double limy = ORC_JAC_CLAMP * (0.5 * cam->height) / cam->fy;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        out->drawn[i] = 0;
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
        if (!(X[2] > ORC_NEAR)) continue;
        if (temporal_cull && !(oh >= ORC_ALPHA_MIN)) continue;
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
        double d[3] = {m[0] - campos[0], m[1] - campos[1], m[2] - campos[2]};
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        d[0] /= dn; d[1] /= dn; d[2] /= dn;
        double Y[16];
        orc_sh_basis(d, sc->sh_degree, Y);
        for (int ch = 0; ch < 3; ch++) {
            double s = 0.0;
            for (int k = 0; k < ncoef; k++) s += sc->sh[((size_t)i * ncoef + k) * 3 + ch] * Y[k];
            out->rgb[3 * (size_t)i + ch] = fmax(0.0, s + 0.5);
        }
        out->drawn[i] = 1;
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
 * Besides the colour it returns T, the number of blended Gaussians, and a
 * per-pixel slack: an upper bound on how far an FP32 evaluation of the same
 * definition may legitimately move the colour because a discrete decision
 * (alpha vs 1/255, T(1-alpha) vs 1e-4, p vs 0, the order of two nearly equal
 * depths) sits within FP32 reach of its threshold; and Tw, the accumulated
 * relative error budget of an FP32 T (the sum over blended Gaussians of the
 * alpha budget times alpha / (1 - alpha), plus 1e-6 per blend).  eps_px is
 * the absolute error budget of an FP32 projected mean in pixels.
 * ------------------------------------------------------------------------- */
typedef struct { double depth; int32_t idx; double alpha; double w; int near_alpha; } orc_cand;

static int cand_cmp(const void *pa, const void *pb) {
    const orc_cand *a = (const orc_cand *)pa, *b = (const orc_cand *)pb;
    if (a->depth < b->depth) return -1;
    if (a->depth > b->depth) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

void orc_render_pixels(const orc_g2d *g, int n, const orc_camera *cam, const double bg[3],
                       int64_t npix, const int32_t *px, const int32_t *py, double eps_px,
                       double *out_rgb, double *out_T, int32_t *out_ncontrib, double *out_slack,
                       double *out_Tw) {
    /* compact list of drawn Gaussians */
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    int nd = 0;
    for (int i = 0; i < n; i++)
        if (g->drawn[i]) ids[nd++] = i;
    const int64_t W = cam->width;
    if (npix < 0) npix = (int64_t)cam->width * cam->height;
#pragma omp parallel
    {
        size_t cap = 1024;
        orc_cand *cand = (orc_cand *)malloc(sizeof(orc_cand) * cap);
#pragma omp for schedule(dynamic, 8)
        for (int64_t q = 0; q < npix; q++) {
            double x = (px ? px[q] : (int32_t)(q % W)) + 0.5;
            double y = (py ? py[q] : (int32_t)(q / W)) + 0.5;
            size_t nc = 0;
            double slack = 0.0;
            for (int k = 0; k < nd; k++) {
                int i = ids[k];
                double dx = g->u[i] - x, dy = g->v[i] - y;
                double a = g->conic[3 * (size_t)i], b = g->conic[3 * (size_t)i + 1], c = g->conic[3 * (size_t)i + 2];
                double p = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
                /* FP32 relative error budget of alpha for this pair */
                double gx = fabs(a * dx + b * dy), gy = fabs(b * dx + c * dy);
                /* FP32 conic: relative error ~ cond * 2^-22 from the cancellation in det */
                const double *cv = g->cov2d + 3 * (size_t)i;
                double cond = (fabs(cv[0] * cv[2]) + cv[1] * cv[1]) / (cv[0] * cv[2] - cv[1] * cv[1]);
                double w = 2e-5 + (gx + gy) * eps_px + fabs(p) * (4e-7 + cond * 2.4e-7);
                int near_p = fabs(p) <= (gx + gy) * eps_px + 1e-6;
                if (p > 0.0 && !near_p) continue;
                double alpha = fmin(ORC_ALPHA_MAX, g->opacity_t[i] * exp(fmin(p, 0.0)));
                int near_alpha = fabs(alpha - ORC_ALPHA_MIN) <= w * ORC_ALPHA_MIN || near_p;
                if (p > 0.0 || alpha < ORC_ALPHA_MIN) {
                    if (!near_alpha) continue;
                    alpha = -alpha; /* excluded here, but within reach of inclusion */
                }
                if (nc == cap) { cap *= 2; cand = (orc_cand *)realloc(cand, sizeof(orc_cand) * cap); }
                cand[nc].depth = g->depth[i];
                cand[nc].idx = i;
                cand[nc].alpha = alpha;
                cand[nc].w = w;
                cand[nc].near_alpha = near_alpha;
                nc++;
            }
            qsort(cand, nc, sizeof(orc_cand), cand_cmp);
            double T = 1.0, C[3] = {0, 0, 0}, wT = 0.0, cmax = 0.0;
            int32_t ncontrib = 0;
            for (size_t k = 0; k < nc; k++) {
                const double *c = g->rgb + 3 * (size_t)cand[k].idx;
                double cm = fmax(c[0], fmax(c[1], c[2]));
                if (cm > cmax) cmax = cm;
            }
            int32_t last = -1;
            double prev_depth = -1.0, prev_alpha = 0.0;
            for (size_t k = 0; k < nc; k++) {
                double alpha = cand[k].alpha;
                if (cand[k].near_alpha) slack += 2.0 * fabs(alpha) * (1.0 + cand[k].w) * cmax * T + 1e-7;
                if (alpha < 0.0) continue; /* not blended in FP64 */
                /* nearly equal depths: FP32 keys may order the pair the other way */
                if (last >= 0 && fabs(cand[k].depth - prev_depth) <= 4e-6 * fmax(fabs(prev_depth), fabs(cand[k].depth)))
                    slack += 2.0 * prev_alpha * alpha * cmax * (T / (1.0 - prev_alpha)) + 1e-7;
                double test = T * (1.0 - alpha);
                /* accumulated FP32 relative error of T, and the stop decision */
                double wstop = wT + cand[k].w * alpha / (1.0 - alpha) + 1e-6;
                if (fabs(test - ORC_T_MIN) <= wstop * ORC_T_MIN) slack += T * alpha * cmax + 2.0 * ORC_T_MIN * cmax;
                if (test < ORC_T_MIN) break;
                const double *c = g->rgb + 3 * (size_t)cand[k].idx;
                for (int ch = 0; ch < 3; ch++) C[ch] += alpha * T * c[ch];
                T = test;
                wT = wstop;
                ncontrib++;
                last = (int32_t)k;
                prev_depth = cand[k].depth;
                prev_alpha = alpha;
            }
            for (int ch = 0; ch < 3; ch++) out_rgb[3 * q + ch] = C[ch] + T * bg[ch];
            if (out_T) out_T[q] = T;
            if (out_ncontrib) out_ncontrib[q] = ncontrib;
            if (out_slack) out_slack[q] = slack;
            if (out_Tw) out_Tw[q] = wT;
        }
        free(cand);
    }
    free(ids);
}

/* ---------------------------------------------------------------------------
 * orc_bin_f32: FP32 mirror of the binning arithmetic (per Gaussian: depth key
 * bits, radius, tile rectangle, tile count) in the fixed operation order that
 * the GPU preprocess also follows, so that tile/key lists can be compared bit
 * for bit.  Every product and sum below is a separately rounded IEEE single
 * operation evaluated left to right as parenthesised; sqrt and division are
 * correctly rounded; this file is compiled with -ffp-contract=off.
 *
 *   tau = t - mu_t;  m_j = mu_j + tau*v_j
 *   X_r = ((R_r0*m_0 + R_r1*m_1) + R_r2*m_2) + T_r
 *   cull !(Z > 0.2)
 *   o = 1/(1 + expf(-logit)); st = expf(lst); o_hat = o * expf((-0.5*(tau*tau))/(st*st))
 *   cull !(o_hat >= 1/255)
 *   xz = X/Z, yz = Y/Z; u = fx*xz + cx; v = fy*yz + cy
 *   limx = 1.3*((0.5*W)/fx); xzc = min(limx, max(-limx, xz)) (same for y)
 *   J00 = fx/Z, J02 = -(fx*xzc)/Z, J11 = fy/Z, J12 = -(fy*yzc)/Z
 *   qn = q / sqrtf(((w*w + x*x) + y*y) + z*z); R(qn) as in orc_quat_to_rot
 *   with 1 - 2*(a*a + b*b) and 2*(a*b -/+ c*d); M_ij = R_ij * expf(ls_j)
 *   Tj_0 = J00*W_0j + J02*W_2j; Tj_1 = J11*W_1j + J12*W_2j   (T = J W)
 *   TM_ij = (T_i0*M_0j + T_i1*M_1j) + T_i2*M_2j              (TM = J W M)
 *   s00 = ((TM00^2 + TM01^2) + TM02^2) + 0.3; s11 likewise;
 *   s01 = (TM00*TM10 + TM01*TM11) + TM02*TM12
 *   det = s00*s11 - s01*s01; cull !(det > 0)
 *   mid = 0.5*(s00 + s11); lam = mid + sqrtf(max(0.1, mid*mid - det))
 *   r = (int) ceilf(3.33 * sqrtf(lam))   (the 2D Gaussian's radius)
 *   cull unless u, v finite
 *   k2 = ((2*logf(255*o_hat))*1.0008) + 0.0008;  rx = ceilf(sqrtf(k2*s00)), ry = ceilf(sqrtf(k2*s11))
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
 * Flags: bit 0 -- sqrt(k2 s00) or sqrt(k2 s11) within 3e-6 relative of an
 * integer (rectangle); bit 1 -- o_hat within 3e-6 relative of 1/255 (cull);
 * bit 2 -- 3.33 sqrt(lambda_max) within 3e-6 of an integer (the radius field
 * only: it does not take part in binning); bit 3 -- a column-cut decision
 * (a against b through ex, lo/tile or hi/tile against an integer) within
 * reach of the same ulp differences.
 * Every operation above is correctly rounded and reproducible on any IEEE
 * machine except expf and logf, whose FP32 results may differ by one or two
 * ulps between math libraries; through the chains (s -> Sigma' -> radii, three
 * exps -> o_hat -> k2) that moves these quantities by at most ~1.5e-6
 * relative, so a decision further than 3e-6 from its threshold is the same
 * everywhere.  A flagged Gaussian is excluded
 * from bit-exact comparison.  A culled Gaussian has depth key 0xFFFFFFFF and
 * 0 tiles.
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t n, sh_degree;
    const float *means, *t_mean, *velocity, *log_scales, *log_t_scale, *quats, *opacity_logit;
} orc_scene_f32;

typedef struct { float R[9], T[3], fx, fy, cx, cy; int32_t width, height; } orc_camera_f32;

void orc_bin_f32(const orc_scene_f32 *sc, const orc_camera_f32 *cam, float t, int32_t tile, int32_t trim,
                 uint32_t *depth_key, int32_t *radius, int32_t *rect /* N x 4: x0,x1,y0,y1 */,
                 uint32_t *tiles_touched, uint64_t *trims, int32_t *flags, float *uv /* N x 2, may be NULL */) {
    const int n = sc->n;
    const int32_t tiles_x = (cam->width + tile - 1) / tile, tiles_y = (cam->height + tile - 1) / tile;
    const float limx = 1.3f * ((0.5f * (float)cam->width) / cam->fx);
    const float limy = 1.3f * ((0.5f * (float)cam->height) / cam->fy);
    const float tilef = (float)tile;
    const float amin = (float)(1.0 / 255.0);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        depth_key[i] = 0xFFFFFFFFu;
        radius[i] = 0;
        rect[4 * (size_t)i + 0] = rect[4 * (size_t)i + 1] = rect[4 * (size_t)i + 2] = rect[4 * (size_t)i + 3] = 0;
        tiles_touched[i] = 0;
        trims[i] = 0;
        flags[i] = 0;
        if (uv) { uv[2 * (size_t)i] = 0.f; uv[2 * (size_t)i + 1] = 0.f; }
        const float *mu = sc->means + 3 * (size_t)i, *vel = sc->velocity + 3 * (size_t)i;
        float tau = t - sc->t_mean[i];
        float m0 = mu[0] + tau * vel[0], m1 = mu[1] + tau * vel[1], m2 = mu[2] + tau * vel[2];
        const float *R = cam->R;
        float X = ((R[0] * m0 + R[1] * m1) + R[2] * m2) + cam->T[0];
        float Y = ((R[3] * m0 + R[4] * m1) + R[5] * m2) + cam->T[1];
        float Z = ((R[6] * m0 + R[7] * m1) + R[8] * m2) + cam->T[2];
        if (!(Z > 0.2f)) continue;
        /* opacity and the temporal factor (transcendental decision) */
        float o = 1.0f / (1.0f + expf(-sc->opacity_logit[i]));
        float st = expf(sc->log_t_scale[i]);
        float oh = o * expf((-0.5f * (tau * tau)) / (st * st));
        if (fabsf(oh - amin) <= 3e-6f * amin) flags[i] |= 2;
        if (!(oh >= amin)) continue;
        float xz = X / Z, yz = Y / Z;
        float u = cam->fx * xz + cam->cx, v = cam->fy * yz + cam->cy;
        float xzc = fminf(limx, fmaxf(-limx, xz)), yzc = fminf(limy, fmaxf(-limy, yz));
        float J00 = cam->fx / Z, J02 = -(cam->fx * xzc) / Z;
        float J11 = cam->fy / Z, J12 = -(cam->fy * yzc) / Z;
        const float *q = sc->quats + 4 * (size_t)i;
        float qn2 = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
        float qn = sqrtf(qn2);
        float w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
        float Rq[9];
        Rq[0] = 1.0f - 2.0f * (y * y + z * z); Rq[1] = 2.0f * (x * y - w * z);       Rq[2] = 2.0f * (x * z + w * y);
        Rq[3] = 2.0f * (x * y + w * z);       Rq[4] = 1.0f - 2.0f * (x * x + z * z); Rq[5] = 2.0f * (y * z - w * x);
        Rq[6] = 2.0f * (x * z - w * y);       Rq[7] = 2.0f * (y * z + w * x);       Rq[8] = 1.0f - 2.0f * (x * x + y * y);
        const float *ls = sc->log_scales + 3 * (size_t)i;
        float s[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
        float M[9];
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) M[3 * r + c] = Rq[3 * r + c] * s[c];
        float Tm[6];
        for (int j = 0; j < 3; j++) {
            Tm[j] = J00 * R[j] + J02 * R[6 + j];
            Tm[3 + j] = J11 * R[3 + j] + J12 * R[6 + j];
        }
        float TM[6];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 3; c++)
                TM[3 * r + c] = (Tm[3 * r + 0] * M[0 * 3 + c] + Tm[3 * r + 1] * M[1 * 3 + c]) + Tm[3 * r + 2] * M[2 * 3 + c];
        float s00 = ((TM[0] * TM[0] + TM[1] * TM[1]) + TM[2] * TM[2]) + 0.3f;
        float s01 = (TM[0] * TM[3] + TM[1] * TM[4]) + TM[2] * TM[5];
        float s11 = ((TM[3] * TM[3] + TM[4] * TM[4]) + TM[5] * TM[5]) + 0.3f;
        float det = s00 * s11 - s01 * s01;
        if (!(det > 0.0f)) continue;
        float mid = 0.5f * (s00 + s11);
        float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
        float rf = ceilf(3.33f * sqrtf(lam));
        if (!(isfinite(u) && isfinite(v))) continue;
        float k2 = ((2.0f * logf(255.0f * oh)) * 1.0008f) + 0.0008f;
        float ex = sqrtf(k2 * s00), ey = sqrtf(k2 * s11);
        float rx = ceilf(ex), ry = ceilf(ey);
        {   /* radii decided within reach of an ulp difference in expf / logf */
            const double rr = 3.33 * sqrt((double)lam);
            if (fabs(rr - nearbyint(rr)) <= 3e-6 * rr) flags[i] |= 4;
            if (fabs((double)ex - nearbyint((double)ex)) <= 3e-6 * ex) flags[i] |= 1;
            if (fabs((double)ey - nearbyint((double)ey)) <= 3e-6 * ey) flags[i] |= 1;
        }
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
        /* ulp differences in expf / logf move k2 and Sigma' by <= ~1.5e-6 relative and
         * the row extents (|offset| <= ey) with them; u, v are the same bits everywhere */
        const double reach = 3e-6 * ((double)ey / tilef);
        uint64_t tw = 0;
        int64_t kept = 0;
        for (int32_t c = x0; c <= x1; c++) {
            const int32_t j = c - x0;
            int32_t cut_t = 0, cut_b = 0;
            if (trim && j < 8) {
                const float left = ((float)c * tilef + 0.5f) - u;
                const float right = fminf((float)c * tilef + tl, wl) - u;
                if (fabs((double)left - ex) <= 3e-6 * ex || fabs((double)right + ex) <= 3e-6 * ex) flags[i] |= 8;
                const float a = fmaxf(left, -ex), b = fminf(right, ex);
                if (!(a <= b)) {
                    cut_t = h < 15 ? h : 15;
                    cut_b = h - cut_t < 15 ? h - cut_t : 15;
                } else {
                    const float xt = fminf(fmaxf(-xl, a), b), xb = fminf(fmaxf(xl, a), b);
                    const float lo = ((v + ((s01 * xt) - sqrtf(fmaxf(0.0f, det * (q2 - xt * xt)))) * i00) - 0.015625f) - tl;
                    const float hi = ((v + ((s01 * xb) + sqrtf(fmaxf(0.0f, det * (q2 - xb * xb)))) * i00) + 0.015625f) - 0.5f;
                    const float flo = lo / tilef, fhi = hi / tilef;
                    if (fabs((double)flo - nearbyint((double)flo)) <= reach + 2e-7 * (fabs((double)flo) + 1.0) ||
                        fabs((double)fhi - nearbyint((double)fhi)) <= reach + 2e-7 * (fabs((double)fhi) + 1.0))
                        flags[i] |= 8;
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

void orc_backward(const orc_scene *sc, const orc_camera *cam, double t, const double *dl_drgb, const double bg[3],
                  orc_scene_grad *out) {
    const int n = sc->n, ncoef = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    const int64_t npix = (int64_t)cam->width * cam->height;
    orc_g2d g;
    g.drawn = (int32_t *)calloc(n > 0 ? n : 1, sizeof(int32_t));
    double *buf = (double *)calloc((size_t)(n > 0 ? n : 1) * 15, sizeof(double));
    g.u = buf; g.v = buf + n; g.depth = buf + 2 * (size_t)n; g.conic = buf + 3 * (size_t)n;
    g.cov2d = buf + 6 * (size_t)n; g.opacity_t = buf + 9 * (size_t)n; g.rgb = buf + 10 * (size_t)n;
    g.lambda_max = buf + 13 * (size_t)n;
    orc_preprocess(sc, cam, t, 1, &g);
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    int nd = 0;
    for (int i = 0; i < n; i++)
        if (g.drawn[i]) ids[nd++] = i;
    /* per-Gaussian gradients of the 2D quantities: u, v, a, b, c, o_hat, r, g, b */
    double *g2 = (double *)calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double));
#pragma omp parallel
    {
        double *loc = (double *)calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double));
        size_t cap = 1024;
        orc_cand *cand = (orc_cand *)malloc(sizeof(orc_cand) * cap);
        orc_blended *bl = (orc_blended *)malloc(sizeof(orc_blended) * cap);
#pragma omp for schedule(dynamic, 8)
        for (int64_t q = 0; q < npix; q++) {
            double x = (double)(q % cam->width) + 0.5, y = (double)(q / cam->width) + 0.5;
            size_t nc = 0;
            for (int k = 0; k < nd; k++) {
                int i = ids[k];
                double dx = g.u[i] - x, dy = g.v[i] - y;
                const double *cn = g.conic + 3 * (size_t)i;
                double p = -0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy;
                if (p > 0.0) continue;
                double alpha = fmin(ORC_ALPHA_MAX, g.opacity_t[i] * exp(p));
                if (alpha < ORC_ALPHA_MIN) continue;
                if (nc == cap) {
                    cap *= 2;
                    cand = (orc_cand *)realloc(cand, sizeof(orc_cand) * cap);
                    bl = (orc_blended *)realloc(bl, sizeof(orc_blended) * cap);
                }
                cand[nc].depth = g.depth[i];
                cand[nc].idx = i;
                cand[nc].alpha = alpha;
                nc++;
            }
            qsort(cand, nc, sizeof(orc_cand), cand_cmp);
            double T = 1.0;
            size_t nb = 0;
            for (size_t k = 0; k < nc; k++) {
                double alpha = cand[k].alpha;
                double test = T * (1.0 - alpha);
                if (test < ORC_T_MIN) break;
                int i = cand[k].idx;
                const double *cn = g.conic + 3 * (size_t)i;
                double dx = g.u[i] - x, dy = g.v[i] - y;
                double p = -0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy;
                bl[nb].idx = i;
                bl[nb].alpha = alpha;
                bl[nb].raw_alpha = g.opacity_t[i] * exp(p);
                bl[nb].T = T;
                nb++;
                T = test;
            }
            const double *G = dl_drgb + 3 * q;
            double B[3] = {bg[0], bg[1], bg[2]};
            for (size_t kk = nb; kk-- > 0;) {
                int i = bl[kk].idx;
                double alpha = bl[kk].alpha, Ti = bl[kk].T;
                const double *c = g.rgb + 3 * (size_t)i;
                double *gi = loc + 9 * (size_t)i;
                double dalpha = 0.0;
                for (int ch = 0; ch < 3; ch++) {
                    gi[6 + ch] += alpha * Ti * G[ch];
                    dalpha += Ti * G[ch] * (c[ch] - B[ch]);
                    B[ch] = alpha * c[ch] + (1.0 - alpha) * B[ch];
                }
                if (bl[kk].raw_alpha > ORC_ALPHA_MAX) continue;   /* clamped: no gradient through alpha */
                const double *cn = g.conic + 3 * (size_t)i;
                double dx = g.u[i] - x, dy = g.v[i] - y;
                double dp = dalpha * alpha;
                gi[5] += dalpha * alpha / g.opacity_t[i];
                gi[0] += -dp * (cn[0] * dx + cn[1] * dy);
                gi[1] += -dp * (cn[1] * dx + cn[2] * dy);
                gi[2] += -0.5 * dp * dx * dx;
                gi[3] += -dp * dx * dy;
                gi[4] += -0.5 * dp * dy * dy;
            }
        }
#pragma omp critical
        for (size_t j = 0; j < (size_t)n * 9; j++) g2[j] += loc[j];
        free(loc);
        free(cand);
        free(bl);
    }
    /* per Gaussian: chain rule back to the raw parameters */
    double campos[3];
    cam_position(cam, campos);
    const double limx = ORC_JAC_CLAMP * (0.5 * cam->width) / cam->fx;
    const double limy = ORC_JAC_CLAMP * (0.5 * cam->height) / cam->fy;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        double *gm = out->means + 3 * (size_t)i, *gv = out->velocity + 3 * (size_t)i;
        double *gls = out->log_scales + 3 * (size_t)i, *gq = out->quats + 4 * (size_t)i;
        double *gsh = out->sh + (size_t)i * ncoef * 3;
        for (int j = 0; j < 3; j++) gm[j] = gv[j] = gls[j] = 0.0;
        for (int j = 0; j < 4; j++) gq[j] = 0.0;
        for (int j = 0; j < ncoef * 3; j++) gsh[j] = 0.0;
        out->t_mean[i] = out->log_t_scale[i] = out->opacity_logit[i] = 0.0;
        if (!g.drawn[i]) continue;
        const double *G2 = g2 + 9 * (size_t)i;
        /* ---- forward quantities */
        double tau = t - sc->t_mean[i];
        double m[3], X[3];
        for (int j = 0; j < 3; j++) m[j] = sc->means[3 * (size_t)i + j] + tau * sc->velocity[3 * (size_t)i + j];
        for (int r = 0; r < 3; r++)
            X[r] = cam->R[3 * r] * m[0] + cam->R[3 * r + 1] * m[1] + cam->R[3 * r + 2] * m[2] + cam->T[r];
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
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) M[3 * r + c] = Rq[3 * r + c] * s[c];
        double Tm[6], TM[6];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 3; c++) Tm[3 * r + c] = J[3 * r] * cam->R[c] + J[3 * r + 1] * cam->R[3 + c] + J[3 * r + 2] * cam->R[6 + c];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 3; c++) TM[3 * r + c] = Tm[3 * r] * M[c] + Tm[3 * r + 1] * M[3 + c] + Tm[3 * r + 2] * M[6 + c];
        const double *cv = g.cov2d + 3 * (size_t)i;
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
        for (int r = 0; r < 2; r++)
            for (int k = 0; k < 3; k++)
                for (int c = 0; c < 3; c++) {
                    dTm[3 * r + k] += dTM[3 * r + c] * M[3 * k + c];
                    dM[3 * k + c] += Tm[3 * r + k] * dTM[3 * r + c];
                }
        for (int r = 0; r < 2; r++)
            for (int k = 0; k < 3; k++)
                for (int c = 0; c < 3; c++) dJ[3 * r + k] += dTm[3 * r + c] * cam->R[3 * k + c];
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
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) dRq[3 * r + c] = dM[3 * r + c] * s[c];
        for (int c = 0; c < 3; c++) {
            double ds = 0.0;
            for (int r = 0; r < 3; r++) ds += dM[3 * r + c] * Rq[3 * r + c];
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
        double oh = g.opacity_t[i], st = exp(sc->log_t_scale[i]);
        double sig = 1.0 / (1.0 + exp(-sc->opacity_logit[i]));
        double goh = G2[5];
        out->opacity_logit[i] = goh * oh * (1.0 - sig);
        dtau += goh * oh * (-tau / (st * st));
        out->log_t_scale[i] = goh * oh * tau * tau / (st * st);
        out->t_mean[i] = -dtau;
    }
    free(g2);
    free(ids);
    free(buf);
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
