// backward.cu -- adjoint of the frame render ("differentiable projection-first
// splatting", Sec. III-B-2), in two kernels:
//
// K7 blend_backward_kernel: one CTA per tile replays the tile's list back to
//   front from the last entry each pixel walked before it stopped (the entry
//   that stopped it is not blended; entries that do not pass the alpha test
//   are skipped as in the forward), recovering T_i = T_{i+1} /
//   (1 - alpha_i) from the stored final T (no per-pixel lists are kept), with
//   G = dL/dC and B = the colour behind (B <- alpha c + (1 - alpha) B):
//     dL/dc_i = alpha_i T_i G,   dL/dalpha_i = T_i G.(c_i - B)
//     alpha = min(0.99, o_hat e^p): dalpha/dp = alpha, dalpha/do_hat = e^p
//     p = -1/2 (a dx^2 + c dy^2) - b dx dy  ->  d/du, d/dv, d/da, d/db, d/dc
//   alpha is recomputed with exactly the forward's single-precision operations,
//   so every skip / blend decision matches the forward.  Per-Gaussian sums
//   (u, v, a, b, c, o_hat, r, g, b) are reduced over each warp only when a
//   lane contributed, gathered per batch in shared memory and added to global
//   memory once per (tile, Gaussian).
// K8 preprocess_backward_kernel: one thread per Gaussian, the chain rule of
//   the preprocess in reverse (conic -> Sigma' -> J W M -> J(X), R(q), scales;
//   (u, v)(X); SH colour and its view direction; X(mu(t)); mu(t) = mu + tau V;
//   o_hat(logit, tau, log s_t); tau = t - mu_t), writing every raw gradient.
#include "blend_common.cuh"
#include "blend_mask.cuh"
#include "d4dgs_internal.cuh"

namespace d4dgs {

namespace {

constexpr int kG2 = 12;   // floats per Gaussian in the 2D gradient buffer (9 used)

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Warp sums of 8 values at once: three exchange steps (offsets 16, 8, 4) each
// hand half of a lane's remaining values to its partner and keep the sums of
// the other half, then two plain steps (offsets 2, 1) finish a single value.
// 9 shuffles instead of 40; afterwards lane L holds the total of value
// ((L >> 4) & 1) * 4 + ((L >> 3) & 1) * 2 + ((L >> 2) & 1).
__device__ __forceinline__ float warp_sum8(const float (&x)[8], int lane) {
    float v4[4], v2[2];
    const bool h16 = (lane >> 4) & 1, h8 = (lane >> 3) & 1, h4 = (lane >> 2) & 1;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const float send = h16 ? x[j] : x[j + 4], keep = h16 ? x[j + 4] : x[j];
        v4[j] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 16);
    }
#pragma unroll
    for (int j = 0; j < 2; j++) {
        const float send = h8 ? v4[j] : v4[j + 2], keep = h8 ? v4[j + 2] : v4[j];
        v2[j] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 8);
    }
    float v = (h4 ? v2[1] : v2[0]) + __shfl_xor_sync(0xFFFFFFFFu, h4 ? v2[0] : v2[1], 4);
    v += __shfl_xor_sync(0xFFFFFFFFu, v, 2);
    v += __shfl_xor_sync(0xFFFFFFFFu, v, 1);
    return v;
}

// K7: one CTA per tile, the forward's pixel layout (a column of PX pixels per
// thread, a warp per 8 x 4PX block).  The tile's list is staged in batches
// from the back (with the forward's per-block masks); each warp walks its
// Gaussians from the highest position down, skipping those whose
// alpha >= 1/255 ellipse misses its block or that lie past every pixel's
// walked range.  Per pixel the exponent is the forward's, so the same pairs
// pass and alpha has the same bits.  A thread's pixels are worked as pixel
// pairs in packed FP32x2 (a pixel that does not take the pair contributes
// alpha = 0: T, B and the sums stay as they are).  Since the thread's pixels
// share dx, the geometric gradients need only three sums per thread,
//   A0 = sum dp, A1 = sum dp dy, A2 = sum dp dy^2   (dp = dL/dalpha alpha),
// and, over the warp, the six moments sum dp, dp dx, dp dx^2, dp dy, dp dx dy,
// dp dy^2 (with dx per thread) plus the colour sums: one 9-value warp
// reduction per (warp, Gaussian) into shared memory.  When a batch is
// flushed the moments become the gradients of the 2D Gaussian, once per
// (tile, Gaussian):
//   dL/du = -(a M_x + b M_y), dL/dv = -(b M_x + c M_y), dL/da = -M_xx / 2,
//   dL/db = -M_xy, dL/dc = -M_yy / 2, dL/do_hat = M_0 / o_hat
// (M_x = sum dp dx, M_y = sum dp dy, ...; p = -(a dx^2 + c dy^2)/2 - b dx dy).
// FLOW: the forward also composited the screen flow; dl_dflow (H x W x 2)
// adds its terms to dL/dalpha and gives dL/d(flow) of every Gaussian.
template <int TS, int BATCH, bool FLOW = false>
__global__ void __launch_bounds__(BlendShape<TS>::NT, TS == 8 ? 16 : (TS == 16 ? 8 : 3))
blend_backward_kernel(const char *__restrict__ ba, const float *__restrict__ dl_drgb,
                      const float *__restrict__ dl_dflow, const __grid_constant__ View v) {
    grid_dependency_wait();
    using S = BlendShape<TS>;
    constexpr int PX = S::PX, NP = S::NP, BH = S::BH, NT = S::NT, BX = S::BX;
    constexpr int NA = FLOW ? 11 : 9;   // shared sums per staged Gaussian
    const uint32_t id_mask = v.packed ? (uint32_t)((1ull << v.id_bits) - 1ull) : 0xFFFFFFFFu;
    const uint32_t *ids = v.packed ? v.tkeys[v.tile_passes & 1] : v.tvals[v.tile_passes & 1];
    const float4 *rec = v.rec;
    const uint32_t n = (uint32_t)v.n, cap = v.cap;
    const int width = v.cam.width, height = v.cam.height, tiles_x = v.cam.tiles_x;
    float *g2 = v.grad2d;
    // the staged batch in dynamic shared memory (k7_smem bytes)
    extern __shared__ float4 s_dyn4[];
    float4 *s_ua = s_dyn4;            // u, u, A, A (forward exponent form, pairs)
    float4 *s_bc = s_ua + BATCH;      // B, B, C, C
    float4 *s_vl = s_bc + BATCH;      // v, v, L, L
    float4 *s_c = s_vl + BATCH;       // r, g, b
    float4 *s_k = s_c + BATCH;        // a, b, c, o_hat (natural conic)
    uint32_t *s_m = reinterpret_cast<uint32_t *>(s_k + BATCH);   // blocks the alpha >= 1/255 ellipse reaches
    uint32_t *s_id = s_m + BATCH;
    float2 *s_f = reinterpret_cast<float2 *>(s_id + BATCH);      // screen flow (FLOW)
    // moments M_0, M_x, M_xx, M_y, M_xy, M_yy, colour sums r, g, b (, flow u, v)
    float (*s_acc)[NA] = reinterpret_cast<float (*)[NA]>(s_f + (FLOW ? BATCH : 0));
    __shared__ uint32_t s_maxw;

    int tile = blockIdx.x;
    {   // the forward's tile order: longest lists first; kept in range whatever the buffer holds
        const uint32_t o = v.tile_order[tile];
        if (o < (uint32_t)v.ntiles) tile = (int)o;
    }
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int x0 = tx * TS, y0 = ty * TS;
    const int lane = (int)(threadIdx.x & 31u), warp = (int)(threadIdx.x >> 5);
    const int px = x0 + 8 * (warp % BX) + (lane & 7);
    const int py = y0 + BH * (warp / BX) + PX * (lane >> 3);
    const float pxf = (float)px + 0.5f;
    const float2 pxf2 = make_float2(pxf, pxf);
    uint2 rg = v.ranges[tile];
    rg.y = min(rg.y, cap);
    rg.x = min(rg.x, rg.y);
    const uint32_t len = rg.y - rg.x;

    float2 pyf[NP], T[NP], G[NP][3], Bc[NP][3], GF[FLOW ? NP : 1][2], BF[FLOW ? NP : 1][2];
    uint32_t walked[PX];
    uint32_t tmax = 0;
#pragma unroll
    for (int j = 0; j < NP; j++) {
        pyf[j] = make_float2((float)(py + 2 * j) + 0.5f, (float)(py + 2 * j + 1) + 0.5f);
        T[j] = make_float2(1.0f, 1.0f);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            G[j][c] = make_float2(0.0f, 0.0f);
            Bc[j][c] = make_float2(v.bg[c], v.bg[c]);
        }
        if (FLOW) {
            GF[FLOW ? j : 0][0] = GF[FLOW ? j : 0][1] = make_float2(0.0f, 0.0f);
            BF[FLOW ? j : 0][0] = BF[FLOW ? j : 0][1] = make_float2(0.0f, 0.0f);
        }
    }
#pragma unroll
    for (int i = 0; i < PX; i++) {
        walked[i] = 0;
        if (px < width && py + i < height) {
            const size_t p = (size_t)(py + i) * width + px;
            float *tj = (i & 1) ? &T[i >> 1].y : &T[i >> 1].x;
            *tj = v.final_T[p];
            walked[i] = min(v.n_contrib[p], len);
#pragma unroll
            for (int c = 0; c < 3; c++) ((i & 1) ? G[i >> 1][c].y : G[i >> 1][c].x) = dl_drgb[3 * p + c];
            if (FLOW) {
                ((i & 1) ? GF[FLOW ? i >> 1 : 0][0].y : GF[FLOW ? i >> 1 : 0][0].x) = dl_dflow[2 * p];
                ((i & 1) ? GF[FLOW ? i >> 1 : 0][1].y : GF[FLOW ? i >> 1 : 0][1].x) = dl_dflow[2 * p + 1];
            }
        }
        tmax = max(tmax, walked[i]);
    }
    const uint32_t wmax = __reduce_max_sync(0xFFFFFFFFu, tmax);
    if (threadIdx.x == 0) s_maxw = 0;
    __syncthreads();
    if (lane == 0) atomicMax(&s_maxw, wmax);
    __syncthreads();
    const uint32_t maxw = s_maxw;
    const uint32_t wbit = 1u << warp;
    const float2 one2 = make_float2(1.0f, 1.0f);
    const float2 zero2 = make_float2(0.0f, 0.0f);

    // positions are 1-based: list entry rg.x + pos - 1; walk pos = maxw .. 1 in batches
    for (int32_t hi = (int32_t)maxw; hi > 0; hi -= BATCH) {
        const int32_t lo = max(hi - BATCH, 0);   // this batch covers positions lo+1 .. hi
        const int nb = hi - lo;
        for (int k = threadIdx.x; k < nb; k += NT) {
            uint32_t id = ids[rg.x + (uint32_t)(lo + k)] & id_mask;
            if (id >= n) id = 0;
            const float4 r0 = rec[3 * (size_t)id + 0];
            const float4 r1 = rec[3 * (size_t)id + 1];
            const float4 r2 = rec[3 * (size_t)id + 2];
            const float A = -0.5f * kLog2e * r0.z, B = -kLog2e * r0.w, C = -0.5f * kLog2e * r1.x;
            s_ua[k] = make_float4(r0.x, r0.x, A, A);
            s_bc[k] = make_float4(B, B, C, C);
            s_vl[k] = make_float4(r0.y, r0.y, r2.w, r2.w);
            s_c[k] = r2;
            s_k[k] = make_float4(r0.z, r0.w, r1.x, r1.y);
            s_m[k] = d4dgs::block_mask<TS, BH>(r0.x, r0.y, A, B, C, r2.w, x0, y0);
            s_id[k] = id;
            if (FLOW) s_f[FLOW ? k : 0] = v.flow2d[id];
#pragma unroll
            for (int j = 0; j < NA; j++) s_acc[k][j] = 0.0f;
        }
        __syncthreads();
        if ((uint32_t)lo < wmax) {
            // chunks of 32 from the top of the batch; within a chunk, set bits from the highest
            for (int k0 = ((nb - 1) / 32) * 32; k0 >= 0; k0 -= 32) {
                const int kl = k0 + lane;
                const bool want = kl < nb && (s_m[kl] & wbit) != 0u && (uint32_t)(lo + kl) < wmax;
                uint32_t bits = __ballot_sync(0xFFFFFFFFu, want);
                while (bits) {
                    const int b = 31 - __clz((int)bits);
                    bits &= ~(1u << b);
                    const int k = k0 + b;
                    const uint32_t pos = (uint32_t)(lo + k + 1);
                    const float4 ua = s_ua[k], bc = s_bc[k], vl = s_vl[k];
                    const float2 dx2 = f2_sub(make_float2(ua.x, ua.y), pxf2);
                    const float2 axx = f2_mul(f2_mul(make_float2(ua.z, ua.w), dx2), dx2);
                    const float2 bx = f2_mul(make_float2(bc.x, bc.y), dx2);
                    float2 dy[NP], qv[NP];
                    bool e[PX];
                    bool any = false;
#pragma unroll
                    for (int j = 0; j < NP; j++) {
                        const float2 d = f2_sub(make_float2(vl.x, vl.y), pyf[j]);
                        const float2 pp = f2_fma(f2_fma(make_float2(bc.z, bc.w), d, bx), d, axx);
                        qv[j] = f2_add(pp, make_float2(vl.z, vl.w));
                        dy[j] = d;
                        e[2 * j] = pos <= walked[2 * j] && pp.x <= 0.0f && qv[j].x >= kLog2AlphaMin;
                        e[2 * j + 1] = pos <= walked[2 * j + 1] && pp.y <= 0.0f && qv[j].y >= kLog2AlphaMin;
                        any |= e[2 * j] | e[2 * j + 1];
                    }
                    // per thread: colour sums and the three dp moments (FLOW: flow sums), as pairs
                    float2 sr = zero2, sg = zero2, sb = zero2, m0 = zero2, m1 = zero2, m2 = zero2;
                    float2 sfu = zero2, sfv = zero2;
                    if (any) {
                        const float4 c = s_c[k];
                        const float2 cr = make_float2(c.x, c.x), cg = make_float2(c.y, c.y), cb = make_float2(c.z, c.z);
                        const float2 fl = FLOW ? s_f[FLOW ? k : 0] : make_float2(0.0f, 0.0f);
#pragma unroll
                        for (int j = 0; j < NP; j++) {
                            const bool ex = e[2 * j], ey = e[2 * j + 1];
                            if (!(ex | ey)) continue;
                            const float rx = ex ? alpha_exp2(qv[j].x) : 0.0f, ry = ey ? alpha_exp2(qv[j].y) : 0.0f;
                            const float2 al = make_float2(fminf(kAlphaMax, rx), fminf(kAlphaMax, ry));
                            const float2 Ti = make_float2(__fdividef(T[j].x, 1.0f - al.x), __fdividef(T[j].y, 1.0f - al.y));
                            const float2 w = f2_mul(al, Ti);
                            sr = f2_fma(w, G[j][0], sr);
                            sg = f2_fma(w, G[j][1], sg);
                            sb = f2_fma(w, G[j][2], sb);
                            const float2 d0 = f2_sub(cr, Bc[j][0]), d1 = f2_sub(cg, Bc[j][1]), d2 = f2_sub(cb, Bc[j][2]);
                            float2 gs = f2_fma(G[j][2], d2, f2_fma(G[j][1], d1, f2_mul(G[j][0], d0)));
                            Bc[j][0] = f2_fma(al, d0, Bc[j][0]);
                            Bc[j][1] = f2_fma(al, d1, Bc[j][1]);
                            Bc[j][2] = f2_fma(al, d2, Bc[j][2]);
                            if (FLOW) {
                                const int fj = FLOW ? j : 0;
                                sfu = f2_fma(w, GF[fj][0], sfu);
                                sfv = f2_fma(w, GF[fj][1], sfv);
                                const float2 fu = f2_sub(make_float2(fl.x, fl.x), BF[fj][0]);
                                const float2 fv = f2_sub(make_float2(fl.y, fl.y), BF[fj][1]);
                                gs = f2_fma(GF[fj][1], fv, f2_fma(GF[fj][0], fu, gs));
                                BF[fj][0] = f2_fma(al, fu, BF[fj][0]);
                                BF[fj][1] = f2_fma(al, fv, BF[fj][1]);
                            }
                            T[j] = Ti;
                            // dL/dp = dL/dalpha * alpha, none through a clamped alpha
                            float2 dp = f2_mul(f2_mul(Ti, gs), al);
                            if (rx > kAlphaMax) dp.x = 0.0f;
                            if (ry > kAlphaMax) dp.y = 0.0f;
                            const float2 dpy = f2_mul(dp, dy[j]);
                            m0 = f2_add(m0, dp);
                            m1 = f2_add(m1, dpy);
                            m2 = f2_fma(dpy, dy[j], m2);
                        }
                    }
                    if (__any_sync(0xFFFFFFFFu, any)) {
                        const float dx = dx2.x;
                        const float a0 = m0.x + m0.y, a1 = m1.x + m1.y;
                        const float x8[8] = {a0, dx * a0, dx * dx * a0, a1, dx * a1, m2.x + m2.y, sr.x + sr.y, sg.x + sg.y};
                        const float tot = warp_sum8(x8, lane);
                        const float tb = warp_sum(sb.x + sb.y);
                        if ((lane & 3) == 0) {   // lanes 0, 4, .., 28 hold values 0..7
                            const int idx = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
                            atomicAdd(&s_acc[k][idx], tot);
                        }
                        if (lane == 0) atomicAdd(&s_acc[k][8], tb);
                        if (FLOW) {
                            const float tfu = warp_sum(sfu.x + sfu.y), tfv = warp_sum(sfv.x + sfv.y);
                            if (lane == 0) {
                                atomicAdd(&s_acc[k][FLOW ? 9 : 0], tfu);
                                atomicAdd(&s_acc[k][FLOW ? 10 : 0], tfv);
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        // flush: moments -> gradients of (u, v, a, b, c, o_hat, r, g, b) (, flow), one set of
        // global atomics per (tile, Gaussian) that received anything
        for (int k = threadIdx.x; k < nb; k += NT) {
            bool anyg = false;
#pragma unroll
            for (int j = 0; j < NA; j++) anyg |= s_acc[k][j] != 0.0f;
            if (anyg) {
                const float4 kk = s_k[k];   // a, b, c, o_hat
                const float M0 = s_acc[k][0], Mx = s_acc[k][1], Mxx = s_acc[k][2], My = s_acc[k][3];
                const float Mxy = s_acc[k][4], Myy = s_acc[k][5];
                float gv[NA];
                gv[0] = -(kk.x * Mx + kk.y * My);
                gv[1] = -(kk.y * Mx + kk.z * My);
                gv[2] = -0.5f * Mxx;
                gv[3] = -Mxy;
                gv[4] = -0.5f * Myy;
                gv[5] = __fdividef(M0, kk.w);
                gv[6] = s_acc[k][6];
                gv[7] = s_acc[k][7];
                gv[8] = s_acc[k][8];
                if (FLOW) {
                    gv[FLOW ? 9 : 0] = s_acc[k][FLOW ? 9 : 0];
                    gv[FLOW ? 10 : 0] = s_acc[k][FLOW ? 10 : 0];
                }
                float *dst = g2 + (size_t)s_id[k] * kG2;
#pragma unroll
                for (int j = 0; j < NA; j++)
                    if (gv[j] != 0.0f) atomicAdd(dst + j, gv[j]);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// K8
constexpr float kC1 = 0.48860251190291992f;   // sqrt(3/(4 pi))
constexpr float kC2a = 1.0925484305920792f;   // sqrt(15/pi)/2
constexpr float kC2b = 0.31539156525252005f;  // sqrt(5/pi)/4
constexpr float kC2c = 0.54627421529603959f;  // sqrt(15/pi)/4
constexpr float kC3e = 0.59004358992664352f;  // sqrt(35/(2 pi))/4
constexpr float kC3f = 2.8906114426405538f;   // sqrt(105/pi)/2
constexpr float kC3g = 0.45704579946446577f;  // sqrt(21/(2 pi))/4
constexpr float kC3h = 0.3731763325901154f;   // sqrt(7/pi)/4
constexpr float kC3k = 1.4453057213202769f;   // sqrt(105/pi)/4
constexpr float kC0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))

// SH basis and its partial derivatives in x, y, z (independent variables).
template <int DEG>
__device__ __forceinline__ void sh_basis_and_grad(float x, float y, float z, float *Y, float (*dY)[3]) {
#pragma unroll
    for (int k = 0; k < 16; k++) dY[k][0] = dY[k][1] = dY[k][2] = 0.0f;
    Y[0] = kC0;
    if (DEG >= 1) {
        Y[1] = -kC1 * y; dY[1][1] = -kC1;
        Y[2] = kC1 * z;  dY[2][2] = kC1;
        Y[3] = -kC1 * x; dY[3][0] = -kC1;
    }
    if (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kC2a * x * y;                 dY[4][0] = kC2a * y; dY[4][1] = kC2a * x;
        Y[5] = -kC2a * y * z;                dY[5][1] = -kC2a * z; dY[5][2] = -kC2a * y;
        Y[6] = kC2b * (2.0f * zz - xx - yy); dY[6][0] = -2.0f * kC2b * x; dY[6][1] = -2.0f * kC2b * y; dY[6][2] = 4.0f * kC2b * z;
        Y[7] = -kC2a * x * z;                dY[7][0] = -kC2a * z; dY[7][2] = -kC2a * x;
        Y[8] = kC2c * (xx - yy);             dY[8][0] = 2.0f * kC2c * x; dY[8][1] = -2.0f * kC2c * y;
        if (DEG >= 3) {
            Y[9] = -kC3e * y * (3.0f * xx - yy);
            dY[9][0] = -6.0f * kC3e * x * y; dY[9][1] = -kC3e * (3.0f * xx - 3.0f * yy);
            Y[10] = kC3f * x * y * z;
            dY[10][0] = kC3f * y * z; dY[10][1] = kC3f * x * z; dY[10][2] = kC3f * x * y;
            Y[11] = -kC3g * y * (4.0f * zz - xx - yy);
            dY[11][0] = 2.0f * kC3g * x * y; dY[11][1] = -kC3g * (4.0f * zz - xx - 3.0f * yy); dY[11][2] = -8.0f * kC3g * y * z;
            Y[12] = kC3h * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
            dY[12][0] = -6.0f * kC3h * x * z; dY[12][1] = -6.0f * kC3h * y * z; dY[12][2] = kC3h * (6.0f * zz - 3.0f * xx - 3.0f * yy);
            Y[13] = -kC3g * x * (4.0f * zz - xx - yy);
            dY[13][0] = -kC3g * (4.0f * zz - 3.0f * xx - yy); dY[13][1] = 2.0f * kC3g * x * y; dY[13][2] = -8.0f * kC3g * x * z;
            Y[14] = kC3k * z * (xx - yy);
            dY[14][0] = 2.0f * kC3k * x * z; dY[14][1] = -2.0f * kC3k * y * z; dY[14][2] = kC3k * (xx - yy);
            Y[15] = -kC3e * x * (xx - 3.0f * yy);
            dY[15][0] = -kC3e * (3.0f * xx - 3.0f * yy); dY[15][1] = 6.0f * kC3e * x * y;
        }
    }
}

struct SceneArgs {
    const float *means, *t_mean, *velocity, *log_scales, *log_t_scale, *quats, *opacity_logit, *sh;
};
struct GradArgs {
    float *means, *t_mean, *velocity, *log_scales, *log_t_scale, *quats, *opacity_logit, *sh;
};

// ACC: add to the gradient arrays instead of overwriting them (several views of one step).
template <int DEG, bool ACC>
__global__ void __launch_bounds__(256)
preprocess_backward_kernel(const char *__restrict__ ba, GradArgs o, const __grid_constant__ View vw) {
    grid_dependency_wait();
    const SceneArgs s{vw.means, vw.t_mean, vw.velocity, vw.log_scales, vw.log_t_scale, vw.quats, vw.opacity_logit,
                      vw.sh};
    const CamArgs &c = vw.cam;
    const float t = vw.t;
    const int n = vw.n;
    const float4 *__restrict__ rec = vw.rec;
    const uint32_t *__restrict__ tiles_touched = vw.tiles_touched;
    const float *__restrict__ g2 = vw.grad2d;
    constexpr int K = (DEG + 1) * (DEG + 1);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float *gsh = o.sh + (size_t)i * 3 * K;
    if (tiles_touched[i] == 0) {   // culled or off screen: no pixel depends on it
        if (ACC) return;
        for (int j = 0; j < 3; j++) o.means[3 * i + j] = o.velocity[3 * i + j] = o.log_scales[3 * i + j] = 0.0f;
        for (int j = 0; j < 4; j++) o.quats[4 * i + j] = 0.0f;
        for (int j = 0; j < 3 * K; j++) gsh[j] = 0.0f;
        o.t_mean[i] = o.log_t_scale[i] = o.opacity_logit[i] = 0.0f;
        return;
    }
    // stores of the raw gradients: overwrite, or add (ACC)
    auto put = [](float *p, float v) {
        if (ACC) *p += v;
        else *p = v;
    };
    // the 2D gradient sums (12 floats, 16-byte aligned): three vector loads
    const float4 *G4 = reinterpret_cast<const float4 *>(g2 + (size_t)i * kG2);
    const float4 Ga = G4[0], Gb = G4[1], Gc = G4[2];
    const float gU = Ga.x, gV = Ga.y, gA = Ga.z, gB = Ga.w, gCc = Gb.x, gO = Gb.y;
    const float gcol[3] = {Gb.z, Gb.w, Gc.x};
    const float gFu = Gc.y, gFv = Gc.z;   // screen flow (zero unless the frame had a flow channel)
    // ---- forward quantities (the decisions use the forward's rounded operations)
    const float tau = __fsub_rn(t, s.t_mean[i]);
    const float vel[3] = {s.velocity[3 * i], s.velocity[3 * i + 1], s.velocity[3 * i + 2]};
    const float m[3] = {__fadd_rn(s.means[3 * i], __fmul_rn(tau, vel[0])),
                        __fadd_rn(s.means[3 * i + 1], __fmul_rn(tau, vel[1])),
                        __fadd_rn(s.means[3 * i + 2], __fmul_rn(tau, vel[2]))};
    const float *R = c.R;
    float Xc[3];
#pragma unroll
    for (int r = 0; r < 3; r++)
        Xc[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(R[3 * r], m[0]), __fmul_rn(R[3 * r + 1], m[1])),
                                    __fmul_rn(R[3 * r + 2], m[2])), c.T[r]);
    const float Z = Xc[2];
    const float xz = __fdiv_rn(Xc[0], Z), yz = __fdiv_rn(Xc[1], Z);
    const float limx = c.limx, limy = c.limy;
    const bool clx = xz < -limx || xz > limx, cly = yz < -limy || yz > limy;
    const float xzc = fminf(limx, fmaxf(-limx, xz)), yzc = fminf(limy, fmaxf(-limy, yz));
    const float iz = 1.0f / Z;
    const float J00 = c.fx * iz, J02 = -c.fx * xzc * iz, J11 = c.fy * iz, J12 = -c.fy * yzc * iz;
    const float4 q4 = reinterpret_cast<const float4 *>(s.quats)[i];
    const float qraw[4] = {q4.x, q4.y, q4.z, q4.w};
    const float qn = sqrtf(qraw[0] * qraw[0] + qraw[1] * qraw[1] + qraw[2] * qraw[2] + qraw[3] * qraw[3]);
    const float qw = qraw[0] / qn, qx = qraw[1] / qn, qy = qraw[2] / qn, qz = qraw[3] / qn;
    const float Rq[9] = {1.0f - 2.0f * (qy * qy + qz * qz), 2.0f * (qx * qy - qw * qz), 2.0f * (qx * qz + qw * qy),
                         2.0f * (qx * qy + qw * qz), 1.0f - 2.0f * (qx * qx + qz * qz), 2.0f * (qy * qz - qw * qx),
                         2.0f * (qx * qz - qw * qy), 2.0f * (qy * qz + qw * qx), 1.0f - 2.0f * (qx * qx + qy * qy)};
    const float sc[3] = {expf(s.log_scales[3 * i]), expf(s.log_scales[3 * i + 1]), expf(s.log_scales[3 * i + 2])};
    float M[9];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int k = 0; k < 3; k++) M[3 * r + k] = Rq[3 * r + k] * sc[k];
    float Tm[6];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        Tm[j] = J00 * R[j] + J02 * R[6 + j];
        Tm[3 + j] = J11 * R[3 + j] + J12 * R[6 + j];
    }
    float TM[6];
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
        for (int k = 0; k < 3; k++) TM[3 * r + k] = Tm[3 * r] * M[k] + Tm[3 * r + 1] * M[3 + k] + Tm[3 * r + 2] * M[6 + k];
    const float s00 = TM[0] * TM[0] + TM[1] * TM[1] + TM[2] * TM[2] + kDilation;
    const float s01 = TM[0] * TM[3] + TM[1] * TM[4] + TM[2] * TM[5];
    const float s11 = TM[3] * TM[3] + TM[4] * TM[4] + TM[5] * TM[5] + kDilation;
    const float det = s00 * s11 - s01 * s01;
    const float id2 = 1.0f / (det * det), idet = 1.0f / det;
    // ---- conic -> Sigma'
    const float d00 = gA * (-s11 * s11 * id2) + gB * (s01 * s11 * id2) + gCc * (idet - s00 * s11 * id2);
    const float d11 = gA * (idet - s11 * s00 * id2) + gB * (s01 * s00 * id2) + gCc * (-s00 * s00 * id2);
    const float d01 = gA * (2.0f * s11 * s01 * id2) + gB * (-idet - 2.0f * s01 * s01 * id2) + gCc * (2.0f * s00 * s01 * id2);
    // ---- Sigma' = TM TM^T + 0.3 I -> TM -> Tm, M -> J
    float dTM[6];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        dTM[k] = 2.0f * d00 * TM[k] + d01 * TM[3 + k];
        dTM[3 + k] = 2.0f * d11 * TM[3 + k] + d01 * TM[k];
    }
    float dTm[6], dM[9];
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
        for (int k = 0; k < 3; k++) dTm[3 * r + k] = dTM[3 * r] * M[3 * k] + dTM[3 * r + 1] * M[3 * k + 1] + dTM[3 * r + 2] * M[3 * k + 2];
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int cc = 0; cc < 3; cc++) dM[3 * k + cc] = Tm[k] * dTM[cc] + Tm[3 + k] * dTM[3 + cc];
    const float dJ00 = dTm[0] * R[0] + dTm[1] * R[1] + dTm[2] * R[2];
    const float dJ02 = dTm[0] * R[6] + dTm[1] * R[7] + dTm[2] * R[8];
    const float dJ11 = dTm[3] * R[3] + dTm[4] * R[4] + dTm[5] * R[5];
    const float dJ12 = dTm[3] * R[6] + dTm[4] * R[7] + dTm[5] * R[8];
    // ---- J(X), (u, v)(X) -> X
    float dX[3] = {0.0f, 0.0f, 0.0f};
    const float iz2 = iz * iz;
    dX[2] += -dJ00 * c.fx * iz2 - dJ11 * c.fy * iz2;
    if (!clx) { dX[0] += -dJ02 * c.fx * iz2; dX[2] += dJ02 * 2.0f * c.fx * Xc[0] * iz2 * iz; }
    else dX[2] += dJ02 * c.fx * xzc * iz2;
    if (!cly) { dX[1] += -dJ12 * c.fy * iz2; dX[2] += dJ12 * 2.0f * c.fy * Xc[1] * iz2 * iz; }
    else dX[2] += dJ12 * c.fy * yzc * iz2;
    dX[0] += gU * c.fx * iz;
    dX[2] += -gU * c.fx * Xc[0] * iz2;
    dX[1] += gV * c.fy * iz;
    dX[2] += -gV * c.fy * Xc[1] * iz2;
    // ---- screen flow f = (fx Vc_x / Z, fy Vc_y / Z), Vc = R V: depth and camera-frame velocity
    const float Vcx = R[0] * vel[0] + R[1] * vel[1] + R[2] * vel[2], Vcy = R[3] * vel[0] + R[4] * vel[1] + R[5] * vel[2];
    dX[2] += -(gFu * c.fx * Vcx + gFv * c.fy * Vcy) * iz2;
    const float dVc0 = gFu * c.fx * iz, dVc1 = gFv * c.fy * iz;
    // ---- M = R(qn) diag(s) -> quaternion, log-scales
    float dR[9];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int k = 0; k < 3; k++) dR[3 * r + k] = dM[3 * r + k] * sc[k];
#pragma unroll
    for (int k = 0; k < 3; k++)
        put(&o.log_scales[3 * i + k], (dM[k] * Rq[k] + dM[3 + k] * Rq[3 + k] + dM[6 + k] * Rq[6 + k]) * sc[k]);
    float dq[4];
    dq[0] = 2.0f * (-qz * dR[1] + qy * dR[2] + qz * dR[3] - qx * dR[5] - qy * dR[6] + qx * dR[7]);
    dq[1] = 2.0f * (qy * dR[1] + qz * dR[2] + qy * dR[3] - 2.0f * qx * dR[4] - qw * dR[5] + qz * dR[6] + qw * dR[7] - 2.0f * qx * dR[8]);
    dq[2] = 2.0f * (-2.0f * qy * dR[0] + qx * dR[1] + qw * dR[2] + qx * dR[3] + qz * dR[5] - qw * dR[6] + qz * dR[7] - 2.0f * qy * dR[8]);
    dq[3] = 2.0f * (-2.0f * qz * dR[0] - qw * dR[1] + qx * dR[2] + qw * dR[3] - 2.0f * qz * dR[4] + qy * dR[5] + qx * dR[6] + qy * dR[7]);
    const float qdot = dq[0] * qw + dq[1] * qx + dq[2] * qy + dq[3] * qz;
    const float qv[4] = {qw, qx, qy, qz};
#pragma unroll
    for (int j = 0; j < 4; j++) put(&o.quats[4 * i + j], (dq[j] - qv[j] * qdot) / qn);
    // ---- colour: clamp, SH coefficients, view direction
    float dir[3] = {m[0] - c.campos[0], m[1] - c.campos[1], m[2] - c.campos[2]};
    const float inv_n = rsqrtf(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    const float d[3] = {dir[0] * inv_n, dir[1] * inv_n, dir[2] * inv_n};
    float Yb[16], dY[16][3];
    sh_basis_and_grad<DEG>(d[0], d[1], d[2], Yb, dY);
    const float *shp = s.sh + (size_t)i * 3 * K;
    float dd[3] = {0.0f, 0.0f, 0.0f};
    if constexpr ((3 * K) % 4 == 0) {
        // 16-byte aligned rows (degree 1 and 3): the coefficients and their gradients as float4s;
        // flat index f = 3 k + ch.  Pass 1: the raw colour (clamp decisions); pass 2 (the row again,
        // from L1): the gradients of the coefficients and of the view direction.
        const float4 *sh4 = reinterpret_cast<const float4 *>(shp);
        float4 *gsh4 = reinterpret_cast<float4 *>(gsh);
        float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
        for (int j = 0; j < (3 * K) / 4; j++) {
            const float4 w4 = __ldg(sh4 + j);
            const float w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int e = 0; e < 4; e++) raw[(4 * j + e) % 3] = fmaf(w[e], Yb[(4 * j + e) / 3], raw[(4 * j + e) % 3]);
        }
        float gch[3];
#pragma unroll
        for (int ch = 0; ch < 3; ch++) gch[ch] = raw[ch] < 0.0f ? 0.0f : gcol[ch];
#pragma unroll
        for (int j = 0; j < (3 * K) / 4; j++) {
            const float4 w4 = __ldg(sh4 + j);
            const float w[4] = {w4.x, w4.y, w4.z, w4.w};
            float o[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int k = (4 * j + e) / 3, ch = (4 * j + e) % 3;
                o[e] = gch[ch] * Yb[k];
                const float gw = gch[ch] * w[e];
                dd[0] += gw * dY[k][0];
                dd[1] += gw * dY[k][1];
                dd[2] += gw * dY[k][2];
            }
            float4 ov = make_float4(o[0], o[1], o[2], o[3]);
            if (ACC) {
                const float4 prev = gsh4[j];
                ov = make_float4(prev.x + ov.x, prev.y + ov.y, prev.z + ov.z, prev.w + ov.w);
            }
            gsh4[j] = ov;
        }
    } else {
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            float raw = 0.5f;
#pragma unroll
            for (int k = 0; k < K; k++) raw = fmaf(shp[3 * k + ch], Yb[k], raw);
            const float gch = raw < 0.0f ? 0.0f : gcol[ch];
#pragma unroll
            for (int k = 0; k < K; k++) {
                put(&gsh[3 * k + ch], gch * Yb[k]);
                dd[0] += gch * shp[3 * k + ch] * dY[k][0];
                dd[1] += gch * shp[3 * k + ch] * dY[k][1];
                dd[2] += gch * shp[3 * k + ch] * dY[k][2];
            }
        }
    }
    const float ddot = dd[0] * d[0] + dd[1] * d[1] + dd[2] * d[2];
    float dm[3];
#pragma unroll
    for (int j = 0; j < 3; j++) dm[j] = (dd[j] - d[j] * ddot) * inv_n + R[j] * dX[0] + R[3 + j] * dX[1] + R[6 + j] * dX[2];
    // ---- mu(t) = mu + tau V; o_hat(tau); tau = t - mu_t
    float dtau = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        put(&o.means[3 * i + j], dm[j]);
        put(&o.velocity[3 * i + j], tau * dm[j] + R[j] * dVc0 + R[3 + j] * dVc1);
        dtau += vel[j] * dm[j];
    }
    const float oh = rec[3 * (size_t)i + 1].y;
    const float st = expf(s.log_t_scale[i]);
    const float sig = 1.0f / (1.0f + expf(-s.opacity_logit[i]));
    put(&o.opacity_logit[i], gO * oh * (1.0f - sig));
    dtau += gO * oh * (-tau / (st * st));
    put(&o.log_t_scale[i], gO * oh * tau * tau / (st * st));
    put(&o.t_mean[i], -dtau);
}

// ---------------------------------------------------------------------------
// Tile order of the replay.  A tile's replay time follows the list entries its
// pixels walked in the forward, which the blend left per tile (tile_work); taken
// in row-major order, the heaviest tiles can be among the last to start and
// leave most SMs idle while they finish.  So the replay takes the tiles
// heaviest first: (one CTA) quarter-octave classes of the work counted,
// scanned from the heaviest down and the tiles scattered (order within a
// class: whatever the atomics give; any order gives the same gradients up to
// the order of their floating-point sums).
// Block 0 orders the replay's tiles; the other blocks clear the per-Gaussian
// 2D gradient sums (n4 float4) that the replay adds into.
__global__ void __launch_bounds__(1024) backward_prologue_kernel(const char *__restrict__ ba, float4 *__restrict__ g2,
                                                                 int64_t n4, const __grid_constant__ View v) {
    grid_dependency_wait();
    if (blockIdx.x > 0) {
        const int64_t stride = (int64_t)(gridDim.x - 1) * blockDim.x;
        for (int64_t i = (int64_t)(blockIdx.x - 1) * blockDim.x + threadIdx.x; i < n4; i += stride)
            g2[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        return;
    }
    __shared__ uint32_t s_cls[kWorkClasses];
    const int T = v.ntiles, tid = threadIdx.x;
    for (int i = tid; i < kWorkClasses; i += 1024) s_cls[i] = 0u;
    __syncthreads();
    for (int t = tid; t < T; t += 1024) atomicAdd(&s_cls[work_class(v.tile_work[t])], 1u);
    __syncthreads();
    if (tid < 32) work_class_scan(s_cls);
    __syncthreads();
    for (int t = tid; t < T; t += 1024) v.tile_order[atomicAdd(&s_cls[work_class(v.tile_work[t])], 1u)] = (uint32_t)t;
}

// dynamic shared memory of a K7 CTA: the staged batch (5 float4, 2 words, the flow and the sums
// per Gaussian)
constexpr size_t k7_smem(int batch, bool flow) {
    return (size_t)batch * (5 * 16 + 2 * 4 + (flow ? 8 : 0) + 4 * (flow ? 11 : 9));
}

template <int TS, int BATCH>
void launch_bb(const char *ba, int ntiles, const float *dl, const float *dlf, cudaStream_t st, const View &v) {
    static bool attr = false;
    if (!attr) {   // above the 48 KB default
        cudaFuncSetAttribute(blend_backward_kernel<TS, BATCH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)k7_smem(BATCH, true));
        cudaFuncSetAttribute(blend_backward_kernel<TS, BATCH, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)k7_smem(BATCH, false));
        attr = true;
    }
    if (dlf)
        launch_chained(blend_backward_kernel<TS, BATCH, true>, ntiles, BlendShape<TS>::NT, k7_smem(BATCH, true), st, ba,
                       dl, dlf, v);
    else
        launch_chained(blend_backward_kernel<TS, BATCH, false>, ntiles, BlendShape<TS>::NT, k7_smem(BATCH, false), st,
                       ba, dl, static_cast<const float *>(nullptr), v);
}

template <bool ACC>
void launch_k8(int deg, int blocks, const char *ba, const GradArgs &o, cudaStream_t st, const View &v) {
    switch (deg) {
        case 0: launch_chained(preprocess_backward_kernel<0, ACC>, blocks, 256, 0, st, ba, o, v); break;
        case 1: launch_chained(preprocess_backward_kernel<1, ACC>, blocks, 256, 0, st, ba, o, v); break;
        case 2: launch_chained(preprocess_backward_kernel<2, ACC>, blocks, 256, 0, st, ba, o, v); break;
        default: launch_chained(preprocess_backward_kernel<3, ACC>, blocks, 256, 0, st, ba, o, v); break;
    }
}

}  // namespace

cudaError_t launch_backward(const BatchArgs &args, char *batch_area, const float *dl_drgb, const float *dl_dflow,
                            const d4dgs_scene_grad &g, cudaStream_t st, int num_sms, bool accumulate) {
    const View &v = args.v[0];
    if (v.n == 0) return cudaSuccess;
    // the replay's order from this frame's tile work, beside the clearing of the gradient sums; the
    // three launches chained like the forward's
    cudaError_t e = launch_chained(backward_prologue_kernel, 1 + 2 * num_sms, 1024, 0, st, (const char *)batch_area,
                                   reinterpret_cast<float4 *>(v.grad2d), (int64_t)v.n * kG2 / 4, v);
    if (e != cudaSuccess) return e;
    switch (args.tile) {   // the staging depth of the backward follows the tile size
        case 8: launch_bb<8, 64>(batch_area, v.ntiles, dl_drgb, dl_dflow, st, v); break;
        case 16: launch_bb<16, 128>(batch_area, v.ntiles, dl_drgb, dl_dflow, st, v); break;
        default: launch_bb<32, 512>(batch_area, v.ntiles, dl_drgb, dl_dflow, st, v); break;
    }
    GradArgs o{g.means, g.t_mean, g.velocity, g.log_scales, g.log_t_scale, g.quats, g.opacity_logit, g.sh};
    const int blocks = (v.n + 255) / 256;
    if (accumulate) launch_k8<true>(v.sh_degree, blocks, batch_area, o, st, v);
    else launch_k8<false>(v.sh_degree, blocks, batch_area, o, st, v);
    return cudaGetLastError();
}

}  // namespace d4dgs
