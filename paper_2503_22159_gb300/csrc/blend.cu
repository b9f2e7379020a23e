// blend.cu -- K6: per-pixel front-to-back alpha compositing over each tile's
// depth-ordered list (Eq. 4; alpha_i = o_hat_i G'_i with the 2D Gaussian of
// Eq. 1 evaluated through its conic):
//
//   p = -1/2 (a dx^2 + c dy^2) - b dx dy,  skip p > 0
//   alpha = min(0.99, o_hat e^p),          skip alpha < 1/255
//   stop (before blending) once T (1 - alpha) < 1e-4
//   C += alpha T c;  T *= 1 - alpha;       out = C + T bg
//
// One CTA per tile; each thread owns two vertically adjacent pixels, so dx and
// its products are shared, and a warp covers a compact TS x (64/TS) block whose
// pixels tend to stop at similar depths.  The CTA walks the tile's list in
// batches: each batch of Gaussians is gathered once into shared memory (already
// scaled to base-2 exponent form) and read back by every thread as broadcast
// loads; a CTA leaves as soon as all of its pixels have stopped.
//
// Exponent form: with A = -a/2 log2(e), B = -b log2(e), C = -c/2 log2(e) and
// L = log2(o_hat), q = A dx^2 + B dx dy + C dy^2 + L and alpha = min(0.99, 2^q),
// so the alpha >= 1/255 test is q >= log2(1/255), taken before the exp: most
// pairs are rejected with five FMAs and two compares.  No tensor cores:
// nothing here is a dense contraction; the bound is FP32 issue.
#include "d4dgs_internal.cuh"

namespace d4dgs {

namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLog2AlphaMin = -7.9943534368588578f;   // log2(1/255)

struct PixelState {
    float T, c0, c1, c2;
    uint32_t last;
    bool done;
};

// One (pixel, Gaussian) step; returns true if the pixel blended it.
__device__ __forceinline__ bool blend_step(PixelState &px, float p, float L, const float4 *col, uint32_t pos) {
    if (p > 0.0f) return false;
    const float q = p + L;
    if (q < kLog2AlphaMin) return false;
    const float alpha = fminf(kAlphaMax, exp2f(q));
    const float test = px.T * (1.0f - alpha);
    if (test < kTMin) {
        px.done = true;
        return false;
    }
    const float4 c = *col;
    const float w = alpha * px.T;
    px.c0 = fmaf(w, c.x, px.c0);
    px.c1 = fmaf(w, c.y, px.c1);
    px.c2 = fmaf(w, c.z, px.c2);
    px.T = test;
    px.last = pos;
    return true;
}

// COUNT: instrumented variant for profiling, which also totals the (pixel,
// Gaussian) pairs evaluated and blended into counts[0..1] (not used on the
// render path).
template <int TS, int BATCH, bool COUNT>
__global__ void __launch_bounds__(TS *TS / 2)
blend_kernel(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ ids, uint32_t id_mask,
             const float4 *__restrict__ rec, uint32_t n, uint32_t cap, int width, int height, int tiles_x,
             float bg0, float bg1, float bg2, float *__restrict__ out_rgb, float *__restrict__ out_T,
             uint32_t *__restrict__ out_nc, unsigned long long *counts) {
    constexpr int NT = TS * TS / 2;
    __shared__ float4 s_g[BATCH];    // u, v, A, B
    __shared__ float2 s_h[BATCH];    // C, L
    __shared__ float4 s_c[BATCH];    // r, g, b

    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int lx = (int)(threadIdx.x % TS), ly = 2 * (int)(threadIdx.x / TS);
    const int px = tx * TS + lx, py0 = ty * TS + ly, py1 = py0 + 1;
    const bool in0 = px < width && py0 < height, in1 = px < width && py1 < height;
    const float pxf = (float)px + 0.5f, pyf0 = (float)py0 + 0.5f, pyf1 = (float)py1 + 0.5f;
    uint2 rg = ranges[tile];
    rg.y = min(rg.y, cap);   // ranges are written clamped; this keeps every read in bounds regardless
    rg.x = min(rg.x, rg.y);

    PixelState a{1.0f, 0.0f, 0.0f, 0.0f, 0u, !in0};
    PixelState b{1.0f, 0.0f, 0.0f, 0.0f, 0u, !in1};
    uint32_t n_eval = 0, n_blend = 0;

    for (uint32_t start = rg.x; start < rg.y; start += BATCH) {
        if (__syncthreads_count(!(a.done && b.done)) == 0) break;
        for (int k = threadIdx.x; k < BATCH; k += NT) {
            const uint32_t j = start + (uint32_t)k;
            if (j < rg.y) {
                uint32_t id = ids[j] & id_mask;
                if (id >= n) id = 0;   // only after a timed-out sort pass; keeps the gather in bounds
                const float4 r0 = rec[3 * (size_t)id + 0];
                const float4 r1 = rec[3 * (size_t)id + 1];
                const float4 r2 = rec[3 * (size_t)id + 2];
                s_g[k] = make_float4(r0.x, r0.y, -0.5f * kLog2e * r0.z, -kLog2e * r0.w);
                s_h[k] = make_float2(-0.5f * kLog2e * r1.x, r2.w);
                s_c[k] = r2;
            }
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)BATCH, rg.y - start);
        if (!(a.done && b.done)) {
            for (int k = 0; k < nb; k++) {
                const float4 g = s_g[k];
                const float2 h = s_h[k];
                const float dx = g.x - pxf;
                const float axx = g.z * dx * dx, bx = g.w * dx;
                const uint32_t pos = start - rg.x + (uint32_t)k + 1u;
                if (!a.done) {
                    const float dy = g.y - pyf0;
                    const float p = fmaf(fmaf(h.x, dy, bx), dy, axx);
                    const bool bl = blend_step(a, p, h.y, &s_c[k], pos);
                    if (COUNT) { n_eval++; n_blend += bl; }
                }
                if (!b.done) {
                    const float dy = g.y - pyf1;
                    const float p = fmaf(fmaf(h.x, dy, bx), dy, axx);
                    const bool bl = blend_step(b, p, h.y, &s_c[k], pos);
                    if (COUNT) { n_eval++; n_blend += bl; }
                }
                if (a.done && b.done) break;
            }
        }
    }
    if (in0) {
        const size_t p = (size_t)py0 * width + px;
        out_rgb[3 * p + 0] = a.c0 + a.T * bg0;
        out_rgb[3 * p + 1] = a.c1 + a.T * bg1;
        out_rgb[3 * p + 2] = a.c2 + a.T * bg2;
        out_T[p] = a.T;
        out_nc[p] = a.last;
    }
    if (in1) {
        const size_t p = (size_t)py1 * width + px;
        out_rgb[3 * p + 0] = b.c0 + b.T * bg0;
        out_rgb[3 * p + 1] = b.c1 + b.T * bg1;
        out_rgb[3 * p + 2] = b.c2 + b.T * bg2;
        out_T[p] = b.T;
        out_nc[p] = b.last;
    }
    if (COUNT) {
        const unsigned long long e = __reduce_add_sync(0xFFFFFFFFu, n_eval);
        const unsigned long long bb = __reduce_add_sync(0xFFFFFFFFu, n_blend);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(counts + 0, e);
            atomicAdd(counts + 1, bb);
        }
    }
}

// The Gaussian id of sorted pair j is ids[j] & id_mask.
const uint32_t *pair_ids(const Layout &L, void *ws) {
    return at<uint32_t>(ws, L.packed ? L.tile_keys[L.final_buf()] : L.tile_vals[L.final_buf()]);
}
uint32_t id_mask(const Layout &L) { return L.packed ? (uint32_t)((1ull << L.id_bits) - 1ull) : 0xFFFFFFFFu; }

template <int TS, int BATCH>
cudaError_t launch_ts(const Layout &L, const d4dgs_config &cfg, void *ws, float *out_rgb, cudaStream_t st,
                      unsigned long long *counts) {
    auto args = [&](auto kernel) {
        kernel<<<L.ntiles, TS * TS / 2, 0, st>>>(at<uint2>(ws, L.ranges), pair_ids(L, ws), id_mask(L),
                                                 at<float4>(ws, L.records), (uint32_t)L.n, (uint32_t)L.cap,
                                                 L.width, L.height, L.tiles_x, cfg.bg[0], cfg.bg[1], cfg.bg[2],
                                                 out_rgb, at<float>(ws, L.final_T), at<uint32_t>(ws, L.n_contrib),
                                                 counts);
    };
    if (counts) args(blend_kernel<TS, BATCH, true>);
    else args(blend_kernel<TS, BATCH, false>);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blend(const Layout &L, const d4dgs_config &cfg, void *ws, float *out_rgb, cudaStream_t st,
                         unsigned long long *counts) {
    if (L.ntiles == 0) return cudaSuccess;
#define D4DGS_BATCHES(TS)                                                           \
    if (cfg.batch == 64) return launch_ts<TS, 64>(L, cfg, ws, out_rgb, st, counts);   \
    if (cfg.batch == 128) return launch_ts<TS, 128>(L, cfg, ws, out_rgb, st, counts); \
    if (cfg.batch == 256) return launch_ts<TS, 256>(L, cfg, ws, out_rgb, st, counts); \
    return cudaErrorInvalidValue;
    switch (L.tile) {
        case 8: D4DGS_BATCHES(8)
        case 16: D4DGS_BATCHES(16)
        case 32: D4DGS_BATCHES(32)
        default: return cudaErrorInvalidValue;
    }
#undef D4DGS_BATCHES
}

}  // namespace d4dgs
