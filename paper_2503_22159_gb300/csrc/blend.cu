// blend.cu -- K6: per-pixel front-to-back alpha compositing over each tile's
// depth-ordered list (Eq. 4; alpha_i = o_hat_i G'_i with the 2D Gaussian of
// Eq. 1 evaluated through its conic):
//
//   p = -1/2 (a dx^2 + c dy^2) - b dx dy,  skip p > 0
//   alpha = min(0.99, o_hat e^p),          skip alpha < 1/255
//   stop (before blending) once T (1 - alpha) < 1e-4
//   C += alpha T c;  T *= 1 - alpha;       out = C + T bg
//
// One CTA per tile, one thread per pixel.  The CTA walks the tile's list in
// batches: each batch of Gaussian records is gathered once into shared memory
// and read back by every pixel as broadcast loads; a CTA leaves as soon as all
// of its pixels have stopped (__syncthreads_count).  No tensor cores: nothing
// here is a dense contraction; the bound is FP32 issue.
#include "d4dgs_internal.cuh"

namespace d4dgs {

namespace {

// COUNT: instrumented variant for profiling, which also totals the (pixel,
// Gaussian) pairs evaluated and blended into counts[0..1] (not used on the
// render path).
template <int TS, int BATCH, bool COUNT>
__global__ void __launch_bounds__(TS *TS)
blend_kernel(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ ids, uint32_t id_mask,
             const float4 *__restrict__ rec, uint32_t n, uint32_t cap, int width, int height, int tiles_x, float bg0, float bg1, float bg2, float *__restrict__ out_rgb,
             float *__restrict__ out_T, uint32_t *__restrict__ out_nc, unsigned long long *counts) {
    constexpr int NT = TS * TS;
    __shared__ float4 s_g[BATCH];    // u, v, A = -a/2, B = -b
    __shared__ float4 s_h[BATCH];    // C = -c/2, o_hat, r, g
    __shared__ float s_b[BATCH];     // blue

    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int px = tx * TS + (int)(threadIdx.x % TS), py = ty * TS + (int)(threadIdx.x / TS);
    const bool inside = px < width && py < height;
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    uint2 rg = ranges[tile];
    rg.y = min(rg.y, cap);   // ranges are written clamped; this keeps every read in bounds regardless
    rg.x = min(rg.x, rg.y);

    float T = 1.0f, c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
    uint32_t last = 0;
    bool done = !inside;
    uint32_t n_eval = 0, n_blend = 0;

    for (uint32_t start = rg.x; start < rg.y; start += BATCH) {
        if (__syncthreads_count(!done) == 0) break;
        for (int k = threadIdx.x; k < BATCH; k += NT) {
            const uint32_t j = start + (uint32_t)k;
            if (j < rg.y) {
                uint32_t id = ids[j] & id_mask;
                if (id >= n) id = 0;   // only after a timed-out sort pass; keeps the gather in bounds
                const float4 r0 = rec[3 * (size_t)id + 0];
                const float4 r1 = rec[3 * (size_t)id + 1];
                const float4 r2 = rec[3 * (size_t)id + 2];
                s_g[k] = make_float4(r0.x, r0.y, -0.5f * r0.z, -r0.w);
                s_h[k] = make_float4(-0.5f * r1.x, r1.y, r2.x, r2.y);
                s_b[k] = r2.z;
            }
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)BATCH, rg.y - start);
        if (!done) {
            for (int b = 0; b < nb; b++) {
                if (COUNT) n_eval++;
                const float4 g = s_g[b];
                const float dx = g.x - pxf, dy = g.y - pyf;
                const float4 h = s_h[b];
                const float power = g.z * dx * dx + h.x * dy * dy + g.w * dx * dy;
                if (power > 0.0f) continue;
                const float alpha = fminf(kAlphaMax, h.y * __expf(power));
                if (alpha < kAlphaMin) continue;
                const float test = T * (1.0f - alpha);
                if (test < kTMin) {
                    done = true;
                    break;
                }
                if (COUNT) n_blend++;
                const float w = alpha * T;
                c0 += w * h.z;
                c1 += w * h.w;
                c2 += w * s_b[b];
                T = test;
                last = start - rg.x + (uint32_t)b + 1u;
            }
        }
    }
    if (inside) {
        const size_t p = (size_t)py * width + px;
        out_rgb[3 * p + 0] = c0 + T * bg0;
        out_rgb[3 * p + 1] = c1 + T * bg1;
        out_rgb[3 * p + 2] = c2 + T * bg2;
        out_T[p] = T;
        out_nc[p] = last;
    }
    if (COUNT) {
        const unsigned long long e = __reduce_add_sync(0xFFFFFFFFu, n_eval);
        const unsigned long long b = __reduce_add_sync(0xFFFFFFFFu, n_blend);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(counts + 0, e);
            atomicAdd(counts + 1, b);
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
    if (counts)
        blend_kernel<TS, BATCH, true><<<L.ntiles, TS * TS, 0, st>>>(
            at<uint2>(ws, L.ranges), pair_ids(L, ws), id_mask(L), at<float4>(ws, L.records),
            (uint32_t)L.n, (uint32_t)L.cap, L.width, L.height, L.tiles_x, cfg.bg[0], cfg.bg[1], cfg.bg[2], out_rgb, at<float>(ws, L.final_T),
            at<uint32_t>(ws, L.n_contrib), counts);
    else
        blend_kernel<TS, BATCH, false><<<L.ntiles, TS * TS, 0, st>>>(
            at<uint2>(ws, L.ranges), pair_ids(L, ws), id_mask(L), at<float4>(ws, L.records),
            (uint32_t)L.n, (uint32_t)L.cap, L.width, L.height, L.tiles_x, cfg.bg[0], cfg.bg[1], cfg.bg[2], out_rgb, at<float>(ws, L.final_T),
            at<uint32_t>(ws, L.n_contrib), nullptr);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blend(const Layout &L, const d4dgs_config &cfg, void *ws, float *out_rgb, cudaStream_t st,
                         unsigned long long *counts) {
    if (L.ntiles == 0) return cudaSuccess;
#define D4DGS_BATCHES(TS)                                                   \
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
