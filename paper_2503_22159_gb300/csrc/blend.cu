// blend.cu -- K6: per-pixel front-to-back alpha compositing over each tile's
// depth-ordered list (Eq. 4; alpha_i = o_hat_i G'_i with the 2D Gaussian of
// Eq. 1 evaluated through its conic):
//
//   p = -1/2 (a dx^2 + c dy^2) - b dx dy,  skip p > 0
//   alpha = min(0.99, o_hat e^p),          skip alpha < 1/255
//   stop (before blending) once T (1 - alpha) < 1e-4
//   C += alpha T c;  T *= 1 - alpha;       out = C + T bg
//
// One CTA per tile; each warp owns an 8 x 8 pixel block of it and each thread
// two vertically adjacent pixels of that block, so dx and its products are
// shared.  The CTA walks the tile's list in batches: each batch of Gaussians is
// gathered once into shared memory (already scaled to base-2 exponent form)
// together with a bit mask of the 8 x 8 blocks its alpha >= 1/255 ellipse
// reaches, and each warp visits only the Gaussians whose mask holds its bit
// (a ballot per 32 Gaussians, then the set bits in ascending order).  Skipped
// (block, Gaussian) pairs have alpha < 1/255 at every pixel of the block, so
// the image is the one the full walk gives.  A warp stops when its 64 pixels
// have stopped, a CTA when all of its pixels have.
//
// Exponent form: with A = -a/2 log2(e), B = -b log2(e), C = -c/2 log2(e) and
// L = log2(o_hat), q = A dx^2 + B dx dy + C dy^2 + L and alpha = min(0.99, 2^q),
// so the alpha >= 1/255 test is q >= log2(1/255), taken before the exp: most
// pairs are rejected with five FMAs and two compares.  No tensor cores:
// nothing here is a dense contraction; the bound is FP32 issue.
#include "blend_mask.cuh"
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

// Composite one Gaussian (already known to pass p <= 0 and q >= log2(1/255))
// into a pixel: stop before blending once T (1 - alpha) < 1e-4.
__device__ __forceinline__ bool composite(PixelState &px, float q, const float4 &c, uint32_t pos) {
    const float alpha = fminf(kAlphaMax, alpha_exp2(q));
    const float test = px.T * (1.0f - alpha);
    if (test < kTMin) {
        px.done = true;
        return false;
    }
    const float w = alpha * px.T;
    px.c0 = fmaf(w, c.x, px.c0);
    px.c1 = fmaf(w, c.y, px.c1);
    px.c2 = fmaf(w, c.z, px.c2);
    px.T = test;
    px.last = pos;
    return true;
}

// COUNT: instrumented variant for profiling (not used on the render path),
// which also totals into counts[0..2]: (pixel, Gaussian) pairs the warps
// evaluated, pairs blended, and the tile-algorithm work sum over tiles of
// (pixels in the image) x (list entries up to the one at which the tile's
// last pixel stopped, or the whole list).
// PERSIST: CTAs take tiles from an atomic counter until all are done (fixed
// grid, for batched and graph-captured launches); otherwise one CTA per tile.
template <int TS, int BATCH, bool COUNT, bool PERSIST>
__global__ void __launch_bounds__(TS *TS / 2, TS == 8 ? 16 : (TS == 16 ? 8 : 2))
blend_kernel(char *__restrict__ ba, float *__restrict__ out0, unsigned long long *counts) {
    constexpr int NT = TS * TS / 2;
    constexpr int BX = TS / 8;       // 8 x 8 blocks per tile row; warp w owns block (w % BX, w / BX)
    static_assert(NT / 32 == BX * BX, "one warp per 8 x 8 block");
    __shared__ float4 s_g[BATCH];    // u, v, A, B
    __shared__ float2 s_h[BATCH];    // C, L
    __shared__ float4 s_c[BATCH];    // r, g, b
    __shared__ uint32_t s_m[BATCH];  // blocks the Gaussian's alpha >= 1/255 ellipse reaches
    __shared__ int32_t s_item;
    __shared__ uint32_t s_stop;
    uint32_t *bw = reinterpret_cast<uint32_t *>(ba);
    const int nviews = (int)bw[kBaNViews];
    const int total = (int)bw[kBaTotalTiles];
    const int lane = (int)(threadIdx.x & 31u), warp = (int)(threadIdx.x >> 5);
    uint32_t n_eval = 0, n_blend = 0;
    unsigned long long n_work = 0;

    for (int pass = 0;; pass++) {
        int item;
        if (PERSIST) {
            if (threadIdx.x == 0) s_item = (int32_t)atomicAdd(bw + kBaBlend, 1u);
            __syncthreads();
            item = s_item;
            __syncthreads();
        } else {
            item = pass == 0 ? (int)blockIdx.x : total;
        }
        if (item >= total) break;
        int vi = 0;
        for (int u = 1; u < nviews; u++)
            if (view_of(ba, u).tile_base <= item) vi = u;
        const View &v = view_of(ba, vi);
        const int tile = item - v.tile_base;
        const int tiles_x = v.cam.tiles_x, width = v.cam.width, height = v.cam.height;
        const uint32_t n = (uint32_t)v.n, cap = v.cap;
        const bool packed = v.packed != 0;
        const uint32_t id_mask = packed ? (uint32_t)((1ull << v.id_bits) - 1ull) : 0xFFFFFFFFu;
        const uint32_t *ids = packed ? v.tkeys[v.tile_passes & 1] : v.tvals[v.tile_passes & 1];
        const float4 *rec = v.rec;
        float *out_rgb = (out0 && vi == 0) ? out0 : v.out_rgb;

        const int tx = tile % tiles_x, ty = tile / tiles_x;
        const int x0 = tx * TS, y0 = ty * TS;
        const int lx = 8 * (warp % BX) + (lane & 7), ly = 8 * (warp / BX) + 2 * (lane >> 3);
        const int px = x0 + lx, py0 = y0 + ly, py1 = py0 + 1;
        const bool in0 = px < width && py0 < height, in1 = px < width && py1 < height;
        const float pxf = (float)px + 0.5f, pyf0 = (float)py0 + 0.5f, pyf1 = (float)py1 + 0.5f;
        uint2 rg = v.ranges[tile];
        rg.y = min(rg.y, cap);   // ranges are written clamped; this keeps every read in bounds regardless
        rg.x = min(rg.x, rg.y);

        PixelState a{1.0f, 0.0f, 0.0f, 0.0f, 0u, !in0};
        PixelState b{1.0f, 0.0f, 0.0f, 0.0f, 0u, !in1};
        uint32_t stop_a = rg.y - rg.x, stop_b = stop_a;   // COUNT only

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
                    const float A = -0.5f * kLog2e * r0.z, B = -kLog2e * r0.w, C = -0.5f * kLog2e * r1.x;
                    s_g[k] = make_float4(r0.x, r0.y, A, B);
                    s_h[k] = make_float2(C, r2.w);
                    s_c[k] = r2;
                    s_m[k] = d4dgs::block_mask<TS>(r0.x, r0.y, A, B, C, r2.w, x0, y0);
                }
            }
            __syncthreads();
            const int nb = (int)min((uint32_t)BATCH, rg.y - start);
            // warp-uniform from here to the end of the batch
            if (__any_sync(0xFFFFFFFFu, !(a.done && b.done))) {
                for (int k0 = 0; k0 < nb; k0 += 32) {
                    const int kl = k0 + lane;
                    uint32_t bits = __ballot_sync(0xFFFFFFFFu, kl < nb && ((s_m[kl] >> warp) & 1u));
                    while (bits) {
                        const int k = k0 + __ffs((int)bits) - 1;
                        bits &= bits - 1u;
                        // both pixels' exponents, branch free; most pairs stop here
                        const float4 g = s_g[k];
                        const float2 h = s_h[k];
                        const float dx = g.x - pxf;
                        const float axx = g.z * dx * dx, bx = g.w * dx;
                        const float dya = g.y - pyf0, dyb = g.y - pyf1;
                        const float pa = fmaf(fmaf(h.x, dya, bx), dya, axx);
                        const float pb = fmaf(fmaf(h.x, dyb, bx), dyb, axx);
                        const float qa = pa + h.y, qb = pb + h.y;
                        const bool ea = !a.done && pa <= 0.0f && qa >= kLog2AlphaMin;
                        const bool eb = !b.done && pb <= 0.0f && qb >= kLog2AlphaMin;
                        if (COUNT) n_eval += (uint32_t)!a.done + (uint32_t)!b.done;
                        if (ea || eb) {
                            const float4 c = s_c[k];
                            const uint32_t pos = start - rg.x + (uint32_t)k + 1u;
                            if (ea) {
                                const bool bl = composite(a, qa, c, pos);
                                if (COUNT) {
                                    n_blend += bl;
                                    if (!bl) stop_a = pos;
                                }
                            }
                            if (eb) {
                                const bool bl = composite(b, qb, c, pos);
                                if (COUNT) {
                                    n_blend += bl;
                                    if (!bl) stop_b = pos;
                                }
                            }
                        }
                    }
                    if (__all_sync(0xFFFFFFFFu, a.done && b.done)) break;
                }
            }
        }
        if (COUNT) {
            // tile work: in-image pixels x entries up to the tile's last stop
            if (threadIdx.x == 0) s_stop = 0u;
            __syncthreads();
            const uint32_t st = max(in0 ? stop_a : 0u, in1 ? stop_b : 0u);
            const uint32_t wst = __reduce_max_sync(0xFFFFFFFFu, st);
            if (lane == 0) atomicMax(&s_stop, wst);
            __syncthreads();
            const int npx = min(TS, width - x0) * min(TS, height - y0);
            if (threadIdx.x == 0) n_work += (unsigned long long)npx * s_stop;
            __syncthreads();
        }
        const float bg0 = v.bg[0], bg1 = v.bg[1], bg2 = v.bg[2];
        if (in0) {
            const size_t p = (size_t)py0 * width + px;
            out_rgb[3 * p + 0] = a.c0 + a.T * bg0;
            out_rgb[3 * p + 1] = a.c1 + a.T * bg1;
            out_rgb[3 * p + 2] = a.c2 + a.T * bg2;
            v.final_T[p] = a.T;
            v.n_contrib[p] = a.last;
        }
        if (in1) {
            const size_t p = (size_t)py1 * width + px;
            out_rgb[3 * p + 0] = b.c0 + b.T * bg0;
            out_rgb[3 * p + 1] = b.c1 + b.T * bg1;
            out_rgb[3 * p + 2] = b.c2 + b.T * bg2;
            v.final_T[p] = b.T;
            v.n_contrib[p] = b.last;
        }
    }
    if (COUNT) {
        const unsigned long long e = __reduce_add_sync(0xFFFFFFFFu, n_eval);
        const unsigned long long bb = __reduce_add_sync(0xFFFFFFFFu, n_blend);
        if (lane == 0) {
            atomicAdd(counts + 0, e);
            atomicAdd(counts + 1, bb);
        }
        if (threadIdx.x == 0) atomicAdd(counts + 2, n_work);
    }
}

template <int TS, int BATCH>
cudaError_t launch_ts(char *ba, int total_tiles, bool persist, cudaStream_t st, int num_sms, float *out0,
                      unsigned long long *counts) {
    auto go = [&](auto kernel) {
        static int occ = 0;   // per instantiation; queried once, before any graph capture uses it
        if (!occ && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, TS * TS / 2, 0) != cudaSuccess ||
                     occ < 1))
            occ = 1;
        kernel<<<occ * num_sms, TS * TS / 2, 0, st>>>(ba, out0, counts);
    };
    if (persist) {
        if (counts) go(blend_kernel<TS, BATCH, true, true>);
        else go(blend_kernel<TS, BATCH, false, true>);
    } else if (counts) {
        blend_kernel<TS, BATCH, true, false><<<total_tiles, TS * TS / 2, 0, st>>>(ba, out0, counts);
    } else {
        blend_kernel<TS, BATCH, false, false><<<total_tiles, TS * TS / 2, 0, st>>>(ba, out0, counts);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blend(const BatchArgs &args, char *batch_area, cudaStream_t st, int num_sms, float *out0,
                         unsigned long long *counts, bool persist) {
    if (args.total_tiles == 0) return cudaSuccess;
    const int nt = args.total_tiles;
#define D4DGS_BATCHES(TS)                                                                              \
    if (args.batch == 64) return launch_ts<TS, 64>(batch_area, nt, persist, st, num_sms, out0, counts);   \
    if (args.batch == 128) return launch_ts<TS, 128>(batch_area, nt, persist, st, num_sms, out0, counts); \
    if (args.batch == 256) return launch_ts<TS, 256>(batch_area, nt, persist, st, num_sms, out0, counts); \
    return cudaErrorInvalidValue;
    switch (args.tile) {
        case 8: D4DGS_BATCHES(8)
        case 16: D4DGS_BATCHES(16)
        case 32: D4DGS_BATCHES(32)
        default: return cudaErrorInvalidValue;
    }
#undef D4DGS_BATCHES
}

}  // namespace d4dgs
