// blend.cu -- K6: per-pixel front-to-back alpha compositing over each tile's
// depth-ordered list (Eq. 4; alpha_i = o_hat_i G'_i with the 2D Gaussian of
// Eq. 1 evaluated through its conic):
//
//   p = -1/2 (a dx^2 + c dy^2) - b dx dy,  skip p > 0
//   alpha = min(0.99, o_hat e^p),          skip alpha < 1/255
//   stop (before blending) once T (1 - alpha) < 1e-4
//   C += alpha T c;  T *= 1 - alpha;       out = C + T bg
//
// One CTA per tile.  Each thread owns a column of PX pixels (4; 2 at 8-px
// tiles), so dx and its products are shared, and works on them as pixel
// pairs with Blackwell's packed FP32x2 add/mul/fma (one instruction for both
// pixels of a pair, each lane rounded as the scalar operation).  Each warp
// owns an 8 x 4PX block of the tile.  The CTA walks the tile's list in
// batches: each batch of Gaussians is gathered once into shared memory
// (already in base-2 exponent form, every scalar stored twice so that a
// 128-bit broadcast load fills register pairs) together with a bit mask of
// the blocks its alpha >= 1/255 ellipse reaches, and each warp visits only
// the Gaussians whose mask holds its bit (a ballot per 32 Gaussians, then the
// set bits in ascending order).  Skipped (block, Gaussian) pairs have
// alpha < 1/255 at every pixel of the block, so the image is the one the full
// walk gives.  When any pixel of a thread passes, all of its pixels take the
// compositing step, with alpha = 0 for the ones that do not (T and C then
// stay as they are).  A warp stops when all of its pixels have stopped, a CTA
// when all of its warps have.
//
// Exponent form: with A = -a/2 log2(e), B = -b log2(e), C = -c/2 log2(e) and
// L = log2(o_hat), q = A dx^2 + B dx dy + C dy^2 + L and alpha = min(0.99, 2^q),
// so the alpha >= 1/255 test is q >= log2(1/255), taken before the exp.  No
// tensor cores: nothing here is a dense contraction; the bound is instruction
// issue.
#include "blend_common.cuh"
#include "blend_mask.cuh"

namespace d4dgs {

namespace {


// warps of a forward CTA
template <int TS>
struct FwdWarps {
    static constexpr int value = BlendShape<TS>::NT / 32;
};

// COUNT: instrumented variant for profiling (not used on the render path),
// which also totals into counts[0..2]: (pixel, Gaussian) pairs the warps
// evaluated, pairs blended, and the tile-algorithm work sum over tiles of
// (pixels in the image) x (list entries up to the one at which the tile's
// last pixel stopped, or the whole list).
// PERSIST: CTAs take tiles from an atomic counter until all are done (fixed
// grid, for batched and graph-captured launches); otherwise one CTA per tile.
// FLOW: also composites the per-Gaussian screen flow into the view's flow
// output (two channels, background 0) with the same weights.
// PARAM: a launch of one view whose descriptor also travels as the kernel parameter v0.
// 32-px tiles: 4 CTAs per SM (64 registers; a 512-deep staging takes 51 KB).
template <int TS, int BATCH, bool COUNT, bool PERSIST, bool FLOW = false, bool PARAM = false>
__global__ void __launch_bounds__(BlendShape<TS>::NT, TS == 8 ? 24 : (TS == 16 ? 10 : 4))
blend_kernel(char *__restrict__ ba, float *__restrict__ out0, unsigned long long *counts,
             const __grid_constant__ View v0) {
    using S = BlendShape<TS>;
    constexpr int PX = S::PX, NP = S::NP, BH = S::BH, NT = S::NT, BX = S::BX;
    // one 96-byte record per staged Gaussian (a 128-byte stride put the 16-byte staging stores of
    // a warp's lanes in the same four banks; at 96 bytes they spread over all of them):
    // [0] u, u, A, A  [1] B, B, C, C  [2] v, v, L, L  [3] r, r, g, g  [4] b, b
    // [5] flow u, u, v, v (FLOW)
    extern __shared__ float4 s_dynb[];   // blend_smem(BATCH) bytes
    float4 (*s_rec)[6] = reinterpret_cast<float4 (*)[6]>(s_dynb);
    uint32_t *s_m = reinterpret_cast<uint32_t *>(s_dynb + BATCH * 6);   // blocks the Gaussian's alpha >= 1/255 ellipse reaches
    __shared__ int32_t s_item;
    __shared__ uint32_t s_stop;
    __shared__ float s_wsum[FwdWarps<TS>::value];   // per warp: list entries its pixels walked
    grid_dependency_wait();
    uint32_t *bw = reinterpret_cast<uint32_t *>(ba);
    const int nviews = PARAM ? 1 : (int)bw[kBaNViews];
    const int total = PARAM ? v0.ntiles : (int)bw[kBaTotalTiles];
    const int lane = (int)(threadIdx.x & 31u), warp = (int)(threadIdx.x >> 5);
    uint32_t n_eval = 0, n_blend = 0;
    unsigned long long n_work = 0;
    const float2 one2 = make_float2(1.0f, 1.0f);

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
        const View &v = PARAM ? v0 : view_of(ba, vi);
        int tile = item - v.tile_base;
        {   // heaviest tiles first (the order the binning derived from the previous frame's walked
            // entries: nearby frames load nearby tiles alike); kept in range whatever the buffer holds
            const uint32_t o = v.tile_order[tile];
            if (o < (uint32_t)v.ntiles) tile = (int)o;
        }
        const int tiles_x = v.cam.tiles_x, width = v.cam.width, height = v.cam.height;
        const uint32_t n = (uint32_t)v.n, cap = v.cap;
        const bool packed = v.packed != 0;
        const uint32_t id_mask = packed ? (uint32_t)((1ull << v.id_bits) - 1ull) : 0xFFFFFFFFu;
        const uint32_t *ids = packed ? v.tkeys[v.tile_passes & 1] : v.tvals[v.tile_passes & 1];
        const float4 *rec = v.rec;
        float *out_rgb = (out0 && vi == 0) ? out0 : v.out_rgb;

        const int tx = tile % tiles_x, ty = tile / tiles_x;
        const int x0 = tx * TS, y0 = ty * TS;
        const int px = x0 + 8 * (warp % BX) + (lane & 7);
        const int py = y0 + BH * (warp / BX) + PX * (lane >> 3);
        const float pxf = (float)px + 0.5f;
        const float2 pxf2 = make_float2(pxf, pxf);
        float2 pyf[NP], T[NP], c0[NP], c1[NP], c2[NP], fa[NP], fb[NP];
        // walked[i]: list entries the pixel walks before the one at which it stops (the
        // whole list if it never stops); the backward replays those entries
        uint32_t walked[PX], stop[PX];
        float thr[PX];   // per-pixel pass threshold of q: log2(1/255), +inf once the pixel has stopped
        uint2 rg = v.ranges[tile];
        rg.y = min(rg.y, cap);   // ranges are written clamped; this keeps every read in bounds regardless
        rg.x = min(rg.x, rg.y);
#pragma unroll
        for (int j = 0; j < NP; j++) {
            pyf[j] = make_float2((float)(py + 2 * j) + 0.5f, (float)(py + 2 * j + 1) + 0.5f);
            T[j] = one2;
            c0[j] = c1[j] = c2[j] = make_float2(0.0f, 0.0f);
            fa[j] = fb[j] = make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int i = 0; i < PX; i++) {
            walked[i] = rg.y - rg.x;
            stop[i] = rg.y - rg.x;   // COUNT only
            thr[i] = (px < width && py + i < height) ? kLog2AlphaMin : kInf;
        }

        for (uint32_t start = rg.x; start < rg.y; start += BATCH) {
            bool live = false;
#pragma unroll
            for (int i = 0; i < PX; i++) live |= thr[i] < kInf;
            if (__syncthreads_count(live) == 0) break;
            for (int k = threadIdx.x; k < BATCH; k += NT) {
                const uint32_t j = start + (uint32_t)k;
                if (j < rg.y) {
                    uint32_t id = ids[j] & id_mask;
                    if (id >= n) id = 0;   // only after a timed-out sort pass; keeps the gather in bounds
                    const float4 r0 = rec[3 * (size_t)id + 0];
                    const float4 r1 = rec[3 * (size_t)id + 1];
                    const float4 r2 = rec[3 * (size_t)id + 2];
                    const float A = -0.5f * kLog2e * r0.z, B = -kLog2e * r0.w, C = -0.5f * kLog2e * r1.x;
                    s_rec[k][0] = make_float4(r0.x, r0.x, A, A);
                    s_rec[k][1] = make_float4(B, B, C, C);
                    s_rec[k][2] = make_float4(r0.y, r0.y, r2.w, r2.w);
                    s_rec[k][3] = make_float4(r2.x, r2.x, r2.y, r2.y);
                    s_rec[k][4] = make_float4(r2.z, r2.z, 0.0f, 0.0f);
                    if (FLOW) {
                        const float2 fl = v.flow2d[id];
                        s_rec[k][5] = make_float4(fl.x, fl.x, fl.y, fl.y);
                    }
                    const float det4 = fmaf(4.0f * A, C, -(B * B)), tr = -(A + C);
                    const bool fast = r2.w <= kLog2FastOpacity && det4 > kFastConditioning * tr * tr;
                    s_m[k] = d4dgs::block_mask<TS, BH>(r0.x, r0.y, A, B, C, r2.w, x0, y0) | (fast ? 0u : kSlowBit);
                }
            }
            __syncthreads();
            const int nb = (int)min((uint32_t)BATCH, rg.y - start);
            // Visit Gaussian k of the batch (warp-uniform).  FAST: no clamp and no
            // p > 0 test (see kLog2FastOpacity).  In both bodies the stop test
            // T (1 - alpha) < 1e-4 is taken for all pixels at once, and the
            // per-pixel selects run only when one of the thread's pixels stops.
            auto visit = [&](auto fast_c, int k) {
                constexpr bool FAST = decltype(fast_c)::value;
                const float4 ua = s_rec[k][0], bc = s_rec[k][1], vl = s_rec[k][2];
                const float2 dx = f2_sub(make_float2(ua.x, ua.y), pxf2);
                const float2 axx = f2_mul(f2_mul(make_float2(ua.z, ua.w), dx), dx);
                const float2 bx = f2_mul(make_float2(bc.x, bc.y), dx);
                float2 al[NP];
                bool e[PX];
#pragma unroll
                for (int j = 0; j < NP; j++) {
                    const float2 dy = f2_sub(make_float2(vl.x, vl.y), pyf[j]);
                    const float2 p = f2_fma(f2_fma(make_float2(bc.z, bc.w), dy, bx), dy, axx);
                    const float2 q = f2_add(p, make_float2(vl.z, vl.w));
                    if (FAST) {
                        e[2 * j] = q.x >= thr[2 * j];
                        e[2 * j + 1] = q.y >= thr[2 * j + 1];
                        al[j] = make_float2(e[2 * j] ? alpha_exp2(q.x) : 0.0f, e[2 * j + 1] ? alpha_exp2(q.y) : 0.0f);
                    } else {
                        e[2 * j] = p.x <= 0.0f && q.x >= thr[2 * j];
                        e[2 * j + 1] = p.y <= 0.0f && q.y >= thr[2 * j + 1];
                        al[j] = make_float2(e[2 * j] ? fminf(kAlphaMax, alpha_exp2(q.x)) : 0.0f,
                                            e[2 * j + 1] ? fminf(kAlphaMax, alpha_exp2(q.y)) : 0.0f);
                    }
                }
                if (COUNT) {
#pragma unroll
                    for (int i = 0; i < PX; i++) n_eval += (uint32_t)(thr[i] < kInf);
                }
                // a pixel that does not pass has alpha = 0 and keeps T >= 1e-4, so only passing ones can stop
                float2 test[NP];
                bool any_stop = false;
#pragma unroll
                for (int j = 0; j < NP; j++) {
                    test[j] = f2_mul(T[j], f2_sub(one2, al[j]));
                    any_stop |= (test[j].x < kTMin) | (test[j].y < kTMin);
                }
                const float4 rgc = s_rec[k][3];
                const float2 bl = make_float2(s_rec[k][4].x, s_rec[k][4].y);
                const uint32_t pos = start - rg.x + (uint32_t)k + 1u;
                if (!__any_sync(0xFFFFFFFFu, any_stop)) {   // warp-uniform: no pixel of the warp stops here
#pragma unroll
                    for (int j = 0; j < NP; j++) {
                        const float2 w = f2_mul(al[j], T[j]);
                        T[j] = test[j];
                        c0[j] = f2_fma(w, make_float2(rgc.x, rgc.y), c0[j]);
                        c1[j] = f2_fma(w, make_float2(rgc.z, rgc.w), c1[j]);
                        c2[j] = f2_fma(w, bl, c2[j]);
                        if (FLOW) {
                            const float4 fr = s_rec[k][5];
                            fa[j] = f2_fma(w, make_float2(fr.x, fr.y), fa[j]);
                            fb[j] = f2_fma(w, make_float2(fr.z, fr.w), fb[j]);
                        }
                    }
                    if (COUNT) {
#pragma unroll
                        for (int i = 0; i < PX; i++) n_blend += (uint32_t)e[i];
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < NP; j++) {
                        const bool sa = test[j].x < kTMin, sb = test[j].y < kTMin;
                        const bool ba = e[2 * j] && !sa, bb = e[2 * j + 1] && !sb;
                        if (sa) {
                            thr[2 * j] = kInf;
                            walked[2 * j] = pos - 1u;
                        }
                        if (sb) {
                            thr[2 * j + 1] = kInf;
                            walked[2 * j + 1] = pos - 1u;
                        }
                        const float2 w = f2_mul(make_float2(sa ? 0.0f : al[j].x, sb ? 0.0f : al[j].y), T[j]);
                        T[j].x = sa ? T[j].x : test[j].x;
                        T[j].y = sb ? T[j].y : test[j].y;
                        c0[j] = f2_fma(w, make_float2(rgc.x, rgc.y), c0[j]);
                        c1[j] = f2_fma(w, make_float2(rgc.z, rgc.w), c1[j]);
                        c2[j] = f2_fma(w, bl, c2[j]);
                        if (COUNT) {
                            n_blend += (uint32_t)ba + (uint32_t)bb;
                            if (sa) stop[2 * j] = pos;
                            if (sb) stop[2 * j + 1] = pos;
                        }
                    }
                }
            };
            // warp-uniform from here to the end of the batch
            if (__any_sync(0xFFFFFFFFu, live)) {
                const uint32_t wbit = 1u << warp;
                for (int k0 = 0; k0 < nb; k0 += 32) {
                    const int kl = k0 + lane;
                    const uint32_t m = kl < nb ? s_m[kl] : 0u;
                    uint32_t bits = __ballot_sync(0xFFFFFFFFu, (m & wbit) != 0u);
                    const uint32_t slow = __ballot_sync(0xFFFFFFFFu, (m & wbit) != 0u && (m & kSlowBit) != 0u);
                    if (slow == 0u) {
                        while (bits) {
                            const int b = __ffs((int)bits) - 1;
                            bits &= bits - 1u;
                            visit(BoolC<true>{}, k0 + b);
                        }
                    } else {
                        while (bits) {
                            const int b = __ffs((int)bits) - 1;
                            bits &= bits - 1u;
                            if ((slow >> b) & 1u) visit(BoolC<false>{}, k0 + b);
                            else visit(BoolC<true>{}, k0 + b);
                        }
                    }
                    bool all_done = true;
#pragma unroll
                    for (int i = 0; i < PX; i++) all_done &= thr[i] == kInf;
                    if (__all_sync(0xFFFFFFFFu, all_done)) break;
                }
            }
        }
        if (COUNT) {
            // tile work: in-image pixels x entries up to the tile's last stop
            if (threadIdx.x == 0) s_stop = 0u;
            __syncthreads();
            uint32_t st = 0u;
#pragma unroll
            for (int i = 0; i < PX; i++)
                if (px < width && py + i < height) st = max(st, stop[i]);
            const uint32_t wst = __reduce_max_sync(0xFFFFFFFFu, st);
            if (lane == 0) atomicMax(&s_stop, wst);
            __syncthreads();
            const int npx = min(TS, width - x0) * min(TS, height - y0);
            if (threadIdx.x == 0) n_work += (unsigned long long)npx * s_stop;
            __syncthreads();
        }
        {   // this tile's work for the next frame's order and this frame's backward: entries walked,
            // summed over the tile's pixels (a float weight: no overflow)
            float ws = 0.0f;
#pragma unroll
            for (int i = 0; i < PX; i++)
                if (px < width && py + i < height) ws += (float)walked[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ws += __shfl_xor_sync(0xFFFFFFFFu, ws, o);
            if (lane == 0) s_wsum[warp] = ws;
            __syncthreads();
            if (threadIdx.x == 0) {
                float t = 0.0f;
#pragma unroll
                for (int w = 0; w < FwdWarps<TS>::value; w++) t += s_wsum[w];
                v.tile_work[tile] = t >= 4.0e9f ? 4000000000u : (uint32_t)t;
            }
        }
        const float bg0 = v.bg[0], bg1 = v.bg[1], bg2 = v.bg[2];
#pragma unroll
        for (int i = 0; i < PX; i++) {
            if (px < width && py + i < height) {
                const int j = i >> 1;
                const bool hi = (i & 1) != 0;
                const float Ti = hi ? T[j].y : T[j].x;
                const size_t p = (size_t)(py + i) * width + px;
                out_rgb[3 * p + 0] = (hi ? c0[j].y : c0[j].x) + Ti * bg0;
                out_rgb[3 * p + 1] = (hi ? c1[j].y : c1[j].x) + Ti * bg1;
                out_rgb[3 * p + 2] = (hi ? c2[j].y : c2[j].x) + Ti * bg2;
                v.final_T[p] = Ti;
                v.n_contrib[p] = walked[i];
                if (FLOW) {
                    v.out_flow[2 * p + 0] = hi ? fa[j].y : fa[j].x;
                    v.out_flow[2 * p + 1] = hi ? fb[j].y : fb[j].x;
                }
            }
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

// dynamic shared memory of a blend CTA: the staged records and block masks
constexpr size_t blend_smem(int batch) { return (size_t)batch * (6 * 16 + 4); }

template <int TS, int BATCH>
cudaError_t launch_ts(char *ba, int total_tiles, bool persist, cudaStream_t st, int num_sms, float *out0,
                      unsigned long long *counts, bool flow, const View &v0) {
    constexpr size_t smem = blend_smem(BATCH);
    static bool attr = false;
    if (!attr && smem > 48 * 1024) {   // above the default
        for (const void *fn : {(const void *)blend_kernel<TS, BATCH, false, false, true, true>,
                               (const void *)blend_kernel<TS, BATCH, true, true>, (const void *)blend_kernel<TS, BATCH, false, true>,
                               (const void *)blend_kernel<TS, BATCH, true, false, false, true>,
                               (const void *)blend_kernel<TS, BATCH, false, false, false, true>})
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    attr = true;
    if (flow)   // single frames only
        return launch_chained(blend_kernel<TS, BATCH, false, false, true, true>, total_tiles, BlendShape<TS>::NT, smem, st,
                              ba, out0, counts, v0);
    auto go = [&](auto kernel) {
        static int occ = 0;   // per instantiation; queried once, before any graph capture uses it
        if (!occ && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, BlendShape<TS>::NT, smem) != cudaSuccess ||
                     occ < 1))
            occ = 1;
        return launch_chained(kernel, occ * num_sms, BlendShape<TS>::NT, smem, st, ba, out0, counts, v0);
    };
    if (persist) {
        if (counts) return go(blend_kernel<TS, BATCH, true, true>);
        return go(blend_kernel<TS, BATCH, false, true>);
    } else if (counts) {
        return launch_chained(blend_kernel<TS, BATCH, true, false, false, true>, total_tiles, BlendShape<TS>::NT, smem, st,
                              ba, out0, counts, v0);
    } else {
        return launch_chained(blend_kernel<TS, BATCH, false, false, false, true>, total_tiles, BlendShape<TS>::NT, smem, st,
                              ba, out0, counts, v0);
    }
}

}  // namespace

cudaError_t launch_blend(const BatchArgs &args, char *batch_area, cudaStream_t st, int num_sms, float *out0,
                         unsigned long long *counts, bool persist) {
    if (args.total_tiles == 0) return cudaSuccess;
    const int nt = args.total_tiles;
    const bool flow = args.nviews == 1 && args.v[0].out_flow != nullptr && !counts && !persist;
#define D4DGS_BATCHES(TS)                                                                                    \
    if (args.batch == 64) return launch_ts<TS, 64>(batch_area, nt, persist, st, num_sms, out0, counts, flow, args.v[0]);   \
    if (args.batch == 128) return launch_ts<TS, 128>(batch_area, nt, persist, st, num_sms, out0, counts, flow, args.v[0]); \
    if (args.batch == 256) return launch_ts<TS, 256>(batch_area, nt, persist, st, num_sms, out0, counts, flow, args.v[0]); \
    return cudaErrorInvalidValue;
    switch (args.tile) {
        case 8: D4DGS_BATCHES(8)
        case 16: D4DGS_BATCHES(16)
        case 32:   // 32-px tiles also stage 512 Gaussians a batch
            if (args.batch == 512) return launch_ts<32, 512>(batch_area, nt, persist, st, num_sms, out0, counts, flow, args.v[0]);
            D4DGS_BATCHES(32)
        default: return cudaErrorInvalidValue;
    }
#undef D4DGS_BATCHES
}

}  // namespace d4dgs
