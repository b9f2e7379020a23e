// api.cu -- the C ABI (include/d4dgs.h): workspace layout, argument checks,
// stage sequencing on the caller's stream, status readback.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include "d4dgs_internal.cuh"

namespace d4dgs {

namespace {

int64_t align256(int64_t x) { return (x + 255) & ~(int64_t)255; }

int ceil_log2(int64_t v) {
    int b = 0;
    while (((int64_t)1 << b) < v) b++;
    return b;
}

bool valid_camera(const d4dgs_camera *c) {
    if (!c) return false;
    if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384) return false;
    for (int i = 0; i < 9; i++)
        if (!isfinite(c->R[i])) return false;
    for (int i = 0; i < 3; i++)
        if (!isfinite(c->T[i])) return false;
    if (!isfinite(c->fx) || !isfinite(c->fy) || !isfinite(c->cx) || !isfinite(c->cy)) return false;
    return c->fx > 0.0f && c->fy > 0.0f;
}

bool valid_config(const d4dgs_config *g) {
    if (!g) return false;
    if (g->tile != 8 && g->tile != 16 && g->tile != 32) return false;
    if (g->batch != 64 && g->batch != 128 && g->batch != 256 && !(g->batch == 512 && g->tile == 32)) return false;
    if (g->trim != 0 && g->trim != 1) return false;
    if (g->colour_cache != 0 && g->colour_cache != 1) return false;
    if (g->binning < 0 || g->binning > 3) return false;
    for (int i = 0; i < 3; i++)
        if (!isfinite(g->bg[i])) return false;
    return isfinite(g->near) && g->near >= 0.0f;
}

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

int check_scene(const d4dgs_scene *s) {
    if (!s || s->n < 0 || s->sh_degree < 0 || s->sh_degree > 3) return D4DGS_ERR_INVALID_ARG;
    if (s->n == 0) return D4DGS_OK;
    const void *ps[] = {s->means, s->t_mean, s->velocity, s->log_scales, s->log_t_scale, s->quats, s->opacity_logit, s->sh};
    for (const void *p : ps)
        if (!p || !aligned(p, 4)) return D4DGS_ERR_INVALID_ARG;
    if (!aligned(s->quats, 16)) return D4DGS_ERR_INVALID_ARG;
    if ((s->sh_degree == 1 || s->sh_degree == 3) && !aligned(s->sh, 16)) return D4DGS_ERR_INVALID_ARG;
    return D4DGS_OK;
}

int check_scene4d(const d4dgs_scene4d *s) {
    if (!s || s->n < 0 || s->sh_degree < 0 || s->sh_degree > 3) return D4DGS_ERR_INVALID_ARG;
    if (s->n == 0) return D4DGS_OK;
    const void *ps[] = {s->means4, s->log_scales4, s->quat_l, s->quat_r};
    for (const void *p : ps)
        if (!p || !aligned(p, 16)) return D4DGS_ERR_INVALID_ARG;
    if (!s->opacity_logit || !aligned(s->opacity_logit, 4) || !s->sh || !aligned(s->sh, 4)) return D4DGS_ERR_INVALID_ARG;
    if ((s->sh_degree == 1 || s->sh_degree == 3) && !aligned(s->sh, 16)) return D4DGS_ERR_INVALID_ARG;
    return D4DGS_OK;
}

int num_sms_current() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < 64 && cache[dev]) return cache[dev];
    int v = 1;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
    if (dev >= 0 && dev < 64) cache[dev] = v;
    return v;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? D4DGS_OK : D4DGS_ERR_CUDA; }

}  // namespace

bool make_layout(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, int64_t cap, Layout *L) {
    if (n < 0 || !valid_camera(cam) || !valid_config(cfg) || cap < 0 || cap > (int64_t)((1u << 30) - 1u)) return false;
    Layout l;
    l.n = n;
    l.width = cam->width;
    l.height = cam->height;
    l.tile = cfg->tile;
    l.tiles_x = (cam->width + cfg->tile - 1) / cfg->tile;
    l.tiles_y = (cam->height + cfg->tile - 1) / cfg->tile;
    l.ntiles = l.tiles_x * l.tiles_y;
    l.pixels = (int64_t)cam->width * cam->height;
    l.depth_passes = 4;
    if (l.tiles_x > kMaxCols) return false;
    l.col_bits = ceil_log2(l.tiles_x);
    l.row_bits = ceil_log2(l.tiles_y);
    // a pair's key holds its tile row only: the emission buckets the pairs by
    // column (pass 0) and the stable row passes keep that order within a row
    l.tile_bits = l.row_bits;
    const int row_passes = (l.row_bits + 7) / 8 < 1 ? 1 : (l.row_bits + 7) / 8;
    // binning 0: the column path (on the 300k-Gaussian 1352x1014 frame at 32-px tiles the direct
    // path's counts, scan and emission measured 33 + 16 + 57 us against 50 + 52 us for the column
    // emission and its row pass)
    l.direct = cfg->binning == 2;
    l.rank_lists = cfg->binning == 3;
    if (l.direct && l.ntiles > kDirMaxTiles) return false;
    l.tile_passes = l.rank_lists ? 0 : l.direct ? 1 : 1 + row_passes;
    l.tile_shift[0] = 0;
    l.tile_pass_bits[0] = l.col_bits;
    int sh = 0;
    for (int p = 1; p < l.tile_passes; p++) {
        const int left = l.tile_bits - sh, passes_left = l.tile_passes - p;
        const int b = (left + passes_left - 1) / passes_left;
        l.tile_shift[p] = sh;
        l.tile_pass_bits[p] = b;
        sh += b;
    }
    l.id_bits = ceil_log2(n > 1 ? n : 2);
    l.packed = (l.id_bits + l.tile_bits) <= 32;
    l.trim_on = cfg->trim;
    l.cap = cap;
    l.parts_depth = n > 0 ? ((int64_t)n + kDepthItems - 1) / kDepthItems : 1;
    l.parts_dup = n > 0 ? ((int64_t)n + kDupItems - 1) / kDupItems : 1;
    l.parts_tile = cap > 0 ? (cap + kTileItems - 1) / kTileItems : 1;
    l.parts_dir = n > 0 ? ((int64_t)n + kDirItems - 1) / kDirItems : 1;
    l.parts_rank = n > 0 ? ((int64_t)n + kRankItems - 1) / kRankItems : 1;
    int64_t off = 0;
    l.control = off; off += align256((int64_t)kCtlWords * 4);
    l.grid = off; off += align256((int64_t)(l.tiles_x + 1) * (l.tiles_y + 1) * 4);
    l.lb_depth = off; off += align256((int64_t)l.depth_passes * l.parts_depth * kRadix * 4);
    l.lb_col = off; off += l.direct || l.rank_lists ? 0 : align256(l.parts_dup * l.tiles_x * 4);
    l.lb_tile = off; off += l.tile_passes > 1 ? align256((int64_t)(l.tile_passes - 1) * l.parts_tile * kRadix * 4) : 0;
    l.cursor = off; off += l.rank_lists ? align256((int64_t)l.ntiles * 4) : 0;
    l.zero_end = off;
    l.colbase = off; off += align256((int64_t)l.tiles_x * 4);
    l.cmat = off; off += l.direct ? align256(l.parts_dir * l.ntiles * 4) : 0;
    l.cgrp = off; off += l.direct ? align256(l.parts_dir * l.ntiles * 8) : 0;
    l.batch = off; off += align256(kBatchAreaBytes);
    l.ranges = off; off += align256((int64_t)l.ntiles * 8);
    l.tile_order = off; off += align256((int64_t)l.ntiles * 4);
    l.tile_work = off; off += align256((int64_t)l.ntiles * 4);
    l.records = off; off += align256((int64_t)n * 48);
    for (int b = 0; b < 2; b++) { l.depth_keys[b] = off; off += align256((int64_t)n * 4); }
    for (int b = 0; b < 2; b++) { l.depth_vals[b] = off; off += align256((int64_t)n * 4); }
    l.tiles_touched = off; off += align256((int64_t)n * 4);
    l.rect = off; off += align256((int64_t)n * 8);
    l.trim = off; off += align256((int64_t)n * 8);
    l.final_T = off; off += align256(l.pixels * 4);
    l.n_contrib = off; off += align256(l.pixels * 4);
    l.grad2d = off; off += align256((int64_t)n * 48);
    l.flow2d = off; off += align256((int64_t)n * 8);
    for (int b = 0; b < 2; b++) { l.tile_keys[b] = off; off += align256(cap * 4); }
    if (!l.packed)
        for (int b = 0; b < 2; b++) { l.tile_vals[b] = off; off += align256(cap * 4); }
    l.total = off;
    *L = l;
    return true;
}

bool layout_for_bytes(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, size_t ws_bytes, Layout *L) {
    Layout l0;
    if (!make_layout(n, cam, cfg, 0, &l0) || (size_t)l0.total > ws_bytes) return false;
    int64_t lo = 0, hi = (int64_t)((ws_bytes - (size_t)l0.total) / 8) + 1;
    if (hi > (int64_t)((1u << 30) - 1u)) hi = (int64_t)((1u << 30) - 1u);
    Layout t;
    while (lo < hi) {   // largest cap whose layout fits
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (make_layout(n, cam, cfg, mid, &t) && (size_t)t.total <= ws_bytes) lo = mid; else hi = mid - 1;
    }
    return make_layout(n, cam, cfg, lo, L);
}

void make_view(const d4dgs_scene &s, const d4dgs_camera &cam, float t, const d4dgs_config &cfg, const Layout &L,
               void *ws, float *out_rgb, View *v) {
    View x;
    memset(&x, 0, sizeof(x));
    x.means = s.means; x.t_mean = s.t_mean; x.velocity = s.velocity; x.log_scales = s.log_scales;
    x.log_t_scale = s.log_t_scale; x.quats = s.quats; x.opacity_logit = s.opacity_logit; x.sh = s.sh;
    x.n = s.n;
    x.sh_degree = s.sh_degree;
    x.t = t;
    for (int i = 0; i < 3; i++) x.bg[i] = cfg.bg[i];
    x.cam = make_cam_args(&cam, cfg.tile, cfg.near > 0.0f ? cfg.near : kNear);
    x.spin_limit = cfg.spin_limit ? cfg.spin_limit : kSpinLimit;
    x.colour_cache = cfg.colour_cache;
    x.out_rgb = out_rgb;
    x.zero_base = at<char>(ws, 0);
    x.zero_bytes = L.zero_end;
    x.ctl = at<uint32_t>(ws, L.control);
    x.grid = at<int>(ws, L.grid);
    x.rec = at<float4>(ws, L.records);
    for (int b = 0; b < 2; b++) {
        x.dkeys[b] = at<uint32_t>(ws, L.depth_keys[b]);
        x.dvals[b] = at<uint32_t>(ws, L.depth_vals[b]);
        x.tkeys[b] = at<uint32_t>(ws, L.tile_keys[b]);
        x.tvals[b] = L.packed ? nullptr : at<uint32_t>(ws, L.tile_vals[b]);
    }
    x.tiles_touched = at<uint32_t>(ws, L.tiles_touched);
    x.rect = at<ushort4>(ws, L.rect);
    x.trim = at<unsigned long long>(ws, L.trim);
    x.ranges = at<uint2>(ws, L.ranges);
    x.tile_order = at<uint32_t>(ws, L.tile_order);
    x.tile_work = at<uint32_t>(ws, L.tile_work);
    x.final_T = at<float>(ws, L.final_T);
    x.n_contrib = at<uint32_t>(ws, L.n_contrib);
    x.grad2d = at<float>(ws, L.grad2d);
    x.flow2d = at<float2>(ws, L.flow2d);
    x.lb_depth = at<uint32_t>(ws, L.lb_depth);
    x.lb_tile = at<uint32_t>(ws, L.lb_tile);
    x.lb_col = at<uint32_t>(ws, L.lb_col);
    x.colbase = at<uint32_t>(ws, L.colbase);
    x.cmat = L.direct ? at<uint32_t>(ws, L.cmat) : nullptr;
    x.cgrp = L.direct ? at<unsigned long long>(ws, L.cgrp) : nullptr;
    x.cursor = L.rank_lists ? at<uint32_t>(ws, L.cursor) : nullptr;
    x.cap = (uint32_t)L.cap;
    x.id_bits = L.id_bits;
    x.col_bits = L.col_bits;
    x.packed = L.packed ? 1 : 0;
    x.tile_passes = L.tile_passes;
    x.trim_on = L.trim_on;
    x.ntiles = L.ntiles;
    for (int p = 0; p < 3; p++) {
        x.tile_shift[p] = L.tile_shift[p];
        x.tile_mask[p] = L.tile_pass_bits[p] ? (1u << L.tile_pass_bits[p]) - 1u : 0u;
    }
    x.parts_depth = (int32_t)L.parts_depth;
    x.parts_dup = (int32_t)L.parts_dup;
    x.parts_tile = (int32_t)L.parts_tile;
    x.parts_dir = (int32_t)L.parts_dir;
    x.parts_rank = (int32_t)L.parts_rank;
    *v = x;
}

// Same scene arrays and camera (the time may differ): views that can share one
// read of each Gaussian in the preprocess.
static bool same_scene_and_camera(const View &a, const View &b) {
    return a.kind == b.kind && a.means == b.means && a.t_mean == b.t_mean && a.velocity == b.velocity &&
           a.log_scales == b.log_scales && a.log_t_scale == b.log_t_scale && a.quats == b.quats &&
           a.means4 == b.means4 && a.log_scales4 == b.log_scales4 && a.quat_l == b.quat_l && a.quat_r == b.quat_r &&
           a.opacity_logit == b.opacity_logit && a.sh == b.sh && a.n == b.n && a.sh_degree == b.sh_degree &&
           a.colour_cache == b.colour_cache && memcmp(&a.cam, &b.cam, sizeof(CamArgs)) == 0;
}

bool finish_batch(BatchArgs *b) {
    if (b->nviews < 1 || b->nviews > kMaxViews) return false;
    int64_t chunks = 0, dparts = 0, uparts = 0, tiles = 0, xparts = 0, bands = 0, rparts = 0;
    b->max_n = 0;
    b->col_cap = 32;
    b->tile_cap = 256;
    b->cells_cap = 256;
    b->packed = b->v[0].packed;
    b->tile_passes = b->v[0].tile_passes;
    b->trim_on = b->v[0].trim_on;
    int lead = -1;
    for (int i = 0; i < b->nviews; i++) {
        View &v = b->v[i];
        if (v.packed != b->packed || v.tile_passes != b->tile_passes || v.cam.tile != b->tile || v.trim_on != b->trim_on ||
            v.kind != b->v[0].kind || v.colour_cache != b->v[0].colour_cache ||
            (v.cmat != nullptr) != (b->v[0].cmat != nullptr) || (v.cursor != nullptr) != (b->v[0].cursor != nullptr))
            return false;
        // time groups: a view joins the group of the view before it when it shares its scene and camera
        if (lead >= 0 && b->v[lead].group_size < kMaxGroup && same_scene_and_camera(b->v[lead], v)) {
            b->v[lead].group_size++;
            v.group_size = 0;
            v.chunk_base = b->v[lead].chunk_base;
        } else {
            lead = i;
            v.group_size = 1;
            v.chunk_base = (int32_t)chunks;
            chunks += (v.n + kPreChunk - 1) / kPreChunk;
        }
        v.depth_part_base = (int32_t)dparts;
        v.dup_part_base = (int32_t)uparts;
        v.tile_base = (int32_t)tiles;
        v.dir_part_base = (int32_t)xparts;
        v.band_base = (int32_t)bands;
        v.rank_part_base = (int32_t)rparts;
        dparts += v.parts_depth;
        uparts += v.parts_dup;
        tiles += v.ntiles;
        if (v.cursor) rparts += v.parts_rank;   // rank lists (every view of the launch)
        if (v.cmat) {   // direct binning (tile_passes 1, so every view of the launch)
            xparts += v.parts_dir;
            bands += (v.ntiles + kDirBand - 1) / kDirBand;
        }
        if (v.n > b->max_n) b->max_n = v.n;
        while (b->col_cap < v.cam.tiles_x) b->col_cap *= 2;
        while (b->tile_cap < v.ntiles) b->tile_cap += 256;
        while (b->cells_cap < (v.cam.tiles_x + 1) * (v.cam.tiles_y + 1)) b->cells_cap += 256;
    }
    if (chunks > INT32_MAX || tiles > INT32_MAX || xparts > INT32_MAX || rparts > INT32_MAX) return false;
    b->total_rank_parts = (int32_t)rparts;
    b->total_dir_parts = (int32_t)xparts;
    b->total_bands = (int32_t)bands;
    b->total_chunks = (int32_t)chunks;
    b->total_depth_parts = (int32_t)dparts;
    b->total_dup_parts = (int32_t)uparts;
    b->total_tiles = (int32_t)tiles;
    return true;
}

}  // namespace d4dgs

namespace d4dgs {
thread_local LaunchTimer *g_launch_timer = nullptr;
}  // namespace d4dgs

using namespace d4dgs;

extern "C" {

size_t d4dgs_workspace_bytes(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, int64_t key_capacity) {
    Layout L;
    if (!make_layout(n, cam, cfg, key_capacity, &L)) return 0;
    return (size_t)L.total;
}

int d4dgs_workspace_layout(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, size_t ws_bytes,
                           d4dgs_layout *out) {
    if (!out || n < 0 || !valid_camera(cam) || !valid_config(cfg)) return D4DGS_ERR_INVALID_ARG;
    Layout L;
    if (!layout_for_bytes(n, cam, cfg, ws_bytes, &L)) return D4DGS_ERR_WORKSPACE_TOO_SMALL;
    out->records = L.records;
    out->depth_keys = L.depth_keys[0];
    out->tiles_touched = L.tiles_touched;
    out->rect = L.rect;
    out->trims = L.trim;
    out->depth_order = L.depth_vals[L.depth_passes & 1];
    out->tile_keys = L.tile_keys[L.final_buf()];
    out->tile_vals = L.packed ? -1 : L.tile_vals[L.final_buf()];
    out->ranges = L.ranges;
    out->tile_order = L.tile_order;
    out->final_T = L.final_T;
    out->n_contrib = L.n_contrib;
    out->control = L.control;
    out->key_capacity = L.cap;
    out->tiles_x = L.tiles_x;
    out->tiles_y = L.tiles_y;
    out->depth_passes = L.depth_passes;
    out->tile_passes = L.tile_passes;
    out->id_bits = L.id_bits;
    out->packed = L.packed ? 1 : 0;
    out->col_bits = L.col_bits;
    return D4DGS_OK;
}

static int prepare(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, void *ws, size_t ws_bytes,
                   Layout *L) {
    if (n < 0 || !valid_camera(cam) || !valid_config(cfg) || !ws || !aligned(ws, 256)) return D4DGS_ERR_INVALID_ARG;
    if (!layout_for_bytes(n, cam, cfg, ws_bytes, L)) return D4DGS_ERR_WORKSPACE_TOO_SMALL;
    return D4DGS_OK;
}

// One frame as a batch of one view; the scene may be null for stages that
// only read the table the preprocess installed (its n must then match).
static int single(const d4dgs_scene *scene, int32_t n, const d4dgs_camera *cam, float t, const d4dgs_config *cfg,
                  void *ws, size_t ws_bytes, float *out_rgb, BatchArgs *b, Layout *L) {
    int rc = prepare(n, cam, cfg, ws, ws_bytes, L);
    if (rc) return rc;
    d4dgs_scene empty{};
    empty.n = n;
    memset(b, 0, offsetof(BatchArgs, v) + sizeof(View));
    b->nviews = 1;
    b->tile = cfg->tile;
    b->batch = cfg->batch;
    make_view(scene ? *scene : empty, *cam, t, *cfg, *L, ws, out_rgb, &b->v[0]);
    return finish_batch(b) ? D4DGS_OK : D4DGS_ERR_INVALID_ARG;
}

int d4dgs_preprocess(const d4dgs_scene *scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg,
                     void *ws, size_t ws_bytes, d4dgs_stream_t stream) {
    int rc = check_scene(scene);
    if (rc) return rc;
    if (!isfinite(t)) return D4DGS_ERR_INVALID_ARG;
    static thread_local BatchArgs b;
    Layout L;
    if ((rc = single(scene, scene->n, cam, t, cfg, ws, ws_bytes, nullptr, &b, &L))) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ba = at<char>(ws, L.batch);
    const int sms = num_sms_current();
    cudaError_t e = launch_clear(b, nullptr, ba, st, sms);
    if (e == cudaSuccess) e = launch_preprocess(b, ba, st, sms, true);
    return cuda_status(e);
}

int d4dgs_sort(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, void *ws, size_t ws_bytes,
               d4dgs_stream_t stream) {
    static thread_local BatchArgs b;
    Layout L;
    int rc = single(nullptr, n, cam, 0.0f, cfg, ws, ws_bytes, nullptr, &b, &L);
    if (rc) return rc;
    return cuda_status(launch_sort(b, at<char>(ws, L.batch), reinterpret_cast<cudaStream_t>(stream), num_sms_current(), true));
}

int d4dgs_blend(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, void *ws, size_t ws_bytes,
                float *out_rgb, d4dgs_stream_t stream) {
    if (!out_rgb || !aligned(out_rgb, 4)) return D4DGS_ERR_INVALID_ARG;
    static thread_local BatchArgs b;
    Layout L;
    int rc = single(nullptr, n, cam, 0.0f, cfg, ws, ws_bytes, out_rgb, &b, &L);
    if (rc) return rc;
    return cuda_status(launch_blend(b, at<char>(ws, L.batch), reinterpret_cast<cudaStream_t>(stream),
                                    num_sms_current(), out_rgb));
}

int d4dgs_blend_profile(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, void *ws, size_t ws_bytes,
                        float *out_rgb, uint64_t *counts, d4dgs_stream_t stream) {
    if (!out_rgb || !counts || !aligned(counts, 8)) return D4DGS_ERR_INVALID_ARG;
    static thread_local BatchArgs b;
    Layout L;
    int rc = single(nullptr, n, cam, 0.0f, cfg, ws, ws_bytes, out_rgb, &b, &L);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ba = at<char>(ws, L.batch);
    // the blend's work counter is reset so that the same frame can be blended again
    if (cudaMemsetAsync(ba + 4 * kBaBlend, 0, 4, st) != cudaSuccess) return D4DGS_ERR_CUDA;
    if (cudaMemsetAsync(counts, 0, 3 * sizeof(uint64_t), st) != cudaSuccess) return D4DGS_ERR_CUDA;
    return cuda_status(launch_blend(b, ba, st, num_sms_current(), out_rgb, reinterpret_cast<unsigned long long *>(counts)));
}

int d4dgs_render(const d4dgs_scene *scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg, void *ws,
                 size_t ws_bytes, float *out_rgb, d4dgs_stream_t stream) {
    if (!out_rgb || !aligned(out_rgb, 4)) return D4DGS_ERR_INVALID_ARG;
    int rc = check_scene(scene);
    if (rc) return rc;
    if (!isfinite(t)) return D4DGS_ERR_INVALID_ARG;
    static thread_local BatchArgs b;
    Layout L;
    if ((rc = single(scene, scene->n, cam, t, cfg, ws, ws_bytes, out_rgb, &b, &L))) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ba = at<char>(ws, L.batch);
    const int sms = num_sms_current();
    cudaError_t e = launch_clear(b, nullptr, ba, st, sms);
    if (e == cudaSuccess) e = launch_preprocess(b, ba, st, sms, true);
    if (e == cudaSuccess) e = launch_sort(b, ba, st, sms, true);
    if (e == cudaSuccess) e = launch_blend(b, ba, st, sms, nullptr);
    return cuda_status(e);
}

// A slicing-first frame as a batch of one view.
static int single4d(const d4dgs_scene4d *s, const d4dgs_camera *cam, float t, const d4dgs_config *cfg, void *ws,
                    size_t ws_bytes, float *out_rgb, BatchArgs *b, Layout *L) {
    int rc = check_scene4d(s);
    if (rc) return rc;
    if (!isfinite(t)) return D4DGS_ERR_INVALID_ARG;
    if ((rc = single(nullptr, s->n, cam, t, cfg, ws, ws_bytes, out_rgb, b, L))) return rc;
    View &v = b->v[0];
    v.kind = 1;
    v.means4 = s->means4; v.log_scales4 = s->log_scales4; v.quat_l = s->quat_l; v.quat_r = s->quat_r;
    v.opacity_logit = s->opacity_logit; v.sh = s->sh;
    v.sh_degree = s->sh_degree;
    return D4DGS_OK;
}

int d4dgs_preprocess_slicing(const d4dgs_scene4d *scene, const d4dgs_camera *cam, float t,
                             const d4dgs_config *cfg, void *ws, size_t ws_bytes, d4dgs_stream_t stream) {
    static thread_local BatchArgs b;
    Layout L;
    int rc = single4d(scene, cam, t, cfg, ws, ws_bytes, nullptr, &b, &L);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ba = at<char>(ws, L.batch);
    const int sms = num_sms_current();
    cudaError_t e = launch_clear(b, nullptr, ba, st, sms);
    if (e == cudaSuccess) e = launch_preprocess(b, ba, st, sms, true);
    return cuda_status(e);
}

int d4dgs_render_slicing(const d4dgs_scene4d *scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg,
                         void *ws, size_t ws_bytes, float *out_rgb, d4dgs_stream_t stream) {
    if (!out_rgb || !aligned(out_rgb, 4)) return D4DGS_ERR_INVALID_ARG;
    static thread_local BatchArgs b;
    Layout L;
    int rc = single4d(scene, cam, t, cfg, ws, ws_bytes, out_rgb, &b, &L);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ba = at<char>(ws, L.batch);
    const int sms = num_sms_current();
    cudaError_t e = launch_clear(b, nullptr, ba, st, sms);
    if (e == cudaSuccess) e = launch_preprocess(b, ba, st, sms, true);
    if (e == cudaSuccess) e = launch_sort(b, ba, st, sms, true);
    if (e == cudaSuccess) e = launch_blend(b, ba, st, sms, nullptr);
    return cuda_status(e);
}

static int backward_common(const d4dgs_scene *scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg,
                           void *ws, size_t ws_bytes, const float *dl_drgb, d4dgs_scene_grad *grad,
                           d4dgs_stream_t stream, bool accumulate) {
    int rc = check_scene(scene);
    if (rc) return rc;
    if (!isfinite(t) || !dl_drgb || !grad) return D4DGS_ERR_INVALID_ARG;
    if (scene->n > 0) {
        float *gp[] = {grad->means, grad->t_mean, grad->velocity, grad->log_scales, grad->log_t_scale, grad->quats,
                       grad->opacity_logit, grad->sh};
        for (float *p : gp)
            if (!p || !aligned(p, 4)) return D4DGS_ERR_INVALID_ARG;
        // the coefficient gradients are written as float4 rows (degree 1 and 3), like the scene's rows
        if ((scene->sh_degree == 1 || scene->sh_degree == 3) && !aligned(grad->sh, 16)) return D4DGS_ERR_INVALID_ARG;
    }
    static thread_local BatchArgs b;
    Layout L;
    if ((rc = single(scene, scene->n, cam, t, cfg, ws, ws_bytes, nullptr, &b, &L))) return rc;
    return cuda_status(launch_backward(b, at<char>(ws, L.batch), dl_drgb, nullptr, *grad,
                                       reinterpret_cast<cudaStream_t>(stream), num_sms_current(), accumulate));
}

int d4dgs_render_backward(const d4dgs_scene *scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg,
                          void *ws, size_t ws_bytes, const float *dl_drgb, d4dgs_scene_grad *grad,
                          d4dgs_stream_t stream) {
    return backward_common(scene, cam, t, cfg, ws, ws_bytes, dl_drgb, grad, stream, false);
}

int d4dgs_render_backward_accumulate(const d4dgs_scene *scene, const d4dgs_camera *cam, float t,
                                     const d4dgs_config *cfg, void *ws, size_t ws_bytes, const float *dl_drgb,
                                     d4dgs_scene_grad *grad, d4dgs_stream_t stream) {
    return backward_common(scene, cam, t, cfg, ws, ws_bytes, dl_drgb, grad, stream, true);
}

int d4dgs_launch_timer(void *const *events, int32_t n_events) {
    static thread_local LaunchTimer timer;
    if (!events || n_events < 1) return D4DGS_ERR_INVALID_ARG;
    timer.events = reinterpret_cast<cudaEvent_t *>(const_cast<void **>(events));
    timer.n = n_events;
    timer.used = 0;
    g_launch_timer = &timer;
    return D4DGS_OK;
}

int32_t d4dgs_launch_timer_stop(void) {
    LaunchTimer *t = g_launch_timer;
    g_launch_timer = nullptr;
    return t ? t->used : 0;
}

int d4dgs_render_flow(const d4dgs_scene *scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg, void *ws,
                      size_t ws_bytes, float *out_rgb, float *out_flow, d4dgs_stream_t stream) {
    if (!out_rgb || !aligned(out_rgb, 4) || !out_flow || !aligned(out_flow, 4)) return D4DGS_ERR_INVALID_ARG;
    int rc = check_scene(scene);
    if (rc) return rc;
    if (!isfinite(t)) return D4DGS_ERR_INVALID_ARG;
    static thread_local BatchArgs b;
    Layout L;
    if ((rc = single(scene, scene->n, cam, t, cfg, ws, ws_bytes, out_rgb, &b, &L))) return rc;
    b.v[0].out_flow = out_flow;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ba = at<char>(ws, L.batch);
    const int sms = num_sms_current();
    cudaError_t e = launch_clear(b, nullptr, ba, st, sms);
    if (e == cudaSuccess) e = launch_preprocess(b, ba, st, sms, true);
    if (e == cudaSuccess) e = launch_sort(b, ba, st, sms, true);
    if (e == cudaSuccess) e = launch_blend(b, ba, st, sms, nullptr);
    return cuda_status(e);
}

int d4dgs_render_backward_flow(const d4dgs_scene *scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg,
                               void *ws, size_t ws_bytes, const float *dl_drgb, const float *dl_dflow,
                               d4dgs_scene_grad *grad, d4dgs_stream_t stream) {
    int rc = check_scene(scene);
    if (rc) return rc;
    if (!isfinite(t) || !dl_drgb || !dl_dflow || !grad) return D4DGS_ERR_INVALID_ARG;
    if (scene->n > 0) {
        float *gp[] = {grad->means, grad->t_mean, grad->velocity, grad->log_scales, grad->log_t_scale, grad->quats,
                       grad->opacity_logit, grad->sh};
        for (float *p : gp)
            if (!p || !aligned(p, 4)) return D4DGS_ERR_INVALID_ARG;
        // the coefficient gradients are written as float4 rows (degree 1 and 3), like the scene's rows
        if ((scene->sh_degree == 1 || scene->sh_degree == 3) && !aligned(grad->sh, 16)) return D4DGS_ERR_INVALID_ARG;
    }
    static thread_local BatchArgs b;
    Layout L;
    if ((rc = single(scene, scene->n, cam, t, cfg, ws, ws_bytes, nullptr, &b, &L))) return rc;
    return cuda_status(launch_backward(b, at<char>(ws, L.batch), dl_drgb, dl_dflow, *grad,
                                       reinterpret_cast<cudaStream_t>(stream), num_sms_current()));
}

size_t d4dgs_batch_args_bytes(void) { return sizeof(BatchArgs); }
size_t d4dgs_batch_area_bytes(void) { return (size_t)kBatchAreaBytes; }

int d4dgs_batch_encode(int32_t nviews, const d4dgs_view *views, const d4dgs_config *cfg, void *args_host,
                       size_t args_bytes) {
    if (nviews < 1 || nviews > kMaxViews || !views || !valid_config(cfg) || !args_host ||
        args_bytes < sizeof(BatchArgs))
        return D4DGS_ERR_INVALID_ARG;
    BatchArgs *b = static_cast<BatchArgs *>(args_host);
    memset(b, 0, sizeof(BatchArgs));
    b->nviews = nviews;
    b->tile = cfg->tile;
    b->batch = cfg->batch;
    for (int i = 0; i < nviews; i++) {
        const d4dgs_view &q = views[i];
        int rc = check_scene(q.scene);
        if (rc) return rc;
        if (!isfinite(q.t) || !q.out_rgb || !aligned(q.out_rgb, 4)) return D4DGS_ERR_INVALID_ARG;
        Layout L;
        if ((rc = prepare(q.scene->n, &q.cam, cfg, q.ws, q.ws_bytes, &L))) return rc;
        make_view(*q.scene, q.cam, q.t, *cfg, L, q.ws, q.out_rgb, &b->v[i]);
    }
    return finish_batch(b) ? D4DGS_OK : D4DGS_ERR_INVALID_ARG;
}

int d4dgs_render_batch_stages(const void *args_host, const void *args_dev, void *batch_area,
                              size_t batch_area_bytes, int32_t stages, d4dgs_stream_t stream) {
    if (!args_host || !batch_area || !aligned(batch_area, 256) || batch_area_bytes < (size_t)kBatchAreaBytes ||
        stages < 0 || stages > 7)
        return D4DGS_ERR_INVALID_ARG;
    if (args_dev && !aligned(args_dev, 16)) return D4DGS_ERR_INVALID_ARG;
    const BatchArgs &b = *static_cast<const BatchArgs *>(args_host);
    if (b.nviews < 1 || b.nviews > kMaxViews) return D4DGS_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ba = static_cast<char *>(batch_area);
    const int sms = num_sms_current();
    cudaError_t e = cudaSuccess;
    if (stages & 1) e = launch_clear(b, args_dev, ba, st, sms);
    if (e == cudaSuccess && (stages & 1)) e = launch_preprocess(b, ba, st, sms, args_dev == nullptr);
    if (e == cudaSuccess && (stages & 2)) e = launch_sort(b, ba, st, sms, args_dev == nullptr);
    if (e == cudaSuccess && (stages & 4)) e = launch_blend(b, ba, st, sms, nullptr, nullptr, /*persist=*/true);
    return cuda_status(e);
}

int d4dgs_render_batch(const void *args_host, const void *args_dev, void *batch_area, size_t batch_area_bytes,
                       d4dgs_stream_t stream) {
    return d4dgs_render_batch_stages(args_host, args_dev, batch_area, batch_area_bytes, 7, stream);
}

int d4dgs_read_stats(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, const void *ws, size_t ws_bytes,
                     d4dgs_stats *out, d4dgs_stream_t stream) {
    if (!out) return D4DGS_ERR_INVALID_ARG;
    Layout L;
    int rc = prepare(n, cam, cfg, const_cast<void *>(ws), ws_bytes, &L);
    if (rc) return rc;
    if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return D4DGS_ERR_CUDA;
    uint32_t words[4] = {0, 0, 0, 0};
    if (cudaMemcpy(words, static_cast<const char *>(ws) + L.control, sizeof(words), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return D4DGS_ERR_CUDA;
    out->status = (words[kCtlStatus] & kStatusTimeout) ? D4DGS_ERR_TIMEOUT
                  : (words[kCtlStatus] & kStatusCapacity) ? D4DGS_ERR_CAPACITY
                                                          : D4DGS_OK;
    out->n_keys = words[kCtlNumKeys];
    out->key_capacity = L.cap;
    out->n_visible = words[kCtlNumVisible];
    return out->status;
}

size_t d4dgs_scene_bytes(int32_t n, int32_t sh_degree) {
    if (n < 0 || sh_degree < 0 || sh_degree > 3) return 0;
    const int64_t k = (int64_t)(sh_degree + 1) * (sh_degree + 1);
    const int64_t cols[8] = {3, 1, 3, 3, 1, 4, 1, 3 * k};
    int64_t off = 0;
    for (int64_t c : cols) off += (((int64_t)n * c * 4) + 255) & ~(int64_t)255;
    return (size_t)off;
}

// Copies in, frame, copy out, all on `stream`; waits for the stream when `sync`.
static int render_host(const d4dgs_scene *host_scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg,
                       void *dev_scene_buf, size_t dev_scene_bytes, void *ws, size_t ws_bytes, void *dev_rgb,
                       float *out_rgb_host, d4dgs_stream_t stream, bool sync) {
    if (!host_scene || host_scene->n < 0 || host_scene->sh_degree < 0 || host_scene->sh_degree > 3)
        return D4DGS_ERR_INVALID_ARG;
    if (!dev_scene_buf || !aligned(dev_scene_buf, 256) || !dev_rgb || !out_rgb_host || !valid_camera(cam))
        return D4DGS_ERR_INVALID_ARG;
    const int32_t n = host_scene->n;
    if (dev_scene_bytes < d4dgs_scene_bytes(n, host_scene->sh_degree)) return D4DGS_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t k = (int64_t)(host_scene->sh_degree + 1) * (host_scene->sh_degree + 1);
    const float *src[8] = {host_scene->means, host_scene->t_mean, host_scene->velocity, host_scene->log_scales,
                           host_scene->log_t_scale, host_scene->quats, host_scene->opacity_logit, host_scene->sh};
    const int64_t cols[8] = {3, 1, 3, 3, 1, 4, 1, 3 * k};
    float *dst[8];
    int64_t off = 0;
    for (int a = 0; a < 8; a++) {
        dst[a] = reinterpret_cast<float *>(static_cast<char *>(dev_scene_buf) + off);
        const size_t bytes = (size_t)n * cols[a] * 4;
        if (n > 0) {
            if (!src[a]) return D4DGS_ERR_INVALID_ARG;
            if (cudaMemcpyAsync(dst[a], src[a], bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return D4DGS_ERR_CUDA;
        }
        off += ((int64_t)bytes + 255) & ~(int64_t)255;
    }
    d4dgs_scene dev{dst[0], dst[1], dst[2], dst[3], dst[4], dst[5], dst[6], dst[7], n, host_scene->sh_degree};
    int rc = d4dgs_render(&dev, cam, t, cfg, ws, ws_bytes, static_cast<float *>(dev_rgb), stream);
    if (rc) return rc;
    const size_t img = (size_t)cam->width * cam->height * 3 * sizeof(float);
    if (cudaMemcpyAsync(out_rgb_host, dev_rgb, img, cudaMemcpyDeviceToHost, st) != cudaSuccess) return D4DGS_ERR_CUDA;
    if (sync && cudaStreamSynchronize(st) != cudaSuccess) return D4DGS_ERR_CUDA;
    return D4DGS_OK;
}

int d4dgs_render_host(const d4dgs_scene *host_scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg,
                      void *dev_scene_buf, size_t dev_scene_bytes, void *ws, size_t ws_bytes, void *dev_rgb,
                      float *out_rgb_host, d4dgs_stream_t stream) {
    return render_host(host_scene, cam, t, cfg, dev_scene_buf, dev_scene_bytes, ws, ws_bytes, dev_rgb, out_rgb_host,
                       stream, true);
}

int d4dgs_render_host_async(const d4dgs_scene *host_scene, const d4dgs_camera *cam, float t,
                            const d4dgs_config *cfg, void *dev_scene_buf, size_t dev_scene_bytes, void *ws,
                            size_t ws_bytes, void *dev_rgb, float *out_rgb_host, d4dgs_stream_t stream) {
    return render_host(host_scene, cam, t, cfg, dev_scene_buf, dev_scene_bytes, ws, ws_bytes, dev_rgb, out_rgb_host,
                       stream, false);
}

int d4dgs_launches_per_frame(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg) {
    Layout L;
    if (!make_layout(n, cam, cfg, 0, &L)) return D4DGS_ERR_INVALID_ARG;
    // clear + preprocess + sort stages + blend
    return 1 + (n > 0 ? 1 : 0) + sort_launch_count(n, L.tile_passes, (L.tiles_x + 1) * (L.tiles_y + 1)) + 1;
}

const char *d4dgs_strerror(int code) {
    switch (code) {
        case D4DGS_OK: return "ok";
        case D4DGS_ERR_INVALID_ARG: return "invalid argument";
        case D4DGS_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
        case D4DGS_ERR_CAPACITY: return "more (tile, Gaussian) pairs than the workspace key capacity";
        case D4DGS_ERR_TIMEOUT: return "a bounded device spin-wait timed out";
        case D4DGS_ERR_CUDA: return "CUDA runtime error";
        default: return "unknown status";
    }
}

}  // extern "C"
