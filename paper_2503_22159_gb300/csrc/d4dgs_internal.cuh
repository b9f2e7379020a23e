// d4dgs_internal.cuh -- shared definitions of the sm_103a renderer: workspace
// layout, control-block words, kernel entry declarations.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/d4dgs.h"

namespace d4dgs {

// ---- rasteriser constants (3DGS conventions the paper reuses, Sec. III-B-2)
constexpr float kNear = 0.2f;          // default near plane on camera z (config near = 0)
constexpr float kDilation = 0.3f;      // px^2 added to the 2D covariance diagonal
constexpr float kJacClamp = 1.3f;      // x/z, y/z clamp, times half the field of view
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kRadiusK = 3.33f;      // 3.33^2 > 2 ln 255: covers every alpha >= 1/255
// margin on k^2 = 2 ln(255 o_hat) of the binning ellipse (k^2 * kK2Scale + kK2Pad)
constexpr float kK2Scale = 1.0008f;
constexpr float kK2Pad = 0.0008f;

// ---- sort geometry
constexpr int kSortThreads = 256;
constexpr int kTileIPT = 20;                              // pair keys per thread (tile passes; 15: +2.7 us)
constexpr int kTileItems = kSortThreads * kTileIPT;       // 5120 pairs per partition
// tile-count grids of at most this many cells ride with the first depth pass
constexpr int kTileCountCells = 6144;
constexpr int kMaxCols = 2048;                            // tile columns of a view (16384 px at 8-px tiles)
constexpr int kDepthIPT = 8;                              // depth keys per thread: 2048-key partitions
constexpr int kDepthItems = kSortThreads * kDepthIPT;     // (A/B: 14.3 against 16.4 us per pass at 1024)
constexpr int kRadix = 256;                               // digit bins (<= 8 bits per pass)
constexpr int kDupThreads = 256;
constexpr int kDupItems = kDupThreads;                    // depth-ordered Gaussians per scan partition
// direct binning (config binning 2): per-(partition, tile) pair counts over
// partitions of kDirItems depth-ordered Gaussians, scanned down each tile's
// column of the count matrix in bands of kDirBand tiles
constexpr int kDirItems = 256;
constexpr int kDirMaxTiles = 2048;
constexpr int kDirBand = 8;
// rank lists (config binning 3): emission partitions of kRankItems depth-ordered
// Gaussians; the list kernel's depth-order bitmap is at most kRankMaxWords words
constexpr int kRankThreads = 1024;
constexpr int kRankItems = 1024;
constexpr int kRankListThreads = 256;
constexpr int kRankMaxWords = 40960;   // 160 KB: one window covers 1.3 M Gaussians

// ---- control block (uint32 words at layout.control)
enum : int {
    kCtlStatus = 0,        // bit 0: key capacity exceeded, bit 1: spin-wait timeout
    kCtlNumKeys = 1,       // total (tile, Gaussian) pairs of the frame (clamped reads use min(cap))
    kCtlNumVisible = 2,    // Gaussians with at least one tile
    kCtlPartBase = 4,      // partition counters: depth passes 4..7, scan+emit 8, tile passes 9..11
    kCtlDepthHist = 64,    // 4 x 256 digit counts of the depth keys
    kCtlTileHist = 64 + 4 * kRadix,   // 3 x 256 digit counts of the pair keys (tile rows)
    kCtlWords = 2048
};
constexpr uint32_t kStatusCapacity = 1u;
constexpr uint32_t kStatusTimeout = 2u;

// Bounded spin: polls before a wait gives up and latches kStatusTimeout
// (the default of config spin_limit).
constexpr uint32_t kSpinLimit = 1u << 20;

struct Layout {
    int32_t n = 0, width = 0, height = 0, tile = 0, tiles_x = 0, tiles_y = 0, ntiles = 0;
    int64_t pixels = 0;
    int32_t depth_passes = 4;
    // pass 0 of the tile sort is the column bucketing done by the emission;
    // passes 1.. sort stably by the tile row, so a pair's key is its tile row
    // (tile_bits = row_bits; tile_shift / tile_pass_bits of passes 1.. are
    // relative to it); direct binning has the one pass of its emission
    int32_t col_bits = 0, row_bits = 0, tile_bits = 0, tile_passes = 0;
    int32_t tile_shift[3] = {0, 0, 0}, tile_pass_bits[3] = {0, 0, 0};
    // pairs are packed as (row << id_bits | id) in one uint32 when they fit,
    // else kept as a row key plus a separate Gaussian-id value
    int32_t id_bits = 0;
    bool packed = true;
    int32_t trim_on = 0;   // config trim: 1 rectangles cut per column (tile_trim.cuh), 0 whole
    int64_t cap = 0;
    int64_t parts_depth = 0, parts_dup = 0, parts_tile = 0, parts_dir = 0;
    bool direct = false;   // config binning 2: pairs emitted straight into their tiles' lists (tile_passes 1)
    // config binning 3: ranks emitted unordered, each tile's list built from a depth-order bitmap
    // (tile_passes 0: the lists end in tile_keys[0], the unordered ranks go to tile_keys[1])
    bool rank_lists = false;
    int64_t parts_rank = 0;
    // zero-initialised region [0, zero_end)
    int64_t control = 0, grid = 0, lb_depth = 0, lb_col = 0, lb_tile = 0, cursor = 0, zero_end = 0;
    // the rest
    int64_t tile_order = 0, tile_work = 0;   // ntiles uint32 each, written by the backward
    int64_t cmat = 0;      // direct binning: parts_dir x ntiles uint32 (not cleared: every entry is written)
    int64_t cgrp = 0;      // direct binning: parts_dir x ntiles uint64 group counts (likewise)
    int64_t colbase = 0, ranges = 0, records = 0, depth_keys[2] = {0, 0}, depth_vals[2] = {0, 0}, tiles_touched = 0, rect = 0;
    int64_t trim = 0;   // per-Gaussian column trims of the rectangle (tile_trim.cuh)
    int64_t final_T = 0, n_contrib = 0, grad2d = 0, flow2d = 0, batch = 0, tile_keys[2] = {0, 0}, tile_vals[2] = {-1, -1};
    int64_t total = 0;
    int32_t grid_w() const { return tiles_x + 1; }
    // index of the final sorted pair buffer
    int final_buf() const { return tile_passes & 1; }
};

// Fills `L` for a workspace holding `cap` keys; returns false on bad arguments.
bool make_layout(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, int64_t cap, Layout *L);
// Largest capacity whose layout fits in ws_bytes; false if none fits.
bool layout_for_bytes(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, size_t ws_bytes, Layout *L);

template <typename T>
__host__ __device__ inline T *at(void *ws, int64_t off) {
    return reinterpret_cast<T *>(static_cast<char *>(ws) + off);
}

// Camera constants of one view.
struct CamArgs {
    float R[9], T[3];
    float fx, fy, cx, cy;
    float campos[3];       // -R^T T, for the SH view direction
    float near;            // near plane on camera z
    // limits of the Jacobian's x/z and y/z clamp, 1.3 times the half field of view:
    // kJacClamp * ((width / 2) / fx) with each operation rounded to single precision
    float limx, limy;
    int32_t width, height, tile, tiles_x, tiles_y;
};
CamArgs make_cam_args(const d4dgs_camera *cam, int32_t tile, float near);

// Everything the kernels need about one frame (scene, camera, time, settings
// and the absolute addresses of its workspace buffers).  A launch processes a
// table of up to kMaxViews of them; a single frame is a table of one.
constexpr int kMaxViews = 32;
constexpr int kMaxGroup = 4;     // views per time group
struct View {
    const float *means, *t_mean, *velocity, *log_scales, *log_t_scale, *quats, *opacity_logit, *sh;
    // slicing-first scenes (kind 1): 4D means, 4D log-scales, rotation quaternion pair
    const float *means4, *log_scales4, *quat_l, *quat_r;
    int32_t kind;                    // 0: disentangled, 1: slicing-first
    int32_t n, sh_degree;
    float t;
    float bg[3];
    CamArgs cam;
    float *out_rgb;
    char *zero_base;                 // [zero_base, zero_base + zero_bytes) is cleared per frame
    int64_t zero_bytes;
    uint32_t *ctl;
    int *grid;
    float4 *rec;
    uint32_t *dkeys[2], *dvals[2], *tiles_touched;
    ushort4 *rect;
    unsigned long long *trim;        // column trims of each rectangle (tile_trim.cuh)
    uint2 *ranges;
    uint32_t *tile_order;            // tiles, most walked entries first (written by the backward)
    uint32_t *tile_work;             // per tile: list entries the forward walked, summed over its pixels
    float *final_T;
    uint32_t *n_contrib;
    float *grad2d;
    float2 *flow2d;                  // per-Gaussian screen flow (pixels per unit time), flow frames only
    float *out_flow;                 // H x W x 2 blended flow output, or null (no flow channel)
    uint32_t *tkeys[2], *tvals[2];
    uint32_t *lb_depth, *lb_tile, *lb_col;
    uint32_t *colbase;               // first position of each tile column's bucket (clamped to cap)
    uint32_t *cmat;                  // direct binning: parts_dir x ntiles pair counts, then list offsets
    unsigned long long *cgrp;        // direct binning: parts_dir x ntiles, byte g = pairs of group g
    uint32_t *cursor;                // rank lists: per tile, the pairs reserved so far (zeroed per frame)
    uint32_t cap;
    int32_t id_bits, col_bits, packed, tile_passes, ntiles;
    int32_t trim_on;                 // config trim: 1 rectangles cut per column
    uint32_t spin_limit;             // polls before a look-back gives up (config spin_limit)
    int32_t colour_cache;            // config colour_cache: SH colour towards the static mean
    int32_t tile_shift[3];
    uint32_t tile_mask[3];
    int32_t parts_depth, parts_dup, parts_tile, parts_dir, parts_rank;
    // time group: consecutive views of one scene seen by one camera (times may
    // differ) are preprocessed together, reading each Gaussian once; the
    // group's first view carries group_size (others 0) and the chunk base
    int32_t group_size;
    // first flattened work item of this view within its table
    int32_t chunk_base, depth_part_base, dup_part_base, tile_base, dir_part_base, band_base, rank_part_base;
};

// Descriptor table as kernel parameters (it travels by value: 32 views fit in
// the parameter space) plus the totals of the flattened work spaces.
struct BatchArgs {
    int32_t nviews;
    int32_t tile, batch, packed, tile_passes;   // shared by every view of a launch
    int32_t col_cap;                            // power of two >= every view's tile columns
    int32_t trim_on;                            // config trim, shared by every view of a launch
    int32_t tile_cap;                           // direct binning: multiple of 256 >= every view's tiles
    int32_t cells_cap;                          // direct binning: multiple of 256 >= every (tiles_x+1)(tiles_y+1)
    int32_t total_chunks, total_depth_parts, total_dup_parts, total_tiles, total_dir_parts, total_bands;
    int32_t total_rank_parts;                   // rank lists: emission partitions of every view
    int32_t max_n;
    View v[kMaxViews];
};

// Batch area (device): work counters of every launch, launch totals, and the
// descriptor table written by the first kernel of a frame.
enum : int {
    kBaChunk = 0,          // preprocess chunk counter
    kBaDepth = 1,          // 1..4 depth passes
    kBaDup = 5,            // scan + emit
    kBaTile = 6,           // 6..8 tile passes
    kBaBlend = 9,
    kBaBack = 10,
    kBaDirCount = 11,      // direct binning: counts, emission
    kBaDirEmit = 12,
    kBaRankEmit = 13,      // rank lists: emission, list building
    kBaRankList = 14,
    kBaNViews = 16, kBaTotalChunks, kBaTotalDepthParts, kBaTotalDupParts, kBaTotalTiles, kBaTotalDirParts,
    kBaTotalBands, kBaTotalRankParts,
    kBaWords = 64
};
constexpr int64_t kBatchTableOffset = 256;
constexpr int64_t kBatchAreaBytes = kBatchTableOffset + (int64_t)sizeof(View) * kMaxViews;
constexpr int kPreChunk = 256;   // Gaussians per preprocess work item

// Fill `v` for one frame in workspace `ws` with layout `L`.
void make_view(const d4dgs_scene &s, const d4dgs_camera &cam, float t, const d4dgs_config &cfg, const Layout &L,
               void *ws, float *out_rgb, View *v);
// Fill the flattened bases and totals; false if the views cannot share a launch.
bool finish_batch(BatchArgs *b);

// ---- launchers (each returns the cudaError_t of its launches).  `args` is the
// host copy; `args_dev`, when not null, is a device copy the first kernel reads
// instead of its by-value parameter (for CUDA graphs whose descriptors change).
cudaError_t launch_clear(const BatchArgs &args, const void *args_dev, char *batch_area, cudaStream_t st, int num_sms);
// host_views: args is the batch the kernels will read (false when the first
// kernel takes the descriptors from device memory instead)
cudaError_t launch_preprocess(const BatchArgs &args, const char *batch_area, cudaStream_t st, int num_sms,
                              bool host_views);
cudaError_t launch_sort(const BatchArgs &args, char *batch_area, cudaStream_t st, int num_sms, bool host_views);
cudaError_t launch_blend(const BatchArgs &args, char *batch_area, cudaStream_t st, int num_sms, float *out0,
                         unsigned long long *counts = nullptr, bool persist = false);
cudaError_t launch_backward(const BatchArgs &args, char *batch_area, const float *dl_drgb, const float *dl_dflow,
                            const d4dgs_scene_grad &g, cudaStream_t st, int num_sms, bool accumulate = false);
int sort_launch_count(int n, int tile_passes, int grid_cells);   // tile_passes 1: direct binning

__device__ __forceinline__ const View &view_of(const char *batch_area, int v) {
    return reinterpret_cast<const View *>(batch_area + kBatchTableOffset)[v];
}

// ---- device helpers
__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_volatile_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_volatile_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// 2^x for the compositing alpha (x in [log2(1/255), 0], so no denormal handling
// is needed); the forward and backward blends share it so that the backward
// recomputes the forward's alpha exactly.
__device__ __forceinline__ float alpha_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// Class of a tile's work (list entries walked, summed over its pixels) for the
// heaviest-first tile orders: 0 for none, else 1 + 4 floor(log2 k) + the two
// bits below k's leading one (quarter octaves).
constexpr int kWorkClasses = 1 + 4 * 32;
__device__ __forceinline__ int work_class(uint32_t k) {
    if (k == 0u) return 0;
    const int l = 31 - __clz(k);
    const uint32_t f = l >= 2 ? (k >> (l - 2)) & 3u : (k << (2 - l)) & 3u;
    return 1 + 4 * l + (int)f;
}
// The work classes' first positions from the heaviest down (s_cls[c]: the count of class c in,
// its first position out), by one whole warp: lane l takes kWorkClassRun consecutive classes
// below the heaviest l * kWorkClassRun, then a warp scan of the lanes' totals.
constexpr int kWorkClassRun = (kWorkClasses + 31) / 32;
__device__ __forceinline__ void work_class_scan(uint32_t *s_cls) {
    const int lane = (int)(threadIdx.x & 31u);
    uint32_t cnt[kWorkClassRun], sum = 0;
#pragma unroll
    for (int j = 0; j < kWorkClassRun; j++) {
        const int c = kWorkClasses - 1 - lane * kWorkClassRun - j;
        cnt[j] = c >= 0 ? s_cls[c] : 0u;
        sum += cnt[j];
    }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    uint32_t pos = x - sum;
#pragma unroll
    for (int j = 0; j < kWorkClassRun; j++) {
        const int c = kWorkClasses - 1 - lane * kWorkClassRun - j;
        if (c >= 0) s_cls[c] = pos;
        pos += cnt[j];
    }
}
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Chained launches (programmatic dependent launch): the forward kernels of a
// frame are launched with programmatic stream serialisation, so the launch of
// a kernel overlaps the end of the one before it in the stream.  Every such
// kernel calls grid_dependency_wait() before its first memory access; it
// returns once the preceding kernel has completed and its writes are visible
// (at once for a kernel launched without the attribute).
constexpr bool kChainedLaunch = true;

__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch timer (d4dgs_launch_timer): while one is installed on a host thread,
// every kernel launch of that thread is followed by a record of the next of
// the caller's events on the launch's stream.
struct LaunchTimer {
    cudaEvent_t *events;
    int n, used;
};
extern thread_local LaunchTimer *g_launch_timer;
inline void note_launch(cudaStream_t st) {
    LaunchTimer *t = g_launch_timer;
    if (t && t->used < t->n && cudaEventRecord(t->events[t->used], st) == cudaSuccess) t->used++;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                           Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = kChainedLaunch ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
    if (e == cudaSuccess) note_launch(st);
    return e;
}

}  // namespace d4dgs
