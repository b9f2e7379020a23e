/*
 * d4dgs.h -- C ABI of the GB300 (sm_103a) renderer for disentangled 4D
 * Gaussian splatting (Feng et al., "Disentangled 4D Gaussian Splatting",
 * arXiv 2503.22159).
 *
 * The library renders one frame of a dynamic scene at time t: the temporal
 * terms of every Gaussian are applied in the paper's deferred, disentangled
 * form (a time-shifted mean and a temporally modulated opacity, Sec. III-B-1,
 * Eq. 7-8), the Gaussian is projected to a dynamic 2D Gaussian (Sec.
 * III-B-2, Eq. 9-16; Algorithm 1), binned into screen tiles by (tile | depth)
 * keys and alpha-composited front to back per pixel (Sec. III-A, Eq. 4; the
 * 3DGS "fast rasterization" the paper reuses).
 *
 * Conventions shared by every entry point
 *   - All array pointers are DEVICE pointers owned by the caller (except the
 *     *_host entry points, which take host pointers).  The library never
 *     allocates device memory inside a call; scratch lives in a caller-owned
 *     workspace whose size d4dgs_workspace_bytes() returns.
 *   - Calls are asynchronous and stream-ordered on `stream`.  Argument errors
 *     are returned at call time.  Errors found on the device (key capacity
 *     exceeded, a bounded spin-wait that gave up) are latched in a status word
 *     inside the workspace and reported by d4dgs_read_stats() after the stream
 *     has been synchronised.
 *   - Parameters are raw (pre-activation): scales and temporal scale as logs,
 *     opacity as a logit, quaternions (w,x,y,z) not necessarily normalised.
 *   - Thread safety: calls on different workspaces may run concurrently; two
 *     calls in flight on the same workspace race.
 *   - Return value: D4DGS_OK (0) or a negative D4DGS_ERR_* code.
 */
#ifndef D4DGS_H
#define D4DGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *d4dgs_stream_t;

enum {
    D4DGS_OK = 0,
    D4DGS_ERR_INVALID_ARG = -1,          /* a pointer, size or enum out of range */
    D4DGS_ERR_WORKSPACE_TOO_SMALL = -2,  /* ws_bytes below what the call needs */
    D4DGS_ERR_CAPACITY = -3,             /* more (tile, Gaussian) keys than the workspace holds */
    D4DGS_ERR_TIMEOUT = -4,              /* a bounded spin-wait on the device gave up */
    D4DGS_ERR_CUDA = -5                  /* a CUDA runtime call or launch failed */
};

/* Per-Gaussian raw parameters, structure of arrays, float32, N rows each.
 * This is the paper's disentangled parameter set (Eq. 8): 4D scale (three
 * log spatial scales + log temporal scale s_t), 4D mean (mu_xyz, mu_t),
 * quaternion q and velocity V3D, plus the 3DGS opacity and SH colour. */
typedef struct {
    const float *means;          /* N x 3 : mu_x, mu_y, mu_z                        */
    const float *t_mean;         /* N     : mu_t                                    */
    const float *velocity;       /* N x 3 : V3D = V / W (Sec. III-B-1)              */
    const float *log_scales;     /* N x 3 : log s_x, log s_y, log s_z               */
    const float *log_t_scale;    /* N     : log s_t, s_t = sqrt(W)                  */
    const float *quats;          /* N x 4 : (w, x, y, z), any non-zero norm         */
    const float *opacity_logit;  /* N     : sigmoid gives the 3DGS opacity          */
    const float *sh;             /* N x (deg+1)^2 x 3 : real SH coefficients, RGB   */
    int32_t n;                   /* N >= 0                                          */
    int32_t sh_degree;           /* 0..3                                            */
} d4dgs_scene;

/* Gradients with respect to the raw parameters, same shapes as d4dgs_scene,
 * device float32, caller-owned; every array is overwritten. */
typedef struct {
    float *means, *t_mean, *velocity, *log_scales, *log_t_scale, *quats, *opacity_logit, *sh;
} d4dgs_scene_grad;

/* Pinhole camera (Algorithm 1 inputs P_camera, R_camera).  World -> camera
 * X_cam = R X_world + T, R row-major; the camera looks along +z, x right,
 * y down; u = fx X/Z + cx, v = fy Y/Z + cy; pixel (x, y) has its centre at
 * (x + 0.5, y + 0.5). */
typedef struct {
    float R[9];
    float T[3];
    float fx, fy, cx, cy;
    int32_t width, height;       /* 1 .. 16384 */
} d4dgs_camera;

/* Rasteriser settings.  tile: 8, 16 or 32 pixels; batch: Gaussians staged
 * per shared-memory batch in the blend, 64, 128 or 256, or 512 at 32-px
 * tiles;
 * bg: background colour added with the final transmittance; trim: 0 bins
 * each Gaussian into its whole tile rectangle, 1 cuts the rectangle's first
 * 8 columns to the tile rows its alpha >= 1/255 ellipse reaches (fewer
 * pairs, more binning arithmetic: worth it for large splats; the image is
 * the same either way); near: the near plane on camera z (Sec. III-B-2
 * defers to the 3DGS rasteriser, whose plane is 0.2; 0 selects 0.2), a
 * Gaussian is drawn only when its time-shifted mean lies beyond it;
 * spin_limit: polls before a bounded device spin-wait (the sort's decoupled
 * look-back) gives up and the frame reports D4DGS_ERR_TIMEOUT (0 selects
 * 2^20; a small value makes the waits give up early, for failure-detection
 * tests); colour_cache: 0 evaluates each Gaussian's SH colour in the
 * direction of its time-shifted mean (the definition), 1 in the direction of
 * its static mean -- an approximation that makes the colour depend on the
 * camera only, so the views of a time group (one scene and camera, several
 * times; Algorithm 1's camera-change caching) share one evaluation of it
 * (disentangled scenes; the slicing-first form ignores it); binning: how
 * the depth-ordered pairs reach their tiles' lists -- 1 column buckets then
 * a stable radix sort by tile row (any grid), 2 straight into each tile's
 * list from per-(256-Gaussian partition, tile) counts (grids of at most
 * 2048 tiles; a larger grid makes the config invalid), 3 each pair's depth
 * rank into its tile's range in no order, then per tile a bitmap over the
 * depth order read back in order (any grid), 0 the library's choice
 * (currently 1).  The lists are the same, entry for entry, every way. */
typedef struct {
    int32_t tile;
    int32_t batch;
    float bg[3];
    int32_t trim;
    float near;
    uint32_t spin_limit;
    int32_t colour_cache;
    int32_t binning;
} d4dgs_config;

/* Counters read back after a frame (host struct). */
typedef struct {
    int32_t status;              /* D4DGS_OK or the first device-side error      */
    int64_t n_keys;              /* total (tile, Gaussian) pairs of the frame     */
    int64_t key_capacity;        /* pairs the workspace can hold                  */
    int64_t n_visible;           /* Gaussians that touch at least one tile        */
} d4dgs_stats;

/* Byte offsets of the workspace buffers (test and profiling hook).  All
 * offsets are from the workspace base; buffers are 256-byte aligned. */
typedef struct {
    int64_t records;             /* N x 12 float: (u,v,a,b) (c,o_hat,depth,radius) (r,g,b,log2 o_hat) */
    int64_t depth_keys;          /* N uint32: float bits of camera z, 0xFFFFFFFF if culled   */
    int64_t tiles_touched;       /* N uint32: tiles kept of the trimmed rectangle, 0 if culled */
    int64_t rect;                /* N x 4 uint16: x0, x1, y0, y1 (inclusive tile indices)    */
    int64_t depth_order;         /* N uint32: Gaussian ids sorted by (depth key, id)         */
    int64_t tile_keys;           /* key_capacity uint32, sorted by tile: (tile row << id_bits) | id
                                    when packed, else the tile row; a tile's pairs are
                                    [ranges[t].x, ranges[t].y)                                */
    int64_t tile_vals;           /* key_capacity uint32 Gaussian ids when not packed, else -1  */
    int64_t ranges;              /* tiles x 2 uint32: [start, end) of each tile's list        */
    int64_t final_T;             /* H x W float: transmittance after the last blend           */
    int64_t n_contrib;           /* H x W uint32: list entries walked before the pixel stopped */
    int64_t control;             /* device status word and counters                           */
    int64_t key_capacity;
    int32_t tiles_x, tiles_y;
    int32_t depth_passes, tile_passes;   /* tile_passes 0: binning 3 (no pass sorts the pairs) */
    int32_t id_bits;             /* ceil(log2 N) */
    int32_t packed;              /* 1: pairs packed in one uint32 (row bits + id_bits <= 32) */
    int32_t col_bits;            /* ceil(log2 tiles_x) (the pair keys carry the row only)     */
    int64_t trims;               /* N uint64: per-column trims of the rectangle (config trim = 1,
                                    else 0); byte j (column x0 + j, j < 8) = rows cut at the
                                    top | rows cut at the bottom << 4 (0..15 each); the
                                    Gaussian's tiles are the rectangle minus these cuts,
                                    tiles_touched of them                                    */
    int64_t tile_order;          /* tiles uint32: the order in which the blend and the
                                    backward's tile replay take the tiles, most work first
                                    (quarter-octave classes of the list entries walked over
                                    each tile's pixels: for the blend those of the frame last
                                    blended in this workspace, for the backward those of its
                                    own frame).  Any order gives the same image.               */
} d4dgs_layout;

/* Bytes of workspace for N Gaussians, this camera and config, and room for
 * key_capacity (tile, Gaussian) pairs.  Returns 0 on invalid arguments. */
size_t d4dgs_workspace_bytes(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, int64_t key_capacity);

/* Layout of a workspace of ws_bytes for (n, cam, cfg); the key capacity is
 * whatever fits.  Returns D4DGS_ERR_WORKSPACE_TOO_SMALL if not even zero
 * keys fit. */
int d4dgs_workspace_layout(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, size_t ws_bytes,
                           d4dgs_layout *out);

/* Stage 1 -- per-Gaussian preprocess at time t (Algorithm 1: the camera
 * transform of the mean and velocity, the deferred temporal slice
 * P_view,t = P_view + tau V_view with tau = t - mu_t (Eq. 7, 15), the
 * temporal opacity factor exp(-tau^2 / (2 s_t^2)) (Eq. 6), projection of
 * the mean (Eq. 12) and of the covariance Sigma' = J W Sigma3D W^T J^T + 0.3 I
 * (Eq. 14, 16), the conic, the tile rectangle of radius
 * ceil(3.33 sqrt(lambda_max)), the depth key and the SH colour in the
 * direction of the time-shifted mean).  Writes the 2D records, depth keys,
 * tile counts and rectangles into the workspace; resets the workspace's
 * status word and counters for a new frame. */
int d4dgs_preprocess(const d4dgs_scene *scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg,
                     void *ws, size_t ws_bytes, d4dgs_stream_t stream);

/* Stage 2 -- binning of the preprocessed frame (the 3DGS fast rasteriser's
 * tile/depth ordering, Sec. III-B-2): onesweep radix sort of the depth keys,
 * then the duplication of one (tile, Gaussian) pair per covered tile in
 * depth order, either (config binning 2) straight into each tile's list at
 * offsets from per-(256-Gaussian partition, tile) counts and their column
 * scan, or (binning 1) into per-tile-column buckets followed by a onesweep
 * radix sort of the pairs by tile row (stable, so each tile's list stays in
 * (depth, id) order), or (binning 3) as depth ranks into each tile's range
 * in no order, each list then read back in depth order from a bitmap of its
 * ranks; per-tile [start, end) ranges.  Widths up to 2048 tiles. */
int d4dgs_sort(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, void *ws, size_t ws_bytes,
               d4dgs_stream_t stream);

/* Stage 3 -- per-pixel front-to-back alpha compositing over the tile's
 * list (Eq. 4 with alpha = min(0.99, o_hat exp(p)), p = -1/2 d^T conic d,
 * skip alpha < 1/255, stop before blending once T (1 - alpha) < 1e-4).
 * out_rgb: H x W x 3 float32 device, caller-owned, overwritten with
 * C + T bg; also stores T and, per pixel, the number of list entries walked
 * before the one at which it stopped (the whole list if it never stopped)
 * in the workspace for the backward pass. */
int d4dgs_blend(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, void *ws, size_t ws_bytes,
                float *out_rgb, d4dgs_stream_t stream);

/* Profiling variant of d4dgs_blend: the same compositing, plus three totals
 * over the frame, accumulated into `counts` (3 x uint64 DEVICE memory,
 * caller-owned, zeroed by the call): counts[0] (pixel, Gaussian) pairs the
 * kernel evaluated, counts[1] pairs blended, counts[2] the work of the plain
 * tile algorithm (Sec. III-B-2), the sum over tiles of the tile's in-image
 * pixels times the list entries walked until its last pixel stopped.  Slower
 * than d4dgs_blend; used to turn a blend time into an FP32 throughput. */
int d4dgs_blend_profile(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, void *ws, size_t ws_bytes,
                        float *out_rgb, uint64_t *counts, d4dgs_stream_t stream);

/* Stages 1-3 in order: one frame of `scene` seen by `cam` at time t
 * (Algorithm 1 for one timestamp). */
int d4dgs_render(const d4dgs_scene *scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg,
                 void *ws, size_t ws_bytes, float *out_rgb, d4dgs_stream_t stream);

/* Backward of d4dgs_render (Sec. III-B-2, "differentiable projection-first
 * splatting"): given dL/dC (H x W x 3 float32 device) and the workspace of
 * the forward call with the same scene, camera, t and config, writes
 * dL/d(raw parameters) into `grad` (overwritten; for SH degree 1 and 3 the
 * coefficient gradients, like the coefficients, must be 16-byte aligned:
 * D4DGS_ERR_INVALID_ARG otherwise).  The per-tile lists are
 * replayed back to front from the stored final T; no per-pixel lists are
 * kept. */
int d4dgs_render_backward(const d4dgs_scene *scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg,
                          void *ws, size_t ws_bytes, const float *dl_drgb, d4dgs_scene_grad *grad,
                          d4dgs_stream_t stream);

/* d4dgs_render_backward for a step over several views: the same gradients,
 * ADDED to the arrays of `grad` instead of overwriting them (the caller zeroes
 * them once per step).  Same arguments, workspace rules and return codes. */
int d4dgs_render_backward_accumulate(const d4dgs_scene *scene, const d4dgs_camera *cam, float t,
                                     const d4dgs_config *cfg, void *ws, size_t ws_bytes, const float *dl_drgb,
                                     d4dgs_scene_grad *grad, d4dgs_stream_t stream);

/* The L1 photometric term of a training step (the 3DGS image loss the paper's
 * training keeps, Sec. III-C) and its gradient, in one pass over `count`
 * float32 values (device, caller-owned; img and target read, dl_dimg
 * overwritten, all 4-byte aligned, 16 bytes for the vector path):
 *   *loss += scale * sum_k |img_k - target_k|     (loss: one device float,
 *                                                  accumulated, not zeroed)
 *   dl_dimg_k = scale * sign(img_k - target_k)    (sign(0) = 0)
 * scale = 1 / (values per image x views) gives the mean over a step's views.
 * Stream-ordered; D4DGS_ERR_INVALID_ARG on a negative count, a non-finite
 * scale, a null or misaligned pointer. */
int d4dgs_l1_loss(const float *img, const float *target, int64_t count, float scale, float *dl_dimg, float *loss,
                  d4dgs_stream_t stream);

/* Launch timer (profiling; the paper has no counterpart): while installed on
 * the calling host thread, every kernel launch that thread makes through this
 * library (and each memset of the backward) is followed by a record of the
 * next of `events` (cudaEvent_t handles, created by the caller with timing
 * enabled) on the launch's stream; once they are used up, further launches
 * record nothing.  With an event the caller records just before the first
 * call, elapsed times between consecutive events are the device times of the
 * individual launches, in order.  d4dgs_launch_timer_stop() uninstalls it and
 * returns how many events were recorded.  INVALID_ARG for a null array or
 * n_events < 1. */
int d4dgs_launch_timer(void *const *events, int32_t n_events);
int32_t d4dgs_launch_timer_stop(void);

/* ---- optical-flow channel and flow-gradient consistency loss (Sec. III-C) -
 * A Gaussian's screen flow is its ray-space velocity (Eq. 13) in pixels per
 * unit time, (fx V_x / Z, fy V_y / Z) with V the camera-frame velocity and Z
 * the depth of the time-shifted mean; the flow image composites it with the
 * colour weights (background 0).
 * out_flow: H x W x 2 float32 device, caller-owned, overwritten.  Otherwise
 * as d4dgs_render, whose outputs (image, T, walked entries) it also writes. */
int d4dgs_render_flow(const d4dgs_scene *scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg,
                      void *ws, size_t ws_bytes, float *out_rgb, float *out_flow, d4dgs_stream_t stream);
/* Backward of d4dgs_render_flow: as d4dgs_render_backward, with dL/dF
 * (H x W x 2 float32 device) of the flow image as well; the workspace must
 * hold the d4dgs_render_flow frame with the same arguments. */
int d4dgs_render_backward_flow(const d4dgs_scene *scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg,
                               void *ws, size_t ws_bytes, const float *dl_drgb, const float *dl_dflow,
                               d4dgs_scene_grad *grad, d4dgs_stream_t stream);
/* Scratch bytes of d4dgs_flow_loss for a W x H image (0 on bad sizes). */
size_t d4dgs_flow_loss_scratch_bytes(int32_t width, int32_t height);
/* The flow-gradient consistency loss (Eq. 17-18) of an image I (H x W x 3)
 * and a flow F (H x W x 2), all float32 device:
 *   M = sqrt(u^2 + v^2 + eps),
 *   L = lambda / (W H) * sum |grad M| * (1 - |grad I| / max |grad I|),
 * with 3x3 Sobel gradients on replicated borders, |grad M| divided by the
 * kernel weight 8, |grad I| over the three channels and its guide held fixed
 * (1 where the image is flat).  Writes L to *loss (one float, device) and,
 * when dl_dflow is not null, dL/dF (H x W x 2) there.  scratch: device,
 * 256-byte aligned, >= d4dgs_flow_loss_scratch_bytes. */
int d4dgs_flow_loss(const float *rgb, const float *flow, int32_t width, int32_t height, float lambda, float eps,
                    void *scratch, size_t scratch_bytes, float *loss, float *dl_dflow, d4dgs_stream_t stream);

/* ---- temporal and spatial splitting (Sec. III-C) ----------------------------
 * Training-side densification: time-domain splitting guided by the gradient
 * of t, spatial splitting by the gradients of xyz, the two scales split
 * independently.  d4dgs_split_accumulate adds |dL/d mean| (3-vector norm),
 * |dL/d t_mean| and 1 to stats (N x 3 float32 device, caller-owned, zeroed by
 * the caller before the first step) for every Gaussian with a nonzero mean or
 * t_mean gradient.  d4dgs_split decides, from the float32 averages
 * g = sum / max(count, 1): in space when g_xyz > tau_xyz and the largest
 * log-scale > log_min_xyz; in time when g_t > tau_t and log s_t > log_min_t.
 * A split Gaussian becomes two: child 1 keeps its index, child 2 is appended
 * after the first N in index order; means mu +- R(q) diag(s) n_xyz and spatial
 * log-scales - log(factor) for a spatial split, t_mean +- s_t n_t and
 * log s_t - log(factor) for a temporal one, the other fields copied.
 * normals: N x 4 standard normal samples (three spatial, one temporal),
 * device.  out: arrays of capacity >= 2N Gaussians (device, caller-owned);
 * *out_n (device int32) receives the new count.  scratch: device,
 * >= d4dgs_split_scratch_bytes(N). */
typedef struct {
    float tau_xyz, tau_t;            /* thresholds on the average gradient norms */
    float log_min_xyz, log_min_t;    /* thresholds on the log-scales              */
    float factor;                    /* scale divisor of a split (> 1, e.g. 1.6)  */
} d4dgs_split_params;
int d4dgs_split_accumulate(const d4dgs_scene_grad *grad, int32_t n, float *stats, d4dgs_stream_t stream);
size_t d4dgs_split_scratch_bytes(int32_t n);
int d4dgs_split(const d4dgs_scene *scene, const float *stats, const float *normals, const d4dgs_split_params *params,
                const d4dgs_scene_grad *out, int32_t capacity, int32_t *out_n, void *scratch, size_t scratch_bytes,
                d4dgs_stream_t stream);

/* ---- slicing-first baseline (comparison, Eq. 5-7) --------------------------
 * The 4D Gaussian form the paper compares against: a 4D mean, 4D scales and
 * a 4D rotation, sliced at every frame into a 3D Gaussian before projection.
 * The rotation is the pair of unit quaternions (q_l, q_r) acting as
 * p -> q_l p q_r on p = t + x i + y j + z k (one reading of the 4D rotations
 * the paper cites; q_r = conj(q_l) is the 3D rotation of q_l).  Per Gaussian
 * and frame: Sigma4D = R4 S4^2 R4^T = [[U, V], [V^T, W]] (Eq. 5),
 * Sigma3D = U - V V^T / W, mean mu + (t - mu_t) V / W, opacity times
 * exp(-(t - mu_t)^2 / (2 W)) (Eq. 6-7); then the same projection, binning and
 * blending as the disentangled path (same workspace, d4dgs_sort and
 * d4dgs_blend apply).  All arrays device, caller-owned, read-only. */
typedef struct {
    const float *means4;         /* N x 4: x, y, z, t                                */
    const float *log_scales4;    /* N x 4                                            */
    const float *quat_l;         /* N x 4 (w, x, y, z), any norm, 16-byte aligned    */
    const float *quat_r;         /* N x 4 (w, x, y, z), any norm, 16-byte aligned    */
    const float *opacity_logit;  /* N                                                */
    const float *sh;             /* N x (deg+1)^2 x 3                                */
    int32_t n, sh_degree;
} d4dgs_scene4d;

/* Stage 1 for a slicing-first scene (then d4dgs_sort and d4dgs_blend). */
int d4dgs_preprocess_slicing(const d4dgs_scene4d *scene, const d4dgs_camera *cam, float t,
                             const d4dgs_config *cfg, void *ws, size_t ws_bytes, d4dgs_stream_t stream);
/* Stages 1-3 for a slicing-first scene. */
int d4dgs_render_slicing(const d4dgs_scene4d *scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg,
                         void *ws, size_t ws_bytes, float *out_rgb, d4dgs_stream_t stream);

/* ---- batched multi-view rendering (serving) -------------------------------
 * V <= 32 frames rendered by ONE launch of each kernel (preprocess, sort
 * passes, blend), each frame with its own scene, camera, time, resolution,
 * workspace and output -- the multi-frame parallel rendering the paper notes
 * for fixed viewpoints (Sec. IV-C), generalised to mixed requests.  All views
 * of a batch share the config (tile, batch, bg) and must agree on the layout
 * class that d4dgs_workspace_layout reports (packed, tile_passes).
 * Kernels are persistent with device-side work distribution, so the launch
 * sequence of d4dgs_render_batch does not depend on the batch's contents and
 * can be captured once as a CUDA graph; with args_dev the first kernel reads
 * the descriptors from device memory, which the caller refreshes (e.g. by a
 * captured host-to-device copy) before each replay.
 * Time groups: consecutive views (up to 4) with the same scene arrays and the
 * same camera -- the paper's fixed-viewpoint multi-timestamp case (Alg. 1
 * caches the camera-dependent terms; Sec. IV-C renders such frames in
 * parallel) -- are preprocessed together: each Gaussian's parameters are read
 * from DRAM once for all times of the group.  Every view's outputs are the
 * same, bit for bit, as when it is rendered alone. */
typedef struct {
    const d4dgs_scene *scene;    /* host struct of device arrays                     */
    d4dgs_camera cam;
    float t;
    void *ws;                    /* this view's workspace (as for d4dgs_render)      */
    size_t ws_bytes;
    float *out_rgb;              /* H x W x 3 float32 device output                  */
} d4dgs_view;

/* Size of one encoded batch (host or device copy). */
size_t d4dgs_batch_args_bytes(void);
/* Device scratch of a batched launch (work counters + descriptor table). */
size_t d4dgs_batch_area_bytes(void);
/* Host only: validates the views and encodes them into args_host (at least
 * d4dgs_batch_args_bytes()).  D4DGS_ERR_INVALID_ARG if they cannot share a
 * launch. */
int d4dgs_batch_encode(int32_t nviews, const d4dgs_view *views, const d4dgs_config *cfg, void *args_host,
                       size_t args_bytes);
/* Renders an encoded batch on `stream`.  args_host: the encoded batch (read
 * on the host for the launch configuration); args_dev: NULL (descriptors
 * travel as kernel parameters) or a device copy of the same bytes, 16-byte
 * aligned, read by the first kernel.  batch_area: >= d4dgs_batch_area_bytes()
 * of device memory, 256-byte aligned, caller-owned.  Per-view status via
 * d4dgs_read_stats on each view's workspace. */
int d4dgs_render_batch(const void *args_host, const void *args_dev, void *batch_area, size_t batch_area_bytes,
                       d4dgs_stream_t stream);
/* The stages of d4dgs_render_batch one at a time (profiling hook): stages is
 * a bit set, 1 = clear + preprocess, 2 = binning, 4 = blend; a batch's stages
 * must be launched in that order on one stream and batch_area. */
int d4dgs_render_batch_stages(const void *args_host, const void *args_dev, void *batch_area,
                              size_t batch_area_bytes, int32_t stages, d4dgs_stream_t stream);

/* Synchronises `stream`, then copies the status word and counters of the
 * last frame rendered in `ws` into *out (host).  Returns out->status. */
int d4dgs_read_stats(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg, const void *ws,
                     size_t ws_bytes, d4dgs_stats *out, d4dgs_stream_t stream);

/* d4dgs_render with HOST inputs and output: copies the scene (host arrays,
 * same layout as d4dgs_scene, ideally pinned) into the device staging area
 * `dev_scene_buf` (at least d4dgs_scene_bytes(n, deg) bytes, caller-owned),
 * renders, and copies the image back into host `out_rgb_host`; all on
 * `stream`, and the call returns after the stream has finished. */
size_t d4dgs_scene_bytes(int32_t n, int32_t sh_degree);
int d4dgs_render_host(const d4dgs_scene *host_scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg,
                      void *dev_scene_buf, size_t dev_scene_bytes, void *ws, size_t ws_bytes,
                      void *dev_rgb, float *out_rgb_host, d4dgs_stream_t stream);
/* d4dgs_render_host without the final wait: the copies and the frame are
 * queued on `stream` and the image is in out_rgb_host once the stream has
 * reached this point (cudaStreamSynchronize, or an event recorded after the
 * call).  Until then the host scene arrays, out_rgb_host, dev_scene_buf, ws
 * and dev_rgb belong to the call.  Callers that give consecutive frames
 * their own slot (staging buffer, workspace, device image, stream) overlap
 * one frame's copies with another's kernels.  Same arguments, checks and
 * return codes as d4dgs_render_host (CUDA errors of the queued work surface
 * at the wait). */
int d4dgs_render_host_async(const d4dgs_scene *host_scene, const d4dgs_camera *cam, float t,
                            const d4dgs_config *cfg, void *dev_scene_buf, size_t dev_scene_bytes, void *ws,
                            size_t ws_bytes, void *dev_rgb, float *out_rgb_host, d4dgs_stream_t stream);

/* d4dgs_render for callers that cannot allocate device memory when they
 * render (the paper has no counterpart; this is a library convenience).  The
 * scratch is a fixed 64 MiB array inside the library's device module: each
 * GPU that loads the library holds it until the process exits, and the call
 * itself allocates nothing.  The caller passes the scene and the output image
 * (H x W x 3 float32 device) as for d4dgs_render.
 *   - Every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress), so a device reset or a new primary context is
 *     followed safely; the first call on a device also loads the library's
 *     module there, so make that first call before any stream capture.
 *   - Returns D4DGS_ERR_WORKSPACE_TOO_SMALL when N and the image size leave
 *     no room for keys in 64 MiB; a frame with more (tile, Gaussian) pairs
 *     than fit is reported as D4DGS_ERR_CAPACITY only through `stats`.
 *   - stats: optional host struct; when non-NULL the call synchronises
 *     `stream` and fills it (returning stats->status), otherwise the call is
 *     asynchronous -- and then a frame whose pairs overflowed the array's
 *     key capacity comes back incomplete with return code D4DGS_OK: callers
 *     that cannot re-render elsewhere should pass stats.
 *   - All calls share the array; calls whose work overlaps on the GPU race. */
int d4dgs_render_static(const d4dgs_scene *scene, const d4dgs_camera *cam, float t, const d4dgs_config *cfg,
                        float *out_rgb, d4dgs_stats *stats, d4dgs_stream_t stream);

/* Number of kernel launches one d4dgs_render issues for (n, cam, cfg) (the
 * launch count of a frame, not counting memsets). */
int d4dgs_launches_per_frame(int32_t n, const d4dgs_camera *cam, const d4dgs_config *cfg);

/* Human-readable text of a status code (static storage). */
const char *d4dgs_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* D4DGS_H */
