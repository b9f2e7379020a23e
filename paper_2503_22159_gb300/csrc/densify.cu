// densify.cu -- temporal and spatial splitting of the disentangled Gaussians
// (Sec. III-C: time-domain splitting guided by the gradient of t, spatial
// splitting by the gradients of xyz, the two scales split independently).
//
// Accumulation: per Gaussian, |dL/d mean| (3-vector norm) and |dL/d t_mean|
// are summed over the training steps that gave it a nonzero gradient.
// Split: with the averages g_xyz, g_t (float32, sum / max(count, 1)), a
// Gaussian splits in space when g_xyz > tau_xyz and its largest log-scale
// exceeds log_min_xyz, in time when g_t > tau_t and log s_t > log_min_t.  A
// split Gaussian becomes two: child 1 stays at its index, child 2 is appended
// after the first N in index order; means mu +- R(q) diag(s) n_xyz and
// spatial log-scales - log(factor) when splitting in space, t_mean +- s_t n_t
// and log s_t - log(factor) when splitting in time, the rest copied; n are the
// caller's standard normal samples (N x 4).  Three launches: per-block decide
// and count, scan of the block totals (one CTA; writes the new N to the
// device), write.
#include "d4dgs_internal.cuh"

namespace d4dgs {

namespace {

constexpr int kSplitThreads = 256;

struct SplitArgs {
    const float *means, *t_mean, *velocity, *log_scales, *log_t_scale, *quats, *opacity_logit, *sh;
    float *o_means, *o_t_mean, *o_velocity, *o_log_scales, *o_log_t_scale, *o_quats, *o_opacity_logit, *o_sh;
    const float *stats, *normals;
    int32_t n, sh_degree;
    float tau_xyz, tau_t, log_min_xyz, log_min_t, log_factor;
};

__device__ __forceinline__ void decide(const SplitArgs &a, int i, bool &ss, bool &tt) {
    const float cnt = fmaxf(a.stats[3 * i + 2], 1.0f);
    const float gx = __fdiv_rn(a.stats[3 * i], cnt), gt = __fdiv_rn(a.stats[3 * i + 1], cnt);
    const float mx = fmaxf(fmaxf(a.log_scales[3 * i], a.log_scales[3 * i + 1]), a.log_scales[3 * i + 2]);
    ss = gx > a.tau_xyz && mx > a.log_min_xyz;
    tt = gt > a.tau_t && a.log_t_scale[i] > a.log_min_t;
}

__global__ void __launch_bounds__(256) split_stats_kernel(const float *__restrict__ gm, const float *__restrict__ gt,
                                                           int n, float *__restrict__ stats) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = gm[3 * i], y = gm[3 * i + 1], z = gm[3 * i + 2], t = gt[i];
    const float nm = sqrtf(x * x + y * y + z * z);
    if (nm == 0.0f && t == 0.0f) return;
    stats[3 * i] += nm;
    stats[3 * i + 1] += fabsf(t);
    stats[3 * i + 2] += 1.0f;
}

__global__ void __launch_bounds__(kSplitThreads) split_count_kernel(const SplitArgs a, uint32_t *block_tot) {
    __shared__ uint32_t s[kSplitThreads / 32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool ss = false, tt = false;
    if (i < a.n) decide(a, i, ss, tt);
    const uint32_t c = __popc(__ballot_sync(0xFFFFFFFFu, ss || tt));
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kSplitThreads / 32; w++) t += s[w];
        block_tot[blockIdx.x] = t;
    }
}

// One CTA: exclusive scan of the block totals in place; writes n + total to *out_n.
__global__ void __launch_bounds__(1024) split_scan_kernel(uint32_t *block_tot, int nblocks, int n, int32_t *out_n) {
    __shared__ uint32_t s_carry;
    __shared__ uint32_t s_w[32];
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < nblocks; base += 1024) {
        const int j = base + (int)threadIdx.x;
        const uint32_t v = j < nblocks ? block_tot[j] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        uint32_t before = 0, all = 0;
        for (int w = 0; w < 32; w++) {
            if (w < warp) before += s_w[w];
            all += s_w[w];
        }
        const uint32_t carry = s_carry;
        if (j < nblocks) block_tot[j] = carry + before + x - v;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + all;
        __syncthreads();
    }
    if (threadIdx.x == 0) *out_n = n + (int32_t)s_carry;
}

__device__ __forceinline__ void quat_rot(const float *q4, float R[9]) {
    const float qn = sqrtf(q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3]);
    const float w = q4[0] / qn, x = q4[1] / qn, y = q4[2] / qn, z = q4[3] / qn;
    R[0] = 1.0f - 2.0f * (y * y + z * z); R[1] = 2.0f * (x * y - w * z); R[2] = 2.0f * (x * z + w * y);
    R[3] = 2.0f * (x * y + w * z); R[4] = 1.0f - 2.0f * (x * x + z * z); R[5] = 2.0f * (y * z - w * x);
    R[6] = 2.0f * (x * z - w * y); R[7] = 2.0f * (y * z + w * x); R[8] = 1.0f - 2.0f * (x * x + y * y);
}

__global__ void __launch_bounds__(kSplitThreads) split_write_kernel(const SplitArgs a, const uint32_t *block_off) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool ss = false, tt = false;
    if (i < a.n) decide(a, i, ss, tt);
    const bool two = ss || tt;
    const uint32_t mask = __ballot_sync(0xFFFFFFFFu, two);
    __shared__ uint32_t s[kSplitThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s[warp] = __popc(mask);
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; w++) before += s[w];
    if (i >= a.n) return;
    const int j2 = a.n + (int)(block_off[blockIdx.x] + before + __popc(mask & lanemask_lt()));
    const int K = (a.sh_degree + 1) * (a.sh_degree + 1);
    float d[3] = {0.0f, 0.0f, 0.0f}, dt = 0.0f;
    if (ss) {
        float R[9];
        quat_rot(a.quats + 4 * i, R);
        float sn[3];
        for (int k = 0; k < 3; k++) sn[k] = expf(a.log_scales[3 * i + k]) * a.normals[4 * i + k];
        for (int r = 0; r < 3; r++) d[r] = R[3 * r] * sn[0] + R[3 * r + 1] * sn[1] + R[3 * r + 2] * sn[2];
    }
    if (tt) dt = expf(a.log_t_scale[i]) * a.normals[4 * i + 3];
    const float dls = ss ? a.log_factor : 0.0f, dlt = tt ? a.log_factor : 0.0f;
    auto put = [&](int o, float sign) {
        for (int k = 0; k < 3; k++) {
            a.o_means[3 * o + k] = a.means[3 * i + k] + sign * d[k];
            a.o_velocity[3 * o + k] = a.velocity[3 * i + k];
            a.o_log_scales[3 * o + k] = a.log_scales[3 * i + k] - dls;
        }
        a.o_t_mean[o] = a.t_mean[i] + sign * dt;
        a.o_log_t_scale[o] = a.log_t_scale[i] - dlt;
        for (int k = 0; k < 4; k++) a.o_quats[4 * o + k] = a.quats[4 * i + k];
        a.o_opacity_logit[o] = a.opacity_logit[i];
        for (int k = 0; k < 3 * K; k++) a.o_sh[(size_t)3 * K * o + k] = a.sh[(size_t)3 * K * i + k];
    };
    put(i, 1.0f);
    if (two) put(j2, -1.0f);
}

}  // namespace

}  // namespace d4dgs

using namespace d4dgs;

extern "C" {

int d4dgs_split_accumulate(const d4dgs_scene_grad *grad, int32_t n, float *stats, d4dgs_stream_t stream) {
    if (!grad || n < 0 || (n > 0 && (!grad->means || !grad->t_mean || !stats))) return D4DGS_ERR_INVALID_ARG;
    if (n == 0) return D4DGS_OK;
    split_stats_kernel<<<(n + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(grad->means, grad->t_mean,
                                                                                            n, stats);
    return cudaGetLastError() == cudaSuccess ? D4DGS_OK : D4DGS_ERR_CUDA;
}

size_t d4dgs_split_scratch_bytes(int32_t n) { return n < 0 ? 0 : ((size_t)(n + kSplitThreads - 1) / kSplitThreads + 1) * 4; }

int d4dgs_split(const d4dgs_scene *scene, const float *stats, const float *normals, const d4dgs_split_params *p,
                const d4dgs_scene_grad *out, int32_t capacity, int32_t *out_n, void *scratch, size_t scratch_bytes,
                d4dgs_stream_t stream) {
    if (!scene || !p || !out || !out_n || !scratch || scene->n < 0 || scene->sh_degree < 0 || scene->sh_degree > 3 ||
        capacity < 2 * scene->n || scratch_bytes < d4dgs_split_scratch_bytes(scene->n) || !(p->factor > 1.0f))
        return D4DGS_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int n = scene->n;
    if (n == 0) return cudaMemsetAsync(out_n, 0, 4, st) == cudaSuccess ? D4DGS_OK : D4DGS_ERR_CUDA;
    if (!stats || !normals) return D4DGS_ERR_INVALID_ARG;
    SplitArgs a{scene->means, scene->t_mean, scene->velocity, scene->log_scales, scene->log_t_scale, scene->quats,
                scene->opacity_logit, scene->sh, out->means, out->t_mean, out->velocity, out->log_scales,
                out->log_t_scale, out->quats, out->opacity_logit, out->sh, stats, normals, n, scene->sh_degree,
                p->tau_xyz, p->tau_t, p->log_min_xyz, p->log_min_t, logf(p->factor)};
    const int nb = (n + kSplitThreads - 1) / kSplitThreads;
    uint32_t *blocks = static_cast<uint32_t *>(scratch);
    split_count_kernel<<<nb, kSplitThreads, 0, st>>>(a, blocks);
    split_scan_kernel<<<1, 1024, 0, st>>>(blocks, nb, n, out_n);
    split_write_kernel<<<nb, kSplitThreads, 0, st>>>(a, blocks);
    return cudaGetLastError() == cudaSuccess ? D4DGS_OK : D4DGS_ERR_CUDA;
}

}  // extern "C"
