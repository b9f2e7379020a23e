// flowloss.cu -- the flow-gradient consistency loss (Sec. III-C, Eq. 17-18)
// on a rendered image I (H x W x 3) and flow F (H x W x 2), and its gradient
// with respect to F:
//
//   M = sqrt(u^2 + v^2 + eps)                                  (Eq. 17)
//   L = lambda / N * sum |grad M| * (1 - |grad I| / max |grad I|)   (Eq. 18)
//
// Gradients are 3x3 Sobel responses with replicated borders; |grad M| is
// divided by the kernel weight 8; |grad I| is taken over the three channels
// and normalised by its maximum over the image (where the image is flat the
// guide is 1); the guide is held fixed (no gradient to I).  dL/dM is the
// transposed Sobel of the per-pixel coefficients, scattered with atomics, then
// dL/du = dL/dM u / M and likewise for v.  Four launches, one thread per pixel.
#include "d4dgs_internal.cuh"

namespace d4dgs {

namespace {

__device__ __forceinline__ int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

// Sobel responses at (x, y) of a single-channel image read through `at`.
template <typename F>
__device__ __forceinline__ void sobel(int x, int y, int W, int H, F at, float &gx, float &gy) {
    const int xm = clampi(x - 1, 0, W - 1), xp = clampi(x + 1, 0, W - 1);
    const int ym = clampi(y - 1, 0, H - 1), yp = clampi(y + 1, 0, H - 1);
    const float a = at(xm, ym), b = at(x, ym), c = at(xp, ym);
    const float d = at(xm, y), f = at(xp, y);
    const float g = at(xm, yp), h = at(x, yp), k = at(xp, yp);
    gx = (c + 2.0f * f + k) - (a + 2.0f * d + g);
    gy = (g + 2.0f * h + k) - (a + 2.0f * b + c);
}

__device__ __forceinline__ float block_sum(float v, float *s) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s[warp] = v;
    __syncthreads();
    float t = 0.0f;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s[w];
    return t;
}

// |grad I| per pixel and its maximum (non-negative floats order as their bits).
__global__ void __launch_bounds__(256) flow_edges_kernel(const float *__restrict__ rgb, int W, int H,
                                                          float *__restrict__ gI, unsigned *maxbits) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    float g = 0.0f;
    if (p < W * H) {
        const int x = p % W, y = p / W;
        float g2 = 0.0f;
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            float gx, gy;
            sobel(x, y, W, H, [&](int xx, int yy) { return rgb[3 * ((size_t)yy * W + xx) + ch]; }, gx, gy);
            g2 += gx * gx + gy * gy;
        }
        g = sqrtf(g2);
        gI[p] = g;
    }
    for (int o = 16; o > 0; o >>= 1) g = fmaxf(g, __shfl_xor_sync(0xFFFFFFFFu, g, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxbits, __float_as_uint(g));
}

__global__ void __launch_bounds__(256) flow_magnitude_kernel(const float *__restrict__ flow, int W, int H, float eps,
                                                              float *__restrict__ M, float *__restrict__ dM) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= W * H) return;
    const float u = flow[2 * p], v = flow[2 * p + 1];
    M[p] = sqrtf(u * u + v * v + eps);
    if (dM) dM[p] = 0.0f;
}

__global__ void __launch_bounds__(256) flow_loss_kernel(const float *__restrict__ M, const float *__restrict__ gI,
                                                         const unsigned *maxbits, int W, int H, float scale,
                                                         float *loss, float *dM) {
    __shared__ float s[8];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    float contrib = 0.0f;
    if (p < W * H) {
        const int x = p % W, y = p / W;
        float gx, gy;
        sobel(x, y, W, H, [&](int xx, int yy) { return M[(size_t)yy * W + xx]; }, gx, gy);
        const float nrm = sqrtf(gx * gx + gy * gy) * 0.125f;
        const float mx = __uint_as_float(*maxbits);
        const float wgt = mx > 0.0f ? 1.0f - gI[p] / mx : 1.0f;
        contrib = scale * nrm * wgt;
        if (dM && nrm > 0.0f) {
            // d nrm / d gx = gx / (64 nrm); gx, gy are linear in the 3 x 3 (clamped) neighbours
            const float cx = scale * wgt * gx / (64.0f * nrm), cy = scale * wgt * gy / (64.0f * nrm);
            const int xs[3] = {clampi(x - 1, 0, W - 1), x, clampi(x + 1, 0, W - 1)};
            const int ys[3] = {clampi(y - 1, 0, H - 1), y, clampi(y + 1, 0, H - 1)};
            const float kx[3][3] = {{-1.f, 0.f, 1.f}, {-2.f, 0.f, 2.f}, {-1.f, 0.f, 1.f}};   // [row][col]
            const float ky[3][3] = {{-1.f, -2.f, -1.f}, {0.f, 0.f, 0.f}, {1.f, 2.f, 1.f}};
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    const float w = cx * kx[r][q] + cy * ky[r][q];
                    if (w != 0.0f) atomicAdd(dM + (size_t)ys[r] * W + xs[q], w);
                }
        }
    }
    const float t = block_sum(contrib, s);
    if (threadIdx.x == 0 && t != 0.0f) atomicAdd(loss, t);
}

__global__ void __launch_bounds__(256) flow_grad_kernel(const float *__restrict__ flow, const float *__restrict__ M,
                                                         const float *__restrict__ dM, int W, int H,
                                                         float *__restrict__ dl_dflow) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= W * H) return;
    const float g = dM[p] / M[p];
    dl_dflow[2 * p] = g * flow[2 * p];
    dl_dflow[2 * p + 1] = g * flow[2 * p + 1];
}

constexpr size_t kHeader = 256;

}  // namespace

}  // namespace d4dgs

using namespace d4dgs;

extern "C" {

size_t d4dgs_flow_loss_scratch_bytes(int32_t width, int32_t height) {
    if (width < 1 || height < 1) return 0;
    return kHeader + 3 * (((size_t)width * height * 4 + 255) / 256 * 256);
}

int d4dgs_flow_loss(const float *rgb, const float *flow, int32_t width, int32_t height, float lambda, float eps,
                    void *scratch, size_t scratch_bytes, float *loss, float *dl_dflow, d4dgs_stream_t stream) {
    if (!rgb || !flow || !scratch || !loss || width < 1 || height < 1 || width > 16384 || height > 16384 ||
        !(eps >= 0.0f) || !isfinite(lambda) || scratch_bytes < d4dgs_flow_loss_scratch_bytes(width, height) ||
        (reinterpret_cast<uintptr_t>(scratch) & 255) || (reinterpret_cast<uintptr_t>(loss) & 3))
        return D4DGS_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t plane = ((size_t)width * height * 4 + 255) / 256 * 256;
    char *base = static_cast<char *>(scratch);
    unsigned *maxbits = reinterpret_cast<unsigned *>(base);
    float *gI = reinterpret_cast<float *>(base + kHeader);
    float *M = reinterpret_cast<float *>(base + kHeader + plane);
    float *dM = dl_dflow ? reinterpret_cast<float *>(base + kHeader + 2 * plane) : nullptr;
    const int npx = width * height, blocks = (npx + 255) / 256;
    if (cudaMemsetAsync(maxbits, 0, 4, st) != cudaSuccess || cudaMemsetAsync(loss, 0, 4, st) != cudaSuccess)
        return D4DGS_ERR_CUDA;
    flow_edges_kernel<<<blocks, 256, 0, st>>>(rgb, width, height, gI, maxbits);
    flow_magnitude_kernel<<<blocks, 256, 0, st>>>(flow, width, height, eps, M, dM);
    flow_loss_kernel<<<blocks, 256, 0, st>>>(M, gI, maxbits, width, height, lambda / (float)npx, loss, dM);
    if (dl_dflow) flow_grad_kernel<<<blocks, 256, 0, st>>>(flow, M, dM, width, height, dl_dflow);
    return cudaGetLastError() == cudaSuccess ? D4DGS_OK : D4DGS_ERR_CUDA;
}

}  // extern "C"
