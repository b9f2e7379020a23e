// loss.cu -- K10: the L1 photometric term of a training step and its gradient
// (the 3DGS L1 image loss the paper's training keeps, Sec. III-C; here
// against a caller-given target), one pass over the image:
//
//   loss += scale * sum_k |img_k - target_k|,   dl_dimg_k = scale * sign(img_k - target_k)
//
// (sign(0) = 0).  HBM-bound: 8 B read and 4 B written per value.  A
// grid-stride loop over float4 quadruples (a scalar tail when the count is not a
// multiple of 4 or a pointer is not 16-byte aligned), a warp-shuffle and
// shared-memory block reduction, one atomicAdd per block into the device scalar.
#include <math.h>

#include "d4dgs_internal.cuh"

namespace d4dgs {
namespace {

constexpr int kLossThreads = 256;

__device__ __forceinline__ float l1_term(float a, float b, float scale, float *g) {
    const float d = a - b;
    *g = d > 0.0f ? scale : (d < 0.0f ? -scale : 0.0f);
    return fabsf(d);
}

__global__ void __launch_bounds__(kLossThreads) l1_loss_kernel(const float *__restrict__ img,
                                                               const float *__restrict__ target, int64_t count,
                                                               float scale, float *__restrict__ grad,
                                                               float *__restrict__ loss, bool vec) {
    float acc = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t done = 0;
    if (vec) {
        const int64_t n4 = count / 4;
        const float4 *a4 = reinterpret_cast<const float4 *>(img), *b4 = reinterpret_cast<const float4 *>(target);
        float4 *g4 = reinterpret_cast<float4 *>(grad);
        for (int64_t i = tid; i < n4; i += stride) {
            const float4 a = __ldcs(a4 + i), b = __ldcs(b4 + i);
            float4 g;
            acc += l1_term(a.x, b.x, scale, &g.x) + l1_term(a.y, b.y, scale, &g.y) + l1_term(a.z, b.z, scale, &g.z) +
                   l1_term(a.w, b.w, scale, &g.w);
            __stcs(g4 + i, g);
        }
        done = n4 * 4;
    }
    for (int64_t i = done + tid; i < count; i += stride) {
        float g;
        acc += l1_term(img[i], target[i], scale, &g);
        grad[i] = g;
    }
    // block reduction
    __shared__ float s_warp[kLossThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < kLossThreads / 32 ? s_warp[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        if (threadIdx.x == 0 && v != 0.0f) atomicAdd(loss, scale * v);
    }
}

}  // namespace
}  // namespace d4dgs

using namespace d4dgs;

extern "C" int d4dgs_l1_loss(const float *img, const float *target, int64_t count, float scale, float *dl_dimg,
                             float *loss, d4dgs_stream_t stream) {
    if (count < 0 || !isfinite(scale)) return D4DGS_ERR_INVALID_ARG;
    if (count == 0) return D4DGS_OK;
    if (!img || !target || !dl_dimg || !loss) return D4DGS_ERR_INVALID_ARG;
    const uintptr_t align = reinterpret_cast<uintptr_t>(img) | reinterpret_cast<uintptr_t>(target) |
                            reinterpret_cast<uintptr_t>(dl_dimg);
    if (align & 3) return D4DGS_ERR_INVALID_ARG;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return D4DGS_ERR_CUDA;
    const bool vec = (align & 15) == 0;
    const int64_t work = vec ? count / 4 : count;
    int64_t blocks = (work + kLossThreads - 1) / kLossThreads;
    const int64_t cap = (int64_t)sms * 8;   // a few waves of 256-thread blocks, then grid-stride
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    l1_loss_kernel<<<(unsigned)blocks, kLossThreads, 0, st>>>(img, target, count, scale, dl_dimg, loss, vec);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) note_launch(st);
    return e == cudaSuccess ? D4DGS_OK : D4DGS_ERR_CUDA;
}
