// noalloc.cu -- d4dgs_render_static: the frame render with its scratch in a
// fixed, file-scope device array instead of a caller-allocated workspace.
//
// Some callers cannot allocate device memory when they want a frame: a host
// application whose device memory is owned by another allocator and that
// forbids cudaMalloc inside its per-frame callback, or a real-time loop where
// cudaMalloc/cudaFree would block on the device and stall other streams.  This
// entry point lets them render without ever allocating: the scratch below is
// part of the loaded module, so every GPU that loads this library holds
// kStaticScratchBytes of it until the process exits.
//
// The caller still owns the scene arrays and the output image.  Every call
// shares the one array: a call overwrites what the previous call left there
// (the render clears the parts that must start at zero itself), and two calls
// whose work overlaps on the GPU (different streams, no ordering between
// them) race on it.
#include <cuda_runtime.h>

#include "d4dgs_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;   // 64 MiB, stated in include/d4dgs.h

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch on the current device.  In host code the
// name g_static_scratch is only a host-side stand-in and must never be handed
// to a kernel.  The address is looked up on every call (once the module is
// loaded this is a table lookup, far cheaper than a frame) rather than cached:
// after cudaDeviceReset, or when the primary context is torn down and made
// again, the module is loaded anew and the array may move, and a cache shared
// by several host threads would need synchronising.  The first call on a
// device loads the module, which is why that call must come before any stream
// capture.
int scratch_address(void **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return D4DGS_ERR_CUDA;
    *out = p;
    return D4DGS_OK;
}

}  // namespace

extern "C" int d4dgs_render_static(const d4dgs_scene *scene, const d4dgs_camera *cam, float t,
                                   const d4dgs_config *cfg, float *out_rgb, d4dgs_stats *stats,
                                   d4dgs_stream_t stream) {
    if (!scene || scene->n < 0) return D4DGS_ERR_INVALID_ARG;
    d4dgs::Layout L;
    if (!d4dgs::make_layout(scene->n, cam, cfg, 0, &L)) return D4DGS_ERR_INVALID_ARG;
    // N and the image must fit with room for at least one key; otherwise refuse
    if (!d4dgs::layout_for_bytes(scene->n, cam, cfg, kStaticScratchBytes, &L) || L.cap < 1)
        return D4DGS_ERR_WORKSPACE_TOO_SMALL;
    void *ws = nullptr;
    int rc = scratch_address(&ws);
    if (rc) return rc;
    rc = d4dgs_render(scene, cam, t, cfg, ws, kStaticScratchBytes, out_rgb, stream);
    if (rc || !stats) return rc;
    return d4dgs_read_stats(scene->n, cam, cfg, ws, kStaticScratchBytes, stats, stream);
}
