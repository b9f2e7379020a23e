// backward.cu -- K7/K8: adjoint of the frame render.
#include "d4dgs_internal.cuh"

namespace d4dgs {

cudaError_t launch_backward(const d4dgs_scene &, const CamArgs &, float, const d4dgs_config &, const Layout &, void *,
                            const float *, const d4dgs_scene_grad &, cudaStream_t, int) {
    return cudaErrorNotSupported;
}

}  // namespace d4dgs
