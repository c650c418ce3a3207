// backward.cu -- placeholder launchers until the backward kernels land.
#include "geer_internal.cuh"

namespace geer {

cudaError_t launch_render_bwd(const geer_workspace *, const float *, cudaStream_t) { return cudaErrorNotSupported; }

cudaError_t launch_preprocess_bwd(const geer_workspace *, const geer_gaussians *, float *, float *, float *, float *,
                                  float *, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace geer
