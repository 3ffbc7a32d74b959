// FP32 trial kernel on 64 x 64 tiles split over a 4-CTA thread-block cluster
// (both models): rank r of a cluster takes filter groups r, r + 4, r + 8 of
// its tile.  For batches of mid-size images (a few 64 x 64 tiles per SM)
// whose trial time is set by one CTA's filter groups; instantiated in its
// own unit so that it compiles in parallel with the others.  The kernel
// template is in fe_fp32_kernel.cuh.
#include <cuda_runtime.h>

#include "fe_fp32_kernel.cuh"

namespace fe {

cudaError_t fp32cl64_prepare() {
    cudaError_t e = prepare_tile<64, 0, 4>();
    if (e == cudaSuccess) e = prepare_tile<64, 1, 4>();
    return e;
}

cudaError_t fp32cl64_launch(int mode, const KParams &p, int ngrid, cudaStream_t s, int model) {
    return model == 1 ? launch_tile<64, 1, 4>(mode, p, ngrid, s) : launch_tile<64, 0, 4>(mode, p, ngrid, s);
}

const void *fp32cl64_trial_entry(int model) {
    return model == 1 ? reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_TRIAL, 64, 1, 4>)
                      : reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_TRIAL, 64, 0, 4>);
}

}  // namespace fe
