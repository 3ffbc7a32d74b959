// FP32 trial kernel instantiated for the combined model (Eq. newmodel,
// Sec. III-A) in w = log u; the template is in fe_fp32_kernel.cuh.
#include <cuda_runtime.h>

#include "fe_fp32_kernel.cuh"

namespace fe {

cudaError_t fp32c_prepare() {
    cudaError_t e = prepare_tile<64, 1>();
    return e != cudaSuccess ? e : prepare_tile<32, 1>();
}

cudaError_t fp32c_launch(int mode, const KParams &p, int ngrid, cudaStream_t s, int T) {
    if (T == 64) return launch_tile<64, 1>(mode, p, ngrid, s);
    if (T == 32) return launch_tile<32, 1>(mode, p, ngrid, s);
    return cudaErrorInvalidValue;
}

const void *fp32c_trial_entry(int T) {
    return T == 32 ? reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_TRIAL, 32, 1>)
                   : reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_TRIAL, 64, 1>);
}

}  // namespace fe
