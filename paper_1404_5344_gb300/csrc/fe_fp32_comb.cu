// FP32 trial kernel instantiated for the combined model (Eq. newmodel,
// Sec. III-A) in w = log u; the template is in fe_fp32_kernel.cuh.
#include <cuda_runtime.h>

#include "fe_fp32_kernel.cuh"

namespace fe {

cudaError_t fp32c_prepare() {
    cudaError_t e = prepare_tile<64, 1>();
    if (e == cudaSuccess) e = prepare_tile<32, 1>();
    if (e == cudaSuccess) e = prepare_tile<32, 1, 4>();
    return e;
}

cudaError_t fp32c_launch(int mode, const KParams &p, int ngrid, cudaStream_t s, int T, int cl) {
    if (T == 64 && cl == 1) return launch_tile<64, 1>(mode, p, ngrid, s);
    if (T == 32 && cl == 1) return launch_tile<32, 1>(mode, p, ngrid, s);
    if (T == 32 && cl == 4) return launch_tile<32, 1, 4>(mode, p, ngrid, s);
    return cudaErrorInvalidValue;
}

const void *fp32c_trial_entry(int T, int cl) {
    if (T == 32)
        return cl == 4 ? reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_TRIAL, 32, 1, 4>)
                       : reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_TRIAL, 32, 1, 1>);
    return reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_TRIAL, 64, 1, 1>);
}

const void *fp32c_ptrial_entry(int T) {
    return T == 32 ? reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_PTRIAL, 32, 1, 1>)
                   : reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_PTRIAL, 64, 1, 1>);
}

}  // namespace fe
