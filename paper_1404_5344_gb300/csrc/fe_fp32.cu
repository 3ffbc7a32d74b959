// FP32 trial kernel: entry points of the FP32 form.  The kernel template is in
// fe_fp32_kernel.cuh; this unit instantiates it for the model with the
// I-divergence data term (Eq. variant) and dispatches the combined model to
// fe_fp32_comb.cu (instantiated there, compiled in parallel).
#include <cuda_runtime.h>

#include "fe_fp32_kernel.cuh"

namespace fe {

bool fp32_tile_supported(int T) { return T == 64 || T == 32; }
size_t fp32_smem_bytes(int T) { return T == 32 ? Geo<32>::SM_BYTES : Geo<64>::SM_BYTES; }
int fp32_tile() { return fp32_tile_size; }
int fp32_threads(int T) { return T == 32 ? Geo<32>::NT : Geo<64>::NT; }
int fp32_ctas_per_sm(int T) { return T == 32 ? Geo<32>::MINB : Geo<64>::MINB; }

cudaError_t fp32_prepare() {
    cudaError_t e = prepare_tile<64, 0>();
    if (e == cudaSuccess) e = prepare_tile<32, 0>();
    if (e == cudaSuccess) e = prepare_tile<32, 0, 4>();
    if (e == cudaSuccess) e = fp32c_prepare();
    if (e == cudaSuccess) e = fp32cl64_prepare();
    return e;
}

cudaError_t fp32_launch(int mode, const KParams &p, int ngrid, cudaStream_t s, int T, int model, int cl) {
    if (T == 64 && cl == 4) return fp32cl64_launch(mode, p, ngrid, s, model);
    if (model == 1) return fp32c_launch(mode, p, ngrid, s, T, cl);
    if (T == 64 && cl == 1) return launch_tile<64, 0>(mode, p, ngrid, s);
    if (T == 32 && cl == 1) return launch_tile<32, 0>(mode, p, ngrid, s);
    if (T == 32 && cl == 4) return launch_tile<32, 0, 4>(mode, p, ngrid, s);
    return cudaErrorInvalidValue;
}

const void *fp32_trial_entry(int T, int model, int cl) {
    if (T == 64 && cl == 4) return fp32cl64_trial_entry(model);
    if (model == 1) return fp32c_trial_entry(T, cl);
    if (T == 32)
        return cl == 4 ? reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_TRIAL, 32, 0, 4>)
                       : reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_TRIAL, 32, 0, 1>);
    return reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_TRIAL, 64, 0, 1>);
}

const void *fp32_ptrial_entry(int T, int model) {
    if (model == 1) return fp32c_ptrial_entry(T);
    return T == 32 ? reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_PTRIAL, 32, 0, 1>)
                   : reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_PTRIAL, 64, 0, 1>);
}

}  // namespace fe
