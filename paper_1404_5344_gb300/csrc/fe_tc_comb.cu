// Tensor-core trial kernel instantiated for the combined model (Eq. newmodel,
// Sec. III-A) in w = log u; the template is in fe_tc_kernel.cuh.
#include "fe_tc_kernel.cuh"

namespace fe {

cudaError_t tcc_prepare() {
    cudaError_t e = prepare_fmt<1, 1>();
    if (e == cudaSuccess) e = prepare_fmt<2, 1>();
    return e != cudaSuccess ? e : prepare_fmt<3, 1>();
}

cudaError_t tcc_launch(int mode, int fmt, const KParams &p, int ngrid, cudaStream_t s) {
    return fmt == 1 ? launch_fmt<1, 1>(mode, p, ngrid, s)
                    : (fmt == 3 ? launch_fmt<3, 1>(mode, p, ngrid, s) : launch_fmt<2, 1>(mode, p, ngrid, s));
}

const void *tcc_trial_entry(int fmt) { return trial_entry<1>(fmt); }
const void *tcc_ptrial_entry(int fmt) { return ptrial_entry<1>(fmt); }

}  // namespace fe
