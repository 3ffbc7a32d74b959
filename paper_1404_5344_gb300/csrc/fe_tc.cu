// Tensor-core forms: host side (rounding of the bank, operand tables, entry
// points) and the instantiation for the model with the I-divergence data
// term; the kernel template is in fe_tc_kernel.cuh, the combined model's
// instantiation in fe_tc_comb.cu.
#include <cstring>
#include <vector>

#include "fe_tc_kernel.cuh"

namespace fe {
namespace {

// Host rounding of the filter bank: BF16 round-to-nearest-even, TF32
// round-to-nearest with ties away from zero (as cvt.rna.tf32.f32).
uint32_t f2u(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return u;
}
float u2f(uint32_t u) {
    float x;
    std::memcpy(&x, &u, 4);
    return x;
}

}  // namespace

float tc_round(int fmt, float x) {
    uint32_t u = f2u(x);
    if (fmt != 2) {  // BF16 (forms 1 and 3)
        u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    } else {
        u = (u + 0x1000u) & 0xFFFFE000u;
    }
    return u2f(u);
}

void tc_build_weights(int fmt, const float *filters, int nf, std::vector<unsigned char> &fwd,
                      std::vector<unsigned char> &adj) {
    const int eb = fmt != 2 ? 2 : 4, kpass = fmt != 2 ? 64 : 56;
    fwd.assign((size_t)NF * kpass * eb, 0);
    adj.assign((size_t)NTAP * NF * eb, 0);
    auto put = [&](std::vector<unsigned char> &buf, int r, int k, int K, float v) {
        const uint32_t off = tc::kmajor_offset(r, k, K, eb);
        const uint32_t bits = f2u(tc_round(fmt, v));
        if (eb == 2) {
            const uint16_t h = (uint16_t)(bits >> 16);
            std::memcpy(&buf[off], &h, 2);
        } else {
            std::memcpy(&buf[off], &bits, 4);
        }
    };
    for (int i = 0; i < nf && i < NF; ++i)
        for (int t = 0; t < KT; ++t) {
            // forward: K index 8a + b reads u(p + (a, b)) of the window, i.e.
            // correlation with the flipped filter (index 8a + 7 stays 0)
            const int a = t / KS, b = t % KS;
            put(fwd, i, 8 * a + b, kpass, filters[(size_t)i * KT + (KT - 1 - t)]);
            // adjoint: S[q, t] = sum_i k_i[t] r_i(q)
            put(adj, t, i, NF, filters[(size_t)i * KT + t]);
        }
}

size_t tc_smem_bytes(int fmt) { return fmt == 1 ? Cfg<1>::BYTES : (fmt == 3 ? Cfg<3>::BYTES : Cfg<2>::BYTES); }
int tc_threads() { return NT; }
int tc_ctas_per_sm(int fmt) { return fmt != 2 ? 3 : 2; }

cudaError_t tc_prepare() {
    cudaError_t e = prepare_fmt<1, 0>();
    if (e == cudaSuccess) e = prepare_fmt<2, 0>();
    if (e == cudaSuccess) e = prepare_fmt<3, 0>();
    if (e == cudaSuccess) e = tcc_prepare();
    return e;
}

cudaError_t tc_launch(int mode, int fmt, const KParams &p, int ngrid, cudaStream_t s, int model) {
    if (model == 1) return tcc_launch(mode, fmt, p, ngrid, s);
    return fmt == 1 ? launch_fmt<1, 0>(mode, p, ngrid, s)
                    : (fmt == 3 ? launch_fmt<3, 0>(mode, p, ngrid, s) : launch_fmt<2, 0>(mode, p, ngrid, s));
}

const void *tc_trial_entry(int fmt, int model) { return model == 1 ? tcc_trial_entry(fmt) : trial_entry<0>(fmt); }
const void *tc_ptrial_entry(int fmt, int model) { return model == 1 ? tcc_ptrial_entry(fmt) : ptrial_entry<0>(fmt); }

}  // namespace fe
