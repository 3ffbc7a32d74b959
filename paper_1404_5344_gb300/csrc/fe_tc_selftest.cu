// fe_tc_gemm_selftest: D[128 x N] = A[128 x K] * B[N x K]^T through one CTA
// of tcgen05.mma with the operand layout and descriptors of tc_ptx.cuh.
// It exercises, in isolation, the tensor-core building block of the precision
// forms, so that a test can pin the layout against a plain reference.
#include <cuda_runtime.h>

#include <cstring>

#include "fe_internal.cuh"
#include "tc_ptx.cuh"

namespace fe {
namespace {

constexpr int ST_M = 128, ST_NMAX = 64, ST_KMAX = 128;

template <int FMT>
__global__ void __launch_bounds__(128, 1)
    tc_selftest_kernel(const float *A, const float *B, float *D, int N, int K, int *status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int EB = FMT == 1 ? 2 : 4;  // operand bytes
    unsigned char *sA = sm;
    unsigned char *sB = sm + ST_M * ST_KMAX * 4;
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5;

    // operands in the K-major core-matrix layout
    for (int e = tid; e < ST_M * K; e += blockDim.x) {
        const int r = e / K, k = e % K;
        const float v = A[e];
        if (FMT == 1)
            *reinterpret_cast<__nv_bfloat16 *>(sA + tc::kmajor_offset(r, k, K, EB)) = __float2bfloat16_rn(v);
        else
            *reinterpret_cast<float *>(sA + tc::kmajor_offset(r, k, K, EB)) = tc::round_tf32(v);
    }
    for (int e = tid; e < N * K; e += blockDim.x) {
        const int r = e / K, k = e % K;
        const float v = B[e];
        if (FMT == 1)
            *reinterpret_cast<__nv_bfloat16 *>(sB + tc::kmajor_offset(r, k, K, EB)) = __float2bfloat16_rn(v);
        else
            *reinterpret_cast<float *>(sB + tc::kmajor_offset(r, k, K, EB)) = tc::round_tf32(v);
    }
    if (tid == 0) tc::mbar_init(&bar, 1);
    if (warp == 0) tc::tmem_alloc(&tbase, 64);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tbase;

    if (tid == 0) {
        const int kstep = FMT == 1 ? 16 : 8;
        const uint32_t sbo = (uint32_t)(K * EB / 16) * 128;
        const uint32_t idesc = tc::make_idesc(FMT, ST_M, N);
        for (int ks = 0; ks < K / kstep; ++ks) {
            const uint64_t ad = tc::make_smem_desc(tc::smem_u32(sA) + ks * 2 * tc::LBO_BYTES, tc::LBO_BYTES, sbo);
            const uint64_t bd = tc::make_smem_desc(tc::smem_u32(sB) + ks * 2 * tc::LBO_BYTES, tc::LBO_BYTES, sbo);
            tc::mma<FMT>(taddr, ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
        tc::mma_commit(&bar);
    }
    bool ok = tc::mbar_wait(&bar, 0);
    if (!ok) {
        if (tid == 0) atomicExch(status, 1);
        ok = tc::mbar_wait(&bar, 0);  // give in-flight MMAs a second bounded chance before freeing TMEM
    }
    tc::fence_after_sync();
    if (ok) {
        const int row = warp * 32 + (tid & 31);
        for (int c = 0; c < N; c += 8) {
            float v[8];
            tc::tmem_ld8(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            tc::tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 8; ++j) D[row * N + c + j] = v[j];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 64);
}

// Bounded-wait self-test: one CTA allocates tensor memory, waits with a
// bounded loop on an mbarrier that nothing ever arrives on, then frees the
// tensor memory and reports whether the wait gave up.  It exercises the
// time-out path of the trial kernels' MMA waits without faulting or hanging
// the GPU.
__global__ void __launch_bounds__(128, 1) tc_wait_selftest_kernel(uint32_t max_iter, int *timed_out) {
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) tc::mbar_init(&bar, 1);
    if (warp == 0) tc::tmem_alloc(&tbase, 32);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const bool ok = tc::mbar_wait(&bar, 0, max_iter);  // no arrival: must give up
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 32);
    if (tid == 0) *timed_out = ok ? 0 : 1;
}

}  // namespace
}  // namespace fe

using namespace fe;

extern "C" fe_status fe_tc_wait_selftest(unsigned max_iter, int *timed_out) {
    if (!timed_out || max_iter == 0 || max_iter > (1u << 24)) return FE_EINVAL;
    int *d = nullptr, h = -1;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return FE_ENOMEM;
    fe_status st = FE_OK;
    tc_wait_selftest_kernel<<<1, 128>>>(max_iter, d);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        st = FE_ECUDA;
    cudaFree(d);
    *timed_out = h;
    if (st == FE_OK && h == 1) st = FE_ETIMEOUT;
    return st;
}

extern "C" fe_status fe_tc_gemm_selftest(int prec, int N, int K, const float *A, const float *B, float *D) {
    if ((prec != FE_BF16 && prec != FE_TF32) || !A || !B || !D) return FE_EINVAL;
    const int kstep = prec == FE_BF16 ? 16 : 8;
    if (N < 16 || N > ST_NMAX || N % 16 || K < kstep || K > ST_KMAX || K % kstep) return FE_EINVAL;
    float *dA = nullptr, *dB = nullptr, *dD = nullptr;
    int *dS = nullptr;
    fe_status st = FE_OK;
    const size_t smem = (size_t)ST_M * ST_KMAX * 4 + (size_t)ST_NMAX * ST_KMAX * 4;
    int hs = 0;
    if (cudaMalloc(&dA, sizeof(float) * ST_M * K) != cudaSuccess || cudaMalloc(&dB, sizeof(float) * N * K) != cudaSuccess ||
        cudaMalloc(&dD, sizeof(float) * ST_M * N) != cudaSuccess || cudaMalloc(&dS, sizeof(int)) != cudaSuccess) {
        st = FE_ENOMEM;
        goto done;
    }
    if (cudaMemcpy(dA, A, sizeof(float) * ST_M * K, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(dB, B, sizeof(float) * N * K, cudaMemcpyDefault) != cudaSuccess || cudaMemset(dS, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(dD, 0xff, sizeof(float) * ST_M * N) != cudaSuccess) {
        st = FE_ECUDA;
        goto done;
    }
    if (prec == FE_BF16) {
        cudaFuncSetAttribute(tc_selftest_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        tc_selftest_kernel<1><<<1, 128, smem>>>(dA, dB, dD, N, K, dS);
    } else {
        cudaFuncSetAttribute(tc_selftest_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        tc_selftest_kernel<2><<<1, 128, smem>>>(dA, dB, dD, N, K, dS);
    }
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        st = FE_ECUDA;
        goto done;
    }
    if (cudaMemcpy(&hs, dS, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(D, dD, sizeof(float) * ST_M * N, cudaMemcpyDefault) != cudaSuccess) {
        st = FE_ECUDA;
        goto done;
    }
    if (hs) st = FE_ETIMEOUT;
done:
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(dS);
    return st;
}
