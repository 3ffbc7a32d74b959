// fe_peak: peak-rate microbenchmarks of the units the solver's kernels are
// bound by, timed on the device in isolation, so that the roofline
// denominators of the benchmark are measured on the GPU at hand rather than
// derived from nominal unit counts.
//
//   FE_PEAK_FFMA       scalar FP32 fused multiply-add (fma.rn.f32), 2 flop each
//   FE_PEAK_FFMA2      packed FP32 fused multiply-add on pairs (fma.rn.f32x2), 4 flop each
//   FE_PEAK_DFMA       FP64 fused multiply-add, 2 flop each
//   FE_PEAK_MUFU_RCP   rcp.approx.ftz.f32 on the special-function unit, 1 op each
//   FE_PEAK_MUFU_LG2   lg2.approx.ftz.f32 on the special-function unit, 1 op each
//   FE_PEAK_TC_BF16    tcgen05.mma kind::f16 (BF16 operands, FP32 accumulation),
//                      M 128 x N 256 x K 16 per instruction, 2 M N K flop each
//   FE_PEAK_TC_TF32    tcgen05.mma kind::tf32, M 128 x N 256 x K 8
//
// The CUDA-core kinds run 8 independent dependency chains per thread (more
// than the pipeline latency needs with 64 warps per SM), fully unrolled 16
// deep so that the loop's own instructions are about 2 % of the stream, on
// every SM at full occupancy.  The tensor-core kinds run one CTA per SM whose
// elected thread issues a stream of MMAs into one tensor-memory accumulator
// (the K loop of a GEMM), with operands resident in shared memory.  The
// completion wait is bounded by a clock limit (about 2 s at full clock): a
// wait that gives up records a status and still frees the tensor memory.
//
// Rates are operations per second of the whole GPU (best of reps timings of
// one launch each, CUDA events on a private stream, after one warm-up launch
// that also scales the work to about target_ms).  No device memory is
// allocated: the results sink and the status word are static device
// variables.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdio>

#include "fe_internal.cuh"
#include "tc_ptx.cuh"

namespace fe {
namespace {

__device__ float pk_sink[1];
__device__ int pk_status[1];

constexpr int PK_CHAINS = 8, PK_UNROLL = 16, PK_THREADS = 256;

template <int KIND>
__global__ void __launch_bounds__(PK_THREADS) peak_alu_kernel(long long iters) {
    const float s0 = 1.0f + 1e-3f * (float)(threadIdx.x & 63);
    float acc = 0.0f;
    if (KIND == FE_PEAK_FFMA) {
        float a[PK_CHAINS];
#pragma unroll
        for (int j = 0; j < PK_CHAINS; ++j) a[j] = s0 + 0.01f * j;
        const float b = 0.9999f, c = 1e-4f;  // contracts toward 1: stays normal
        for (long long it = 0; it < iters; ++it)
#pragma unroll
            for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
                for (int j = 0; j < PK_CHAINS; ++j) a[j] = fmaf(a[j], b, c);
#pragma unroll
        for (int j = 0; j < PK_CHAINS; ++j) acc += a[j];
    } else if (KIND == FE_PEAK_FFMA2) {
        uint64_t a[PK_CHAINS];
        const uint64_t b = ((uint64_t)__float_as_uint(0.9999f) << 32) | __float_as_uint(0.9998f);
        const uint64_t c = ((uint64_t)__float_as_uint(1e-4f) << 32) | __float_as_uint(2e-4f);
#pragma unroll
        for (int j = 0; j < PK_CHAINS; ++j)
            a[j] = ((uint64_t)__float_as_uint(s0 + 0.01f * j) << 32) | __float_as_uint(s0 - 0.01f * j);
        for (long long it = 0; it < iters; ++it)
#pragma unroll
            for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
                for (int j = 0; j < PK_CHAINS; ++j)
                    asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[j]) : "l"(b), "l"(c));
#pragma unroll
        for (int j = 0; j < PK_CHAINS; ++j)
            acc += __uint_as_float((uint32_t)a[j]) + __uint_as_float((uint32_t)(a[j] >> 32));
    } else if (KIND == FE_PEAK_DFMA) {
        double a[PK_CHAINS];
#pragma unroll
        for (int j = 0; j < PK_CHAINS; ++j) a[j] = (double)s0 + 0.01 * j;
        const double b = 0.9999, c = 1e-4;
        for (long long it = 0; it < iters; ++it)
#pragma unroll
            for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
                for (int j = 0; j < PK_CHAINS; ++j) a[j] = fma(a[j], b, c);
#pragma unroll
        for (int j = 0; j < PK_CHAINS; ++j) acc += (float)a[j];
    } else if (KIND == FE_PEAK_MUFU_RCP) {
        float a[PK_CHAINS];
#pragma unroll
        for (int j = 0; j < PK_CHAINS; ++j) a[j] = s0 + 0.01f * j;
        // x <- 1/x + 1/2 (fixed point 1.28, contracting), one FADD per rcp, so
        // that no pair of reciprocals can be folded away
        for (long long it = 0; it < iters; ++it)
#pragma unroll
            for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
                for (int j = 0; j < PK_CHAINS; ++j) {
                    asm volatile("rcp.approx.ftz.f32 %0, %0;" : "+f"(a[j]));
                    a[j] += 0.5f;
                }
#pragma unroll
        for (int j = 0; j < PK_CHAINS; ++j) acc += a[j];
    } else {  // FE_PEAK_MUFU_LG2: x <- lg2(x) + 2 (fixed point 4, contracting), one FADD per lg2
        float a[PK_CHAINS];
#pragma unroll
        for (int j = 0; j < PK_CHAINS; ++j) a[j] = 3.0f + s0 + 0.01f * j;
        for (long long it = 0; it < iters; ++it)
#pragma unroll
            for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
                for (int j = 0; j < PK_CHAINS; ++j) {
                    asm volatile("lg2.approx.ftz.f32 %0, %0;" : "+f"(a[j]));
                    a[j] += 2.0f;
                }
#pragma unroll
        for (int j = 0; j < PK_CHAINS; ++j) acc += a[j];
    }
    if (acc == -1.25f) pk_sink[0] = acc;  // never true; keeps the chains live
}

// Tensor-core peak: one CTA per SM (its shared memory admits no second one),
// thread 0 issues `iters` MMAs D += A B^T (M 128, N 256) from shared memory.
constexpr int PK_TC_M = 128, PK_TC_N = 256, PK_TC_SMEM = 160 * 1024;

__device__ __forceinline__ uint32_t pk_hash(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

template <int FMT>
__global__ void __launch_bounds__(128, 1) peak_tc_kernel(int iters) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int EB = FMT == 1 ? 2 : 4, K = FMT == 1 ? 16 : 8;  // one MMA: 32 bytes of K per row
    unsigned char *sA = sm;
    unsigned char *sB = sm + PK_TC_M * K * EB;
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5;
    // small pseudo-random operands (values in [-1, 1)) in the K-major layout
    for (int e = tid; e < (PK_TC_M + PK_TC_N) * K; e += blockDim.x) {
        const bool isA = e < PK_TC_M * K;
        const int ee = isA ? e : e - PK_TC_M * K, r = ee / K, k = ee % K;
        const float v = (float)(int)(pk_hash((uint32_t)e * 2654435761u + blockIdx.x) & 0xFFFF) / 32768.0f - 1.0f;
        unsigned char *dst = (isA ? sA : sB) + tc::kmajor_offset(r, k, K, EB);
        if (FMT == 1)
            *reinterpret_cast<__nv_bfloat16 *>(dst) = __float2bfloat16_rn(v);
        else
            *reinterpret_cast<float *>(dst) = tc::round_tf32(v);
    }
    if (tid == 0) tc::mbar_init(&bar, 1);
    if (warp == 0) tc::tmem_alloc(&tbase, PK_TC_N);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tbase;
    if (tid == 0) {
        const uint32_t sbo = (uint32_t)(K * EB / 16) * 128;
        const uint64_t ad = tc::make_smem_desc(tc::smem_u32(sA), tc::LBO_BYTES, sbo);
        const uint64_t bd = tc::make_smem_desc(tc::smem_u32(sB), tc::LBO_BYTES, sbo);
        constexpr uint32_t idesc = tc::make_idesc(FMT, PK_TC_M, PK_TC_N);
        for (int i = 0; i < iters; ++i) tc::mma<FMT>(taddr, ad, bd, idesc, i > 0 ? 1u : 0u);
        tc::mma_commit(&bar);
    }
    // bounded wait: about 4e9 SM clocks (2 s at 2 GHz), then a status
    auto wait = [&]() {
        const long long t0 = clock64();
        for (;;) {
            if (tc::mbar_try_wait(&bar, 0)) return true;
            if (clock64() - t0 > 4000000000ll) return false;
        }
    };
    bool ok = wait();
    if (!ok) {
        if (tid == 0) atomicExch(pk_status, 1);
        ok = wait();  // a second bounded chance for MMAs in flight before the memory is freed
    }
    tc::fence_after_sync();
    // warp 0 reads one accumulator row (a warp-wide load, so the whole warp
    // must agree that the MMAs completed) so that the result is used
    const bool wok = __all_sync(0xffffffffu, ok);
    if (wok && warp == 0) {
        float v[8];
        tc::tmem_ld8(taddr, v);
        tc::tmem_ld_wait();
        if (tid == 0 && v[0] == -1.25f) pk_sink[0] = v[0];
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, PK_TC_N);
}

cudaError_t launch_peak(int kind, long long iters, int sms, int bps, cudaStream_t s) {
    const dim3 g(sms * bps);
    switch (kind) {
        case FE_PEAK_FFMA: peak_alu_kernel<FE_PEAK_FFMA><<<g, PK_THREADS, 0, s>>>(iters); break;
        case FE_PEAK_FFMA2: peak_alu_kernel<FE_PEAK_FFMA2><<<g, PK_THREADS, 0, s>>>(iters); break;
        case FE_PEAK_DFMA: peak_alu_kernel<FE_PEAK_DFMA><<<g, PK_THREADS, 0, s>>>(iters); break;
        case FE_PEAK_MUFU_RCP: peak_alu_kernel<FE_PEAK_MUFU_RCP><<<g, PK_THREADS, 0, s>>>(iters); break;
        case FE_PEAK_MUFU_LG2: peak_alu_kernel<FE_PEAK_MUFU_LG2><<<g, PK_THREADS, 0, s>>>(iters); break;
        case FE_PEAK_TC_BF16: peak_tc_kernel<1><<<sms, 128, PK_TC_SMEM, s>>>((int)iters); break;
        case FE_PEAK_TC_TF32: peak_tc_kernel<2><<<sms, 128, PK_TC_SMEM, s>>>((int)iters); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Operations (flop for the FMA and tensor kinds, instructions for the MUFU
// kinds) of one launch.
double peak_ops(int kind, long long iters, int sms, int bps) {
    const double thr = (double)sms * bps * PK_THREADS, per = (double)PK_CHAINS * PK_UNROLL * (double)iters;
    switch (kind) {
        case FE_PEAK_FFMA: return thr * per * 2.0;
        case FE_PEAK_FFMA2: return thr * per * 4.0;
        case FE_PEAK_DFMA: return thr * per * 2.0;
        case FE_PEAK_MUFU_RCP:
        case FE_PEAK_MUFU_LG2: return thr * per;
        case FE_PEAK_TC_BF16: return (double)sms * iters * 2.0 * PK_TC_M * PK_TC_N * 16;
        case FE_PEAK_TC_TF32: return (double)sms * iters * 2.0 * PK_TC_M * PK_TC_N * 8;
        default: return 0.0;
    }
}

}  // namespace
}  // namespace fe

using namespace fe;

extern "C" fe_status fe_peak(int kind, double target_ms, int reps, double *rate, double *best_ms, int *sms_out) {
    if (kind < FE_PEAK_FFMA || kind > FE_PEAK_TC_TF32 || !rate || reps < 1 || reps > 100 || !(target_ms > 0.0) ||
        target_ms > 2000.0) {
        set_global_error("fe_peak: kind outside 0..6, reps outside 1..100, target_ms outside (0, 2000] or rate NULL");
        return FE_EINVAL;
    }
    int dev = 0, sms = 0, bps = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        set_global_error("fe_peak: no CUDA device");
        return FE_ECUDA;
    }
    const bool tc = kind == FE_PEAK_TC_BF16 || kind == FE_PEAK_TC_TF32;
    cudaError_t e = cudaSuccess;
    if (tc) {
        e = cudaFuncSetAttribute(kind == FE_PEAK_TC_BF16 ? (const void *)peak_tc_kernel<1> : (const void *)peak_tc_kernel<2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, PK_TC_SMEM);
    } else {
        const void *fn = nullptr;
        switch (kind) {
            case FE_PEAK_FFMA: fn = (const void *)peak_alu_kernel<FE_PEAK_FFMA>; break;
            case FE_PEAK_FFMA2: fn = (const void *)peak_alu_kernel<FE_PEAK_FFMA2>; break;
            case FE_PEAK_DFMA: fn = (const void *)peak_alu_kernel<FE_PEAK_DFMA>; break;
            case FE_PEAK_MUFU_RCP: fn = (const void *)peak_alu_kernel<FE_PEAK_MUFU_RCP>; break;
            default: fn = (const void *)peak_alu_kernel<FE_PEAK_MUFU_LG2>; break;
        }
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, PK_THREADS, 0);
        if (e == cudaSuccess && bps < 1) bps = 1;
    }
    if (e != cudaSuccess) {
        set_global_error("fe_peak: kernel set-up failed");
        return FE_ECUDA;
    }
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    fe_status st = FE_OK;
    const int zero = 0;
    int hstat = 0;
    float ms = 0.f, best = 0.f;
    long long iters = tc ? 4096 : (kind == FE_PEAK_DFMA ? 8 : 256);
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaMemcpyToSymbolAsync(pk_status, &zero, sizeof zero, 0,
                                                                       cudaMemcpyHostToDevice, s) != cudaSuccess) {
        st = FE_ECUDA;
        goto done;
    }
    // warm-up, which also scales the work to about target_ms per launch
    for (int pass = 0; pass < 2; ++pass) {
        if (cudaEventRecord(e0, s) != cudaSuccess || launch_peak(kind, iters, sms, bps, s) != cudaSuccess ||
            cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            st = FE_ECUDA;
            goto done;
        }
        if (pass == 0) {
            const double scale = target_ms / std::max(1e-3, (double)ms);
            iters = std::max<long long>(1, (long long)(iters * std::min(scale, 1e5)));
            if (tc) iters = std::min<long long>(iters, 1 << 22);  // the wait bound covers this many MMAs
        }
    }
    for (int r = 0; r < reps; ++r) {
        if (cudaEventRecord(e0, s) != cudaSuccess || launch_peak(kind, iters, sms, bps, s) != cudaSuccess ||
            cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            st = FE_ECUDA;
            goto done;
        }
        if (r == 0 || ms < best) best = ms;
    }
    if (cudaMemcpyFromSymbolAsync(&hstat, pk_status, sizeof hstat, 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        st = FE_ECUDA;
        goto done;
    }
    if (hstat) {
        set_global_error("fe_peak: a tensor-core completion wait ran out");
        st = FE_ETIMEOUT;
        goto done;
    }
    *rate = peak_ops(kind, iters, sms, bps) / (best * 1e-3);
    if (best_ms) *best_ms = best;
    if (sms_out) *sms_out = sms;
done:
    if (st == FE_ECUDA) set_global_error("fe_peak: a CUDA call failed");
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    return st;
}

extern "C" fe_status fe_device_sms(int *sms) {
    int dev = 0;
    if (!sms) return FE_EINVAL;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_global_error("fe_device_sms: no CUDA device");
        return FE_ECUDA;
    }
    return FE_OK;
}
