// Quality measures the paper reports (Sec. III): PSNR, and the SSIM index of
// Wang, Bovik, Sheikh and Simoncelli (2004) as the paper cites it.
//
// SSIM: at every position where an 11 x 11 window fits in the image, local
// means, variances and covariance under the circular Gaussian window
// (sigma = 1.5, normalised to sum 1) give
//   ((2 mx my + C1)(2 sxy + C2)) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2)),
// C1 = (0.01 peak)^2, C2 = (0.03 peak)^2; the index is the mean over those
// positions.  The window is separable, so each CTA filters its tile's rows
// and then its columns.  The moments are accumulated in FP64: E[x^2] - mx^2
// cancels badly in FP32 at speckle intensities, and this routine is an
// evaluation, not the solver's hot path.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <vector>

#include "fe_internal.cuh"

namespace fe {
namespace {

constexpr int SW = 11, SR = 5;       // window side and radius
constexpr int ST = 32;               // output tile (ST x ST SSIM positions)
constexpr int SIN = ST + SW - 1;     // input tile side (42)
constexpr int SNT = 256;

__constant__ double c_gauss[SW];

// one CTA: SSIM of an ST x ST block of window positions; per-CTA sum into part
__global__ void __launch_bounds__(SNT) ssim_kernel(const float *__restrict__ x, const float *__restrict__ y, int H,
                                                    int W, double C1, double C2, double *__restrict__ part) {
    extern __shared__ double sh[];
    double *hx = sh;                      // row-filtered moments: 5 planes of SIN x ST
    float *sx = reinterpret_cast<float *>(sh + 5 * SIN * ST);  // input tiles
    float *sy = sx + SIN * SIN;
    __shared__ double red[SNT / 32];
    const int Ho = H - SW + 1, Wo = W - SW + 1;  // positions (top-left corners)
    const int oy0 = blockIdx.y * ST, ox0 = blockIdx.x * ST;
    const int tid = threadIdx.x;
    for (int i = tid; i < SIN * SIN; i += SNT) {
        const int r = i / SIN, c = i % SIN;
        const int yy = min(oy0 + r, H - 1), xx = min(ox0 + c, W - 1);  // clamped reads feed only unused outputs
        sx[i] = x[(size_t)yy * W + xx];
        sy[i] = y[(size_t)yy * W + xx];
    }
    __syncthreads();
    // horizontal pass: SIN rows x ST output columns, 5 moments each
    for (int i = tid; i < SIN * ST; i += SNT) {
        const int r = i / ST, c = i % ST;
        double m1 = 0, m2 = 0, m3 = 0, m4 = 0, m5 = 0;
#pragma unroll
        for (int t = 0; t < SW; ++t) {
            const double a = sx[r * SIN + c + t], b = sy[r * SIN + c + t], g = c_gauss[t];
            m1 += g * a;
            m2 += g * b;
            m3 += g * a * a;
            m4 += g * b * b;
            m5 += g * a * b;
        }
        hx[0 * SIN * ST + i] = m1;
        hx[1 * SIN * ST + i] = m2;
        hx[2 * SIN * ST + i] = m3;
        hx[3 * SIN * ST + i] = m4;
        hx[4 * SIN * ST + i] = m5;
    }
    __syncthreads();
    // vertical pass and the index
    double acc = 0.0;
    for (int i = tid; i < ST * ST; i += SNT) {
        const int r = i / ST, c = i % ST;
        if (oy0 + r >= Ho || ox0 + c >= Wo) continue;
        double m[5] = {0, 0, 0, 0, 0};
#pragma unroll
        for (int t = 0; t < SW; ++t) {
            const double g = c_gauss[t];
#pragma unroll
            for (int q = 0; q < 5; ++q) m[q] += g * hx[q * SIN * ST + (r + t) * ST + c];
        }
        const double mx = m[0], my = m[1];
        const double vx = m[2] - mx * mx, vy = m[3] - my * my, cxy = m[4] - mx * my;
        acc += ((2.0 * mx * my + C1) * (2.0 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2));
    }
    // CTA sum in a fixed order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < SNT / 32; ++w) s += red[w];
        part[blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

constexpr int PB = 256;  // blocks of the PSNR reduction
__global__ void __launch_bounds__(256) sqdiff_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                                     size_t n, double *__restrict__ part) {
    __shared__ double red[8];
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double d = (double)x[i] - (double)y[i];
        s += d * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

bool device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

fe_status fail(fe_status s, const char *msg) {
    set_global_error(msg);
    return s;
}

// per-block partial sums -> one double, summed on the host in block order
fe_status finish(double *d_part, int nparts, cudaStream_t s, double *sum) {
    std::vector<double> h(nparts);
    cudaError_t e = cudaMemcpyAsync(h.data(), d_part, sizeof(double) * nparts, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaError_t e2 = cudaFreeAsync(d_part, s);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return fail(FE_ECUDA, cudaGetErrorString(e));
    double t = 0.0;
    for (double v : h) t += v;
    *sum = t;
    return FE_OK;
}

}  // namespace
}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_ssim(const float *x, const float *y, int H, int W, double peak, double *out, void *stream) {
    set_global_error("");
    if (!x || !y || !out) return fail(FE_EINVAL, "fe_ssim: NULL argument");
    if (H < SW || W < SW) return fail(FE_EINVAL, "fe_ssim: the image must be at least 11 x 11");
    if (!(peak > 0.0) || !std::isfinite(peak)) return fail(FE_EINVAL, "fe_ssim: peak must be > 0");
    if (!device_ptr(x) || !device_ptr(y)) return fail(FE_EINVAL, "fe_ssim: x and y must be device pointers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // per-device set-up (the window in constant memory, the kernel's
    // shared-memory opt-in), once per device and process
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fail(FE_ECUDA, "fe_ssim: no device");
    {
        static std::mutex mu;
        static bool ready[64] = {};
        std::lock_guard<std::mutex> lk(mu);
        if (!ready[dev]) {
            double g[SW], sum = 0.0;
            for (int i = 0; i < SW; ++i) sum += (g[i] = std::exp(-0.5 * (i - SR) * (i - SR) / (1.5 * 1.5)));
            for (int i = 0; i < SW; ++i) g[i] /= sum;
            if (cudaMemcpyToSymbol(c_gauss, g, sizeof g) != cudaSuccess)
                return fail(FE_ECUDA, "fe_ssim: window upload failed");
            const int smem = (int)(5 * SIN * ST * sizeof(double) + 2 * SIN * SIN * sizeof(float));
            if (cudaFuncSetAttribute(ssim_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
                return fail(FE_ECUDA, "fe_ssim: shared-memory attribute failed");
            ready[dev] = true;
        }
    }
    const int Ho = H - SW + 1, Wo = W - SW + 1;
    const dim3 grid((Wo + ST - 1) / ST, (Ho + ST - 1) / ST);
    const int nparts = (int)(grid.x * grid.y);
    double *d_part = nullptr;
    if (cudaMallocAsync(&d_part, sizeof(double) * nparts, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(FE_ENOMEM, "fe_ssim: allocation failed");
    }
    const size_t smem = 5 * SIN * ST * sizeof(double) + 2 * SIN * SIN * sizeof(float);
    const double C1 = (0.01 * peak) * (0.01 * peak), C2 = (0.03 * peak) * (0.03 * peak);
    ssim_kernel<<<grid, SNT, smem, s>>>(x, y, H, W, C1, C2, d_part);
    if (cudaGetLastError() != cudaSuccess) {
        cudaFreeAsync(d_part, s);
        return fail(FE_ECUDA, "fe_ssim: launch failed");
    }
    double sum = 0.0;
    fe_status st = finish(d_part, nparts, s, &sum);
    if (st != FE_OK) return st;
    *out = sum / ((double)Ho * (double)Wo);
    return FE_OK;
}

fe_status fe_psnr(const float *x, const float *y, long long n, double peak, double *out, void *stream) {
    set_global_error("");
    if (!x || !y || !out || n <= 0) return fail(FE_EINVAL, "fe_psnr: NULL argument or n <= 0");
    if (!(peak > 0.0) || !std::isfinite(peak)) return fail(FE_EINVAL, "fe_psnr: peak must be > 0");
    if (!device_ptr(x) || !device_ptr(y)) return fail(FE_EINVAL, "fe_psnr: x and y must be device pointers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *d_part = nullptr;
    if (cudaMallocAsync(&d_part, sizeof(double) * PB, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(FE_ENOMEM, "fe_psnr: allocation failed");
    }
    sqdiff_kernel<<<PB, 256, 0, s>>>(x, y, (size_t)n, d_part);
    if (cudaGetLastError() != cudaSuccess) {
        cudaFreeAsync(d_part, s);
        return fail(FE_ECUDA, "fe_psnr: launch failed");
    }
    double sse = 0.0;
    fe_status st = finish(d_part, PB, s, &sse);
    if (st != FE_OK) return st;
    const double mse = sse / (double)n;
    *out = mse == 0.0 ? INFINITY : 10.0 * std::log10(peak * peak / mse);
    return FE_OK;
}

}  // extern "C"
