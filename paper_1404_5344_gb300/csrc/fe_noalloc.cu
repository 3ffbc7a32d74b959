// fe_gradient_noalloc: grad F(u) and F(u) of one image without any device
// allocation.
//
// Who needs this: code that may not call cudaMalloc (or any allocating
// routine) on the path where it evaluates the prior's gradient - e.g. a plugin
// that must live inside a host framework's fixed device-memory pool, or a
// real-time loop where an allocation (and the implicit synchronisation it can
// bring) is not allowed.  Such a caller owns every input and output buffer;
// the per-tile partial sums, counters, tile list and weight tables this kernel
// needs as scratch live in one file-scope device array instead.
//
// The array is a module global: every GPU that loads this library holds it
// (NA_SCRATCH_BYTES, about 0.3 MB) until the process exits.  All calls share
// it and it keeps the last call's contents; each call rewrites everything it
// reads before the gradient kernel runs and the kernel resets its own arrival
// counter.  Two calls whose kernels overlap on the GPU (different streams,
// same device) race on the array and must be serialised by the caller.
//
// Device set-up: the first call on a device makes that device current,
// resolves the device address of the array with cudaGetSymbolAddress (in host
// code the array's name is only a host-side stand-in, not a device address)
// and raises the kernel's shared-memory limit.  That first call should come
// before any stream capture.  Both belong to the device's primary context:
// cudaDeviceReset makes them stale, so a call whose launch fails forgets the
// device's set-up and the next call redoes it.
#include <cuda_runtime.h>

#include <mutex>

#include "fe_internal.cuh"

namespace fe {
namespace {

constexpr int NA_MAX_TILES = 4096;  // e.g. one 4096 x 4096 image (64 x 64 tiles)
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t NA_OFF_WF = 0;
constexpr size_t NA_OFF_WA = align256(NA_OFF_WF + sizeof(float) * KT * NFMAX);
constexpr size_t NA_OFF_TH = align256(NA_OFF_WA + sizeof(float) * NFMAX * KT_PAD);
constexpr size_t NA_OFF_IMG = align256(NA_OFF_TH + sizeof(float) * NFMAX);
constexpr size_t NA_OFF_ARR = align256(NA_OFF_IMG + sizeof(ImgDesc));
constexpr size_t NA_OFF_RES = align256(NA_OFF_ARR + sizeof(unsigned));
constexpr size_t NA_OFF_TILES = align256(NA_OFF_RES + 2 * sizeof(double));
constexpr size_t NA_OFF_PART = align256(NA_OFF_TILES + sizeof(TileDesc) * NA_MAX_TILES);
constexpr size_t NA_SCRATCH_BYTES = align256(NA_OFF_PART + sizeof(double) * NRED * NA_MAX_TILES);

static __device__ __align__(256) unsigned char fe_noalloc_scratch[NA_SCRATCH_BYTES];

constexpr int NA_MAX_DEV = 64;
std::mutex na_mu;
unsigned char *na_base[NA_MAX_DEV] = {};

// Weight tables in the layout the tile kernel reads (see KParams): forward
// taps flipped and tap-major, adjoint taps times 2 theta_i filter-major, zero
// beyond nf.
// Also writes the image and tile descriptors and clears the counters.
__global__ void na_setup_kernel(unsigned char *base, const float *filters, const float *theta, int nf,
                                int H, int W, int tiles_x, int ntiles, const float *u) {
    float *wf = reinterpret_cast<float *>(base + NA_OFF_WF);
    float *wa = reinterpret_cast<float *>(base + NA_OFF_WA);
    float *th = reinterpret_cast<float *>(base + NA_OFF_TH);
    TileDesc *tiles = reinterpret_cast<TileDesc *>(base + NA_OFF_TILES);
    const int T = fp32_tile_size;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < NA_MAX_TILES + KT * NFMAX;
         j += gridDim.x * blockDim.x) {
        if (j < KT * NFMAX) {
            const int t = j / NFMAX, i = j % NFMAX;
            wf[j] = i < nf ? filters[i * KT + (KT - 1 - t)] : 0.0f;
        }
        if (j < NFMAX * KT_PAD) {
            const int i = j / KT_PAD, t = j % KT_PAD;
            wa[j] = (i < nf && t < KT) ? 2.0f * theta[i] * filters[i * KT + t] : 0.0f;
        }
        if (j < NFMAX) th[j] = j < nf ? theta[j] : 0.0f;
        if (j < ntiles) tiles[j] = TileDesc{0, (j / tiles_x) * T, (j % tiles_x) * T, 0};
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ImgDesc d;
        d.H = H;
        d.W = W;
        d.tile_begin = 0;
        d.ntiles = ntiles;
        for (int k = 0; k < 3; ++k) d.u[k] = nullptr;
        for (int k = 0; k < 2; ++k) d.g[k] = nullptr;
        d.f2 = const_cast<float *>(u);  // G is not returned; any valid plane keeps its reads in bounds
        d.lambda = 1.0;
        d.lambda1 = 0.0;
        d.gscale = 0.5;
        d.tmap = nullptr;
        *reinterpret_cast<ImgDesc *>(base + NA_OFF_IMG) = d;
        *reinterpret_cast<unsigned *>(base + NA_OFF_ARR) = 0u;
        reinterpret_cast<double *>(base + NA_OFF_RES)[0] = 0.0;
        reinterpret_cast<double *>(base + NA_OFF_RES)[1] = 0.0;
    }
}

// Once per device, with that device current: the device address of the
// scratch array and the kernel's shared-memory opt-in.
fe_status na_device_base(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        set_global_error("fe_gradient_noalloc: no current CUDA device");
        return FE_ECUDA;
    }
    if (dev < 0 || dev >= NA_MAX_DEV) {
        set_global_error("fe_gradient_noalloc: device index out of range");
        return FE_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(na_mu);
    if (!na_base[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, fe_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_global_error("fe_gradient_noalloc: cudaGetSymbolAddress failed");
            return FE_ECUDA;
        }
        if (fp32_prepare() != cudaSuccess) {
            set_global_error("fe_gradient_noalloc: cudaFuncSetAttribute failed");
            return FE_ECUDA;
        }
        na_base[dev] = static_cast<unsigned char *>(p);
    }
    *out = na_base[dev];
    return FE_OK;
}

// After a failed launch (for example once cudaDeviceReset has torn down the
// context the set-up was made in) the current device's set-up is dropped, so
// that the next call resolves the array's address and the attribute again.
void na_forget_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEV) return;
    std::lock_guard<std::mutex> lock(na_mu);
    na_base[dev] = nullptr;
}

}  // namespace
}  // namespace fe

using namespace fe;

extern "C" fe_status fe_gradient_noalloc(const float *u, float *g, double *F, int H, int W,
                                         const float *filters, const float *theta, int nf,
                                         void *stream) {
    if (!u || !g || !filters || !theta) {
        set_global_error("fe_gradient_noalloc: u, g, filters and theta must be device pointers");
        return FE_EINVAL;
    }
    if (nf < 1 || nf > NFMAX) {
        set_global_error("fe_gradient_noalloc: nf must be in 1..64");
        return FE_EINVAL;
    }
    const int T = fp32_tile();
    if (H < 8 || W < 8 || H > 65536 || W > 65536) {
        set_global_error("fe_gradient_noalloc: H and W must be in 8..65536");
        return FE_EINVAL;
    }
    const long long tiles_x = (W + T - 1) / T, ntiles = tiles_x * ((H + T - 1) / T);
    if (ntiles > NA_MAX_TILES) {
        set_global_error("fe_gradient_noalloc: image needs more than 4096 tiles of 64x64 "
                         "(the size of the static scratch array), e.g. larger than 4096x4096");
        return FE_EINVAL;
    }
    unsigned char *base = nullptr;
    fe_status st = na_device_base(&base);
    if (st != FE_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    na_setup_kernel<<<16, 256, 0, s>>>(base, filters, theta, nf, H, W, (int)tiles_x, (int)ntiles, u);
    if (cudaGetLastError() != cudaSuccess) {
        na_forget_device();
        set_global_error("fe_gradient_noalloc: set-up kernel launch failed");
        return FE_ECUDA;
    }
    KParams kp{};
    kp.imgs = reinterpret_cast<const ImgDesc *>(base + NA_OFF_IMG);
    kp.st = nullptr;  // not read by the gradient mode
    kp.tiles = reinterpret_cast<const TileDesc *>(base + NA_OFF_TILES);
    kp.partials = reinterpret_cast<double *>(base + NA_OFF_PART);
    kp.img_arrivals = reinterpret_cast<unsigned *>(base + NA_OFF_ARR);
    kp.loop = nullptr;  // not read by the gradient mode
    kp.wf = reinterpret_cast<const float *>(base + NA_OFF_WF);
    kp.wa = reinterpret_cast<const float *>(base + NA_OFF_WA);
    kp.theta = reinterpret_cast<const float *>(base + NA_OFF_TH);
    kp.nfp = (nf + 7) / 8 * 8;
    kp.nimg = 1;
    kp.ntiles = (int)ntiles;
    kp.tile0 = 0;
    kp.u_ext = u;
    kp.g_ext = g;
    kp.results = reinterpret_cast<double *>(base + NA_OFF_RES);
    if (fp32_launch(MODE_GRAD_EXT, kp, (int)ntiles, s) != cudaSuccess) {
        na_forget_device();
        set_global_error("fe_gradient_noalloc: gradient kernel launch failed");
        return FE_ECUDA;
    }
    // results[0] is F; results[1] (the data term) is computed from the
    // stand-in f = u set up above, can be NaN for u <= 0, and is never returned
    if (F && cudaMemcpyAsync(F, base + NA_OFF_RES, sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        set_global_error("fe_gradient_noalloc: copy of F failed");
        return FE_ECUDA;
    }
    return FE_OK;
}
