// Host side of the libfe C ABI (include/fe.h): contexts, device memory,
// argument validation, and the device-driven iPiano loop.
//
// The loop over iterations never reads energies back to the host: every
// launch of the trial kernel either performs one trial per active image
// (accepted or rejected on the device) or exits at once for finished images.
// Two drivers are provided: a host loop that launches trial kernels in chunks
// and reads one integer (the active-image count) between chunks, and a CUDA
// graph whose while-node re-launches the trial kernel until the kernel's
// last CTA clears the condition.  Both are bounded by a device-side trial
// budget, so neither can spin forever.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fe_internal.cuh"

using namespace fe;

struct fe_ctx {
    int dev = 0;
    cudaStream_t s = nullptr;
    fe_params prm{};
    std::vector<float> filt, theta;
    int nimg = 0, ntiles = 0, nfp = 0;
    int tile_y = 0, tile_x = 0;  // output tile of the trial kernel (autotuned or given)
    int cluster = 1;             // CTAs per tile (FP32: 4 = a thread-block cluster per 32 x 32 tile)
    std::vector<int> H, W;
    std::vector<ImgDesc> himg;
    std::vector<TileDesc> htile;
    std::vector<void *> allocs;
    ImgDesc *d_imgs = nullptr;
    ImgState *d_st = nullptr;
    TileDesc *d_tiles = nullptr;
    int *d_order = nullptr;  // launch order of the tiles (whole-list launches)
    std::vector<int> horder;
    int *d_porder = nullptr;  // persistent launches: each image's tiles in the order they are taken
    std::vector<int> hporder;
    int *d_sched = nullptr;   // persistent launches: per-image tile counters
    double *d_part = nullptr;
    unsigned *d_arr = nullptr;
    LoopCtl *d_loop = nullptr;
    float *d_wf = nullptr, *d_wa = nullptr, *d_th = nullptr;
    double *d_res = nullptr;
    int *d_flag = nullptr;
    int *d_tc_error = nullptr;
    double *d_gpart = nullptr;  // partial sums of the data-term floor G(f)
    double *d_htarget = nullptr;  // per-image energy targets of fe_solve_to_energy
    unsigned char *d_tcw_fwd = nullptr, *d_tcw_adj = nullptr;
    CUtensorMap *d_tmaps = nullptr;  // tensor-core forms: 6 TMA maps per image (u0..2, g0..1, f2)
    float *d_scratch = nullptr;  // 2 planes of the largest image (host-pointer staging)
    size_t max_plane = 0;
    KParams kp{};
    long long host_launches = 0;
    std::string err;
    int loop_mode = 2;
    // CUDA graphs of the device loop: [0] a while node around per-trial
    // launches, [1] the persistent trial launch
    bool graph_built[2] = {false, false};
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
};

namespace {

fe_status set_err(fe_ctx *c, fe_status s, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

thread_local std::string g_init_err;

#define FE_CUDA(c, call)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return set_err((c), FE_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                           __FILE__, __LINE__);                                            \
    } while (0)

// f^2 and the initial iterate: u^0 (variant model) or w^0 = log u^0
// (combined model, logw != 0); u^{-1} = u^0.
__global__ void prep_kernel(const float *f, const float *u0, float *f2, float *ua, float *ub,
                            size_t N, int logw, int *bad) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
         i += (size_t)gridDim.x * blockDim.x) {
        const float fv = f[i];
        const float f2v = fv * fv;
        const float uv = u0 ? u0[i] : fv;
        const bool ok = fv > 0.0f && isfinite(fv) && f2v > 0.0f && isfinite(f2v) && uv > 0.0f &&
                        isfinite(uv);
        const float xv = logw ? logf(uv) : uv;
        f2[i] = f2v;
        ua[i] = xv;
        ub[i] = xv;
        if (!ok) atomicOr(bad, 1);
    }
}

// u = e^w (combined model: the iterate is w)
__global__ void exp_kernel(const float *w, float *u, size_t N) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
        u[i] = expf(w[i]);
}

// Per-block partial sums of the minimum of the data term (the floor of the
// convergence test), GF_BLOCKS partials per image, summed on the host in
// block order.  Variant: (lambda/2) f^2 (1 - log f^2), the value at u = f.
// Combined: lambda1/2 (2 log f + 1) + lambda2/2 (f^2 - 2 f^2 log f), the value
// at w = log f, where g'(w) = 0.
constexpr int GF_BLOCKS = 64;
__global__ void gfloor_kernel(const float *f2, size_t N, int model, double lam, double lam1, double *part) {
    __shared__ double red[256];
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const double v = (double)f2[i];
        if (model == FE_MODEL_COMBINED) {
            const double lf = 0.5 * log(v);
            s += 0.5 * lam1 * (2.0 * lf + 1.0) + 0.5 * lam * (v - 2.0 * v * lf);
        } else {
            s += 0.5 * lam * v * (1.0 - log(v));
        }
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Start of fe_step / fe_solve: per-image targets, the trial budget (per
// launch for per-trial launches, per image for the persistent launch) and
// the persistent launch's tile counters (0: the first trial's tiles are
// available; images that do not iterate never offer tiles).
__global__ void begin_kernel(ImgState *st, int nimg, long long n, double tol, LoopCtl *lc,
                             long long budget, const double *H_target, int *sched) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int nact = 0;
    for (int j = 0; j < nimg; ++j) {
        st[j].H_target = H_target ? H_target[j] : -INFINITY;
        bool act = false;
        if (st[j].status == FE_OK) {
            st[j].done = 0;
            st[j].converged = 0;
            st[j].bt = 0;
            st[j].target = st[j].n + n;
            st[j].tol = tol;
            st[j].trial_limit = st[j].trials + budget;
            act = n > 0;
        } else {
            st[j].done = 1;
        }
        nact += act;
        sched[j] = act ? 0 : 0x40000000;
    }
    lc->grid_arrivals = 0u;
    lc->active = nact;
    lc->budget = budget;
    lc->abort = 0;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
fe_status dalloc(fe_ctx *c, T **p, size_t count) {
    void *q = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, FE_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    c->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return FE_OK;
}

fe_status validate_params(fe_ctx *c, const fe_params *p) {
    if (!p) return set_err(c, FE_EINVAL, "params is NULL");
    if (p->nf < 1 || p->nf > NFMAX) return set_err(c, FE_EINVAL, "nf=%d outside 1..%d", p->nf, NFMAX);
    if (p->ksize != KS) return set_err(c, FE_EINVAL, "ksize=%d, only 7 is supported", p->ksize);
    if (!p->filters || !p->theta) return set_err(c, FE_EINVAL, "filters or theta is NULL");
    for (int i = 0; i < p->nf * KT; ++i)
        if (!std::isfinite(p->filters[i])) return set_err(c, FE_EINVAL, "filter weight %d not finite", i);
    for (int i = 0; i < p->nf; ++i)
        if (!(p->theta[i] >= 0.0f) || !std::isfinite(p->theta[i]))
            return set_err(c, FE_EINVAL, "theta[%d] must be finite and >= 0", i);
    if (p->model != FE_MODEL_VARIANT && p->model != FE_MODEL_COMBINED)
        return set_err(c, FE_EINVAL, "unknown model %d", p->model);
    if (p->model == FE_MODEL_VARIANT) {
        if (!(p->lambda > 0.0) || !std::isfinite(p->lambda)) return set_err(c, FE_EINVAL, "lambda must be > 0");
    } else {
        if (!(p->lambda >= 0.0) || !std::isfinite(p->lambda) || !(p->lambda1 >= 0.0) || !std::isfinite(p->lambda1) ||
            !(p->lambda + p->lambda1 > 0.0))
            return set_err(c, FE_EINVAL, "combined model: lambda, lambda1 must be finite, >= 0, not both 0");
    }
    if (!(p->beta >= 0.0 && p->beta < 1.0)) return set_err(c, FE_EINVAL, "beta must be in [0,1)");
    if (!(p->L0 > 0.0) || !std::isfinite(p->L0)) return set_err(c, FE_EINVAL, "L0 must be > 0");
    if (!(p->eta > 1.0) || !std::isfinite(p->eta)) return set_err(c, FE_EINVAL, "eta must be > 1");
    if (!(p->c2 >= 0.0) || !std::isfinite(p->c2)) return set_err(c, FE_EINVAL, "c2 must be >= 0");
    if (p->max_backtrack < 0) return set_err(c, FE_EINVAL, "max_backtrack must be >= 0");
    if (p->prec != FE_FP32 && p->prec != FE_TF32 && p->prec != FE_BF16 && p->prec != FE_BF16R)
        return set_err(c, FE_EINVAL, "unknown precision %d", p->prec);
    if (p->prec != FE_FP32 && p->nf > 48)
        return set_err(c, FE_EUNSUPPORTED, "the tensor-core forms take at most 48 filters (nf=%d)", p->nf);
    if (p->prec == FE_FP32 && p->tile != 0 && !fp32_tile_supported(p->tile) && p->tile != (32 | FE_TILE_CLUSTER4) &&
        p->tile != (64 | FE_TILE_CLUSTER4))
        return set_err(c, FE_EUNSUPPORTED, "FP32 tile %d: use 0 (autotune), 32, 64, 32 | FE_TILE_CLUSTER4 or 64 | FE_TILE_CLUSTER4",
                       p->tile);
    if (p->prec != FE_FP32 && p->tile != 0)
        return set_err(c, FE_EUNSUPPORTED, "the tensor-core forms have one tile shape: tile must be 0");
    return FE_OK;
}

// cuTensorMapEncodeTiled from the driver, through the runtime's entry-point
// query (the library links only the runtime); NULL when unavailable, in which
// case the trial kernels read their inputs with plain loads.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *q = nullptr;
        cudaDriverEntryPointQueryResult r;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000, cudaEnableDefault, &r) ==
                cudaSuccess &&
            r == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(q);
        else
            cudaGetLastError();
    });
    return fn;
}

// TMA maps of every plane of every image whose row pitch is a multiple of 16
// bytes (W % 4 == 0): FP32 elements, dims {W, H}, box {tc_box_x, tc_box_y},
// zero fill outside the plane.  Other images keep tmap = NULL (plain loads).
fe_status build_tensor_maps(fe_ctx *c) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return FE_OK;
    std::vector<CUtensorMap> maps((size_t)c->nimg * 6);
    std::vector<int> ok(c->nimg, 0);
    for (int j = 0; j < c->nimg; ++j) {
        const ImgDesc &d = c->himg[j];
        if (d.W % 4 != 0) continue;
        float *planes[6] = {d.u[0], d.u[1], d.u[2], d.g[0], d.g[1], d.f2};
        bool good = true;
        for (int k = 0; k < 6 && good; ++k) {
            const cuuint64_t dims[2] = {(cuuint64_t)d.W, (cuuint64_t)d.H};
            const cuuint64_t strides[1] = {(cuuint64_t)d.W * 4};
            const cuuint32_t box[2] = {(cuuint32_t)tc_box_x, (cuuint32_t)tc_box_y};
            const cuuint32_t es[2] = {1, 1};
            good = enc(&maps[(size_t)j * 6 + k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, planes[k], dims, strides, box,
                       es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        }
        ok[j] = good;
    }
    fe_status st = dalloc(c, &c->d_tmaps, maps.size());
    if (st != FE_OK) return st;
    FE_CUDA(c, cudaMemcpy(c->d_tmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    for (int j = 0; j < c->nimg; ++j) c->himg[j].tmap = ok[j] ? c->d_tmaps + (size_t)j * 6 : nullptr;
    return FE_OK;
}

// Tensor-core kernel format of a precision form: 1 = BF16, 2 = TF32, 3 = BF16
// with r carried as a single BF16 operand.
int tc_format(int prec) { return prec == FE_BF16 ? 1 : (prec == FE_BF16R ? 3 : 2); }

// Launch one tile kernel of the context's precision form.
cudaError_t launch_tiles(const fe_ctx *c, int mode, const KParams &kp, int grid) {
    if (c->prm.prec == FE_FP32) return fp32_launch(mode, kp, grid, c->s, c->tile_y, c->prm.model, c->cluster);
    return tc_launch(mode, tc_format(c->prm.prec), kp, grid, c->s, c->prm.model);
}

// Tile origins and owned extents along one axis of length N with tile T.
// FP32: origins 0, T, 2T, ... (the last tile may hang over the border).
// Tensor-core forms: the last origin is moved back to N - T (when N >= T)
// so that it ends at the border and owns all its rows; the tile before it
// owns only the rows up to that origin.  The first tile always owns the
// first 3 rows: their mirror images (rows -3..-1) lie in its halo only.
// Outputs: origin o_i, owned start relative to the origin rel_i, owned
// length own_i (tile i owns [o_i + rel_i, o_i + rel_i + own_i)).
void axis_tiles(bool tc, int N, int T, std::vector<int> &o, std::vector<int> &rel, std::vector<int> &own) {
    const int n = (N + T - 1) / T;
    std::vector<int> s;
    o.clear();
    rel.clear();
    own.clear();
    for (int i = 0; i < n; ++i) o.push_back(i * T);
    if (tc && n > 1) o[n - 1] = N - T;
    for (int i = 0; i < n; ++i) s.push_back(i == 0 ? 0 : (tc && i == n - 1 ? std::max(o[i], 3) : o[i]));
    for (int i = 0; i < n; ++i) {
        own.push_back((i + 1 < n ? s[i + 1] : N) - s[i]);
        rel.push_back(s[i] - o[i]);
    }
}

// The tile list of every image for a TY x TX tile (host copy only); cl CTAs
// work on each tile.
void build_tiles(fe_ctx *c, int TY, int TX, int cl = 1) {
    const bool tc = c->prm.prec != FE_FP32;
    c->htile.clear();
    for (int j = 0; j < c->nimg; ++j) {
        std::vector<int> oy, ry, ohv, ox, rx, owv;
        axis_tiles(tc, c->H[j], TY, oy, ry, ohv);
        axis_tiles(tc, c->W[j], TX, ox, rx, owv);
        ImgDesc &d = c->himg[j];
        d.tile_begin = (int)c->htile.size();
        d.ntiles = (int)(oy.size() * ox.size());
        for (size_t a = 0; a < oy.size(); ++a)
            for (size_t b = 0; b < ox.size(); ++b)
                c->htile.push_back(TileDesc{j, oy[a], ox[b], ohv[a], owv[b], ry[a], rx[b], 0});
    }
    c->ntiles = (int)c->htile.size();
    c->tile_y = TY;
    c->tile_x = TX;
    c->cluster = cl;
    // launch order of the FP32 64 x 64 tiles: tiles with more image borders
    // first (their frame work makes them the longest), so that the last wave
    // of a launch holds the shortest tiles; ties keep the list order
    // (measured +0.9 % on 24 x 512^2 + 24 x 256^2; the split 32 x 32 tiles
    // on small batches run faster in list order, -2.5 % ordered)
    auto sides = [&](const TileDesc &t) {
        const int H = c->H[t.img], W = c->W[t.img];
        return (t.y0 == 0) + (t.x0 == 0) + (t.y0 + TY > H - 3) + (t.x0 + TX > W - 3);
    };
    c->horder.resize(c->ntiles);
    for (int k = 0; k < c->ntiles; ++k) c->horder[k] = k;
    if (!tc && TY == 64 && cl == 1)
        std::stable_sort(c->horder.begin(), c->horder.end(),
                         [&](int a, int b) { return sides(c->htile[a]) > sides(c->htile[b]); });
    // persistent launches take an image's tiles in the same longest-first
    // order, per image (the order the tiles of one trial become available)
    c->hporder.resize(c->ntiles);
    for (int k = 0; k < c->ntiles; ++k) c->hporder[k] = k;
    for (int j = 0; j < c->nimg; ++j) {
        auto b = c->hporder.begin() + c->himg[j].tile_begin;
        std::stable_sort(b, b + c->himg[j].ntiles,
                         [&](int a, int bb) { return sides(c->htile[a]) > sides(c->htile[bb]); });
    }
}

// FP32 tile candidates: code = T, or T | FE_TILE_CLUSTER4
void build_tiles_code(fe_ctx *c, int code) {
    const int T = code & 0xff;
    build_tiles(c, T, T, (code & FE_TILE_CLUSTER4) ? 4 : 1);
}

size_t count_tiles(const fe_ctx *c, int TY, int TX) {
    size_t n = 0;
    for (int j = 0; j < c->nimg; ++j) n += (size_t)((c->H[j] + TY - 1) / TY) * ((c->W[j] + TX - 1) / TX);
    return n;
}

fe_status upload_tiles(fe_ctx *c) {
    FE_CUDA(c, cudaMemcpyAsync(c->d_imgs, c->himg.data(), sizeof(ImgDesc) * c->nimg, cudaMemcpyHostToDevice, c->s));
    FE_CUDA(c, cudaMemcpyAsync(c->d_tiles, c->htile.data(), sizeof(TileDesc) * c->ntiles, cudaMemcpyHostToDevice,
                               c->s));
    FE_CUDA(c, cudaMemcpyAsync(c->d_order, c->horder.data(), sizeof(int) * c->ntiles, cudaMemcpyHostToDevice, c->s));
    FE_CUDA(c, cudaMemcpyAsync(c->d_porder, c->hporder.data(), sizeof(int) * c->ntiles, cudaMemcpyHostToDevice,
                               c->s));
    c->kp.ntiles = c->ntiles;
    return FE_OK;
}

fe_status load_inputs(fe_ctx *c, const float *const *f, const float *const *u0) {
    if (!f) return set_err(c, FE_EINVAL, "f is NULL");
    FE_CUDA(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->s));
    for (int j = 0; j < c->nimg; ++j) {
        if (!f[j]) return set_err(c, FE_EINVAL, "f[%d] is NULL", j);
        const size_t N = (size_t)c->H[j] * c->W[j];
        ImgDesc &im = c->himg[j];
        // stage f in u[1] and u0 in u[0]; the prep kernel squares f, checks
        // positivity and writes u^0 into u[0] and u[2] (u^{-1} = u^0)
        FE_CUDA(c, cudaMemcpyAsync(im.u[1], f[j], N * 4, cudaMemcpyDefault, c->s));
        const bool has_u0 = u0 && u0[j];
        if (has_u0) FE_CUDA(c, cudaMemcpyAsync(im.u[0], u0[j], N * 4, cudaMemcpyDefault, c->s));
        const int blocks = (int)std::min<size_t>((N + 255) / 256, 4096);
        prep_kernel<<<blocks, 256, 0, c->s>>>(im.u[1], has_u0 ? im.u[0] : nullptr, im.f2, im.u[0], im.u[2],
                                              N, c->prm.model == FE_MODEL_COMBINED ? 1 : 0, c->d_flag);
        FE_CUDA(c, cudaGetLastError());
        ++c->host_launches;
    }
    int bad = 0;
    FE_CUDA(c, cudaMemcpyAsync(&bad, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    FE_CUDA(c, cudaStreamSynchronize(c->s));
    if (bad) return set_err(c, FE_EINVAL, "f and u0 must be finite and > 0 (f^2 must not underflow)");
    // floor of the data term, G(f), for the convergence test
    for (int j = 0; j < c->nimg; ++j) {
        gfloor_kernel<<<GF_BLOCKS, 256, 0, c->s>>>(c->himg[j].f2, (size_t)c->H[j] * c->W[j], c->prm.model,
                                                   c->prm.lambda, c->prm.lambda1,
                                                   c->d_gpart + (size_t)j * GF_BLOCKS);
        FE_CUDA(c, cudaGetLastError());
        ++c->host_launches;
    }
    std::vector<double> gp((size_t)c->nimg * GF_BLOCKS);
    FE_CUDA(c, cudaMemcpyAsync(gp.data(), c->d_gpart, sizeof(double) * gp.size(), cudaMemcpyDeviceToHost, c->s));
    FE_CUDA(c, cudaStreamSynchronize(c->s));
    // fresh state, then grad F(u^0), F(u^0), G(u^0) on the device
    std::vector<ImgState> hs(c->nimg);
    for (int j = 0; j < c->nimg; ++j) {
        ImgState &s = hs[j];
        std::memset(&s, 0, sizeof s);
        s.L = c->prm.L0;
        s.alpha = 2.0 * (1.0 - c->prm.beta) / (c->prm.L0 + 2.0 * c->prm.c2);
        s.status = FE_OK;
        double g = 0.0;
        for (int k = 0; k < GF_BLOCKS; ++k) g += gp[(size_t)j * GF_BLOCKS + k];
        s.Gf = g;
    }
    FE_CUDA(c, cudaMemcpyAsync(c->d_st, hs.data(), sizeof(ImgState) * hs.size(), cudaMemcpyHostToDevice, c->s));
    FE_CUDA(c, cudaMemsetAsync(c->d_arr, 0, sizeof(unsigned) * c->nimg, c->s));
    KParams kp = c->kp;
    kp.tile0 = 0;
    FE_CUDA(c, launch_tiles(c, MODE_INIT, kp, c->ntiles));
    ++c->host_launches;
    FE_CUDA(c, cudaMemcpyAsync(hs.data(), c->d_st, sizeof(ImgState) * hs.size(), cudaMemcpyDeviceToHost, c->s));
    FE_CUDA(c, cudaStreamSynchronize(c->s));
    for (int j = 0; j < c->nimg; ++j)
        if (hs[j].status != FE_OK) return set_err(c, (fe_status)hs[j].status, "image %d: non-finite energy at u^0", j);
    return FE_OK;
}

// Whether this context's trial kernel can run as one persistent launch: the
// tiles that one CTA works on alone (not the thread-block cluster tiles).
bool persist_supported(const fe_ctx *c) { return c->prm.prec != FE_FP32 || c->cluster == 1; }

// CUDA graph of the device loop: a while node whose body is one trial kernel
// node.  Per-trial launches (persist false): one launch per trial of every
// image, the last CTA sets the while condition.  Persistent (persist true):
// the body is one launch of as many CTAs as fit on the GPU at once (at most
// one per tile), which runs every trial of every image and ends the loop.
// Kernel, block size, shared memory and grid of a trial launch: per-trial
// (every tile, times the cluster size) or persistent.
fe_status trial_config(fe_ctx *c, bool persist, const void **fn_out, int *threads_out, size_t *smem_out,
                       int *grid_out) {
    const int fmt = tc_format(c->prm.prec);
    const bool tc = c->prm.prec != FE_FP32;
    const void *fn = persist ? (tc ? tc_ptrial_entry(fmt, c->prm.model) : fp32_ptrial_entry(c->tile_y, c->prm.model))
                             : (tc ? tc_trial_entry(fmt, c->prm.model)
                                   : fp32_trial_entry(c->tile_y, c->prm.model, c->cluster));
    const int threads = tc ? tc_threads() : fp32_threads(c->tile_y);
    const size_t smem = tc ? tc_smem_bytes(fmt) : fp32_smem_bytes(c->tile_y);
    int grid = c->ntiles * (tc ? 1 : c->cluster);
    if (persist) {
        // CTAs per SM: the residency the kernel is built for (its launch
        // bounds and shared memory; the occupancy calculator was measured to
        // report 1 for the tensor-core kernel, which runs 3 per SM), or the
        // calculator's figure if higher.  A CTA that finds no room waits to
        // be scheduled; it holds no tile meanwhile, so no other CTA waits on it.
        int per_sm = 0, sms = 0;
        FE_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
        FE_CUDA(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
        per_sm = std::max(per_sm, tc ? tc_ctas_per_sm(fmt) : fp32_ctas_per_sm(c->tile_y));
        grid = std::max(1, std::min(c->ntiles, per_sm * sms));
    }
    *fn_out = fn;
    *threads_out = threads;
    *smem_out = smem;
    *grid_out = grid;
    return FE_OK;
}

fe_status build_graph(fe_ctx *c, bool persist) {
    const int gi = persist ? 1 : 0;
    if (c->graph_built[gi]) return FE_OK;
    const bool tc = c->prm.prec != FE_FP32;
    const void *fn = nullptr;
    int threads = 0, grid = 0;
    size_t smem = 0;
    fe_status cst = trial_config(c, persist, &fn, &threads, &smem, &grid);
    if (cst != FE_OK) return cst;
    cudaGraph_t g = nullptr;
    FE_CUDA(c, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return set_err(c, FE_EUNSUPPORTED, "conditional graph nodes unavailable: %s", cudaGetErrorString(e));
    }
    // cudaGraphNodeParams has no default constructor in C++ (union member);
    // build it zero-filled in raw storage
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    std::memset(raw, 0, sizeof raw);
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cn;
    e = cudaGraphAddNode(&cn, g, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return set_err(c, FE_EUNSUPPORTED, "cudaGraphAddNode(while): %s", cudaGetErrorString(e));
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    KParams kp = c->kp;
    kp.tile0 = 0;
    kp.cond = (unsigned long long)h;
    kp.use_cond = 1;
    void *args[] = {&kp};
    cudaKernelNodeParams knp;
    std::memset(&knp, 0, sizeof knp);
    knp.func = const_cast<void *>(fn);
    knp.gridDim = dim3((unsigned)grid);
    knp.blockDim = dim3((unsigned)threads);
    knp.sharedMemBytes = (unsigned)smem;
    knp.kernelParams = args;
    cudaGraphNode_t kn;
    e = cudaGraphAddKernelNode(&kn, body, nullptr, 0, &knp);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return set_err(c, FE_ECUDA, "cudaGraphAddKernelNode: %s", cudaGetErrorString(e));
    }
    if (!tc && c->cluster > 1) {  // thread-block clusters of c->cluster CTAs
        cudaKernelNodeAttrValue v;
        std::memset(&v, 0, sizeof v);
        v.clusterDim.x = (unsigned)c->cluster;
        v.clusterDim.y = 1;
        v.clusterDim.z = 1;
        e = cudaGraphKernelNodeSetAttribute(kn, cudaKernelNodeAttributeClusterDimension, &v);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return set_err(c, FE_ECUDA, "cluster dimension of the graph node: %s", cudaGetErrorString(e));
        }
    }
    cudaGraphExec_t ex;
    e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return set_err(c, FE_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
    c->graph[gi] = g;
    c->gexec[gi] = ex;
    c->graph_built[gi] = true;
    return FE_OK;
}

// After a persistent launch (synchronised): a launch that stopped because no
// trial was decided for PERSIST_STALL_NS is reported.
fe_status check_persist(fe_ctx *c) {
    LoopCtl lc;
    FE_CUDA(c, cudaMemcpy(&lc, c->d_loop, sizeof lc, cudaMemcpyDeviceToHost));
    if (lc.abort)
        set_err(c, FE_ETIMEOUT, "persistent launch stopped: no trial was decided for %.0f s",
                1e-9 * (double)PERSIST_STALL_NS);
    return FE_OK;
}

// Run trial launches until no image is active (or the budget is spent).
// Loop mode 2 runs the persistent launch in a CUDA graph where the tile
// allows it (else as mode 1), mode 3 the same launch without a graph (else
// as mode 0), mode 1 the graph of per-trial launches, mode 0 (or a driver
// without conditional graph nodes) host-side chunks of per-trial launches.
fe_status run_loop(fe_ctx *c, long long n_hint, long long budget, bool sync) {
    if (c->loop_mode == 3 && persist_supported(c)) {
        const void *fn = nullptr;
        int threads = 0, grid = 0;
        size_t smem = 0;
        fe_status st = trial_config(c, true, &fn, &threads, &smem, &grid);
        if (st != FE_OK) return st;
        KParams kp = c->kp;
        kp.tile0 = 0;
        kp.use_cond = 0;
        void *args[] = {&kp};
        FE_CUDA(c, cudaLaunchKernel(fn, dim3((unsigned)grid), dim3((unsigned)threads), args, smem, c->s));
        if (sync) {
            FE_CUDA(c, cudaStreamSynchronize(c->s));
            return check_persist(c);
        }
        return FE_OK;
    }
    if (c->loop_mode == 1 || c->loop_mode == 2) {
        const bool persist = c->loop_mode == 2 && persist_supported(c);
        fe_status st = build_graph(c, persist);
        if (st == FE_OK) {
            FE_CUDA(c, cudaGraphLaunch(c->gexec[persist ? 1 : 0], c->s));
            if (sync) {
                FE_CUDA(c, cudaStreamSynchronize(c->s));
                if (persist) return check_persist(c);
            }
            return FE_OK;
        }
        if (st != FE_EUNSUPPORTED) return st;
        c->loop_mode = 0;  // fall back to the chunked host loop of the same kernel
    }
    KParams kp = c->kp;
    kp.tile0 = 0;
    long long launched = 0;
    long long chunk = std::max<long long>(1, std::min<long long>(n_hint, 64));
    for (;;) {
        const long long todo = std::min(chunk, budget - launched);
        for (long long k = 0; k < todo; ++k) FE_CUDA(c, launch_tiles(c, MODE_TRIAL, kp, c->ntiles));
        launched += todo;
        LoopCtl lc;
        FE_CUDA(c, cudaMemcpyAsync(&lc, c->d_loop, sizeof lc, cudaMemcpyDeviceToHost, c->s));
        FE_CUDA(c, cudaStreamSynchronize(c->s));
        if (lc.active == 0 || launched >= budget) break;
        chunk = 16;
    }
    return FE_OK;
}

fe_status fetch_states(fe_ctx *c, std::vector<ImgState> &hs) {
    hs.resize(c->nimg);
    FE_CUDA(c, cudaMemcpyAsync(hs.data(), c->d_st, sizeof(ImgState) * c->nimg, cudaMemcpyDeviceToHost, c->s));
    FE_CUDA(c, cudaStreamSynchronize(c->s));
    return FE_OK;
}

fe_status check_img(fe_ctx *c, int img) {
    if (!c) return FE_EINVAL;
    if (img < 0 || img >= c->nimg) return set_err(c, FE_EINVAL, "image index %d outside 0..%d", img, c->nimg - 1);
    return FE_OK;
}

// Stage a caller pointer for reading by a kernel: device pointers are used
// directly, host pointers are copied into scratch plane `slot`.
fe_status stage_in(fe_ctx *c, const float *src, size_t N, int slot, const float **out) {
    if (is_device_ptr(src)) {
        *out = src;
        return FE_OK;
    }
    float *dst = c->d_scratch + (size_t)slot * c->max_plane;
    FE_CUDA(c, cudaMemcpyAsync(dst, src, N * 4, cudaMemcpyDefault, c->s));
    *out = dst;
    return FE_OK;
}

// Tile autotuner (FP32 form).  The choice depends on the image sizes: a
// batch with too few 64 x 64 tiles to fill 152 SMs x 2 CTAs runs faster
// with 32 x 32 tiles despite their larger recomputed halo.  Each candidate
// is timed on this context's own images with the initial-gradient kernel
// (forward bank, potential, adjoint bank and sums on every tile: the cost of
// a trial without the pointwise prox), which is idempotent, so timing it
// changes no state.  One warm-up launch, then the median of three
// CUDA-event timings.  The choice is cached per device and list of image
// sizes for the life of the process.
fe_status autotune_tile(fe_ctx *c, const std::vector<int> &cand) {
    static std::mutex mu;
    static std::map<std::string, int> cache;
    std::string key = std::to_string(c->dev) + ":" + std::to_string(c->nfp) + ":" + std::to_string(c->prm.model);
    for (int j = 0; j < c->nimg; ++j) key += ":" + std::to_string(c->H[j]) + "x" + std::to_string(c->W[j]);
    int best = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) best = it->second;
    }
    if (best == 0) {
        cudaEvent_t e0, e1;
        FE_CUDA(c, cudaEventCreate(&e0));
        if (cudaEventCreate(&e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            return set_err(c, FE_ECUDA, "cudaEventCreate failed");
        }
        float best_ms = 0.f;
        fe_status st = FE_OK;
        for (int T : cand) {
            build_tiles_code(c, T);
            if ((st = upload_tiles(c)) != FE_OK) break;
            KParams kp = c->kp;
            kp.tile0 = 0;
            float ms[3];
            cudaError_t e = launch_tiles(c, MODE_INIT, kp, c->ntiles);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
                if ((e = cudaEventRecord(e0, c->s)) != cudaSuccess) break;
                if ((e = launch_tiles(c, MODE_INIT, kp, c->ntiles)) != cudaSuccess) break;
                if ((e = cudaEventRecord(e1, c->s)) != cudaSuccess) break;
                if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
                e = cudaEventElapsedTime(&ms[r], e0, e1);
            }
            c->host_launches += 4;
            if (e != cudaSuccess) {
                st = set_err(c, FE_ECUDA, "tile autotune (T=%d): %s", T, cudaGetErrorString(e));
                break;
            }
            std::sort(ms, ms + 3);
            if (best == 0 || ms[1] < best_ms) {
                best = T;
                best_ms = ms[1];
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st != FE_OK) return st;
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = best;
    }
    build_tiles_code(c, best);
    return upload_tiles(c);
}

}  // namespace

void fe::set_global_error(const char *msg) { g_init_err = msg ? msg : ""; }

extern "C" {

int fe_abi_version(void) { return FE_ABI_VERSION; }

const char *fe_status_string(fe_status s) {
    switch (s) {
        case FE_OK: return "ok";
        case FE_EINVAL: return "invalid argument";
        case FE_ENOMEM: return "out of device memory";
        case FE_ECUDA: return "CUDA error";
        case FE_ENONFINITE: return "non-finite value in a trial";
        case FE_EBACKTRACK: return "backtracking limit reached";
        case FE_ETIMEOUT: return "device trial budget exhausted";
        case FE_ENOTCONVERGED: return "not converged within max_iter";
        case FE_EUNSUPPORTED: return "unsupported option";
    }
    return "unknown status";
}

const char *fe_last_error(const fe_ctx *ctx) { return ctx ? ctx->err.c_str() : g_init_err.c_str(); }

void fe_default_params(fe_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->ksize = KS;
    p->lambda = 5.0;
    p->beta = 0.8;
    p->L0 = 1.0;
    p->eta = 2.0;
    p->c2 = 1e-6;
    p->max_backtrack = 30;
    p->prec = FE_FP32;
    p->tile = 0;
    p->model = FE_MODEL_VARIANT;
    p->lambda1 = 0.0;
}

void fe_destroy(fe_ctx *c) {
    if (!c) return;
    if (c->s) cudaStreamSynchronize(c->s);
    for (int k = 0; k < 2; ++k) {
        if (c->gexec[k]) cudaGraphExecDestroy(c->gexec[k]);
        if (c->graph[k]) cudaGraphDestroy(c->graph[k]);
    }
    for (void *p : c->allocs) cudaFree(p);
    delete c;
}

fe_status fe_init_batch(fe_ctx **out, const fe_params *p, int nimg, const int *H, const int *W,
                        const float *const *f, const float *const *u0, void *stream) {
    g_init_err.clear();
    if (!out) return FE_EINVAL;
    *out = nullptr;
    fe_ctx *c = new fe_ctx();
    auto bail = [&](fe_status s) {
        g_init_err = c->err;
        fe_destroy(c);
        return s;
    };
    fe_status st = validate_params(c, p);
    if (st != FE_OK) return bail(st);
    if (nimg < 1 || !H || !W || !f) return bail(set_err(c, FE_EINVAL, "need nimg >= 1 and non-NULL H, W, f"));
    c->prm = *p;
    c->nimg = nimg;
    c->s = static_cast<cudaStream_t>(stream);
    c->filt.assign(p->filters, p->filters + (size_t)p->nf * KT);
    c->theta.assign(p->theta, p->theta + p->nf);
    c->nfp = ((p->nf + 7) / 8) * 8;
    const bool tc = p->prec != FE_FP32;
    size_t plane_total = 0;
    for (int j = 0; j < nimg; ++j) {
        if (H[j] < 8 || W[j] < 8 || H[j] > 65536 || W[j] > 65536)
            return bail(set_err(c, FE_EINVAL, "image %d: size %dx%d outside 8..65536", j, H[j], W[j]));
        c->H.push_back(H[j]);
        c->W.push_back(W[j]);
        const size_t N = (size_t)H[j] * W[j];
        c->max_plane = std::max(c->max_plane, (N + 63) / 64 * 64);
        plane_total += 6 * ((N + 63) / 64 * 64);
        ImgDesc d{};
        d.H = H[j];
        d.W = W[j];
        d.lambda = p->lambda;
        d.lambda1 = p->model == FE_MODEL_COMBINED ? p->lambda1 : 0.0;
        d.gscale = p->model == FE_MODEL_COMBINED ? 1.0 : 0.5 * p->lambda;
        c->himg.push_back(d);
    }
    // candidate tile shapes: the tensor-core forms have one; FP32 has 64 and
    // 32, each also split over a 4-CTA cluster (autotuned when p->tile == 0)
    std::vector<int> cand;
    if (tc)
        cand.push_back(0);
    else if (p->tile != 0)
        cand.push_back(p->tile);
    else
        cand = {64, 32, 32 | FE_TILE_CLUSTER4, 64 | FE_TILE_CLUSTER4};
    size_t max_tiles = 0;
    for (int T : cand)
        max_tiles = std::max(max_tiles, tc ? count_tiles(c, tc_tile_y, tc_tile_x) : count_tiles(c, T & 0xff, T & 0xff));
    if (max_tiles > (size_t)0x7fffffff) return bail(set_err(c, FE_EINVAL, "too many tiles"));
    if (tc)
        build_tiles(c, tc_tile_y, tc_tile_x);
    else
        build_tiles_code(c, cand[0]);
    if (cudaGetDevice(&c->dev) != cudaSuccess) return bail(set_err(c, FE_ECUDA, "no CUDA device"));

    if (cudaError_t e = tc ? tc_prepare() : fp32_prepare(); e != cudaSuccess)
        return bail(set_err(c, FE_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e)));

    float *planes = nullptr;
    if ((st = dalloc(c, &planes, plane_total)) != FE_OK) return bail(st);
    size_t off = 0;
    for (int j = 0; j < nimg; ++j) {
        const size_t N = (size_t)H[j] * W[j], P = (N + 63) / 64 * 64;
        ImgDesc &d = c->himg[j];
        for (int k = 0; k < 3; ++k) d.u[k] = planes + off + k * P;
        for (int k = 0; k < 2; ++k) d.g[k] = planes + off + (3 + k) * P;
        d.f2 = planes + off + 5 * P;
        off += 6 * P;
    }
    if ((st = dalloc(c, &c->d_imgs, nimg)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_st, nimg)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_tiles, max_tiles)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_order, max_tiles)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_porder, max_tiles)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_sched, nimg)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_part, max_tiles * NRED)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_arr, nimg)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_loop, 1)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_wf, (size_t)KT * NFMAX)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_wa, (size_t)NFMAX * KT_PAD)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_th, NFMAX)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_res, 2 * (size_t)nimg)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_flag, 4)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_tc_error, 1)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_gpart, (size_t)nimg * GF_BLOCKS)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_htarget, (size_t)nimg)) != FE_OK) return bail(st);
    if ((st = dalloc(c, &c->d_scratch, 2 * c->max_plane)) != FE_OK) return bail(st);
    if (tc) {
        std::vector<unsigned char> bf, ba;
        tc_build_weights(tc_format(p->prec), p->filters, p->nf, bf, ba);
        if ((st = dalloc(c, &c->d_tcw_fwd, bf.size())) != FE_OK) return bail(st);
        if ((st = dalloc(c, &c->d_tcw_adj, ba.size())) != FE_OK) return bail(st);
        if (cudaMemcpy(c->d_tcw_fwd, bf.data(), bf.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c->d_tcw_adj, ba.data(), ba.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(set_err(c, FE_ECUDA, "upload of the rounded filter bank failed"));
    }
    if (cudaMemset(c->d_tc_error, 0, sizeof(int)) != cudaSuccess)
        return bail(set_err(c, FE_ECUDA, "cudaMemset failed"));
    if (tc && (st = build_tensor_maps(c)) != FE_OK) return bail(st);

    // weight tables: forward = flipped taps (convolution as correlation),
    // tap-major; adjoint = taps as stored times 2 theta_i (the factor of
    // theta_i rho'), filter-major (correlation = K^T)
    std::vector<float> wf((size_t)KT * NFMAX, 0.f), wa((size_t)NFMAX * KT_PAD, 0.f), th(NFMAX, 0.f);
    for (int i = 0; i < p->nf; ++i) {
        for (int t = 0; t < KT; ++t) {
            wf[(size_t)t * NFMAX + i] = p->filters[(size_t)i * KT + (KT - 1 - t)];
            wa[(size_t)i * KT_PAD + t] = 2.0f * p->theta[i] * p->filters[(size_t)i * KT + t];
        }
        th[i] = p->theta[i];
    }
    if (cudaMemcpy(c->d_wf, wf.data(), wf.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_wa, wa.data(), wa.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_th, th.data(), th.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_imgs, c->himg.data(), sizeof(ImgDesc) * nimg, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_tiles, c->htile.data(), sizeof(TileDesc) * c->ntiles, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(c->d_order, c->horder.data(), sizeof(int) * c->ntiles, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_porder, c->hporder.data(), sizeof(int) * c->ntiles, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(set_err(c, FE_ECUDA, "upload of descriptors failed: %s", cudaGetErrorString(cudaGetLastError())));

    KParams &kp = c->kp;
    std::memset(&kp, 0, sizeof kp);
    kp.imgs = c->d_imgs;
    kp.st = c->d_st;
    kp.tiles = c->d_tiles;
    kp.order = c->d_order;
    kp.partials = c->d_part;
    kp.img_arrivals = c->d_arr;
    kp.loop = c->d_loop;
    kp.wf = c->d_wf;
    kp.wa = c->d_wa;
    kp.theta = c->d_th;
    kp.nfp = c->nfp;
    kp.nimg = nimg;
    kp.ntiles = c->ntiles;
    kp.beta = p->beta;
    kp.eta = p->eta;
    kp.c2 = p->c2;
    kp.max_bt = p->max_backtrack;
    kp.results = c->d_res;
    kp.tcw_fwd = c->d_tcw_fwd;
    kp.tcw_adj = c->d_tcw_adj;
    kp.tc_error = c->d_tc_error;
    kp.sched = c->d_sched;
    kp.porder = c->d_porder;

    if (cudaMemset(c->d_loop, 0, sizeof(LoopCtl)) != cudaSuccess)
        return bail(set_err(c, FE_ECUDA, "cudaMemset: %s", cudaGetErrorString(cudaGetLastError())));
    if ((st = load_inputs(c, f, u0)) != FE_OK) return bail(st);
    if (cand.size() > 1) {
        if ((st = autotune_tile(c, cand)) != FE_OK) return bail(st);
        if ((st = load_inputs(c, f, u0)) != FE_OK) return bail(st);  // state of the chosen tiling
    }
    *out = c;
    return FE_OK;
}

fe_status fe_init(fe_ctx **out, const fe_params *p, int H, int W, const float *f, const float *u0, void *stream) {
    const float *fa[1] = {f};
    const float *ua[1] = {u0};
    return fe_init_batch(out, p, 1, &H, &W, fa, u0 ? ua : nullptr, stream);
}

fe_status fe_reset(fe_ctx *c, const float *const *f, const float *const *u0) {
    if (!c) return FE_EINVAL;
    return load_inputs(c, f, u0);
}

fe_status fe_set_loop_mode(fe_ctx *c, int mode) {
    if (!c || mode < 0 || mode > 3) return FE_EINVAL;
    c->loop_mode = mode;
    return FE_OK;
}

fe_status fe_step(fe_ctx *c, int n, fe_status *worst) {
    if (!c) return FE_EINVAL;
    if (n < 0) return set_err(c, FE_EINVAL, "n must be >= 0");
    if (n > 0) {
        const long long budget = (long long)n * (c->prm.max_backtrack + 1) + 1;
        begin_kernel<<<1, 32, 0, c->s>>>(c->d_st, c->nimg, n, 0.0, c->d_loop, budget, nullptr, c->d_sched);
        FE_CUDA(c, cudaGetLastError());
        ++c->host_launches;
        fe_status st = run_loop(c, n, budget, worst != nullptr);
        if (st != FE_OK) return st;
    }
    if (worst) {
        std::vector<ImgState> hs;
        fe_status st = fetch_states(c, hs);
        if (st != FE_OK) return st;
        *worst = FE_OK;
        for (auto &s : hs)
            if (s.status != FE_OK) {
                *worst = (fe_status)s.status;
                break;
            }
    }
    return FE_OK;
}

fe_status fe_solve(fe_ctx *c, int max_iter, double rel_tol) { return fe_solve_to_energy(c, max_iter, rel_tol, nullptr); }

fe_status fe_solve_to_energy(fe_ctx *c, int max_iter, double rel_tol, const double *H_target) {
    if (!c) return FE_EINVAL;
    if (max_iter < 0 || !(rel_tol >= 0.0)) return set_err(c, FE_EINVAL, "max_iter >= 0 and rel_tol >= 0 required");
    const long long budget = (long long)max_iter * (c->prm.max_backtrack + 1) + 1;
    const double *d_target = nullptr;
    if (H_target) {
        for (int j = 0; j < c->nimg; ++j)
            if (std::isnan(H_target[j])) return set_err(c, FE_EINVAL, "H_target[%d] is NaN", j);
        FE_CUDA(c, cudaMemcpyAsync(c->d_htarget, H_target, sizeof(double) * c->nimg, cudaMemcpyHostToDevice, c->s));
        d_target = c->d_htarget;
    }
    begin_kernel<<<1, 32, 0, c->s>>>(c->d_st, c->nimg, max_iter, rel_tol, c->d_loop, budget, d_target,
                                     c->d_sched);
    FE_CUDA(c, cudaGetLastError());
    ++c->host_launches;
    fe_status st = run_loop(c, std::min(max_iter, 32), budget, true);
    if (st != FE_OK) return st;
    std::vector<ImgState> hs;
    if ((st = fetch_states(c, hs)) != FE_OK) return st;
    for (auto &s : hs)
        if (s.status != FE_OK) return (fe_status)s.status;
    for (auto &s : hs)
        if (!s.converged) return FE_ENOTCONVERGED;
    return FE_OK;
}

fe_status fe_get_info(fe_ctx *c, int img, fe_info *out) {
    fe_status st = check_img(c, img);
    if (st != FE_OK) return st;
    if (!out) return set_err(c, FE_EINVAL, "out is NULL");
    ImgState s;
    FE_CUDA(c, cudaMemcpyAsync(&s, c->d_st + img, sizeof s, cudaMemcpyDeviceToHost, c->s));
    FE_CUDA(c, cudaStreamSynchronize(c->s));
    out->n = s.n;
    out->trials = s.trials;
    out->backtracks = s.backtracks;
    out->L = s.L;
    out->alpha = s.alpha;
    out->F = s.F;
    out->G = s.G;
    out->H = s.H;
    out->H_prev = s.H_prev;
    out->rel_change = s.rel_change;
    out->last_gd = s.last_gd;
    out->last_dd = s.last_dd;
    out->last_dp = s.last_dp;
    out->status = s.status;
    out->converged = s.converged;
    out->G_floor = s.Gf;
    return FE_OK;
}

fe_status fe_get_state(fe_ctx *c, int img, float *u, float *u_prev, float *g, fe_info *info) {
    fe_status st = check_img(c, img);
    if (st != FE_OK) return st;
    ImgState s;
    FE_CUDA(c, cudaMemcpyAsync(&s, c->d_st + img, sizeof s, cudaMemcpyDeviceToHost, c->s));
    FE_CUDA(c, cudaStreamSynchronize(c->s));
    const ImgDesc &d = c->himg[img];
    const size_t N = (size_t)d.H * d.W;
    if (u) FE_CUDA(c, cudaMemcpyAsync(u, d.u[s.cur], N * 4, cudaMemcpyDefault, c->s));
    if (u_prev) FE_CUDA(c, cudaMemcpyAsync(u_prev, d.u[(s.cur + 2) % 3], N * 4, cudaMemcpyDefault, c->s));
    if (g) FE_CUDA(c, cudaMemcpyAsync(g, d.g[s.gcur], N * 4, cudaMemcpyDefault, c->s));
    FE_CUDA(c, cudaStreamSynchronize(c->s));
    if (info) return fe_get_info(c, img, info);
    return FE_OK;
}

fe_status fe_set_state(fe_ctx *c, int img, const float *u, const float *u_prev, const float *g, const fe_info *info) {
    fe_status st = check_img(c, img);
    if (st != FE_OK) return st;
    if (!u || !u_prev || !g || !info) return set_err(c, FE_EINVAL, "u, u_prev, g and info are required");
    ImgState s;
    FE_CUDA(c, cudaMemcpyAsync(&s, c->d_st + img, sizeof s, cudaMemcpyDeviceToHost, c->s));
    FE_CUDA(c, cudaStreamSynchronize(c->s));
    const ImgDesc &d = c->himg[img];
    const size_t N = (size_t)d.H * d.W;
    FE_CUDA(c, cudaMemcpyAsync(d.u[s.cur], u, N * 4, cudaMemcpyDefault, c->s));
    FE_CUDA(c, cudaMemcpyAsync(d.u[(s.cur + 2) % 3], u_prev, N * 4, cudaMemcpyDefault, c->s));
    FE_CUDA(c, cudaMemcpyAsync(d.g[s.gcur], g, N * 4, cudaMemcpyDefault, c->s));
    s.n = info->n;
    s.trials = info->trials;
    s.backtracks = info->backtracks;
    s.L = info->L;
    s.alpha = info->alpha;
    s.F = info->F;
    s.G = info->G;
    s.H = info->H;
    s.H_prev = info->H_prev;
    s.rel_change = info->rel_change;
    s.last_gd = info->last_gd;
    s.last_dd = info->last_dd;
    s.last_dp = info->last_dp;
    s.status = info->status;
    s.converged = info->converged;
    s.bt = 0;
    s.done = 0;
    FE_CUDA(c, cudaMemcpyAsync(c->d_st + img, &s, sizeof s, cudaMemcpyHostToDevice, c->s));
    FE_CUDA(c, cudaStreamSynchronize(c->s));
    return FE_OK;
}

fe_status fe_get_u(fe_ctx *c, int img, float *out) {
    if (c && c->prm.model != FE_MODEL_COMBINED) return fe_get_state(c, img, out, nullptr, nullptr, nullptr);
    fe_status st = check_img(c, img);
    if (st != FE_OK) return st;
    if (!out) return set_err(c, FE_EINVAL, "out is NULL");
    ImgState s;
    FE_CUDA(c, cudaMemcpyAsync(&s, c->d_st + img, sizeof s, cudaMemcpyDeviceToHost, c->s));
    FE_CUDA(c, cudaStreamSynchronize(c->s));
    const ImgDesc &d = c->himg[img];
    const size_t N = (size_t)d.H * d.W;
    // u = e^w into the caller's device buffer, or via the scratch plane
    const bool dev = is_device_ptr(out);
    float *dst = dev ? out : c->d_scratch;
    exp_kernel<<<(int)std::min<size_t>((N + 255) / 256, 4096), 256, 0, c->s>>>(d.u[s.cur], dst, N);
    FE_CUDA(c, cudaGetLastError());
    ++c->host_launches;
    if (!dev) FE_CUDA(c, cudaMemcpyAsync(out, dst, N * 4, cudaMemcpyDefault, c->s));
    FE_CUDA(c, cudaStreamSynchronize(c->s));
    return FE_OK;
}

static fe_status ext_launch(fe_ctx *c, int mode, int img, const float *u, float *g, double *F, double *G) {
    fe_status st = check_img(c, img);
    if (st != FE_OK) return st;
    if (!u) return set_err(c, FE_EINVAL, "u is NULL");
    const ImgDesc &d = c->himg[img];
    const size_t N = (size_t)d.H * d.W;
    const float *ud;
    if ((st = stage_in(c, u, N, 0, &ud)) != FE_OK) return st;
    float *gd = nullptr;
    const bool g_dev = g && is_device_ptr(g);
    if (mode == MODE_GRAD_EXT) gd = g_dev ? g : c->d_scratch + c->max_plane;
    // positivity of u is required by log u in G
    FE_CUDA(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->s));
    KParams kp = c->kp;
    kp.tile0 = d.tile_begin;
    kp.order = nullptr;  // one image's tiles in list order
    kp.u_ext = ud;
    kp.g_ext = gd;
    FE_CUDA(c, launch_tiles(c, mode, kp, d.ntiles));
    ++c->host_launches;
    double res[2];
    FE_CUDA(c, cudaMemcpyAsync(res, c->d_res + 2 * img, sizeof res, cudaMemcpyDeviceToHost, c->s));
    if (mode == MODE_GRAD_EXT && g && !g_dev) FE_CUDA(c, cudaMemcpyAsync(g, gd, N * 4, cudaMemcpyDefault, c->s));
    FE_CUDA(c, cudaStreamSynchronize(c->s));
    if (F) *F = res[0];
    if (G) *G = res[1];
    return FE_OK;
}

fe_status fe_energy(fe_ctx *c, int img, const float *u, double *E, double *F, double *G) {
    double f_ = 0, g_ = 0;
    fe_status st = ext_launch(c, MODE_ENERGY_EXT, img, u, nullptr, &f_, &g_);
    if (st != FE_OK) return st;
    if (E) *E = f_ + g_;
    if (F) *F = f_;
    if (G) *G = g_;
    return FE_OK;
}

fe_status fe_gradient(fe_ctx *c, int img, const float *u, float *g, double *F) {
    if (c && !g) return set_err(c, FE_EINVAL, "g is NULL");
    return ext_launch(c, MODE_GRAD_EXT, img, u, g, F, nullptr);
}

int fe_num_images(const fe_ctx *c) { return c ? c->nimg : 0; }

fe_status fe_tile_size(const fe_ctx *c, int *tile_y, int *tile_x) {
    if (!c || !tile_y || !tile_x) return FE_EINVAL;
    *tile_y = c->tile_y;
    *tile_x = c->tile_x;
    return FE_OK;
}

int fe_tile_cluster(const fe_ctx *c) { return c ? c->cluster : 0; }

fe_status fe_image_size(const fe_ctx *c, int img, int *H, int *W) {
    if (!c || img < 0 || img >= c->nimg) return FE_EINVAL;
    if (H) *H = c->H[img];
    if (W) *W = c->W[img];
    return FE_OK;
}

long long fe_launch_count(const fe_ctx *c) {
    if (!c) return 0;
    LoopCtl lc;
    if (cudaMemcpyAsync(&lc, c->d_loop, sizeof lc, cudaMemcpyDeviceToHost, c->s) != cudaSuccess ||
        cudaStreamSynchronize(c->s) != cudaSuccess)
        return -1;
    // trial kernels are counted on the device (host loop and graph alike),
    // every other kernel on the host
    return c->host_launches + lc.launches;
}

}  // extern "C"
