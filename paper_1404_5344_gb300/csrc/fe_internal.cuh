// Internal declarations of libfe shared by its translation units.
//
// Device data model (per image j of a context):
//   u[0..2]  three rotating FP32 planes: u^n = u[cur], u^{n-1} = u[(cur+2)%3],
//            the trial writes u^{n+1} into u[(cur+1)%3]
//   g[0..1]  grad F(u^n) = g[gcur]; the trial writes grad F(u^{n+1}) into g[gcur^1]
//   f2       f^2 (the data term and its prox only use f^2)
// A rejected trial leaves cur/gcur untouched, so its outputs are simply
// overwritten by the next trial.  All planes are row-major with pitch W.
//
// Each launch of a tile kernel covers every tile of every image; the last
// block to finish an image reduces that image's per-tile partial sums in a
// fixed order (deterministic) and takes the accept/reject decision of the
// backtracking rule on the device; the last block of the grid updates the
// device-side loop control (count of active images, trial budget, and the
// while-condition of the CUDA graph when the loop runs as a graph).
//
// Persistent trial launches (MODE_PTRIAL): one launch runs every trial of
// every image.  Its CTAs (as many as fit on the GPU at once) take tiles from
// per-image counters sched[j]: the block that decides image j's trial resets
// sched[j] to 0 when the image goes on, so that the tiles of its next trial
// become available at once, while other images' trials still run.  Each
// image's trials, and each trial's arithmetic and reduction order, are those
// of the per-trial launches: the results are the same bit for bit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fe.h"

namespace fe {

constexpr int NRED = 5;  // F(u1), G(u1), <g,D>, |D|^2, <D, u^n - u^{n-1}>
constexpr int NFMAX = 64;
constexpr int KS = 7;
constexpr int KT = KS * KS;  // 49 taps
constexpr int KT_PAD = 52;   // per-filter stride of the adjoint weight table

enum Mode : int {
    MODE_TRIAL = 0,       // one iPiano trial from u^n, u^{n-1}, g^n
    MODE_INIT = 1,        // g = grad F(u[0]) into g[0]; F, G; initialise the state
    MODE_GRAD_EXT = 2,    // g_ext = grad F(u_ext); F, G into results
    MODE_ENERGY_EXT = 3,  // F(u_ext), G(u_ext) into results
    MODE_PTRIAL = 4,      // persistent: one launch runs every trial of every image
};

struct ImgDesc {
    int H, W;
    int tile_begin, ntiles;
    float *u[3];
    float *g[2];
    float *f2;
    double lambda;   // variant model: lambda; combined model: lambda2 (variant term)
    double lambda1;  // combined model: weight of the log-domain term
    double gscale;   // factor applied to the summed data-term partials (variant: lambda/2;
                     // combined: 1, the kernel sums the full per-pixel value)
    // tensor-core forms: six TMA tensor maps (CUtensorMap, 128 bytes each) of
    // the planes u[0], u[1], u[2], g[0], g[1], f2 in device memory, for the
    // trial's box loads of tile + 6-pixel halo; NULL where the plane pitch is
    // not a multiple of 16 bytes (W % 4 != 0): those images use plain loads
    const void *tmap;
};

struct ImgState {
    double F, G, H, H_prev;
    double L, alpha;
    double rel_change, last_gd, last_dd, last_dp;
    double tol;
    double H_target;  // stop once an accepted H <= H_target (-inf: no energy target)
    double Gf;  // min of the data term: at u = f (variant), at w = log f (combined)
    long long n, trials, backtracks, target;
    long long trial_limit;  // persistent launches: trials allowed before FE_ETIMEOUT
    int cur, gcur, bt, status, done, converged;
};

// A tile covers rows [y0, y0 + TY) and columns [x0, x0 + TX) of an image; it
// owns (writes, sums) rows [y0 + sy, y0 + sy + oh) and columns
// [x0 + sx, x0 + sx + ow).  The FP32 kernel tiles without overlap (sy = sx =
// 0); the tensor-core kernel shifts the last tile of a row/column back so
// that it ends at the image border, leaving the previous tile to own the rows
// before it, and keeps the first three rows/columns with the first tile.
struct TileDesc {
    int img, y0, x0, oh, ow, sy, sx, pad;
};

struct LoopCtl {
    unsigned grid_arrivals;  // blocks arrived in the current launch
    int active;              // images still iterating after the last launch
    long long budget;        // trial launches left before FE_ETIMEOUT
    long long launches;      // trial launches executed (for launch accounting)
    unsigned long long decisions;  // persistent launches: trial decisions taken (progress)
    int abort;               // persistent launches: a wait for work ran out
    int pad;
};

// A persistent launch's wait for work gives up when no trial of any image has
// been decided for this long (one trial of the largest image takes
// milliseconds): the launch then stops with LoopCtl::abort set instead of
// spinning on.
constexpr unsigned long long PERSIST_STALL_NS = 4000000000ull;

struct KParams {
    const ImgDesc *imgs;
    ImgState *st;
    const TileDesc *tiles;
    double *partials;        // [ntiles][NRED]
    unsigned *img_arrivals;  // [nimg]
    LoopCtl *loop;
    const float *wf;     // forward weights, flipped, tap-major: wf[t * NFMAX + i] = k_i[48 - t]
    const float *wa;     // adjoint weights, filter-major: wa[i * KT_PAD + t] = 2 theta_i k_i[t]
    const float *theta;  // [NFMAX], zero beyond nf
    int nfp;             // nf rounded up to the filter-group size
    int nimg, ntiles;
    double beta, eta, c2;
    int max_bt;
    int tile0;                  // first global tile of this launch (grid covers tile0 ..)
    const int *order;           // whole-list launches: block b runs tile order[b] (NULL: tile0 + b)
    const float *u_ext;         // input of the EXT modes (one image per launch)
    float *g_ext;               // gradient output of MODE_GRAD_EXT
    double *results;            // [nimg][2]: F, G of the EXT modes
    unsigned long long cond;    // cudaGraphConditionalHandle of the while node
    int use_cond;
    // tensor-core forms: filter bank rounded to the operand type, in the
    // K-major shared-memory byte layout of the forward and adjoint GEMMs
    const void *tcw_fwd;
    const void *tcw_adj;
    int *tc_error;              // set when a tensor-core wait runs out
    // persistent trial launches: per-image tile counters ([nimg]; the tiles
    // of image j's current trial are sched[j] .. ntiles - 1 still to take)
    // and each image's tiles in the order they are taken (global indices)
    int *sched;
    const int *porder;
    unsigned long long persist_stall_ns;  // wait limit of the claim (0: PERSIST_STALL_NS)
};

// FP32 fused tile kernel (fe_fp32.cu)
constexpr int fp32_tile_size = 64;  // default square output tile of the FP32 kernel
bool fp32_tile_supported(int T);     // T = 64 or 32
size_t fp32_smem_bytes(int T = fp32_tile_size);
int fp32_tile();                                    // the default tile, fp32_tile_size
int fp32_threads(int T = fp32_tile_size);           // block size of the tile kernel
int fp32_ctas_per_sm(int T);  // CTAs per SM the tile kernel is built for (launch bounds, shared memory)
cudaError_t fp32_prepare();  // opt in to the large shared-memory carve-out (every tile and model)
// model: 0 = Eq. variant (iterate u), 1 = combined model (iterate w = log u);
// cl: CTAs per tile (1, or 4 = a thread-block cluster per 32 x 32 tile);
// grid = tiles (the launch multiplies by cl)
cudaError_t fp32_launch(int mode, const KParams &p, int grid, cudaStream_t s, int T = fp32_tile_size,
                        int model = 0, int cl = 1);
const void *fp32_trial_entry(int T = fp32_tile_size, int model = 0, int cl = 1);
const void *fp32_ptrial_entry(int T, int model);  // persistent trial kernel (one CTA per tile)
cudaError_t fp32c_prepare();  // combined-model instantiations (fe_fp32_comb.cu)
cudaError_t fp32c_launch(int mode, const KParams &p, int grid, cudaStream_t s, int T, int cl);
const void *fp32c_trial_entry(int T, int cl);
const void *fp32c_ptrial_entry(int T);
cudaError_t fp32cl64_prepare();  // 64 x 64 tiles on 4-CTA clusters, both models (fe_fp32_cl64.cu)
cudaError_t fp32cl64_launch(int mode, const KParams &p, int grid, cudaStream_t s, int model);
const void *fp32cl64_trial_entry(int model);

// Tensor-core tile kernel (fe_tc.cu); fmt 1 = BF16, 2 = TF32 operands
constexpr int tc_tile_y = 58, tc_tile_x = 26;  // output tile; tile + 3-pixel halo = 64 x 32
// TMA box of the trial's inputs: the tile + 6-pixel halo (70 rows x 38
// columns) from a start column rounded down to a multiple of 4 (16 bytes)
constexpr int tc_box_x = 44, tc_box_y = 70;
size_t tc_smem_bytes(int fmt);
int tc_threads();
int tc_ctas_per_sm(int fmt);  // CTAs per SM the kernel is built for (launch bounds, shared memory)
cudaError_t tc_prepare();  // every format and model
// model: 0 = Eq. variant (iterate u), 1 = combined model (iterate w = log u)
cudaError_t tc_launch(int mode, int fmt, const KParams &p, int grid, cudaStream_t s, int model = 0);
const void *tc_trial_entry(int fmt, int model = 0);
const void *tc_ptrial_entry(int fmt, int model = 0);  // persistent trial kernel
cudaError_t tcc_prepare();  // combined-model instantiations (fe_tc_comb.cu)
cudaError_t tcc_launch(int mode, int fmt, const KParams &p, int grid, cudaStream_t s);
const void *tcc_trial_entry(int fmt);
const void *tcc_ptrial_entry(int fmt);
// Host: filter bank rounded to the operand type (BF16 round-to-nearest-even,
// TF32 round-to-nearest-away) in the byte layout of the two GEMM B operands.
void tc_build_weights(int fmt, const float *filters, int nf, std::vector<unsigned char> &fwd,
                      std::vector<unsigned char> &adj);
float tc_round(int fmt, float x);

// Message returned by fe_last_error(NULL) for calls without a context (fe_api.cu)
void set_global_error(const char *msg);
}  // namespace fe
