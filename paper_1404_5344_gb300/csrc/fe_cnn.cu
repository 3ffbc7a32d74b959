// Learned warm start: a small CNN that predicts u^0 from the observation f,
// with hand-written inference and training kernels.
//
// Network (depth D = 5, width C = 32): 3x3 convolutions with zero padding,
// 1 -> C -> C -> C -> C -> 1 channels, bias, ReLU after every layer but the
// last.  Input x = log f - M0; output d; the prediction is
//   u^0 = f exp(d)        (positive by construction),
// trained with the loss mean_p (d_p - t_p)^2, t = log u* - log f, where u* is
// the output of the iPiano solver run on f.  Weights are kept in FP32 (Adam
// state) and used in BF16 (rounded to nearest even) by every convolution;
// activations and accumulation are FP32.
//
// Kernels: conv3x3 forward (bias + ReLU fused; with an optional ReLU mask on
// the input it also serves as the data gradient, given transposed and
// flipped weights), weight/bias gradient with per-CTA partial sums and a
// fixed-order reduction (deterministic), loss + output gradient, Adam.
//
// The 32 -> 32 convolutions (three in the forward pass, three data
// gradients in the backward pass) run on the tensor cores as implicit GEMMs
// (conv32_tc_kernel): a CTA computes 16 x 8 output pixels (M = 128) times
// 32 output channels (N = 32) in tensor memory; K = 9 taps x 32 input
// channels, each activation carried as a BF16 hi + lo pair (K doubles), so
// the products of the BF16 weights with the FP32 activations keep about 16
// bits and the sums are FP32.  No im2col copy is made: the 18 x 10 halo
// tile is stored channel-chunk-major in shared memory (chunk of 8 channels,
// then pixel, 16 bytes per pixel and chunk), so the A operand of tap (dy,
// dx) is the same tile read from a descriptor start shifted by (dy x 10 +
// dx) pixels, its 8-pixel core-matrix groups (one output row each) 160
// bytes apart and its two channel chunks of one MMA 2880 bytes apart.  The
// 1 -> 32 and 32 -> 1 layers (K = 9 or N = 1) stay on the CUDA cores.  The
// weight gradients of the 32 -> 32 layers run on the tensor cores as well
// (wgrad32_tc_kernel: the pixels as K); those of the other two layers on the
// CUDA cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "fe_internal.cuh"
#include "fe_tile_common.cuh"
#include "tc_ptx.cuh"

namespace fe {
namespace {

constexpr int CW = 32;       // width
constexpr int DEPTH = 5;     // layers
constexpr float M0 = 4.5f;   // input offset of log f
constexpr int TS = 16;       // output tile side of the conv kernels
constexpr int NT = TS * TS;  // 256 threads

__host__ __device__ constexpr int cin_of(int l) { return l == 0 ? 1 : CW; }
__host__ __device__ constexpr int cout_of(int l) { return l == DEPTH - 1 ? 1 : CW; }

// y[b][o][p] = act(bias[o] + sum_c sum_tap w[c][tap][o] * x'[b][c][p + off(tap)])
// x' = x, or x * (mask > 0) when mask != nullptr.  w is [CIN][9][COUT]
// (FP32 values of the BF16 weights).  Zero padding.
template <int CIN, int COUT, bool RELU>
__global__ void __launch_bounds__(NT) conv3x3_kernel(const float *__restrict__ x, const float *__restrict__ mask,
                                                     const float *__restrict__ w, const float *__restrict__ bias,
                                                     float *__restrict__ y, int H, int W) {
    extern __shared__ __align__(16) float csm[];
    float *sw = csm;                                                     // [CIN * 9 * COUT]
    float(*sx)[TS + 2][TS + 2] = reinterpret_cast<float(*)[TS + 2][TS + 2]>(csm + CIN * 9 * COUT);
    const int b = blockIdx.z, tx0 = blockIdx.x * TS, ty0 = blockIdx.y * TS;
    const int tid = threadIdx.x, ly = tid / TS, lx = tid % TS;
    const size_t plane = (size_t)H * W;
    for (int j = tid; j < CIN * 9 * COUT; j += NT) sw[j] = w[j];
    for (int j = tid; j < CIN * (TS + 2) * (TS + 2); j += NT) {
        const int c = j / ((TS + 2) * (TS + 2)), r = j % ((TS + 2) * (TS + 2));
        const int yy = ty0 - 1 + r / (TS + 2), xx = tx0 - 1 + r % (TS + 2);
        float v = 0.f;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
            const size_t o = ((size_t)b * CIN + c) * plane + (size_t)yy * W + xx;
            v = x[o];
            if (mask && !(mask[o] > 0.f)) v = 0.f;
        }
        sx[c][r / (TS + 2)][r % (TS + 2)] = v;
    }
    __syncthreads();
    float acc[COUT];
#pragma unroll
    for (int o = 0; o < COUT; ++o) acc[o] = bias ? bias[o] : 0.f;
    for (int c = 0; c < CIN; ++c) {
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const float v = sx[c][ly + t / 3][lx + t % 3];
            const float *wp = sw + (c * 9 + t) * COUT;
#pragma unroll
            for (int o = 0; o < COUT; ++o) acc[o] = fmaf(wp[o], v, acc[o]);
        }
    }
    const int yy = ty0 + ly, xx = tx0 + lx;
    if (yy < H && xx < W) {
#pragma unroll
        for (int o = 0; o < COUT; ++o)
            y[((size_t)b * COUT + o) * plane + (size_t)yy * W + xx] = RELU ? fmaxf(acc[o], 0.f) : acc[o];
    }
}

// ---- tensor-core 3x3 convolution, 32 -> 32 channels --------------------------
constexpr int TC_OY = 16, TC_OX = 8;                  // output tile: 128 pixels (M)
constexpr int TC_IY = TC_OY + 2, TC_IX = TC_OX + 2;   // 18 x 10 halo tile
constexpr int TC_NPX = TC_IY * TC_IX;                 // 180 pixels
constexpr int TC_CHUNK = TC_NPX * 16;                 // one 8-channel chunk of the tile: 2880 bytes
constexpr int TC_PLANE = 4 * TC_CHUNK;                // 32 channels (hi or lo): 11520 bytes
constexpr int TC_A_BYTES = 2 * TC_PLANE;              // hi, lo
constexpr int TC_B_TAP = CW * CW * 2;                 // one tap's B operand: N 32 x K 32 BF16
constexpr int TC_B_BYTES = 9 * TC_B_TAP;
constexpr int TC_SMEM = TC_A_BYTES + TC_B_BYTES;      // 41472 bytes
static_assert(TC_A_BYTES % 128 == 0, "B operand alignment");

// B operands of the nine taps in the K-major core-matrix byte layout:
// (tap t, output channel n, input channel k) at t * 2048 + (n / 8) * 512 +
// (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2, from a [CIN][9][COUT] weight
// array of BF16-valued floats (the forward layout, or the transposed and
// flipped one of the data gradient).
__global__ void cnn_tc_weights_kernel(const float *__restrict__ w, unsigned short *__restrict__ wq) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= CW * 9 * CW) return;
    const int k = e / (9 * CW), t = (e / CW) % 9, n = e % CW;
    const int off = t * TC_B_TAP + (n >> 3) * 512 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
    wq[off / 2] = (unsigned short)(__float_as_uint(w[e]) >> 16);  // exact: w is BF16-valued
}

// y[b][o][p] = act(bias[o] + sum_c sum_tap w[c][tap][o] x'[b][c][p + off(tap)]),
// x' = x or x * (mask > 0), zero padding; the convolution of conv3x3_kernel
// for CIN = COUT = 32, on the tensor cores.  Persistent: a CTA loads the B
// operands and allocates tensor memory once, then runs the 16 x 8 output
// tiles blockIdx.x, blockIdx.x + gridDim.x, ... of all B images.  128
// threads: thread m holds output pixel (m / 8, m % 8) of a tile in TMEM lane
// m.  A completion wait that runs out sets *err and the CTA stops.
template <bool RELU>
__global__ void __launch_bounds__(128) conv32_tc_kernel(const float *__restrict__ x, const float *__restrict__ mask,
                                                        const unsigned short *__restrict__ wq,
                                                        const float *__restrict__ bias, float *__restrict__ y, int B,
                                                        int H, int W, int *err) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    unsigned char *sA = tsm;                // [hi | lo][chunk][pixel][8 channels] BF16
    unsigned char *sB = tsm + TC_A_BYTES;   // [tap] B operands
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5;
    const size_t plane = (size_t)H * W;
    const int tiles_x = (W + TC_OX - 1) / TC_OX, tiles_img = tiles_x * ((H + TC_OY - 1) / TC_OY);
    const int ntiles = tiles_img * B;
    for (int j = tid; j < TC_B_BYTES / 16; j += 128)
        reinterpret_cast<uint4 *>(sB)[j] = __ldg(reinterpret_cast<const uint4 *>(wq) + j);
    if (tid == 0) tc::mbar_init(&bar, 1);
    if (warp == 0) tc::tmem_alloc(&tbase, 32);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tbase;
    float bv[CW];
#pragma unroll
    for (int o = 0; o < CW; ++o) bv[o] = bias ? __ldg(bias + o) : 0.f;
    uint32_t phase = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int b = tile / tiles_img, tr = tile - b * tiles_img;
        const int ty0 = (tr / tiles_x) * TC_OY, tx0 = (tr % tiles_x) * TC_OX;
        // halo tile: one task per (pixel, chunk of 8 channels): hi and lo runs;
        // a thread's (up to) 6 tasks issue all their global loads first, so
        // that their latencies overlap, then convert and store
        constexpr int NTASK = (4 * TC_NPX + 127) / 128;
        float v[NTASK][8];
#pragma unroll
        for (int k = 0; k < NTASK; ++k) {
            const int task = tid + 128 * k;
            const int q = task / TC_NPX, px = task - q * TC_NPX;
            const int iy = px / TC_IX, ix = px - iy * TC_IX;
            const int yy = ty0 - 1 + iy, xx = tx0 - 1 + ix;
            const bool in = task < 4 * TC_NPX && yy >= 0 && yy < H && xx >= 0 && xx < W;
            const size_t o0 = ((size_t)b * CW + q * 8) * plane + (size_t)yy * W + xx;
#pragma unroll
            for (int c = 0; c < 8; ++c) v[k][c] = in ? __ldg(x + o0 + c * plane) : 0.f;
            if (mask) {
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (in && !(__ldg(mask + o0 + c * plane) > 0.f)) v[k][c] = 0.f;
            }
        }
#pragma unroll
        for (int k = 0; k < NTASK; ++k) {
            const int task = tid + 128 * k;
            if (task >= 4 * TC_NPX) break;
            const int q = task / TC_NPX, px = task - q * TC_NPX;
            uint32_t h[4], l[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                h[j] = bf16x2_rn(v[k][2 * j], v[k][2 * j + 1]);
                l[j] = bf16x2_rn(v[k][2 * j] - __uint_as_float(h[j] << 16),
                                 v[k][2 * j + 1] - __uint_as_float(h[j] & 0xffff0000u));
            }
            unsigned char *dst = sA + q * TC_CHUNK + px * 16;
            *reinterpret_cast<uint4 *>(dst) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4 *>(dst + TC_PLANE) = make_uint4(l[0], l[1], l[2], l[3]);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            constexpr uint32_t idesc = tc::make_idesc(1, 128, CW);
            const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
            uint32_t acc = 0u;
#pragma unroll 1
            for (int t = 0; t < 9; ++t) {
                const uint32_t shift = (uint32_t)(((t / 3) * TC_IX + (t % 3)) * 16);
#pragma unroll
                for (int pl = 0; pl < 2; ++pl)
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t ad =
                            tc::make_smem_desc(a0 + pl * TC_PLANE + 2 * ks * TC_CHUNK + shift, TC_CHUNK, TC_IX * 16);
                        const uint64_t bd = tc::make_smem_desc(b0 + t * TC_B_TAP + ks * 256, 128, 512);
                        tc::mma<1>(taddr, ad, bd, idesc, acc);
                        acc = 1u;
                    }
            }
            tc::mma_commit(&bar);
        }
        bool ok = tc::mbar_wait(&bar, phase);
        if (!ok) {
            if (tid == 0) atomicExch(err, 1);
            ok = tc::mbar_wait(&bar, phase);  // a second bounded chance for MMAs in flight
        }
        phase ^= 1u;
        tc::fence_after_sync();
        const bool wok = __all_sync(0xffffffffu, ok);
        if (wok) {
            float a[CW];
#pragma unroll
            for (int j = 0; j < CW / 8; ++j) {
                float t8[8];
                tc::tmem_ld8(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(8 * j), t8);
#pragma unroll
                for (int k = 0; k < 8; ++k) a[8 * j + k] = t8[k];
            }
            tc::tmem_ld_wait();
            const int oy = ty0 + tid / TC_OX, ox = tx0 + tid % TC_OX;
            if (oy < H && ox < W) {
#pragma unroll
                for (int o = 0; o < CW; ++o) {
                    const float r = a[o] + bv[o];
                    y[((size_t)b * CW + o) * plane + (size_t)oy * W + ox] = RELU ? fmaxf(r, 0.f) : r;
                }
            }
        }
        // the next tile rewrites the operands and the accumulator
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (!__syncthreads_and(ok)) break;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 32);
}

// Per-CTA partial sums of the weight and bias gradients of one layer (the
// 1 -> 32 and 32 -> 1 layers):
//   dW[o][c][tap] += sum_p g[b][o][p] x[b][c][p + off(tap)],  dB[o] += sum_p g[b][o][p]
// with g = dY * (Y > 0) for a ReLU layer (Y = the layer's output) or dY.  The
// CTAs are persistent over the 16 x 16 tiles (blockIdx.x, + gridDim.x, ...);
// a thread owns the parameters tid and tid + NT, sums a tile's 256 pixels in
// FP32 and the tiles in FP64.  part[blockIdx.x][COUT*CIN*9 + COUT].
template <int CIN, int COUT, bool RELU>
__global__ void __launch_bounds__(NT, CIN == 1 ? 1 : 2) wgrad_kernel(const float *__restrict__ x, const float *__restrict__ dy,
                                                   const float *__restrict__ yout, float *__restrict__ part, int B,
                                                   int H, int W) {
    constexpr int NW = COUT * CIN * 9, NE = NW + COUT;
    static_assert(NE <= 2 * NT, "two parameters per thread");
    extern __shared__ __align__(16) float wsm[];
    // [COUT][TS*TS + 1]: the odd channel stride puts the channels a warp reads at once in distinct banks
    float(*sg)[TS * TS + 1] = reinterpret_cast<float(*)[TS * TS + 1]>(wsm);
    float(*sx)[TS + 2][TS + 2] = reinterpret_cast<float(*)[TS + 2][TS + 2]>(wsm + COUT * (TS * TS + 1));
    const int tid = threadIdx.x;
    const size_t plane = (size_t)H * W;
    const int tiles_x = (W + TS - 1) / TS, tiles_img = tiles_x * ((H + TS - 1) / TS), ntiles = tiles_img * B;
    // 32 -> 1 layer: the next tile's inputs are loaded into registers while
    // the current one is summed (halo pixel r = tid + NT k, all CIN channels of
    // it; G element tid + NT i).  1 -> 32 layer (32 G values per thread): each
    // tile is staged directly, more CTAs per SM hiding the loads.  Zero
    // padding; g masked by the ReLU.
    constexpr bool PRE = CIN > 1;
    constexpr int RX = (TS + 2) * (TS + 2), NR = (RX + NT - 1) / NT, NGL = COUT * TS * TS / NT;
    static_assert(COUT * TS * TS % NT == 0, "whole G rounds");
    float xr[NR][CIN], gr[NGL];
    auto load = [&](int tile) {
        const int b = tile / tiles_img, tr = tile - b * tiles_img;
        const int ty0 = (tr / tiles_x) * TS, tx0 = (tr % tiles_x) * TS;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            const int r = tid + k * NT;
            const int yy = ty0 - 1 + r / (TS + 2), xx = tx0 - 1 + r % (TS + 2);
            const bool in = r < RX && yy >= 0 && yy < H && xx >= 0 && xx < W;
            const float *src = x + (size_t)b * CIN * plane + (in ? (size_t)yy * W + xx : 0);
#pragma unroll
            for (int c = 0; c < CIN; ++c) xr[k][c] = in ? __ldg(src + (size_t)c * plane) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < NGL; ++i) {
            const int j = tid + i * NT;
            const int o = j / (TS * TS), r = j % (TS * TS);
            const int yy = ty0 + r / TS, xx = tx0 + r % TS;
            float g = 0.f;
            if (yy < H && xx < W) {
                const size_t idx = ((size_t)b * COUT + o) * plane + (size_t)yy * W + xx;
                g = __ldg(dy + idx);
                if (RELU && !(__ldg(yout + idx) > 0.f)) g = 0.f;
            }
            gr[i] = g;
        }
    };
    double acc[2] = {0.0, 0.0};
    if (PRE && (int)blockIdx.x < ntiles) load(blockIdx.x);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();  // the previous tile's reads of sg and sx are done
        if constexpr (PRE) {
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const int r = tid + k * NT;
                if (r < RX)
#pragma unroll
                    for (int c = 0; c < CIN; ++c) (&sx[c][0][0])[r] = xr[k][c];
            }
#pragma unroll
            for (int i = 0; i < NGL; ++i) {
                const int j = tid + i * NT;
                sg[j / (TS * TS)][j % (TS * TS)] = gr[i];
            }
        } else {
            const int b = tile / tiles_img, tr = tile - b * tiles_img;
            const int ty0 = (tr / tiles_x) * TS, tx0 = (tr % tiles_x) * TS;
            for (int j = tid; j < CIN * RX; j += NT) {
                const int c = j / RX, r = j % RX;
                const int yy = ty0 - 1 + r / (TS + 2), xx = tx0 - 1 + r % (TS + 2);
                sx[c][r / (TS + 2)][r % (TS + 2)] =
                    (yy >= 0 && yy < H && xx >= 0 && xx < W) ? x[((size_t)b * CIN + c) * plane + (size_t)yy * W + xx] : 0.f;
            }
            for (int j = tid; j < COUT * TS * TS; j += NT) {
                const int o = j / (TS * TS), r = j % (TS * TS);
                const int yy = ty0 + r / TS, xx = tx0 + r % TS;
                float g = 0.f;
                if (yy < H && xx < W) {
                    const size_t idx = ((size_t)b * COUT + o) * plane + (size_t)yy * W + xx;
                    g = dy[idx];
                    if (RELU && !(yout[idx] > 0.f)) g = 0.f;
                }
                sg[o][r] = g;
            }
        }
        __syncthreads();
        if (PRE && tile + (int)gridDim.x < ntiles) load(tile + gridDim.x);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int e = tid + k * NT;
            if (e >= NE) continue;
            float s = 0.f;
            if (e < NW) {
                const int o = e / (CIN * 9), c = (e / 9) % CIN, t = e % 9;
                for (int r = 0; r < TS * TS; ++r) s = fmaf(sg[o][r], sx[c][r / TS + t / 3][r % TS + t % 3], s);
            } else {
                for (int r = 0; r < TS * TS; ++r) s += sg[e - NW][r];
            }
            acc[k] += (double)s;
        }
    }
    float *out = part + (size_t)blockIdx.x * NE;
#pragma unroll
    for (int k = 0; k < 2; ++k)
        if (tid + k * NT < NE) out[tid + k * NT] = (float)acc[k];
}

// ---- tensor-core weight gradient of the 32 -> 32 layers -----------------------
// dW[o][c][tap] = sum_p g[o][p] x[c][p + off(tap)] as GEMMs with the pixels as
// K.  Per 16 x 8 tile (K = 128 pixels: 8 MMA steps of two pixel rows) and tap
// column dx, D[(dy, c), o] (M = 128 = dy 0..3 x 32 input channels, the dy = 3
// rows unused; N = 32 output channels) accumulates in tensor memory over
// every tile the CTA takes (persistent CTAs; three tap columns = 96 TMEM
// columns), and the CTA writes its sums once.  A operand: a table of 16-byte
// entries X[dx][iy][c] = x[c][iy][dx .. dx + 7] (8 pixels of one halo row), so
// that row (dy, c) of step s is entry X[dx][2s + dy][c] (rows 16 bytes apart:
// SBO 128) and its second pixel row one halo row further (LBO 512).  B
// operand: G[py][o] = g[o][py][0 .. 7].  Both are carried as BF16 hi + lo
// (products hi*hi + lo*hi + hi*lo: about 16 bits), summed in FP32.
// Loads are spread over the lanes so that a warp instruction touches few
// cache lines: five lanes per halo row (iy, c), lane q holding the pixels 2q
// and 2q + 1 of the row's 10, which give the words of its three entries
// (dx = 0 and 2: the pair (2q, 2q + 1); dx = 1: (2q + 1, 2q + 2), the second
// value from lane q + 1); two lanes per G row (py, o), lane h holding the
// pixels 4h .. 4h + 3 (one 16-byte load when W % 4 == 0).  Each value is
// rounded to BF16 hi + lo once per word it enters.  The loads of the next tile are issued while the MMAs of the
// current one run.
constexpr int WG_IY = TC_OY + 3;              // 19 halo rows: the last is read only by the unused dy = 3 rows
constexpr int WG_ROW = CW * 16;               // one halo row of the table: 32 channels x 16 bytes
constexpr int WG_DX = WG_IY * WG_ROW;         // one tap column of the table
constexpr int WG_XPL = 3 * WG_DX;             // the hi (or lo) table
constexpr int WG_GPL = TC_OY * WG_ROW;        // the hi (or lo) G: 16 pixel rows x 32 channels x 16 bytes
constexpr int WG_XT = TC_IY * CW / 6 / 4;     // halo-row tasks (6 rows x 5 lanes) per warp: 24
constexpr int WG_GT = TC_OY / 2;              // G tasks (16 channels x 2 pixel quads) per warp: 8
constexpr int WG_SMEM = 2 * WG_XPL + 2 * WG_GPL;
static_assert(WG_XPL % 128 == 0 && WG_GPL % 128 == 0, "operand alignment");
static_assert(TC_IX == 10 && TC_OX == 8, "a halo row is 10 values, an entry 8");
static_assert(TC_IY * CW == 4 * 6 * WG_XT, "the halo rows split into 6-row tasks over 4 warps");
static_assert(3 * (WG_SMEM + 2048) <= 228 * 1024, "three CTAs per SM (1 KB static, 1 KB reserved each)");

// part[blockIdx.x][COUT*CIN*9 + COUT] (as wgrad_kernel's), the grid = the
// persistent CTAs (each takes at least one tile).  128 threads, three CTAs
// per SM.  A completion wait that runs out sets *err and the CTA stops.
template <bool RELU>
__global__ void __launch_bounds__(128, 3) wgrad32_tc_kernel(const float *__restrict__ x, const float *__restrict__ dy,
                                                            const float *__restrict__ yout, float *__restrict__ part,
                                                            int B, int H, int W, int *err) {
    extern __shared__ __align__(1024) unsigned char gsm[];
    unsigned char *sX = gsm;                                      // [hi | lo][dx][iy][c][8 pixels]
    unsigned char *sG = gsm + 2 * WG_XPL;                         // [hi | lo][py][o][8 pixels]
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t plane = (size_t)H * W;
    const int tiles_x = (W + TC_OX - 1) / TC_OX, tiles_img = tiles_x * ((H + TC_OY - 1) / TC_OY);
    const int ntiles = tiles_img * B;
    if (tid == 0) tc::mbar_init(&bar, 1);
    if (warp == 0) tc::tmem_alloc(&tbase, 128);
    // the table's last halo row (read only by the unused dy = 3 rows) holds zeros
    for (int j = tid; j < 2 * 3 * CW; j += 128) {
        const int pl = j / (3 * CW), dx = (j / CW) % 3, c = j % CW;
        *reinterpret_cast<uint4 *>(sX + pl * WG_XPL + dx * WG_DX + (WG_IY - 1) * WG_ROW + c * 16) =
            make_uint4(0u, 0u, 0u, 0u);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tbase;

    // registers of one tile.  Halo rows: task t of this warp = rows
    // 6 (warp + 4 t) + r6, r6 = lane / 5 (lanes 30, 31 idle), row R -> (iy, c) =
    // (R / 32, R % 32); lane q = lane % 5 holds pixels 2q, 2q + 1.  G rows: task
    // t = row py = (warp >> 1) + 2 t, channel o = 16 (warp & 1) + lane / 2, lane
    // h = lane % 2 holds pixels 4h .. 4h + 3.  Zero outside the image.
    const int q = lane % 5, r6 = lane / 5;
    const int o_g = 16 * (warp & 1) + (lane >> 1), h_g = lane & 1;
    const bool vec = (W & 3) == 0;  // 16-byte G loads (every row start is then 16-byte aligned)
    float xa[WG_XT], xb[WG_XT], dv[WG_GT][4], yv[WG_GT][4];
    auto load = [&](int tile) {
        const int b = tile / tiles_img, tr = tile - b * tiles_img;
        const int ty0 = (tr / tiles_x) * TC_OY, tx0 = (tr % tiles_x) * TC_OX;
        const int xx = tx0 - 1 + 2 * q;
#pragma unroll
        for (int t = 0; t < WG_XT; ++t) {
            const int R = 6 * (warp + 4 * t) + r6, iy = R >> 5, c = R & 31;
            const int yy = ty0 - 1 + iy;
            const bool rowok = lane < 30 && yy >= 0 && yy < H;
            const float *src = x + ((size_t)b * CW + c) * plane + (size_t)(rowok ? yy : 0) * W;
            xa[t] = (rowok && xx >= 0 && xx < W) ? __ldg(src + xx) : 0.f;
            xb[t] = (rowok && xx + 1 < W) ? __ldg(src + xx + 1) : 0.f;  // xx + 1 >= 0
        }
        const int gx = tx0 + 4 * h_g;
#pragma unroll
        for (int t = 0; t < WG_GT; ++t) {
            const int yy = ty0 + (warp >> 1) + 2 * t;
            const size_t base = ((size_t)b * CW + o_g) * plane + (size_t)(yy < H ? yy : 0) * W + gx;
            if (vec && yy < H && gx < W) {  // W % 4 == 0: the quad lies in the row
                const float4 d = __ldg(reinterpret_cast<const float4 *>(dy + base));
                dv[t][0] = d.x, dv[t][1] = d.y, dv[t][2] = d.z, dv[t][3] = d.w;
                if (RELU) {
                    const float4 y = __ldg(reinterpret_cast<const float4 *>(yout + base));
                    yv[t][0] = y.x, yv[t][1] = y.y, yv[t][2] = y.z, yv[t][3] = y.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool in = yy < H && gx + j < W;
                    dv[t][j] = in ? __ldg(dy + base + j) : 0.f;
                    if (RELU) yv[t][j] = in ? __ldg(yout + base + j) : 1.f;
                }
            }
        }
    };

    __shared__ float sBias[2][CW];
    float bsum = 0.f;  // this thread's share of dB[o_g]
    uint32_t phase = 0;
    bool first = true, ok = true;
    if ((int)blockIdx.x < ntiles) load(blockIdx.x);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // (the MMAs of the previous tile have completed: the operands are free)
#pragma unroll
        for (int t = 0; t < WG_XT; ++t) {
            const float a = xa[t], bv = xb[t];
            const float nx = __shfl_down_sync(0xffffffffu, a, 1);  // pixel 2q + 2 (lane q + 1 of the row)
            const uint32_t he = bf16x2_rn(a, bv);
            const uint32_t le = bf16x2_rn(a - __uint_as_float(he << 16), bv - __uint_as_float(he & 0xffff0000u));
            const uint32_t ho = bf16x2_rn(bv, nx);
            const uint32_t lo = bf16x2_rn(bv - __uint_as_float(ho << 16), nx - __uint_as_float(ho & 0xffff0000u));
            const int R = 6 * (warp + 4 * t) + r6;
            unsigned char *e = sX + (R >> 5) * WG_ROW + (R & 31) * 16;
            if (lane < 30) {
                if (q < 4) {  // dx = 0 and dx = 1, word q
                    *reinterpret_cast<uint32_t *>(e + 4 * q) = he;
                    *reinterpret_cast<uint32_t *>(e + WG_XPL + 4 * q) = le;
                    *reinterpret_cast<uint32_t *>(e + WG_DX + 4 * q) = ho;
                    *reinterpret_cast<uint32_t *>(e + WG_DX + WG_XPL + 4 * q) = lo;
                }
                if (q > 0) {  // dx = 2, word q - 1
                    *reinterpret_cast<uint32_t *>(e + 2 * WG_DX + 4 * (q - 1)) = he;
                    *reinterpret_cast<uint32_t *>(e + 2 * WG_DX + WG_XPL + 4 * (q - 1)) = le;
                }
            }
        }
#pragma unroll
        for (int t = 0; t < WG_GT; ++t) {
            uint32_t hw[2], lw[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                // g = dY, masked by Y > 0 after a ReLU
                const float g0 = (RELU && !(yv[t][2 * k] > 0.f)) ? 0.f : dv[t][2 * k];
                const float g1 = (RELU && !(yv[t][2 * k + 1] > 0.f)) ? 0.f : dv[t][2 * k + 1];
                bsum += g0;
                bsum += g1;
                hw[k] = bf16x2_rn(g0, g1);
                lw[k] = bf16x2_rn(g0 - __uint_as_float(hw[k] << 16), g1 - __uint_as_float(hw[k] & 0xffff0000u));
            }
            unsigned char *e = sG + ((warp >> 1) + 2 * t) * WG_ROW + o_g * 16 + 8 * h_g;
            *reinterpret_cast<uint2 *>(e) = make_uint2(hw[0], hw[1]);
            *reinterpret_cast<uint2 *>(e + WG_GPL) = make_uint2(lw[0], lw[1]);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            constexpr uint32_t idesc = tc::make_idesc(1, 128, CW);
            const uint32_t a0 = tc::smem_u32(sX), g0 = tc::smem_u32(sG);
#pragma unroll 1
            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                for (int st = 0; st < TC_OY / 2; ++st)
#pragma unroll
                    for (int ps = 0; ps < 3; ++ps) {  // x hi * g hi, x lo * g hi, x hi * g lo
                        const int xp = ps == 1, gp = ps == 2;
                        const uint64_t ad = tc::make_smem_desc(a0 + xp * WG_XPL + dx * WG_DX + 2 * st * WG_ROW, WG_ROW, 128);
                        const uint64_t bd = tc::make_smem_desc(g0 + gp * WG_GPL + 2 * st * WG_ROW, WG_ROW, 128);
                        tc::mma<1>(taddr + (uint32_t)(dx * CW), ad, bd, idesc, (first && st == 0 && ps == 0) ? 0u : 1u);
                    }
            tc::mma_commit(&bar);
        }
        first = false;
        // the next tile's loads (registers only) overlap the MMAs
        if (tile + (int)gridDim.x < ntiles) load(tile + gridDim.x);
        ok = tc::mbar_wait(&bar, phase);
        if (!ok) {
            if (tid == 0) atomicExch(err, 1);
            ok = tc::mbar_wait(&bar, phase);  // a second bounded chance for MMAs in flight
        }
        phase ^= 1u;
        // the next tile rewrites the operands
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (!__syncthreads_and(ok)) break;
    }
    // the CTA's partial sums: lane (dy, c) = tid of warps 0..2, columns dx*32 + o
    const size_t nw = (size_t)CW * CW * 9;
    float *out = part + (size_t)blockIdx.x * (nw + CW);
    if (!first && ok) {
#pragma unroll 1
        for (int dx = 0; dx < 3; ++dx)
#pragma unroll
            for (int j = 0; j < CW / 8; ++j) {
                float t8[8];
                tc::tmem_ld8(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(dx * CW + 8 * j), t8);
                tc::tmem_ld_wait();
                if (warp < 3) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) out[(size_t)(8 * j + k) * CW * 9 + lane * 9 + warp * 3 + dx] = t8[k];
                }
            }
    } else if (first) {
        for (size_t e = tid; e < nw; e += 128) out[e] = 0.f;
    }
    // dB[o]: the two lanes of channel o in each of its two warps, added as
    // (h0 + h1) of warp o / 16, then + (h0 + h1) of warp o / 16 + 2
    bsum += __shfl_xor_sync(0xffffffffu, bsum, 1);
    if (h_g == 0) sBias[warp >> 1][o_g] = bsum;
    __syncthreads();
    if (tid < CW) out[nw + tid] = sBias[0][tid] + sBias[1][tid];
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 128);
}


// Fixed-order reduction of per-CTA partials: out[e] = sum_k part[k][e] in
// FP64.  A block (1024 threads) takes 32 parameters (one per lane); its warp
// w adds the partials k = w, w + 32, ... in order, and the 32 warp sums are
// added in warp order (the result depends only on nblocks, not on
// scheduling).
__global__ void __launch_bounds__(1024) reduce_parts_kernel(const float *__restrict__ part, int nblocks, int n,
                                                            float *__restrict__ out) {
    __shared__ double red[32][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, e = blockIdx.x * 32 + lane;
    double s = 0.0;
    if (e < n) {
#pragma unroll 4
        for (int k = w; k < nblocks; k += 32) s += part[(size_t)k * n + e];
    }
    red[w][lane] = s;
    __syncthreads();
    if (w == 0 && e < n) {
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < 32; ++j) t += red[j][lane];
        out[e] = (float)t;
    }
}

__global__ void prep_input_kernel(const float *__restrict__ f, float *__restrict__ x, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] = logf(f[i]) - M0;
}

// u0 = f exp(d)
__global__ void output_kernel(const float *__restrict__ f, const float *__restrict__ d, float *__restrict__ u0, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        u0[i] = f[i] * expf(d[i]);
}

// loss = sum_p (d - t)^2 (per-block partials in FP64), dd = 2 (d - t) / n,
// t = log u* - log f
__global__ void loss_kernel(const float *__restrict__ d, const float *__restrict__ f, const float *__restrict__ ut,
                            float *__restrict__ dd, double *__restrict__ part, size_t n) {
    __shared__ double red[256];
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float e = d[i] - (logf(ut[i]) - logf(f[i]));
        s += (double)e * (double)e;
        dd[i] = 2.0f * e / (float)n;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Adam on the FP32 master parameters; refreshes the BF16-valued copy used by
// the convolutions (weights only: biases stay FP32).
__global__ void adam_kernel(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, const unsigned char *__restrict__ is_w,
                            float *__restrict__ pq, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pq[i] = is_w[i] ? __bfloat162float(__float2bfloat16_rn(pi)) : pi;
}

}  // namespace
}  // namespace fe

using namespace fe;

struct fe_cnn {
    cudaStream_t s = nullptr;
    int np = 0;
    std::vector<int> woff, boff;  // per layer: offset of W ([COUT][CIN][9]) and b in the parameter vector
    float *p = nullptr, *pq = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    unsigned char *is_w = nullptr;
    float *wl[DEPTH] = {}, *wt[DEPTH] = {};  // conv layouts [CIN][9][COUT] and transposed-flipped [COUT][9][CIN]
    // tensor-core B operands of the 32 -> 32 layers (1..3): forward and data gradient
    unsigned short *wqf[DEPTH] = {}, *wqt[DEPTH] = {};
    int *tc_err = nullptr;  // set when a tensor-core completion wait runs out
    int sms = 1;            // multiprocessors of the device (grid of the persistent convolutions)
    float *act = nullptr, *dact = nullptr, *part = nullptr, *tmp = nullptr;
    double *lpart = nullptr;
    size_t cap_pix = 0, cap_part = 0;
    long long step = 0;
    std::string err;
};

namespace fe {
namespace {

fe_status cnn_err(fe_cnn *n, fe_status s, const std::string &msg) {
    if (n) n->err = msg;
    return s;
}

#define CNN_CUDA(n, call)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return cnn_err((n), FE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// conv layouts from the (BF16-valued) parameters: forward [CIN][9][COUT],
// data-gradient [COUT][9][CIN] with the taps flipped
__global__ void layout_kernel(const float *__restrict__ pq, int woff, int cin, int cout, float *__restrict__ wl,
                              float *__restrict__ wt) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cin * cout * 9) return;
    const int o = e / (cin * 9), c = (e / 9) % cin, t = e % 9;
    const float w = pq[woff + e];
    wl[(c * 9 + t) * cout + o] = w;
    wt[(o * 9 + (8 - t)) * cin + c] = w;
}

fe_status refresh_layouts(fe_cnn *n) {
    for (int l = 0; l < DEPTH; ++l) {
        const int ne = cin_of(l) * cout_of(l) * 9;
        layout_kernel<<<(ne + 255) / 256, 256, 0, n->s>>>(n->pq, n->woff[l], cin_of(l), cout_of(l), n->wl[l], n->wt[l]);
        CNN_CUDA(n, cudaGetLastError());
        if (cin_of(l) == CW && cout_of(l) == CW) {
            cnn_tc_weights_kernel<<<(CW * 9 * CW + 255) / 256, 256, 0, n->s>>>(n->wl[l], n->wqf[l]);
            cnn_tc_weights_kernel<<<(CW * 9 * CW + 255) / 256, 256, 0, n->s>>>(n->wt[l], n->wqt[l]);
            CNN_CUDA(n, cudaGetLastError());
        }
    }
    return FE_OK;
}

// A 32 -> 32 convolution on the tensor cores (conv32_tc_kernel).
template <bool RELU>
void conv32(const fe_cnn *n, const float *x, const float *mask, const unsigned short *wq, const float *bias, float *y,
            int B, int H, int W) {
    // persistent: four CTAs per SM (41.5 KB of shared memory each), every
    // CTA several tiles
    const int tiles = ((W + TC_OX - 1) / TC_OX) * ((H + TC_OY - 1) / TC_OY) * B;
    const int grid = std::min(tiles, 4 * n->sms);
    conv32_tc_kernel<RELU><<<grid, 128, TC_SMEM, n->s>>>(x, mask, wq, bias, y, B, H, W, n->tc_err);
}

// FE_ETIMEOUT if a tensor-core completion wait ran out since creation
// (the stream has been synchronised by the caller).
fe_status check_tc(fe_cnn *n) {
    int e = 0;
    CNN_CUDA(n, cudaMemcpy(&e, n->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    return e ? cnn_err(n, FE_ETIMEOUT, "a tensor-core completion wait of the CNN ran out") : FE_OK;
}

fe_status ensure_capacity(fe_cnn *n, size_t pix, size_t parts) {
    if (pix > n->cap_pix) {
        cudaFree(n->act);
        cudaFree(n->dact);
        cudaFree(n->tmp);
        // activations of all layers + input: (1 + 4 C + 1) planes; two work planes of C channels
        CNN_CUDA(n, cudaMalloc(&n->act, sizeof(float) * pix * (2 + (DEPTH - 1) * CW)));
        CNN_CUDA(n, cudaMalloc(&n->dact, sizeof(float) * pix * 2 * CW));
        CNN_CUDA(n, cudaMalloc(&n->tmp, sizeof(float) * pix * 4));
        n->cap_pix = pix;
    }
    if (parts > n->cap_part) {
        cudaFree(n->part);
        CNN_CUDA(n, cudaMalloc(&n->part, sizeof(float) * parts));
        n->cap_part = parts;
    }
    return FE_OK;
}

template <int CIN, int COUT>
constexpr size_t conv_smem() { return sizeof(float) * ((size_t)CIN * 9 * COUT + (size_t)CIN * (TS + 2) * (TS + 2)); }
template <int CIN, int COUT>
constexpr size_t wgrad_smem() { return sizeof(float) * ((size_t)COUT * (TS * TS + 1) + (size_t)CIN * (TS + 2) * (TS + 2)); }

// CTAs of the tensor-core weight gradient: three per SM (73.5 KB of shared
// memory each), at most one per 16 x 8 tile
int wgrad32_ctas(const fe_cnn *n, int B, int H, int W) {
    const long long tiles = (long long)((W + TC_OX - 1) / TC_OX) * ((H + TC_OY - 1) / TC_OY) * B;
    return (int)std::max<long long>(1, std::min<long long>(tiles, 3LL * n->sms));
}

// CTAs of the CUDA-core weight gradient (1 -> 32 and 32 -> 1 layers): as
// many as are resident at once, at most one per 16 x 16 tile
template <int CIN, int COUT, bool RELU>
int wgrad_ctas(const fe_cnn *n, int B, int H, int W) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, wgrad_kernel<CIN, COUT, RELU>, NT, wgrad_smem<CIN, COUT>()) !=
            cudaSuccess ||
        occ < 1)
        occ = 1;
    const long long tiles = (long long)((W + TS - 1) / TS) * ((H + TS - 1) / TS) * B;
    return (int)std::max<long long>(1, std::min<long long>(tiles, (long long)occ * n->sms));
}

// CTAs of partial weight-gradient sums a loss_grad needs room for
size_t grad_parts(const fe_cnn *n, int B, int H, int W) {
    return (size_t)std::max({wgrad_ctas<1, CW, true>(n, B, H, W), wgrad_ctas<CW, 1, false>(n, B, H, W),
                             wgrad32_ctas(n, B, H, W)});
}

template <int CIN, int COUT, bool RELU>
void conv(const fe_cnn *n, const float *x, const float *mask, const float *w, const float *bias, float *y, int B, int H,
          int W) {
    const dim3 grid((W + TS - 1) / TS, (H + TS - 1) / TS, B);
    conv3x3_kernel<CIN, COUT, RELU><<<grid, NT, conv_smem<CIN, COUT>(), n->s>>>(x, mask, w, bias, y, H, W);
}

cudaError_t cnn_prepare() {
    cudaError_t e = cudaSuccess;
#define FE_SMEM(k, b) \
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(b))) != cudaSuccess) return e
    FE_SMEM((conv3x3_kernel<1, CW, true>), (conv_smem<1, CW>()));
    FE_SMEM((conv3x3_kernel<CW, CW, true>), (conv_smem<CW, CW>()));
    FE_SMEM((conv3x3_kernel<CW, 1, false>), (conv_smem<CW, 1>()));
    FE_SMEM((conv3x3_kernel<1, CW, false>), (conv_smem<1, CW>()));
    FE_SMEM((conv3x3_kernel<CW, CW, false>), (conv_smem<CW, CW>()));
    FE_SMEM((wgrad_kernel<CW, 1, false>), (wgrad_smem<CW, 1>()));
    FE_SMEM((wgrad_kernel<1, CW, true>), (wgrad_smem<1, CW>()));
    FE_SMEM((conv32_tc_kernel<true>), TC_SMEM);
    FE_SMEM((wgrad32_tc_kernel<true>), WG_SMEM);
    FE_SMEM((conv32_tc_kernel<false>), TC_SMEM);
#undef FE_SMEM
    return e;
}

// pointer to the activation of layer l (l = -1: the input x)
float *act_ptr(fe_cnn *n, int l, size_t pix) {
    if (l < 0) return n->act;
    return n->act + pix * (1 + (size_t)l * CW);
}

fe_status forward(fe_cnn *n, const float *f_dev, int B, int H, int W) {
    const size_t pix = (size_t)B * H * W;
    prep_input_kernel<<<(unsigned)std::min<size_t>((pix + 255) / 256, 4096), 256, 0, n->s>>>(f_dev, act_ptr(n, -1, pix), pix);
    conv<1, CW, true>(n, act_ptr(n, -1, pix), nullptr, n->wl[0], n->pq + n->boff[0], act_ptr(n, 0, pix), B, H, W);
    conv32<true>(n, act_ptr(n, 0, pix), nullptr, n->wqf[1], n->pq + n->boff[1], act_ptr(n, 1, pix), B, H, W);
    conv32<true>(n, act_ptr(n, 1, pix), nullptr, n->wqf[2], n->pq + n->boff[2], act_ptr(n, 2, pix), B, H, W);
    conv32<true>(n, act_ptr(n, 2, pix), nullptr, n->wqf[3], n->pq + n->boff[3], act_ptr(n, 3, pix), B, H, W);
    conv<CW, 1, false>(n, act_ptr(n, 3, pix), nullptr, n->wl[4], n->pq + n->boff[4], act_ptr(n, 4, pix), B, H, W);
    CNN_CUDA(n, cudaGetLastError());
    return FE_OK;
}

template <int CIN, int COUT, bool RELU>
fe_status wgrad(fe_cnn *n, const float *x, const float *dy, const float *y, int B, int H, int W, int layer) {
    int nb;
    const int ne = COUT * CIN * 9 + COUT;
    if constexpr (CIN == CW && COUT == CW) {
        nb = wgrad32_ctas(n, B, H, W);
        wgrad32_tc_kernel<RELU><<<nb, 128, WG_SMEM, n->s>>>(x, dy, y, n->part, B, H, W, n->tc_err);
    } else {
        nb = wgrad_ctas<CIN, COUT, RELU>(n, B, H, W);
        wgrad_kernel<CIN, COUT, RELU><<<nb, NT, wgrad_smem<CIN, COUT>(), n->s>>>(x, dy, y, n->part, B, H, W);
    }
    // weights then bias of this layer are contiguous in the parameter vector
    reduce_parts_kernel<<<(ne + 31) / 32, 1024, 0, n->s>>>(n->part, nb, ne, n->g + n->woff[layer]);
    CNN_CUDA(n, cudaGetLastError());
    return FE_OK;
}

// loss and gradients of all parameters into n->g (device); *loss host
fe_status loss_grad(fe_cnn *n, const float *f_dev, const float *ut_dev, int B, int H, int W, double *loss) {
    const size_t pix = (size_t)B * H * W;
    fe_status st = ensure_capacity(n, pix, grad_parts(n, B, H, W) * (CW * CW * 9 + CW));
    if (st != FE_OK) return st;
    if ((st = forward(n, f_dev, B, H, W)) != FE_OK) return st;
    const int lb = 256;
    if (!n->lpart) CNN_CUDA(n, cudaMalloc(&n->lpart, sizeof(double) * lb));
    float *dd = n->dact;  // d loss / d output, 1 channel
    loss_kernel<<<lb, 256, 0, n->s>>>(act_ptr(n, 4, pix), f_dev, ut_dev, dd, n->lpart, pix);
    CNN_CUDA(n, cudaGetLastError());
    // backward: layer 4 (no ReLU), then 3..0 (ReLU on their outputs)
    float *g_in = dd, *g_out = n->dact + pix * CW;  // ping-pong C-channel gradient planes
    if ((st = wgrad<CW, 1, false>(n, act_ptr(n, 3, pix), g_in, nullptr, B, H, W, 4)) != FE_OK) return st;
    conv<1, CW, false>(n, g_in, nullptr, n->wt[4], nullptr, g_out, B, H, W);
    std::swap(g_in, g_out);
    // g_in = d loss / d act3 (post-ReLU)
    if ((st = wgrad<CW, CW, true>(n, act_ptr(n, 2, pix), g_in, act_ptr(n, 3, pix), B, H, W, 3)) != FE_OK) return st;
    conv32<false>(n, g_in, act_ptr(n, 3, pix), n->wqt[3], nullptr, g_out, B, H, W);
    std::swap(g_in, g_out);
    if ((st = wgrad<CW, CW, true>(n, act_ptr(n, 1, pix), g_in, act_ptr(n, 2, pix), B, H, W, 2)) != FE_OK) return st;
    conv32<false>(n, g_in, act_ptr(n, 2, pix), n->wqt[2], nullptr, g_out, B, H, W);
    std::swap(g_in, g_out);
    if ((st = wgrad<CW, CW, true>(n, act_ptr(n, 0, pix), g_in, act_ptr(n, 1, pix), B, H, W, 1)) != FE_OK) return st;
    conv32<false>(n, g_in, act_ptr(n, 1, pix), n->wqt[1], nullptr, g_out, B, H, W);
    std::swap(g_in, g_out);
    if ((st = wgrad<1, CW, true>(n, act_ptr(n, -1, pix), g_in, act_ptr(n, 0, pix), B, H, W, 0)) != FE_OK) return st;
    CNN_CUDA(n, cudaGetLastError());
    std::vector<double> lp(lb);
    CNN_CUDA(n, cudaMemcpyAsync(lp.data(), n->lpart, sizeof(double) * lb, cudaMemcpyDeviceToHost, n->s));
    CNN_CUDA(n, cudaStreamSynchronize(n->s));
    double s = 0.0;
    for (double v : lp) s += v;
    if (loss) *loss = s / (double)pix;
    return check_tc(n);
}

const float *stage(fe_cnn *n, const float *src, size_t count, int slot, fe_status *st) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, src) == cudaSuccess && (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged))
        return src;
    cudaGetLastError();
    float *dst = n->tmp + (size_t)slot * (n->cap_pix);
    if (cudaMemcpyAsync(dst, src, sizeof(float) * count, cudaMemcpyDefault, n->s) != cudaSuccess) {
        *st = cnn_err(n, FE_ECUDA, "staging copy failed");
        return nullptr;
    }
    return dst;
}

}  // namespace
}  // namespace fe

extern "C" {

fe_status fe_cnn_create(fe_cnn **out, unsigned long long seed, void *stream) {
    if (!out) return FE_EINVAL;
    *out = nullptr;
    if (cnn_prepare() != cudaSuccess) return FE_ECUDA;
    fe_cnn *n = new fe_cnn();
    n->s = static_cast<cudaStream_t>(stream);
    int off = 0;
    for (int l = 0; l < DEPTH; ++l) {
        n->woff.push_back(off);
        off += cin_of(l) * cout_of(l) * 9;
        n->boff.push_back(off);
        off += cout_of(l);
    }
    n->np = off;
    // He-style initialisation scaled down for the last layer (start near d = 0)
    std::vector<float> p(off, 0.f);
    std::vector<unsigned char> isw(off, 0);
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    for (int l = 0; l < DEPTH; ++l) {
        const float sd = std::sqrt(2.0f / (9.0f * cin_of(l))) * (l == DEPTH - 1 ? 0.1f : 1.0f);
        for (int e = 0; e < cin_of(l) * cout_of(l) * 9; ++e) {
            p[n->woff[l] + e] = sd * nd(rng);
            isw[n->woff[l] + e] = 1;
        }
    }
    auto fail = [&](fe_status s) {
        fe_cnn_destroy(n);
        return s;
    };
    if (cudaMalloc(&n->p, sizeof(float) * off) || cudaMalloc(&n->pq, sizeof(float) * off) ||
        cudaMalloc(&n->m, sizeof(float) * off) || cudaMalloc(&n->v, sizeof(float) * off) ||
        cudaMalloc(&n->g, sizeof(float) * off) || cudaMalloc(&n->is_w, off))
        return fail(FE_ENOMEM);
    for (int l = 0; l < DEPTH; ++l) {
        const size_t ne = (size_t)cin_of(l) * cout_of(l) * 9;
        if (cudaMalloc(&n->wl[l], sizeof(float) * ne) || cudaMalloc(&n->wt[l], sizeof(float) * ne)) return fail(FE_ENOMEM);
        if (cin_of(l) == CW && cout_of(l) == CW &&
            (cudaMalloc(&n->wqf[l], TC_B_BYTES) || cudaMalloc(&n->wqt[l], TC_B_BYTES)))
            return fail(FE_ENOMEM);
    }
    if (cudaMalloc(&n->tc_err, sizeof(int))) return fail(FE_ENOMEM);
    {
        int dev = 0;
        if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, dev))
            return fail(FE_ECUDA);
    }
    if (cudaMemset(n->tc_err, 0, sizeof(int)) ||
        cudaMemcpy(n->is_w, isw.data(), off, cudaMemcpyHostToDevice) || cudaMemset(n->m, 0, sizeof(float) * off) ||
        cudaMemset(n->v, 0, sizeof(float) * off) || cudaMemset(n->g, 0, sizeof(float) * off))
        return fail(FE_ECUDA);
    *out = n;
    fe_status st = fe_cnn_set_params(n, p.data());
    if (st != FE_OK) {
        *out = nullptr;
        return fail(st);
    }
    return FE_OK;
}

void fe_cnn_destroy(fe_cnn *n) {
    if (!n) return;
    if (n->s) cudaStreamSynchronize(n->s);
    cudaFree(n->p);
    cudaFree(n->pq);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->g);
    cudaFree(n->is_w);
    for (int l = 0; l < DEPTH; ++l) {
        cudaFree(n->wl[l]);
        cudaFree(n->wt[l]);
        cudaFree(n->wqf[l]);
        cudaFree(n->wqt[l]);
    }
    cudaFree(n->act);
    cudaFree(n->dact);
    cudaFree(n->part);
    cudaFree(n->tmp);
    cudaFree(n->lpart);
    cudaFree(n->tc_err);
    delete n;
}

int fe_cnn_num_params(const fe_cnn *n) { return n ? n->np : 0; }

const char *fe_cnn_last_error(const fe_cnn *n) { return n ? n->err.c_str() : ""; }

fe_status fe_cnn_set_params(fe_cnn *n, const float *params) {
    if (!n || !params) return FE_EINVAL;
    std::vector<float> p(n->np), pq(n->np);
    CNN_CUDA(n, cudaMemcpy(p.data(), params, sizeof(float) * n->np, cudaMemcpyDefault));
    for (int l = 0; l < DEPTH; ++l)
        for (int i = n->woff[l]; i < n->boff[l] + cout_of(l); ++i)
            pq[i] = i < n->boff[l] ? tc_round(1, p[i]) : p[i];
    CNN_CUDA(n, cudaMemcpy(n->p, p.data(), sizeof(float) * n->np, cudaMemcpyHostToDevice));
    CNN_CUDA(n, cudaMemcpy(n->pq, pq.data(), sizeof(float) * n->np, cudaMemcpyHostToDevice));
    return refresh_layouts(n);
}

fe_status fe_cnn_get_params(fe_cnn *n, float *params) {
    if (!n || !params) return FE_EINVAL;
    CNN_CUDA(n, cudaMemcpyAsync(params, n->p, sizeof(float) * n->np, cudaMemcpyDefault, n->s));
    CNN_CUDA(n, cudaStreamSynchronize(n->s));
    return FE_OK;
}

fe_status fe_cnn_forward(fe_cnn *n, const float *f, int B, int H, int W, float *u0, float *d) {
    if (!n || !f || B < 1 || H < 1 || W < 1) return FE_EINVAL;
    const size_t pix = (size_t)B * H * W;
    fe_status st = ensure_capacity(n, pix, 1);
    if (st != FE_OK) return st;
    const float *fd = stage(n, f, pix, 0, &st);
    if (!fd) return st;
    if ((st = forward(n, fd, B, H, W)) != FE_OK) return st;
    float *dout = act_ptr(n, 4, pix);
    if (u0) {
        cudaPointerAttributes a;
        const bool dev = cudaPointerGetAttributes(&a, u0) == cudaSuccess && a.type == cudaMemoryTypeDevice;
        cudaGetLastError();
        float *dst = dev ? u0 : n->tmp + n->cap_pix;
        output_kernel<<<(unsigned)std::min<size_t>((pix + 255) / 256, 4096), 256, 0, n->s>>>(fd, dout, dst, pix);
        CNN_CUDA(n, cudaGetLastError());
        if (!dev) CNN_CUDA(n, cudaMemcpyAsync(u0, dst, sizeof(float) * pix, cudaMemcpyDefault, n->s));
    }
    if (d) CNN_CUDA(n, cudaMemcpyAsync(d, dout, sizeof(float) * pix, cudaMemcpyDefault, n->s));
    CNN_CUDA(n, cudaStreamSynchronize(n->s));
    return check_tc(n);
}

fe_status fe_cnn_loss_grad(fe_cnn *n, const float *f, const float *u_target, int B, int H, int W, double *loss,
                           float *grad) {
    if (!n || !f || !u_target || B < 1 || H < 1 || W < 1) return FE_EINVAL;
    const size_t pix = (size_t)B * H * W;
    fe_status st = ensure_capacity(n, pix, grad_parts(n, B, H, W) * (CW * CW * 9 + CW));
    if (st != FE_OK) return st;
    const float *fd = stage(n, f, pix, 0, &st);
    if (!fd) return st;
    const float *ud = stage(n, u_target, pix, 1, &st);
    if (!ud) return st;
    if ((st = loss_grad(n, fd, ud, B, H, W, loss)) != FE_OK) return st;
    if (grad) {
        CNN_CUDA(n, cudaMemcpyAsync(grad, n->g, sizeof(float) * n->np, cudaMemcpyDefault, n->s));
        CNN_CUDA(n, cudaStreamSynchronize(n->s));
    }
    return FE_OK;
}

fe_status fe_cnn_train_step(fe_cnn *n, const float *f, const float *u_target, int B, int H, int W, float lr,
                            double *loss) {
    fe_status st = fe_cnn_loss_grad(n, f, u_target, B, H, W, loss, nullptr);
    if (st != FE_OK) return st;
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - std::pow(b1, (float)n->step), c2 = 1.f - std::pow(b2, (float)n->step);
    adam_kernel<<<(n->np + 255) / 256, 256, 0, n->s>>>(n->p, n->m, n->v, n->g, n->is_w, n->pq, n->np, lr, b1, b2, eps, c1, c2);
    CNN_CUDA(n, cudaGetLastError());
    return refresh_layouts(n);
}

}  // extern "C"
