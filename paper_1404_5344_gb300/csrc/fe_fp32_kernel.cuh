// Fused FP32 iPiano trial kernel for the FoE despeckling models (template;
// instantiated by fe_fp32.cu for the model with the I-divergence data term and
// by fe_fp32_comb.cu for the combined model in w = log u).
//
// One CTA handles one TY x TX output tile of one image and does, in shared
// memory, every step of one iPiano trial (Sec. II-C):
//
//   1. load u^n, u^{n-1}, g^n, f^2 on the tile + 6-pixel halo (symmetric
//      reflection at the image border) and form the inertial forward step
//      uhat = u^n - alpha g^n + beta (u^n - u^{n-1})             (update rule)
//   2. closed-form prox of alpha G, pointwise, on tile + halo 6 (Sec. II-C):
//      u = (uhat + sqrt(uhat^2 + 4(1+t l) t l f^2)) / (2 (1 + t l)), evaluated
//      as 2 t l f^2 / (sqrt(D) - uhat) when uhat < 0 (no cancellation)
//   3. forward filter bank z_i = k_i * u on tile + halo 3, 7x7 taps, FFMA
//   4. s_i = z_i / (1 + z_i^2) (zero outside the image), and the energy term
//      theta_i log(1 + z_i^2) on the tile; theta_i rho'(z_i) = 2 theta_i s_i,
//      and the factor 2 theta_i is folded into the adjoint weights
//   5. adjoint bank g = sum_i (2 theta_i K_i)^T s_i on the tile (correlation),
//      plus the transpose of the symmetric extension: values of K_i^T r on
//      the 3-pixel frame outside the image are folded back onto the pixels
//      they mirror
//   6. per-tile FP64 partial sums of F(u^{n+1}), G(u^{n+1}), <g^n, D>, |D|^2,
//      <D, u^n - u^{n-1}>; the last CTA of the image reduces them in a fixed
//      order and applies the backtracking test (accept / L <- eta L).
//
// Filters are processed in groups of G = 4 so that the 4 response planes of
// the tile + halo fit in shared memory; the adjoint accumulators stay in
// registers across groups.
//
// Two tile shapes, T x T output pixels per CTA, each also split by filter
// group over a 4-CTA thread-block cluster (CL = 4; the autotuner of the host
// side picks one of the four per context):
//   T = 64: 256 threads, two CTAs per SM so that one CTA's barrier waits are
//           covered by the other; forward units of 1 column x 10 rows x 4
//           filters over the 70 x 70 response region (490 units, two rounds);
//           adjoint units of 4 x 4 output pixels (one per thread)
//   T = 32: 128 threads, four CTAs per SM, for images too small to fill the
//           GPU with 64 x 64 tiles; forward units of 1 column x 13 rows over
//           a 39-row (one padding row) x 38-column region (114 units, one
//           round); adjoint units of 2 x 4 output pixels (one per thread)
// The weights of a filter group (forward taps, adjoint taps, theta) are
// staged in shared memory, double-buffered: asynchronous copies (cp.async)
// fetch the next group's weights while the current group runs.  A forward
// unit slides its column window over the 7 kernel columns, reading weight
// vectors as uniform 128-bit shared loads.  An adjoint unit reads each window
// row with three LDS.128 and holds each filter's 49 weights in registers
// while its window rows stream through.  The frame of the symmetric-boundary
// transpose (the 3-pixel ring outside the image) is computed per group as
// strip tasks and folded onto the pixels it mirrors after the last group.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cooperative_groups.h>

#include "fe_internal.cuh"
#include "fe_tile_common.cuh"

namespace fe {
namespace {

constexpr int G = 4;  // filters per group (response planes held in shared memory)

template <int T>
struct Cfg;
template <>
struct Cfg<64> {
    static constexpr int NT = 256, MINB = 2, FWD_ROWS = 10, AUR = 4;
    static constexpr int SU_LD = 87;  // 10*87 = 70 (mod 32): unit rows wrap without bank conflicts
    static constexpr int SR_LD = 72;
};
template <>
struct Cfg<32> {
    static constexpr int NT = 128, MINB = 4, FWD_ROWS = 13, AUR = 2;
    static constexpr int SU_LD = 62;  // 13*62 = 6 (mod 32), 38 = 6 (mod 32): as above
    static constexpr int SR_LD = 40;
};

template <int T>
struct Geo {
    using C = Cfg<T>;
    static constexpr int TY = T, TX = T, NT = C::NT, MINB = C::MINB;
    static constexpr int FWD_ROWS = C::FWD_ROWS, AUR = C::AUR, SU_LD = C::SU_LD, SR_LD = C::SR_LD;
    static constexpr int R3Y = TY + 6, R3X = TX + 6;  // response region (tile + 3)
    // rows the forward units cover: R3Y rounded up to whole units (the extra
    // row is computed from clamped loads and never read)
    static constexpr int R3YA = (R3Y + FWD_ROWS - 1) / FWD_ROWS * FWD_ROWS;
    static constexpr int R6Y = R3YA + 6, R6X = TX + 12;  // u^{n+1} region (tile + 6, padded)
    static constexpr int NWARP = NT / 32;
    static constexpr int FWD_WIN = FWD_ROWS + KS - 1;       // column window of a forward unit
    static constexpr int FWD_UNITS = R3X * (R3YA / FWD_ROWS);
    static constexpr int AUX = TX / 4;                      // adjoint units per tile row
    static constexpr int ADJ_UNITS = (TY / AUR) * AUX;
    static constexpr int RING = 2 * 3 * R3X + 2 * 3 * TY;   // frame positions
    // sR follows sU: round sU up to 4 floats so that sR is 16-byte aligned
    // for the adjoint's 128-bit loads
    static constexpr size_t SM_U = ((size_t)R6Y * SU_LD + 3) / 4 * 4;
    static constexpr size_t SM_R = (size_t)G * R3YA * SR_LD;
    // one group's weights: forward taps (tap-major, G per tap), adjoint taps
    // (filter-major, KT_PAD per filter), theta; two buffers
    static constexpr int WB_F = 0, WB_A = KT * G, WB_T = WB_A + G * KT_PAD, WBUF = WB_T + G;
    static constexpr size_t SM_W = 2 * (size_t)WBUF;
    static constexpr size_t SM_FLOATS = SM_U + SM_R + SM_W;
    static constexpr size_t SM_BYTES = SM_FLOATS * 4 + (size_t)NWARP * NRED * 8;
    static_assert(NT == ADJ_UNITS, "one adjoint unit per thread");
    static_assert(SU_LD >= R6X && SR_LD >= R3X, "row pitches hold a region row");
    static_assert(SR_LD % 4 == 0 && SR_LD >= 4 * (AUX - 1) + 12, "adjoint window loads stay in the row");
    static_assert((AUR - 1) + (TY - AUR) + KS <= R3Y, "adjoint windows stay in the response region");
    static_assert(SM_U % 4 == 0 && SM_R % 4 == 0 && (SR_LD * R3YA) % 4 == 0,
                  "every plane and row of sR starts on a 16-byte boundary");
    static_assert(SM_FLOATS % 2 == 0, "double scratch alignment");
    static_assert(WB_A % 4 == 0 && WB_T % 4 == 0 && WBUF % 4 == 0 && (SM_U + SM_R) % 4 == 0,
                  "weight buffers and their parts start on 16-byte boundaries");
    static_assert(KT * G / 4 + G * KT_PAD / 4 + 1 <= NT, "one 16-byte copy per thread stages a group");
    static_assert(MINB * (SM_BYTES + 1024) <= 228 * 1024, "MINB CTAs per SM");
    static_assert(RING <= SM_R, "the frame ring reuses sR");
    static_assert(3 * R3Y <= NT && 3 * TX <= NT, "one frame-strip task per thread and strip");
};

constexpr float LN2 = 0.69314718055994530942f;

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Stage the weights of filter group grp in wb (one 16-byte copy per thread):
// forward taps wf[t * NFMAX + grp G .. + G) -> wb[WB_F + t G ..], adjoint taps
// wa[(grp G + i) KT_PAD + t] -> wb[WB_A + i KT_PAD + t], theta -> wb[WB_T ..].
template <int T>
__device__ __forceinline__ void stage_weights(float *wb, const KParams &p, int grp, int tid) {
    using Q = Geo<T>;
    constexpr int NA4 = G * KT_PAD / 4;  // float4 of adjoint taps
    static_assert(G == 4, "one float4 of forward taps per tap");
    if (tid < KT)
        cp_async16(wb + Q::WB_F + tid * G, p.wf + tid * NFMAX + grp * G);
    else if (tid < KT + NA4)
        cp_async16(wb + Q::WB_A + (tid - KT) * 4, p.wa + (size_t)grp * G * KT_PAD + (tid - KT) * 4);
    else if (tid == KT + NA4)
        cp_async16(wb + Q::WB_T, p.theta + grp * G);
    cp_async_commit();
}

template <int T>
__device__ __forceinline__ int pos_to_ring(int pr, int pc) {
    constexpr int TY = T, TX = T, R3X = T + 6;
    if (pr < 3) return pr * R3X + pc;
    if (pr >= TY + 3) return 3 * R3X + (pr - TY - 3) * R3X + pc;
    if (pc < 3) return 6 * R3X + (pr - 3) * 3 + pc;
    return 6 * R3X + 3 * TY + (pr - 3) * 3 + (pc - TX - 3);
}

// Forward bank of one unit (1 column x FWD_ROWS rows x G filters of group
// grp) and its epilogue: s_i = z_i / (1 + z_i^2) into sR (theta_i rho'(z_i) =
// 2 theta_i s_i; the adjoint weights carry 2 theta_i), theta_i log2(1 + z_i^2)
// summed over the unit's tile pixels.  MASK: some pixel of the unit lies outside the image (a
// run-time flag: one inlined copy of this function instead of two keeps the
// kernel's code small enough for the instruction cache, measured 7 % faster).
template <int T, int MODE>
__device__ __forceinline__ float forward_unit(const float *__restrict__ sU, float *__restrict__ sR,
                                              const float *__restrict__ wb, int c, int rb, int y0, int x0, int H,
                                              int W, bool MASK) {
    using Q = Geo<T>;
    constexpr int FWD_ROWS = Q::FWD_ROWS, FWD_WIN = Q::FWD_WIN, SU_LD = Q::SU_LD, SR_LD = Q::SR_LD;
    constexpr int TY = Q::TY, TX = Q::TX, R3YA = Q::R3YA;
    float z[FWD_ROWS][G];
    const float *ucol = sU + rb * FWD_ROWS * SU_LD + c;
    const float *wcol = wb + Q::WB_F;
    if constexpr (FWD_ROWS <= 10) {
    // accumulators of filter pairs (0, 1) and (2, 3) as packed FP32 pairs:
    // one fma.rn.f32x2 updates both filters of a pair at a row (each element
    // rounded as the scalar FMA, in the same order), with the window value
    // duplicated into both halves of its operand; half the FMA instructions
    // of the scalar form (the 13-row units of the 32 x 32 tile keep the
    // scalar form: their packed window does not fit the register budget)
    static_assert(G == 4, "two filter pairs per group");
    uint64_t z2[FWD_ROWS][2];
#pragma unroll
    for (int r = 0; r < FWD_ROWS; ++r) z2[r][0] = z2[r][1] = 0ull;
#pragma unroll 1
    for (int bb = 0; bb < KS; ++bb) {
        uint64_t vd[FWD_WIN];
#pragma unroll
        for (int r = 0; r < FWD_WIN; ++r) {
            const float v = ucol[r * SU_LD + bb];
            vd[r] = f2_pack(v, v);
        }
#pragma unroll
        for (int aa = 0; aa < KS; ++aa) {
            const float4 w0 = *reinterpret_cast<const float4 *>(wcol + (aa * KS + bb) * G);
            const uint64_t w01 = f2_pack(w0.x, w0.y), w23 = f2_pack(w0.z, w0.w);
#pragma unroll
            for (int r = 0; r < FWD_ROWS; ++r) z2[r][0] = f2_fma(w01, vd[r + aa], z2[r][0]);
#pragma unroll
            for (int r = 0; r < FWD_ROWS; ++r) z2[r][1] = f2_fma(w23, vd[r + aa], z2[r][1]);
        }
    }
#pragma unroll
    for (int r = 0; r < FWD_ROWS; ++r) {
        f2_unpack(z2[r][0], z[r][0], z[r][1]);
        f2_unpack(z2[r][1], z[r][2], z[r][3]);
    }
    } else {
#pragma unroll
    for (int r = 0; r < FWD_ROWS; ++r)
#pragma unroll
        for (int i = 0; i < G; ++i) z[r][i] = 0.f;
#pragma unroll 1
    for (int bb = 0; bb < KS; ++bb) {
        float v[FWD_WIN];
#pragma unroll
        for (int r = 0; r < FWD_WIN; ++r) v[r] = ucol[r * SU_LD + bb];
#pragma unroll
        for (int aa = 0; aa < KS; ++aa) {
            const float4 w0 = *reinterpret_cast<const float4 *>(wcol + (aa * KS + bb) * G);
            const float w[G] = {w0.x, w0.y, w0.z, w0.w};
#pragma unroll
            for (int i = 0; i < G; ++i)
#pragma unroll
                for (int r = 0; r < FWD_ROWS; ++r) z[r][i] = fmaf(w[i], v[r + aa], z[r][i]);
        }
    }
    }
    float th[G];
#pragma unroll
    for (int i = 0; i < G; ++i) th[i] = wb[Q::WB_T + i];
    const int x = x0 - 3 + c;
    const bool colin = x >= 0 && x < W, colint = c >= 3 && c < 3 + TX;
    float fsum = 0.f;
#pragma unroll
    for (int r = 0; r < FWD_ROWS; ++r) {
        const int pr = rb * FWD_ROWS + r;
        const int y = y0 - 3 + pr;
        const bool inimg = !MASK || (colin && y >= 0 && y < H);
        const bool inner = colint && pr >= 3 && pr < 3 + TY && (!MASK || inimg);
        float psum = 0.f;
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const float zz = z[r][i];
            const float q = fmaf(zz, zz, 1.0f);
            if (MODE != MODE_ENERGY_EXT) {
                float rv = zz * rcp_ftz(q);
                if (MASK && !inimg) rv = 0.0f;
                sR[(i * R3YA + pr) * SR_LD + c] = rv;
            }
            psum = fmaf(th[i], lg2_ftz(q), psum);
        }
        if (inner) fsum += psum;
    }
    return fsum * LN2;
}

// MODEL 0: Eq. variant, iterate u.  MODEL 1: Eq. newmodel, iterate w = log u
// (the filter bank sees u = e^w; grad_w F = e^w (.) sum_i theta_i K_i^T rho'(z_i);
// the prox is prox_w).
// CL > 1: the tile is split over a thread-block cluster of CL CTAs by filter
// group (rank r takes groups r, r + CL, ...), for images too small to fill
// the GPU otherwise.  Every rank recomputes the prologue (only rank 0 writes
// u^{n+1} and keeps the step sums); after the groups each rank leaves its
// partial K^T r, frame values and F sum in its shared memory, rank 0 adds
// the other ranks' partials in rank order through distributed shared memory
// and finishes the tile.  Launched with a cluster dimension of CL.
template <int MODE, int T, int MODEL, int CL>
__global__ void __launch_bounds__(Geo<T>::NT, Geo<T>::MINB) fp32_tile_kernel(const KParams p) {
    using Q = Geo<T>;
    constexpr int TY = Q::TY, TX = Q::TX, NT = Q::NT, R3Y = Q::R3Y, R3X = Q::R3X, R3YA = Q::R3YA;
    constexpr int R6Y = Q::R6Y, R6X = Q::R6X, SU_LD = Q::SU_LD, SR_LD = Q::SR_LD, AUR = Q::AUR;
    constexpr int FWD_ROWS = Q::FWD_ROWS, FWD_UNITS = Q::FWD_UNITS;
    constexpr size_t SM_U = Q::SM_U, SM_R = Q::SM_R;
    extern __shared__ __align__(16) float smem[];
    float *sU = smem;
    float *sR = sU + SM_U;
    float *sW = sR + SM_R;  // two weight buffers
    double *sRed = reinterpret_cast<double *>(sW + Q::SM_W);
    __shared__ int sLast;

    const int tid = threadIdx.x;
    int rank = 0;
    if constexpr (CL > 1) rank = (int)cooperative_groups::this_cluster().block_rank();
    // persistent launches (MODE_PTRIAL, one CTA per tile): the CTA runs tiles
    // until every image has stopped, taking each from the per-image counters;
    // otherwise the launch's block index names the one tile
    constexpr bool PERSIST = MODE == MODE_PTRIAL;
    constexpr bool TRIAL = MODE == MODE_TRIAL || PERSIST;
    static_assert(!PERSIST || CL == 1, "persistent launches run tiles of one CTA");
    __shared__ int sTask;
    int pref = p.nimg > 0 ? (int)blockIdx.x % p.nimg : 0;  // image of the last tile taken
    for (;;) {
        int gtile;
        if constexpr (PERSIST) {
            __syncthreads();  // the previous tile is done with shared memory and sTask
            if (tid < 32) {
                const int t = persist_grab(p, pref);
                if (tid == 0) sTask = t;
            }
            __syncthreads();
            gtile = sTask;  // claimed with an acquire fence (persist_grab)
            if (gtile < 0) break;
        } else {
            const int bt = p.tile0 + (int)blockIdx.x / CL;
            gtile = p.order ? p.order[bt] : bt;
        }
        const TileDesc td = p.tiles[gtile];
        const int img = td.img;
        const ImgDesc im = p.imgs[img];
        ImgState *st = p.st + img;
        const int H = im.H, W = im.W, y0 = td.y0, x0 = td.x0;

        bool active = true;
        int gcur_out = 0;
        if (TRIAL) {
            active = (st->done == 0) && (st->n < st->target);
            gcur_out = st->gcur ^ 1;
        }

        if (active) {
            // ---- 1+2: inertial step and prox on tile + 6 ---------------------
            // per-thread sums: compensated FP32 for F and G (large terms), plain
            // FP32 for the small step-test terms
            Sum2 accF{0.f, 0.f}, accG{0.f, 0.f};
            float accGD = 0.f, accDD = 0.f, accDP = 0.f;
            {
                int cur = 0, gcur = 0;
                float a = 0.f, b = 0.f, tl = 0.f;
                const float l1 = (float)im.lambda1, l2 = (float)im.lambda;  // combined model
                if (TRIAL) {
                    cur = st->cur;
                    gcur = st->gcur;
                    const double alpha = st->alpha;
                    a = (float)alpha;
                    b = (float)p.beta;
                    tl = (float)(alpha * im.lambda);
                }
                const float *uc = (TRIAL || MODE == MODE_INIT) ? im.u[cur] : p.u_ext;
                const float *upv = im.u[(cur + 2) % 3];
                const float *gc = im.g[gcur];
                float *un = im.u[(cur + 1) % 3];
                const float *f2p = im.f2;
                // UNR positions per thread at a time: their loads are issued
                // together before the arithmetic (positions past the region
                // load the last one's values and are skipped); the 32 x 32
                // tile takes one (its register budget is smaller)
                constexpr int UNR = T == 64 ? 4 : 1, NPIX = R6Y * R6X;
                for (int base = 0; base < NPIX; base += UNR * NT) {
                    size_t offk[UNR];
                    float u0k[UNR], u1k[UNR], g0k[UNR], f2k[UNR];
#pragma unroll
                    for (int k = 0; k < UNR; ++k) {
                        const int idx = base + k * NT + tid;
                        const int idc = idx < NPIX ? idx : NPIX - 1;
                        const int ry = idc / R6X, rx = idc - ry * R6X;
                        offk[k] = (size_t)reflect(y0 - 6 + ry, H) * W + reflect(x0 - 6 + rx, W);
                        f2k[k] = __ldg(f2p + offk[k]);
                        if (TRIAL) {
                            // L2 loads: a persistent launch rewrites these planes while it runs
                            u0k[k] = __ldcg(uc + offk[k]);
                            u1k[k] = __ldcg(upv + offk[k]);
                            g0k[k] = __ldcg(gc + offk[k]);
                        } else {
                            u0k[k] = __ldg(uc + offk[k]);
                            u1k[k] = g0k[k] = 0.f;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < UNR; ++k) {
                        const int idx = base + k * NT + tid;
                        if (idx >= NPIX) continue;
                        const int ry = idx / R6X, rx = idx - ry * R6X;
                        const int y = y0 - 6 + ry, x = x0 - 6 + rx;
                        const size_t off = offk[k];
                        const bool inner = ry >= 6 && ry < 6 + TY && rx >= 6 && rx < 6 + TX && y < H && x < W;
                        const float u0 = u0k[k], f2 = f2k[k];
                        float v;
                        if (TRIAL) {
                            const float u_1 = u1k[k], g0 = g0k[k];
                            const float dprev = u0 - u_1;
                            const float uhat = fmaf(-a, g0, fmaf(b, dprev, u0));
                            v = MODEL == 0 ? prox_g(uhat, f2, tl) : prox_w(uhat, f2, a, l1, l2);
                            if (inner && rank == 0) {
                                un[off] = v;
                                const float d = v - u0;
                                accGD = fmaf(g0, d, accGD);
                                accDD = fmaf(d, d, accDD);
                                accDP = fmaf(d, dprev, accDP);
                                sum2_add(accG, MODEL == 0 ? v * v - 2.0f * f2 * logf(v) : data_w(v, f2, l1, l2));
                            }
                        } else {
                            v = u0;
                            if (inner && rank == 0)
                                sum2_add(accG, MODEL == 0 ? v * v - 2.0f * f2 * logf(v) : data_w(v, f2, l1, l2));
                        }
                        sU[ry * SU_LD + rx] = MODEL == 0 ? v : expf(v);  // the bank sees u
                    }
                }
            }

            float acc[AUR][4];
    #pragma unroll
            for (int i = 0; i < AUR; ++i)
    #pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
            // frame values of this thread's strip tasks (left, right, top, bottom)
            float fr[4] = {0.f, 0.f, 0.f, 0.f};
            const int aux = tid % Q::AUX, auy = tid / Q::AUX;  // adjoint unit of this thread
            const bool sLft = x0 == 0, sTop = y0 == 0, sRgt = x0 + TX > W - 3, sBot = y0 + TY > H - 3;
            const bool border = sLft || sTop || sRgt || sBot;

            const int ngrp = p.nfp / G;
            if (rank < ngrp) stage_weights<T>(sW, p, rank, tid);
            for (int grp = rank, gi = 0; grp < ngrp; grp += CL, ++gi) {
                const float *wb = sW + (gi & 1) * Q::WBUF;
                cp_async_wait_all();  // this thread's copies of the group's weights
                __syncthreads();      // sU / weights ready; previous group's sR and weight reads done
                // the next group's weights into the other buffer (its last readers,
                // the previous group, finished before the barrier above)
                if (grp + CL < ngrp) stage_weights<T>(sW + ((gi + 1) & 1) * Q::WBUF, p, grp + CL, tid);
                // ---- 3+4: forward bank and potential on tile + 3 -------------
                for (int unit = tid; unit < FWD_UNITS; unit += NT) {
                    const int c = unit % R3X, rb = unit / R3X;
                    const int x = x0 - 3 + c, ylo = y0 - 3 + rb * FWD_ROWS;
                    const bool full = x >= 0 && x < W && ylo >= 0 && ylo + FWD_ROWS <= H;
                    const float fs = forward_unit<T, MODE>(sU, sR, wb, c, rb, y0, x0, H, W, !full);
                    sum2_add(accF, fs);
                }
                if (MODE == MODE_ENERGY_EXT) continue;
                __syncthreads();  // sR complete

                // ---- 5: adjoint bank on the tile (AUR x 4 unit per thread) -----
                for (int i = 0; i < G; ++i) {
                    const float *wrow = wb + Q::WB_A + i * KT_PAD;
                    float kw[KT_PAD];
    #pragma unroll
                    for (int j = 0; j < KT_PAD / 4; ++j) {
                        const float4 t = reinterpret_cast<const float4 *>(wrow)[j];
                        kw[4 * j] = t.x;
                        kw[4 * j + 1] = t.y;
                        kw[4 * j + 2] = t.z;
                        kw[4 * j + 3] = t.w;
                    }
                    const float *Ri = sR + (size_t)i * R3YA * SR_LD + (AUR * auy) * SR_LD + 4 * aux;
    #pragma unroll
                    for (int rr = 0; rr < AUR + KS - 1; ++rr) {
                        const float4 a0 = *reinterpret_cast<const float4 *>(Ri + rr * SR_LD);
                        const float4 a1 = *reinterpret_cast<const float4 *>(Ri + rr * SR_LD + 4);
                        const float4 a2 = *reinterpret_cast<const float4 *>(Ri + rr * SR_LD + 8);
                        const float v[12] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w};
    #pragma unroll
                        for (int pp = 0; pp < AUR; ++pp) {
                            const int aa = rr - pp;
                            if (aa < 0 || aa >= KS) continue;
    #pragma unroll
                            for (int bb = 0; bb < KS; ++bb)
    #pragma unroll
                                for (int q = 0; q < 4; ++q) acc[pp][q] = fmaf(kw[aa * KS + bb], v[q + bb], acc[pp][q]);
                        }
                    }
                }
                // ---- 5b: K^T s on the frame outside the image (border tiles) --
                // frame value at (j, jx) = sum_i sum_ab 2 theta_i k_i[a][b]
                // s_i(j - 3 + a, jx - 3 + b), s_i zero off-image, so only the taps
                // that reach into the image count.  The frame is cut into strips
                // of depth d = 1..3, one (line, depth) task per thread and strip,
                // with static tap loops: the left / right strips run over the
                // ring's rows l in [0, R3Y) (axis_pos maps l to the image row j,
                // the corner rows included), the top / bottom strips over the
                // tile's columns.
                if (border) {
                    if (tid < 3 * R3Y && (sLft || sRgt)) {
                        // depth fastest: the lanes of a load read 3 columns of ~11
                        // rows (a column of 32 rows would hit every bank 8 times:
                        // SR_LD = 8 mod 32)
                        const int d = 1 + tid % 3, l = tid / 3;
                        int j;
                        if (axis_pos(l, y0, TY, H, j)) {
                            // rows of s inside the image and in the response region;
                            // sR row of tap a: j - y0 + a
                            const int alo = max(max(0, 3 - j), y0 - j), ahi = min(min(KS, H + 3 - j), R3Y + y0 - j);
                            const int r0 = j - y0;
                            if (sLft) {
                                // frame column -d: taps b >= 3 + d, sR column b - d
                                float sv = 0.f;
    #pragma unroll
                                for (int i = 0; i < G; ++i) {
                                    const float *wrow = wb + Q::WB_A + i * KT_PAD;
                                    const float *Ri = sR + (size_t)i * R3YA * SR_LD;
    #pragma unroll
                                    for (int aa = 0; aa < KS; ++aa) {
                                        if (aa < alo || aa >= ahi) continue;
    #pragma unroll
                                        for (int bb = 4; bb < KS; ++bb)
                                            if (bb >= 3 + d)
                                                sv = fmaf(wrow[aa * KS + bb], Ri[(r0 + aa) * SR_LD + bb - d], sv);
                                    }
                                }
                                fr[0] += sv;
                            }
                            if (sRgt && W - d >= x0 && W - d < x0 + TX) {
                                // frame column W - 1 + d: taps b <= 3 - d, sR column W - x0 - 1 + d + b
                                float sv = 0.f;
    #pragma unroll
                                for (int i = 0; i < G; ++i) {
                                    const float *wrow = wb + Q::WB_A + i * KT_PAD;
                                    const float *Ri = sR + (size_t)i * R3YA * SR_LD + (W - x0 - 1 + d);
    #pragma unroll
                                    for (int aa = 0; aa < KS; ++aa) {
                                        if (aa < alo || aa >= ahi) continue;
    #pragma unroll
                                        for (int bb = 0; bb < 3; ++bb)
                                            if (bb <= 3 - d) sv = fmaf(wrow[aa * KS + bb], Ri[(r0 + aa) * SR_LD + bb], sv);
                                    }
                                }
                                fr[1] += sv;
                            }
                        }
                    }
                    if (tid < 3 * TX && (sTop || sBot)) {
                        const int d = 1 + tid / TX, c = tid - (d - 1) * TX;  // image column x0 + c
                        if (x0 + c < W) {
                            if (sTop) {
                                // frame row -d: taps a >= 3 + d, sR row a - d, sR column c + b
                                float sv = 0.f;
    #pragma unroll
                                for (int i = 0; i < G; ++i) {
                                    const float *wrow = wb + Q::WB_A + i * KT_PAD;
                                    const float *Ri = sR + (size_t)i * R3YA * SR_LD + c;
    #pragma unroll
                                    for (int aa = 4; aa < KS; ++aa) {
                                        if (aa < 3 + d) continue;
    #pragma unroll
                                        for (int bb = 0; bb < KS; ++bb)
                                            sv = fmaf(wrow[aa * KS + bb], Ri[(aa - d) * SR_LD + bb], sv);
                                    }
                                }
                                fr[2] += sv;
                            }
                            if (sBot && H - d >= y0 && H - d < y0 + TY) {
                                // frame row H - 1 + d: taps a <= 3 - d, sR row H - y0 - 1 + d + a
                                float sv = 0.f;
    #pragma unroll
                                for (int i = 0; i < G; ++i) {
                                    const float *wrow = wb + Q::WB_A + i * KT_PAD;
                                    const float *Ri = sR + (size_t)i * R3YA * SR_LD + (H - y0 - 1 + d) * SR_LD + c;
    #pragma unroll
                                    for (int aa = 0; aa < 3; ++aa) {
                                        if (aa > 3 - d) continue;
    #pragma unroll
                                        for (int bb = 0; bb < KS; ++bb) sv = fmaf(wrow[aa * KS + bb], Ri[aa * SR_LD + bb], sv);
                                    }
                                }
                                fr[3] += sv;
                            }
                        }
                    }
                }
            }

            if constexpr (CL > 1) {
                // ---- combine the ranks' partials at rank 0 (distributed shared memory)
                auto cluster = cooperative_groups::this_cluster();
                __syncthreads();  // this CTA's sR reads are done
                constexpr int NA = AUR * 4;
                constexpr int NFR = 4;
                float *part = sR;  // per thread: NA adjoint sums, NFR frame values, F (s, c)
                static_assert(NT * (NA + NFR + 2) <= (int)SM_R, "partials fit in sR");
    #pragma unroll
                for (int pp = 0; pp < AUR; ++pp)
    #pragma unroll
                    for (int q = 0; q < 4; ++q) part[tid * NA + pp * 4 + q] = acc[pp][q];
    #pragma unroll
                for (int k = 0; k < NFR; ++k) part[NT * NA + tid * NFR + k] = fr[k];
                part[NT * (NA + NFR) + 2 * tid] = accF.s;
                part[NT * (NA + NFR) + 2 * tid + 1] = accF.c;
                cluster.sync();  // every rank's partials are visible in the cluster
                if (rank == 0) {
                    for (int r = 1; r < CL; ++r) {
                        const float *rp = cluster.map_shared_rank(part, r);
    #pragma unroll
                        for (int pp = 0; pp < AUR; ++pp)
    #pragma unroll
                            for (int q = 0; q < 4; ++q) acc[pp][q] += rp[tid * NA + pp * 4 + q];
    #pragma unroll
                        for (int k = 0; k < NFR; ++k) fr[k] += rp[NT * NA + tid * NFR + k];
                        accF = sum2_merge(accF, Sum2{rp[NT * (NA + NFR) + 2 * tid],
                                                    rp[NT * (NA + NFR) + 2 * tid + 1]});
                    }
                }
                cluster.sync();  // rank 0 has read the other ranks' shared memory
            }

            if (MODE != MODE_ENERGY_EXT && rank == 0) {
                // ---- fold the frame back onto the pixels it mirrors ----------
                if (border) {
                    __syncthreads();  // all sR reads done; reuse sR for the ring
                    // each ring slot is written by the one task that computed it
                    // (slots of lines outside this tile's frame are never read)
                    if (tid < 3 * R3Y) {
                        const int d = 1 + tid % 3, l = tid / 3;
                        if (sLft) sR[pos_to_ring<T>(l, 3 - d)] = fr[0];
                        if (sRgt) sR[pos_to_ring<T>(l, TX + 2 + d)] = fr[1];
                    }
                    if (tid < 3 * TX) {
                        const int d = 1 + tid / TX, c = tid - (d - 1) * TX;
                        if (sTop) sR[pos_to_ring<T>(3 - d, c + 3)] = fr[2];
                        if (sBot) sR[pos_to_ring<T>(TY + 2 + d, c + 3)] = fr[3];
                    }
                    __syncthreads();
                }
                {
                    float *gout;
                    if (MODE == MODE_GRAD_EXT)
                        gout = p.g_ext;
                    else if (MODE == MODE_INIT)
                        gout = im.g[0];
                    else
                        gout = im.g[gcur_out];
    #pragma unroll
                    for (int pp = 0; pp < AUR; ++pp) {
                        const int y = y0 + AUR * auy + pp;
                        if (y >= H) continue;
    #pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int x = x0 + 4 * aux + q;
                            if (x >= W) continue;
                            float gv = acc[pp][q];  // (K^T r)(y, x); the fold follows
                            if (border && (y < 3 || y >= H - 3 || x < 3 || x >= W - 3)) {
                                // frame positions that the symmetric extension maps onto
                                // (y, x): at most one per axis (H, W >= 8); scalars, so
                                // that nothing is indexed dynamically (local memory)
                                const int oy = y - y0 + 3, ox = x - x0 + 3;
                                const int qy = y < 3 ? 2 - y : (y >= H - 3 ? TY + 2 + H - y : -1);  // j = -y-1 | 2H-1-y
                                const int qx = x < 3 ? 2 - x : (x >= W - 3 ? TX + 2 + W - x : -1);
                                if (qx >= 0) gv += sR[pos_to_ring<T>(oy, qx)];
                                if (qy >= 0) {
                                    gv += sR[pos_to_ring<T>(qy, ox)];
                                    if (qx >= 0) gv += sR[pos_to_ring<T>(qy, qx)];
                                }
                            }
                            // combined model: grad_w F = e^w (.) K^T r, u = e^w from sU
                            if (MODEL == 1) gv *= sU[(y - y0 + 6) * SU_LD + (x - x0 + 6)];
                            gout[(size_t)y * W + x] = gv;
                        }
                    }
                }
            }

            // ---- 6: per-tile FP64 partial sums, last-CTA decision -------------
            if (rank == 0) {
                const Sum2 vals[NRED] = {accF, accG, {accGD, 0.f}, {accDD, 0.f}, {accDP, 0.f}};
                tile_finish<NT>(p, MODE, gtile, img, im, st, vals, sRed, &sLast);
            }
        }
        if constexpr (!PERSIST) break;
    }

    // ---- loop control: the last rank-0 CTA of the launch -------------------
    if constexpr (PERSIST) persist_exit(p, gridDim.x);
    if (MODE == MODE_TRIAL && rank == 0) loop_control(p, gridDim.x / CL);
}

template <int T, int MODEL, int CL = 1>
cudaError_t prepare_tile() {
    const int b = (int)Geo<T>::SM_BYTES;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(fp32_tile_kernel<MODE_TRIAL, T, MODEL, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)) !=
        cudaSuccess)
        return e;
    if constexpr (CL == 1)
        if ((e = cudaFuncSetAttribute(fp32_tile_kernel<MODE_PTRIAL, T, MODEL, 1>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, b)) != cudaSuccess)
            return e;
    if ((e = cudaFuncSetAttribute(fp32_tile_kernel<MODE_INIT, T, MODEL, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(fp32_tile_kernel<MODE_GRAD_EXT, T, MODEL, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  b)) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(fp32_tile_kernel<MODE_ENERGY_EXT, T, MODEL, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}

// ngrid = tiles; CL CTAs per tile, launched as clusters of CL
template <int T, int MODEL, int CL = 1>
cudaError_t launch_tile(int mode, const KParams &p, int ngrid, cudaStream_t s) {
    const void *fn;
    switch (mode) {
        case MODE_TRIAL: fn = reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_TRIAL, T, MODEL, CL>); break;
        case MODE_INIT: fn = reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_INIT, T, MODEL, CL>); break;
        case MODE_GRAD_EXT: fn = reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_GRAD_EXT, T, MODEL, CL>); break;
        case MODE_ENERGY_EXT:
            fn = reinterpret_cast<const void *>(&fp32_tile_kernel<MODE_ENERGY_EXT, T, MODEL, CL>);
            break;
        default: return cudaErrorInvalidValue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ngrid * CL);
    cfg.blockDim = dim3(Geo<T>::NT);
    cfg.dynamicSmemBytes = Geo<T>::SM_BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (CL > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    void *args[] = {const_cast<KParams *>(&p)};
    return cudaLaunchKernelExC(&cfg, fn, args);
}


}  // namespace
}  // namespace fe
