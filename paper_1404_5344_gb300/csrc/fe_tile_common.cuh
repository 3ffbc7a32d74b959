// Device code shared by the tile kernels (FP32 and tensor-core forms):
// boundary reflection, the closed-form prox, the backtracking decision, the
// per-tile FP64 partial sums with the last-CTA reduction, and the loop
// control run by the last CTA of a trial launch.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fe_internal.cuh"

namespace fe {
namespace {

// Approximate reciprocal and base-2 logarithm on the special-function unit
// with subnormal inputs and results flushed to zero.  The response epilogues
// apply them to q = 1 + z^2 >= 1, where the flush never triggers, so they give
// the same values as the non-flushing forms without the extra instructions
// those spend on subnormal operands.
__device__ __forceinline__ float rcp_ftz(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_ftz(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Packed FP32 pairs (two floats in one 64-bit register, element 0 in the low
// half): one fma / mul / sub instruction operates on both elements, each with
// its own IEEE round-to-nearest rounding (the results equal two scalar ops).
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// BF16 pair of (lo, hi) rounded to nearest even, lo in the low 16 bits
__device__ __forceinline__ uint32_t bf16x2_rn(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// Symmetric (half-sample) reflection for j in [-6, n+6) when n >= 6; indices
// further out only feed responses outside the image and are clamped.
__device__ __forceinline__ int reflect(int j, int n) {
    j = j < 0 ? -j - 1 : j;
    j = j >= n ? 2 * n - 1 - j : j;
    return min(max(j, 0), n - 1);
}

// Closed-form prox of t*G at uhat (Sec. II-C), tl = t * lambda: the positive
// root of (1+tl) u^2 - uhat u - tl f^2 = 0, as 2 tl f^2 / (sqrt(D) - uhat) when
// uhat < 0 (no cancellation).
__device__ __forceinline__ float prox_g(float uhat, float f2, float tl) {
    const float D = fmaf(uhat, uhat, 4.0f * (1.0f + tl) * tl * f2);
    const float sD = sqrtf(D);
    return uhat >= 0.0f ? (uhat + sD) / (2.0f * (1.0f + tl)) : (2.0f * tl * f2) / (sD - uhat);
}

// Combined model (Eq. newmodel, Sec. III-A) in w = log u, one pixel: the
// data term lambda1/2 (2w + f^2 e^{-2w}) + lambda2/2 (e^{2w} - 2 f^2 w).
__device__ __forceinline__ float data_w(float w, float f2, float l1, float l2) {
    const float e2 = expf(2.0f * w), em2 = expf(-2.0f * w);
    return 0.5f * l1 * fmaf(f2, em2, 2.0f * w) + 0.5f * l2 * fmaf(-2.0f * f2, w, e2);
}

// Prox of tau*G for the combined model, one pixel, by Newton's method (the
// paper's choice, Sec. III-A): the root of phi(w) = w - what + tau g'(w),
// g'(w) = l1 (1 - f^2 e^{-2w}) + l2 (e^{2w} - f^2).  phi is increasing
// (phi' = 1 + tau g'' > 0) and g'(log f) = 0, so the root lies between what
// and log f; a Newton step that leaves that closed bracket is replaced by
// bisection.  At most 20 steps; stops once a step is below 2^-22 (1 + |w|).
// The bracket test is inclusive: near the root a step that rounds onto the
// bracket end just updated (w itself) must count as converged; a strict
// test bisects away from the root there, and in FP32 the iteration then
// bounced until the step limit (every warp ran 20 steps, with errors up to
// 1e-4 against the FP64 root; inclusive: 4-10 steps, 1e-7).
__device__ __forceinline__ float prox_w(float what, float f2, float tau, float l1, float l2) {
    const float lf = 0.5f * logf(f2);
    float lo = fminf(what, lf), hi = fmaxf(what, lf);
    float w = what;
    for (int it = 0; it < 20; ++it) {
        const float e2 = expf(2.0f * w), em2 = expf(-2.0f * w);
        const float ph = w - what + tau * (l1 * fmaf(-f2, em2, 1.0f) + l2 * (e2 - f2));
        if (ph == 0.0f) break;
        if (ph > 0.0f)
            hi = w;
        else
            lo = w;
        const float d2 = fmaf(2.0f * tau, fmaf(l1 * f2, em2, l2 * e2), 1.0f);
        float wn = w - ph / d2;
        if (!(wn >= lo && wn <= hi)) wn = 0.5f * (lo + hi);
        const float step = fabsf(wn - w);
        w = wn;
        if (step <= 2.4e-7f * (1.0f + fabsf(w))) break;
    }
    return w;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Compensated FP32 sum s + c (TwoSum, Knuth): c collects the exact rounding
// error of every addition, so a thread's partial sum keeps about twice the
// FP32 precision without FP64 instructions (FP64 issues at about 2 lanes per
// clock per SM on this GPU, 64x below FP32).  Per-thread and per-warp sums
// use it; the per-warp results are combined in FP64.
struct Sum2 {
    float s, c;
};
__device__ __forceinline__ void sum2_add(Sum2 &a, float x) {
    const float t = a.s + x;
    const float bp = t - a.s;
    a.c += (a.s - (t - bp)) + (x - bp);
    a.s = t;
}
__device__ __forceinline__ Sum2 sum2_merge(Sum2 a, Sum2 b) {
    const float t = a.s + b.s;
    const float bp = t - a.s;
    return Sum2{t, (a.c + b.c) + ((a.s - (t - bp)) + (b.s - bp))};
}
__device__ __forceinline__ Sum2 warp_sum2(Sum2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const Sum2 w{__shfl_xor_sync(0xffffffffu, v.s, o), __shfl_xor_sync(0xffffffffu, v.c, o)};
        v = sum2_merge(v, w);
    }
    return v;
}

// Position p in [0, T+6) of the frame/tile grid along one axis -> image
// coordinate j; returns whether that position belongs to this tile (main
// rows inside the image, or frame rows whose mirror image lies in the tile).
__device__ __forceinline__ bool axis_pos(int p, int t0, int T, int N, int &j) {
    if (p < 3) {
        j = p - 3;
        return t0 == 0;
    }
    if (p < T + 3) {
        j = t0 + p - 3;
        return j < N;
    }
    j = N + (p - T - 3);
    const int tgt = 2 * N - 1 - j;
    return tgt >= t0 && tgt < t0 + T;
}

// Accept / reject of the backtracking rule for one image (one thread).
__device__ void decide(const KParams &p, ImgState *st, const double *t, int mode) {
    const double F1 = t[0], G1 = t[1], gd = t[2], dd = t[3], dp = t[4];
    if (mode == MODE_INIT) {
        st->F = F1;
        st->G = G1;
        st->H = F1 + G1;
        st->H_prev = F1 + G1;
        st->alpha = 2.0 * (1.0 - p.beta) / (st->L + 2.0 * p.c2);
        if (!isfinite(F1) || !isfinite(G1)) {
            st->status = FE_ENONFINITE;
            st->done = 1;
        }
        return;
    }
    st->trials += 1;
    // a non-finite F1 (e^w overflowed in the combined model: inf, or inf - inf
    // = NaN inside the bank) fails the descent test like any other trial and
    // is rejected (L <- eta L, bounded by max_backtrack); non-finite step sums,
    // or an accepted step with a non-finite data term, stop the image
    if (!isfinite(gd) || !isfinite(dd)) {
        st->status = FE_ENONFINITE;
        st->done = 1;
        return;
    }
    if (isfinite(F1) && F1 <= st->F + gd + 0.5 * st->L * dd) {
        if (!isfinite(G1)) {
            st->status = FE_ENONFINITE;
            st->done = 1;
            return;
        }
        const double H1 = F1 + G1;
        // relative change of the energy above its data-term floor G(f) =
        // min_u G(u): H - G(f) = F(u) + (G(u) - G(f)) >= 0
        const double num = fabs(H1 - st->H), den = fabs(H1 - st->Gf);
        st->rel_change = num == 0.0 ? 0.0 : num / den;
        st->H_prev = st->H;
        st->F = F1;
        st->G = G1;
        st->H = H1;
        st->last_gd = gd;
        st->last_dd = dd;
        st->last_dp = dp;
        st->cur = (st->cur + 1) % 3;
        st->gcur ^= 1;
        st->n += 1;
        st->bt = 0;
        if ((st->tol > 0.0 && st->rel_change < st->tol) || H1 <= st->H_target) {
            st->converged = 1;
            st->done = 1;
        }
    } else {
        st->backtracks += 1;
        if (st->bt >= p.max_bt) {
            st->status = FE_EBACKTRACK;
            st->done = 1;
            return;
        }
        st->bt += 1;
        st->L *= p.eta;
        st->alpha = 2.0 * (1.0 - p.beta) / (st->L + 2.0 * p.c2);
    }
}

// ---- persistent trial launches ---------------------------------------------

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The next tile of a persistent launch (warp 0 of the CTA, all 32 lanes):
// the lanes look at 32 images at a time, starting with the image the CTA
// took its last tile from (pref), and the first image with tiles left is
// claimed by one atomic increment of its counter.  Returns the global tile
// index, or -1 when every image has stopped or the launch aborts.
__device__ int persist_grab(const KParams &p, int &pref) {
    const int lane = threadIdx.x & 31;
    LoopCtl *lc = p.loop;
    const unsigned long long limit = p.persist_stall_ns ? p.persist_stall_ns : PERSIST_STALL_NS;
    unsigned long long seen = ~0ull, t0 = 0;
    for (;;) {
        // lane 0 reads the shared words and broadcasts them: every lane takes
        // the same branches (the ballots below need the whole warp)
        int stop = 0;
        if (lane == 0) stop = *(volatile int *)&lc->abort != 0 || *(volatile int *)&lc->active <= 0;
        if (__shfl_sync(0xffffffffu, stop, 0)) return -1;
        for (int base = 0; base < p.nimg; base += 32) {
            const int k = base + lane;
            int j = pref + k;
            if (j >= p.nimg) j -= p.nimg;
            const int nt = k < p.nimg ? __ldg(&p.imgs[j].ntiles) : 0;
            const bool avail = k < p.nimg && *(volatile int *)(p.sched + j) < nt;
            unsigned m = __ballot_sync(0xffffffffu, avail);
            while (m) {
                const int l = __ffs(m) - 1;
                m &= m - 1u;
                int t = 0;
                if (lane == l) t = atomicAdd(p.sched + j, 1);
                t = __shfl_sync(0xffffffffu, t, l);
                const int jl = __shfl_sync(0xffffffffu, j, l), ntl = __shfl_sync(0xffffffffu, nt, l);
                if (t < ntl) {
                    pref = jl;
                    // acquire: the image's decision and the planes of its
                    // previous trial (the CTA's barrier passes them on)
                    __threadfence();
                    return __ldg(p.porder + __ldg(&p.imgs[jl].tile_begin) + t);
                }
            }
        }
        // nothing to take now: tiles come back when a trial is decided
        int stalled = 0;
        if (lane == 0) {
            const unsigned long long d = *(volatile unsigned long long *)&lc->decisions, now = global_ns();
            if (d != seen) {
                seen = d;
                t0 = now;
            } else if (now - t0 > limit) {
                atomicExch(&lc->abort, 1);
                stalled = 1;
            }
        }
        if (__shfl_sync(0xffffffffu, stalled, 0)) return -1;
        __nanosleep(200);
    }
}

// After the decision of image img's trial (thread 0 of the deciding CTA):
// the image's next trial is released (its tile counter back to 0), or the
// image leaves the launch.  The trial budget of the per-trial launches
// (FE_ETIMEOUT once it is spent) applies per image.
__device__ void persist_next(const KParams &p, ImgState *st, int img) {
    if (st->done == 0 && st->n < st->target && st->trials >= st->trial_limit) {
        st->status = FE_ETIMEOUT;
        st->done = 1;
    }
    const bool more = st->done == 0 && st->n < st->target;
    __threadfence();  // the state, the planes and the reset arrival count first
    if (more)
        atomicExch(p.sched + img, 0);
    else
        atomicSub(&p.loop->active, 1);
    atomicAdd(&p.loop->decisions, 1ull);
}

// End of a persistent launch (thread 0 of every CTA): the last CTA to leave
// marks images that a stalled launch left unfinished (FE_ETIMEOUT), and ends
// the graph's while loop.
__device__ void persist_exit(const KParams &p, unsigned participants) {
    if (threadIdx.x != 0) return;
    __threadfence();
    const unsigned prev = atomicAdd(&p.loop->grid_arrivals, 1u);
    if (prev != participants - 1u) return;
    __threadfence();
    LoopCtl *lc = p.loop;
    lc->grid_arrivals = 0u;
    for (int j = 0; j < p.nimg; ++j) {
        volatile ImgState *s = p.st + j;
        if (s->done == 0 && s->n < s->target) {
            s->status = FE_ETIMEOUT;
            s->done = 1;
        }
    }
    lc->active = 0;
    lc->launches += 1;
    __threadfence();
    if (p.use_cond) cudaGraphSetConditional(p.cond, 0u);
}

// Per-tile partial sums -> partials[gtile] (FP64): each thread's compensated
// FP32 sums are reduced per warp, the warps' results in FP64.  The last CTA
// of the image reduces the image's partials in FP64 in a fixed order (so the
// result does not depend on which CTA finishes last) and applies the
// decision (TRIAL/INIT) or stores F, G (EXT modes).  sRed: NT/32 * NRED
// doubles of shared memory.
template <int NT>
__device__ void tile_finish(const KParams &p, int mode, int gtile, int img, const ImgDesc &im, ImgState *st,
                            const Sum2 (&vals)[NRED], double *sRed, int *sLast) {
    constexpr int NWARP = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // (the CTA's plane and gradient writes are released to the deciding CTA,
    // and through it to the image's next trial, by the barriers below and
    // thread 0's fence before its arrival: the pattern of a grid barrier)
#pragma unroll
    for (int k = 0; k < NRED; ++k) {
        const Sum2 v = warp_sum2(vals[k]);
        if (lane == 0) sRed[warp * NRED + k] = (double)v.s + (double)v.c;
    }
    __syncthreads();
    if (tid < NRED) {
        double s = 0.0;
        for (int w = 0; w < NWARP; ++w) s += sRed[w * NRED + tid];
        p.partials[(size_t)gtile * NRED + tid] = s;
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(p.img_arrivals + img, 1u);
        *sLast = (prev == (unsigned)im.ntiles - 1u);
    }
    __syncthreads();
    if (*sLast) {
        __threadfence();
        // only the warps that hold partials reduce (FP64 issue is scarce)
        const int nw = min(NWARP, (im.ntiles + 31) / 32);
        if (warp < nw) {
            double part[NRED];
#pragma unroll
            for (int k = 0; k < NRED; ++k) part[k] = 0.0;
            for (int t = tid; t < im.ntiles; t += nw * 32)
#pragma unroll
                for (int k = 0; k < NRED; ++k) part[k] += __ldcg(p.partials + (size_t)(im.tile_begin + t) * NRED + k);
#pragma unroll
            for (int k = 0; k < NRED; ++k) {
                const double v = warp_sum(part[k]);
                if (lane == 0) sRed[warp * NRED + k] = v;
            }
        }
        __syncthreads();
        if (tid == 0) {
            double tot[NRED];
            for (int k = 0; k < NRED; ++k) {
                double s = 0.0;
                for (int w = 0; w < nw; ++w) s += sRed[w * NRED + k];
                tot[k] = s;
            }
            tot[1] *= im.gscale;  // variant: G = (lambda/2) sum_p (u^2 - 2 f^2 log u)
            if (mode == MODE_TRIAL || mode == MODE_PTRIAL || mode == MODE_INIT) {
                decide(p, st, tot, mode == MODE_PTRIAL ? MODE_TRIAL : mode);
            } else {
                p.results[2 * img] = tot[0];
                p.results[2 * img + 1] = tot[1];
            }
            p.img_arrivals[img] = 0u;
            __threadfence();
            if (mode == MODE_PTRIAL) persist_next(p, st, img);
        }
    }
}

// Loop control of a trial launch (thread 0 of every participating CTA: all
// CTAs, or the rank-0 CTA of every cluster): the last of the `participants`
// to arrive - each after its own tile's reduction and decision - counts the
// images still iterating, spends one unit of the trial budget, and sets the
// while-condition of the CUDA graph.
__device__ void loop_control(const KParams &p, unsigned participants) {
    if (threadIdx.x != 0) return;
    __threadfence();
    const unsigned prev = atomicAdd(&p.loop->grid_arrivals, 1u);
    if (prev != participants - 1u) return;
    __threadfence();
    LoopCtl *lc = p.loop;
    lc->grid_arrivals = 0u;
    long long budget = lc->budget - 1;
    int nact = 0;
    for (int j = 0; j < p.nimg; ++j) {
        volatile ImgState *s = p.st + j;
        if (s->done == 0 && s->n < s->target) {
            if (budget <= 0) {
                s->status = FE_ETIMEOUT;
                s->done = 1;
            } else {
                ++nact;
            }
        }
    }
    lc->budget = budget;
    lc->active = nact;
    lc->launches += 1;
    __threadfence();
    if (p.use_cond) cudaGraphSetConditional(p.cond, nact > 0 ? 1u : 0u);
}

}  // namespace
}  // namespace fe
