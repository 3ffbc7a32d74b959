/*
 * FP64 CPU oracle for the FoE despeckling models minimised by iPiano
 * (Sec. II-C): the model with the I-divergence data term (Eq. variant,
 * Sec. II-B) in u, and the combined model (Eq. newmodel, Sec. III-A) in
 * w = log u, whose special case lambda_2 = 0 is Eq. original.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library, and it never includes a CUDA header.
 *
 * Everything is computed in double precision with plain loops, in the order
 * the paper states the operations:
 *
 *   E_FoE(u) = sum_i theta_i sum_p rho((k_i * u)_p)           Eq. FOEmodel
 *   rho(x) = log(1 + x^2),  rho'(x) = 2x / (1 + x^2)          Sec. II-A/II-C
 *   G(u)    = (lambda/2) <u^2 - 2 f^2 log u, 1>                Eq. dataterm2
 *   H(u)    = F(u) + G(u),  F = E_FoE                          Eq. fplusg
 *   grad F  = sum_i theta_i K_i^T rho'(K_i u)                  Sec. II-C
 *   prox    = positive root of (1+t*l) u^2 - uhat u - t*l f^2  Sec. II-C
 *   u^{n+1} = prox_{alpha G}(u^n - alpha grad F(u^n) + beta (u^n - u^{n-1}))
 *
 * Readings of points the paper leaves open (each one is a parameter or a
 * stated convention, listed with the design notes):
 *   - K_i is "k_i * u" with symmetric (half-sample, edge-repeating) boundary
 *     extension by 3 pixels, then a true 2-D convolution ("valid" part).
 *     K_i^T is the exact matrix transpose: the full correlation onto the
 *     padded grid followed by the transpose of the padding map, which adds
 *     every padded pixel back onto the image pixel it was copied from.
 *   - Step size / backtracking (the paper names alpha, beta only; the rule
 *     is the one of the cited iPiano paper): alpha_n = 2(1-beta)/(L_n + 2 c2),
 *     a trial is accepted iff
 *       F(u^{n+1}) <= F(u^n) + <grad F(u^n), u^{n+1}-u^n> + L_n/2 |u^{n+1}-u^n|^2,
 *     otherwise L_n <- eta L_n and the trial is recomputed.  L is never
 *     decreased; u^{-1} = u^0.  A trial with a non-finite F (overflow) fails
 *     the test: it is rejected, not an error.
 *   - Stopping: a fixed number of accepted iterations, or
 *     |H^{n+1} - H^n| / |H^{n+1} - G(f)| < tol: the relative change of the
 *     energy above the floor of the data term, G(f) = min_u G(u) (a constant
 *     of the problem; with intensities of order 100 it dominates |H|).
 *
 * Parallelism: OpenMP over image rows inside each operator (each row is an
 * independent plain loop; sums over rows are combined serially in row order
 * so results do not depend on the thread count).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_API __attribute__((visibility("default")))

/* ----------------------------------------------------------------------- */
/* Boundary extension (reading of the unstated boundary condition)         */
/* ----------------------------------------------------------------------- */

/* Half-sample symmetric index map: ... c b a | a b c ... d e | e d ...
 * Repeated reflection covers extensions wider than the image. */
ORC_API long orc_mirror(long j, long n)
{
    for (;;) {
        if (j < 0)
            j = -j - 1;
        else if (j >= n)
            j = 2 * n - 1 - j;
        else
            return j;
    }
}

/* P: R^{H x W} -> R^{(H+2p) x (W+2p)}, symmetric extension by p pixels. */
ORC_API void orc_pad(const double *u, int H, int W, int p, double *up)
{
    const int Wp = W + 2 * p, Hp = H + 2 * p;
    for (int Y = 0; Y < Hp; ++Y)
        for (int X = 0; X < Wp; ++X)
            up[(long)Y * Wp + X] =
                u[orc_mirror(Y - p, H) * W + orc_mirror(X - p, W)];
}

/* P^T: adds every padded pixel onto the image pixel it was copied from. */
ORC_API void orc_pad_adjoint(const double *up, int H, int W, int p, double *u)
{
    const int Wp = W + 2 * p, Hp = H + 2 * p;
    memset(u, 0, sizeof(double) * (size_t)H * W);
    for (int Y = 0; Y < Hp; ++Y)
        for (int X = 0; X < Wp; ++X)
            u[orc_mirror(Y - p, H) * W + orc_mirror(X - p, W)] +=
                up[(long)Y * Wp + X];
}

/* ----------------------------------------------------------------------- */
/* Linear filter operators K_i and K_i^T (Sec. II-C: K_i u <=> k_i * u)     */
/* ----------------------------------------------------------------------- */

/* True 2-D convolution, "valid" part: z(y,x) = sum_ab k[a][b] up(y+ks-1-a, x+ks-1-b)
 * with up of size Hp x Wp, z of size (Hp-ks+1) x (Wp-ks+1). */
ORC_API void orc_conv_valid(const double *up, int Hp, int Wp,
                            const double *k, int ks, double *z)
{
    const int Ho = Hp - ks + 1, Wo = Wp - ks + 1;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < Ho; ++y)
        for (int x = 0; x < Wo; ++x) {
            double s = 0.0;
            for (int a = 0; a < ks; ++a)
                for (int b = 0; b < ks; ++b)
                    s += k[a * ks + b] *
                         up[(long)(y + ks - 1 - a) * Wp + (x + ks - 1 - b)];
            z[(long)y * Wo + x] = s;
        }
}

/* Transpose of orc_conv_valid: the "full" correlation of r (Ho x Wo, zero
 * outside) with k onto the Hp x Wp grid:
 *   s(Y,X) = sum_ab k[a][b] r(Y-(ks-1)+a, X-(ks-1)+b). */
ORC_API void orc_conv_valid_adjoint(const double *r, int Ho, int Wo,
                                    const double *k, int ks, double *s)
{
    const int Hp = Ho + ks - 1, Wp = Wo + ks - 1;
#pragma omp parallel for schedule(static)
    for (int Y = 0; Y < Hp; ++Y)
        for (int X = 0; X < Wp; ++X) {
            double acc = 0.0;
            for (int a = 0; a < ks; ++a) {
                const int y = Y - (ks - 1) + a;
                if (y < 0 || y >= Ho)
                    continue;
                for (int b = 0; b < ks; ++b) {
                    const int x = X - (ks - 1) + b;
                    if (x < 0 || x >= Wo)
                        continue;
                    acc += k[a * ks + b] * r[(long)y * Wo + x];
                }
            }
            s[(long)Y * Wp + X] = acc;
        }
}

/* z = K u : pad symmetrically by ks/2, convolve, keep the H x W result. */
ORC_API void orc_K(const double *u, int H, int W, const double *k, int ks, double *z)
{
    const int p = ks / 2;
    double *up = (double *)malloc(sizeof(double) * (size_t)(H + 2 * p) * (W + 2 * p));
    orc_pad(u, H, W, p, up);
    orc_conv_valid(up, H + 2 * p, W + 2 * p, k, ks, z);
    free(up);
}

/* g = K^T r = P^T C^T r. */
ORC_API void orc_KT(const double *r, int H, int W, const double *k, int ks, double *g)
{
    const int p = ks / 2;
    double *sp = (double *)malloc(sizeof(double) * (size_t)(H + 2 * p) * (W + 2 * p));
    orc_conv_valid_adjoint(r, H, W, k, ks, sp);
    orc_pad_adjoint(sp, H, W, p, g);
    free(sp);
}

/* ----------------------------------------------------------------------- */
/* Potential, energies, gradient                                           */
/* ----------------------------------------------------------------------- */

ORC_API double orc_rho(double x) { return log(1.0 + x * x); }
ORC_API double orc_drho(double x) { return 2.0 * x / (1.0 + x * x); }

/* Sum of a row-major H x W array, rows summed in parallel and combined in
 * row order (independent of the thread count). */
static double sum_rows(const double *v, int H, int W)
{
    double *rs = (double *)malloc(sizeof(double) * (size_t)H);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        double s = 0.0;
        for (int x = 0; x < W; ++x)
            s += v[(long)y * W + x];
        rs[y] = s;
    }
    double t = 0.0;
    for (int y = 0; y < H; ++y)
        t += rs[y];
    free(rs);
    return t;
}

/* F(u) = E_FoE(u) = sum_i theta_i sum_p rho((K_i u)_p)   (Eq. FOEmodel) */
ORC_API double orc_F(const double *u, int H, int W, const double *bank,
                     const double *theta, int nf, int ks)
{
    const size_t N = (size_t)H * W;
    double *z = (double *)malloc(sizeof(double) * N);
    double *t = (double *)malloc(sizeof(double) * N);
    double F = 0.0;
    for (int i = 0; i < nf; ++i) {
        orc_K(u, H, W, bank + (size_t)i * ks * ks, ks, z);
        for (size_t p = 0; p < N; ++p)
            t[p] = orc_rho(z[p]);
        F += theta[i] * sum_rows(t, H, W);
    }
    free(z);
    free(t);
    return F;
}

/* G(u) = (lambda/2) sum_p (u_p^2 - 2 f_p^2 log u_p)   (Eq. dataterm2) */
ORC_API double orc_G(const double *u, const double *f, long N, double lambda)
{
    double s = 0.0;
    for (long p = 0; p < N; ++p)
        s += u[p] * u[p] - 2.0 * f[p] * f[p] * log(u[p]);
    return 0.5 * lambda * s;
}

/* grad F(u) = sum_i theta_i K_i^T rho'(K_i u)   (Sec. II-C, model variant).
 * Returns F(u) as a by-product (same z). */
ORC_API double orc_gradF(const double *u, int H, int W, const double *bank,
                         const double *theta, int nf, int ks, double *g)
{
    const size_t N = (size_t)H * W;
    double *z = (double *)malloc(sizeof(double) * N);
    double *r = (double *)malloc(sizeof(double) * N);
    double *t = (double *)malloc(sizeof(double) * N);
    double *gi = (double *)malloc(sizeof(double) * N);
    double F = 0.0;
    memset(g, 0, sizeof(double) * N);
    for (int i = 0; i < nf; ++i) {
        const double *k = bank + (size_t)i * ks * ks;
        orc_K(u, H, W, k, ks, z);
        for (size_t p = 0; p < N; ++p) {
            r[p] = orc_drho(z[p]);
            t[p] = orc_rho(z[p]);
        }
        F += theta[i] * sum_rows(t, H, W);
        orc_KT(r, H, W, k, ks, gi);
        for (size_t p = 0; p < N; ++p)
            g[p] += theta[i] * gi[p];
    }
    free(z);
    free(r);
    free(t);
    free(gi);
    return F;
}

/* grad F at one pixel (y,x), for sampled checks on large images; needs
 * H, W >= ks/2 so that every padded pixel is a single reflection. */
static double K_at(const double *u, int H, int W, const double *k, int ks, int y, int x)
{
    const int p = ks / 2;
    double s = 0.0;
    for (int a = 0; a < ks; ++a)
        for (int b = 0; b < ks; ++b)
            s += k[a * ks + b] *
                 u[orc_mirror(y + p - a, H) * W + orc_mirror(x + p - b, W)];
    return s;
}

ORC_API double orc_gradF_at(const double *u, int H, int W, const double *bank,
                            const double *theta, int nf, int ks, int y, int x)
{
    const int p = ks / 2;
    /* padded rows / cols (in image coordinates j in [-p, H+p)) that the
     * padding map sends to y / x */
    int jy[3], ny = 0, jx[3], nx = 0;
    const int cy[3] = {y, -y - 1, 2 * H - 1 - y}, cx[3] = {x, -x - 1, 2 * W - 1 - x};
    for (int c = 0; c < 3; ++c) {
        int dup = 0;
        for (int d = 0; d < ny; ++d) dup |= (jy[d] == cy[c]);
        if (!dup && cy[c] >= -p && cy[c] < H + p && orc_mirror(cy[c], H) == y)
            jy[ny++] = cy[c];
        dup = 0;
        for (int d = 0; d < nx; ++d) dup |= (jx[d] == cx[c]);
        if (!dup && cx[c] >= -p && cx[c] < W + p && orc_mirror(cx[c], W) == x)
            jx[nx++] = cx[c];
    }
    double g = 0.0;
    for (int i = 0; i < nf; ++i) {
        const double *k = bank + (size_t)i * ks * ks;
        double gi = 0.0;
        for (int m = 0; m < ny; ++m)
            for (int n = 0; n < nx; ++n)
                /* (C^T r)(Y,X) = sum_ab k[a][b] r(Y-p+a, X-p+b) with r zero off-image */
                for (int a = 0; a < ks; ++a) {
                    const int yy = jy[m] - p + a;
                    if (yy < 0 || yy >= H) continue;
                    for (int b = 0; b < ks; ++b) {
                        const int xx = jx[n] - p + b;
                        if (xx < 0 || xx >= W) continue;
                        gi += k[a * ks + b] * orc_drho(K_at(u, H, W, k, ks, yy, xx));
                    }
                }
        g += theta[i] * gi;
    }
    return g;
}

/* ----------------------------------------------------------------------- */
/* Proximal map of tau*G (Sec. II-C, closed form for the variant model)    */
/* ----------------------------------------------------------------------- */

/* The paper's formula, written literally. */
ORC_API double orc_prox_literal(double uhat, double f, double tau, double lambda)
{
    const double tl = tau * lambda;
    return (uhat + sqrt(uhat * uhat + 4.0 * (1.0 + tl) * tl * f * f)) / (2.0 * (1.0 + tl));
}

/* Same root; for uhat < 0 the numerator uhat + sqrt(D) is rewritten as
 * (D - uhat^2)/(sqrt(D) - uhat) to avoid cancellation. */
ORC_API double orc_prox(double uhat, double f, double tau, double lambda)
{
    const double tl = tau * lambda;
    const double D = uhat * uhat + 4.0 * (1.0 + tl) * tl * f * f;
    if (uhat >= 0.0)
        return (uhat + sqrt(D)) / (2.0 * (1.0 + tl));
    return 2.0 * tl * f * f / (sqrt(D) - uhat);
}

/* ----------------------------------------------------------------------- */
/* Combined model (Eq. newmodel) in w = log u                              */
/*   F(w) = E_FoE(e^w)                                                     */
/*   G(w) = sum_p lambda1/2 (2w + f^2 e^{-2w}) + lambda2/2 (e^{2w} - 2f^2 w) */
/* lambda2 = 0: Eq. original (Sec. II-C).                                  */
/* ----------------------------------------------------------------------- */

ORC_API double orc_Fw(const double *w, int H, int W, const double *bank,
                      const double *theta, int nf, int ks)
{
    const long N = (long)H * W;
    double *u = (double *)malloc(sizeof(double) * N);
    for (long q = 0; q < N; ++q)
        u[q] = exp(w[q]);
    const double F = orc_F(u, H, W, bank, theta, nf, ks);
    free(u);
    return F;
}

/* grad_w F = sum_i theta_i W K_i^T rho'(K_i e^w), W = diag(e^w) (Sec. II-C).
 * Returns F(w). */
ORC_API double orc_gradFw(const double *w, int H, int W, const double *bank,
                          const double *theta, int nf, int ks, double *g)
{
    const long N = (long)H * W;
    double *u = (double *)malloc(sizeof(double) * N);
    for (long q = 0; q < N; ++q)
        u[q] = exp(w[q]);
    const double F = orc_gradF(u, H, W, bank, theta, nf, ks, g);
    for (long q = 0; q < N; ++q)
        g[q] *= u[q];
    free(u);
    return F;
}

/* Data term of one pixel and its first two derivatives in w. */
static double gc_term(double w, double f, double l1, double l2)
{
    return 0.5 * l1 * (2.0 * w + f * f * exp(-2.0 * w)) + 0.5 * l2 * (exp(2.0 * w) - 2.0 * f * f * w);
}
static double gc_d1(double w, double f, double l1, double l2)
{
    return l1 * (1.0 - f * f * exp(-2.0 * w)) + l2 * (exp(2.0 * w) - f * f);
}
static double gc_d2(double w, double f, double l1, double l2)
{
    return 2.0 * l1 * f * f * exp(-2.0 * w) + 2.0 * l2 * exp(2.0 * w);
}

ORC_API double orc_Gc(const double *w, const double *f, long N, double lambda1, double lambda2)
{
    double s = 0.0;
    for (long p = 0; p < N; ++p)
        s += gc_term(w[p], f[p], lambda1, lambda2);
    return s;
}

/* Proximal map of tau*G for the combined model, one pixel: the root of
 * phi(w) = w - what + tau g'(w) by Newton's method (Sec. III-A: the prox is
 * solved with Newton's method).  phi is strictly increasing (phi' = 1 +
 * tau g'' > 0) and g'(log f) = 0, so the root lies in the closed interval
 * between what and log f; a Newton step that leaves that interval is
 * replaced by bisection (a step onto its end stays a Newton step).
 * Iterates until the step is below 1e-15 (1 + |w|) or 200 iterations;
 * *iters (may be NULL) receives the number of steps taken. */
ORC_API double orc_proxc_iters(double what, double f, double tau, double lambda1, double lambda2, int *iters)
{
    const double lf = log(f);
    double lo = what < lf ? what : lf, hi = what < lf ? lf : what;
    double w = what;
    int it = 0;
    while (it < 200) {
        ++it;
        const double ph = w - what + tau * gc_d1(w, f, lambda1, lambda2);
        if (ph == 0.0)
            break;
        if (ph > 0.0)
            hi = w;
        else
            lo = w;
        double wn = w - ph / (1.0 + tau * gc_d2(w, f, lambda1, lambda2));
        if (!(wn >= lo && wn <= hi))
            wn = 0.5 * (lo + hi);
        const double step = fabs(wn - w);
        w = wn;
        if (step <= 1e-15 * (1.0 + fabs(w)))
            break;
    }
    if (iters)
        *iters = it;
    return w;
}

ORC_API double orc_proxc(double what, double f, double tau, double lambda1, double lambda2)
{
    return orc_proxc_iters(what, f, tau, lambda1, lambda2, NULL);
}

/* ----------------------------------------------------------------------- */
/* iPiano                                                                  */
/* ----------------------------------------------------------------------- */

enum { ORC_MODEL_VARIANT = 0, ORC_MODEL_COMBINED = 1 };

typedef struct {
    double lambda, beta, L0, eta, c2;
    int max_backtrack;
    int max_iter;     /* accepted iterations */
    double tol;       /* <= 0: no energy-change test */
    int model;        /* ORC_MODEL_VARIANT: x = u, G with lambda;
                         ORC_MODEL_COMBINED: x = w = log u, G with lambda1
                         (Eq. original term) and lambda2 = lambda (variant term) */
    double lambda1;
} orc_params;

/* The model's F, grad F, G, prox and data-term floor in its variable x. */
static double obj_gradF(const orc_params *p, const double *x, int H, int W, const double *bank,
                        const double *theta, int nf, int ks, double *g)
{
    return p->model == ORC_MODEL_COMBINED ? orc_gradFw(x, H, W, bank, theta, nf, ks, g)
                                          : orc_gradF(x, H, W, bank, theta, nf, ks, g);
}
static double obj_F(const orc_params *p, const double *x, int H, int W, const double *bank,
                    const double *theta, int nf, int ks)
{
    return p->model == ORC_MODEL_COMBINED ? orc_Fw(x, H, W, bank, theta, nf, ks)
                                          : orc_F(x, H, W, bank, theta, nf, ks);
}
static double obj_G(const orc_params *p, const double *x, const double *f, long N)
{
    return p->model == ORC_MODEL_COMBINED ? orc_Gc(x, f, N, p->lambda1, p->lambda) : orc_G(x, f, N, p->lambda);
}
static double obj_prox(const orc_params *p, double xhat, double f, double tau)
{
    return p->model == ORC_MODEL_COMBINED ? orc_proxc(xhat, f, tau, p->lambda1, p->lambda)
                                          : orc_prox(xhat, f, tau, p->lambda);
}
/* min_x G(x): reached at u = f (variant) and at w = log f (combined: g'(log f) = 0). */
static double obj_Gfloor(const orc_params *p, const double *f, long N)
{
    if (p->model != ORC_MODEL_COMBINED)
        return orc_G(f, f, N, p->lambda);
    double s = 0.0;
    for (long q = 0; q < N; ++q)
        s += gc_term(log(f[q]), f[q], p->lambda1, p->lambda);
    return s;
}

/* Per accepted iteration record (9 doubles):
 *  [L_n, alpha_n, F, G, H, backtracks, <g,D>, |D|^2, <D, D_prev>]
 * where D = u^{n+1} - u^n, D_prev = u^n - u^{n-1}, g = grad F(u^n). */
#define ORC_REC 9

enum { ORC_OK = 0, ORC_EBACKTRACK = 5, ORC_ENONFINITE = 4 };

static double step_size(const orc_params *p, double L)
{
    return 2.0 * (1.0 - p->beta) / (L + 2.0 * p->c2);
}

/* One iPiano iteration from (u, up) with gradient g = grad F(u), F = F(u),
 * starting from the estimate *L.  On acceptance writes u1 (and g1 = grad F(u1),
 * F1, G1) and returns ORC_OK; *L holds the accepted L_n. */
static int ipiano_iteration(const double *u, const double *up, const double *g,
                            double F, int H, int W, const double *f,
                            const double *bank, const double *theta, int nf, int ks,
                            const orc_params *p, double *L, double *u1, double *g1,
                            double *F1_out, double *G1_out, double *rec)
{
    const long N = (long)H * W;
    double *uhat = (double *)malloc(sizeof(double) * N);
    int bt = 0, status = ORC_EBACKTRACK;
    for (;;) {
        const double alpha = step_size(p, *L);
        /* forward (explicit) step with inertia, then the prox of alpha G */
        for (long q = 0; q < N; ++q) {
            uhat[q] = u[q] - alpha * g[q] + p->beta * (u[q] - up[q]);
            u1[q] = obj_prox(p, uhat[q], f[q], alpha);
        }
        const double F1 = obj_F(p, u1, H, W, bank, theta, nf, ks);
        double gd = 0.0, dd = 0.0, dp = 0.0;
        for (long q = 0; q < N; ++q) {
            const double d = u1[q] - u[q];
            gd += g[q] * d;
            dd += d * d;
            dp += d * (u[q] - up[q]);
        }
        /* a non-finite F1 (e^w overflowed in the combined model: inf, or
         * inf - inf = NaN inside the bank) fails the descent test like any
         * other trial and is rejected; non-finite step sums stop the solve */
        if (!isfinite(gd) || !isfinite(dd)) {
            status = ORC_ENONFINITE;
            break;
        }
        if (isfinite(F1) && F1 <= F + gd + 0.5 * (*L) * dd) {
            obj_gradF(p, u1, H, W, bank, theta, nf, ks, g1);
            *F1_out = F1;
            *G1_out = obj_G(p, u1, f, N);
            if (rec) {
                rec[0] = *L;
                rec[1] = alpha;
                rec[2] = F1;
                rec[3] = *G1_out;
                rec[4] = F1 + *G1_out;
                rec[5] = bt;
                rec[6] = gd;
                rec[7] = dd;
                rec[8] = dp;
            }
            status = ORC_OK;
            break;
        }
        if (bt >= p->max_backtrack)
            break;
        *L *= p->eta;
        ++bt;
    }
    free(uhat);
    return status;
}

/* Full solve.  u_io: on entry u^0 (copied as u^{-1} too); on exit u^n.
 * u_prev_out (may be NULL): u^{n-1}.  rec (may be NULL): ORC_REC doubles per
 * accepted iteration.  *n_done: accepted iterations.  *L_io: L_{-1} on entry
 * (params L0 if <= 0), the last accepted L on exit.  h0 (may be NULL): F, G
 * of u^0.  Returns ORC_OK, ORC_EBACKTRACK or ORC_ENONFINITE. */
ORC_API int orc_ipiano(const double *f, int H, int W, const double *bank,
                       const double *theta, int nf, int ks, const orc_params *p,
                       double *u_io, double *u_prev_out, double *rec,
                       int *n_done, double *L_io, double *h0, int *converged)
{
    const long N = (long)H * W;
    double *u = u_io;
    double *up = (double *)malloc(sizeof(double) * N);
    double *u1 = (double *)malloc(sizeof(double) * N);
    double *g = (double *)malloc(sizeof(double) * N);
    double *g1 = (double *)malloc(sizeof(double) * N);
    memcpy(up, u, sizeof(double) * N);
    double L = (L_io && *L_io > 0.0) ? *L_io : p->L0;
    double F = obj_gradF(p, u, H, W, bank, theta, nf, ks, g);
    double G = obj_G(p, u, f, N);
    const double Gfloor = obj_Gfloor(p, f, N);
    if (h0) {
        h0[0] = F;
        h0[1] = G;
    }
    int n = 0, status = ORC_OK;
    if (converged) *converged = 0;
    while (n < p->max_iter) {
        double F1, G1;
        status = ipiano_iteration(u, up, g, F, H, W, f, bank, theta, nf, ks, p,
                                  &L, u1, g1, &F1, &G1, rec ? rec + (size_t)n * ORC_REC : NULL);
        if (status != ORC_OK)
            break;
        const double Hn = F + G, H1 = F1 + G1;
        memcpy(up, u, sizeof(double) * N);
        memcpy(u, u1, sizeof(double) * N);
        memcpy(g, g1, sizeof(double) * N);
        F = F1;
        G = G1;
        ++n;
        if (p->tol > 0.0 && fabs(H1 - Hn) / fabs(H1 - Gfloor) < p->tol) {
            if (converged) *converged = 1;
            break;
        }
    }
    if (u_prev_out)
        memcpy(u_prev_out, up, sizeof(double) * N);
    if (n_done)
        *n_done = n;
    if (L_io)
        *L_io = L;
    free(up);
    free(u1);
    free(g);
    free(g1);
    return status;
}

/* One iteration from a given state (u^n, u^{n-1}) and estimate L_in; the
 * gradient and F at u^n are recomputed here in FP64.  Writes u^{n+1} and the
 * record; *L_out = accepted L_n. */
ORC_API int orc_ipiano_step(const double *f, int H, int W, const double *bank,
                            const double *theta, int nf, int ks, const orc_params *p,
                            const double *u, const double *up, double L_in,
                            double *u1, double *rec, double *L_out)
{
    const long N = (long)H * W;
    double *g = (double *)malloc(sizeof(double) * N);
    double *g1 = (double *)malloc(sizeof(double) * N);
    const double F = obj_gradF(p, u, H, W, bank, theta, nf, ks, g);
    double L = L_in, F1, G1;
    const int status = ipiano_iteration(u, up, g, F, H, W, f, bank, theta, nf, ks,
                                        p, &L, u1, g1, &F1, &G1, rec);
    if (L_out)
        *L_out = L;
    free(g);
    free(g1);
    return status;
}

/* iPiano with a prescribed sequence L_0..L_{n-1} and no backtracking test:
 * alpha_k = 2(1-beta)/(L_k + 2 c2) and the Sec. II-C update.  Starts from
 * (u_io, u_prev_io) = (u^0, u^{-1}) and returns (u^n, u^{n-1}) in them.
 * rec (n x ORC_REC) as orc_ipiano, except rec[5] = the margin of the
 * descent test F(u^k) + <g,D> + L_k/2 |D|^2 - F(u^{k+1}) (>= 0 means the
 * backtracking rule would accept the step). */
ORC_API int orc_ipiano_fixed(const double *f, int H, int W, const double *bank,
                             const double *theta, int nf, int ks, const orc_params *p,
                             const double *Lseq, int n, double *u_io, double *u_prev_io,
                             double *rec)
{
    const long N = (long)H * W;
    double *u = u_io, *up = u_prev_io;
    double *u1 = (double *)malloc(sizeof(double) * N);
    double *g = (double *)malloc(sizeof(double) * N);
    int status = ORC_OK;
    double F = obj_gradF(p, u, H, W, bank, theta, nf, ks, g);
    for (int k = 0; k < n; ++k) {
        const double L = Lseq[k], alpha = step_size(p, L);
        double gd = 0.0, dd = 0.0, dp = 0.0;
        for (long q = 0; q < N; ++q) {
            const double uhat = u[q] - alpha * g[q] + p->beta * (u[q] - up[q]);
            u1[q] = obj_prox(p, uhat, f[q], alpha);
            const double d = u1[q] - u[q];
            gd += g[q] * d;
            dd += d * d;
            dp += d * (u[q] - up[q]);
        }
        const double F1 = obj_gradF(p, u1, H, W, bank, theta, nf, ks, g);
        const double G1 = obj_G(p, u1, f, N);
        if (!isfinite(F1) || !isfinite(G1)) {
            status = ORC_ENONFINITE;
            break;
        }
        if (rec) {
            double *r = rec + (size_t)k * ORC_REC;
            r[0] = L;
            r[1] = alpha;
            r[2] = F1;
            r[3] = G1;
            r[4] = F1 + G1;
            r[5] = F + gd + 0.5 * L * dd - F1;
            r[6] = gd;
            r[7] = dd;
            r[8] = dp;
        }
        memcpy(up, u, sizeof(double) * N);
        memcpy(u, u1, sizeof(double) * N);
        F = F1;
    }
    free(u1);
    free(g);
    return status;
}

ORC_API int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

ORC_API void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}
