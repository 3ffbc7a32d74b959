/*
 * fe.h - C ABI of libfe, the GB300 (sm_103a) iPiano solver for the
 * Fields-of-Experts despeckling model with the I-divergence data term.
 *
 * Problem (Chen et al., "A higher-order MRF based variational model for
 * multiplicative noise reduction"; Eq. variant of Sec. II-B):
 *
 *     argmin_{u > 0}  H(u) = F(u) + G(u)
 *     F(u) = sum_i theta_i sum_p log(1 + (k_i * u)_p^2)      (Eq. FOEmodel)
 *     G(u) = (lambda / 2) sum_p (u_p^2 - 2 f_p^2 log u_p)    (Eq. dataterm2)
 *
 * solved by iPiano (Sec. II-C, Eq. fplusg and the update rule under it):
 *
 *     u^{n+1} = prox_{alpha_n G}(u^n - alpha_n grad F(u^n) + beta (u^n - u^{n-1}))
 *     grad F(u) = sum_i theta_i K_i^T rho'(K_i u),  rho'(z) = 2z / (1 + z^2)
 *     prox: u_p = (uhat_p + sqrt(uhat_p^2 + 4(1+tau l) tau l f_p^2)) / (2(1+tau l))
 *
 * Second model (fe_params.model = FE_MODEL_COMBINED, every precision form): the
 * combined model of Eq. newmodel (Sec. III-A), iterated in w = log u:
 *
 *     argmin_w  F(e^w) + sum_p lambda1/2 (2 w_p + f_p^2 e^{-2 w_p})
 *                      + lambda2/2 (e^{2 w_p} - 2 f_p^2 w_p)
 *     grad_w F = e^w (.) sum_i theta_i K_i^T rho'(K_i e^w)            (Sec. II-C)
 *
 * with the prox of the (convex) data term solved per pixel by Newton's
 * method (Sec. III-A), safeguarded by the bracket [min(what, log f),
 * max(what, log f)] that always holds the root.  lambda2 = fe_params.lambda,
 * lambda1 = fe_params.lambda1; lambda2 = 0 gives Eq. original (Sec. II-C).
 * For this model the solver's iterate is w: fe_get_state / fe_set_state
 * exchange (w^n, w^{n-1}, grad_w F), fe_energy and fe_gradient take w, and
 * fe_get_u returns u = e^w.  The data-term floor of the convergence test is
 * its value at w = log f, where it is minimal.
 *
 * Conventions that the paper leaves open (fixed here, identical to the FP64
 * oracle used by the tests):
 *   - k_i * u is a true 2-D convolution of the image extended by 3 pixels with
 *     half-sample symmetric reflection (... c b a | a b c ...); K_i^T is the
 *     exact transpose of that linear map (boundary fold included).
 *   - alpha_n = 2 (1 - beta) / (L_n + 2 c2).  A trial is accepted iff
 *       F(u^{n+1}) <= F(u^n) + <grad F(u^n), u^{n+1} - u^n> + L_n/2 |u^{n+1} - u^n|^2
 *     else L_n <- eta L_n and the trial is redone (at most max_backtrack
 *     times per iteration).  L is never decreased.  u^{-1} = u^0.  A trial
 *     whose F(u^{n+1}) is not finite fails the test (it is rejected).
 *   - Convergence: |H^{n+1} - H^n| / |H^{n+1} - G(f)| < tol, i.e. the relative
 *     change of the energy measured above the floor of the data term,
 *     G(f) = min_u G(u) = (lambda/2) sum_p f_p^2 (1 - log f_p^2).  (With
 *     intensities of order 100 the constant G(f) dominates |H|, and a test on
 *     |H| alone would stop after the first step.)
 *
 * Data layout: every image is a dense row-major float32 array, pitch = W.
 * Pointers named "any" may be host (pageable or pinned) or device pointers of
 * the current device; copies use cudaMemcpyDefault.  Device pointers must be
 * 4-byte aligned.  The library keeps its own device state (iterates, gradient,
 * f^2, per-tile partial sums) and frees it in fe_destroy.
 *
 * Errors: no call aborts or throws across the ABI.  Every call returns an
 * fe_status; fe_last_error() gives a message for the last failure on a
 * context.  Calls are stream-ordered on the stream given to fe_init; calls
 * that return host values synchronise that stream.
 *
 * Threads: a context must not be used by two host threads at once.
 */
#ifndef FE_H
#define FE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FE_ABI_VERSION 2

#if defined(__GNUC__)
#define FE_API __attribute__((visibility("default")))
#else
#define FE_API
#endif

typedef enum {
    FE_OK = 0,
    FE_EINVAL = 1,          /* bad argument (null, size < 8, f <= 0 or not finite, ...) */
    FE_ENOMEM = 2,          /* device allocation failed */
    FE_ECUDA = 3,           /* a CUDA runtime call failed */
    FE_ENONFINITE = 4,      /* a trial produced non-finite step sums, or an accepted
                               step a non-finite energy (a trial whose F is not
                               finite, e.g. e^w overflowing, is only rejected) */
    FE_EBACKTRACK = 5,      /* more than max_backtrack rejections in one iteration */
    FE_ETIMEOUT = 6,        /* the device-side trial budget ran out */
    FE_ENOTCONVERGED = 7,   /* fe_solve hit max_iter before the tolerance */
    FE_EUNSUPPORTED = 8     /* option not available in this build */
} fe_status;

typedef enum {
    FE_FP32 = 0,            /* filter bank in FP32 FFMA (parity-grade) */
    FE_TF32 = 1,            /* filter bank on the tensor cores, TF32 operands */
    FE_BF16 = 2,            /* filter bank on the tensor cores, BF16 operands */
    FE_BF16R = 3            /* as FE_BF16, but the response r_i = theta_i rho'(z_i) enters
                               the adjoint bank rounded once to BF16 (no lo part: half
                               the adjoint GEMM's K); the energy is that of FE_BF16 and
                               grad F carries the rounding of r (about 2^-9 relative
                               per response), a stated-bound variant of the form */
} fe_precision;

#define FE_TILE_CLUSTER4 0x100  /* fe_params.tile flag: a 4-CTA cluster per tile */

typedef enum {
    FE_MODEL_VARIANT = 0,   /* Eq. variant in u (all precision forms) */
    FE_MODEL_COMBINED = 1   /* Eq. newmodel in w = log u */
} fe_model;

/* Solver parameters.  All pointers are HOST pointers, copied by fe_init. */
typedef struct {
    int nf;                 /* number of filters, 1..64 (48 in the paper) */
    int ksize;              /* filter side; must be 7 */
    const float *filters;   /* nf * 7 * 7, filter i at filters + 49 i, row-major k_i[a][b] */
    const float *theta;     /* nf weights theta_i >= 0 (Eq. FOEmodel) */
    double lambda;          /* weight of the I-divergence term: lambda > 0 (Eq. variant);
                               lambda2 >= 0 of Eq. newmodel (FE_MODEL_COMBINED) */
    double beta;            /* inertia, 0 <= beta < 1 */
    double L0;              /* initial Lipschitz estimate L_{-1} > 0 */
    double eta;             /* backtracking factor > 1 */
    double c2;              /* step-size margin c2 >= 0 */
    int max_backtrack;      /* rejections allowed per iteration, >= 0 */
    int prec;               /* fe_precision */
    int tile;               /* output tile of the trial kernel: 0 = autotune.  FP32:
                               0, 64, 32 (T x T), or 32 | FE_TILE_CLUSTER4 /
                               64 | FE_TILE_CLUSTER4 (T x T tiles, each split by
                               filter group over a cluster of 4 CTAs that combine
                               through distributed shared memory: for images too
                               small to fill the GPU); at 0 fe_init_batch times the
                               four on the context's own
                               images (the initial gradient kernel, 4 launches
                               each) and keeps the fastest, cached per device and
                               list of image sizes.
                               Tensor-core forms: 0 only (one shape, 58 rows x
                               26 columns).
                               Other values: FE_EUNSUPPORTED. */
    int model;              /* fe_model */
    double lambda1;         /* FE_MODEL_COMBINED: weight lambda1 >= 0 of the
                               log-domain term (lambda + lambda1 > 0); ignored
                               by FE_MODEL_VARIANT */
} fe_params;

/* Per-image solver state summary (host struct, filled by fe_get_info). */
typedef struct {
    long long n;            /* accepted iterations since fe_init */
    long long trials;       /* trial evaluations (accepted + rejected) */
    long long backtracks;   /* rejected trials in total */
    double L;               /* current Lipschitz estimate L_n */
    double alpha;           /* alpha_n for the current L_n */
    double F, G, H;         /* energies at u^n */
    double H_prev;          /* H at u^{n-1} */
    double rel_change;      /* |H^n - H^{n-1}| / |H^n - G(f)| of the last accepted step */
    double last_gd;         /* <grad F(u^{n-1}), u^n - u^{n-1}> of the last accepted step */
    double last_dd;         /* |u^n - u^{n-1}|^2 */
    double last_dp;         /* <u^n - u^{n-1}, u^{n-1} - u^{n-2}> */
    int status;             /* fe_status of this image */
    int converged;          /* 1 once the tolerance of the last fe_solve was met */
    double G_floor;         /* G(f), the floor of the data term (read-only) */
} fe_info;

typedef struct fe_ctx fe_ctx;

/* Default parameters: nf = 0 and filters = NULL (caller sets them),
 * lambda 5, beta 0.8, L0 1, eta 2, c2 1e-6, max_backtrack 30, FP32.
 * Defines: the parameters of the problem of Eq. variant (Sec. II-B: filters
 * k_i, weights theta_i, lambda) and of iPiano's update rule (Sec. II-C: alpha
 * from L_n, beta).  The paper gives no values for beta, L0, eta, c2 or the
 * backtracking cap; these defaults are the readings stated above.
 * p: host pointer, overwritten in full.  No error: a NULL p is ignored. */
FE_API void fe_default_params(fe_params *p);

/* Create a context for nimg images of sizes H[j] x W[j] (each >= 8) with
 * observations f[j] (any pointer, H[j]*W[j] floats, all > 0 and finite) and
 * optional starting points u0[j] (any pointer, > 0; u0 == NULL or u0[j] ==
 * NULL means u^0 = f).  Allocates the device state, computes grad F(u^0),
 * F(u^0), G(u^0).  stream is a cudaStream_t (NULL = legacy default stream).
 * Defines: the problem argmin_{u>0} F(u) + G(u) of Eq. variant (Sec. II-B,
 * with the FoE prior of Eq. FOEmodel and the data term of Eq. dataterm2), or
 * of Eq. newmodel in w = log u (Sec. III-A), cast as Eq. fplusg (Sec. II-C);
 * the start u^{-1} = u^0 = f is a reading (the paper states no start).
 * Ownership: f, u0 and p are read during the call only; the context owns its
 * device state until fe_destroy.  *out receives the context (NULL on error).
 * Errors: FE_EINVAL, FE_ENOMEM, FE_ECUDA, FE_EUNSUPPORTED (*out is NULL). */
FE_API fe_status fe_init_batch(fe_ctx **out, const fe_params *p, int nimg,
                        const int *H, const int *W,
                        const float *const *f, const float *const *u0, void *stream);

/* Single-image form of fe_init_batch (same definition, arguments and
 * errors with nimg = 1). */
FE_API fe_status fe_init(fe_ctx **out, const fe_params *p, int H, int W,
                  const float *f, const float *u0, void *stream);

/* Restart every image from new observations (and optional starts) of the
 * same sizes, without reallocating.  Same argument rules as fe_init_batch.
 * Defines: the initialisation step of iPiano (Sec. II-C: u^{-1} = u^0, g^0 =
 * grad F(u^0)) on new data f; the counters n, trials, backtracks restart at 0
 * and L at fe_params.L0.  Errors: FE_EINVAL, FE_ECUDA. */
FE_API fe_status fe_reset(fe_ctx *ctx, const float *const *f, const float *const *u0);

/* Free the context and every device buffer it allocated (stream-ordered,
 * then synchronised).  Resource management: no counterpart in the paper.
 * ctx == NULL is a no-op.  The context must not be used afterwards. */
FE_API void fe_destroy(fe_ctx *ctx);

/* Run n accepted iPiano iterations on every image that has no error.
 * Defines: the basic update rule of iPiano, Sec. II-C,
 *   u^{n+1} = (I + alpha dG)^{-1}(u^n - alpha grad F(u^n) + beta (u^n - u^{n-1})),
 * with grad F and the closed-form prox of Eq. variant given there (or the
 * Newton prox of Eq. newmodel, Sec. III-A), and alpha_n from the backtracking
 * rule above (a reading: the paper names alpha and beta only).  The whole loop
 * runs on the device: one fused trial kernel per trial, accept/reject decided
 * on the device.  n >= 0 (0 is a no-op).  Asynchronous unless worst != NULL,
 * in which case it synchronises and stores the first non-OK per-image status
 * (or FE_OK) in *worst (host pointer).  Errors: FE_EINVAL, FE_ECUDA. */
FE_API fe_status fe_step(fe_ctx *ctx, int n, fe_status *worst);

/* Iterate until |H^{n+1}-H^n|/|H^{n+1}-G(f)| < rel_tol or max_iter accepted
 * iterations (counted from this call) on every image.  Synchronises.
 * Defines: the iPiano update rule of Sec. II-C (as fe_step) run to the
 * stopping rule above, which is a reading (the paper states none): the
 * relative change of H = F + G of Eq. fplusg, measured above the data-term
 * floor G(f).  rel_tol >= 0, max_iter >= 0.
 * Returns FE_OK if all images converged, FE_ENOTCONVERGED if some hit
 * max_iter, else the first error status (FE_EINVAL, FE_ECUDA, or a per-image
 * FE_ENONFINITE / FE_EBACKTRACK / FE_ETIMEOUT). */
FE_API fe_status fe_solve(fe_ctx *ctx, int max_iter, double rel_tol);

/* fe_solve with an energy target per image: image j also stops at the first
 * accepted iterate whose energy H = F + G (Eq. fplusg, Sec. II-C) is <=
 * H_target[j] (a stopping reading of this library; the paper states no
 * stopping rule).  H_target: host array of nimg doubles (-inf disables the
 * target of an image; NaN is rejected), or NULL (fe_solve).  rel_tol = 0
 * disables the relative-change rule.  It compares runs from different
 * starting points at the same energy (the learned warm start against plain
 * iPiano).  Returns as fe_solve: FE_OK when every image met a stopping rule,
 * FE_ENOTCONVERGED when some hit max_iter first, else the first error. */
FE_API fe_status fe_solve_to_energy(fe_ctx *ctx, int max_iter, double rel_tol, const double *H_target);

/* Summary of image img (synchronises): n, L_n, alpha_n of the update rule
 * (Sec. II-C) and F, G, H = F + G of Eq. fplusg at u^n.  out: host pointer.
 * Errors: FE_EINVAL (NULL, img out of range), FE_ECUDA. */
FE_API fe_status fe_get_info(fe_ctx *ctx, int img, fe_info *out);

/* Copy u^n of image img to out (any pointer, H*W floats, caller-owned);
 * FE_MODEL_COMBINED: u^n = e^{w^n}, the change of variables u = e^w of
 * Eq. original (Sec. II-C).  Synchronises.  Errors: FE_EINVAL, FE_ECUDA. */
FE_API fe_status fe_get_u(fe_ctx *ctx, int img, float *out);

/* Energies of an arbitrary iterate u (any pointer, H*W floats of image img's
 * size; u > 0 for FE_MODEL_VARIANT, w = log u for FE_MODEL_COMBINED) against
 * image img's f: E = F + G.  Any output pointer may be NULL (host pointers).
 * Defines: F = E_FoE of Eq. FOEmodel (Sec. II-A, rho(x) = log(1 + x^2)) and G =
 * the data term of Eq. dataterm2 (Sec. II-B), i.e. the objective of
 * Eq. variant; FE_MODEL_COMBINED: the objective of Eq. newmodel (Sec. III-A).
 * Sums in FP64.  Synchronises.  Errors: FE_EINVAL, FE_ECUDA. */
FE_API fe_status fe_energy(fe_ctx *ctx, int img, const float *u, double *E, double *F, double *G);

/* grad F at an arbitrary iterate (u, or w for FE_MODEL_COMBINED; any
 * pointer) into g (any pointer, caller-owned), both H*W floats of image img's
 * size; F into *F (host) if F != NULL.
 * Defines: grad_u F = sum_i theta_i K_i^T rho'(K_i u) (Sec. II-C, model
 * Eq. variant); grad_w F = sum_i theta_i W K_i^T rho'(K_i e^w), W = diag(e^w)
 * (Sec. II-C, models in w).  Synchronises.  Errors: FE_EINVAL, FE_ECUDA. */
FE_API fe_status fe_gradient(fe_ctx *ctx, int img, const float *u, float *g, double *F);

/* Checkpoint: copy u^n, u^{n-1}, grad F(u^n) (any pointers, H*W floats each;
 * any may be NULL) and the scalar state of image img.  These are the
 * quantities the update rule of Sec. II-C reads; the checkpoint itself has no
 * counterpart in the paper.  Synchronises.  Errors: FE_EINVAL, FE_ECUDA. */
FE_API fe_status fe_get_state(fe_ctx *ctx, int img, float *u, float *u_prev, float *g, fe_info *info);

/* Restore a checkpoint taken with fe_get_state (same sizes and params):
 * continuing from it reproduces the uninterrupted run bit for bit.  No
 * counterpart in the paper (see fe_get_state).  u, u_prev, g: any pointers,
 * none NULL; info: host pointer.  Errors: FE_EINVAL, FE_ECUDA. */
FE_API fe_status fe_set_state(fe_ctx *ctx, int img, const float *u, const float *u_prev,
                       const float *g, const fe_info *info);

/* Number of images / size of image img (H, W: host pointers).  Bookkeeping,
 * no counterpart in the paper.  fe_num_images(NULL) = 0; fe_image_size:
 * FE_EINVAL on NULL or an index out of range. */
FE_API int fe_num_images(const fe_ctx *ctx);
FE_API fe_status fe_image_size(const fe_ctx *ctx, int img, int *H, int *W);

/* Quality measures the paper reports (Sec. III), context-free.
 *
 * fe_ssim: mean SSIM index of x against the reference y (Wang, Bovik,
 * Sheikh, Simoncelli 2004, as cited in Sec. III): for every position where
 * an 11 x 11 window fits, the local means, variances and covariance under a
 * circular Gaussian window (sigma 1.5, weights summing to 1) give
 * ((2 mx my + C1)(2 sxy + C2)) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2)),
 * C1 = (0.01 peak)^2, C2 = (0.03 peak)^2; *out = the mean over the
 * (H - 10) x (W - 10) positions.  Moments in FP64.
 * fe_psnr: 10 log10(peak^2 / MSE) over n pixels (+inf if x == y).
 * x, y: DEVICE pointers (H*W or n floats, row-major); stream-ordered on
 * stream, synchronises it; allocates its partial sums with cudaMallocAsync.
 * Errors: FE_EINVAL (NULL, H or W < 11, peak <= 0, host pointers),
 * FE_ENOMEM, FE_ECUDA; message in fe_last_error(NULL). */
FE_API fe_status fe_ssim(const float *x, const float *y, int H, int W, double peak, double *out, void *stream);
FE_API fe_status fe_psnr(const float *x, const float *y, long long n, double peak, double *out, void *stream);

/* Output tile (rows x columns) of the context's trial kernel, as chosen by
 * the autotuner or given in fe_params.tile.  The paper has no counterpart
 * (a launch parameter of this implementation).  FE_EINVAL on NULL arguments. */
FE_API fe_status fe_tile_size(const fe_ctx *ctx, int *tile_y, int *tile_x);

/* CTAs that work on one tile (1, or 4 for a thread-block cluster per tile);
 * 0 for a NULL context.  No counterpart in the paper (launch parameter). */
FE_API int fe_tile_cluster(const fe_ctx *ctx);

/* Device kernel launches issued by this context since creation (trial,
 * gradient, energy and bookkeeping kernels), for launch accounting.  No
 * counterpart in the paper.  Synchronises the context's stream; 0 for NULL,
 * -1 if reading the device counter failed. */
FE_API long long fe_launch_count(const fe_ctx *ctx);

/* Select how fe_step/fe_solve drive the device loop of Sec. II-C's
 * iterations: 0 = host loop of per-trial kernel launches in chunks; 1 = one
 * CUDA graph whose device-side while node repeats a per-trial launch over
 * every tile of every active image; 2 (the default) = one CUDA graph holding
 * ONE persistent launch that runs every trial of every image: its CTAs take
 * tiles from per-image counters, and the block that decides an image's
 * trial releases the tiles of that image's next trial at once, so images
 * advance independently instead of in lockstep.  Mode 2 applies where a tile
 * runs on one CTA (every tensor-core form; the FP32 tiles without a
 * thread-block cluster) and runs as mode 1 otherwise; 3 = the persistent
 * launch of mode 2 issued directly, without a graph (for profilers that do
 * not follow kernels into conditional graph nodes; runs as mode 0 where
 * mode 2 runs as mode 1); modes 1 and 2 run as mode 0 on a driver without
 * conditional graph nodes.  All modes compute
 * the same iterates, energies and decisions bit for bit (each image's trials
 * and each trial's reduction order are the same).  A persistent launch in
 * which no trial is decided for 4 s stops; the images it left unfinished get
 * FE_ETIMEOUT.  The choice has no counterpart in the paper.  FE_EINVAL for
 * other modes or a NULL context. */
FE_API fe_status fe_set_loop_mode(fe_ctx *ctx, int mode);

/* Allocation-free gradient of one image: grad F(u) into g and F(u) into *F,
 * the same computation as fe_gradient, without a context.  The paper has no
 * counterpart; this entry exists for callers that may not allocate device
 * memory on the path where they call it (for example a plugin confined to a
 * host framework's fixed memory pool, or a real-time loop that forbids the
 * allocation calls and the synchronisation they can bring).
 *
 * All pointers are DEVICE pointers owned by the caller: u and g hold H*W
 * floats (row-major, pitch W; g must not alias u), filters holds nf*49 floats
 * (k_i[a][b] row-major), theta holds nf floats, F (may be NULL) one double.
 * Asynchronous on stream (a cudaStream_t, NULL = legacy default stream).
 *
 * No cudaMalloc, cudaFree or other allocating call is made.  The scratch
 * (tile list, weight tables, per-tile partial sums, counters) is one static
 * device array of about 0.3 MB that every GPU loading this library holds
 * until the process exits, which limits the image to at most 4096 tiles of
 * 64x64 pixels (e.g. 4096 x 4096); larger images return FE_EINVAL.  All calls
 * share that array and it keeps the last call's contents (each call rewrites
 * what it reads); calls whose kernels overlap on the GPU race on it and must
 * be serialised by the caller.  The first call on a device does a one-time
 * set-up with that device current (device address of the array, kernel
 * attribute) and should come before any stream capture.  That set-up belongs
 * to the device's primary context: after cudaDeviceReset the next call must
 * redo it, which happens by itself when a launch fails (the failed call
 * returns FE_ECUDA and forgets the set-up), so the call after it succeeds.
 * Errors: FE_EINVAL (NULL pointer, nf outside 1..64, H or W < 8, too many
 * tiles), FE_ECUDA; the message is in fe_last_error(NULL). */
FE_API fe_status fe_gradient_noalloc(const float *u, float *g, double *F, int H, int W,
                                     const float *filters, const float *theta, int nf,
                                     void *stream);

/* ---- Learned warm start ---------------------------------------------------
 * A small CNN predicts the starting point u^0 of iPiano from f.  The paper
 * has no counterpart (it starts from the observation); this is the warm-start
 * form of the solver, trained on (f, u*) pairs produced by the solver itself.
 *
 * Network: five 3x3 convolutions with zero padding, 1 -> 32 -> 32 -> 32 -> 32
 * -> 1 channels, bias, ReLU after the first four.  Input log f - 4.5, output
 * d, prediction u^0 = f exp(d) (positive by construction).  Loss
 * mean_p (d_p - (log u*_p - log f_p))^2.  Weights are stored in FP32 and used
 * in BF16 (round-to-nearest-even) by every convolution; activations and
 * accumulation are FP32; training uses Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * Parameter vector: for each layer, W[cout][cin][3][3] then b[cout].
 * Batches are B images of H x W, row-major, consecutive ("any" pointers).
 * All calls synchronise the stream given at creation.  Gradients are sums of
 * per-CTA partials added in FP64 in a fixed order, so the same inputs and
 * parameters give the same loss and gradient bit for bit on a given device.
 * Errors: FE_EINVAL (NULL net or required pointer, B, H or W < 1), FE_ENOMEM
 * (an allocation at creation), FE_ECUDA (a CUDA call failed, including
 * growing the activation buffers), FE_ETIMEOUT (a tensor-core completion
 * wait ran out: the results of that call are not valid); the message is in
 * fe_cnn_last_error(net). */
typedef struct fe_cnn fe_cnn;

/* Create with seeded He-normal weights (last layer scaled by 0.1). */
FE_API fe_status fe_cnn_create(fe_cnn **out, unsigned long long seed, void *stream);
FE_API void fe_cnn_destroy(fe_cnn *net);
FE_API int fe_cnn_num_params(const fe_cnn *net);
FE_API const char *fe_cnn_last_error(const fe_cnn *net);
/* Copy the FP32 parameters in/out (any pointer, fe_cnn_num_params floats). */
FE_API fe_status fe_cnn_set_params(fe_cnn *net, const float *params);
FE_API fe_status fe_cnn_get_params(fe_cnn *net, float *params);
/* Inference: u0 = f exp(d) and/or d (any pointers, may be NULL). */
FE_API fe_status fe_cnn_forward(fe_cnn *net, const float *f, int B, int H, int W, float *u0, float *d);
/* Loss and its gradient with respect to every parameter (grad may be NULL). */
FE_API fe_status fe_cnn_loss_grad(fe_cnn *net, const float *f, const float *u_target, int B, int H, int W,
                                  double *loss, float *grad);
/* One Adam step with learning rate lr; *loss = the loss before the step. */
FE_API fe_status fe_cnn_train_step(fe_cnn *net, const float *f, const float *u_target, int B, int H, int W,
                                   float lr, double *loss);

/* Diagnostic of the tensor-core building block used by the FE_TF32 / FE_BF16
 * forms (no counterpart in the paper: it tests the GEMM that the filter banks
 * k_i * u and K_i^T r of Sec. II-C run on): D = A * B^T with A 128 x K, B N x K (row-major float, any pointers)
 * rounded to the form's operand type (BF16 round-to-nearest-even, TF32
 * round-to-nearest), accumulated in FP32 by tcgen05.mma in tensor memory,
 * D 128 x N row-major float (any pointer).  prec = FE_BF16 (K multiple of 16)
 * or FE_TF32 (K multiple of 8), K <= 128, N in 16..64 multiple of 16.
 * Allocates and frees its own device buffers; synchronises the device.
 * Errors: FE_EINVAL, FE_ENOMEM, FE_ECUDA, FE_ETIMEOUT (MMA completion never
 * signalled within the wait bound). */
FE_API fe_status fe_tc_gemm_selftest(int prec, int N, int K, const float *A, const float *B, float *D);

/* Bounded-wait self-test (no counterpart in the paper): one CTA allocates
 * tensor memory, waits on an mbarrier that nothing ever completes with at
 * most max_iter polls (1 .. 2^24), frees the tensor memory and stores 1 in
 * *timed_out if the wait gave up (0 if it did not).  Returns FE_ETIMEOUT when
 * it gave up (the expected outcome), FE_EINVAL, FE_ENOMEM, FE_ECUDA.  The
 * trial kernels' MMA waits take the same bounded path. */
FE_API fe_status fe_tc_wait_selftest(unsigned max_iter, int *timed_out);

/* Bounded-wait self-test of the persistent trial launch (loop mode 2; no
 * counterpart in the paper): one warp runs the launch's tile claim against
 * one image whose only tile is taken, with the image still counted active
 * and no trial ever decided, and a wait limit of stall_s seconds (0 <
 * stall_s <= 5; the solver uses 4 s).  *aborted = 1 if the claim gave up
 * and raised the launch's abort flag (0 otherwise), *waited_s = the
 * kernel's duration.  Returns FE_ETIMEOUT when it gave up (the expected
 * outcome), FE_EINVAL, FE_ENOMEM, FE_ECUDA.  Allocates and frees its own
 * device buffer; synchronises the device. */
FE_API fe_status fe_persist_wait_selftest(double stall_s, int *aborted, double *waited_s);

/* ---- Peak-rate microbenchmarks ---------------------------------------------
 * Measured roofline denominators (no counterpart in the paper): the rate of
 * the units the solver's kernels are bound by, on the current device, each
 * timed in isolation (one warm-up launch that scales the work to about
 * target_ms, then the best of reps launches; CUDA events on a private stream,
 * synchronised).  CUDA-core kinds run every SM at full occupancy with 8
 * independent dependency chains per thread; tensor-core kinds run one CTA per
 * SM issuing a stream of M 128 x N 256 MMAs into one tensor-memory
 * accumulator (operands in shared memory).
 * *rate: operations per second of the whole device - flop for the FMA and
 * tensor kinds (2 per FMA, 4 per packed FMA, 2 M N K per MMA), instructions
 * (per thread) for the MUFU kinds.  *best_ms (may be NULL): the best launch
 * time; *sms (may be NULL): multiprocessors of the device.  Allocates no
 * device memory.  Errors: FE_EINVAL (kind outside the enum, reps outside
 * 1..100, target_ms outside (0, 2000], rate NULL), FE_ECUDA, FE_ETIMEOUT (a
 * tensor-core completion wait gave up; bounded by about 4e9 SM clocks). */
typedef enum {
    FE_PEAK_FFMA = 0,       /* fma.rn.f32 */
    FE_PEAK_FFMA2 = 1,      /* fma.rn.f32x2 (two FP32 FMAs per instruction) */
    FE_PEAK_DFMA = 2,       /* fma.rn.f64 */
    FE_PEAK_MUFU_RCP = 3,   /* rcp.approx.ftz.f32 */
    FE_PEAK_MUFU_LG2 = 4,   /* lg2.approx.ftz.f32 */
    FE_PEAK_TC_BF16 = 5,    /* tcgen05.mma kind::f16, BF16 operands, FP32 accumulation */
    FE_PEAK_TC_TF32 = 6     /* tcgen05.mma kind::tf32 */
} fe_peak_kind;
FE_API fe_status fe_peak(int kind, double target_ms, int reps, double *rate, double *best_ms, int *sms);

/* Multiprocessor count of the current device (cudaDevAttrMultiProcessorCount)
 * into *sms.  Errors: FE_EINVAL (NULL), FE_ECUDA. */
FE_API fe_status fe_device_sms(int *sms);

/* Error reporting and versioning (no counterpart in the paper).
 * fe_last_error: message of the last failure on ctx, or of the last
 * context-free call (ctx == NULL) on this host thread; the string is owned by
 * the library and valid until the next call on the same context / thread.
 * fe_status_string: static name of a status.  fe_abi_version: FE_ABI_VERSION
 * of the built library. */
FE_API const char *fe_last_error(const fe_ctx *ctx);
FE_API const char *fe_status_string(fe_status s);
FE_API int fe_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FE_H */
