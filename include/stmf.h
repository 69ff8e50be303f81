/*
 * stmf.h -- C ABI of the GB300 library for implicit symmetric CP fitting of moment tensors.
 *
 * The method (Sherman & Kolda, "Estimating Higher-Order Moments Using Symmetric Tensor
 * Decomposition", arXiv 1911.03813) fits a rank-r symmetric model
 *     M = sum_j lambda_j a_j^{(x)d}                                   (Sec. 1, eq. cp_element)
 * to the d-th moment tensor of p weighted samples
 *     X = sum_l nu_l v_l^{(x)d}                                       (Sec. 3, eq. tensorX)
 * by minimising f = ||X - M||^2 (Sec. 2.6, eq. optFunc) without ever forming X: the function
 * and gradient come from Alg. 2 (fg_implicit, Sec. 3.4), whose cost is one pass over the
 * samples.
 *
 * Conventions for every entry point
 * ---------------------------------
 *  - Memory: every array argument is a DEVICE pointer on the context's device unless the
 *    comment says "host". The caller owns all arrays it passes; the library never frees them.
 *    The library owns only its context (and the workspace the context allocates).
 *  - Layouts: the sample matrix V (the paper's n x p, one sample per column) is stored
 *    sample-major: p rows of `ld` elements, row l holding v_l in its first n entries (V stored
 *    column-major with leading dimension ld). The factor matrix A (n x r) is column-major with
 *    leading dimension n; G_A has the same layout. lambda and g_lambda hold r entries.
 *    All model parameters and outputs are FP64.
 *  - Errors: every call returns an stmf_status and never throws. Arguments are validated on
 *    the host before anything is launched; on a validation error nothing is launched and
 *    stmf_last_error() describes the failing argument. Kernel launch failures return
 *    STMF_ECUDA. Errors found on the device (a non-finite result, a bounded wait that ran out)
 *    are recorded in the context's device status word and surface through
 *    stmf_device_status().
 *  - Asynchrony: stmf_fg and stmf_norm_x only enqueue work on `stream` (NULL = the legacy
 *    default stream) and return; their outputs are valid once the stream reaches that point.
 *  - Devices: a context is bound to the device it was created on. Make that device current
 *    (cudaSetDevice) on the calling thread before each call, as for a cuBLAS handle; a call
 *    made with another device current returns STMF_EINVAL before anything is launched.
 *  - Threads and streams: a context may be used from one host thread at a time, and calls on
 *    different streams that share a context must not overlap on the device (they share the
 *    context's workspace). Use one context per concurrent stream.
 *  - Workspace: a context allocates its device workspace on first use and grows it when a call
 *    needs more. A call that grows it synchronises the device, so make the first call of each
 *    shape (or stmf_reserve) before capturing a CUDA graph.
 */
#ifndef STMF_H
#define STMF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define STMF_API __attribute__((visibility("default")))
#else
#define STMF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* stmf_stream_t; /* a cudaStream_t */

typedef enum {
  STMF_OK = 0,
  STMF_EINVAL = 1,      /* an argument is out of range or misaligned */
  STMF_ENOMEM = 2,      /* device allocation failed, or a request exceeds the memory budget */
  STMF_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  STMF_ETIMEOUT = 4,    /* a bounded device wait ran out */
  STMF_ENONFINITE = 5,  /* a result is NaN or infinite */
  STMF_ENOTREADY = 6,   /* the request is still running */
  STMF_ECANCELLED = 7,  /* the request was cancelled */
  STMF_EBUSY = 8,       /* no slot free */
  STMF_EUNSUPPORTED = 9 /* the device is not a GB300-class part (sm_103) */
} stmf_status;

typedef enum {
  STMF_F64 = 0,  /* IEEE binary64 */
  STMF_F32 = 1,  /* IEEE binary32 */
  STMF_BF16 = 2, /* bfloat16 */
  STMF_E4M3 = 3  /* OCP FP8 E4M3 with one FP32 scale per sample: v_l = scale[l] * q_l */
} stmf_dtype;

/* The samples V (the paper's n x p data matrix, Sec. 3), stored sample-major. */
typedef struct {
  const void* data;   /* device; p rows of ld elements of `dtype`; 16-byte aligned */
  const float* scale; /* device; p FP32 per-sample scales for STMF_E4M3, else NULL */
  int64_t n;          /* features per sample, 1 <= n <= 512 (see stmf_fg for n x r limits) */
  int64_t p;          /* number of samples, p >= 1 */
  int64_t ld;         /* row stride in elements, ld >= n, ld * sizeof(dtype) % 16 == 0 */
  int32_t dtype;      /* stmf_dtype */
  int32_t reserved;
} stmf_samples;

typedef struct stmf_ctx* stmf_ctx_t;

/* Library version, as 10000*major + 100*minor + patch. */
STMF_API int stmf_version(void);

/* Human-readable name of a status code (static storage). */
STMF_API const char* stmf_status_string(int status);

/* Create a context on CUDA device `device`. Fails with STMF_EUNSUPPORTED when the device is
 * not compute capability 10.3 (the kernels are built for sm_103a only). *out is set on
 * success. */
STMF_API stmf_status stmf_create(int device, stmf_ctx_t* out);

/* Destroy a context and free its workspace. Synchronises the device. NULL is accepted. */
STMF_API stmf_status stmf_destroy(stmf_ctx_t ctx);

/* Text describing the last error returned on this context (static per context; valid until
 * the next call on it). */
STMF_API const char* stmf_last_error(stmf_ctx_t ctx);

/* Grow the workspace so that stmf_fg / stmf_norm_x on V with rank r need no allocation.
 * Synchronises the device when it allocates. */
STMF_API stmf_status stmf_reserve(stmf_ctx_t ctx, const stmf_samples* V, int64_t r);

/* Read the device status word (STMF_OK or the first device-side error since the last read),
 * waiting for `stream`, and reset it to STMF_OK. *out_host is a host pointer. */
STMF_API stmf_status stmf_device_status(stmf_ctx_t ctx, stmf_stream_t stream, int32_t* out_host);

/*
 * stmf_fg -- function value and gradient by Alg. 2 (fg_implicit, Sec. 3.4):
 *     Y   = V D_nu [V^T A]^{d-1}            (Lemma 3.3, eq. Y)
 *     w_j = a_j^T y_j                       (Lemma 3.5: <X, M> = w^T lambda)
 *     B = A^T A, C = B^{d-1}, u = (B * C) lambda   (Lemma 3.4: ||M||^2 = lambda^T u)
 *     f   = alpha + lambda^T u - 2 w^T lambda     (eq. optFunc expanded)
 *     g_lambda = -2 (w - u)                        (eq. gradl)
 *     G_A = -2 d (Y - A D_lambda C) D_lambda       (eq. gradb)
 * Powers of matrices are element-wise (Sec. 2).
 *
 *  V        samples (see stmf_samples). BF16 and E4M3 samples are contracted on the tensor
 *           cores with FP32 accumulation (n <= 256, r <= 16); F32 with FP32 FMA; F64 with FP64
 *           FMA; other shapes on the CUDA cores in FP32 (FP64 for F64). Per-block partial sums
 *           are combined in FP64 and every step after Y runs in FP64. The CUDA-core pass stages 64
 *           samples in shared memory and holds Y in registers: it needs n x ceil4(r) <= 16384
 *           and 64 (n + 1) elements plus n x ceil4(r) of the compute type (FP32, or FP64 for
 *           F64 samples) within 227 KB; outside that the call returns STMF_EINVAL (for example
 *           F64 samples with n = 512, or n = 512 with r > 32).
 *  nu       device, p FP64 positive sample weights (Sec. 3 allows any positive vector), or NULL
 *           for the paper's default nu_l = 1/p.
 *  d        tensor order, 2 <= d <= 8 (d = 2 is the matrix case).
 *  r        rank, 1 <= r <= 64.
 *  lambda   device, r FP64.             A  device, n x r FP64 column-major (lda = n).
 *  alpha    device pointer to the FP64 constant alpha = ||X||^2 (e.g. from stmf_norm_x), or NULL
 *           for alpha = 0 (the shifted objective, Sec. 3.4).
 *  f        device, 1 FP64 (out).   g_lambda  device, r FP64 (out).   G_A  device, n x r (out).
 * Outputs may not alias inputs. Enqueued on `stream`; asynchronous.
 */
STMF_API stmf_status stmf_fg(stmf_ctx_t ctx, const stmf_samples* V, const double* nu, int32_t d,
                    int64_t r, const double* lambda, const double* A, const double* alpha,
                    double* f, double* g_lambda, double* G_A, stmf_stream_t stream);

/*
 * stmf_fg_host -- stmf_fg with every array in HOST memory (the end-to-end call). V (and nu, the
 * E4M3 scales) are streamed to the device in chunks of about 256 MB through three library-owned
 * staging buffers on one copy stream, so the copy of one chunk overlaps the pass over the
 * previous ones; chunk partials are summed in FP64 in chunk order; f, g_lambda and G_A are
 * copied back. Use pinned host memory for V: from pageable memory the copies do not overlap.
 *  V        host samples (stmf_samples with host pointers).   nu  host p FP64 or NULL (1/p).
 *  lambda   host r.   A  host n x r column-major.   alpha  the constant ||X||^2 of f (0: shifted).
 *  f, g_lambda, G_A   host outputs.
 * Synchronous: returns when the outputs are in host memory. The first call, and a call with
 * larger rows than before, allocates the staging buffers (synchronising the device).
 */
STMF_API stmf_status stmf_fg_host(stmf_ctx_t ctx, const stmf_samples* V, const double* nu,
                                  int32_t d, int64_t r, const double* lambda, const double* A,
                                  double alpha, double* f, double* g_lambda, double* G_A,
                                  stmf_stream_t stream);

/*
 * Sample-sharded evaluation. Every sum of Alg. 2 over samples (eq. Y, Lemma 3.5) splits over
 * disjoint shards of V, so G devices holding shards V_g each compute their partial (w, Y), the
 * partials are summed (one all-reduce of r + n r FP64 values), and the model terms follow:
 *
 * stmf_fg_partial -- yw = [w; vec(Y)] summed over this shard: w_j = sum_l nu_l (v_l^T a_j)^d,
 *   Y = sum_l nu_l (v_l^T A)^{d-1} v_l^T (n x r column-major after the r entries of w).
 *   nu       device weights of this shard's samples, or NULL for nu_l = 1 / p_total.
 *   p_total  the number of samples over all shards (used when nu is NULL; >= V->p).
 *   yw       device, r + n r FP64 (out).
 * stmf_fg_finish -- f, g_lambda, G_A from a summed yw (B = A^T A, C, u, then f and the gradients).
 *   n        features.   Other arguments as for stmf_fg.
 * Both enqueue on `stream`; asynchronous.
 */
STMF_API stmf_status stmf_fg_partial(stmf_ctx_t ctx, const stmf_samples* V, const double* nu,
                                     int64_t p_total, int32_t d, int64_t r, const double* lambda,
                                     const double* A, double* yw, stmf_stream_t stream);
STMF_API stmf_status stmf_fg_finish(stmf_ctx_t ctx, const double* yw, int64_t n, int32_t d,
                                    int64_t r, const double* lambda, const double* A,
                                    const double* alpha, double* f, double* g_lambda, double* G_A,
                                    stmf_stream_t stream);

/*
 * stmf_norm_x -- alpha = ||X||^2, the constant of Alg. 2 (Sec. 3.3), by the cheaper of the two
 * methods of stmf_norm_x_method (method 0).
 *
 * stmf_norm_x_method -- alpha = ||X||^2 by a chosen method:
 *  1  the Gram form nu^T (V^T V)^d nu (Lemma 3.4 applied to X), n p^2 / 2 multiply-adds, over
 *     the upper triangle of sample-tile pairs without forming the p x p Gram matrix;
 *  2  the distinct entries of the symmetric X (Sec. 3.3 notes that forming X can be cheaper than
 *     the implicit O(n p^2) route): X_m = sum_l nu_l prod_{i in m} v_li for every multiset m of
 *     d features and ||X||^2 = sum_m (d! / prod of the multiplicities' factorials) X_m^2, about
 *     p C(n+d-1, d) multiply-adds; needs C(n+d-2, d-1) <= 2^22 and, for FP64 samples, n <= 384
 *     (the first call for an (n, d) builds a prefix table and synchronises the device);
 *  0  the cheaper of the two by their operation counts.
 * Per-block sums are combined in FP64 in a fixed order (reproducible bit for bit).
 *  V, nu, d   as for stmf_fg.     alpha_out  device, 1 FP64 (out).
 * Enqueued on `stream`; asynchronous. STMF_EINVAL for an unknown method or a method-2 request
 * past its limits.
 */
STMF_API stmf_status stmf_norm_x(stmf_ctx_t ctx, const stmf_samples* V, const double* nu, int32_t d,
                        double* alpha_out, stmf_stream_t stream);
STMF_API stmf_status stmf_norm_x_method(stmf_ctx_t ctx, const stmf_samples* V, const double* nu,
                                        int32_t d, int32_t method, double* alpha_out,
                                        stmf_stream_t stream);

/*
 * stmf_set_pass_tiles -- launch shape of this context's tensor-core passes (not part of the
 * method): each CTA takes at least `min_tiles` tiles of 128 samples, so a pass over p samples
 * runs on min(#SMs, ceil(p / (128 min_tiles))) CTAs. A CTA of these passes holds a whole SM (its
 * shared memory): the default, 1, spreads every pass over all SMs, which is fastest for one
 * evaluation at a time; code that runs many small evaluations at once on other streams (the
 * server's fit slots use STMF_SERVER_PASS_TILES) gets more of them onto the GPU together with a
 * larger value. The grouping of per-CTA partial sums depends on the launch shape, so two contexts
 * give bit-identical results only with the same setting. STMF_EINVAL outside [1, 2^20].
 */
#define STMF_SERVER_PASS_TILES 128
STMF_API stmf_status stmf_set_pass_tiles(stmf_ctx_t ctx, int32_t min_tiles);

/*
 * Kernel timing for benchmarks (not part of the method). While enabled, every stmf_fg records
 * a pair of CUDA events around its fused pass over V, on the call's stream. stmf_profile_read
 * waits for the recorded events, returns the summed pass time in milliseconds and the number of
 * passes (host pointers), and clears the record. At most 65536 passes are recorded.
 */
STMF_API stmf_status stmf_profile_enable(stmf_ctx_t ctx, int32_t enable);
STMF_API stmf_status stmf_profile_read(stmf_ctx_t ctx, double* total_ms_host, int64_t* count_host);

/*
 * Optimiser options of stmf_fit. The paper (Sec. 4) runs L-BFGS-B without bounds, memory m = 5,
 * at most 10,000 iterations and 50,000 function evaluations, and a gradient tolerance pgtol that
 * varies by experiment (0.05 in Sec. 4.1, 1e-4 in Sec. 4.2). The other settings are this
 * library's readings of the solver's defaults (strong-Wolfe line search with c1 = 1e-3, c2 = 0.9).
 */
typedef struct {
  int32_t m;           /* number of stored correction pairs, 1..64 (paper: 5) */
  int32_t max_ls;      /* evaluations per line search (20) */
  double pgtol;        /* stop when max_i |g_i| <= pgtol */
  double factr;        /* stop when the relative decrease of f <= factr * DBL_EPSILON (1e7); the
                          decrease is measured against max(|f|, 1), so with F32/BF16/E4M3 samples,
                          whose evaluations carry ~1e-7 relative noise in f, use factr >= 1e9 or 0 */
  int64_t max_iters;   /* outer iterations (10,000) */
  int64_t max_evals;   /* function/gradient evaluations (50,000) */
  int32_t alpha_mode;  /* 1: f includes alpha = ||X||^2 (computed first); 0: shifted f, alpha = 0 */
  int32_t chunk;       /* evaluations enqueued between host reads of the done flag (16) */
} stmf_fit_opts;

/* Outcome of stmf_fit (host struct). stop_reason: 1 pgtol, 2 factr, 3 max_iters, 4 max_evals,
 * 5 line search failed, 6 non-finite value. status: the device status word (STMF_OK unless a
 * kernel reported an error). */
typedef struct {
  double f;          /* objective at the returned iterate (includes alpha when alpha_mode = 1) */
  double alpha;      /* ||X||^2 when alpha_mode = 1, else 0 */
  double g_inf;      /* max |g_i| at the returned iterate */
  int64_t iters;     /* outer iterations */
  int64_t evals;     /* function/gradient evaluations (the inner iterations of Sec. 4.1) */
  int32_t stop_reason;
  int32_t status;
} stmf_fit_result;

/* Fill *opts with the defaults listed above (pgtol = 1e-5). */
STMF_API stmf_status stmf_fit_default_opts(stmf_fit_opts* opts);

/*
 * stmf_fit -- minimise f(lambda, A) = ||X - M||^2 (eq. optFunc) from the start (lambda, A) with
 * the on-device L-BFGS described above; each evaluation is stmf_fg's Alg. 2. The optimiser state
 * (iterate, gradient, m correction pairs, line-search points) stays in device memory; the host
 * only reads a done flag once per `chunk` evaluations.
 *  V, nu, d, r   as for stmf_fg.
 *  opts          host pointer (see stmf_fit_default_opts).
 *  lambda, A     device; the start on entry (r FP64; n x r FP64 column-major), the final iterate
 *                on return.
 *  out           host; the result.
 * Synchronous: returns when the optimiser has stopped (work is issued on `stream`).
 */
STMF_API stmf_status stmf_fit(stmf_ctx_t ctx, const stmf_samples* V, const double* nu, int32_t d,
                     int64_t r, const stmf_fit_opts* opts, double* lambda, double* A,
                     stmf_fit_result* out, stmf_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * Serving: continuously batched fits (not part of the paper; a request is a fit of Sec. 4 with
 * several starts, of which the best final f is kept, as in Sec. 4.2's best-of-ten protocol).
 *
 * A server owns a scheduler thread and `max_fits` fit slots (a context, a CUDA stream and
 * preallocated workspaces each). Each start of a request occupies one slot and runs the
 * on-device L-BFGS of stmf_fit. Requests are admitted first-come first-served as soon as enough
 * slots are free and their device footprint fits the memory budget; fits of different requests
 * run at the same time on their own streams, so work that arrives while others run overlaps with
 * them on the GPU. Each fit's kernels use a fixed launch shape and fixed-order reductions, so a
 * result does not depend on what else is running. The slots' contexts take
 * STMF_SERVER_PASS_TILES tiles per CTA (stmf_set_pass_tiles), so that passes of many small fits
 * share the GPU.
 * ------------------------------------------------------------------------------------------ */
typedef struct stmf_server* stmf_server_t;

typedef struct {
  int32_t device;
  int32_t max_fits;      /* fit slots (concurrent starts), >= 1 */
  int32_t n_max;         /* largest n of any request (<= 512) */
  int32_t r_max;         /* largest r of any request (<= 64) */
  int32_t m_max;         /* largest L-BFGS memory of any request */
  int32_t reserved;
  size_t mem_budget;     /* device bytes: slot workspaces + admitted requests' footprints */
} stmf_server_config;

typedef struct {
  stmf_samples V;          /* data: device pointers, or host pointers when V_on_host = 1 */
  int32_t V_on_host;       /* 1: V.data (and V.scale) are host memory; the server copies them to
                              device memory it allocates at admission and frees at completion */
  int32_t d;
  int64_t r;
  int32_t n_starts;        /* >= 1 */
  int32_t reserved;
  const double* nu;        /* device p FP64 or NULL (1/p); must stay valid until completion */
  const double* x0;        /* host: n_starts start points, each [lambda (r); A (n x r, col-major)] */
  double* lambda_out;      /* device, r: best start's final lambda (NULL: not copied) */
  double* A_out;           /* device, n x r: best start's final A (NULL: not copied) */
  stmf_fit_opts opts;
} stmf_request;

typedef struct {
  int32_t state;           /* STMF_OK (done), STMF_ENOTREADY, STMF_ECANCELLED, or an error */
  int32_t best_start;
  stmf_fit_result best;    /* result of the start with the lowest final f */
  int64_t total_evals;     /* evaluations over all starts */
  double t_submit, t_admit, t_done;  /* seconds on the server's clock */
  size_t footprint;        /* device bytes charged to the request at admission */
} stmf_request_result;

typedef struct {
  int64_t submitted, admitted, completed, cancelled, failed;
  int32_t active_fits, queued;
  size_t bytes_in_use;     /* admitted footprints (excluding slot workspaces) */
  size_t peak_bytes_in_use;
  size_t slot_bytes;       /* preallocated slot workspaces */
  double now;              /* server clock, seconds */
  int32_t peak_active_fits; /* most fits that held a slot at the same time since creation */
  int32_t reserved;
} stmf_server_stats;

/* Create a server: allocates max_fits slots (fails with STMF_ENOMEM when they alone exceed
 * mem_budget) and starts the scheduler thread. */
STMF_API stmf_status stmf_server_create(const stmf_server_config* cfg, stmf_server_t* out);

/* Stop the scheduler (running requests are cancelled), free everything. */
STMF_API stmf_status stmf_server_destroy(stmf_server_t srv);

/* Queue a request. The struct and the start points x0 are copied at submission; samples given
 * in host memory (V_on_host = 1) are copied to the device at admission, so they (and device
 * samples, nu and the output buffers) must stay valid until the request has finished.
 * *ticket identifies the request. STMF_EINVAL for invalid arguments; STMF_ENOMEM when its
 * footprint alone exceeds what the budget leaves after the slots. */
STMF_API stmf_status stmf_submit(stmf_server_t srv, const stmf_request* req, uint64_t* ticket);

/* Wait up to timeout_ms (0: do not wait, < 0: no limit) for the request; fills *out (host) and
 * returns STMF_OK once it has finished (successfully or not: see out->state), STMF_ENOTREADY
 * while it is queued or running, STMF_EINVAL for an unknown ticket. The call that returns
 * STMF_OK delivers the result once and releases the ticket: later polls or cancels of it
 * return STMF_EINVAL, so a long-running server holds no memory for delivered requests. */
STMF_API stmf_status stmf_poll(stmf_server_t srv, uint64_t ticket, stmf_request_result* out,
                      int32_t timeout_ms);

/* Cancel a queued or running request; it finishes with state STMF_ECANCELLED. */
STMF_API stmf_status stmf_cancel(stmf_server_t srv, uint64_t ticket);

/* Counters of the server (host struct). */
STMF_API stmf_status stmf_server_get_stats(stmf_server_t srv, stmf_server_stats* out);

/*
 * stmf_rrf_start -- the randomized-range-finder start of eq. rrf (Sec. 4.2): A0 = V Omega with
 * unit-norm columns, Omega a p x r_hat Gaussian test matrix. Omega is never stored: entry (l, j)
 * is drawn inside the pass from Philox4x32-10 (Salmon et al., SC 2011) with counter
 * (l mod 2^32, l div 2^32, j, 0) and key (seed mod 2^32, seed div 2^32); the first two output
 * words give u1, u2 = (x + 1/2) 2^-32 and omega = sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller). FP64
 * samples: the draw, products and sums in FP64 on the CUDA cores. BF16 and E4M3 samples with
 * n <= 256 and r_hat <= 16: the tensor-core pass, the draw in FP32 as a BF16 hi/lo pair, FP32
 * accumulation folded every 8 tiles. Other samples: the draw and products in FP32 on the CUDA
 * cores, sums over 16 tiles folded into FP64. Either way about 1e-6 relative to the FP64 result;
 * the column normalisation is FP64.
 *  V        samples (any type).     r_hat  1..64 columns (n * r_hat limited by shared memory).
 *  seed     key of the generator.   A0     device, n x r_hat FP64 column-major (out).
 * Enqueued on `stream`; asynchronous.
 */
STMF_API stmf_status stmf_rrf_start(stmf_ctx_t ctx, const stmf_samples* V, int64_t r_hat, uint64_t seed,
                           double* A0, stmf_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * Sec. 5: massive or online data.
 * ------------------------------------------------------------------------------------------ */

/*
 * stmf_fg_sampled -- Alg. 2 on the stochastic Kruskal tensor of Lemma 5.1: the s rows
 * idx[0..s) of V (drawn with replacement by the caller; a row may repeat) with weights 1/s, whose
 * TTSVs X~ a^{d-1} are unbiased for X a^{d-1}. Arguments as for stmf_fg, plus
 *  idx   device, s int64 row indices in [0, V->p); an index outside that range reads as a zero
 *        sample and sets STMF_EINVAL in the device status word.
 * BF16, E4M3 and FP32 rows with n <= 256 and r <= 16 take the tensor-core passes, whose warps
 * copy the rows into the pass's stages; FP64 rows take the CUDA-core pass. Enqueued on `stream`;
 * asynchronous.
 */
STMF_API stmf_status stmf_fg_sampled(stmf_ctx_t ctx, const stmf_samples* V, const int64_t* idx, int64_t s,
                            int32_t d, int64_t r, const double* lambda, const double* A,
                            const double* alpha, double* f, double* g_lambda, double* G_A,
                            stmf_stream_t stream);

/* Adam (Kingma & Ba, 2015) with the schedule of Sec. 5 (paper values as defaults). */
typedef struct {
  double lr0;          /* initial learning rate (0.01) */
  double lr1;          /* rate after the first non-decrease (0.001) */
  double beta1, beta2, eps;   /* 0.9, 0.999, 1e-8 */
  int64_t epoch;       /* iterations per epoch (100) */
  int64_t max_epochs;  /* 0: no limit besides the index rows given */
} stmf_adam_opts;

typedef struct {
  double f_est;        /* estimated shifted f at the returned iterate */
  int64_t epochs;      /* epochs completed */
  int64_t iters;       /* Adam steps in the returned state */
  int32_t drops;       /* times the estimate did not decrease (2 = stopped) */
  int32_t status;      /* device status word */
} stmf_adam_result;

STMF_API stmf_status stmf_adam_default_opts(stmf_adam_opts* opts);

/*
 * stmf_adam -- Sec. 5's stochastic method: Adam on (lambda, A) with one sampled stochastic
 * gradient per iteration (Lemma 5.1), an estimate of the shifted objective after every epoch on
 * the fixed rows est_idx (Sec. 5 uses 1,000), the learning rate dropping to lr1 and the state
 * returning to the prior epoch at the first non-decrease, and a stop (returning the prior epoch's
 * iterate) at the second. Returning to the prior epoch restores the Adam moments and step count
 * too (this library's reading). All state stays on the device; the host reads one flag per epoch.
 *  sample_idx  device, iters x s int64: row t holds the s sampled rows of iteration t.
 *  est_idx     device, est_s int64: the fixed estimation rows.
 *  lambda, A   device; start on entry, final iterate on return.   out  host.
 * Synchronous (work on `stream`). Runs at most floor(iters / epoch) epochs.
 */
STMF_API stmf_status stmf_adam(stmf_ctx_t ctx, const stmf_samples* V, int32_t d, int64_t r,
                      const stmf_adam_opts* opts, const int64_t* sample_idx, int64_t iters,
                      int64_t s, const int64_t* est_idx, int64_t est_s, double* lambda, double* A,
                      stmf_adam_result* out, stmf_stream_t stream);

/*
 * stmf_fg_noalloc -- the evaluation of stmf_fg for callers that cannot allocate device memory.
 * The paper has no counterpart: this is an interface variant of stmf_fg (same kernels, same
 * arguments and results), added for callers such as code running inside a memory arena owned
 * by another runtime that forbids outside allocations, or a launch path where an allocation
 * would synchronise the device at the wrong time. stmf_fg cannot serve them because its context
 * allocates a status word and grows a workspace with cudaMalloc.
 *
 * No context: the scratch (block partial sums, reduced Y and w, A^T A, a status word) is one fixed
 * 8 MiB array of device globals in the library, held by every GPU that loads the library until
 * the process exits. The call never calls cudaMalloc, cudaFree or any allocating routine. The
 * first call on a device, with that device current, looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any stream capture.
 *
 * Limits: as for stmf_fg (n <= 512, r <= 64, 2 <= d <= 8). The pass runs at most
 * floor((2^20 - r^2) / ((n + 1) r)) - 1 blocks so that every request within these limits fits the
 * scratch (a request outside them returns STMF_EINVAL before any work; STMF_ENOMEM would mean
 * the scratch cannot hold two blocks' partials, which no valid n, r reaches).
 *
 * All calls on a device share the array and leave their contents in it. A call writes every
 * block partial it reads unless a block of its pass gave up on a bounded wait; such a block
 * records STMF_ETIMEOUT in the status word, and whenever the status word is nonzero by the time
 * the model terms run, f, g_lambda and G_A are written as NaN instead of a result, so partials
 * left by an earlier call never reach an output. Calls whose work overlaps on the GPU (other
 * streams or host threads) race on the array: serialise them. The cached address of the array
 * is looked up again on every call whose stream is not capturing (so a cudaDeviceReset between
 * calls is harmless); a call on a capturing stream returns STMF_EINVAL if no earlier call on
 * this device cached it.
 *
 *  V, nu, d, r, lambda, A, alpha, f, g_lambda, G_A   as for stmf_fg (device pointers).
 *  status   device, 1 int32 owned by the caller, or NULL. When given, device-side errors
 *           (STMF_ENONFINITE, STMF_ETIMEOUT) are recorded there; the call does not clear it,
 *           so a word still holding an earlier error also makes the outputs NaN. When NULL,
 *           errors go to a word inside the scratch that the call clears first, and the NaN
 *           outputs are the only sign of them.
 * Enqueued on `stream`; asynchronous; the current device must be the device of all pointers.
 */
STMF_API stmf_status stmf_fg_noalloc(const stmf_samples* V, const double* nu, int32_t d, int64_t r,
                            const double* lambda, const double* A, const double* alpha,
                            double* f, double* g_lambda, double* G_A, int32_t* status,
                            stmf_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* STMF_H */
