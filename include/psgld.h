/*
 * psgld.h -- C ABI of the GB300 (sm_103a) implementation of Parallel SGLD
 * (PSGLD) for matrix factorisation: Simsekli, Koptagel, Guldas, Cemgil,
 * Oztoprak, Birbil, "Parallel Stochastic Gradient Markov Chain Monte Carlo
 * for Matrix Factorisation Models" (2015).
 *
 * Model (Sec. 1 Eq. generative, Sec. 4 Eq. tweedienmf): V (I x J) ~ W H with
 * W (I x K), H (K x J); v_ij ~ Tweedie(mean sum_k w_ik h_kj, dispersion phi,
 * power p).  The paper writes the power as beta on the beta-divergence; the
 * two are related by p = 2 - beta (p = 0 Gaussian, 1 Poisson, 2 gamma,
 * 1 < p < 2 compound Poisson, 3 inverse Gaussian).
 *
 * Sampler (Sec. 3 Eq. psgld_w, Eq. psgld_h, Algorithm 1): [I] and [J] are cut
 * into B pieces; block (r, c) is row piece r x column piece c.  At iteration t
 * (1-based) the part holds the B blocks (r, (r + (t-1) mod B) mod B); every
 * block of the part updates its W rows and H columns at once, from the
 * factors of iteration t-1:
 *   w_ik += eps_t (S_t sum_{j in block} dlog p(v_ij)/dw_ik + dlog p(w_ik)/dw_ik)
 *           + sqrt(2 eps_t) z,   z ~ N(0, 1)
 * and the same for h_kj; S_t = N / |Pi_t| (observed entries over observed
 * entries of the part).  Non-negative models (exponential priors) mirror the
 * result, w <- |w| (Sec. 3.2).  A sweep is B consecutive iterations; together
 * they visit every block once.
 *
 * Conventions for every call:
 *   - Pointers named *_dev must be device memory of the context's GPU; pointers
 *     named *_host must be host memory.  Pointers named plainly (no suffix)
 *     may be either: the library copies through unified addressing.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream only enqueue work on it unless they
 *     return a host value, in which case they synchronise that stream.
 *   - No call is thread-safe on one context; distinct contexts are
 *     independent.  Nothing throws across the ABI; every failure returns a
 *     negative psgld_status and records a message for psgld_last_error().
 *   - All device memory the library allocates belongs to the context and is
 *     freed by psgld_destroy().  Caller buffers stay the caller's.
 */
#ifndef PSGLD_H
#define PSGLD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PSGLD_API __attribute__((visibility("default")))
#else
#define PSGLD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct psgld_ctx psgld_ctx;

typedef enum {
    PSGLD_OK = 0,
    PSGLD_ERR_ARG = -1,     /* invalid argument or input data */
    PSGLD_ERR_OOM = -2,     /* device allocation failed */
    PSGLD_ERR_CUDA = -3,    /* a CUDA runtime call failed */
    PSGLD_ERR_STATE = -4,   /* call not valid in the current state */
    PSGLD_ERR_TIMEOUT = -5, /* a bounded device wait ran out */
    PSGLD_ERR_SIZE = -6     /* input larger than a fixed maximum of the call */
} psgld_status;

/* Prior families.  Exponential priors (Sec. 4, Eq. tweedienmf) make the
 * model non-negative and turn on mirroring (Sec. 3.2).  Gaussian priors give
 * the unconstrained BPMF-like model the paper names in Sec. 1. */
typedef enum { PSGLD_PRIOR_EXPONENTIAL = 0, PSGLD_PRIOR_GAUSSIAN = 1 } psgld_prior_kind;

typedef struct {
    int32_t kind;             /* psgld_prior_kind */
    double lambda_w, lambda_h; /* exponential rates (kind 0), > 0 */
    double sigma_w, sigma_h;   /* Gaussian standard deviations (kind 1), > 0 */
} psgld_prior;

/* Step-size rule (Sec. 2 Eq. eps; Sec. 4.1 uses eps_t = (a/t)^b). */
typedef enum { PSGLD_EPS_FIXED = 0, PSGLD_EPS_POLY = 1 } psgld_eps_mode;
/* Likelihood scale S_t: N/|Pi_t| as in Eq. psgld_1, or the block count B. */
typedef enum { PSGLD_SCALE_N_OVER_PART = 0, PSGLD_SCALE_B = 1 } psgld_scale_mode;

typedef struct {
    uint64_t seed;            /* Philox key of the Langevin noise */
    int32_t eps_mode;         /* psgld_eps_mode */
    double eps;               /* fixed step (eps_mode 0), > 0 */
    double eps_a, eps_b;      /* eps_t = (a/t)^b (eps_mode 1), a > 0, b in (0.5, 1] */
    int32_t scale_mode;       /* psgld_scale_mode */
    double mu_min;            /* lower clamp of mu inside mu^(-p) when p > 0 */
    int32_t freeze_W;         /* 1: W is held fixed */
    int32_t freeze_H;         /* 1: H is held fixed */
    int64_t burn_in_sweeps;   /* sweeps discarded before posterior sums start */
    int32_t use_graphs;       /* 1: each sweep replays one captured CUDA graph */
    int32_t profile;          /* 1: time every part-step launch with CUDA events */
    int32_t dense_path;       /* dense V on the tensor cores, read when data is set:
                               * 0: off (dense V becomes the sparse layout of all
                               *    I*J entries, FP32 gather path);
                               * 1: on, kernel chosen by shape: single-pass for
                               *    blocks of at most 128 rows with K <= 128,
                               *    else two-sided;
                               * 2: on, two-sided kernel (K <= 256);
                               * 3: on, single-pass kernel (K <= 128, FP32 V) */
    int32_t dense_v_bf16;     /* 1: the two-sided kernel keeps V in BF16 */
    int32_t part_mode;        /* 0: cyclic part order, part (t-1) mod B at iteration t
                               * (Sec. 4.1); 1: at every iteration part s with
                               * probability |Pi_s| / N (condition C2, Sec. 3.1),
                               * drawn from the Philox stream of the seed with the
                               * counter (0, 0xFFFFFFFF, t_lo, 2 t_hi): with x the
                               * 64-bit number (word 1, word 0), r = floor(x N /
                               * 2^64) and s is the part whose range of the running
                               * sum of part sizes (parts 0 .. B-1) holds r.  Sweeps
                               * then run without CUDA graphs. */
    int32_t dense_fp8;        /* 1: the single-pass tensor-core kernel computes
                               * mu = W_b H_b from E4M3 (FP8) copies of the
                               * factors, each 128-row W tile and each 128-column
                               * H tile scaled by its largest |x| / 448, FP32
                               * accumulation; E and the gradient contractions
                               * stay BF16.  Needs dense_path 1 or 3, K <= 128,
                               * FP32 V (dense_path 1 then always takes the
                               * single-pass kernel). */
    int32_t gather_bf16;      /* 1: on the sparse path the gradient kernel gathers
                               * BF16 copies of the other factor's rows (half the
                               * bytes; the own row, the products and all sums stay
                               * FP32); the copies are rebuilt by psgld_set_factors
                               * and rewritten by every update.  Set it before
                               * psgld_set_factors. */
    int32_t max_sms;          /* > 0: the two-sided tensor-core kernel (persistent,
                               * one CTA per SM) runs on at most this many SMs, so
                               * that kernels of other streams find SMs free while
                               * it runs (a long-running chain beside short jobs);
                               * 0: every SM.  psgld_batch_sweep's shared launches
                               * use every SM regardless. */
    int32_t batch_ctas;       /* psgld_batch_sweep, read from the list's first
                               * context: CTAs of each persistent two-sided batch
                               * launch (0: one per SM).  Every item is computed by
                               * one CTA whichever CTA takes it, so the chains do
                               * not depend on it (a knob for the autotuner). */
    int32_t batch_update_blocks; /* psgld_batch_sweep: thread blocks of each batch
                               * update launch, a grid-stride loop over all items
                               * (0: one per 256 items, at most 2432); results do
                               * not depend on it. */
    int32_t debug_wait_polls; /* for testing the timeout path; 0 (the default): the
                               * normal limit of every bounded device wait (2^24
                               * polls or about one second of SM clock).  > 0: the
                               * sparse gradient kernel's first wait for its row
                               * gathers makes at most this many polls, without
                               * suspending and before it issues the copies, then
                               * gives up -- a wait that surely runs out, on
                               * purpose: the kernel sets the context's error
                               * flag, waits for its own copies with the normal
                               * limit, and the next synchronising call returns
                               * PSGLD_ERR_TIMEOUT naming the kernel and the wait.
                               * The part-step's result is then undefined; the
                               * context stays usable (set the factors again). */
    int32_t wide_col_blocks;  /* two-sided tensor-core kernel: the first this many
                               * blocks of a part have columns items of 256 H^T
                               * rows (two accumulators sharing each W tile), the
                               * rest 128-row items, which even out the end of the
                               * launch; -1 (the default): half the blocks.  Every
                               * G row is the same sum either way, so the chains do
                               * not depend on it (a knob for the autotuner). */
    int32_t dense_share_e;    /* two-sided tensor-core kernel, read when the data are
                               * set: 1: the columns items take E from the rows items
                               * of their block (mu and E formed once per entry, E
                               * through HBM, columns items wait for their block's
                               * rows items); 0: every item forms its own mu and E
                               * (V kept in both orientations); -1 (the default): 1
                               * for row pieces of at least 512 rows whose part fills
                               * more than one wave of CTAs, else 0.  The chains
                               * differ by rounding only (mu = W H^T from either
                               * orientation's MMAs). */
} psgld_options;

/* Device memory.  By default the library allocates with cudaMalloc and frees
 * with cudaFree (which waits for the whole device).  A caller that runs many
 * contexts side by side on streams (a serving loop) can hand in its own
 * allocator instead: alloc returns `bytes` of device memory of the current
 * device, aligned to at least 256 bytes, or NULL; `stream` is the stream of
 * the call that allocates (NULL for psgld_create); free returns memory that
 * alloc gave.  The library frees a buffer only after the work that uses it has
 * finished.  Contexts created after the call use the allocator (each keeps a
 * copy); NULL restores cudaMalloc / cudaFree.  Not thread-safe with concurrent
 * psgld_create calls. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, void *stream, void *user);
    void *user;
} psgld_allocator;

PSGLD_API psgld_status psgld_set_allocator(const psgld_allocator *allocator_host);

/* Defaults: seed 0, fixed eps 1e-4, a = 0.01, b = 0.51, scale N/|Pi_t|,
 * mu_min 1e-10, nothing frozen, no burn-in, graphs on, profiling off,
 * dense_path off, cyclic parts. */
PSGLD_API void psgld_default_options(psgld_options *opt_host);

/* Create a context on the current CUDA device.
 * I, J >= 1; 1 <= B <= min(I, J); 1 <= K <= 512; phi > 0; tweedie_p not in
 * (0, 1) (no Tweedie model exists for 1 < beta < 2, Sec. 4); I, J and
 * B * max(I, J) below 2^31.
 * *out receives the new context, or NULL on failure. */
PSGLD_API psgld_status psgld_create(int64_t I, int64_t J, int32_t K, int32_t B,
                          double tweedie_p, double phi,
                          const psgld_prior *prior_host, psgld_ctx **out);

PSGLD_API psgld_status psgld_set_options(psgld_ctx *ctx, const psgld_options *opt_host);

/* Observed entries in coordinate form: i[n] in [0, I), j[n] in [0, J),
 * v[n] (float), n < nnz.  Pairs must be unique; non-negative models require
 * v >= 0.  The library builds its own part-major layouts on the device
 * (rows of each part sorted by column, columns of each part sorted by row)
 * and keeps no reference to the caller's arrays after the call returns.
 * Synchronises `stream`.  Resets the iteration counter and posterior sums. */
PSGLD_API psgld_status psgld_set_data_coo(psgld_ctx *ctx, int64_t nnz, const int32_t *i,
                                const int32_t *j, const float *v, void *stream);

/* Dense V (every entry observed), row-major with leading dimension ld >= J;
 * non-negative models require V >= 0, and every entry must be finite.
 * With dense_path = 0: the same effect as psgld_set_data_coo over all I*J
 * entries.  With dense_path > 0: the library keeps its own copies of V and
 * each block of a part (Definitions 1-2) computes its gradient terms as a
 * GEMM -> Tweedie epilogue -> GEMM chain on the tensor cores (Sec. 4,
 * Eq. psgld_w, Eq. psgld_h): mu = W_b H_b with BF16 operands and FP32
 * accumulation, E = (V_b - mu) max(mu, mu_min)^(-p) / phi rounded to BF16,
 * E H_b^T and E^T W_b with FP32 accumulation; the update, noise and mirror
 * stay FP32 as on the sparse path.  The single-pass kernel computes mu once
 * per entry; the two-sided kernel computes it once for the W rows and once
 * for the H columns, so that every gradient row is summed by one CTA.
 * PSGLD_ERR_ARG if K > 256 (K > 128 for dense_path = 3).
 * psgld_part_layout is not available for such data (PSGLD_ERR_STATE).
 * Synchronises `stream`.  Resets the iteration counter and posterior sums. */
PSGLD_API psgld_status psgld_set_data_dense(psgld_ctx *ctx, const float *V, int64_t ld,
                                  void *stream);

/* Factors in: W is I x K row-major; Ht is H transposed, J x K row-major.
 * Non-negative models require all entries >= 0. */
PSGLD_API psgld_status psgld_set_factors(psgld_ctx *ctx, const float *W, const float *Ht,
                               void *stream);
/* Factors out, same layouts.  Either pointer may be NULL. */
PSGLD_API psgld_status psgld_get_factors(psgld_ctx *ctx, float *W, float *Ht, void *stream);

/* One PSGLD iteration t (1-based): Algorithm 1's loop body for part
 * Pi_t, on `stream`.  Does not touch the posterior sums. */
PSGLD_API psgld_status psgld_part_step(psgld_ctx *ctx, int64_t t, void *stream);

/* n_sweeps sweeps of B iterations each, continuing from the iteration
 * counter, which must sit at a sweep boundary (a multiple of B).  After each
 * sweep past burn-in the FP64 posterior sums of W, W^2, H, H^2 are updated. */
PSGLD_API psgld_status psgld_sweep(psgld_ctx *ctx, int32_t n_sweeps, void *stream);

/* n_sweeps sweeps of each of the n contexts, their part-steps sharing
 * launches: at every part of a sweep one gradient launch per group of
 * contexts on the same tensor-core kernel variant covers the blocks of all
 * of them -- single-pass contexts grouped by K class (K rounded up to 16,
 * 32, 64 or 128) and GEMM1 precision, two-sided contexts by K width (K
 * rounded up to 64), V type and Tweedie power, the latter as one persistent
 * launch over all their items -- and one update launch covers all the
 * contexts' rows; then each context's posterior sums as in psgld_sweep.
 * Every context must hold dense data on a tensor-core kernel (dense_path 1,
 * 2 or 3), the same B, cyclic parts and its iteration counter at a sweep
 * boundary; sizes, powers, priors, seeds and step sizes may differ.  Each
 * context ends in the same state, bit for bit, as after psgld_sweep(ctx,
 * n_sweeps).  The work is enqueued on `stream` (the call returns before it
 * runs, like psgld_sweep); the launches' parameter tables are kept by the
 * first context of the list and reused by its next batch.  A context may be
 * in one batch at a time: a call whose list shares a context with a batch
 * still running on another stream must be ordered after it by the caller.
 * With use_graphs (the first context's option, and profile off), each sweep
 * of the batch replays one captured CUDA graph holding all its launches,
 * kept by the first context per parity of the ping-pong buffers and per
 * posterior-accumulation flag, and captured again when the batch's launch
 * structure (contexts per kernel variant, grid sizes, knobs) changes. */
PSGLD_API psgld_status psgld_batch_sweep(psgld_ctx *const *ctxs_host, int32_t n, int32_t n_sweeps,
                                         void *stream);

/* Monte Carlo posterior mean and variance of W (I x K) and H^T (J x K), FP64,
 * over the samples kept so far (population variance): the Monte Carlo
 * averages over the samples after burn-in that the paper reports for its
 * audio experiment (Sec. 4, shared-memory setting, experiments on audio:
 * the samples of the burn-in phase are discarded),
 * here one sample per sweep.  Any output pointer may be NULL.  Waits for the
 * context's last enqueued work. */
PSGLD_API psgld_status psgld_posterior_mean(psgld_ctx *ctx, double *Wmean_host,
                                  double *Wvar_host, double *Hmean_host,
                                  double *Hvar_host, int64_t *n_samples_host);

/* -(1/phi) sum over observed entries of d_beta(v || mu) at the current
 * factors (the log-likelihood up to the mu-free normaliser, Sec. 4), FP64.
 * mu is formed in FP64 for every observed entry: over dense data that is an
 * FP64 product W H of I x J x K multiply-adds, bounded by the GPU's FP64
 * rate (about 0.57 s at 32768 x 32768, K = 256, on GB300). */
PSGLD_API psgld_status psgld_log_lik(psgld_ctx *ctx, double *out_host, void *stream);

/* sqrt(mean over observed entries of (v - mu)^2), FP64; mu from the current
 * factors (use_posterior_mean = 0) or from the posterior means (1).  The
 * root mean squared error between V and W H that the paper monitors over
 * the iterations of its MovieLens experiment (Sec. 4, distributed-hybrid
 * setting), on the observed entries. */
PSGLD_API psgld_status psgld_rmse(psgld_ctx *ctx, int32_t use_posterior_mean,
                        double *out_host, void *stream);

/* ---- checkpoint and resume ----------------------------------------------
 * A chain's whole state is its factors (psgld_get_factors / _set_factors),
 * the FP64 posterior sums and three counters; the options (seed included)
 * and the data are the caller's.  The Langevin noise of iteration t is a
 * function of (seed, t, matrix, row, column) only (Sec. 2's N(0, 2 eps)
 * drawn from a counter-based Philox stream), so a chain restored into a
 * fresh context with the same options and data continues bit for bit as if
 * it had not stopped. */

/* Copies the state out: sums of W and W^2 (I x K) and of H^T and (H^T)^2
 * (J x K), row-major FP64 host arrays (any may be NULL), and
 * counters_host[0..2] = iterations done t, sweeps done, posterior samples
 * kept (may be NULL).  Waits for the context's last enqueued work. */
PSGLD_API psgld_status psgld_get_state(psgld_ctx *ctx, double *sW_host, double *sW2_host,
                                       double *sH_host, double *sH2_host, int64_t *counters_host);

/* Restores a state taken with psgld_get_state, after psgld_set_data_* and
 * psgld_set_factors (setting data clears the sums and counters).  All four
 * sums and the counters are required; PSGLD_ERR_ARG if a pointer is NULL or
 * the counters are inconsistent (t < 0, sweeps < 0, samples outside
 * [0, sweeps]); PSGLD_ERR_STATE before the factors are set.  Synchronous. */
PSGLD_API psgld_status psgld_set_state(psgld_ctx *ctx, const double *sW_host, const double *sW2_host,
                                       const double *sH_host, const double *sH2_host,
                                       const int64_t *counters_host);

/* ---- introspection: the schedule and layouts, for bit-exact checks ------ */

/* Piece boundaries (Definition 1): row_starts[r] = floor(r I / B) for
 * r = 0..B, the same for columns.  Host arrays of B+1 entries. */
PSGLD_API psgld_status psgld_piece_bounds(const psgld_ctx *ctx, int64_t *row_starts_host,
                                int64_t *col_starts_host);
/* Part of iteration t (Definition 2): col_piece_host[r] is the column piece
 * joined with row piece r, r = 0..B-1.  With part_mode = 1 the part depends
 * on the data's part sizes: PSGLD_ERR_STATE before data is set. */
PSGLD_API psgld_status psgld_part_schedule(const psgld_ctx *ctx, int64_t t,
                                 int32_t *col_piece_host);
/* Row-major layout of part s (0 <= s < B): row_ptr_host[0..I] offsets
 * (relative to the part's first entry) and the column of every entry of the
 * part, rows in order, columns ascending.  cols_host may be NULL to query the
 * count, which is written to *n_entries_host. */
PSGLD_API psgld_status psgld_part_layout(psgld_ctx *ctx, int32_t s, int32_t *row_ptr_host,
                               int32_t *cols_host, int64_t *n_entries_host);
/* Device time of the part-step kernels recorded since the last call, with
 * profile = 1: *total_ms_host receives their summed CUDA-event durations and
 * *launches_host their count.  Events are recorded on the launch stream
 * around each part-step kernel, also inside captured sweep graphs; each
 * iteration of a part owns one event pair, so read after every call that
 * runs at most B iterations (one sweep) for complete figures (with
 * part_mode = 1 a part can recur within a sweep: read after every
 * part-step).  Synchronises
 * the context's last stream. */
PSGLD_API psgld_status psgld_profile_read(psgld_ctx *ctx, double *total_ms_host,
                                          int64_t *launches_host);
/* The same split at the end of the gradient kernel (the sparse gather kernel
 * or the tensor-core chain): *grad_ms_host and *update_ms_host receive the
 * summed durations of the gradient and of the update launches. */
PSGLD_API psgld_status psgld_profile_read_split(psgld_ctx *ctx, double *grad_ms_host,
                                                double *update_ms_host, int64_t *launches_host);

/* Last completed iteration t (0 before the first). */
PSGLD_API int64_t psgld_iterations_done(const psgld_ctx *ctx);

/* Device bytes a context holds once its data is set (psgld_create plus
 * psgld_set_data_*; scratch that those calls free before returning is not
 * counted), for a scheduler that admits work against a memory budget.
 * nnz: observed entries (ignored when dense_path > 0, where V is I x J).
 * -1 on invalid sizes.  Needs no GPU. */
PSGLD_API int64_t psgld_estimate_device_bytes(int64_t I, int64_t J, int32_t K, int32_t B,
                                              int64_t nnz, int32_t dense_path,
                                              int32_t dense_v_bf16);

/* ---- log-likelihood without allocation ----------------------------------
 * No counterpart in the paper: a convenience for callers that cannot
 * allocate device memory when they need the number (their device memory is
 * reserved by another allocator, or they run where an allocation would
 * synchronise the device or is not allowed).  It needs no context and
 * allocates nothing: its only scratch, one FP64 partial sum per 4096 entries,
 * is a fixed 32 KB array compiled into the library, present on every GPU that
 * loads the library until the process exits.
 *
 * Writes to *out_dev (device memory) -(1/phi) sum_n d_beta(v[n] || mu_n),
 * mu_n = sum_k W[i[n]*K + k] * Ht[j[n]*K + k] (max(mu, mu_min) when
 * tweedie_p > 0), the value psgld_log_lik reports for the same entries and
 * factors.  i_dev, j_dev, v_dev hold nnz entries; W_dev is I x K and Ht_dev
 * J x K, row-major without padding; all are device memory and stay the
 * caller's.  Enqueued on `stream` (NULL = legacy default stream); nothing is
 * synchronised.
 *
 * Limits and errors: nnz <= PSGLD_STATIC_MAX_NNZ, else PSGLD_ERR_SIZE;
 * PSGLD_ERR_ARG for other invalid arguments (nnz < 0, I, J or K < 1, a null
 * pointer, phi <= 0, tweedie_p in (0, 1), mu_min <= 0); PSGLD_ERR_CUDA if a
 * launch fails.  Entry indices are checked on the device: an entry with i
 * outside [0, I) or j outside [0, J) is never read, and *out_dev becomes NaN.
 * There is no context, so no message is recorded.
 *
 * The first call on a device looks up the scratch array's device address
 * (with that device current) and caches it per device ordinal: make that
 * first call before any stream capture.  The cached address is that of the
 * device's primary context (the CUDA runtime's and PyTorch's); it is not
 * valid after cudaDeviceReset or under a context made with the driver API.
 * All calls share the array; calls that can overlap on the same GPU
 * (different streams without ordering) race and must be serialised by the
 * caller.  Each call writes every partial slot it reads, so no state
 * carries over from one call to the next. */
#define PSGLD_STATIC_MAX_NNZ (4096ll * 4096ll)
PSGLD_API psgld_status psgld_log_lik_static(int64_t nnz, const int32_t *i_dev,
                                            const int32_t *j_dev, const float *v_dev,
                                            const float *W_dev, const float *Ht_dev,
                                            int64_t I, int64_t J, int32_t K,
                                            double tweedie_p, double phi, double mu_min,
                                            double *out_dev, void *stream);

/* Message of the last failure on this context ("" if none).  Valid until the
 * next call on the context. */
PSGLD_API const char *psgld_last_error(const psgld_ctx *ctx);

PSGLD_API void psgld_destroy(psgld_ctx *ctx);

/* ---- Native serving loop --------------------------------------------------
 * Continuous batching of dense factorisation jobs on one GPU, run by two
 * worker threads inside the library.  Submitted jobs wait in arrival order
 * until the device memory their context will hold (psgld_estimate_device_bytes)
 * fits in what the budget has left; the admission thread then sets them up
 * (context, data and factor copies with their input checks, on the server's
 * admission stream) and later reads back and releases finished ones.  The
 * batch thread keeps up to `max_inflight` psgld_batch_sweep calls of one
 * sweep each queued on its batch stream, each over every set-up job with
 * sweeps left, so jobs arriving meanwhile join at the next sweep, and never
 * waits for a set-up or a read-back.  Contexts allocate from a CUDA
 * stream-ordered memory pool, so releasing one does not wait for the whole
 * device.  A job's chain depends only on its own inputs and seed: its result
 * is the same alone and in any mix.  Not the paper's (its experiments run
 * one chain at a time); this is the serving form of Algorithm 1 for many
 * concurrent chains. */
typedef struct psgld_server psgld_server;

typedef struct {
    int64_t I, J;
    int32_t K, B;
    double tweedie_p, phi;
    psgld_prior prior;
    psgld_options options;    /* seed, step size, burn_in_sweeps, dense_path
                               * (1, 2 or 3), dense_v_bf16, ... as for a context */
    int32_t sweeps;           /* sweeps to run, > 0 */
    const float *V_dev;       /* I x J, row stride ldv >= J, FP32, device memory */
    int64_t ldv;
    const float *W0_dev;      /* I x K initial W, device memory */
    const float *Ht0_dev;     /* J x K initial H^T, device memory */
    double *Wmean_host;       /* I x K posterior mean of W (or NULL) */
    double *Hmean_host;       /* J x K posterior mean of H^T (or NULL) */
} psgld_job;
/* The caller keeps V, W0, Ht0 and the output buffers valid and unchanged
 * until the job is reported done by psgld_server_poll. */

/* hbm_budget: bytes the admitted jobs' contexts may hold together; a job
 * whose own estimate exceeds it is refused at submission (PSGLD_ERR_SIZE).
 * max_inflight >= 1: batch sweeps queued at a time. */
PSGLD_API psgld_status psgld_server_create(size_t hbm_budget, int32_t max_inflight,
                                           psgld_server **srv_out);
/* Queues a job (copied; the pointers it holds are not) and returns its id.
 * Thread-safe with respect to polling. */
PSGLD_API psgld_status psgld_server_submit(psgld_server *srv, const psgld_job *job,
                                           int64_t *id_out);
/* Up to `max` jobs finished since the last poll: their ids and their latency
 * (seconds from submission to the read-back of their results; negative if
 * the job failed, with psgld_server_last_error naming why).  Returns the
 * number written. */
PSGLD_API int32_t psgld_server_poll(psgld_server *srv, int64_t *ids_host, double *latency_s_host,
                                    int32_t max);
/* Waits until every submitted job has finished (PSGLD_ERR_TIMEOUT after
 * timeout_s seconds). */
PSGLD_API psgld_status psgld_server_wait_idle(psgld_server *srv, double timeout_s);
/* Batch sweeps issued, mean jobs per batch sweep, peak bytes held. */
PSGLD_API psgld_status psgld_server_stats(psgld_server *srv, int64_t *sweeps_out,
                                          double *jobs_per_sweep_out, size_t *peak_bytes_out);
/* Message of the latest failed job ("" if none); valid until the next call. */
PSGLD_API const char *psgld_server_last_error(psgld_server *srv);
/* Finishes every submitted job, stops the worker and frees the server. */
PSGLD_API void psgld_server_destroy(psgld_server *srv);

#ifdef __cplusplus
}
#endif
#endif
