/*
 * psgld_oracle.h -- plain FP64 CPU oracle of Parallel SGLD for matrix
 * factorisation (Simsekli et al., "Parallel Stochastic Gradient Markov Chain
 * Monte Carlo for Matrix Factorisation Models", 2015).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library.  It
 * is called only by the test suite, by the smoke check and by the CPU-baseline
 * leg of the benchmark.  The product library never links, loads or calls it,
 * and it shares no code, header, table or constant with the CUDA path.
 *
 * Everything here is slow and literal on purpose: FP64 throughout, one loop
 * per equation, no blocking and no reordering beyond what the equations state.
 *
 * Parity pins (what fixes each function independently of itself) are listed
 * in the test files; every function below is pinned.
 */
#ifndef PSGLD_ORACLE_H
#define PSGLD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Prior kinds.  Exponential priors (Sec. 4, Eq. tweedienmf) come with the
 * mirroring step of Sec. 3.2 and Algorithm 1; Gaussian priors are the
 * BPMF-like special case named in Sec. 1. */
enum { OR_PRIOR_EXPONENTIAL = 0, OR_PRIOR_GAUSSIAN = 1 };
/* Step-size rules: fixed epsilon, or epsilon_t = (a/t)^b (Sec. 4.1). */
enum { OR_EPS_FIXED = 0, OR_EPS_POLY = 1 };
/* Likelihood scale: N/|Pi_t| (Eq. psgld_1) or the block count B. */
enum { OR_SCALE_N_OVER_PART = 0, OR_SCALE_B = 1 };

typedef struct or_model or_model;

/* ---- the model (Sec. 1 Eq. generative, Sec. 4 Eq. tweedienmf) ---------- */
or_model *or_create(int64_t I, int64_t J, int32_t K, int32_t B, double p,
                    double phi, int32_t prior_kind, double lambda_w,
                    double lambda_h, double sigma_w, double sigma_h);
void or_destroy(or_model *m);
void or_set_options(or_model *m, uint64_t seed, int32_t eps_mode, double eps,
                    double eps_a, double eps_b, int32_t scale_mode,
                    double mu_min, int32_t freeze_W, int32_t freeze_H,
                    int64_t burn_in_sweeps);
/* Observed entries (i, j, v), 0-based.  Returns 0, or -1 on a duplicate or
 * out-of-range index. */
int or_set_data(or_model *m, int64_t nnz, const int32_t *i, const int32_t *j,
                const double *v);
/* W is I x K row-major; H is K x J row-major (the paper's orientation). */
void or_set_factors(or_model *m, const double *W, const double *H);
void or_get_factors(const or_model *m, double *W, double *H);

/* ---- partition and part schedule (Definitions 1-2, Sec. 4.1) ----------- */
int64_t or_piece_start(int64_t r, int64_t n, int32_t B);
int32_t or_piece_of(int64_t x, int64_t n, int32_t B);
/* Column piece of the block that row piece r joins in the part used at
 * iteration t (1-based). */
int32_t or_part_col_piece(int64_t t, int32_t B, int32_t r);
/* Entries of block (r, c), in the oracle's block-sorted order (row, then
 * column).  Returns the count; copies up to cap entries. */
int64_t or_block_entries(const or_model *m, int32_t r, int32_t c, int64_t cap,
                         int32_t *i_out, int32_t *j_out);
int64_t or_part_size(const or_model *m, int64_t t);
/* Part order: 0 cyclic (Sec. 4.1, the default), 1 size-proportional random
 * choice at every iteration (condition C2 of Sec. 3.1). */
void or_set_part_mode(or_model *m, int32_t mode);
/* Index s of the part used at iteration t (its blocks are (r, (r+s) mod B)). */
int32_t or_part_index(const or_model *m, int64_t t);

/* ---- random numbers ------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                      uint32_t out[4]);
/* Standard normal used for element k of factor row `row` of matrix `mat`
 * (0 = W, 1 = H; for H the row is the column index j) at iteration t. */
double or_noise(uint64_t seed, int64_t t, int32_t mat, int64_t row, int32_t k);
/* The same normals for rows 0..nrows-1, elements 0..K-1: out[row*K + k]. */
void or_noise_matrix(uint64_t seed, int64_t t, int32_t mat, int64_t nrows,
                     int32_t K, double *out);

/* ---- one iteration of Algorithm 1 ---------------------------------------- */
double or_eps(const or_model *m, int64_t t);
double or_scale(const or_model *m, int64_t t);
/* Drift of Eq. psgld_w / psgld_h at iteration t, evaluated at the current
 * factors: S * sum_{(i,j) in Pi_t} grad log p(v_ij | .) + grad log p(.). */
void or_drift(const or_model *m, int64_t t, double *dW, double *dH);
void or_part_step(or_model *m, int64_t t);
/* n full sweeps of B part-steps from the current iteration counter (which
 * must sit at a sweep boundary); accumulates the posterior sums at the end of
 * every sweep past burn-in.  Returns 0, or -1 if not at a boundary. */
int or_sweep(or_model *m, int32_t n);
int64_t or_iterations_done(const or_model *m);
/* Threads for the blocks of a part (OpenMP); results do not depend on it.
 * n <= 0 only queries.  Returns the number now in use. */
int32_t or_set_threads(int32_t n);

/* ---- posterior summaries and diagnostics --------------------------------- */
void or_posterior(const or_model *m, double *Wmean, double *Wvar,
                  double *Hmean, double *Hvar, int64_t *n_samples);
/* beta-divergence d_beta(v || mu) with beta = 2 - p (Sec. 4). */
double or_beta_div(double v, double mu, double p);
/* -(1/phi) sum_obs d_beta(v || mu) at the current factors. */
double or_log_lik(const or_model *m);
/* the same sum restricted to the part used at iteration t */
double or_log_lik_part(const or_model *m, int64_t t);
/* log-likelihood part plus the log-prior terms (up to constants). */
double or_log_post(const or_model *m);
/* RMSE of v against the reconstruction on the observed entries; from the
 * current factors (use_mean = 0) or the posterior means (use_mean = 1). */
double or_rmse(const or_model *m, int32_t use_mean);

#ifdef __cplusplus
}
#endif
#endif
