/*
 * psgld_oracle.c -- plain FP64 CPU oracle of Parallel SGLD (PSGLD) for
 * matrix factorisation, Simsekli et al. 2015.
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product library.  It shares no
 * code with the CUDA path.
 *
 * Passages followed (section / equation / algorithm of the paper):
 *   model ............. Sec. 1 Eq. generative, Eq. fullbayes; Sec. 4 Eq. tweedienmf
 *   Tweedie density ... Sec. 4: TW(v; mu, phi, beta) ~ exp(-d_beta(v||mu)/phi)
 *   blocks, parts ..... Sec. 3 Definitions 1 and 2; cyclic part order, Sec. 4.1
 *   updates ........... Sec. 3 Eq. psgld_1, Eq. psgld_w, Eq. psgld_h
 *   noise ............. Sec. 2: N(0, 2 eps) entries of the noise matrices
 *   step size ......... Sec. 2 Eq. eps; eps_t = (a/t)^b, Sec. 4.1
 *   mirroring ......... Sec. 3.2 and Algorithm 1
 *   Algorithm 1 ....... the loop over t with a ForPar over the blocks of a part
 *   posterior means ... Monte Carlo averages after burn-in, Sec. 4.1.2
 *
 * Readings of points the paper leaves open (each one is listed with its
 * reason in the design notes of the repository):
 *   - the W and H updates of one iteration both read (W^(t-1), H^(t-1));
 *   - N is the number of observed entries, |Pi_t| the observed entries of
 *     the part;
 *   - piece r of [n] is [floor(r n / B), floor((r+1) n / B));
 *   - at iteration t the part pairs row piece r with column piece
 *     (r + (t-1) mod B) mod B;
 *   - mu is clamped below by mu_min in the Tweedie factor when p > 0;
 *   - exponential priors: the state is kept non-negative (mirroring), so the
 *     prior gradient is -lambda; Gaussian priors: -w / sigma^2;
 *   - noise: Philox4x32-10 keyed by the seed, counter (k/4, row, t, matrix),
 *     Box-Muller on the two pairs of 23-bit uniforms.
 */
#include "psgld_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

struct or_model {
    int64_t I, J;
    int32_t K, B;
    double p, phi;
    int32_t prior_kind;
    double lambda_w, lambda_h, sigma_w, sigma_h;
    /* options */
    uint64_t seed;
    int32_t eps_mode;
    double eps, eps_a, eps_b;
    int32_t scale_mode;
    int32_t part_mode;        /* 0: cyclic order; 1: size-proportional draw (C2) */
    double mu_min;
    int32_t freeze_W, freeze_H;
    int64_t burn_in;
    /* observed entries grouped by block (r, c) at index r*B + c, each block
     * sorted by row then column */
    int64_t N;
    int64_t *blk_ptr;
    int32_t *ent_i, *ent_j;
    double *ent_v;
    /* state */
    double *W; /* I x K, row-major */
    double *H; /* K x J, row-major */
    int64_t t_done;
    int64_t sweeps_done;
    /* posterior sums */
    double *sW, *sW2, *sH, *sH2;
    int64_t n_samples;
};

/* ------------------------------------------------------------------------ */
/* Partition and schedule (Definitions 1 and 2)                             */
/* ------------------------------------------------------------------------ */

int64_t or_piece_start(int64_t r, int64_t n, int32_t B)
{
    return (r * n) / B;
}

int32_t or_piece_of(int64_t x, int64_t n, int32_t B)
{
    for (int32_t r = 0; r < B; ++r)
        if (x >= or_piece_start(r, n, B) && x < or_piece_start(r + 1, n, B))
            return r;
    return -1;
}

int32_t or_part_col_piece(int64_t t, int32_t B, int32_t r)
{
    int64_t s = (t - 1) % B;
    return (int32_t)((r + s) % B);
}

/* ------------------------------------------------------------------------ */
/* Model set-up                                                             */
/* ------------------------------------------------------------------------ */

or_model *or_create(int64_t I, int64_t J, int32_t K, int32_t B, double p,
                    double phi, int32_t prior_kind, double lambda_w,
                    double lambda_h, double sigma_w, double sigma_h)
{
    or_model *m = (or_model *)calloc(1, sizeof(or_model));
    m->I = I; m->J = J; m->K = K; m->B = B;
    m->p = p; m->phi = phi;
    m->prior_kind = prior_kind;
    m->lambda_w = lambda_w; m->lambda_h = lambda_h;
    m->sigma_w = sigma_w; m->sigma_h = sigma_h;
    m->seed = 0;
    m->eps_mode = OR_EPS_FIXED;
    m->eps = 1e-4;
    m->eps_a = 0.01; m->eps_b = 0.51;
    m->scale_mode = OR_SCALE_N_OVER_PART;
    m->mu_min = 1e-10;
    m->blk_ptr = (int64_t *)calloc((size_t)B * B + 1, sizeof(int64_t));
    m->W = (double *)calloc((size_t)(I * K), sizeof(double));
    m->H = (double *)calloc((size_t)(K * J), sizeof(double));
    m->sW = (double *)calloc((size_t)(I * K), sizeof(double));
    m->sW2 = (double *)calloc((size_t)(I * K), sizeof(double));
    m->sH = (double *)calloc((size_t)(K * J), sizeof(double));
    m->sH2 = (double *)calloc((size_t)(K * J), sizeof(double));
    return m;
}

void or_destroy(or_model *m)
{
    if (!m) return;
    free(m->blk_ptr); free(m->ent_i); free(m->ent_j); free(m->ent_v);
    free(m->W); free(m->H); free(m->sW); free(m->sW2); free(m->sH); free(m->sH2);
    free(m);
}

void or_set_options(or_model *m, uint64_t seed, int32_t eps_mode, double eps,
                    double eps_a, double eps_b, int32_t scale_mode,
                    double mu_min, int32_t freeze_W, int32_t freeze_H,
                    int64_t burn_in_sweeps)
{
    m->seed = seed;
    m->eps_mode = eps_mode;
    m->eps = eps; m->eps_a = eps_a; m->eps_b = eps_b;
    m->scale_mode = scale_mode;
    m->mu_min = mu_min;
    m->freeze_W = freeze_W; m->freeze_H = freeze_H;
    m->burn_in = burn_in_sweeps;
}

/* Sort key used inside one block: row, then column. */
static const int32_t *g_sort_i, *g_sort_j;
static int cmp_row_col(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    if (g_sort_i[x] != g_sort_i[y]) return g_sort_i[x] < g_sort_i[y] ? -1 : 1;
    if (g_sort_j[x] != g_sort_j[y]) return g_sort_j[x] < g_sort_j[y] ? -1 : 1;
    return 0;
}

int or_set_data(or_model *m, int64_t nnz, const int32_t *i, const int32_t *j,
                const double *v)
{
    int32_t B = m->B;
    int64_t nb = (int64_t)B * B;
    for (int64_t e = 0; e < nnz; ++e)
        if (i[e] < 0 || i[e] >= m->I || j[e] < 0 || j[e] >= m->J) return -1;

    /* block of every entry (Definition 1) */
    int64_t *blk = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz ? nnz : 1));
    memset(m->blk_ptr, 0, sizeof(int64_t) * (size_t)(nb + 1));
    for (int64_t e = 0; e < nnz; ++e) {
        int32_t r = or_piece_of(i[e], m->I, B);
        int32_t c = or_piece_of(j[e], m->J, B);
        blk[e] = (int64_t)r * B + c;
        m->blk_ptr[blk[e] + 1] += 1;
    }
    for (int64_t b = 0; b < nb; ++b) m->blk_ptr[b + 1] += m->blk_ptr[b];

    /* group by block, then sort each block by (row, column) */
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz ? nnz : 1));
    int64_t *fill = (int64_t *)calloc((size_t)(nb > 0 ? nb : 1), sizeof(int64_t));
    for (int64_t e = 0; e < nnz; ++e)
        order[m->blk_ptr[blk[e]] + fill[blk[e]]++] = e;
    g_sort_i = i; g_sort_j = j;
    for (int64_t b = 0; b < nb; ++b)
        qsort(order + m->blk_ptr[b], (size_t)(m->blk_ptr[b + 1] - m->blk_ptr[b]),
              sizeof(int64_t), cmp_row_col);

    free(m->ent_i); free(m->ent_j); free(m->ent_v);
    m->ent_i = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    m->ent_j = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    m->ent_v = (double *)malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
    int dup = 0;
    for (int64_t n = 0; n < nnz; ++n) {
        int64_t e = order[n];
        m->ent_i[n] = i[e]; m->ent_j[n] = j[e]; m->ent_v[n] = v[e];
        if (n > 0 && m->ent_i[n] == m->ent_i[n - 1] && m->ent_j[n] == m->ent_j[n - 1])
            dup = 1;
    }
    m->N = nnz;
    free(blk); free(order); free(fill);
    return dup ? -1 : 0;
}

void or_set_factors(or_model *m, const double *W, const double *H)
{
    memcpy(m->W, W, sizeof(double) * (size_t)(m->I * m->K));
    memcpy(m->H, H, sizeof(double) * (size_t)(m->K * m->J));
}

void or_get_factors(const or_model *m, double *W, double *H)
{
    if (W) memcpy(W, m->W, sizeof(double) * (size_t)(m->I * m->K));
    if (H) memcpy(H, m->H, sizeof(double) * (size_t)(m->K * m->J));
}

int64_t or_block_entries(const or_model *m, int32_t r, int32_t c, int64_t cap,
                         int32_t *i_out, int32_t *j_out)
{
    int64_t b = (int64_t)r * m->B + c;
    int64_t lo = m->blk_ptr[b], hi = m->blk_ptr[b + 1];
    for (int64_t n = lo; n < hi && n - lo < cap; ++n) {
        i_out[n - lo] = m->ent_i[n];
        j_out[n - lo] = m->ent_j[n];
    }
    return hi - lo;
}

/* |Pi_t|: observed entries in the B blocks of the part used at iteration t */
/* Observed entries of part s (blocks (r, (r + s) mod B), Definition 2). */
static int64_t part_entries(const or_model *m, int32_t s)
{
    int64_t n = 0;
    for (int32_t r = 0; r < m->B; ++r) {
        int64_t b = (int64_t)r * m->B + (r + s) % m->B;
        n += m->blk_ptr[b + 1] - m->blk_ptr[b];
    }
    return n;
}

void or_set_part_mode(or_model *m, int32_t mode) { m->part_mode = mode; }

/* The part used at iteration t.  Cyclic: s = (t - 1) mod B (Sec. 4.1).
 * Size-proportional (condition C2 of Sec. 3.1): part s with probability
 * |Pi_s| / N, drawn independently at every t from the Philox stream keyed by
 * the seed, counter (0, 0xFFFFFFFF, t_lo, 2 t_hi) -- a counter no noise draw
 * uses (their second word is a row index below 2^31).  With x the 64-bit
 * number (word 1, word 0) of the draw, r = floor(x N / 2^64) is uniform on
 * [0, N) up to 2^-64, and s is the part whose range of the running sum of
 * part sizes (parts in order 0 .. B-1) holds r. */
int32_t or_part_index(const or_model *m, int64_t t)
{
    if (m->part_mode == 0 || m->N == 0) return (int32_t)((t - 1) % m->B);
    const uint32_t ctr[4] = {0u, 0xFFFFFFFFu, (uint32_t)(uint64_t)t,
                             (uint32_t)((uint64_t)t >> 32) << 1};
    const uint32_t key[2] = {(uint32_t)m->seed, (uint32_t)(m->seed >> 32)};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    const uint64_t x64 = ((uint64_t)x[1] << 32) | x[0];
    const uint64_t r = (uint64_t)(((unsigned __int128)x64 * (uint64_t)m->N) >> 64);
    uint64_t cum = 0;
    for (int32_t s = 0; s < m->B; ++s) {
        cum += (uint64_t)part_entries(m, s);
        if (r < cum) return s;
    }
    return m->B - 1;
}

static int32_t col_piece(const or_model *m, int64_t t, int32_t r)
{
    return (r + or_part_index(m, t)) % m->B;
}

int64_t or_part_size(const or_model *m, int64_t t)
{
    return part_entries(m, or_part_index(m, t));
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 and Box-Muller                                             */
/* ------------------------------------------------------------------------ */

/* One Philox4x32 round: two 32x32->64 products of words 0 and 2 with the
 * round multipliers, the high halves mixed with words 1, 3 and the key. */
static void philox_round(uint32_t x[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x[2];
    uint32_t y0 = (uint32_t)(p1 >> 32) ^ x[1] ^ k[0];
    uint32_t y1 = (uint32_t)p1;
    uint32_t y2 = (uint32_t)(p0 >> 32) ^ x[3] ^ k[1];
    uint32_t y3 = (uint32_t)p0;
    x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3;
}

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {          /* Weyl key schedule */
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(x, k);
    }
    out[0] = x[0]; out[1] = x[1]; out[2] = x[2]; out[3] = x[3];
}

/* Four standard normals for elements 4q..4q+3 of one factor row. */
static void or_noise4(uint64_t seed, int64_t t, int32_t mat, int64_t row,
                      int64_t q, double z[4])
{
    uint32_t ctr[4] = {(uint32_t)q, (uint32_t)row, (uint32_t)(uint64_t)t,
                       (uint32_t)(((uint64_t)t >> 32) << 1) | (uint32_t)mat};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    double u[4];
    for (int n = 0; n < 4; ++n)               /* uniform on (0, 1) */
        u[n] = ((double)(x[n] >> 9) + 0.5) / 8388608.0;
    const double two_pi = 6.283185307179586476925286766559;
    double r0 = sqrt(-2.0 * log(u[0])), r1 = sqrt(-2.0 * log(u[2]));
    z[0] = r0 * cos(two_pi * u[1]);
    z[1] = r0 * sin(two_pi * u[1]);
    z[2] = r1 * cos(two_pi * u[3]);
    z[3] = r1 * sin(two_pi * u[3]);
}

double or_noise(uint64_t seed, int64_t t, int32_t mat, int64_t row, int32_t k)
{
    double z[4];
    or_noise4(seed, t, mat, row, k / 4, z);
    return z[k % 4];
}

void or_noise_matrix(uint64_t seed, int64_t t, int32_t mat, int64_t nrows,
                     int32_t K, double *out)
{
    for (int64_t row = 0; row < nrows; ++row)
        for (int32_t k = 0; k < K; ++k)
            out[row * K + k] = or_noise(seed, t, mat, row, k);
}

/* ------------------------------------------------------------------------ */
/* One PSGLD iteration                                                      */
/* ------------------------------------------------------------------------ */

double or_eps(const or_model *m, int64_t t)
{
    if (m->eps_mode == OR_EPS_POLY) return pow(m->eps_a / (double)t, m->eps_b);
    return m->eps;
}

double or_scale(const or_model *m, int64_t t)
{
    if (m->scale_mode == OR_SCALE_B) return (double)m->B;
    int64_t n = or_part_size(m, t);
    return n > 0 ? (double)m->N / (double)n : 0.0;
}

/* d/dmu log TW(v; mu, phi, p) = (v - mu) mu^(-p) / phi  (from d_beta, Sec. 4) */
static double tweedie_grad(const or_model *m, double v, double mu)
{
    if (m->p == 0.0) return (v - mu) / m->phi;
    double mc = mu > m->mu_min ? mu : m->mu_min;
    return (v - mu) * pow(mc, -m->p) / m->phi;
}

static double prior_grad(const or_model *m, int32_t mat, double x)
{
    if (m->prior_kind == OR_PRIOR_EXPONENTIAL) return mat == 0 ? -m->lambda_w : -m->lambda_h;
    double s = mat == 0 ? m->sigma_w : m->sigma_h;
    return -x / (s * s);
}

void or_drift(const or_model *m, int64_t t, double *dW, double *dH)
{
    const int64_t I = m->I, J = m->J;
    const int32_t K = m->K, B = m->B;
    const double S = or_scale(m, t);
    memset(dW, 0, sizeof(double) * (size_t)(I * K));
    memset(dH, 0, sizeof(double) * (size_t)(K * J));

    /* likelihood part, one block of the part at a time (blocks share no rows
     * and no columns, so they write disjoint parts of dW and dH) */
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t r = 0; r < B; ++r) {
        int32_t c = col_piece(m, t, r);
        int64_t b = (int64_t)r * B + c;
        for (int64_t n = m->blk_ptr[b]; n < m->blk_ptr[b + 1]; ++n) {
            int64_t i = m->ent_i[n], j = m->ent_j[n];
            double mu = 0.0;
            for (int32_t k = 0; k < K; ++k) mu += m->W[i * K + k] * m->H[(int64_t)k * J + j];
            double e = tweedie_grad(m, m->ent_v[n], mu);
            for (int32_t k = 0; k < K; ++k) {
                dW[i * K + k] += e * m->H[(int64_t)k * J + j];
                dH[(int64_t)k * J + j] += e * m->W[i * K + k];
            }
        }
    }
    /* scale and prior */
#pragma omp parallel for
    for (int64_t i = 0; i < I; ++i)
        for (int32_t k = 0; k < K; ++k)
            dW[i * K + k] = S * dW[i * K + k] + prior_grad(m, 0, m->W[i * K + k]);
#pragma omp parallel for
    for (int64_t j = 0; j < J; ++j)
        for (int32_t k = 0; k < K; ++k)
            dH[(int64_t)k * J + j] = S * dH[(int64_t)k * J + j] + prior_grad(m, 1, m->H[(int64_t)k * J + j]);
}

void or_part_step(or_model *m, int64_t t)
{
    const int64_t I = m->I, J = m->J;
    const int32_t K = m->K;
    const double eps = or_eps(m, t);
    const double sd = sqrt(2.0 * eps);          /* noise variance is 2 eps */
    const int mirror = m->prior_kind == OR_PRIOR_EXPONENTIAL;
    double *dW = (double *)malloc(sizeof(double) * (size_t)(I * K));
    double *dH = (double *)malloc(sizeof(double) * (size_t)(K * J));

    /* both drifts from (W^(t-1), H^(t-1)) */
    or_drift(m, t, dW, dH);

    if (!m->freeze_W) {
#pragma omp parallel for
        for (int64_t i = 0; i < I; ++i)
            for (int32_t q = 0; 4 * q < K; ++q) {
                double z[4];
                or_noise4(m->seed, t, 0, i, q, z);
                for (int32_t n = 0; n < 4 && 4 * q + n < K; ++n) {
                    int64_t a = i * K + 4 * q + n;
                    double w = m->W[a] + eps * dW[a] + sd * z[n];
                    m->W[a] = mirror ? fabs(w) : w;
                }
            }
    }
    if (!m->freeze_H) {
#pragma omp parallel for
        for (int64_t j = 0; j < J; ++j)
            for (int32_t q = 0; 4 * q < K; ++q) {
                double z[4];
                or_noise4(m->seed, t, 1, j, q, z);
                for (int32_t n = 0; n < 4 && 4 * q + n < K; ++n) {
                    int64_t a = (int64_t)(4 * q + n) * J + j;
                    double h = m->H[a] + eps * dH[a] + sd * z[n];
                    m->H[a] = mirror ? fabs(h) : h;
                }
            }
    }
    free(dW); free(dH);
    m->t_done = t;
}

int64_t or_iterations_done(const or_model *m) { return m->t_done; }

int32_t or_set_threads(int32_t n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int or_sweep(or_model *m, int32_t n)
{
    if (m->t_done % m->B != 0) return -1;
    for (int32_t s = 0; s < n; ++s) {
        for (int32_t b = 0; b < m->B; ++b) or_part_step(m, m->t_done + 1);
        if (m->sweeps_done >= m->burn_in) {
            for (int64_t a = 0; a < m->I * m->K; ++a) {
                m->sW[a] += m->W[a];
                m->sW2[a] += m->W[a] * m->W[a];
            }
            for (int64_t a = 0; a < (int64_t)m->K * m->J; ++a) {
                m->sH[a] += m->H[a];
                m->sH2[a] += m->H[a] * m->H[a];
            }
            m->n_samples += 1;
        }
        m->sweeps_done += 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Posterior summaries and diagnostics                                      */
/* ------------------------------------------------------------------------ */

void or_posterior(const or_model *m, double *Wmean, double *Wvar, double *Hmean,
                  double *Hvar, int64_t *n_samples)
{
    double n = (double)m->n_samples;
    for (int64_t a = 0; a < m->I * m->K; ++a) {
        double mean = n > 0 ? m->sW[a] / n : 0.0;
        if (Wmean) Wmean[a] = mean;
        if (Wvar) Wvar[a] = n > 0 ? m->sW2[a] / n - mean * mean : 0.0;
    }
    for (int64_t a = 0; a < (int64_t)m->K * m->J; ++a) {
        double mean = n > 0 ? m->sH[a] / n : 0.0;
        if (Hmean) Hmean[a] = mean;
        if (Hvar) Hvar[a] = n > 0 ? m->sH2[a] / n - mean * mean : 0.0;
    }
    if (n_samples) *n_samples = m->n_samples;
}

double or_beta_div(double v, double mu, double p)
{
    double beta = 2.0 - p;
    if (beta == 2.0) return 0.5 * (v - mu) * (v - mu);       /* Euclidean */
    if (beta == 1.0)                                         /* Kullback-Leibler */
        return (v > 0.0 ? v * log(v / mu) : 0.0) - v + mu;
    if (beta == 0.0) return v / mu - log(v / mu) - 1.0;       /* Itakura-Saito */
    return pow(v, beta) / (beta * (beta - 1.0)) - v * pow(mu, beta - 1.0) / (beta - 1.0)
           + pow(mu, beta) / beta;
}

static double or_mu(const or_model *m, const double *W, const double *H, int64_t i, int64_t j)
{
    double mu = 0.0;
    for (int32_t k = 0; k < m->K; ++k) mu += W[i * m->K + k] * H[(int64_t)k * m->J + j];
    return mu;
}

static double log_lik_range(const or_model *m, int64_t lo, int64_t hi)
{
    double s = 0.0;
    for (int64_t n = lo; n < hi; ++n) {
        double mu = or_mu(m, m->W, m->H, m->ent_i[n], m->ent_j[n]);
        if (m->p > 0.0 && mu < m->mu_min) mu = m->mu_min;
        s += or_beta_div(m->ent_v[n], mu, m->p);
    }
    return -s / m->phi;
}

double or_log_lik(const or_model *m)
{
    return log_lik_range(m, 0, m->N);
}

/* -(1/phi) sum over the part used at iteration t */
double or_log_lik_part(const or_model *m, int64_t t)
{
    double s = 0.0;
    for (int32_t r = 0; r < m->B; ++r) {
        int64_t b = (int64_t)r * m->B + col_piece(m, t, r);
        s += log_lik_range(m, m->blk_ptr[b], m->blk_ptr[b + 1]);
    }
    return s;
}

double or_log_post(const or_model *m)
{
    double lp = 0.0;
    for (int64_t a = 0; a < m->I * m->K; ++a)
        lp += m->prior_kind == OR_PRIOR_EXPONENTIAL
                  ? -m->lambda_w * m->W[a]
                  : -m->W[a] * m->W[a] / (2.0 * m->sigma_w * m->sigma_w);
    for (int64_t a = 0; a < (int64_t)m->K * m->J; ++a)
        lp += m->prior_kind == OR_PRIOR_EXPONENTIAL
                  ? -m->lambda_h * m->H[a]
                  : -m->H[a] * m->H[a] / (2.0 * m->sigma_h * m->sigma_h);
    return or_log_lik(m) + lp;
}

double or_rmse(const or_model *m, int32_t use_mean)
{
    const double *W = m->W, *H = m->H;
    double *Wm = NULL, *Hm = NULL;
    if (use_mean) {
        Wm = (double *)malloc(sizeof(double) * (size_t)(m->I * m->K));
        Hm = (double *)malloc(sizeof(double) * (size_t)(m->K * m->J));
        or_posterior(m, Wm, NULL, Hm, NULL, NULL);
        W = Wm; H = Hm;
    }
    double s = 0.0;
    for (int64_t n = 0; n < m->N; ++n) {
        double d = m->ent_v[n] - or_mu(m, W, H, m->ent_i[n], m->ent_j[n]);
        s += d * d;
    }
    free(Wm); free(Hm);
    return m->N > 0 ? sqrt(s / (double)m->N) : 0.0;
}
