// psgld_reduce.cu -- FP64 posterior sums and the log-likelihood / RMSE
// reductions.
//
// Posterior (Monte Carlo averages after burn-in, Sec. 4.1.2): after every
// sweep past burn-in each factor element x adds x and x^2 to FP64 running
// sums; mean = sum/n, variance = sum2/n - mean^2.
//
// Log-likelihood (Sec. 4): -(1/phi) sum_obs d_beta(v || mu), beta = 2 - p,
// with the named limits at beta = 2, 1, 0 (Euclidean, Kullback-Leibler,
// Itakura-Saito).  RMSE: sqrt(mean_obs (v - mu)^2).  Both run in FP64 over the
// row-major layout (or the dense V of the tensor-core path); per-CTA partial
// sums are added on the host in CTA order, so the result is deterministic.
#include <algorithm>
#include <cstring>

#include "psgld_internal.cuh"

namespace psgld {
namespace {

__global__ void accumulate_kernel(const float4 *__restrict__ x, int64_t n4, double *__restrict__ s,
                                  double *__restrict__ s2)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n4;
         a += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = x[a];
        double2 *ps = reinterpret_cast<double2 *>(s) + 2 * a;
        double2 *ps2 = reinterpret_cast<double2 *>(s2) + 2 * a;
        double2 p0 = ps[0], p1 = ps[1], q0 = ps2[0], q1 = ps2[1];
        const double a0 = v.x, a1 = v.y, a2 = v.z, a3 = v.w;
        p0.x += a0; p0.y += a1; p1.x += a2; p1.y += a3;
        q0.x += a0 * a0; q0.y += a1 * a1; q1.x += a2 * a2; q1.y += a3 * a3;
        ps[0] = p0; ps[1] = p1; ps2[0] = q0; ps2[1] = q1;
    }
}

// One context's share of a batched accumulation: its current factors, its
// sums, and when to take the sample (Sec. 4.1's averages after burn-in).
struct AccParams {
    const float4 *W, *Ht;        // current factors (I x ldk, J x ldk)
    int64_t nW4, nH4;            // their float4 counts
    double *sW, *sW2, *sH, *sH2;
    int64_t *t_dev;              // iteration at the start of the running sweep
    int64_t t0;                  // *t_dev when the batched call began
    int64_t acc_from;            // first sweep of the call whose sample is taken
    int64_t B;
};

// Every context's factors added to its sums in one launch: context i owns
// float4 units [unit_start[i], unit_start[i + 1]) (W first, then H^T); the
// arithmetic per unit is accumulate_kernel's.
__global__ void accumulate_batch_kernel(const AccParams *__restrict__ Ps, const int64_t *__restrict__ unit_start,
                                        int n)
{
    const int64_t total = __ldg(unit_start + n);
    int ci = -1;
    bool take = false;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < total;
         a += (int64_t)gridDim.x * blockDim.x) {
        if (ci < 0 || __ldg(unit_start + ci + 1) <= a) {
            int lo = ci < 0 ? 0 : ci, hi = n - 1;   // last i with unit_start[i] <= a
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(unit_start + mid) <= a) lo = mid; else hi = mid - 1;
            }
            ci = lo;
            const AccParams &P = Ps[ci];
            take = (*P.t_dev - P.t0) / P.B >= P.acc_from;
        }
        if (!take) continue;
        const AccParams &P = Ps[ci];
        int64_t u = a - __ldg(unit_start + ci);
        const float4 *x = P.W;
        double *s = P.sW, *s2 = P.sW2;
        if (u >= P.nW4) {
            u -= P.nW4;
            x = P.Ht;
            s = P.sH;
            s2 = P.sH2;
        }
        const float4 v = x[u];
        double2 *ps = reinterpret_cast<double2 *>(s) + 2 * u;
        double2 *ps2 = reinterpret_cast<double2 *>(s2) + 2 * u;
        double2 p0 = ps[0], p1 = ps[1], q0 = ps2[0], q1 = ps2[1];
        const double a0 = v.x, a1 = v.y, a2 = v.z, a3 = v.w;
        p0.x += a0; p0.y += a1; p1.x += a2; p1.y += a3;
        q0.x += a0 * a0; q0.y += a1 * a1; q1.x += a2 * a2; q1.y += a3 * a3;
        ps[0] = p0; ps[1] = p1; ps2[0] = q0; ps2[1] = q1;
    }
}

// mode 0: *t_dev = t0 for every context; mode 1: *t_dev += B
__global__ void t_batch_kernel(const AccParams *__restrict__ Ps, int n, int mode)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const AccParams &P = Ps[i];
        if (mode == 0) *P.t_dev = P.t0;
        else *P.t_dev += P.B;
    }
}

__global__ void advance_t_kernel(int64_t *t, int64_t by)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *t += by;
}

__device__ double beta_div(double v, double mu, double p)
{
    const double beta = 2.0 - p;
    if (beta == 2.0) return 0.5 * (v - mu) * (v - mu);
    if (beta == 1.0) return (v > 0.0 ? v * log(v / mu) : 0.0) - v + mu;
    if (beta == 0.0) return v / mu - log(v / mu) - 1.0;
    return pow(v, beta) / (beta * (beta - 1.0)) - v * pow(mu, beta - 1.0) / (beta - 1.0) +
           pow(mu, beta) / beta;
}

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 1216;   // 8 per SM

// mode 0: log-likelihood; mode 1: sum of squared residuals.
// Factors: fp32 (W, Ht) or, when Ws is non-null, fp64 sums scaled by inv_n.
__global__ void __launch_bounds__(kRedThreads)
reduce_kernel(int mode, const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
              const float *__restrict__ val, int64_t nslots, int64_t I, int ldk, int K,
              const float *__restrict__ W, const float *__restrict__ Ht,
              const double *__restrict__ Ws, const double *__restrict__ Hs, double inv_n,
              double p, double phi, double mu_min, double *__restrict__ out)
{
    double acc = 0.0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nslots;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = s % I;
        for (int32_t e = ptr[s]; e < ptr[s + 1]; ++e) {
            const int64_t j = idx[e];
            double mu = 0.0;
            if (Ws) {
                for (int k = 0; k < K; ++k) mu += (Ws[i * ldk + k] * inv_n) * (Hs[j * ldk + k] * inv_n);
            } else {
                for (int k = 0; k < K; ++k) mu += (double)W[i * ldk + k] * (double)Ht[j * ldk + k];
            }
            const double v = val[e];
            if (mode == 0) {
                const double m = (p > 0.0 && mu < mu_min) ? mu_min : mu;
                acc -= beta_div(v, m, p) / phi;
            } else {
                acc += (v - mu) * (v - mu);
            }
        }
    }
    __shared__ double sm[kRedThreads];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sm[0];
}

// The same sums over a dense V (every entry observed), in 64 x 64 tiles of
// entries, the CTAs of the grid taking tiles in turn.  mu of each entry is
// the FP64 dot product over k in order 0 .. K-1 (one multiply-add per k, as
// for a single entry), computed for a tile at once: 16-wide slices of the
// tile's W rows and H^T rows (scaled by inv_n for posterior means) in shared
// memory, each thread 4 x 4 entries 16 rows and 16 columns apart (so a
// warp's shared-memory reads and V loads fall on consecutive addresses).
constexpr int kTileMN = 64, kTileK = 16;
static_assert(kRedThreads == 256, "16 x 16 threads, 4 x 4 entries each, per 64 x 64 tile");

__device__ __forceinline__ double tile_factor(const float *X, const double *Xs, double inv_n, int64_t row,
                                              int64_t n, int k, int K, int ldk)
{
    if (row >= n || k >= K) return 0.0;
    return Xs ? Xs[row * ldk + k] * inv_n : (double)X[row * ldk + k];
}

__global__ void __launch_bounds__(kRedThreads)
reduce_dense_tiled_kernel(int mode, const float *__restrict__ V, int64_t ldv, int64_t I, int64_t J,
                          int ldk, int K, const float *__restrict__ W, const float *__restrict__ Ht,
                          const double *__restrict__ Ws, const double *__restrict__ Hs, double inv_n,
                          double p, double phi, double mu_min, double *__restrict__ out)
{
    __shared__ double sw[kTileK][kTileMN + 1], sh[kTileK][kTileMN + 1];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int64_t ti = (I + kTileMN - 1) / kTileMN, tj = (J + kTileMN - 1) / kTileMN;
    double acc = 0.0;
    for (int64_t t = blockIdx.x; t < ti * tj; t += gridDim.x) {
        const int64_t i0 = (t / tj) * kTileMN, j0 = (t % tj) * kTileMN;
        double mu[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) mu[a][b] = 0.0;
        for (int k0 = 0; k0 < K; k0 += kTileK) {
            __syncthreads();
            // 64 rows x 16 k of each factor: four values per thread and factor
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = tid + q * kRedThreads;          // 0 .. 1023
                const int r = e >> 4, kk = e & 15;
                sw[kk][r] = tile_factor(W, Ws, inv_n, i0 + r, I, k0 + kk, K, ldk);
                sh[kk][r] = tile_factor(Ht, Hs, inv_n, j0 + r, J, k0 + kk, K, ldk);
            }
            __syncthreads();
            const int kn = K - k0 < kTileK ? K - k0 : kTileK;
            for (int kk = 0; kk < kn; ++kk) {
                double wv[4], hv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) wv[a] = sw[kk][ty + 16 * a];
#pragma unroll
                for (int b = 0; b < 4; ++b) hv[b] = sh[kk][tx + 16 * b];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) mu[a][b] = fma(wv[a], hv[b], mu[a][b]);
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t i = i0 + ty + 16 * a;
            if (i >= I) continue;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int64_t j = j0 + tx + 16 * b;
                if (j >= J) continue;
                const double v = V[i * ldv + j];
                const double m = mu[a][b];
                if (mode == 0) {
                    const double mc = (p > 0.0 && m < mu_min) ? mu_min : m;
                    acc -= beta_div(v, mc, p) / phi;
                } else {
                    acc += (v - m) * (v - m);
                }
            }
        }
    }
    __shared__ double red[kRedThreads];
    red[tid] = acc;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    if (tid == 0) out[blockIdx.x] = red[0];
}

}  // namespace

int reduce_blocks() { return kRedBlocks; }

psgld_status launch_accumulate(psgld_ctx *c, cudaStream_t st)
{
    const int64_t nW4 = c->I * c->ldk / 4, nH4 = c->J * c->ldk / 4;
    accumulate_kernel<<<(unsigned)std::min<int64_t>((nW4 + 255) / 256, 152 * 16), 256, 0, st>>>(
        reinterpret_cast<const float4 *>(c->W[c->wcur]), nW4, c->sW.s, c->sW.s2);
    accumulate_kernel<<<(unsigned)std::min<int64_t>((nH4 + 255) / 256, 152 * 16), 256, 0, st>>>(
        reinterpret_cast<const float4 *>(c->Ht[c->hcur]), nH4, c->sH.s, c->sH.s2);
    PSGLD_CK(c, cudaGetLastError());
    return PSGLD_OK;
}

size_t acc_param_bytes() { return sizeof(AccParams); }

int64_t fill_acc_param(psgld_ctx *c, int64_t t0, int64_t acc_from, void *dst)
{
    AccParams P;
    P.W = reinterpret_cast<const float4 *>(c->W[c->wcur]);
    P.Ht = reinterpret_cast<const float4 *>(c->Ht[c->hcur]);
    P.nW4 = c->I * c->ldk / 4;
    P.nH4 = c->J * c->ldk / 4;
    P.sW = c->sW.s;
    P.sW2 = c->sW.s2;
    P.sH = c->sH.s;
    P.sH2 = c->sH.s2;
    P.t_dev = c->t_dev;
    P.t0 = t0;
    P.acc_from = acc_from;
    P.B = c->B;
    std::memcpy(dst, &P, sizeof P);
    return P.nW4 + P.nH4;
}

psgld_status launch_accumulate_batch(psgld_ctx *c0, const void *params, const int64_t *unit_start, int n,
                                     int64_t total_units, cudaStream_t st)
{
    const unsigned grid = (unsigned)std::min<int64_t>((total_units + 255) / 256, 152 * 16);
    if (grid > 0)
        accumulate_batch_kernel<<<grid, 256, 0, st>>>(static_cast<const AccParams *>(params), unit_start, n);
    PSGLD_CK(c0, cudaGetLastError());
    return PSGLD_OK;
}

psgld_status launch_t_batch(psgld_ctx *c0, const void *params, int n, int mode, cudaStream_t st)
{
    t_batch_kernel<<<(n + 255) / 256, 256, 0, st>>>(static_cast<const AccParams *>(params), n, mode);
    PSGLD_CK(c0, cudaGetLastError());
    return PSGLD_OK;
}

psgld_status launch_advance_t(psgld_ctx *c, int64_t by, cudaStream_t st)
{
    advance_t_kernel<<<1, 32, 0, st>>>(c->t_dev, by);
    PSGLD_CK(c, cudaGetLastError());
    return PSGLD_OK;
}

psgld_status reduce_loglik_rmse(psgld_ctx *c, int mode, int use_mean, cudaStream_t st, double *out)
{
    const SideLayout &L = c->side[0];
    const double inv_n = c->n_samples > 0 ? 1.0 / (double)c->n_samples : 0.0;
    if (c->dense)
        reduce_dense_tiled_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(
            mode, c->Vd, c->ldv, c->I, c->J, c->ldk, c->K, c->W[c->wcur], c->Ht[c->hcur],
            use_mean ? c->sW.s : nullptr, use_mean ? c->sH.s : nullptr, inv_n, c->p, c->phi,
            c->opt.mu_min, c->red);
    else
        reduce_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(
            mode, L.ptr, L.idx, L.val, (int64_t)c->B * c->I, c->I, c->ldk, c->K, c->W[c->wcur],
            c->Ht[c->hcur], use_mean ? c->sW.s : nullptr, use_mean ? c->sH.s : nullptr, inv_n,
            c->p, c->phi, c->opt.mu_min, c->red);
    PSGLD_CK(c, cudaGetLastError());
    PSGLD_CK(c, cudaMemcpyAsync(c->red_host.data(), c->red, sizeof(double) * kRedBlocks,
                                cudaMemcpyDeviceToHost, st));
    PSGLD_CK(c, cudaStreamSynchronize(st));
    {
        psgld_status fs = check_kernel_flag(c);
        if (fs != PSGLD_OK) return fs;
    }
    double s = 0.0;
    for (int b = 0; b < kRedBlocks; ++b) s += c->red_host[b];
    *out = s;
    return PSGLD_OK;
}

}  // namespace psgld
