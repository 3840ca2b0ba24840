// psgld_step.cu -- one PSGLD iteration (Algorithm 1's loop body) as a single
// fused kernel launch.
//
// For part Pi_t every block (r, c) updates the W rows of row piece r and the
// H columns of column piece c from (W^(t-1), H^(t-1))  (Eq. psgld_w and
// Eq. psgld_h).  Because the B blocks of a part cover every row piece and
// every column piece exactly once, one iteration updates every row of W and
// every column of H:
//
//   w_i <- w_i + eps (S sum_{j in row i of Pi_t} e_ij h_j + dlog p(w_i)) + sqrt(2 eps) z
//   h_j <- h_j + eps (S sum_{i in col j of Pi_t} e_ij w_i + dlog p(h_j)) + sqrt(2 eps) z
//   e_ij = (v_ij - mu_ij) max(mu_ij, mu_min)^(-p) / phi,  mu_ij = w_i . h_j
//
// followed by |.| for non-negative models (Sec. 3.2).  This is the Tweedie
// gradient of Sec. 4 (d/dmu of -d_beta(v||mu)/phi with beta = 2 - p).
//
// Design.  Both updates read only the previous factors, so they are
// independent: the W side (rows of the part's CSR) and the H side (columns
// of the part's CSC) run as two halves of one grid.  Factors are ping-pong
// buffers (read X_cur, write X_next), so no block reads a row another block
// is writing and no atomics touch the factors.  A team of T lanes (T = the
// power of two covering ceil(K/4) float4 groups) owns one work record: it
// loads its own row once, streams the record's entries (index and value
// loaded coalesced, one per lane, then broadcast by shuffle), gathers the
// other factor's rows with read-only float4 loads, reduces mu across the
// team by butterfly shuffles, and accumulates the gradient in registers.
// SDDMM (mu), the Tweedie epilogue (e) and the SpMM (sum e h) are therefore
// one pass with e never leaving registers.  Rows with more than seg_len
// entries in the part are split over several records; their partial
// gradients go to a small scratch area and the last record to arrive (an
// arrival counter) sums them in record order, so results are deterministic.
// The same team then draws its Philox normals and writes the updated row.
#include <algorithm>

#include "psgld_internal.cuh"

namespace psgld {
namespace {

struct Side {
    const float *X_cur;   // own rows (n_rows x ldk)
    float *X_next;
    const float *Y_cur;   // gathered rows of the other factor
    const int32_t *idx;   // other index of each entry
    const float *val;
    const int4 *seg;      // this part's records
    const int4 *split;    // this part's split table
    float *partial;
    unsigned *counter;
    int64_t nseg;
    float prior_a, prior_b;   // d log p(x)/dx = prior_a + prior_b * x
    uint32_t mat;             // 0 = W, 1 = H (noise stream)
    int nblocks;              // CTAs of this side
};

struct StepParams {
    Side side[2];
    const int64_t *t_dev;     // if non-null, t = *t_dev + t_add
    int64_t t_add;
    int K, ldk, ngroups;
    float eps, sd, S, phi_inv, p, mu_min;
    int eps_poly;             // 1: eps_t = (a/t)^b computed on the device
    double eps_a, eps_b;
    int p_mode;               // 0: p = 0, 1: p = 1, 2: p = 2, 3: other
    int mirror;
    uint32_t key0, key1;
};

constexpr int kThreads = 256;

template <int T>
__device__ __forceinline__ unsigned team_mask()
{
    if constexpr (T == 32) {
        return 0xffffffffu;
    } else {
        return ((1u << T) - 1u) << ((threadIdx.x & 31) & ~(T - 1));
    }
}

template <int T>
__device__ __forceinline__ float team_sum(float v, unsigned mask)
{
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, T);
    return v;
}

__device__ __forceinline__ float4 ldg4(const float *p)
{
    return __ldg(reinterpret_cast<const float4 *>(p));
}

__device__ __forceinline__ float dot4(const float4 a, const float4 b, float acc)
{
    acc = fmaf(a.x, b.x, acc);
    acc = fmaf(a.y, b.y, acc);
    acc = fmaf(a.z, b.z, acc);
    acc = fmaf(a.w, b.w, acc);
    return acc;
}

__device__ __forceinline__ void axpy4(float4 &acc, float e, const float4 y)
{
    acc.x = fmaf(e, y.x, acc.x);
    acc.y = fmaf(e, y.y, acc.y);
    acc.z = fmaf(e, y.z, acc.z);
    acc.w = fmaf(e, y.w, acc.w);
}

// Tweedie factor: e = (v - mu) * max(mu, mu_min)^(-p) / phi
__device__ __forceinline__ float tweedie_e(const StepParams &P, float v, float mu)
{
    const float d = v - mu;
    if (P.p_mode == 0) return d * P.phi_inv;
    const float mc = fmaxf(mu, P.mu_min);
    if (P.p_mode == 1) return d / mc * P.phi_inv;
    if (P.p_mode == 2) return d / (mc * mc) * P.phi_inv;
    return d * exp2f(-P.p * log2f(mc)) * P.phi_inv;
}

__device__ __forceinline__ float update1(const StepParams &P, const Side &Sd, float x, float g,
                                         float z, float eps, float sd)
{
    const float drift = fmaf(P.S, g, fmaf(Sd.prior_b, x, Sd.prior_a));
    const float y = fmaf(sd, z, fmaf(eps, drift, x));
    return P.mirror ? fabsf(y) : y;
}

template <int T, int G, int U>
__global__ void __launch_bounds__(kThreads) part_step_kernel(const __grid_constant__ StepParams P)
{
    const int sid = (int)blockIdx.x < P.side[0].nblocks ? 0 : 1;
    const Side &Sd = P.side[sid];
    const int cta = sid == 0 ? (int)blockIdx.x : (int)blockIdx.x - P.side[0].nblocks;
    constexpr int kTeams = kThreads / T;
    const int lane = threadIdx.x & (T - 1);
    const int64_t rec = (int64_t)cta * kTeams + threadIdx.x / T;
    if (rec >= Sd.nseg) return;   // team-uniform exit
    const unsigned mask = team_mask<T>();
    const int ldk = P.ldk, ng = P.ngroups;

    const int4 sg = Sd.seg[rec];  // row, beg, end, split
    const int64_t row = sg.x;

    float4 x[G], acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int q = lane + g * T;
        x[g] = q < ng ? ldg4(Sd.X_cur + row * ldk + 4 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
        acc[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    for (int base = sg.y; base < sg.z; base += T) {
        const int n = min(T, sg.z - base);
        int my_j = 0;
        float my_v = 0.f;
        if (lane < n) {
            my_j = __ldg(Sd.idx + base + lane);
            my_v = __ldg(Sd.val + base + lane);
        }
        for (int u = 0; u < n; u += U) {
            float4 y[U][G];
            float vv[U];
#pragma unroll
            for (int uu = 0; uu < U; ++uu) {
                const int src = u + uu;
                const int jj = __shfl_sync(mask, my_j, src, T);
                vv[uu] = __shfl_sync(mask, my_v, src, T);
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int q = lane + g * T;
                    y[uu][g] = (q < ng && src < n) ? ldg4(Sd.Y_cur + (int64_t)jj * ldk + 4 * q)
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int uu = 0; uu < U; ++uu) {
                if (u + uu < n) {   // team-uniform
                    float d = 0.f;
#pragma unroll
                    for (int g = 0; g < G; ++g) d = dot4(x[g], y[uu][g], d);
                    const float mu = team_sum<T>(d, mask);
                    const float e = tweedie_e(P, vv[uu], mu);
#pragma unroll
                    for (int g = 0; g < G; ++g) axpy4(acc[g], e, y[uu][g]);
                }
            }
        }
    }

    if (sg.w >= 0) {
        // Row split over several records: publish the partial gradient; the
        // last record to arrive adds all partials in record order.
        const int4 sp = Sd.split[sg.w];   // first record, count, first slot
        const int64_t slot = sp.z + (rec - sp.x);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int q = lane + g * T;
            if (q < ng) __stcg(reinterpret_cast<float4 *>(Sd.partial + slot * ldk + 4 * q), acc[g]);
        }
        __threadfence();
        __syncwarp(mask);
        unsigned last = 0;
        if (lane == 0) last = atomicAdd(Sd.counter + sg.w, 1u) == (unsigned)(sp.y - 1);
        last = __shfl_sync(mask, last, 0, T);
        if (!last) return;
        __threadfence();
#pragma unroll
        for (int g = 0; g < G; ++g) acc[g] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int o = 0; o < sp.y; ++o) {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int q = lane + g * T;
                if (q < ng) {
                    const float4 a = __ldcg(reinterpret_cast<const float4 *>(
                        Sd.partial + (int64_t)(sp.z + o) * ldk + 4 * q));
                    acc[g].x += a.x; acc[g].y += a.y; acc[g].z += a.z; acc[g].w += a.w;
                }
            }
        }
        if (lane == 0) Sd.counter[sg.w] = 0u;   // ready for the next launch
    }

    // step size and noise scale
    const int64_t t = P.t_dev ? *P.t_dev + P.t_add : P.t_add;
    float eps = P.eps, sd = P.sd;
    if (P.eps_poly) {
        const double e = pow(P.eps_a / (double)t, P.eps_b);
        eps = (float)e;
        sd = (float)sqrt(2.0 * e);
    }
    const uint32_t t_lo = (uint32_t)(uint64_t)t, t_hi = (uint32_t)((uint64_t)t >> 32);
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int q = lane + g * T;
        if (q < ng) {
            const uint4 r = dev::philox4x32_10(
                make_uint4((uint32_t)q, (uint32_t)row, t_lo, (t_hi << 1) | Sd.mat),
                make_uint2(P.key0, P.key1));
            const float4 z = dev::box_muller4(r);
            const int k0 = 4 * q;
            float4 o;
            o.x = update1(P, Sd, x[g].x, acc[g].x, z.x, eps, sd);
            o.y = k0 + 1 < P.K ? update1(P, Sd, x[g].y, acc[g].y, z.y, eps, sd) : 0.f;
            o.z = k0 + 2 < P.K ? update1(P, Sd, x[g].z, acc[g].z, z.z, eps, sd) : 0.f;
            o.w = k0 + 3 < P.K ? update1(P, Sd, x[g].w, acc[g].w, z.w, eps, sd) : 0.f;
            *reinterpret_cast<float4 *>(Sd.X_next + row * ldk + k0) = o;
        }
    }
}

using KernelFn = void (*)(StepParams);

KernelFn pick_kernel(int T, int G)
{
    if (G == 1) {
        switch (T) {
        case 1: return part_step_kernel<1, 1, 4>;
        case 2: return part_step_kernel<2, 1, 4>;
        case 4: return part_step_kernel<4, 1, 4>;
        case 8: return part_step_kernel<8, 1, 4>;
        case 16: return part_step_kernel<16, 1, 4>;
        case 32: return part_step_kernel<32, 1, 4>;
        }
    }
    if (T == 32) {
        switch (G) {
        case 2: return part_step_kernel<32, 2, 4>;
        case 3: return part_step_kernel<32, 3, 2>;
        case 4: return part_step_kernel<32, 4, 2>;
        }
    }
    return nullptr;
}

}  // namespace

void team_shape(int ngroups, int *T, int *G)
{
    int t = 1;
    while (t < ngroups && t < 32) t <<= 1;
    *T = t;
    *G = (ngroups + t - 1) / t;
}

psgld_status launch_part_step(psgld_ctx *c, int64_t t, const int64_t *t_dev, int64_t t_add,
                              cudaStream_t st)
{
    const int B = c->B;
    const int part = (int)((t - 1) % B);
    int T, G;
    team_shape(c->ngroups, &T, &G);
    KernelFn fn = pick_kernel(T, G);
    if (!fn) return fail(c, PSGLD_ERR_ARG, "unsupported K");

    StepParams P{};
    const int teams_per_cta = kThreads / T;
    const bool upd[2] = {!c->opt.freeze_W, !c->opt.freeze_H};
    for (int s = 0; s < 2; ++s) {
        SideLayout &L = c->side[s];
        Side &Sd = P.side[s];
        Sd.X_cur = s == 0 ? c->W[c->wcur] : c->Ht[c->hcur];
        Sd.X_next = s == 0 ? c->W[c->wcur ^ 1] : c->Ht[c->hcur ^ 1];
        Sd.Y_cur = s == 0 ? c->Ht[c->hcur] : c->W[c->wcur];
        Sd.idx = L.idx;
        Sd.val = L.val;
        Sd.seg = L.seg + L.seg_off[part];
        Sd.split = L.split + L.split_off[part];
        Sd.partial = L.partial;
        Sd.counter = L.counter;
        Sd.nseg = upd[s] ? L.seg_off[part + 1] - L.seg_off[part] : 0;
        if (c->prior.kind == PSGLD_PRIOR_EXPONENTIAL) {
            Sd.prior_a = (float)-(s == 0 ? c->prior.lambda_w : c->prior.lambda_h);
            Sd.prior_b = 0.f;
        } else {
            const double sg = s == 0 ? c->prior.sigma_w : c->prior.sigma_h;
            Sd.prior_a = 0.f;
            Sd.prior_b = (float)(-1.0 / (sg * sg));
        }
        Sd.mat = (uint32_t)s;
        Sd.nblocks = (int)((Sd.nseg + teams_per_cta - 1) / teams_per_cta);
    }
    P.t_dev = t_dev;
    P.t_add = t_dev ? t_add : t;
    P.K = c->K;
    P.ldk = c->ldk;
    P.ngroups = c->ngroups;
    const double eps = c->opt.eps;
    P.eps = (float)eps;
    P.sd = (float)std::sqrt(2.0 * eps);
    P.eps_poly = c->opt.eps_mode == PSGLD_EPS_POLY;
    P.eps_a = c->opt.eps_a;
    P.eps_b = c->opt.eps_b;
    const int64_t np = c->part_n[part];
    P.S = c->opt.scale_mode == PSGLD_SCALE_B ? (float)B : (np > 0 ? (float)((double)c->N / (double)np) : 0.f);
    P.phi_inv = (float)(1.0 / c->phi);
    P.p = (float)c->p;
    P.mu_min = (float)c->opt.mu_min;
    P.p_mode = c->p == 0.0 ? 0 : c->p == 1.0 ? 1 : c->p == 2.0 ? 2 : 3;
    P.mirror = c->prior.kind == PSGLD_PRIOR_EXPONENTIAL;
    P.key0 = (uint32_t)c->opt.seed;
    P.key1 = (uint32_t)(c->opt.seed >> 32);

    const int grid = P.side[0].nblocks + P.side[1].nblocks;
    if (grid > 0) fn<<<grid, kThreads, 0, st>>>(P);
    PSGLD_CK(c, cudaGetLastError());
    if (upd[0]) c->wcur ^= 1;
    if (upd[1]) c->hcur ^= 1;
    return PSGLD_OK;
}

}  // namespace psgld
