// psgld_step.cu -- one PSGLD iteration (Algorithm 1's loop body) as two
// kernel launches: the likelihood gradient, then the Langevin update.
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
// Kernel 1, gradient.  Both sums read only the previous factors, so the W
// side (the part's entries in row order) and the H side (in column order)
// run in one grid and write G = sum e h (resp. sum e w) for every row.  The
// entries are cut into units of E consecutive entries, one warp per unit:
// the unit's other-factor rows are gathered into shared memory by bulk
// copies, mu and the Tweedie factor are formed one lane per entry, and the
// gradient is summed by row segments of the unit -- SDDMM, epilogue and SpMM
// in one pass, e never leaves the SM.  A row whose entries span several
// units publishes the sums of its first and last pieces to per-unit head and
// tail slots, which the update kernel adds in unit order, so the result does
// not depend on scheduling (details at the kernel).

// On dense data kept for the tensor cores (dense_path), kernel 1 is the block
// GEMM -> epilogue -> GEMM chain of psgld_dense.cu instead; kernel 2 is the
// same.
//
// Kernel 2, update.  A flat, fully coalesced sweep over every (row, float4
// group) item of both factors: the row's gradient (G, nothing for an empty
// row, or the sum of a split row's partials), Philox4x32-10 normals (counter
// = group, row, t, matrix), prior gradient, step, mirror; reads X_cur, writes
// X_next (ping-pong buffers, so no row is read and written by the same
// launch).  Philox's integer multiplies and Box-Muller make this ALU-bound,
// so it runs at full lane occupancy rather than inside the gather-bound
// kernel 1.
#include <algorithm>
#include <cstring>
#include <vector>
#include <cmath>

#include "psgld_internal.cuh"

namespace psgld {
namespace {

constexpr int kThreads = 256;        // update kernel
constexpr int kGradThreads = 128;    // gradient kernel: four warps, one unit each

struct GradSide {
    const float *X_cur;    // own rows (n_rows x ldk)
    const float *Y_cur;    // gathered rows of the other factor
    float *Gout;           // this side's rows of G
    const int32_t *own;    // own row of each entry
    const int32_t *idx;    // other index of each entry
    const float *val;
    float *partial;        // 2 x units x ldk: head / tail partial sums
    int64_t base;          // first entry of the part
    int64_t n;             // entries of the part
    int64_t units;         // ceil(n / E)
    const uint16_t *Y16;   // BF16 copy of the other factor (rows of ld16), gathered instead of Y_cur
    int prefetch_own;      // 1: own rows go to L2 with the gathers (own factor beyond L2)
};

struct GradParams {
    GradSide side[2];
    int ldk, lds, ngroups;    // row length, shared-memory row stride (floats), float4 groups
    int ld16, lds16;          // BF16 gather: row length and shared-memory row stride (elements)
    float phi_inv, p, mu_min;
    int p_mode;               // 0: p = 0, 1: p = 1, 2: p = 2, 3: other
    int *err;                 // set to 16 when a bulk copy wait runs out
    uint32_t wait_polls;      // > 0: the first wait's poll limit (no suspension), for tests
};

struct UpdSide {
    const float *X_cur;
    float *X_next;
    const float *Gin;
    const int32_t *ptr;       // this part's row offsets (absolute entry indices)
    const float *partial;     // head / tail partial sums of the gradient kernel
    int64_t base;             // first entry of the part
    int64_t items;            // n_rows * ngroups (0 when the factor is frozen)
    int64_t gstride;          // dense path: distance between partial gradient arrays
    int gparts;               // dense path: partial gradient arrays to add (0: sparse path)
    uint16_t *sh;             // two-sided dense kernel: BF16 shadow of X_next (else null)
    int64_t n_rows;           // I or J
    int sh_tiles;             // 64-row shadow tiles per piece
    uint16_t *g16;            // BF16 copy of X_next for the gradient kernel's gathers (else null)
    float prior_a, prior_b;   // d log p(x)/dx = prior_a + prior_b * x
    uint32_t mat;             // 0 = W, 1 = H (noise stream)
};

struct UpdParams {
    UpdSide side[2];
    const int64_t *t_dev;     // if non-null, t = *t_dev + t_add
    int64_t t_add;
    int K, ldk, ngroups, unit_shift;
    uint32_t div_magic;       // ceil(2^32 / ngroups) when item * ngroups < 2^32, else 0
    float eps, sd, S;
    int eps_poly;             // 1: eps_t = (a/t)^b computed on the device
    double eps_a, eps_b;
    int mirror;
    int B, sh_kp;             // pieces; shadow tile width (two-sided dense kernel)
    int ld16;                 // row length of the BF16 gather copies
    uint32_t rk0[10], rk1[10];   // Philox round keys (seed + r * Weyl constants)
};

template <int S>
__device__ __forceinline__ unsigned sub_mask()
{
    if constexpr (S == 32) {
        return 0xffffffffu;
    } else {
        return ((1u << S) - 1u) << ((threadIdx.x & 31) & ~(S - 1));
    }
}

template <int S>
__device__ __forceinline__ float sub_sum(float v, unsigned mask)
{
#pragma unroll
    for (int o = S / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, S);
    return v;
}

__device__ __forceinline__ float4 ldg4(const float *p)
{
    return __ldg(reinterpret_cast<const float4 *>(p));
}

__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }

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

__device__ __forceinline__ void add4(float4 &a, const float4 b)
{
    a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
}

// Tweedie factor: e = (v - mu) * max(mu, mu_min)^(-p) / phi
__device__ __forceinline__ float tweedie_e(const GradParams &P, float v, float mu)
{
    const float d = v - mu;
    if (P.p_mode == 0) return d * P.phi_inv;
    const float mc = fmaxf(mu, P.mu_min);
    if (P.p_mode == 1) return d / mc * P.phi_inv;
    if (P.p_mode == 2) return d / (mc * mc) * P.phi_inv;
    return d * exp2f(-P.p * log2f(mc)) * P.phi_inv;
}

// ---- kernel 1: the likelihood gradient ------------------------------------
//
// A unit is E consecutive entries of the part in this side's order (rows in
// order, the other index ascending), one unit per warp at a time.  Steps:
//   1. lane l holds entry l of the unit: own row, other index j, value v
//      (loaded while the warp worked on its previous unit);
//   2. TMA bulk copies (cp.async.bulk, one instruction per factor row) bring
//      the E gathered rows Y[j] into the warp's shared memory, completing on
//      the warp's mbarrier, so every gather of the unit is in flight at once;
//      meanwhile each row segment's own row X[own] is prefetched into L2
//      (when that factor exceeds L2) and each lane starts loading its own
//      row's first float4 groups;
//   3. SDDMM + epilogue, one lane per entry: mu = X[own] . Y[j], e = Tweedie
//      factor (X rows read through L1; lanes of one row share the lines);
//   4. SpMM by row segments of the unit (their starts tabulated in shared
//      memory), sub-teams of S lanes over the K columns: G[row] = sum_l e_l
//      Y[j_l] over the segment.  A unit holding one row splits its entries
//      over the sub-teams and adds their sums; a unit holding several rows
//      gives each sub-team whole segments;
//   5. a segment whose row also has entries before the unit goes to the
//      unit's head slot, one whose row continues after it to the tail slot,
//      any other straight to G.  The update kernel adds a row's tail and head
//      slots in unit order, so the result does not depend on scheduling.

constexpr uint32_t kWaitLimit = 1u << 24;          // mbarrier polls before giving up
constexpr long long kWaitCycles = 1ll << 31;         // ... or about one second of SM clock
constexpr uint32_t kWaitHintNs = 2000;               // suspension per poll

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Waits (suspended, up to about `hint_ns`) for phase `parity` of the barrier
// to complete; true once it has.  The suspension keeps waiting warps from
// taking issue slots while the copies are in flight.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns) : "memory");
    return ok != 0;
}

// One poll of phase `parity` of the barrier, without suspending.
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

// Bulk prefetch of `bytes` (a multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(src), "r"(bytes) : "memory");
}

// Four gathered entries (q-th float4 group) of row `row` of the warp's
// gathered rows: FP32 rows of lds floats, or (BF) BF16 rows of lds16.
template <bool BF>
__device__ __forceinline__ float4 ys4(const float *ys, int row, int q, int lds, int lds16)
{
    if constexpr (BF) {
        const uint2 v = *reinterpret_cast<const uint2 *>(reinterpret_cast<const uint16_t *>(ys) +
                                                         (size_t)row * lds16 + 4 * q);
        return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xFFFF0000u),
                           __uint_as_float(v.y << 16), __uint_as_float(v.y & 0xFFFF0000u));
    } else {
        return *reinterpret_cast<const float4 *>(ys + (size_t)row * lds + 4 * q);
    }
}

// A unit's entries as each lane loads them, one unit ahead of its work:
// lane l entry l (own row, other index, value); `edge` is, on lane 0, the
// own row of the entry just before the unit and, on lane 1, of the entry
// just after it (-1: none).
struct UnitIn {
    int own, jj;
    float vv;
    int edge;
};

template <int SID, int E>
__device__ __forceinline__ UnitIn load_unit(const GradParams &P, int64_t u)
{
    const GradSide &Sd = P.side[SID];
    const int lane32 = threadIdx.x & 31;
    const int64_t e0 = Sd.base + u * E, rem = Sd.n - u * E;
    UnitIn r{-1, 0, 0.f, -1};
    if (lane32 < E && lane32 < rem) {
        r.own = __ldg(Sd.own + e0 + lane32);
        r.jj = __ldg(Sd.idx + e0 + lane32);
        r.vv = __ldg(Sd.val + e0 + lane32);
    }
    if (lane32 == 0 && u > 0) r.edge = __ldg(Sd.own + e0 - 1);
    if (lane32 == 1 && rem > E) r.edge = __ldg(Sd.own + e0 + E);
    return r;
}

// One unit (E consecutive entries of side SID's part order) on one warp; SID
// is a template parameter so that the side's fields are fixed parameter
// offsets.  BF: the gathered rows are the BF16 copies (half the bytes;
// products and sums stay FP32).  `bar` completes once per unit, phase
// `parity`.  False when the gathers did not land in time (the warp stops).
template <int SID, int S, int NG, int E, bool BF>
__device__ __forceinline__ bool grad_unit(const GradParams &P, int64_t u, const UnitIn &in, float *ys,
                                          float *es, int *ow, int *sg, uint64_t *bar, uint32_t parity)
{
    constexpr int R = 32 / S;      // sub-teams per warp
    constexpr int NGP = S * NG;    // float4 groups a sub-team covers (>= ngroups)
    const int lane32 = threadIdx.x & 31;
    const int ng = P.ngroups, ldk = P.ldk, lds = P.lds;
    const GradSide &Sd = P.side[SID];
    const int n = (int)(Sd.n - u * E < E ? Sd.n - u * E : E);

    // ---- 1. this lane's entry (loaded with the previous unit)
    const bool valid = lane32 < n;
    const int own = in.own, jj = in.jj;
    const float vv = in.vv;
    const int prev_own = __shfl_sync(0xffffffffu, in.edge, 0);   // rows of the entries just outside the unit
    const int next_own = __shfl_sync(0xffffffffu, in.edge, 1);
    const int lds16 = P.lds16;
    const uint32_t row_bytes = BF ? (uint32_t)P.ld16 * 2u : (uint32_t)ldk * 4u;

    // ---- 2. bulk gathers into shared memory, once every lane is done with
    // the previous unit's (its reads ordered before the copies' writes)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane32 == 0) mbar_expect_tx(bar, (uint32_t)n * row_bytes);
    __syncwarp();
    bool done = false;
    if (P.wait_polls) {
        // a test limit: at most wait_polls polls, without suspending, made
        // before the copies are issued -- so the wait surely runs out
        for (uint32_t it = 0; it < P.wait_polls && !done; ++it) done = mbar_test_wait(bar, parity);
    }
    if (valid) {
        if constexpr (BF)
            bulk_g2s(reinterpret_cast<uint16_t *>(ys) + (size_t)lane32 * lds16, Sd.Y16 + (int64_t)jj * P.ld16,
                     row_bytes, bar);
        else
            bulk_g2s(ys + (size_t)lane32 * lds, Sd.Y_cur + (int64_t)jj * ldk, row_bytes, bar);
    }
    // each row segment's own row on its way to L2 while the gathers land
    const int own_prev_lane = __shfl_up_sync(0xffffffffu, own, 1);
    const bool seg_start = valid && (lane32 == 0 || own != own_prev_lane);
    if (seg_start && Sd.prefetch_own) prefetch_l2(Sd.X_cur + (int64_t)own * ldk, (uint32_t)ldk * 4u);
    // the first XP float4 groups of this lane's own row, loaded before the
    // wait (the rest after it, in the mu loop)
    constexpr int XP = NGP < 8 ? NGP : 8;
    float4 xp[XP];
    const float *xrow = Sd.X_cur + (int64_t)(valid ? own : 0) * ldk;
#pragma unroll
    for (int w = 0; w < XP; ++w) xp[w] = (valid && w < ng) ? ldg4(xrow + 4 * w) : zero4();
    const long long t_start = clock64();
    if (!P.wait_polls) {
        for (uint32_t it = 0; it < kWaitLimit && !done && clock64() - t_start < kWaitCycles; ++it)
            done = mbar_try_wait(bar, parity, kWaitHintNs);
    }
    if (!__all_sync(0xffffffffu, done)) {
        // The copies did not land: report it, wait (bounded again) for them
        // so that no copy targets freed shared memory, and give up.
        if (lane32 == 0) atomicOr(P.err, 16);
        const long long t_again = clock64();
        for (uint32_t it = 0; it < kWaitLimit && !done && clock64() - t_again < kWaitCycles; ++it)
            done = mbar_try_wait(bar, parity, kWaitHintNs);
        return false;
    }

    // ---- 3. mu and the Tweedie factor, one lane per entry
    float e = 0.f;
    if (valid) {
        const float *x = Sd.X_cur + (int64_t)own * ldk;
        float d = 0.f;
#pragma unroll
        for (int q = 0; q < NGP; ++q)
            if (q < ng) d = dot4(q < XP ? xp[q < XP ? q : 0] : ldg4(x + 4 * q), ys4<BF>(ys, lane32, q, lds, lds16), d);
        e = tweedie_e(P, vv, d);
    }
    const unsigned smask = __ballot_sync(0xffffffffu, seg_start);
    if (lane32 < E) {
        es[lane32] = e;
        ow[lane32] = own;
    }
    // sg[k]: the unit's entry that starts row segment k; sg[nseg] = n
    if (seg_start) sg[__popc(smask & ((1u << lane32) - 1u))] = lane32;
    if (lane32 == 0) sg[__popc(smask)] = n;
    __syncwarp();

    // ---- 4./5. gradient sums per row segment
    const int sub = lane32 / S, lane = lane32 & (S - 1);
    const int nseg = __popc(smask);
    float4 acc[NG];
    if (nseg == 1) {
        // one row: sub-team s takes entries s, s+R, ...; then add the sub-teams
#pragma unroll
        for (int g = 0; g < NG; ++g) acc[g] = zero4();
#pragma unroll 4
        for (int sl = sub; sl < n; sl += R) {
            const float es_ = es[sl];
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                const int q = lane + g * S;
                if (q < ng) axpy4(acc[g], es_, ys4<BF>(ys, sl, q, lds, lds16));
            }
        }
#pragma unroll
        for (int o = S; o < 32; o <<= 1)
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                acc[g].x += __shfl_xor_sync(0xffffffffu, acc[g].x, o);
                acc[g].y += __shfl_xor_sync(0xffffffffu, acc[g].y, o);
                acc[g].z += __shfl_xor_sync(0xffffffffu, acc[g].z, o);
                acc[g].w += __shfl_xor_sync(0xffffffffu, acc[g].w, o);
            }
        const int row = ow[0];
        float *dst = prev_own == row ? Sd.partial + (2 * u) * (int64_t)ldk
                   : next_own == row ? Sd.partial + (2 * u + 1) * (int64_t)ldk
                                     : Sd.Gout + (int64_t)row * ldk;
        if (sub == 0) {
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                const int q = lane + g * S;
                if (q < ng) *reinterpret_cast<float4 *>(dst + 4 * q) = acc[g];
            }
        }
    } else {
        // several rows: sub-team s takes segments s, s+R, ...
        for (int k = sub; k < nseg; k += R) {
            const int st = sg[k], en = sg[k + 1];
            const int row = ow[st];
#pragma unroll
            for (int g = 0; g < NG; ++g) acc[g] = zero4();
#pragma unroll 4
            for (int sl = st; sl < en; ++sl) {
                const float es_ = es[sl];
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    const int q = lane + g * S;
                    if (q < ng) axpy4(acc[g], es_, ys4<BF>(ys, sl, q, lds, lds16));
                }
            }
            float *dst = (k == 0 && prev_own == row) ? Sd.partial + (2 * u) * (int64_t)ldk
                       : (k == nseg - 1 && next_own == row) ? Sd.partial + (2 * u + 1) * (int64_t)ldk
                                                             : Sd.Gout + (int64_t)row * ldk;
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                const int q = lane + g * S;
                if (q < ng) *reinterpret_cast<float4 *>(dst + 4 * q) = acc[g];
            }
        }
    }
    return true;
}

// Each warp takes units u, u + T, u + 2T, ... (T = warps of the grid: a
// grid of one CTA per 4 units gives every warp one unit; a smaller grid
// keeps warps resident over several), loading the next unit's entries
// before working on the current one.
template <int S, int NG, int E, bool BF>
__global__ void __launch_bounds__(kGradThreads) grad_kernel(const __grid_constant__ GradParams P)
{
    extern __shared__ float4 smem4[];
    const int warp = threadIdx.x >> 5;
    const int lds = P.lds;
    constexpr int kWarpsPerCta = kGradThreads / 32;
    float *base = reinterpret_cast<float *>(smem4);
    float *ys = base + (size_t)warp * E * lds;                      // E gathered rows
    float *es = base + (size_t)kWarpsPerCta * E * lds + warp * E;   // e of each entry
    int *ow = reinterpret_cast<int *>(base + (size_t)kWarpsPerCta * E * lds + kWarpsPerCta * E) + warp * E;
    int *sg = reinterpret_cast<int *>(base + (size_t)kWarpsPerCta * (E * lds + 2 * E)) + warp * (E + 1);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + (size_t)kWarpsPerCta * (E * lds + 3 * E + 1)) + warp;

    const int64_t U0 = P.side[0].units, U = U0 + P.side[1].units;
    const int64_t T = (int64_t)gridDim.x * kWarpsPerCta;
    int64_t u = (int64_t)blockIdx.x * kWarpsPerCta + warp;
    if (u >= U) return;   // warp-uniform
    if ((threadIdx.x & 31) == 0) mbar_init(bar);
    __syncwarp();
    UnitIn cur = u < U0 ? load_unit<0, E>(P, u) : load_unit<1, E>(P, u - U0);
    for (uint32_t parity = 0; u < U; u += T, parity ^= 1u) {
        const int64_t nu = u + T;
        UnitIn nxt{-1, 0, 0.f, -1};
        if (nu < U) nxt = nu < U0 ? load_unit<0, E>(P, nu) : load_unit<1, E>(P, nu - U0);
        const bool ok = u < U0 ? grad_unit<0, S, NG, E, BF>(P, u, cur, ys, es, ow, sg, bar, parity)
                               : grad_unit<1, S, NG, E, BF>(P, u - U0, cur, ys, es, ow, sg, bar, parity);
        if (!ok) return;
        cur = nxt;
    }
}

// ---- kernel 2: the Langevin update --------------------------------------

// Philox4x32-10 (Salmon et al., SC'11) with the round keys precomputed on the
// host: each round multiplies words 0 and 2 into 64-bit products and mixes
// their high halves with words 1, 3 and the round key.
__device__ __forceinline__ uint4 philox(uint4 c, const UpdParams &P)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ P.rk0[r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ P.rk1[r], (uint32_t)p0);
    }
    return c;
}

__device__ __forceinline__ float update1(const UpdParams &P, const UpdSide &Sd, float x, float g,
                                         float z, float eps, float sd)
{
    const float drift = fmaf(P.S, g, fmaf(Sd.prior_b, x, Sd.prior_a));
    const float y = fmaf(sd, z, fmaf(eps, drift, x));
    return P.mirror ? fabsf(y) : y;
}

// One (row, float4 group) item of factor SID (0 = W, 1 = H^T); SID is a
// template parameter so that the side's fields are fixed parameter offsets.
template <int SID>
__device__ __forceinline__ void update_item(const UpdParams &P, int64_t item, float eps, float sd,
                                            uint32_t t_lo, uint32_t t_hi)
{
    const UpdSide &Sd = P.side[SID];
    const int ng = P.ngroups, ldk = P.ldk;
    const int64_t row = P.div_magic ? (int64_t)__umulhi((uint32_t)item, P.div_magic) : item / ng;
    const int q = (int)(item - row * ng);
    const int64_t off = row * ldk + 4 * q;
    const float4 x = ldg4(Sd.X_cur + off);
    // this row's gradient.  Dense path: G, or the sum in M-tile order of
    // the block's partial arrays.  Sparse path: nothing (no entries), G
    // (entries within one unit), or its first unit's tail slot plus the
    // later units' head slots.
    float4 g = zero4();
    if (Sd.gparts > 0) {
        g = ldg4(Sd.Gin + off);
        for (int h = 1; h < Sd.gparts; ++h) add4(g, ldg4(Sd.Gin + h * Sd.gstride + off));
    } else {
        const int64_t p0 = __ldg(Sd.ptr + row) - Sd.base, p1 = __ldg(Sd.ptr + row + 1) - Sd.base;
        if (p1 > p0) {
            const int64_t u0 = p0 >> P.unit_shift, u1 = (p1 - 1) >> P.unit_shift;
            if (u0 == u1) {
                g = ldg4(Sd.Gin + off);
            } else {
                g = __ldcg(reinterpret_cast<const float4 *>(Sd.partial + (2 * u0 + 1) * ldk + 4 * q));
                const float *hp = Sd.partial + 4 * q;
                int64_t uu = u0 + 1;
                for (; uu + 8 <= u1 + 1; uu += 8) {   // eight independent loads in flight
                    float4 v[8];
#pragma unroll
                    for (int w = 0; w < 8; ++w)
                        v[w] = __ldcg(reinterpret_cast<const float4 *>(hp + 2 * (uu + w) * ldk));
#pragma unroll
                    for (int w = 0; w < 8; ++w) add4(g, v[w]);
                }
                for (; uu <= u1; ++uu)
                    add4(g, __ldcg(reinterpret_cast<const float4 *>(hp + 2 * uu * ldk)));
            }
        }
    }
    const uint4 r = philox(make_uint4((uint32_t)q, (uint32_t)row, t_lo, (t_hi << 1) | (uint32_t)SID), P);
    const float4 z = dev::box_muller4(r);
    const int k0 = 4 * q;
    float4 o;
    o.x = update1(P, Sd, x.x, g.x, z.x, eps, sd);
    o.y = k0 + 1 < P.K ? update1(P, Sd, x.y, g.y, z.y, eps, sd) : 0.f;
    o.z = k0 + 2 < P.K ? update1(P, Sd, x.z, g.z, z.z, eps, sd) : 0.f;
    o.w = k0 + 3 < P.K ? update1(P, Sd, x.w, g.w, z.w, eps, sd) : 0.f;
    *reinterpret_cast<float4 *>(Sd.X_next + off) = o;
    if (Sd.sh) dev::shadow_store4(Sd.sh, row, k0, o, Sd.n_rows, P.B, Sd.sh_tiles, P.sh_kp);
    if (Sd.g16) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(o.x, o.y), b = __floats2bfloat162_rn(o.z, o.w);
        *reinterpret_cast<uint2 *>(Sd.g16 + row * P.ld16 + k0) =
            make_uint2(*reinterpret_cast<const uint32_t *>(&a), *reinterpret_cast<const uint32_t *>(&b));
    }
}

__global__ void __launch_bounds__(kThreads, 5) update_kernel(const __grid_constant__ UpdParams P)
{
    const int64_t t = P.t_dev ? *P.t_dev + P.t_add : P.t_add;
    float eps = P.eps, sd = P.sd;
    if (P.eps_poly) {
        const double e = pow(P.eps_a / (double)t, P.eps_b);
        eps = (float)e;
        sd = (float)sqrt(2.0 * e);
    }
    const uint32_t t_lo = (uint32_t)(uint64_t)t, t_hi = (uint32_t)((uint64_t)t >> 32);
    // the flat item sequence: W items, then H^T items
    const int64_t n0 = P.side[0].items, n1 = P.side[1].items;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    int64_t a = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    for (; a < n0; a += stride) update_item<0>(P, a, eps, sd, t_lo, t_hi);
    for (a -= n0; a < n1; a += stride) update_item<1>(P, a, eps, sd, t_lo, t_hi);
}

// The update of the sparse path for one context, with 32-bit index
// arithmetic (every row offset and item index of both factors below 2^31,
// checked on the host) and no BF16 copies to write: the same arithmetic,
// the same result bit for bit as update_item, in fewer instructions.
template <int SID>
__device__ __forceinline__ void update_item32(const UpdParams &P, uint32_t item, float eps, float sd,
                                              uint32_t t_lo, uint32_t t_hi)
{
    const UpdSide &Sd = P.side[SID];
    const uint32_t ng = (uint32_t)P.ngroups;
    const uint32_t row = P.div_magic ? __umulhi(item, P.div_magic) : item / ng;
    const uint32_t q = item - row * ng;
    const uint32_t off = row * (uint32_t)P.ldk + 4u * q;
    const float4 x = ldg4(Sd.X_cur + off);
    float4 g = zero4();
    const int p0 = __ldg(Sd.ptr + row) - (int)Sd.base, p1 = __ldg(Sd.ptr + row + 1) - (int)Sd.base;
    if (p1 > p0) {
        const int u0 = p0 >> P.unit_shift, u1 = (p1 - 1) >> P.unit_shift;
        if (u0 == u1) {
            g = ldg4(Sd.Gin + off);
        } else {
            // the row's first unit's tail slot, then the later units' head slots, in unit order
            const uint32_t ldk = (uint32_t)P.ldk;
            g = __ldcg(reinterpret_cast<const float4 *>(Sd.partial + (2u * u0 + 1u) * ldk + 4u * q));
            const float *hp = Sd.partial + 4u * q;
            int uu = u0 + 1;
            for (; uu + 8 <= u1 + 1; uu += 8) {   // eight independent loads in flight
                float4 v[8];
#pragma unroll
                for (int w = 0; w < 8; ++w)
                    v[w] = __ldcg(reinterpret_cast<const float4 *>(hp + 2u * (uint32_t)(uu + w) * ldk));
#pragma unroll
                for (int w = 0; w < 8; ++w) add4(g, v[w]);
            }
            for (; uu <= u1; ++uu) add4(g, __ldcg(reinterpret_cast<const float4 *>(hp + 2u * (uint32_t)uu * ldk)));
        }
    }
    const uint4 r = philox(make_uint4(q, row, t_lo, (t_hi << 1) | (uint32_t)SID), P);
    const float4 z = dev::box_muller4(r);
    float4 o;
    o.x = update1(P, Sd, x.x, g.x, z.x, eps, sd);
    o.y = update1(P, Sd, x.y, g.y, z.y, eps, sd);
    o.z = update1(P, Sd, x.z, g.z, z.z, eps, sd);
    o.w = update1(P, Sd, x.w, g.w, z.w, eps, sd);
    // the padding columns (k >= K) stay zero: their x, g are zero and the
    // noise is masked (K is a multiple of 4 except in the last group)
    if (4u * q + 4u > (uint32_t)P.K) {
        const uint32_t k0 = 4u * q;
        if (k0 + 1 >= (uint32_t)P.K) o.y = 0.f;
        if (k0 + 2 >= (uint32_t)P.K) o.z = 0.f;
        if (k0 + 3 >= (uint32_t)P.K) o.w = 0.f;
    }
    *reinterpret_cast<float4 *>(Sd.X_next + off) = o;
}

__global__ void __launch_bounds__(kThreads, 5) update_kernel32(const __grid_constant__ UpdParams P)
{
    const int64_t t = P.t_dev ? *P.t_dev + P.t_add : P.t_add;
    float eps = P.eps, sd = P.sd;
    if (P.eps_poly) {
        const double e = pow(P.eps_a / (double)t, P.eps_b);
        eps = (float)e;
        sd = (float)sqrt(2.0 * e);
    }
    const uint32_t t_lo = (uint32_t)(uint64_t)t, t_hi = (uint32_t)((uint64_t)t >> 32);
    const uint32_t n0 = (uint32_t)P.side[0].items, n1 = (uint32_t)P.side[1].items;
    const uint32_t stride = gridDim.x * kThreads;
    uint32_t a = blockIdx.x * kThreads + threadIdx.x;
    for (; a < n0; a += stride) update_item32<0>(P, a, eps, sd, t_lo, t_hi);
    for (a -= n0; a < n1; a += stride) update_item32<1>(P, a, eps, sd, t_lo, t_hi);
}

// The update of the dense path with 32-bit index arithmetic (items, factor
// and gradient offsets and the BF16 shadows' offsets all below 2^31,
// checked on the host): the same arithmetic, the same result bit for bit as
// update_item on the dense path, in fewer instructions.  The shadow's tile
// layout is dev::shadow_store4's, here in 32-bit offsets.
__device__ __forceinline__ void shadow_store4_32(uint16_t *sh, uint32_t row, uint32_t k0, float4 v, uint32_t n,
                                                 uint32_t B, uint32_t tiles, uint32_t KP)
{
    const uint32_t piece = ((row + 1u) * B - 1u) / n;
    const uint32_t rr = row - (piece * n) / B;
    const uint32_t rho = rr & 63u;
    const uint32_t kk = k0 & 63u, c = kk >> 3;
    const uint32_t off = (piece * tiles + (rr >> 6)) * 64u * KP + (k0 >> 6) * 4096u + rho * 64u +
                         ((c ^ (rho & 7u)) << 3) + (kk & 7u);
    __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
    *reinterpret_cast<uint2 *>(sh + off) =
        make_uint2(*reinterpret_cast<uint32_t *>(&lo), *reinterpret_cast<uint32_t *>(&hi));
}

template <int SID>
__device__ __forceinline__ void update_item_dense32(const UpdParams &P, uint32_t item, float eps, float sd,
                                                    uint32_t t_lo, uint32_t t_hi)
{
    const UpdSide &Sd = P.side[SID];
    const uint32_t ng = (uint32_t)P.ngroups;
    const uint32_t row = P.div_magic ? __umulhi(item, P.div_magic) : item / ng;
    const uint32_t q = item - row * ng;
    const uint32_t off = row * (uint32_t)P.ldk + 4u * q;
    const float4 x = ldg4(Sd.X_cur + off);
    // G, or the sum in M-tile order of the block's partial arrays
    float4 g = ldg4(Sd.Gin + off);
    for (int h = 1; h < Sd.gparts; ++h) add4(g, ldg4(Sd.Gin + (uint32_t)h * (uint32_t)Sd.gstride + off));
    const uint4 r = philox(make_uint4(q, row, t_lo, (t_hi << 1) | (uint32_t)SID), P);
    const float4 z = dev::box_muller4(r);
    float4 o;
    o.x = update1(P, Sd, x.x, g.x, z.x, eps, sd);
    o.y = update1(P, Sd, x.y, g.y, z.y, eps, sd);
    o.z = update1(P, Sd, x.z, g.z, z.z, eps, sd);
    o.w = update1(P, Sd, x.w, g.w, z.w, eps, sd);
    const uint32_t k0 = 4u * q;
    if (k0 + 4u > (uint32_t)P.K) {   // padding columns stay zero
        if (k0 + 1 >= (uint32_t)P.K) o.y = 0.f;
        if (k0 + 2 >= (uint32_t)P.K) o.z = 0.f;
        if (k0 + 3 >= (uint32_t)P.K) o.w = 0.f;
    }
    *reinterpret_cast<float4 *>(Sd.X_next + off) = o;
    if (Sd.sh)
        shadow_store4_32(Sd.sh, row, k0, o, (uint32_t)Sd.n_rows, (uint32_t)P.B, (uint32_t)Sd.sh_tiles,
                         (uint32_t)P.sh_kp);
}

__global__ void __launch_bounds__(kThreads, 5) update_kernel_dense32(const __grid_constant__ UpdParams P)
{
    const int64_t t = P.t_dev ? *P.t_dev + P.t_add : P.t_add;
    float eps = P.eps, sd = P.sd;
    if (P.eps_poly) {
        const double e = pow(P.eps_a / (double)t, P.eps_b);
        eps = (float)e;
        sd = (float)sqrt(2.0 * e);
    }
    const uint32_t t_lo = (uint32_t)(uint64_t)t, t_hi = (uint32_t)((uint64_t)t >> 32);
    const uint32_t n0 = (uint32_t)P.side[0].items, n1 = (uint32_t)P.side[1].items;
    const uint32_t stride = gridDim.x * kThreads;
    uint32_t a = blockIdx.x * kThreads + threadIdx.x;
    for (; a < n0; a += stride) update_item_dense32<0>(P, a, eps, sd, t_lo, t_hi);
    for (a -= n0; a < n1; a += stride) update_item_dense32<1>(P, a, eps, sd, t_lo, t_hi);
}

using GradFn = void (*)(GradParams);

struct Shape {
    int S, NG, E, lds;
};

// Sub-team lanes S and float4 groups per lane NG cover K; E entries per unit
// keep a warp's shared memory (E gathered rows) near 17 KB at most; the row
// stride is padded so that its float4 count is odd (each lane reading its own
// row hits distinct banks).
Shape shape_for(int ngroups)
{
    Shape sh;
    if (ngroups <= 4) {            // K <= 16: one float4 group per lane
        sh.S = 1;
        while (sh.S < ngroups) sh.S <<= 1;
        sh.NG = 1;
    } else {                       // two groups per lane, up to 32 lanes
        sh.S = 4;
        while (sh.S * 2 < ngroups && sh.S < 32) sh.S <<= 1;
        sh.NG = (ngroups + sh.S - 1) / sh.S;
    }
    sh.E = ngroups <= 32 ? 32 : ngroups <= 64 ? 16 : 8;
    sh.lds = (ngroups & 1) ? 4 * ngroups : 4 * ngroups + 4;
    return sh;
}

template <bool BF>
GradFn pick_grad_t(const Shape &sh)
{
    if (sh.NG == 1) {
        switch (sh.S) {
        case 1: return grad_kernel<1, 1, 32, BF>;
        case 2: return grad_kernel<2, 1, 32, BF>;
        case 4: return grad_kernel<4, 1, 32, BF>;
        }
    }
    if (sh.NG == 2) {
        switch (sh.S) {
        case 4: return grad_kernel<4, 2, 32, BF>;
        case 8: return grad_kernel<8, 2, 32, BF>;
        case 16: return grad_kernel<16, 2, 32, BF>;
        case 32: return grad_kernel<32, 2, 16, BF>;
        }
    }
    if (sh.S == 32) {
        switch (sh.NG) {
        case 3: return grad_kernel<32, 3, 8, BF>;
        case 4: return grad_kernel<32, 4, 8, BF>;
        }
    }
    return nullptr;
}

// BF: the variant that gathers the BF16 copies of the factors
GradFn pick_grad(const Shape &sh, bool bf)
{
    return bf ? pick_grad_t<true>(sh) : pick_grad_t<false>(sh);
}

// BF16 gather copies: rows of ld16 = ldk rounded up to 8 (16-byte rows for
// the bulk copies); shared-memory stride lds16 >= ld16 with lds16 / 8 odd,
// so that the lanes' 8-byte reads of distinct rows spread over the banks.
int ld16_for(int ldk) { return 8 * ((ldk + 7) / 8); }
int lds16_for(int ldk)
{
    const int m = ld16_for(ldk) / 8;
    return 8 * ((m & 1) ? m : m + 1);
}

size_t grad_smem(const Shape &sh)
{
    const int warps = kGradThreads / 32;
    return sizeof(float) * (size_t)warps * ((size_t)sh.E * sh.lds + 3 * sh.E + 1) +
           sizeof(uint64_t) * warps;
}

}  // namespace

namespace {

// BF16 copy of an n x ldk FP32 factor into rows of ld16 (padding zero)
__global__ void gather_copy_kernel(const float *__restrict__ X, int64_t n, int ldk, int ld16,
                                   uint16_t *__restrict__ Y)
{
    const int64_t total = n * ld16;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < total;
         a += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = a / ld16;
        const int k = (int)(a - r * ld16);
        const float x = k < ldk ? X[r * ldk + k] : 0.f;
        const __nv_bfloat16 b = __float2bfloat16_rn(x);
        Y[a] = *reinterpret_cast<const uint16_t *>(&b);
    }
}

}  // namespace

bool gather_bf16(const psgld_ctx *c) { return c->opt.gather_bf16 && !c->dense && c->W16 && c->H16; }

psgld_status build_gather_shadows(psgld_ctx *c, cudaStream_t st)
{
    if (!c->opt.gather_bf16 || c->dense || !c->has_factors) return PSGLD_OK;
    const int ld16 = ld16_for(c->ldk);
    for (int side = 0; side < 2; ++side) {
        const int64_t n = side == 0 ? c->I : c->J;
        uint16_t *&Y = side == 0 ? c->W16 : c->H16;
        if (!Y) {
            Y = static_cast<uint16_t *>(dev_alloc(c, sizeof(uint16_t) * (size_t)std::max<int64_t>(n * ld16, 1), st));
            if (!Y) return fail(c, PSGLD_ERR_OOM, "device allocation failed");
        }
        const float *X = side == 0 ? c->W[c->wcur] : c->Ht[c->hcur];
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n * ld16 + 255) / 256, 152 * 16));
        gather_copy_kernel<<<grid, 256, 0, st>>>(X, n, c->ldk, ld16, Y);
        PSGLD_CK(c, cudaGetLastError());
    }
    return PSGLD_OK;
}

int unit_entries(int ngroups) { return shape_for(ngroups).E; }

// CTAs of kernel `f` (`threads` threads, `smem` bytes of dynamic shared
// memory each) resident at once on the current device: SMs x CTAs per SM,
// remembered per host thread for the last two kernels asked about (the
// gradient kernels of one context, FP32 and BF16 gathers).
static int64_t resident_wave(const void *f, int threads, size_t smem)
{
    struct Entry {
        const void *f;
        int threads;
        size_t smem;
        int dev;
        int64_t wave;
    };
    thread_local Entry memo[2] = {{nullptr, 0, 0, -1, 0}, {nullptr, 0, 0, -1, 0}};
    thread_local int next = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1ll << 40;
    for (const Entry &e : memo)
        if (e.f == f && e.threads == threads && e.smem == smem && e.dev == dev) return e.wave;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, smem) != cudaSuccess ||
        sms <= 0 || per_sm <= 0)
        return 1ll << 40;   // unknown: no cap
    memo[next] = {f, threads, smem, dev, (int64_t)sms * per_sm};
    next ^= 1;
    return (int64_t)sms * per_sm;
}

psgld_status prepare_kernels(psgld_ctx *c)
{
    const Shape sh = shape_for(c->ngroups);
    for (int bf = 0; bf < 2; ++bf) {
        GradFn gfn = pick_grad(sh, bf != 0);
        if (!gfn) return fail(c, PSGLD_ERR_ARG, "unsupported K");
        PSGLD_CK(c, cudaFuncSetAttribute(gfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)grad_smem(sh)));
    }
    return PSGLD_OK;
}

// Kernel parameters of iteration t (part `part`) for context c: the gradient
// kernel's and the update kernel's.  With t_dev the update kernel reads t
// from *t_dev + t_add (captured graphs).
static void fill_params(psgld_ctx *c, int part, int64_t t, const int64_t *t_dev, int64_t t_add,
                        GradParams &GP, UpdParams &UP)
{
    const int B = c->B;
    const Shape sh = shape_for(c->ngroups);
    const bool dense = c->dense;
    const bool upd[2] = {!c->opt.freeze_W, !c->opt.freeze_H};
    GP = GradParams{};
    UP = UpdParams{};
    for (int s = 0; s < 2; ++s) {
        SideLayout &L = c->side[s];
        GradSide &Gs = GP.side[s];
        UpdSide &Us = UP.side[s];
        const int64_t n_rows = s == 0 ? c->I : c->J;
        float *X_cur = s == 0 ? c->W[c->wcur] : c->Ht[c->hcur];
        float *X_next = s == 0 ? c->W[c->wcur ^ 1] : c->Ht[c->hcur ^ 1];
        float *G_rows = c->G + (s == 0 ? 0 : c->I * c->ldk);
        const int64_t base = dense ? 0 : L.part_first[part];
        const int64_t n = dense ? 0 : L.part_first[part + 1] - base;
        Gs.X_cur = X_cur;
        Gs.Y_cur = s == 0 ? c->Ht[c->hcur] : c->W[c->wcur];
        Gs.Gout = G_rows;
        Gs.own = L.own;
        Gs.idx = L.idx;
        Gs.val = L.val;
        Gs.partial = L.partial;
        Gs.base = base;
        Gs.n = n;
        Gs.units = upd[s] ? (n + sh.E - 1) / sh.E : 0;
        Gs.Y16 = gather_bf16(c) ? (s == 0 ? c->H16 : c->W16) : nullptr;
        Gs.prefetch_own = 4.0 * (double)n_rows * c->ldk > 64.0 * (1 << 20);

        Us.X_cur = X_cur;
        Us.X_next = X_next;
        Us.Gin = G_rows;
        Us.ptr = dense ? nullptr : L.ptr + (int64_t)part * n_rows;
        Us.gparts = dense ? 1 : 0;
        if (dense && c->dense_kind == 1 && s == 1 && c->mtiles > 1) {
            Us.Gin = c->hpart;
            Us.gparts = c->mtiles;
            Us.gstride = c->J * c->ldk;
        }
        Us.n_rows = n_rows;
        if (dense && c->dense_kind == 2) {
            Us.sh = s == 0 ? c->Wsh : c->Hsh;
            Us.sh_tiles = 2 * (s == 0 ? c->mt_max : c->nt_max);
        }
        Us.partial = L.partial;
        Us.g16 = gather_bf16(c) ? (s == 0 ? c->W16 : c->H16) : nullptr;
        Us.base = base;
        Us.items = upd[s] ? n_rows * c->ngroups : 0;
        if (c->prior.kind == PSGLD_PRIOR_EXPONENTIAL) {
            Us.prior_a = (float)-(s == 0 ? c->prior.lambda_w : c->prior.lambda_h);
            Us.prior_b = 0.f;
        } else {
            const double sg = s == 0 ? c->prior.sigma_w : c->prior.sigma_h;
            Us.prior_a = 0.f;
            Us.prior_b = (float)(-1.0 / (sg * sg));
        }
        Us.mat = (uint32_t)s;
    }
    GP.ldk = c->ldk;
    GP.lds = sh.lds;
    GP.ld16 = ld16_for(c->ldk);
    GP.lds16 = lds16_for(c->ldk);
    GP.ngroups = c->ngroups;
    GP.phi_inv = (float)(1.0 / c->phi);
    GP.p = (float)c->p;
    GP.mu_min = (float)c->opt.mu_min;
    GP.p_mode = c->p == 0.0 ? 0 : c->p == 1.0 ? 1 : c->p == 2.0 ? 2 : 3;
    GP.err = c->kflag;
    GP.wait_polls = (uint32_t)c->opt.debug_wait_polls;

    UP.t_dev = t_dev;
    UP.t_add = t_dev ? t_add : t;
    UP.K = c->K;
    UP.ldk = c->ldk;
    UP.ngroups = c->ngroups;
    UP.unit_shift = sh.E == 32 ? 5 : sh.E == 16 ? 4 : 3;
    const int64_t max_items = std::max(UP.side[0].items, UP.side[1].items);
    UP.div_magic = (max_items * c->ngroups < (1ll << 32))
                       ? (uint32_t)(((1ull << 32) + c->ngroups - 1) / c->ngroups)
                       : 0u;
    const double eps = c->opt.eps;
    UP.eps = (float)eps;
    UP.sd = (float)std::sqrt(2.0 * eps);
    UP.eps_poly = c->opt.eps_mode == PSGLD_EPS_POLY;
    UP.eps_a = c->opt.eps_a;
    UP.eps_b = c->opt.eps_b;
    const int64_t np = c->part_n[part];
    UP.S = c->opt.scale_mode == PSGLD_SCALE_B ? (float)B
                                              : (np > 0 ? (float)((double)c->N / (double)np) : 0.f);
    UP.mirror = c->prior.kind == PSGLD_PRIOR_EXPONENTIAL;
    UP.B = B;
    UP.sh_kp = c->KP;
    UP.ld16 = ld16_for(c->ldk);
    uint32_t k0 = (uint32_t)c->opt.seed, k1 = (uint32_t)(c->opt.seed >> 32);
    for (int r = 0; r < 10; ++r) {   // Weyl key schedule of Philox4x32
        UP.rk0[r] = k0;
        UP.rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

psgld_status launch_part_step(psgld_ctx *c, int64_t t, const int64_t *t_dev, int64_t t_add,
                              cudaStream_t st)
{
    const int B = c->B;
    const int part = part_of_iteration(c, t);
    const Shape sh = shape_for(c->ngroups);
    GradFn gfn = pick_grad(sh, gather_bf16(c));
    if (!gfn) return fail(c, PSGLD_ERR_ARG, "unsupported K");
    const bool dense = c->dense;
    const bool upd[2] = {!c->opt.freeze_W, !c->opt.freeze_H};
    GradParams GP;
    UpdParams UP;
    fill_params(c, part, t, t_dev, t_add, GP, UP);

    const int64_t units = GP.side[0].units + GP.side[1].units;
    const int ggrid = (int)((units + kGradThreads / 32 - 1) / (kGradThreads / 32));
    const int64_t items = UP.side[0].items + UP.side[1].items;
    // Inside a stream capture the records must be external, so that they
    // become event-record nodes of the graph (a plain record would only
    // become a dependency edge); outside a capture they are plain records.
    const bool prof = c->opt.profile && (int)c->ev_start.size() == B;
    unsigned rec_flags = cudaEventRecordDefault;
    if (prof) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        PSGLD_CK(c, cudaStreamIsCapturing(st, &cap));
        if (cap == cudaStreamCaptureStatusActive) rec_flags = cudaEventRecordExternal;
        PSGLD_CK(c, cudaEventRecordWithFlags(c->ev_start[part], st, rec_flags));
    }
    // the sparse path takes the 32-bit update kernel when every index fits
    // (items, row offsets of both factors and the partial slots)
    const int64_t lim = (1ll << 31) - 1;
    const int64_t slots = 2 * std::max(c->side[0].max_units, c->side[1].max_units) * c->ldk;
    const bool small = !dense && !gather_bf16(c) && items <= lim &&
                       std::max(c->I, c->J) * c->ldk <= lim && slots <= lim && c->N <= lim;
    // the dense path's 32-bit update: items, factor rows, every partial
    // gradient array and the BF16 shadows within 2^31
    const int64_t sh_elems = c->dense_kind == 2
        ? (int64_t)B * 2 * std::max<int64_t>(c->mt_max, c->nt_max) * 64 * c->KP : 0;
    const bool dense32 = dense && !gather_bf16(c) && items <= lim && std::max(c->I, c->J) * c->ldk <= lim &&
                         (int64_t)std::max(1, c->mtiles) * c->J * c->ldk <= lim && sh_elems <= lim;
    auto update = [&](const UpdParams &U, cudaStream_t ss) {
        const int64_t n = U.side[0].items + U.side[1].items;
        const int grid = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 16);
        if (grid <= 0) return;
        if (small) update_kernel32<<<grid, kThreads, 0, ss>>>(U);
        else if (dense32) update_kernel_dense32<<<grid, kThreads, 0, ss>>>(U);
        else update_kernel<<<grid, kThreads, 0, ss>>>(U);
    };
    // resident: one wave of CTAs whose warps walk several units each (the
    // next unit's entries load during the current one); otherwise one unit
    // per warp, so that two launches on two streams share the SMs
    auto gradient = [&](const GradParams &G, cudaStream_t ss, bool resident) {
        const int64_t n = G.side[0].units + G.side[1].units;
        int64_t grid = (n + kGradThreads / 32 - 1) / (kGradThreads / 32);
        if (resident) grid = std::min<int64_t>(grid, resident_wave((const void *)gfn, kGradThreads, grad_smem(sh)));
        if (grid > 0) gfn<<<(int)grid, kGradThreads, grad_smem(sh), ss>>>(G);
    };
    // W and H^T on two streams when the factors fit in L2 (W and H^T at most
    // 64 MB): each side's gradient, then its update; their outputs are
    // disjoint (G rows, partial slots, next buffers of the ping-ponged
    // factors), so the result is the same bit for bit, and the ALU-bound
    // update of one side overlaps the L2-bound gathers of the other (10 M
    // entries, K = 50: 1.58 to 1.50 ms per sweep).  With factors beyond L2
    // the W side's gradient runs alone on the full (resident) grid first,
    // then the H side's gradient and the W side's update run side by side:
    // the latency-bound gathers leave issue slots that the ALU-bound update
    // fills (10^8 entries, K = 100: 21.4 to 19.9 ms per sweep; the earlier
    // order, both gradients at once and the updates after them, had been
    // slower than one stream).  Not with gather_bf16: the BF16 copies that
    // the gathers read are single-buffered and rewritten by the updates.
    // Inside a capture the fork and join become graph edges.
    const bool l2_fit = 4.0 * (double)(c->I + c->J) * c->ldk <= 64.0 * (1 << 20);
    if (!dense && !prof && !gather_bf16(c) && l2_fit && c->side_stream && upd[0] && upd[1]) {
        GradParams GW = GP, GH = GP;
        GW.side[1].units = 0;
        GH.side[0].units = 0;
        UpdParams UW = UP, UH = UP;
        UW.side[1].items = 0;
        UH.side[0].items = 0;
        PSGLD_CK(c, cudaEventRecord(c->ev_fork, st));
        PSGLD_CK(c, cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0));
        gradient(GH, c->side_stream, false);
        update(UH, c->side_stream);
        gradient(GW, st, false);
        update(UW, st);
        PSGLD_CK(c, cudaGetLastError());
        PSGLD_CK(c, cudaEventRecord(c->ev_join, c->side_stream));
        PSGLD_CK(c, cudaStreamWaitEvent(st, c->ev_join, 0));
    } else if (!dense && !prof && !gather_bf16(c) && c->side_stream && upd[0] && upd[1] && ggrid > 0) {
        GradParams GW = GP, GH = GP;
        GW.side[1].units = 0;
        GH.side[0].units = 0;
        UpdParams UW = UP, UH = UP;
        UW.side[1].items = 0;
        UH.side[0].items = 0;
        gradient(GW, st, true);
        PSGLD_CK(c, cudaEventRecord(c->ev_fork, st));
        PSGLD_CK(c, cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0));
        gradient(GH, c->side_stream, true);   // enqueued ahead of the W update
        update(UH, c->side_stream);
        update(UW, st);
        PSGLD_CK(c, cudaGetLastError());
        PSGLD_CK(c, cudaEventRecord(c->ev_join, c->side_stream));
        PSGLD_CK(c, cudaStreamWaitEvent(st, c->ev_join, 0));
    } else {
        if (dense) {
            if (upd[0] || upd[1]) {
                const psgld_status ds = launch_dense_grad(c, part, st);
                if (ds != PSGLD_OK) return ds;
            }
        } else if (ggrid > 0) {
            gradient(GP, st, true);
        }
        PSGLD_CK(c, cudaGetLastError());
        if (prof) PSGLD_CK(c, cudaEventRecordWithFlags(c->ev_mid[part], st, rec_flags));
        if (items > 0) update(UP, st);
    }
    PSGLD_CK(c, cudaGetLastError());
    if (prof) {
        PSGLD_CK(c, cudaEventRecordWithFlags(c->ev_end[part], st, rec_flags));
        c->ev_pending[part] = 1;
    }
    if (upd[0]) c->wcur ^= 1;
    if (upd[1]) c->hcur ^= 1;
    return PSGLD_OK;
}

namespace {

// ---- many contexts in one update launch ------------------------------------

__global__ void __launch_bounds__(kThreads, 4)
update_batch_kernel(const UpdParams *__restrict__ Ps, const int64_t *__restrict__ item_start, int n)
{
    const int64_t total = __ldg(item_start + n);
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    int ci = -1;
    float eps = 0.f, sd = 0.f;
    uint32_t t_lo = 0, t_hi = 0;
    for (int64_t a = blockIdx.x * (int64_t)kThreads + threadIdx.x; a < total; a += stride) {
        if (ci < 0 || __ldg(item_start + ci + 1) <= a) {
            int lo = ci < 0 ? 0 : ci, hi = n - 1;   // last i with item_start[i] <= a
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(item_start + mid) <= a) lo = mid; else hi = mid - 1;
            }
            ci = lo;
            const UpdParams &P = Ps[ci];
            const int64_t t = P.t_dev ? *P.t_dev + P.t_add : P.t_add;
            eps = P.eps;
            sd = P.sd;
            if (P.eps_poly) {
                const double e = pow(P.eps_a / (double)t, P.eps_b);
                eps = (float)e;
                sd = (float)sqrt(2.0 * e);
            }
            t_lo = (uint32_t)(uint64_t)t;
            t_hi = (uint32_t)((uint64_t)t >> 32);
        }
        const UpdParams &P = Ps[ci];
        const int64_t local = a - __ldg(item_start + ci);
        if (local < P.side[0].items) update_item<0>(P, local, eps, sd, t_lo, t_hi);
        else update_item<1>(P, local - P.side[0].items, eps, sd, t_lo, t_hi);
    }
}

}  // namespace

size_t upd_param_bytes() { return sizeof(UpdParams); }

int64_t fill_upd_param(psgld_ctx *c, int part, const int64_t *t_dev, int64_t t_add, void *dst)
{
    GradParams GP;
    UpdParams UP;
    fill_params(c, part, t_add, t_dev, t_add, GP, UP);
    std::memcpy(dst, &UP, sizeof UP);
    return UP.side[0].items + UP.side[1].items;
}

psgld_status launch_update_batch(psgld_ctx *c0, const void *params, const int64_t *item_start, int n,
                                 int64_t total_items, cudaStream_t st)
{
    const int64_t cap = c0->opt.batch_update_blocks > 0 ? c0->opt.batch_update_blocks : 152 * 16;
    const int grid = (int)std::min<int64_t>((total_items + kThreads - 1) / kThreads, cap);
    if (grid > 0)
        update_batch_kernel<<<grid, kThreads, 0, st>>>(static_cast<const UpdParams *>(params), item_start, n);
    PSGLD_CK(c0, cudaGetLastError());
    return PSGLD_OK;
}

}  // namespace psgld
