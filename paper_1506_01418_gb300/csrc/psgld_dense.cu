// psgld_dense.cu -- the likelihood gradient of one PSGLD iteration on dense V
// with the 5th-generation tensor cores (tcgen05, accumulators in TMEM).
//
// For block b of part Pi_t (rows R_b of row piece b, columns C_b of column
// piece (b + s) mod B; Definitions 1-2) the gradient terms of Eq. psgld_w and
// Eq. psgld_h are three contractions around the Tweedie epilogue (Sec. 4):
//   GEMM1  mu   = W_b H_b                           (|R_b| x |C_b|, inner K)
//   epi    E    = (V_b - mu) max(mu, mu_min)^(-p) / phi
//   GEMM2  G_W  = E H_b^T                           (|R_b| x K, inner |C_b|)
//   GEMM3  G_H  = E^T W_b                           (|C_b| x K, inner |R_b|)
// The update kernel then applies step, prior, noise and mirror as on the
// sparse path.
//
// One CTA of 128 threads per (block, 128-row M-tile); it walks the block's
// columns in 128-column tiles.  Operands are BF16 in shared memory in the
// canonical no-swizzle K-major layout (8-row x 16-byte core matrices, K-
// adjacent core matrices 128 B apart, 8-row groups KD*16 B apart), written by
// the threads from the FP32 factors; each MMA is tcgen05.mma.cta_group::1
// kind::f16 (BF16 x BF16 -> FP32) issued by one thread, 128 x N x 16 per
// instruction, and completes on an mbarrier through tcgen05.commit.
// TMEM holds mu / G_H (columns 0..127) and the running G_W (columns 128..),
// read back with tcgen05.ld (thread t = TMEM lane t = tile row t).  mu never
// leaves the SM: the epilogue turns it into E in shared memory, both
// orientations, for GEMM2 and GEMM3.  G_W accumulates over the block's column
// tiles in TMEM; G_H of a column tile is written once per M-tile (directly
// when the block has one M-tile, else to per-M-tile partial rows that the
// update kernel adds in order).
//
// Every mbarrier wait is bounded (iterations and about one second of SM
// clock); on a timeout the kernel sets the error flag, waits once more
// (bounded) for the MMAs it issued, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "psgld_internal.cuh"

namespace psgld {
namespace {

constexpr int kDenseThreads = 128;
constexpr int kTile = 128;   // rows of an M-tile = columns of an n-tile
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kDenseWaitLimit = 1u << 24;
constexpr long long kDenseWaitCycles = 1ll << 31;

struct DenseParams {
    const float *V;          // I x ldv, FP32
    int64_t ldv;
    const float *W;          // I x ldk (current)
    const float *Ht;         // J x ldk (current)
    float *G;                // (I + J) x ldk
    float *hpart;            // mtiles x J x ldk partial G_H rows (mtiles > 1)
    int64_t I, J;
    int K, ldk, B, part, mtiles;
    float phi_inv, p, mu_min;
    int p_mode;
    int *err;
};

__device__ __forceinline__ uint32_t saddr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (r, k) in an R x KD K-major no-swizzle tile
__device__ __forceinline__ uint32_t cm_off(int r, int k, int KD)
{
    return (uint32_t)((r >> 3) * (KD * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor (no swizzle): start, leading (K) and
// stride (8-row group) byte offsets, descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptor: FP32 accumulate, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                 "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                   "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
                   "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
                   "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
                   "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ bool bar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(saddr(bar)), "r"(parity), "r"(2000u) : "memory");
    return ok != 0;
}

// bounded wait for phase `parity`; false if it ran out
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity)
{
    bool done = false;
    const long long t0 = clock64();
    for (uint32_t it = 0; it < kDenseWaitLimit && !done && clock64() - t0 < kDenseWaitCycles; ++it)
        done = bar_try_wait(bar, parity);
    return done;
}

__device__ __forceinline__ float tweedie(const DenseParams &P, float v, float mu)
{
    const float d = v - mu;
    if (P.p_mode == 0) return d * P.phi_inv;
    const float mc = fmaxf(mu, P.mu_min);
    if (P.p_mode == 1) return d / mc * P.phi_inv;
    if (P.p_mode == 2) return d / (mc * mc) * P.phi_inv;
    return d * exp2f(-P.p * log2f(mc)) * P.phi_inv;
}

__device__ __forceinline__ void st_bf16(unsigned char *base, uint32_t off, float x)
{
    *reinterpret_cast<__nv_bfloat16 *>(base + off) = __float2bfloat16_rn(x);
}

template <int KP>
__global__ void __launch_bounds__(kDenseThreads, 1) dense_grad_kernel(const __grid_constant__ DenseParams P)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr uint32_t kOpBytes = kTile * KP * 2;           // a 128 x KP BF16 tile
    constexpr uint32_t kEBytes = kTile * kTile * 2;         // a 128 x 128 BF16 tile
    unsigned char *A1 = sm;                     // W tile   rows m, K-dim k   (GEMM1 A)
    unsigned char *B1 = A1 + kOpBytes;          // Ht tile  rows n, K-dim k   (GEMM1 B)
    unsigned char *B2 = B1 + kOpBytes;          // H tile   rows k, K-dim n   (GEMM2 B)
    unsigned char *B3 = B2 + kOpBytes;          // Wt tile  rows k, K-dim m   (GEMM3 B)
    unsigned char *A2 = B3 + kOpBytes;          // E        rows m, K-dim n   (GEMM2 A)
    unsigned char *A3 = A2 + kEBytes;           // E^T      rows n, K-dim m   (GEMM3 A)
    uint64_t *bar = reinterpret_cast<uint64_t *>(A3 + kEBytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int B = P.B;
    const int blk = blockIdx.x / P.mtiles, mt = blockIdx.x % P.mtiles;
    const int cpiece = (blk + P.part) % B;
    const int64_t rs = (int64_t)blk * P.I / B, re = (int64_t)(blk + 1) * P.I / B;
    const int64_t cs = (int64_t)cpiece * P.J / B, ce = (int64_t)(cpiece + 1) * P.J / B;
    const int64_t m0 = rs + (int64_t)mt * kTile;
    const int K = P.K, ldk = P.ldk;
    if (m0 >= re) {
        // this block has one M-tile fewer than the largest: its partial G_H
        // rows are zero, so that the update's sum over M-tiles stays exact
        float *dst = P.hpart + ((int64_t)mt * P.J + cs) * ldk;
        const int64_t n = (ce - cs) * ldk;
        for (int64_t a = tid; a < n; a += kDenseThreads) dst[a] = 0.f;
        return;
    }

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(saddr(tslot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    uint32_t phase = 0;
    bool ok = true;

    // own rows of this M-tile: W (GEMM1 A) and W^T (GEMM3 B), BF16, zero padded
    {
        const int64_t row = m0 + tid;
        const bool rv = row < re;
        for (int k = 0; k < KP; k += 4) {
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
            if (rv && k < K) w = *reinterpret_cast<const float4 *>(P.W + row * ldk + k);
            const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                const float x = k + d < K ? wv[d] : 0.f;
                st_bf16(A1, cm_off(tid, k + d, KP), x);
                st_bf16(B3, cm_off(k + d, tid, kTile), x);
            }
        }
    }

    const uint64_t aW = sdesc(saddr(A1), 128, KP * 16);
    const int ntiles = (int)((ce - cs + kTile - 1) / kTile);
    for (int nt = 0; nt < ntiles && ok; ++nt) {
        const int64_t n0 = cs + (int64_t)nt * kTile;
        // column tile: H^T rows (GEMM1 B) and H (GEMM2 B)
        {
            const int64_t col = n0 + tid;
            const bool cv = col < ce;
            for (int k = 0; k < KP; k += 4) {
                float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
                if (cv && k < K) h = *reinterpret_cast<const float4 *>(P.Ht + col * ldk + k);
                const float hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    const float x = k + d < K ? hv[d] : 0.f;
                    st_bf16(B1, cm_off(tid, k + d, KP), x);
                    st_bf16(B2, cm_off(k + d, tid, kTile), x);
                }
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();

        // GEMM1: mu (TMEM columns 0..127) = W_tile . H_tile
        if (tid == 0) {
            const uint64_t bH = sdesc(saddr(B1), 128, KP * 16);
#pragma unroll
            for (int ks = 0; ks < KP / 16; ++ks)
                mma_bf16(tmem, aW + (uint64_t)(ks * 16), bH + (uint64_t)(ks * 16),
                         idesc_bf16(kTile, kTile), ks > 0);
            mma_commit(bar);
        }
        ok = bar_wait(bar, phase);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) { ok = false; break; }
        fence_after();

        // epilogue: E = Tweedie factor of mu, masked to the block, BF16,
        // into E (rows m) and E^T (rows n)
        {
            const int64_t row = m0 + tid;
            const bool rv = row < re;
            for (int c = 0; c < kTile; c += 32) {
                float mu[32];
                tmem_ld32(tmem + lane_base + (uint32_t)c, mu);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int64_t col = n0 + c + j;
                    float e = 0.f;
                    if (rv && col < ce) e = tweedie(P, P.V[row * P.ldv + col], mu[j]);
                    st_bf16(A2, cm_off(tid, c + j, kTile), e);
                    st_bf16(A3, cm_off(c + j, tid, kTile), e);
                }
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();

        // GEMM2: G_W (columns 128..128+KP) += E . H_tile^T;  GEMM3: G_H tile
        // (columns 0..KP, over mu) = E^T . W_tile
        if (tid == 0) {
            const uint64_t aE = sdesc(saddr(A2), 128, kTile * 16);
            const uint64_t bH2 = sdesc(saddr(B2), 128, kTile * 16);
            const uint64_t aEt = sdesc(saddr(A3), 128, kTile * 16);
            const uint64_t bWt = sdesc(saddr(B3), 128, kTile * 16);
#pragma unroll
            for (int ks = 0; ks < kTile / 16; ++ks)
                mma_bf16(tmem + kTile, aE + (uint64_t)(ks * 16), bH2 + (uint64_t)(ks * 16),
                         idesc_bf16(kTile, KP), (nt > 0 || ks > 0));
#pragma unroll
            for (int ks = 0; ks < kTile / 16; ++ks)
                mma_bf16(tmem, aEt + (uint64_t)(ks * 16), bWt + (uint64_t)(ks * 16),
                         idesc_bf16(kTile, KP), ks > 0);
            mma_commit(bar);
        }
        ok = bar_wait(bar, phase);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) { ok = false; break; }
        fence_after();

        // G_H of this column tile: thread t = column n0 + t (every lane takes
        // part in the warp-wide TMEM loads; only real columns store)
        {
            const int64_t col = n0 + tid;
            const bool cv = col < ce;
            float *dst = P.mtiles == 1 ? P.G + (P.I + col) * ldk
                                       : P.hpart + ((int64_t)mt * P.J + col) * ldk;
            for (int c = 0; c < KP; c += 32) {
                float g[32];
                tmem_ld32(tmem + lane_base + (uint32_t)c, g);
                if (cv) {
#pragma unroll
                    for (int j = 0; j < 32; j += 4)
                        if (c + j < ldk)
                            *reinterpret_cast<float4 *>(dst + c + j) =
                                make_float4(g[j], g[j + 1], g[j + 2], g[j + 3]);
                }
            }
        }
        fence_before();
        __syncthreads();
        fence_after();
    }

    if (ok) {
        // G_W: thread t = row m0 + t
        const int64_t row = m0 + tid;
        for (int c = 0; c < KP; c += 32) {
            float g[32];
            tmem_ld32(tmem + lane_base + (uint32_t)(kTile + c), g);
            if (row < re) {
#pragma unroll
                for (int j = 0; j < 32; j += 4)
                    if (c + j < ldk)
                        *reinterpret_cast<float4 *>(P.G + row * ldk + c + j) =
                            make_float4(g[j], g[j + 1], g[j + 2], g[j + 3]);
            }
        }
    } else {
        if (tid == 0) atomicOr(P.err, 16);
        bar_wait(bar, phase ^ 1u);   // give in-flight MMAs one more bounded chance
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"(kTmemCols) : "memory");
}

using DenseFn = void (*)(DenseParams);

DenseFn pick_dense(int kp)
{
    switch (kp) {
    case 16: return dense_grad_kernel<16>;
    case 32: return dense_grad_kernel<32>;
    case 64: return dense_grad_kernel<64>;
    case 128: return dense_grad_kernel<128>;
    }
    return nullptr;
}

int dense_kp(int K)
{
    int kp = 16;
    while (kp < K) kp <<= 1;
    return kp;
}

size_t dense_smem(int kp)
{
    return 4 * (size_t)kTile * kp * 2 + 2 * (size_t)kTile * kTile * 2 + 16;
}

}  // namespace

bool dense_supported(int K) { return K >= 1 && K <= 128; }

int dense_mtiles(const psgld_ctx *c)
{
    const int64_t rows = (c->I + c->B - 1) / c->B;   // largest row piece
    return (int)((rows + kTile - 1) / kTile);
}

psgld_status prepare_dense(psgld_ctx *c)
{
    DenseFn fn = pick_dense(dense_kp(c->K));
    if (!fn) return fail(c, PSGLD_ERR_ARG, "dense tensor-core path supports K <= 128");
    PSGLD_CK(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)dense_smem(dense_kp(c->K))));
    return PSGLD_OK;
}

psgld_status launch_dense_grad(psgld_ctx *c, int part, cudaStream_t st)
{
    const int kp = dense_kp(c->K);
    DenseFn fn = pick_dense(kp);
    if (!fn) return fail(c, PSGLD_ERR_ARG, "dense tensor-core path supports K <= 128");
    DenseParams P{};
    P.V = c->Vd;
    P.ldv = c->ldv;
    P.W = c->W[c->wcur];
    P.Ht = c->Ht[c->hcur];
    P.G = c->G;
    P.hpart = c->hpart;
    P.I = c->I;
    P.J = c->J;
    P.K = c->K;
    P.ldk = c->ldk;
    P.B = c->B;
    P.part = part;
    P.mtiles = dense_mtiles(c);
    P.phi_inv = (float)(1.0 / c->phi);
    P.p = (float)c->p;
    P.mu_min = (float)c->opt.mu_min;
    P.p_mode = c->p == 0.0 ? 0 : c->p == 1.0 ? 1 : c->p == 2.0 ? 2 : 3;
    P.err = c->kflag;
    fn<<<c->B * P.mtiles, kDenseThreads, dense_smem(kp), st>>>(P);
    PSGLD_CK(c, cudaGetLastError());
    return PSGLD_OK;
}

}  // namespace psgld
