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
// leaves the SM: the epilogue turns it into E in shared memory, which GEMM2
// reads K-major and GEMM3 MN-major (transposed), as GEMM3 does the W tile and
// GEMM2 the H tile.  G_W accumulates over the block's column
// tiles in TMEM; G_H of a column tile is written once per M-tile (directly
// when the block has one M-tile, else to per-M-tile partial rows that the
// update kernel adds in order).
//
// Every mbarrier wait is bounded (iterations and about one second of SM
// clock); on a timeout the kernel sets the error flag, waits once more
// (bounded) for the MMAs it issued, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "psgld_internal.cuh"

namespace psgld {
namespace {

constexpr int kDenseThreads = 256;
constexpr int kTile = 128;   // rows of an M-tile = columns of an n-tile
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kDenseWaitLimit = 1u << 30;
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

// shared-memory matrix descriptor (no swizzle): start, leading byte offset
// (between 8 x 16-byte core matrices adjacent along K) and stride byte offset
// (between core matrices adjacent along M or N), descriptor version 1.  The
// same tile serves as a K-major operand and, read the other way, as an
// MN-major one: for a tile stored as (r, c) core matrices (8 r-rows of 16
// bytes of consecutive c), K-major along c has LBO = c-group stride, SBO =
// r-group stride; MN-major along c (K = r) has LBO = r-group stride, SBO =
// c-group stride.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// The same with the 128-byte swizzle (layout type 2): the operand is stored
// in atoms of 8 rows x 128 bytes, 16-byte chunks of row r at chunk position
// c ^ (r % 8), atoms 1024-byte aligned.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return sdesc(addr, lbo, sbo) | (2ull << 61);
}

// instruction descriptor: FP32 accumulate, BF16 A and B; a_mn / b_mn select
// the MN-major (transposed) reading of that operand
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn = 0, int b_mn = 0)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// instruction descriptor of kind::f8f6f4: FP32 accumulate, E4M3 A and B
// (format code 0), both K-major
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}

// The same with A read from TMEM (128 lanes = rows, K packed two BF16 per
// 32-bit column, 8 columns per K step of 16).
__device__ __forceinline__ void mma_bf16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
                 :: "r"(d_tmem), "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}

// Copy of a 128-row x 32-byte operand slice (one K step of 16 BF16) from
// shared memory (described like an MMA operand) into 8 TMEM columns.
__device__ __forceinline__ void tmem_cp_128x256b(uint32_t taddr, uint64_t sdesc_)
{
    asm volatile("tcgen05.cp.cta_group::1.128x256b [%0], %1;" :: "r"(taddr), "l"(sdesc_) : "memory");
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

// One poll of phase `parity` (the instruction may block for a short,
// hardware-chosen time, and returns as soon as the phase completes).
__device__ __forceinline__ bool bar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(saddr(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// bounded wait for phase `parity`; false if it ran out (polls, or about one
// second of SM clock)
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity)
{
    if (bar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t it = 0; it < kDenseWaitLimit; ++it) {
        if (bar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > kDenseWaitCycles) break;
    }
    return false;
}

// Tweedie factor (v - mu) max(mu, mu_min)^-p / phi of one entry with fast
// reciprocal / exp2 / log2 (relative error a few 2^-22, far below the BF16
// rounding of E that follows); p_mode 0..2 for p = 0, 1, 2, else the power.
__device__ __forceinline__ float tweedie_fast(int p_mode, float p, float phi_inv, float mu_min,
                                              float v, float mu)
{
    const float d = (v - mu) * phi_inv;
    if (p_mode == 0) return d;
    const float mc = fmaxf(mu, mu_min);
    if (p_mode == 1) return __fdividef(d, mc);
    if (p_mode == 2) return __fdividef(d, mc * mc);
    return d * exp2f(-p * __log2f(mc));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // lo at the lower address
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Row `src_row` (valid if < end) of an FP32 n x ldk matrix into row r of a
// 128 x KP K-major BF16 tile, zero padded; half h of the K range.  Returns
// the largest |x| this thread staged.
template <int KP>
__device__ __forceinline__ float stage_rows(unsigned char *tile, const float *__restrict__ X, int64_t src_row,
                                            int64_t end, int K, int ldk, int r, int h)
{
    const bool v = src_row < end;
    constexpr int kHalf = KP / 2;
    float amax = 0.f;
#pragma unroll
    for (int k = h * kHalf; k < (h + 1) * kHalf; k += 4) {
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (v && k < K) x = __ldg(reinterpret_cast<const float4 *>(X + src_row * ldk + k));
        const float a = x.x, b = k + 1 < K ? x.y : 0.f, c = k + 2 < K ? x.z : 0.f,
                    d = k + 3 < K ? x.w : 0.f;
        amax = fmaxf(amax, fmaxf(fmaxf(fabsf(a), fabsf(b)), fmaxf(fabsf(c), fabsf(d))));
        *reinterpret_cast<uint2 *>(tile + cm_off(r, k, KP)) = make_uint2(pack_bf16x2(a, b), pack_bf16x2(c, d));
    }
    return amax;
}

// four floats to E4M3 (round to nearest even, saturating), x0 at the lowest byte
__device__ __forceinline__ uint32_t pack_e4m3x4(float x0, float x1, float x2, float x3)
{
    uint16_t lo, hi;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(x1), "f"(x0));
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(x3), "f"(x2));
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

// byte offset of element (r, k) in an R x KD K-major no-swizzle 8-bit tile:
// core matrices of 8 rows x 16 bytes, adjacent along K 128 bytes apart
__device__ __forceinline__ uint32_t cm8_off(int r, int k, int KD)
{
    return (uint32_t)((r >> 3) * (KD * 8) + (k >> 4) * 128 + (r & 7) * 16 + (k & 15));
}

// The same row as stage_rows, times inv_s, into a 128 x KD E4M3 tile (KD =
// KP rounded up to 32, one MMA K step), zero padded; half h of the K range.
template <int KD>
__device__ __forceinline__ void stage_rows_e4m3(unsigned char *tile, const float *__restrict__ X,
                                                int64_t src_row, int64_t end, int K, int ldk, int r, int h,
                                                float inv_s)
{
    const bool v = src_row < end;
    constexpr int kHalf = KD / 2;
#pragma unroll
    for (int k = h * kHalf; k < (h + 1) * kHalf; k += 16) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int kk = k + 4 * q;
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (v && kk < K) x = __ldg(reinterpret_cast<const float4 *>(X + src_row * ldk + kk));
            w[q] = pack_e4m3x4(x.x * inv_s, kk + 1 < K ? x.y * inv_s : 0.f, kk + 2 < K ? x.z * inv_s : 0.f,
                               kk + 3 < K ? x.w * inv_s : 0.f);
        }
        *reinterpret_cast<uint4 *>(tile + cm8_off(r, k, KD)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Largest |x| over the CTA (x >= 0 from every thread), through `slot`
// (zero on entry, left holding the result; all threads must call).
__device__ __forceinline__ float cta_amax(float x, uint32_t *slot)
{
    const uint32_t m = __reduce_max_sync(0xffffffffu, __float_as_uint(x));   // x >= 0: bits order as values
    if ((threadIdx.x & 31) == 0) atomicMax(slot, m);
    __syncthreads();
    return __uint_as_float(*slot);
}

// E4M3 scale of a tile whose largest |x| is amax: the largest finite E4M3
// value is 448.  Returns s (x ~ s q) and sets inv_s.
__device__ __forceinline__ float e4m3_scale(float amax, float *inv_s)
{
    if (!(amax > 0.f)) {
        *inv_s = 1.f;
        return 1.f;
    }
    *inv_s = 448.f / amax;
    return amax / 448.f;
}

// 32-column chunks of a TMEM row block (this thread's lane) to an FP32 row
// in global memory: chunk c goes to half (c / 32) mod 2.
template <int KP>
__device__ __forceinline__ void drain_rows(uint32_t taddr, float *dst, bool valid, int ldk, int h)
{
#pragma unroll
    for (int c = 32 * h; c < KP; c += 64) {
        float g[32];
        tmem_ld32(taddr + (uint32_t)c, g);
        if (valid) {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
                if (c + j < ldk)
                    *reinterpret_cast<float4 *>(dst + c + j) = make_float4(g[j], g[j + 1], g[j + 2], g[j + 3]);
        }
    }
}

// One CTA of the single-pass kernel: CTA number `cta` of the launch for the
// context described by P (P may live in parameter or global memory).  With
// F8, GEMM1 (mu) reads E4M3 copies of the W and H tiles, each scaled by its
// own largest |x| / 448 (one scale per 128-row W tile and per 128-column H
// tile); mu is the FP32 product times both scales.  GEMM2 and GEMM3 stay
// BF16.
template <int KP, bool F8>
__device__ __forceinline__ void dense_grad_cta(const DenseParams &P, int cta)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr uint32_t kOpBytes = kTile * KP * 2;           // a 128 x KP BF16 tile
    constexpr uint32_t kEBytes = kTile * kTile * 2;         // a 128 x 128 BF16 tile
    constexpr int KD = KP < 32 ? 32 : KP;                   // E4M3 tile width (K step 32)
    constexpr uint32_t kOp8Bytes = F8 ? kTile * KD : 0;
    // Each tile is stored once as (row, K-dim) core matrices and read K-major
    // by one GEMM and MN-major by another.
    unsigned char *A1 = sm;                     // W tile  (m, k): GEMM1 A; GEMM3 B (MN-major)
    unsigned char *B1 = A1 + kOpBytes;          // Ht tile (n, k): GEMM1 B; GEMM2 B (MN-major)
    unsigned char *A2 = B1 + kOpBytes;          // E tile  (m, n): GEMM2 A; GEMM3 A (MN-major)
    unsigned char *A8 = A2 + kEBytes;           // E4M3 W tile (F8: GEMM1 A)
    unsigned char *B8 = A8 + kOp8Bytes;         // E4M3 Ht tile (F8: GEMM1 B)
    uint64_t *bar = reinterpret_cast<uint64_t *>(B8 + kOp8Bytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    uint32_t *amax_slot = tslot + 1;            // [0]: W tile, [1]: Ht tile (F8)

    const int tid = threadIdx.x, warp = tid >> 5;
    const int B = P.B;
    const int blk = cta / P.mtiles, mt = cta % P.mtiles;
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
        amax_slot[0] = 0u;
        amax_slot[1] = 0u;
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    // Two warps per TMEM lane quadrant: thread t works on tile row / column
    // r = t mod 128 (its quadrant's lanes) and on half h = t / 128 of the
    // columns it loads, converts or drains.
    const int r = tid & (kTile - 1), h = tid >> 7;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    uint32_t phase = 0;
    bool ok = true;

    // own rows of this M-tile: W (GEMM1 A) and W^T (GEMM3 B), BF16, zero padded
    const float wmax = stage_rows<KP>(A1, P.W, m0 + r, re, K, ldk, r, h);
    float sW = 1.f;
    if constexpr (F8) {
        float inv;
        sW = e4m3_scale(cta_amax(wmax, amax_slot), &inv);
        stage_rows_e4m3<KD>(A8, P.W, m0 + r, re, K, ldk, r, h, inv);
    }

    const uint64_t aW = F8 ? sdesc(saddr(A8), 128, KD * 8) : sdesc(saddr(A1), 128, KP * 16);
    const int ntiles = (int)((ce - cs + kTile - 1) / kTile);
    const float *__restrict__ vbase = P.V;
    const int64_t ldv = P.ldv;
    const int p_mode = P.p_mode;
    const float pw = P.p, phi_inv = P.phi_inv, mu_min = P.mu_min;
    const int64_t row = m0 + r;
    const bool rv = row < re;
    const float *__restrict__ vrow = vbase + (rv ? row : rs) * ldv;
    for (int nt = 0; nt < ntiles && ok; ++nt) {
        const int64_t n0 = cs + (int64_t)nt * kTile;
        // this thread's 64 values of V (row `row`, columns n0 + 64 h ...), all
        // requested before the column tile is staged and GEMM1 runs, so that
        // their latency overlaps both
        float vv[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) {
            const int64_t col = n0 + 64 * h + j;
            vv[j] = (rv && col < ce) ? __ldg(vrow + col) : 0.f;
        }
        // column tile: H^T rows (GEMM1 B) and H (GEMM2 B)
        const float hmax = stage_rows<KP>(B1, P.Ht, n0 + r, ce, K, ldk, r, h);
        float smu = 1.f;                          // scale of the GEMM1 product
        if constexpr (F8) {
            float inv;
            smu = sW * e4m3_scale(cta_amax(hmax, amax_slot + 1), &inv);
            stage_rows_e4m3<KD>(B8, P.Ht, n0 + r, ce, K, ldk, r, h, inv);
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();

        // GEMM1: mu (TMEM columns 0..127) = W_tile . H_tile
        if (tid == 0) {
            if constexpr (F8) {
                amax_slot[1] = 0u;                // every thread has read it (barrier above)
                const uint64_t bH = sdesc(saddr(B8), 128, KD * 8);
#pragma unroll
                for (int ks = 0; ks < KD / 32; ++ks)
                    mma_e4m3(tmem, aW + (uint64_t)(ks * 16), bH + (uint64_t)(ks * 16),
                             idesc_e4m3(kTile, kTile), ks > 0);
            } else {
                const uint64_t bH = sdesc(saddr(B1), 128, KP * 16);
#pragma unroll
                for (int ks = 0; ks < KP / 16; ++ks)
                    mma_bf16(tmem, aW + (uint64_t)(ks * 16), bH + (uint64_t)(ks * 16),
                             idesc_bf16(kTile, kTile), ks > 0);
            }
            mma_commit(bar);
        }
        ok = bar_wait(bar, phase);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) { ok = false; break; }
        fence_after();

        // epilogue: E = Tweedie factor of mu, masked to the block, BF16,
        // into E (rows m) and E^T (rows n); eight columns per 16-byte store
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int c = 64 * h + 32 * cc;
            float mu[32];
            tmem_ld32(tmem + lane_base + (uint32_t)c, mu);
#pragma unroll
            for (int j8 = 0; j8 < 32; j8 += 8) {
                uint32_t pk[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float e2[2];
#pragma unroll
                    for (int d = 0; d < 2; ++d) {
                        const int j = j8 + 2 * q + d;
                        const bool in = rv && n0 + c + j < ce;
                        const float m = F8 ? mu[j] * smu : mu[j];
                        e2[d] = in ? tweedie_fast(p_mode, pw, phi_inv, mu_min, vv[32 * cc + j], m) : 0.f;
                    }
                    pk[q] = pack_bf16x2(e2[0], e2[1]);
                }
                *reinterpret_cast<uint4 *>(A2 + cm_off(r, c + j8, kTile)) =
                    make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();

        // GEMM2: G_W (columns 128..128+KP) += E . H_tile^T   (A = E K-major,
        //        B = Ht tile read MN-major: N = k, K-dim = n)
        // GEMM3: G_H tile (columns 0..KP, over mu) = E^T . W_tile   (A = E read
        //        MN-major: M = n, K-dim = m; B = W tile read MN-major: N = k)
        if (tid == 0) {
            const uint64_t aE = sdesc(saddr(A2), 128, kTile * 16);
            const uint64_t bHt = sdesc(saddr(B1), KP * 16, 128);
            const uint64_t aEt = sdesc(saddr(A2), kTile * 16, 128);
            const uint64_t bW = sdesc(saddr(A1), KP * 16, 128);
#pragma unroll
            for (int ks = 0; ks < kTile / 16; ++ks)
                mma_bf16(tmem + kTile, aE + (uint64_t)(ks * 16), bHt + (uint64_t)(ks * 2 * KP),
                         idesc_bf16(kTile, KP, 0, 1), (nt > 0 || ks > 0));
#pragma unroll
            for (int ks = 0; ks < kTile / 16; ++ks)
                mma_bf16(tmem, aEt + (uint64_t)(ks * 2 * kTile), bW + (uint64_t)(ks * 2 * KP),
                         idesc_bf16(kTile, KP, 1, 1), ks > 0);
            mma_commit(bar);
        }
        ok = bar_wait(bar, phase);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) { ok = false; break; }
        fence_after();

        // G_H of this column tile: thread = column n0 + r, 32-column chunks
        // of TMEM split between the two halves (every lane of a warp takes
        // part in its TMEM loads; only real columns store)
        {
            const int64_t col = n0 + r;
            const bool cv = col < ce;
            float *dst = P.mtiles == 1 ? P.G + (P.I + col) * ldk
                                       : P.hpart + ((int64_t)mt * P.J + col) * ldk;
            drain_rows<KP>(tmem + lane_base, dst, cv, ldk, h);
        }
        fence_before();
        __syncthreads();
        fence_after();
    }

    if (ok) {
        // G_W: thread = row m0 + r
        drain_rows<KP>(tmem + lane_base + (uint32_t)kTile, P.G + row * ldk, rv, ldk, h);
    } else {
        if (tid == 0) atomicOr(P.err, 32);   // single-pass dense kernel
        bar_wait(bar, phase ^ 1u);   // give in-flight MMAs one more bounded chance
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"(kTmemCols) : "memory");
}


template <int KP, bool F8>
__global__ void __launch_bounds__(kDenseThreads, 1) dense_grad_kernel(const __grid_constant__ DenseParams P)
{
    dense_grad_cta<KP, F8>(P, blockIdx.x);
}

// Many contexts in one launch: context i owns CTAs [cta_start[i],
// cta_start[i + 1]) of the grid (cta_start[n] = grid size); its parameters
// are the slot `stride` bytes * i into `tab`.
template <int KP, bool F8>
__global__ void __launch_bounds__(kDenseThreads, 1)
dense_grad_batch_kernel(const unsigned char *__restrict__ tab, size_t stride, const int *__restrict__ cta_start,
                        int n)
{
    const int b = blockIdx.x;
    int lo = 0, hi = n - 1;          // last i with cta_start[i] <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(cta_start + mid) <= b) lo = mid; else hi = mid - 1;
    }
    dense_grad_cta<KP, F8>(*reinterpret_cast<const DenseParams *>(tab + (size_t)lo * stride),
                           b - __ldg(cta_start + lo));
}

// ===========================================================================
// Two-sided pipelined kernel, every item forming its own mu (K <= 256)
// ===========================================================================
//
// The form for short row pieces or parts of a single wave of items (the
// kernel after it, with E shared between the two kinds of items, for long
// pieces in several waves).  A block larger than one 128-row tile would need
// its G_H summed over the block's M-tiles.  Instead the work of a part is
// split into two kinds of items that read only the previous factors: a rows
// item owns 128 rows of W of one block and walks all the block's columns,
// accumulating G_W of those rows in TMEM; a columns item owns 128 rows of H^T
// (columns of V) and walks all the block's rows, accumulating G_H.  Each
// computes its own mu and E (GEMM1 twice per entry: 4 contractions instead
// of 3), so all of a part's items run at once, and every G row is written
// once, complete, by one CTA -- no partial sums, no atomics.
//
// Operands come from HBM already in the MMA layout: BF16 shadows of W and
// H^T cut into 128-row canonical K-major tiles per piece (kept by the update
// kernel), and V cut into 128 x 64 tiles per block, once per orientation, in
// the order the epilogue reads them (4-column FP32 or 8-column BF16 chunks,
// one 16-byte chunk per owned row, so a warp reads 512 contiguous bytes).
// Every tile is one bulk copy.  Items are assigned to CTAs round robin.
//
// One persistent CTA per SM, 10 warps:
//   warp 0               producer: the owned tile once per item, then per
//                         walked tile the other factor's 64-row tile and the
//                         V tile, into two rings of slots (bulk copies);
//   warp 1               MMA issuer: GEMM1 mu_j = A . B_j^T into one of two
//                         TMEM buffers, then GEMM2 G += E_(j-1) . B_(j-1)
//                         (B read MN-major), so GEMM1 of tile j overlaps the
//                         epilogue of tile j-1; completions via tcgen05.commit.
//                         Both warps run their loops with all 32 lanes (the
//                         descriptors stay warp-uniform, in uniform registers)
//                         and lane 0 performs each copy and MMA;
//   warps 2-9            epilogue, two warps per TMEM lane quarter (32 of the
//                         tile's 64 columns each): TMEM mu + V (shared
//                         memory) -> E (BF16, shared memory, two buffers),
//                         and after an item's last tile the G rows from TMEM
//                         to HBM.  The Tweedie power is a template parameter
//                         (p = 0, 1, 2, other), so the epilogue is straight-line.
// TMEM: mu buffers at columns 0 and 64, G at 128 .. 128 + KP, and the owned
// tile (copied from shared memory once per item with tcgen05.cp, so GEMM1
// reads A from TMEM and shared memory serves only B) in the last KP / 2
// columns.
// Padding rows and columns of every tile are zero, so mu and E are zero
// there and need no masks.
namespace two_sided_rc {

constexpr int kThreads = 320;     // warp 0 producer, warp 1 MMA, warps 2..9 epilogue
constexpr int kOwn = 128;          // owned rows per item (TMEM lanes)
constexpr int kBN = 64;            // walked rows per tile
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kGCol = 128;
constexpr int kMaxStages = 4;
constexpr int kEpiWarps = 8;       // two per TMEM lane quarter, 32 walked columns each

struct Side {
    const uint16_t *own_sh;     // BF16 shadow tiles of the owned factor
    const uint16_t *walk_sh;    // ... of the walked factor
    const unsigned char *Vt;    // V tiles in this orientation
    float *G;                   // G rows of the owned factor
    int64_t n_own, n_walk;      // I or J
    int own_tiles;              // 128-row tile slots per owned piece (items, V tiles)
    int walk_tiles;             // 64-row V tile slots per walked piece
    int own_sh64, walk_sh64;    // 64-row shadow tiles per owned / walked piece
};

struct Params {
    Side side[2];
    int B, part, KP, ldk, stages, vstages, items_a, items;
    float phi_inv, p, mu_min;
    int p_mode;
    int *err;
};

struct Bars {
    uint64_t full[kMaxStages], empty[kMaxStages];       // walked factor tiles
    uint64_t vfull[kMaxStages], vempty[kMaxStages];     // V tiles
    uint64_t mu_full[2], mu_empty[2], e_full[2], e_empty[2];
    uint64_t a_full, a_empty, g_full, g_empty;
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ void bar_init(uint64_t *b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(saddr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(saddr(b)) : "memory");
}

// Leader-only forms for warp-uniform loops: every lane executes the
// instruction with the same (uniform) operands and elect.sync picks the one
// lane that performs it (the same lane each time, the whole warp being
// active), so descriptors and addresses stay in uniform registers and each
// MMA issues in a few cycles.  The `leader` argument is unused (kept for the
// call sites' readability).
__device__ __forceinline__ void expect_tx_if(uint32_t, uint64_t *b, uint32_t bytes)
{
    asm volatile("{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
                 "@e mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n\t}"
                 :: "r"(saddr(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s_if(uint32_t, void *dst, const void *src, uint32_t bytes, uint64_t *b)
{
    asm volatile("{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
                 "@e cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n\t}"
                 :: "r"(saddr(dst)), "l"(src), "r"(bytes), "r"(saddr(b)) : "memory");
}

__device__ __forceinline__ void mma_ta_if(uint32_t, uint32_t d, uint32_t a, uint64_t bdesc, uint32_t id,
                                          uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p, e;\n\telect.sync _|e, 0xffffffff;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
                 :: "r"(d), "r"(a), "l"(bdesc), "r"(id), "r"(acc) : "memory");
}

__device__ __forceinline__ void mma_ss_if(uint32_t, uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t id,
                                          uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p, e;\n\telect.sync _|e, 0xffffffff;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(d), "l"(adesc), "l"(bdesc), "r"(id), "r"(acc) : "memory");
}

__device__ __forceinline__ void cp_if(uint32_t, uint32_t taddr, uint64_t sdesc_)
{
    asm volatile("{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
                 "@e tcgen05.cp.cta_group::1.128x256b [%0], %1;\n\t}"
                 :: "r"(taddr), "l"(sdesc_) : "memory");
}

__device__ __forceinline__ void commit_if(uint32_t, uint64_t *b)
{
    asm volatile("{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
                 "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}"
                 :: "r"(saddr(b)) : "memory");
}

// GEMM1 of one walked tile, fully unrolled for the K width KPC: mu (TMEM
// column d) = A (TMEM, tA) . B^T (walked tile at shared address aB, 128-byte
// swizzled K-major atoms of 64 rows x 128 B).  With compile-time K steps the
// descriptors are constants plus one uniform base, so each MMA issues in a
// few cycles.
template <int KPC>
__device__ __forceinline__ void gemm1_tile(uint32_t ld, uint32_t d, uint32_t tA, uint32_t aB, uint32_t id1)
{
    const uint64_t base = sdesc_sw128(aB, 16, 1024);
#pragma unroll
    for (int ks = 0; ks < KPC / 16; ++ks)
        mma_ta_if(ld, d, tA + (uint32_t)ks * 8,
                  base + (uint64_t)(((ks >> 2) * (64 * 128) + (ks & 3) * 32) >> 4), id1, ks > 0);
}

// The owned tile (shared address aA, 128-row atoms) into TMEM at tA.
template <int KPC>
__device__ __forceinline__ void own_to_tmem(uint32_t ld, uint32_t tA, uint32_t aA)
{
    const uint64_t base = sdesc_sw128(aA, 16, 1024);
#pragma unroll
    for (int ks = 0; ks < KPC / 16; ++ks)
        cp_if(ld, tA + (uint32_t)ks * 8, base + (uint64_t)(((ks >> 2) * (128 * 128) + (ks & 3) * 32) >> 4));
}

// Bounded wait by a whole warp, with one warp-uniform answer.  Every lane
// polls (control flow stays uniform, which keeps the MMA warp's operands in
// uniform registers); a completed phase costs one try_wait and one vote.
// The wait gives up (and raises the abort flag) when the CTA is aborting or
// the wait runs out.
__device__ __forceinline__ bool wait32(Bars *S, uint64_t *b, uint32_t parity)
{
    if (__all_sync(0xffffffffu, bar_try_wait(b, parity))) return true;
    const bool stop = __any_sync(0xffffffffu, *(volatile int *)&S->abort != 0);
    bool ok = !stop && bar_wait(b, parity);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && !stop && (threadIdx.x & 31) == 0) {
        // the first warp to give up records its role: 128 producer, 256 MMA, 512 epilogue
        const int warp = threadIdx.x >> 5;
        atomicOr((int *)&S->abort, warp == 0 ? 128 : warp == 1 ? 256 : 512);
    }
    return ok;
}

// Slot and phase of a ring of n slots, advanced one use at a time.
struct Ring {
    uint32_t slot = 0, phase = 0;
    __device__ __forceinline__ void next(uint32_t n)
    {
        if (++slot == n) { slot = 0; phase ^= 1u; }
    }
};

struct Item {
    int side, own_piece, walk_piece, ot, own_rows_in_tile, nj;
    int64_t own_start;
};

__device__ __forceinline__ bool decode(const Params &P, int it, Item &x)
{
    const int B = P.B;
    int side = 0, k = it;
    if (k >= P.items_a) { side = 1; k -= P.items_a; }
    const Side &Sd = P.side[side];
    const int b = k / Sd.own_tiles, ot = k % Sd.own_tiles;
    const int cpiece = (b + P.part) % B;
    x.side = side;
    x.own_piece = side == 0 ? b : cpiece;
    x.walk_piece = side == 0 ? cpiece : b;
    x.ot = ot;
    x.own_start = ((int64_t)x.own_piece * Sd.n_own) / B;
    const int64_t own_rows = ((int64_t)(x.own_piece + 1) * Sd.n_own) / B - x.own_start;
    const int64_t walk_rows = ((int64_t)(x.walk_piece + 1) * Sd.n_walk) / B -
                              ((int64_t)x.walk_piece * Sd.n_walk) / B;
    const int64_t left = own_rows - (int64_t)ot * kOwn;
    x.own_rows_in_tile = (int)(left < kOwn ? left : kOwn);
    x.nj = (int)((walk_rows + kBN - 1) / kBN);
    return left > 0;
}

template <int PM>
__device__ __forceinline__ float tweedie_pm(float p, float phi_inv, float mu_min, float v, float mu)
{
    const float d = (v - mu) * phi_inv;
    if constexpr (PM == 0) {
        return d;
    } else {
        const float mc = fmaxf(mu, mu_min);
        if constexpr (PM == 1) return __fdividef(d, mc);
        if constexpr (PM == 2) return __fdividef(d, mc * mc);
        if constexpr (PM == 3) return d * exp2f(-p * __log2f(mc));
    }
}

// Where the items' parameters come from: one context (the kernel parameter)
// or, batched, a table of contexts in global memory whose items follow one
// another (context i owns items [item_start[i], item_start[i + 1]); slots
// `stride` bytes apart).
struct Src {
    const unsigned char *tab;
    const int *item_start;
    int n;
    size_t stride;
};

template <bool BATCH>
__device__ __forceinline__ const Params &ctx_of(const Params &P0, const Src &src, int it, int &local)
{
    if constexpr (!BATCH) {
        local = it;
        return P0;
    } else {
        int lo = 0, hi = src.n - 1;          // last i with item_start[i] <= it
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(src.item_start + mid) <= it) lo = mid; else hi = mid - 1;
        }
        local = it - __ldg(src.item_start + lo);
        return *reinterpret_cast<const Params *>(src.tab + (size_t)lo * src.stride);
    }
}

// The kernel body.  P0 gives what is uniform over the launch (K width,
// ring depths); each item reads its own context's parameters.
template <typename VT, int PM, bool BATCH>
__device__ __forceinline__ void chain_body(const Params &P0, const Src src, const int total_items)
{
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    // the swizzled operand tiles need 1024-byte alignment (1 KB of slack is allocated)
    unsigned char *sm = sm_raw + ((1024u - (saddr(sm_raw) & 1023u)) & 1023u);
    const int KP = P0.KP;                                       // multiple of 64
    const int NA = KP / 64;                                     // 128-byte atoms along K
    const uint32_t a_bytes = (uint32_t)kOwn * KP * 2;           // owned tile
    const uint32_t b_bytes = (uint32_t)kBN * KP * 2;            // walked tile
    const uint32_t v_bytes = (uint32_t)kOwn * kBN * sizeof(VT); // V tile
    constexpr uint32_t e_bytes = kOwn * kBN * 2;
    unsigned char *sA = sm;
    unsigned char *sE = sA + a_bytes;                           // 2 x e_bytes
    unsigned char *sB = sE + 2 * e_bytes;                       // NS x b_bytes
    unsigned char *sV = sB + (size_t)P0.stages * b_bytes;       // NV x v_bytes
    Bars *S = reinterpret_cast<Bars *>(sV + (size_t)P0.vstages * v_bytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NS = P0.stages, NV = P0.vstages;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) { bar_init(&S->full[s], 1); bar_init(&S->empty[s], 1); }
        for (int s = 0; s < NV; ++s) { bar_init(&S->vfull[s], 1); bar_init(&S->vempty[s], kEpiWarps); }
        for (int b = 0; b < 2; ++b) {
            bar_init(&S->mu_full[b], 1); bar_init(&S->mu_empty[b], kEpiWarps);
            bar_init(&S->e_full[b], kEpiWarps); bar_init(&S->e_empty[b], 1);
        }
        bar_init(&S->a_full, 1); bar_init(&S->a_empty, 1);
        bar_init(&S->g_full, 1); bar_init(&S->g_empty, kEpiWarps);
        S->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(saddr(&S->tmem)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S->tmem;

    if (warp == 0) {
        // ---------------- producer (whole warp, lane 0 performs)
        {
            const uint32_t ld = lane == 0;
            uint32_t ic = 0;
            Ring rb, rv;
            for (int it = blockIdx.x; it < total_items; it += gridDim.x) {
                int lit;
                const Params &P = ctx_of<BATCH>(P0, src, it, lit);
                Item x;
                if (!decode(P, lit, x)) continue;
                const Side &Sd = P.side[x.side];
                if (!wait32(S, &S->a_empty, (ic & 1) ^ 1)) goto done0;
                expect_tx_if(ld, &S->a_full, a_bytes);
                {
                    // rows 0..63 and 64..127 come from two 64-row shadow tiles;
                    // in shared memory each atom holds all 128 rows
                    const uint16_t *t0 = Sd.own_sh + ((int64_t)x.own_piece * Sd.own_sh64 + 2 * x.ot) * 64 * KP;
                    for (int a = 0; a < NA; ++a) {
                        bulk_g2s_if(ld, sA + a * 16384, t0 + a * 4096, 8192, &S->a_full);
                        bulk_g2s_if(ld, sA + a * 16384 + 8192, t0 + 64 * KP + a * 4096, 8192, &S->a_full);
                    }
                }
                const unsigned char *vbase =
                    Sd.Vt + ((((int64_t)x.own_piece * P.B + x.walk_piece) * Sd.own_tiles + x.ot) *
                             Sd.walk_tiles) * (int64_t)v_bytes;
                for (int j = 0; j < x.nj; ++j) {
                    const uint32_t st = rb.slot, sv = rv.slot;
                    if (!wait32(S, &S->empty[st], rb.phase ^ 1)) goto done0;
                    expect_tx_if(ld, &S->full[st], b_bytes);
                    bulk_g2s_if(ld, sB + (size_t)st * b_bytes,
                                Sd.walk_sh + ((int64_t)x.walk_piece * Sd.walk_sh64 + j) * kBN * KP,
                                b_bytes, &S->full[st]);
                    if (!wait32(S, &S->vempty[sv], rv.phase ^ 1)) goto done0;
                    expect_tx_if(ld, &S->vfull[sv], v_bytes);
                    bulk_g2s_if(ld, sV + (size_t)sv * v_bytes, vbase + (int64_t)j * v_bytes, v_bytes, &S->vfull[sv]);
                    rb.next(NS);
                    rv.next(NV);
                }
                ++ic;
            }
        }
    done0:
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer (whole warp, lane 0 performs).  Tile
        // number tc (counted over the CTA's items) uses mu / E buffer tc % 2,
        // for the (tc / 2)-th time.
        {
            const uint32_t ld = lane == 0;
            uint32_t tc = 0, ic = 0;
            Ring r1, r2;     // walked-tile slots of GEMM1 (tile tc) and GEMM2 (tile tc - 1)
            const uint32_t id1 = idesc_bf16(kOwn, kBN);
            const uint32_t id2 = idesc_bf16(kOwn, KP, 0, 1);
            // K-major, 128-byte swizzle: 8-row groups 1024 B apart; a K step of
            // 16 entries moves 32 B inside an atom, 4 steps fill an atom, and the
            // next atom of the owned tile starts 128 rows x 128 B further
            const uint32_t aA = saddr(sA);
            const uint32_t tA = tmem + (kTmemCols - (uint32_t)KP / 2);   // owned tile in TMEM
            for (int it = blockIdx.x; it < total_items; it += gridDim.x) {
                int lit;
                const Params &P = ctx_of<BATCH>(P0, src, it, lit);
                Item x;
                if (!decode(P, lit, x)) continue;
                if (!wait32(S, &S->a_full, ic & 1)) goto done1;
                fence_after();
                // the owned tile into TMEM once per item (ordered after the
                // previous item's MMAs and before this item's: same issuing
                // thread); its shared-memory slot is free when the copies are
                switch (KP) {
                case 64: own_to_tmem<64>(ld, tA, aA); break;
                case 128: own_to_tmem<128>(ld, tA, aA); break;
                case 192: own_to_tmem<192>(ld, tA, aA); break;
                default: own_to_tmem<256>(ld, tA, aA); break;
                }
                commit_if(ld, &S->a_empty);
                for (int j = 0; j <= x.nj; ++j) {
                    if (j < x.nj) {
                        const uint32_t st = r1.slot;
                        const int b = (int)(tc & 1);
                        if (!wait32(S, &S->full[st], r1.phase)) goto done1;
                        if (!wait32(S, &S->mu_empty[b], ((tc >> 1) & 1) ^ 1)) goto done1;
                        fence_after();
                        const uint32_t aB = saddr(sB + (size_t)st * b_bytes);
                        const uint32_t dmu = tmem + (uint32_t)(b * kBN);
                        switch (KP) {
                        case 64: gemm1_tile<64>(ld, dmu, tA, aB, id1); break;
                        case 128: gemm1_tile<128>(ld, dmu, tA, aB, id1); break;
                        case 192: gemm1_tile<192>(ld, dmu, tA, aB, id1); break;
                        default: gemm1_tile<256>(ld, dmu, tA, aB, id1); break;
                        }
                        commit_if(ld, &S->mu_full[b]);
                        ++tc;
                        r1.next(NS);
                    }
                    if (j > 0) {
                        // GEMM2 of tile j - 1 (tile number tp)
                        const uint32_t tp = j < x.nj ? tc - 2 : tc - 1;
                        const int b = (int)(tp & 1);
                        const uint32_t st = r2.slot;
                        if (!wait32(S, &S->e_full[b], (tp >> 1) & 1)) goto done1;
                        if (j == 1 && !wait32(S, &S->g_empty, (ic & 1) ^ 1)) goto done1;
                        fence_after();
                        // A = E (K-major, one atom of 64 walked columns); B = the
                        // walked tile read MN-major: MN atoms (64 entries of k)
                        // 64 rows x 128 B apart (LBO), 8-row K groups 1024 B apart
                        // (SBO), a K step of 16 walked rows = 2048 B
                        const uint64_t dE = sdesc_sw128(saddr(sE + b * e_bytes), 16, 1024);
                        const uint64_t dBt = sdesc_sw128(saddr(sB + (size_t)st * b_bytes), kBN * 128, 1024);
#pragma unroll
                        for (int ks = 0; ks < kBN / 16; ++ks)
                            mma_ss_if(ld, tmem + kGCol, dE + (uint64_t)(ks * 2), dBt + (uint64_t)(ks * 128),
                                      id2, (j > 1 || ks > 0));
                        commit_if(ld, &S->e_empty[b]);
                        commit_if(ld, &S->empty[st]);
                        r2.next(NS);
                    }
                }
                commit_if(ld, &S->g_full);
                ++ic;
            }
        }
    done1:
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 2..9): TMEM lane quarter warp % 4,
        // walked columns 32 h .. 32 h + 31 of each tile, h = (warp - 2) / 4
        const int q = warp & 3, hc = (warp - 2) >> 2;
        const int rho = 32 * q + lane;                      // owned row in the tile
        const int c = 32 * hc;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        uint32_t tc = 0, ic = 0;
        Ring rv;
        for (int it = blockIdx.x; it < total_items; it += gridDim.x) {
            int lit;
            const Params &P = ctx_of<BATCH>(P0, src, it, lit);
            Item x;
            if (!decode(P, lit, x)) continue;
            const Side &Sd = P.side[x.side];
            const float pp = P.p, phi_inv = P.phi_inv, mu_min = P.mu_min;
            for (int j = 0; j < x.nj; ++j, ++tc, rv.next(NV)) {
                const int b = (int)(tc & 1);
                const uint32_t sv = rv.slot;
                const uint32_t ph = (tc >> 1) & 1;
                if (!wait32(S, &S->vfull[sv], rv.phase)) goto done2;
                if (!wait32(S, &S->mu_full[b], ph)) goto done2;
                if (!wait32(S, &S->e_empty[b], ph ^ 1)) goto done2;
                fence_after();
                const unsigned char *vt = sV + (size_t)sv * v_bytes;
                unsigned char *eb = sE + b * e_bytes;
                float mu[32];
                tmem_ld32(tmem + lane_base + (uint32_t)(b * kBN + c), mu);
                float v[32];
                if constexpr (sizeof(VT) == 4) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float4 w = *reinterpret_cast<const float4 *>(
                            vt + ((size_t)((c >> 2) + i) * kOwn + rho) * 16);
                        v[4 * i] = w.x; v[4 * i + 1] = w.y; v[4 * i + 2] = w.z; v[4 * i + 3] = w.w;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const uint4 w = *reinterpret_cast<const uint4 *>(
                            vt + ((size_t)((c >> 3) + i) * kOwn + rho) * 16);
                        const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            v[8 * i + 2 * h] = __uint_as_float(u[h] << 16);
                            v[8 * i + 2 * h + 1] = __uint_as_float(u[h] & 0xffff0000u);
                        }
                    }
                }
                uint32_t pk[16];
#pragma unroll
                for (int h = 0; h < 16; ++h) {
                    const float e0 = tweedie_pm<PM>(pp, phi_inv, mu_min, v[2 * h], mu[2 * h]);
                    const float e1 = tweedie_pm<PM>(pp, phi_inv, mu_min, v[2 * h + 1], mu[2 * h + 1]);
                    __nv_bfloat162 t2 = __floats2bfloat162_rn(e0, e1);
                    pk[h] = *reinterpret_cast<uint32_t *>(&t2);
                }
                // E (owned row rho, walked columns c..c+31): row rho of the
                // 128-byte-swizzled atom column, chunk (c/8 + g) ^ (rho % 8)
#pragma unroll
                for (int g = 0; g < 4; ++g)
                    *reinterpret_cast<uint4 *>(eb + rho * 128 + ((((c >> 3) + g) ^ (rho & 7)) << 4)) =
                        make_uint4(pk[4 * g], pk[4 * g + 1], pk[4 * g + 2], pk[4 * g + 3]);
                fence_async_smem();
                fence_before();
                __syncwarp();
                if (lane == 0) {
                    bar_arrive(&S->vempty[sv]);
                    bar_arrive(&S->mu_empty[b]);
                    bar_arrive(&S->e_full[b]);
                }
            }
            // the item's G rows: this warp's lane quarter, every other 32-column chunk
            if (!wait32(S, &S->g_full, ic & 1)) goto done2;
            fence_after();
            {
                const bool rv = rho < x.own_rows_in_tile;
                float *dst = Sd.G + (x.own_start + (int64_t)x.ot * kOwn + rho) * P.ldk;
                for (int cc = 32 * hc; cc < KP; cc += 64) {
                    float g[32];
                    tmem_ld32(tmem + lane_base + kGCol + (uint32_t)cc, g);
                    if (rv) {
#pragma unroll
                        for (int h = 0; h < 32; h += 4)
                            if (cc + h < P.ldk)
                                *reinterpret_cast<float4 *>(dst + cc + h) = make_float4(g[h], g[h + 1], g[h + 2], g[h + 3]);
                    }
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) bar_arrive(&S->g_empty);
            ++ic;
        }
    done2:
        __syncwarp();
    }

    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x == 0 && S->abort) {                      // two-sided kernel (+ role)
        if constexpr (BATCH) {
            for (int i = 0; i < src.n; ++i)
                atomicOr(reinterpret_cast<const Params *>(src.tab + (size_t)i * src.stride)->err, 64 | S->abort);
        } else {
            atomicOr(P0.err, 64 | S->abort);
        }
    }
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"(kTmemCols) : "memory");
}

template <typename VT, int PM>
__global__ void __launch_bounds__(kThreads, 1) chain_kernel(const __grid_constant__ Params P)
{
    chain_body<VT, PM, false>(P, Src{nullptr, nullptr, 1, 0}, P.items);
}

// Many contexts of one K width, V type and power in one persistent launch.
template <typename VT, int PM>
__global__ void __launch_bounds__(kThreads, 1)
chain_batch_kernel(const unsigned char *tab, size_t stride, const int *item_start, int n)
{
    chain_body<VT, PM, true>(*reinterpret_cast<const Params *>(tab), Src{tab, item_start, n, stride},
                             __ldg(item_start + n));
}

}  // namespace two_sided_rc

// ===========================================================================
// Two-sided pipelined kernel (blocks of any size, K <= 256)
// ===========================================================================
//
// A block larger than one 128-row tile would need its G_H summed over the
// block's M-tiles.  Instead the work of a part is split into two kinds of
// items.  A rows item owns 128 rows of W of one block and walks all the
// block's columns in 64-column tiles: mu = W H^T, E, and G_W += E H in TMEM;
// each E tile (BF16, the image the epilogue built in shared memory) also
// goes to HBM, one bulk store.  A columns item owns 256 rows of H^T (columns
// of V) in two 128-row accumulators; once every rows item of its block has
// stored its E, it walks the block's rows: G_H += E^T W, one contraction,
// each W tile serving both accumulators.  mu and E are formed once per entry (the three
// contractions the gradient needs), and every G row is written once,
// complete, by one CTA: no partial sums, no atomics on data.  E is formed
// without its 1 / phi factor, which multiplies G as G is written.
//
// Items are claimed in order from a counter in HBM (the rows items of every
// block first, then the columns items), and a columns item waits (bounded)
// for a per-block count of finished rows items.  A claimed item waits only
// for items claimed before it, all held by running CTAs, so a launch
// finishes however many of its CTAs the GPU runs at a time.  The last CTA to
// finish sets the counters back to zero for the next launch.
//
// Operands come from HBM already in the MMA layout: BF16 shadows of W and
// H^T cut into 64-row swizzled K-major tiles per piece (kept by the update
// kernel), and V cut into 128 x 64 tiles per block, in the order the
// epilogue reads them (4-column FP32 or 8-column BF16 chunks, one 16-byte
// chunk per owned row, so a warp reads 512 contiguous bytes).  Every tile is
// one bulk copy.
//
// One persistent CTA per SM, 11 warps:
//   warp 0     producer: claims the items and hands them on through a
//              two-slot queue in shared memory; rows item: the owned tile,
//              then per walked tile the H^T tile (a ring of 2 to 6 slots);
//              columns item: per 64 W rows one stage of the W tile and the
//              two 64 x 64 halves of E that cover the owned columns.  A CTA
//              claims all its rows items before its first columns item, so
//              at that point (its last rows item complete) the columns
//              stages take over the whole of shared memory: a ring of 2 to
//              6 stages;
//   warp 1     MMA issuer: rows item: GEMM1 mu_j = A . B_j^T into one of two
//              TMEM buffers, then GEMM2 G += E_(j-1) . B_(j-1) (B read
//              MN-major), so GEMM1 of tile j overlaps the epilogue of tile
//              j-1; columns item: G += E^T . W, both operands read MN-major.
//              Completions via tcgen05.commit.  Both warps run their loops
//              with all 32 lanes (the descriptors stay warp-uniform, in
//              uniform registers) and one elected lane performs each copy
//              and MMA;
//   warps 2-9  epilogue, two warps per TMEM lane quarter (32 of the tile's
//              64 columns each): TMEM mu + V -> E (BF16, into an E buffer),
//              V read from HBM straight into registers two tiles ahead; and
//              after an item's last tile the
//              G rows from TMEM to HBM.  The Tweedie power is a template
//              parameter (p = 0, 1, 2, other), so the epilogue is
//              straight-line;
//   warp 10    E stores: each E tile of a rows item to HBM (one bulk copy
//              from its E buffer), and after the item the count its block's
//              columns items wait for.  The tensor core queues only a few
//              MMAs, so this work stays off the MMA warp.
// TMEM, rows item: mu buffers at columns 0 and 64, G at 128 .. 128 + KP, and
// the owned tile (copied from shared memory once per item with tcgen05.cp,
// so GEMM1 reads A from TMEM and shared memory serves only B) in the last
// KP / 2 columns; columns item: its two accumulators at columns 0 and 256.
// Padding rows and columns of every tile are zero, so mu and E are zero
// there and need no masks.
namespace two_sided {

constexpr int kThreads = 352;     // warp 0 producer, warp 1 MMA, warps 2..9 epilogue, warp 10 E stores
constexpr int kOwn = 128;          // owned rows per rows item (TMEM lanes)
constexpr int kOwnH = 256;         // owned rows per columns item (two accumulators)
constexpr int kBN = 64;            // walked rows per tile
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kGCol = 128;
constexpr int kMaxStages = 6;
constexpr int kEpiWarps = 8;       // two per TMEM lane quarter, 32 walked columns each
constexpr int kQueue = 2;          // claimed items on their way from the producer
constexpr int kMaxHStages = 6;     // columns-item stages (W tile + E halves)
constexpr uint32_t kEBytes = kOwn * kBN * 2;    // one E tile, BF16
constexpr uint32_t kStgBytes = kOwn * 64 * 4;     // G staging: 128 rows x 64 FP32 columns

struct Side {
    const uint16_t *own_sh;     // BF16 shadow tiles of the owned factor (rows items)
    const uint16_t *walk_sh;    // ... of the walked factor
    const unsigned char *Vt;    // V tiles (rows items)
    float *G;                   // G rows of the owned factor
    int64_t n_own, n_walk;      // I or J
    int own_tiles;              // 128-row tile slots per owned piece (items, V tiles)
    int walk_tiles;             // 64-row V tile slots per walked piece
    int own_sh64, walk_sh64;    // 64-row shadow tiles per owned / walked piece
};

struct Params {
    Side side[2];
    uint16_t *Et;               // the part's E tiles: slot (b * side[0].own_tiles + t) * et_cols + j
                                // holds the 128 x 64 BF16 image of W tile t x H^T tile j of block b
    int *sync;                  // [0] items claimed, [1] CTAs finished, [2 + b] rows items of
                                // block b whose E is in HBM; all zero between launches
    int et_cols;                // E slots per W tile (4 x the 256-row columns items per piece)
    int hwide, ht1, ht2;        // blocks 0 .. hwide - 1: 256-row columns items (ht2 per piece), the
                                // rest 128-row ones (ht1 per piece)
    int B, part, KP, ldk, stages, hstages, items_a, items;
    int bars_off;               // shared-memory offset of the barriers (past both layouts)
    float phi_inv, p, mu_min;
    int p_mode;
    int *err;
};

struct Bars {
    uint64_t full[kMaxStages], empty[kMaxStages];       // walked factor tiles
    uint64_t mu_full[2], mu_empty[2], e_full[2], e_empty[2];
    uint64_t a_full, a_empty, g_full, g_empty;
    uint64_t hfull[kMaxHStages], hempty[kMaxHStages];   // columns-item stages
    uint64_t q_full[kQueue], q_empty[kQueue];           // the item queue
    uint64_t stg_full, stg_empty;                       // G staging passes (epilogue warps)
    int q_item[kQueue];
    int items_done;             // epilogue warps done with an item (its MMAs, reads and drain)
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ void bar_init(uint64_t *b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(saddr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(saddr(b)) : "memory");
}

// Leader-only forms for warp-uniform loops: every lane executes the
// instruction with the same (uniform) operands and elect.sync picks the one
// lane that performs it (the same lane each time, the whole warp being
// active), so descriptors and addresses stay in uniform registers and each
// MMA issues in a few cycles.  The `leader` argument is unused (kept for the
// call sites' readability).
__device__ __forceinline__ void expect_tx_if(uint32_t, uint64_t *b, uint32_t bytes)
{
    asm volatile("{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
                 "@e mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n\t}"
                 :: "r"(saddr(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s_if(uint32_t, void *dst, const void *src, uint32_t bytes, uint64_t *b)
{
    asm volatile("{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
                 "@e cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n\t}"
                 :: "r"(saddr(dst)), "l"(src), "r"(bytes), "r"(saddr(b)) : "memory");
}

// L2 prefetch of `bytes` (a multiple of 16) from a 16-byte aligned address
__device__ __forceinline__ void prefetch_l2_if(const void *src, uint32_t bytes)
{
    asm volatile("{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
                 "@e cp.async.bulk.prefetch.L2.global [%0], %1;\n\t}"
                 :: "l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mma_ta_if(uint32_t, uint32_t d, uint32_t a, uint64_t bdesc, uint32_t id,
                                          uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p, e;\n\telect.sync _|e, 0xffffffff;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
                 :: "r"(d), "r"(a), "l"(bdesc), "r"(id), "r"(acc) : "memory");
}

__device__ __forceinline__ void mma_ss_if(uint32_t, uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t id,
                                          uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p, e;\n\telect.sync _|e, 0xffffffff;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(d), "l"(adesc), "l"(bdesc), "r"(id), "r"(acc) : "memory");
}

__device__ __forceinline__ void cp_if(uint32_t, uint32_t taddr, uint64_t sdesc_)
{
    asm volatile("{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
                 "@e tcgen05.cp.cta_group::1.128x256b [%0], %1;\n\t}"
                 :: "r"(taddr), "l"(sdesc_) : "memory");
}

__device__ __forceinline__ void commit_if(uint32_t, uint64_t *b)
{
    asm volatile("{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
                 "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}"
                 :: "r"(saddr(b)) : "memory");
}

// GEMM1 of one walked tile, fully unrolled for the K width KPC: mu (TMEM
// column d) = A (TMEM, tA) . B^T (walked tile at shared address aB, 128-byte
// swizzled K-major atoms of 64 rows x 128 B).  With compile-time K steps the
// descriptors are constants plus one uniform base, so each MMA issues in a
// few cycles.
template <int KPC>
__device__ __forceinline__ void gemm1_tile(uint32_t ld, uint32_t d, uint32_t tA, uint32_t aB, uint32_t id1)
{
    const uint64_t base = sdesc_sw128(aB, 16, 1024);
#pragma unroll
    for (int ks = 0; ks < KPC / 16; ++ks)
        mma_ta_if(ld, d, tA + (uint32_t)ks * 8,
                  base + (uint64_t)(((ks >> 2) * (64 * 128) + (ks & 3) * 32) >> 4), id1, ks > 0);
}

// The owned tile (shared address aA, 128-row atoms) into TMEM at tA.
template <int KPC>
__device__ __forceinline__ void own_to_tmem(uint32_t ld, uint32_t tA, uint32_t aA)
{
    const uint64_t base = sdesc_sw128(aA, 16, 1024);
#pragma unroll
    for (int ks = 0; ks < KPC / 16; ++ks)
        cp_if(ld, tA + (uint32_t)ks * 8, base + (uint64_t)(((ks >> 2) * (128 * 128) + (ks & 3) * 32) >> 4));
}

// Bounded wait by a whole warp, with one warp-uniform answer.  Every lane
// polls (control flow stays uniform, which keeps the MMA warp's operands in
// uniform registers); a completed phase costs one try_wait and one vote.
// The wait gives up (and raises the abort flag) when the CTA is aborting or
// the wait runs out.
__device__ __forceinline__ bool wait32(Bars *S, uint64_t *b, uint32_t parity)
{
    if (__all_sync(0xffffffffu, bar_try_wait(b, parity))) return true;
    const bool stop = __any_sync(0xffffffffu, *(volatile int *)&S->abort != 0);
    bool ok = !stop && bar_wait(b, parity);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && !stop && (threadIdx.x & 31) == 0) {
        // the first warp to give up records its role: 128 producer, 256 MMA, 512 epilogue
        const int warp = threadIdx.x >> 5;
        atomicOr((int *)&S->abort, warp == 0 ? 128 : warp == 1 ? 256 : 512);
    }
    return ok;
}

// 16 bytes of data read once (no L1 allocation)
__device__ __forceinline__ uint4 ldg_stream(const void *p)
{
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}

// Non-blocking test of phase `parity`.
__device__ __forceinline__ bool bar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(saddr(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Two waits with one vote when both phases are already
// complete (the common case in the steady pipeline), else one by one.
__device__ __forceinline__ bool wait32x2(Bars *S, uint64_t *a, uint32_t pa, uint64_t *b, uint32_t pb)
{
    if (__all_sync(0xffffffffu, bar_test(a, pa) && bar_test(b, pb))) return true;
    return wait32(S, a, pa) && wait32(S, b, pb);
}

// Bounded wait of the producer warp until another CTA's count in HBM
// reaches `target` (acquire), then a proxy fence so that the bulk copies
// issued after it read what the counted warps stored.  Gives up (abort
// role 1024) after about a second of SM clock, or when the CTA is aborting.
__device__ __forceinline__ bool wait_count(Bars *S, const int *cnt, int target)
{
    int ok = 1;
    if ((threadIdx.x & 31) == 0) {
        const long long t0 = clock64();
        for (uint32_t it = 0;; ++it) {
            int v;
            asm volatile("ld.acquire.gpu.b32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
            if (v >= target) break;
            if (*(volatile int *)&S->abort != 0) { ok = 0; break; }
            if (it >= kDenseWaitLimit || clock64() - t0 > kDenseWaitCycles) {
                atomicOr((int *)&S->abort, 1024);
                ok = 0;
                break;
            }
            __nanosleep(128);
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    asm volatile("fence.proxy.async.global;" ::: "memory");
    return ok != 0;
}

// Slot and phase of a ring of n slots, advanced one use at a time.
struct Ring {
    uint32_t slot = 0, phase = 0;
    __device__ __forceinline__ void next(uint32_t n)
    {
        if (++slot == n) { slot = 0; phase ^= 1u; }
    }
};

struct Item {
    int side, block, own_piece, walk_piece, ot, own_rows_in_tile, nj;
    int rows_per, row0;         // owned rows of the item (128 or 256) and its first row in the piece
    bool rl;                    // a rows item
    int64_t own_start;
};

// Item k of one side of one context: block b pairs row piece b with column
// piece (b + part) mod B; tile ot of the owned piece.  Rows items: 128 rows,
// own_tiles per block.  Columns items: 256 rows (ht2 per block) in blocks
// 0 .. hwide - 1, then 128 rows (ht1 per block).
__device__ __forceinline__ bool decode(const Params &P, int side, int k, Item &x)
{
    const int B = P.B;
    const Side &Sd = P.side[side];
    int b, ot, rows_per = kOwn;
    x.rl = side == 0;
    if (x.rl) {
        b = k / Sd.own_tiles;
        ot = k % Sd.own_tiles;
    } else if (k < P.hwide * P.ht2) {
        b = k / P.ht2;
        ot = k % P.ht2;
        rows_per = kOwnH;
    } else {
        k -= P.hwide * P.ht2;
        b = P.hwide + k / P.ht1;
        ot = k % P.ht1;
    }
    x.rows_per = rows_per;
    x.row0 = ot * rows_per;
    const int cpiece = (b + P.part) % B;
    x.side = side;
    x.block = b;
    x.own_piece = side == 0 ? b : cpiece;
    x.walk_piece = side == 0 ? cpiece : b;
    x.ot = ot;
    x.own_start = ((int64_t)x.own_piece * Sd.n_own) / B;
    const int64_t own_rows = ((int64_t)(x.own_piece + 1) * Sd.n_own) / B - x.own_start;
    const int64_t walk_rows = ((int64_t)(x.walk_piece + 1) * Sd.n_walk) / B -
                              ((int64_t)x.walk_piece * Sd.n_walk) / B;
    const int64_t left = own_rows - (int64_t)x.row0;
    x.own_rows_in_tile = (int)(left < rows_per ? left : rows_per);
    x.nj = (int)((walk_rows + kBN - 1) / kBN);
    return left > 0;
}

// (v - mu) max(mu, mu_min)^-p; the 1 / phi goes on G when it is written
template <int PM>
__device__ __forceinline__ float tweedie_pm(float p, float mu_min, float v, float mu)
{
    const float d = v - mu;
    if constexpr (PM == 0) {
        return d;
    } else {
        const float mc = fmaxf(mu, mu_min);
        if constexpr (PM == 1) return __fdividef(d, mc);
        if constexpr (PM == 2) return __fdividef(d, mc * mc);
        if constexpr (PM == 3) return d * exp2f(-p * __log2f(mc));
    }
}

// Where the items' parameters come from: one context (the kernel parameter)
// or, batched, a table of contexts in global memory (slots `stride` bytes
// apart).  Batched, the rows items of every context come first, context i
// owning [wstart[i], wstart[i + 1]), then the columns items, context i
// owning [hstart[i], hstart[i + 1]) of those.
struct Src {
    const unsigned char *tab;
    const int *wstart, *hstart;
    int n;
    size_t stride;
};

template <bool BATCH>
__device__ __forceinline__ const Params &item_of(const Params &P0, const Src &src, int it, int &side, int &k)
{
    if constexpr (!BATCH) {
        side = it >= P0.items_a ? 1 : 0;
        k = side ? it - P0.items_a : it;
        return P0;
    } else {
        const int nw = __ldg(src.wstart + src.n);
        const int *pre = src.wstart;
        int r = it;
        bool first = true;
        if (r >= nw) {
            pre = src.hstart;
            r -= nw;
            first = false;
        }
        int lo = 0, hi = src.n - 1;          // last i with pre[i] <= r
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(pre + mid) <= r) lo = mid; else hi = mid - 1;
        }
        k = r - __ldg(pre + lo);
        const Params &P = *reinterpret_cast<const Params *>(src.tab + (size_t)lo * src.stride);
        side = first ? (k >= P.items_a ? 1 : 0) : 1;
        if (first && side == 1) k -= P.items_a;
        return P;
    }
}

// Next claimed item from the queue (MMA and epilogue warps); -1 at the end,
// -2 if the wait gave up.
__device__ __forceinline__ int take_item(Bars *S, Ring &rq)
{
    if (!wait32(S, &S->q_full[rq.slot], rq.phase)) return -2;
    const int it = *(volatile int *)&S->q_item[rq.slot];
    __syncwarp();
    if ((threadIdx.x & 31) == 0) bar_arrive(&S->q_empty[rq.slot]);
    rq.next(kQueue);
    return it;
}

// The kernel body.  P0 gives what is uniform over the launch (K width,
// ring depths, the claim counters); each item reads its own context's
// parameters.
template <typename VT, int PM, bool BATCH>
__device__ __forceinline__ void chain_body(const Params &P0, const Src src, const int total_items)
{
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    // the swizzled operand tiles need 1024-byte alignment (1 KB of slack is allocated)
    unsigned char *sm = sm_raw + ((1024u - (saddr(sm_raw) & 1023u)) & 1023u);
    const int KP = P0.KP;                                       // multiple of 64
    const int NA = KP / 64;                                     // 128-byte atoms along K
    const uint32_t a_bytes = (uint32_t)kOwn * KP * 2;           // owned tile
    const uint32_t b_bytes = (uint32_t)kBN * KP * 2;            // walked tile
    const uint32_t v_bytes = (uint32_t)kOwn * kBN * sizeof(VT); // V tile (HBM)
    unsigned char *sA = sm;
    unsigned char *sE = sA + a_bytes;                           // 2 x kEBytes
    unsigned char *sB = sE + 2 * kEBytes;                       // NS x b_bytes
    Bars *S = reinterpret_cast<Bars *>(sm + P0.bars_off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NS = P0.stages, NH = P0.hstages;
    const uint32_t h_bytes = b_bytes + 2 * kEBytes;             // columns-item stage: W tile, 4 E halves
    unsigned char *sStgH = sm + (size_t)NH * h_bytes;           // columns items' G staging

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) { bar_init(&S->full[s], 1); bar_init(&S->empty[s], 1); }
        for (int b = 0; b < 2; ++b) {
            bar_init(&S->mu_full[b], 1); bar_init(&S->mu_empty[b], kEpiWarps);
            bar_init(&S->e_full[b], kEpiWarps); bar_init(&S->e_empty[b], 2);   // GEMM2 done, E stored
        }
        bar_init(&S->a_full, 1); bar_init(&S->a_empty, 1);
        bar_init(&S->g_full, 1); bar_init(&S->g_empty, kEpiWarps);
        for (int s = 0; s < NH; ++s) { bar_init(&S->hfull[s], 1); bar_init(&S->hempty[s], 1); }
        for (int s = 0; s < kQueue; ++s) { bar_init(&S->q_full[s], 1); bar_init(&S->q_empty[s], 2 + kEpiWarps); }
        bar_init(&S->stg_full, kEpiWarps); bar_init(&S->stg_empty, kEpiWarps);
        S->abort = 0;
        S->items_done = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(saddr(&S->tmem)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S->tmem;

    // E buffer use u (a rows-item tile) takes buffer u % 2 for the (u / 2)-th
    // time; item n completes phase n of g_full.
    if (warp == 0) {
        // ---------------- producer (whole warp, one elected lane performs)
        {
            const uint32_t ld = lane == 0;
            uint32_t iw = 0, ic = 0;
            bool hphase = false;
            Ring rb, rq, rh;
            for (;;) {
                if (!wait32(S, &S->q_empty[rq.slot], rq.phase ^ 1)) goto done0;
                int it = 0;
                if (lane == 0) it = atomicAdd(P0.sync, 1);
                it = __shfl_sync(0xffffffffu, it, 0);
                if (it >= total_items) it = -1;
                if (lane == 0) {
                    S->q_item[rq.slot] = it;
                    bar_arrive(&S->q_full[rq.slot]);
                }
                __syncwarp();
                rq.next(kQueue);
                if (it < 0) break;
                int side, k;
                const Params &P = item_of<BATCH>(P0, src, it, side, k);
                Item x;
                if (!decode(P, side, k, x)) continue;
                const Side &Sd = P.side[side];
                if (x.rl) {
                    // rows item: the owned W tile, then the walked H^T tiles
                    // (and L2 prefetches of the V tiles)
                    if (hphase) {                     // cannot happen: rows items are claimed first
                        atomicOr((int *)&S->abort, 128);
                        goto done0;
                    }
                    if (!wait32(S, &S->a_empty, (iw & 1) ^ 1)) goto done0;
                    expect_tx_if(ld, &S->a_full, a_bytes);
                    {
                        // rows 0..63 and 64..127 come from two 64-row shadow tiles;
                        // in shared memory each atom holds all 128 rows
                        const uint16_t *t0 = Sd.own_sh + ((int64_t)x.own_piece * Sd.own_sh64 + 2 * x.ot) * 64 * KP;
                        for (int a = 0; a < NA; ++a) {
                            bulk_g2s_if(ld, sA + a * 16384, t0 + a * 4096, 8192, &S->a_full);
                            bulk_g2s_if(ld, sA + a * 16384 + 8192, t0 + 64 * KP + a * 4096, 8192, &S->a_full);
                        }
                    }
                    ++iw;
                    // with each walked tile, an L2 prefetch of its V tile: the
                    // epilogue's register loads, two tiles ahead, then hit L2
                    const unsigned char *vbase =
                        Sd.Vt + ((((int64_t)x.own_piece * P.B + x.walk_piece) * Sd.own_tiles + x.ot) *
                                 Sd.walk_tiles) * (int64_t)v_bytes;
                    for (int j = 0; j < x.nj; ++j) {
                        const uint32_t st = rb.slot;
                        if (!wait32(S, &S->empty[st], rb.phase ^ 1)) goto done0;
                        expect_tx_if(ld, &S->full[st], b_bytes);
                        bulk_g2s_if(ld, sB + (size_t)st * b_bytes,
                                    Sd.walk_sh + ((int64_t)x.walk_piece * Sd.walk_sh64 + j) * kBN * KP,
                                    b_bytes, &S->full[st]);
                        prefetch_l2_if(vbase + (int64_t)j * v_bytes, v_bytes);
                        rb.next(NS);
                    }
                } else {
                    // columns item: once the block's rows items have stored E,
                    // per 64 W rows the W tile and the E halves of the owned
                    // columns (E tiles 4 ot .. 4 ot + 3 of each W tile)
                    if (!hphase) {
                        // the first one: once every earlier (rows) item's G is
                        // complete, their MMAs, copies and epilogue reads of
                        // shared memory are all done.  A count, not a wait on
                        // g_full: the producer may be two items ahead, where a
                        // phase parity would already read as complete.
                        int ok = 1;
                        if (lane == 0) {
                            const long long t0 = clock64();
                            while (*(volatile int *)&S->items_done < kEpiWarps * (int)ic) {
                                if (*(volatile int *)&S->abort != 0) { ok = 0; break; }
                                if (clock64() - t0 > kDenseWaitCycles) {
                                    atomicOr((int *)&S->abort, 128);
                                    ok = 0;
                                    break;
                                }
                            }
                        }
                        if (!__shfl_sync(0xffffffffu, ok, 0)) goto done0;
                        hphase = true;
                    }
                    const int64_t wrows = ((int64_t)(x.walk_piece + 1) * Sd.n_walk) / P.B -
                                          ((int64_t)x.walk_piece * Sd.n_walk) / P.B;
                    const int target = (int)((wrows + kOwn - 1) / kOwn);
                    if (!wait_count(S, P.sync + 2 + x.block, target)) goto done0;
                    const uint16_t *e0 =
                        P.Et + (((int64_t)x.block * P.side[0].own_tiles) * P.et_cols + x.row0 / kBN) * (kEBytes / 2);
                    const int nq = x.rows_per / kBN;          // E tiles across the owned rows (4 or 2)
                    const uint32_t stage_tx = b_bytes + (uint32_t)nq * (kEBytes / 2);
                    // stage s: rows 64 (s % 2) .. + 63 of W tile s / 2, in each
                    // of the nq E tiles (8 KB each, consecutive slots)
                    auto e_half = [&](int st_, int q) {
                        return e0 + (int64_t)(st_ >> 1) * P.et_cols * (kEBytes / 2) + q * (kEBytes / 2) +
                               (st_ & 1) * (kEBytes / 4);
                    };
                    // the E halves of the first stages into L2 now, later ones a
                    // ring's length ahead (they come from HBM)
                    for (int s = 0; s < NH && s < x.nj; ++s)
                        for (int q = 0; q < nq; ++q) prefetch_l2_if(e_half(s, q), kEBytes / 2);
                    for (int s = 0; s < x.nj; ++s) {
                        const uint32_t sh = rh.slot;
                        unsigned char *stage = sm + (size_t)sh * h_bytes;
                        if (s + NH < x.nj)
                            for (int q = 0; q < nq; ++q) prefetch_l2_if(e_half(s + NH, q), kEBytes / 2);
                        if (!wait32(S, &S->hempty[sh], rh.phase ^ 1)) goto done0;
                        expect_tx_if(ld, &S->hfull[sh], stage_tx);
                        bulk_g2s_if(ld, stage, Sd.walk_sh + ((int64_t)x.walk_piece * Sd.walk_sh64 + s) * kBN * KP,
                                    b_bytes, &S->hfull[sh]);
                        for (int q = 0; q < nq; ++q)
                            bulk_g2s_if(ld, stage + b_bytes + q * (kEBytes / 2), e_half(s, q), kEBytes / 2,
                                        &S->hfull[sh]);
                        rh.next(NH);
                    }
                }
                ++ic;
            }
        }
    done0:
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer (whole warp, one elected lane performs)
        {
            const uint32_t ld = lane == 0;
            uint32_t iw = 0, ic = 0, tw = 0, te = 0;     // rows items, items, mu uses, E uses
            Ring r1, r2, rq, rh; // walked-tile slots of GEMM1 (tile j) and GEMM2 (tile j - 1); stages
            const uint32_t id1 = idesc_bf16(kOwn, kBN);
            const uint32_t id2 = idesc_bf16(kOwn, KP, 0, 1);
            const uint32_t id3 = idesc_bf16(kOwn, KP, 1, 1);
            // K-major, 128-byte swizzle: 8-row groups 1024 B apart; a K step of
            // 16 entries moves 32 B inside an atom, 4 steps fill an atom, and the
            // next atom of the owned tile starts 128 rows x 128 B further
            const uint32_t aA = saddr(sA);
            const uint32_t tA = tmem + (kTmemCols - (uint32_t)KP / 2);   // owned tile in TMEM
            for (;;) {
                const int it = take_item(S, rq);
                if (it == -2) goto done1;
                if (it < 0) break;
                int side, k;
                const Params &P = item_of<BATCH>(P0, src, it, side, k);
                Item x;
                if (!decode(P, side, k, x)) continue;
                if (x.rl) {
                    if (!wait32(S, &S->a_full, iw & 1)) goto done1;
                    fence_after();
                    // the owned tile into TMEM once per item (ordered after the
                    // previous item's MMAs and before this item's: same issuing
                    // thread); its shared-memory slot is free when the copies are
                    switch (KP) {
                    case 64: own_to_tmem<64>(ld, tA, aA); break;
                    case 128: own_to_tmem<128>(ld, tA, aA); break;
                    case 192: own_to_tmem<192>(ld, tA, aA); break;
                    default: own_to_tmem<256>(ld, tA, aA); break;
                    }
                    commit_if(ld, &S->a_empty);
                    ++iw;
                    for (int j = 0; j <= x.nj; ++j) {
                        if (j < x.nj) {
                            const uint32_t st = r1.slot;
                            const uint32_t bm = tw & 1;
                            if (!wait32x2(S, &S->full[st], r1.phase, &S->mu_empty[bm], ((tw >> 1) & 1) ^ 1))
                                goto done1;
                            fence_after();
                            const uint32_t aB = saddr(sB + (size_t)st * b_bytes);
                            const uint32_t dmu = tmem + bm * (uint32_t)kBN;
                            switch (KP) {
                            case 64: gemm1_tile<64>(ld, dmu, tA, aB, id1); break;
                            case 128: gemm1_tile<128>(ld, dmu, tA, aB, id1); break;
                            case 192: gemm1_tile<192>(ld, dmu, tA, aB, id1); break;
                            default: gemm1_tile<256>(ld, dmu, tA, aB, id1); break;
                            }
                            commit_if(ld, &S->mu_full[bm]);
                            ++tw;
                            r1.next(NS);
                        }
                        if (j > 0) {
                            // GEMM2 of tile j - 1
                            const uint32_t be = te & 1;
                            const uint32_t st = r2.slot;
                            if (!wait32(S, &S->e_full[be], (te >> 1) & 1)) goto done1;
                            if (j == 1 && !wait32(S, &S->g_empty, (ic & 1) ^ 1)) goto done1;
                            fence_after();
                            // A = E (K-major, one atom of 64 walked columns); B = the
                            // walked tile read MN-major: MN atoms (64 entries of k)
                            // 64 rows x 128 B apart (LBO), 8-row K groups 1024 B apart
                            // (SBO), a K step of 16 walked rows = 2048 B
                            const uint64_t dE = sdesc_sw128(saddr(sE + be * kEBytes), 16, 1024);
                            const uint64_t dBt = sdesc_sw128(saddr(sB + (size_t)st * b_bytes), kBN * 128, 1024);
#pragma unroll
                            for (int ks = 0; ks < kBN / 16; ++ks)
                                mma_ss_if(ld, tmem + kGCol, dE + (uint64_t)(ks * 2), dBt + (uint64_t)(ks * 128),
                                          id2, (j > 1 || ks > 0));
                            commit_if(ld, &S->e_empty[be]);
                            commit_if(ld, &S->empty[st]);
                            ++te;
                            r2.next(NS);
                        }
                    }
                } else {
                    // G (owned H^T rows) += E^T . W over the block's W rows, 64
                    // at a time.  A = the two E halves read MN-major (64 owned
                    // rows per 128-byte atom column, the second half 8 KB on,
                    // 8 W rows per 1024 B); B = the W tile read MN-major as in
                    // GEMM2.  A K step of 16 W rows is 2048 B in both.  Two
                    // accumulators (owned rows 0..127 at TMEM column 0, rows
                    // 128..255 at column 256) share each W tile.
                    for (int s = 0; s < x.nj; ++s) {
                        const uint32_t sh = rh.slot;
                        const uint32_t stage = saddr(sm) + sh * h_bytes;
                        if (!wait32(S, &S->hfull[sh], rh.phase)) goto done1;
                        if (s == 0 && !wait32(S, &S->g_empty, (ic & 1) ^ 1)) goto done1;
                        fence_after();
                        const uint64_t dE0 = sdesc_sw128(stage + b_bytes, kEBytes / 2, 1024);
                        const uint64_t dE1 = sdesc_sw128(stage + b_bytes + kEBytes, kEBytes / 2, 1024);
                        const uint64_t dW = sdesc_sw128(stage, kBN * 128, 1024);
                        if (x.rows_per == kOwnH) {
#pragma unroll
                            for (int ks = 0; ks < kBN / 16; ++ks) {
                                mma_ss_if(ld, tmem, dE0 + (uint64_t)(ks * 128), dW + (uint64_t)(ks * 128), id3,
                                          (s > 0 || ks > 0));
                                mma_ss_if(ld, tmem + 256, dE1 + (uint64_t)(ks * 128), dW + (uint64_t)(ks * 128),
                                          id3, (s > 0 || ks > 0));
                            }
                        } else {
#pragma unroll
                            for (int ks = 0; ks < kBN / 16; ++ks)
                                mma_ss_if(ld, tmem, dE0 + (uint64_t)(ks * 128), dW + (uint64_t)(ks * 128), id3,
                                          (s > 0 || ks > 0));
                        }
                        commit_if(ld, &S->hempty[sh]);
                        rh.next(NH);
                    }
                }
                commit_if(ld, &S->g_full);
                ++ic;
            }
        }
    done1:
        __syncwarp();
    } else if (warp == 2 + kEpiWarps) {
        // ---------------- E stores (warp 10, lane 0 performs): each rows-item
        // E tile, once the epilogue has built it, to HBM with one bulk copy;
        // the buffer's second release (the first is GEMM2's commit) once the
        // copy has read it; after the item's last tile, the count that its
        // block's columns items wait for
        uint32_t te = 0;
        Ring rq;
        for (;;) {
            const int it = take_item(S, rq);
            if (it == -2) goto done3;
            if (it < 0) break;
            int side, k;
            const Params &P = item_of<BATCH>(P0, src, it, side, k);
            Item x;
            if (!decode(P, side, k, x) || !x.rl) continue;
            unsigned char *eg = reinterpret_cast<unsigned char *>(
                P.Et + ((int64_t)x.block * P.side[0].own_tiles + x.ot) * P.et_cols * (kEBytes / 2));
            for (int j = 0; j < x.nj; ++j, ++te) {
                const uint32_t be = te & 1;
                if (!wait32(S, &S->e_full[be], (te >> 1) & 1)) goto done3;
                if (lane == 0)
                    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n\t"
                                 "cp.async.bulk.commit_group;\n\t"
                                 "cp.async.bulk.wait_group.read 0;"
                                 :: "l"(eg + (size_t)j * kEBytes), "r"(saddr(sE + be * kEBytes)), "r"(kEBytes)
                                 : "memory");
                __syncwarp();
                if (lane == 0) bar_arrive(&S->e_empty[be]);
            }
            // the item's E complete in HBM: count it (release after the
            // async-proxy writes)
            if (lane == 0) {
                asm volatile("cp.async.bulk.wait_group 0;\n\tfence.proxy.async.global;" ::: "memory");
                __threadfence();
                atomicAdd(P.sync + 2 + x.block, 1);
            }
            __syncwarp();
        }
    done3:
        if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 2..9): TMEM lane quarter warp % 4,
        // walked columns 32 h .. 32 h + 31 of each tile, h = (warp - 2) / 4
        const int q = warp & 3, hc = (warp - 2) >> 2;
        const int rho = 32 * q + lane;                      // owned row in the tile
        const int c = 32 * hc;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        uint32_t ic = 0, tw = 0, te = 0, np = 0;   // items, mu uses, E uses, staging passes
        Ring rq;
        for (;;) {
            const int it = take_item(S, rq);
            if (it == -2) goto done2;
            if (it < 0) break;
            int side, k;
            const Params &P = item_of<BATCH>(P0, src, it, side, k);
            Item x;
            if (!decode(P, side, k, x)) continue;
            const Side &Sd = P.side[side];
            if (x.rl) {
                const float pp = P.p, mu_min = P.mu_min;
                // V straight from HBM into registers, two tiles ahead: this
                // thread's 16-byte chunks (c / (16 / sizeof(VT)) + i, row rho)
                // of each tile, a warp reading 512 contiguous bytes per load
                constexpr int kVQ = sizeof(VT) == 4 ? 8 : 4;
                const unsigned char *vrow =
                    Sd.Vt + (((int64_t)x.own_piece * P.B + x.walk_piece) * Sd.own_tiles + x.ot) * Sd.walk_tiles *
                                (int64_t)v_bytes +
                    ((size_t)(c / (int)(16 / sizeof(VT))) * kOwn + rho) * 16;
                uint4 qa[kVQ], qb[kVQ];
                auto vload = [&](uint4 (&q)[kVQ], int jj) {
                    if (jj < x.nj) {
                        const unsigned char *src_v = vrow + (int64_t)jj * v_bytes;
#pragma unroll
                        for (int i = 0; i < kVQ; ++i) q[i] = ldg_stream(src_v + (size_t)i * kOwn * 16);
                    }
                };
                // one walked tile: E from TMEM mu and the V chunks in q
                auto tile = [&](const uint4 (&q)[kVQ]) -> bool {
                    const uint32_t bm = tw & 1, be = te & 1;
                    if (!wait32x2(S, &S->mu_full[bm], (tw >> 1) & 1, &S->e_empty[be], ((te >> 1) & 1) ^ 1))
                        return false;
                    fence_after();
                    unsigned char *eb = sE + be * kEBytes;
                    float mu[32];
                    tmem_ld32(tmem + lane_base + bm * (uint32_t)kBN + (uint32_t)c, mu);
                    float v[32];
                    if constexpr (sizeof(VT) == 4) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            v[4 * i] = __uint_as_float(q[i].x); v[4 * i + 1] = __uint_as_float(q[i].y);
                            v[4 * i + 2] = __uint_as_float(q[i].z); v[4 * i + 3] = __uint_as_float(q[i].w);
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const uint32_t u[4] = {q[i].x, q[i].y, q[i].z, q[i].w};
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                v[8 * i + 2 * h] = __uint_as_float(u[h] << 16);
                                v[8 * i + 2 * h + 1] = __uint_as_float(u[h] & 0xffff0000u);
                            }
                        }
                    }
                    uint32_t pk[16];
#pragma unroll
                    for (int h = 0; h < 16; ++h) {
                        const float e0 = tweedie_pm<PM>(pp, mu_min, v[2 * h], mu[2 * h]);
                        const float e1 = tweedie_pm<PM>(pp, mu_min, v[2 * h + 1], mu[2 * h + 1]);
                        __nv_bfloat162 t2 = __floats2bfloat162_rn(e0, e1);
                        pk[h] = *reinterpret_cast<uint32_t *>(&t2);
                    }
                    // E (owned row rho, walked columns c..c+31): row rho of the
                    // 128-byte-swizzled atom column, chunk (c/8 + g) ^ (rho % 8)
#pragma unroll
                    for (int g = 0; g < 4; ++g)
                        *reinterpret_cast<uint4 *>(eb + rho * 128 + ((((c >> 3) + g) ^ (rho & 7)) << 4)) =
                            make_uint4(pk[4 * g], pk[4 * g + 1], pk[4 * g + 2], pk[4 * g + 3]);
                    fence_async_smem();
                    fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        bar_arrive(&S->mu_empty[bm]);
                        bar_arrive(&S->e_full[be]);
                    }
                    ++tw;
                    ++te;
                    return true;
                };
                vload(qa, 0);
                vload(qb, 1);
                for (int j = 0; j < x.nj; j += 2) {
                    if (!tile(qa)) goto done2;
                    vload(qa, j + 2);
                    if (j + 1 < x.nj) {
                        if (!tile(qb)) goto done2;
                        vload(qb, j + 3);
                    }
                }
            }
            // the item's G rows (times 1 / phi) to HBM, coalesced through a
            // 32 KB staging buffer: passes of 64 columns; in each, every warp
            // puts its 32 rows x 32 columns (lane quarter q, half hc) in the
            // buffer (16-byte chunk k of row r at chunk position k ^ (r % 8),
            // so both the writes and the reads are free of bank conflicts),
            // then stores 16 whole 256-byte row segments, two rows per
            // instruction.  Staging: the E buffers for a rows item (free once
            // its last GEMM2 and E store have read them), a buffer of its own
            // for a columns item.  The passes are ordered by two mbarriers
            // (bounded waits), so a warp that gives up cannot strand the others.
            if (!wait32(S, &S->g_full, ic & 1)) goto done2;
            {
                unsigned char *stg = sStgH;
                if (x.rl) {
                    if (!wait32x2(S, &S->e_empty[te & 1], ((te >> 1) & 1) ^ 1, &S->e_empty[(te + 1) & 1],
                                  (((te + 1) >> 1) & 1) ^ 1))
                        goto done2;
                    stg = sE;
                }
                fence_after();
                const float phi_inv = P.phi_inv;
                const int w8 = warp - 2;
                // rows item: one accumulator at kGCol; columns item: two, of
                // 128 rows each, at columns 0 and 256
                const int nacc = x.rows_per / kOwn;
                for (int a = 0; a < nacc; ++a)
                for (int cp = 0; cp < KP; cp += 64, ++np) {
                    const uint32_t gcol = x.rl ? kGCol : 256u * (uint32_t)a;
                    float *gbase = Sd.G + (x.own_start + (int64_t)x.row0 + 128 * a) * P.ldk;
                    const int rows = x.own_rows_in_tile - 128 * a;
                    float g[32];
                    tmem_ld32(tmem + lane_base + gcol + (uint32_t)(cp + c), g);
                    if (a == nacc - 1 && cp + 64 >= KP) {
                        // this warp's last TMEM read of the item: G may be reused
                        fence_before();
                        __syncwarp();
                        if (lane == 0) bar_arrive(&S->g_empty);
                    }
                    if (!wait32(S, &S->stg_empty, (np & 1) ^ 1)) goto done2;
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        *reinterpret_cast<float4 *>(stg + rho * 256 + (((hc * 8 + i) ^ (rho & 7)) << 4)) =
                            make_float4(g[4 * i], g[4 * i + 1], g[4 * i + 2], g[4 * i + 3]);
                    __syncwarp();
                    if (lane == 0) bar_arrive(&S->stg_full);
                    if (!wait32(S, &S->stg_full, np & 1)) goto done2;
#pragma unroll
                    for (int s2 = 0; s2 < 8; ++s2) {
                        const int r = 16 * w8 + 2 * s2 + (lane >> 4), ch = lane & 15;
                        const float4 val =
                            *reinterpret_cast<const float4 *>(stg + r * 256 + ((ch ^ (r & 7)) << 4));
                        const int col = cp + 4 * ch;
                        if (r < rows && col < P.ldk)
                            *reinterpret_cast<float4 *>(gbase + (int64_t)r * P.ldk + col) =
                                make_float4(val.x * phi_inv, val.y * phi_inv, val.z * phi_inv, val.w * phi_inv);
                    }
                    __syncwarp();
                    if (lane == 0) bar_arrive(&S->stg_empty);
                }
                // a rows item staged in the E buffers, which this warp fills
                // again with the next item's first tile: first every warp
                // must be done reading the last pass
                if (x.rl && !wait32(S, &S->stg_empty, (np & 1) ^ 1)) goto done2;
            }
            // the item is done with shared memory and TMEM (the producer's
            // columns stages may take over once every earlier item is)
            if (lane == 0) atomicAdd(&S->items_done, 1);
            ++ic;
        }
    done2:
        __syncwarp();
    }

    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x == 0) {
        if (S->abort) {                                      // two-sided kernel (+ role)
            if constexpr (BATCH) {
                for (int i = 0; i < src.n; ++i)
                    atomicOr(reinterpret_cast<const Params *>(src.tab + (size_t)i * src.stride)->err,
                             64 | S->abort);
            } else {
                atomicOr(P0.err, 64 | S->abort);
            }
        }
        // the last CTA to finish (every item claimed and done, or given up)
        // sets the launch's counters back to zero
        __threadfence();
        if (atomicAdd(P0.sync + 1, 1) == (int)gridDim.x - 1) {
            __threadfence();
            if constexpr (BATCH) {
                for (int i = 0; i < src.n; ++i) {
                    const Params &Pi = *reinterpret_cast<const Params *>(src.tab + (size_t)i * src.stride);
                    for (int b = 0; b < Pi.B; ++b) Pi.sync[2 + b] = 0;
                }
            } else {
                for (int b = 0; b < P0.B; ++b) P0.sync[2 + b] = 0;
            }
            P0.sync[0] = 0;
            P0.sync[1] = 0;
        }
    }
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"(kTmemCols) : "memory");
}

template <typename VT, int PM>
__global__ void __launch_bounds__(kThreads, 1) chain_kernel(const __grid_constant__ Params P)
{
    chain_body<VT, PM, false>(P, Src{nullptr, nullptr, nullptr, 1, 0}, P.items);
}

// Many contexts of one K width, V type and power in one persistent launch.
template <typename VT, int PM>
__global__ void __launch_bounds__(kThreads, 1)
chain_batch_kernel(const unsigned char *tab, size_t stride, const int *wstart, const int *hstart, int n)
{
    chain_body<VT, PM, true>(*reinterpret_cast<const Params *>(tab), Src{tab, wstart, hstart, n, stride},
                             __ldg(wstart + n) + __ldg(hstart + n));
}

}  // namespace two_sided

using DenseFn = void (*)(DenseParams);

DenseFn pick_dense(int kp, bool f8)
{
    switch (kp) {
    case 16: return f8 ? dense_grad_kernel<16, true> : dense_grad_kernel<16, false>;
    case 32: return f8 ? dense_grad_kernel<32, true> : dense_grad_kernel<32, false>;
    case 64: return f8 ? dense_grad_kernel<64, true> : dense_grad_kernel<64, false>;
    case 128: return f8 ? dense_grad_kernel<128, true> : dense_grad_kernel<128, false>;
    }
    return nullptr;
}

using DenseBatchFn = void (*)(const unsigned char *, size_t, const int *, int);

DenseBatchFn pick_dense_batch(int kp, bool f8)
{
    switch (kp) {
    case 16: return f8 ? dense_grad_batch_kernel<16, true> : dense_grad_batch_kernel<16, false>;
    case 32: return f8 ? dense_grad_batch_kernel<32, true> : dense_grad_batch_kernel<32, false>;
    case 64: return f8 ? dense_grad_batch_kernel<64, true> : dense_grad_batch_kernel<64, false>;
    case 128: return f8 ? dense_grad_batch_kernel<128, true> : dense_grad_batch_kernel<128, false>;
    }
    return nullptr;
}

int dense_kp(int K)
{
    int kp = 16;
    while (kp < K) kp <<= 1;
    return kp;
}

// At least half of an SM's shared memory, so that at most one of the
// library's TMEM-holding CTAs (this kernel's 256 columns, the two-sided
// kernel's 512) is resident per SM: a tcgen05.alloc that cannot be met
// blocks, and a CTA holding TMEM beside it must never wait on that.
size_t dense_smem(int kp, bool f8)
{
    const size_t e4m3 = f8 ? 2 * (size_t)kTile * std::max(kp, 32) : 0;
    // tiles, then the mbarrier (8 bytes), the TMEM address and two scale slots (4 each)
    return std::max<size_t>(2 * (size_t)kTile * kp * 2 + (size_t)kTile * kTile * 2 + e4m3 + 32,
                            116 * 1024);
}

}  // namespace

bool dense_supported(int K) { return K >= 1 && K <= 256; }

int dense_mtiles(const psgld_ctx *c)
{
    const int64_t rows = (c->I + c->B - 1) / c->B;   // largest row piece
    return (int)((rows + kTile - 1) / kTile);
}

namespace {

int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

__device__ __forceinline__ int64_t piece_start_d(int64_t r, int64_t n, int B) { return (r * n) / B; }
__device__ __forceinline__ int64_t piece_of_d(int64_t x, int64_t n, int B) { return ((x + 1) * B - 1) / n; }

// V (I x J, FP32, row-major) into the tiles of one orientation (side 0: owned
// = rows of V, side 1: owned = columns); padding stays zero.
template <typename VT>
__global__ void build_vtiles_kernel(const float *__restrict__ V, int64_t I, int64_t J, int B, int side,
                                    int own_tiles, int walk_tiles, VT *__restrict__ out)
{
    const int64_t n_own = side == 0 ? I : J, n_walk = side == 0 ? J : I;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < I * J;
         a += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = a / J, j = a - i * J;
        const int64_t own = side == 0 ? i : j, walk = side == 0 ? j : i;
        const int64_t op = piece_of_d(own, n_own, B), wp = piece_of_d(walk, n_walk, B);
        const int64_t orow = own - piece_start_d(op, n_own, B), wrow = walk - piece_start_d(wp, n_walk, B);
        const int64_t tile = ((op * B + wp) * own_tiles + (orow >> 7)) * walk_tiles + (wrow >> 6);
        const int rho = (int)(orow & 127), kap = (int)(wrow & 63);
        int64_t e;
        if constexpr (sizeof(VT) == 4)
            e = tile * 8192 + ((int64_t)(kap >> 2) * 128 + rho) * 4 + (kap & 3);
        else
            e = tile * 8192 + ((int64_t)(kap >> 3) * 128 + rho) * 8 + (kap & 7);
        if constexpr (sizeof(VT) == 4)
            out[e] = V[a];
        else
            out[e] = __float2bfloat16_rn(V[a]);
    }
}

__global__ void build_shadow_kernel(const float *__restrict__ X, int64_t n, int ngroups, int ldk, int B,
                                    int tiles, int KP, uint16_t *__restrict__ sh)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n * ngroups;
         a += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = a / ngroups;
        const int q = (int)(a - row * ngroups);
        const float4 x = *reinterpret_cast<const float4 *>(X + row * ldk + 4 * q);
        dev::shadow_store4(sh, row, 4 * q, x, n, B, tiles, KP);
    }
}

using ChainRcFn = void (*)(two_sided_rc::Params);

ChainRcFn pick_chain_rc(bool vb, int pm)
{
    static const ChainRcFn f[2][4] = {
        {two_sided_rc::chain_kernel<float, 0>, two_sided_rc::chain_kernel<float, 1>,
         two_sided_rc::chain_kernel<float, 2>, two_sided_rc::chain_kernel<float, 3>},
        {two_sided_rc::chain_kernel<__nv_bfloat16, 0>, two_sided_rc::chain_kernel<__nv_bfloat16, 1>,
         two_sided_rc::chain_kernel<__nv_bfloat16, 2>, two_sided_rc::chain_kernel<__nv_bfloat16, 3>}};
    return f[vb ? 1 : 0][pm];
}

using ChainRcBatchFn = void (*)(const unsigned char *, size_t, const int *, int);

ChainRcBatchFn pick_chain_batch_rc(bool vb, int pm)
{
    static const ChainRcBatchFn f[2][4] = {
        {two_sided_rc::chain_batch_kernel<float, 0>, two_sided_rc::chain_batch_kernel<float, 1>,
         two_sided_rc::chain_batch_kernel<float, 2>, two_sided_rc::chain_batch_kernel<float, 3>},
        {two_sided_rc::chain_batch_kernel<__nv_bfloat16, 0>, two_sided_rc::chain_batch_kernel<__nv_bfloat16, 1>,
         two_sided_rc::chain_batch_kernel<__nv_bfloat16, 2>, two_sided_rc::chain_batch_kernel<__nv_bfloat16, 3>}};
    return f[vb ? 1 : 0][pm];
}

size_t rc_bytes(int KP, int vsize, int stages, int vstages)
{
    return (size_t)two_sided_rc::kOwn * KP * 2 + 2 * (size_t)two_sided_rc::kOwn * two_sided_rc::kBN * 2 +
           (size_t)stages * two_sided_rc::kBN * KP * 2 +
           (size_t)vstages * two_sided_rc::kOwn * two_sided_rc::kBN * vsize + sizeof(two_sided_rc::Bars) + 16 +
           1024;   // alignment slack
}

// At least half of an SM's shared memory, so that one CTA (and one 512-column
// TMEM allocation) runs per SM.
size_t rc_smem(int KP, int vsize, int stages, int vstages)
{
    return std::max<size_t>(rc_bytes(KP, vsize, stages, vstages), 120 * 1024);
}

// Ring depths: two V slots (they free as soon as the epilogue has read
// them), then as many walked-factor slots as fit (2 .. 4), then a third V
// slot if it still fits.
void rc_stages(int KP, int vsize, int *stages, int *vstages)
{
    int s = two_sided_rc::kMaxStages;
    while (s > 2 && rc_bytes(KP, vsize, s, 2) > 232448) --s;
    int v = 2;
    if (rc_bytes(KP, vsize, s, 3) <= 232448) v = 3;
    *stages = s;
    *vstages = v;
}

using ChainFn = void (*)(two_sided::Params);

ChainFn pick_chain(bool vb, int pm)
{
    static const ChainFn f[2][4] = {
        {two_sided::chain_kernel<float, 0>, two_sided::chain_kernel<float, 1>,
         two_sided::chain_kernel<float, 2>, two_sided::chain_kernel<float, 3>},
        {two_sided::chain_kernel<__nv_bfloat16, 0>, two_sided::chain_kernel<__nv_bfloat16, 1>,
         two_sided::chain_kernel<__nv_bfloat16, 2>, two_sided::chain_kernel<__nv_bfloat16, 3>}};
    return f[vb ? 1 : 0][pm];
}

using ChainBatchFn = void (*)(const unsigned char *, size_t, const int *, const int *, int);

ChainBatchFn pick_chain_batch(bool vb, int pm)
{
    static const ChainBatchFn f[2][4] = {
        {two_sided::chain_batch_kernel<float, 0>, two_sided::chain_batch_kernel<float, 1>,
         two_sided::chain_batch_kernel<float, 2>, two_sided::chain_batch_kernel<float, 3>},
        {two_sided::chain_batch_kernel<__nv_bfloat16, 0>, two_sided::chain_batch_kernel<__nv_bfloat16, 1>,
         two_sided::chain_batch_kernel<__nv_bfloat16, 2>, two_sided::chain_batch_kernel<__nv_bfloat16, 3>}};
    return f[vb ? 1 : 0][pm];
}

// Shared memory: the rows items' layout (owned tile, E buffers, walked-tile
// ring) and the columns items' (stages, G staging) share one region; the
// barriers follow it.
size_t two_sided_rows_layout(int KP, int stages)
{
    return (size_t)two_sided::kOwn * KP * 2 + 2 * (size_t)two_sided::kEBytes +
           (size_t)stages * two_sided::kBN * KP * 2;
}

constexpr size_t kTwoSidedExtra = sizeof(two_sided::Bars) + 16 + 1024;   // barriers, alignment slack
constexpr size_t kTwoSidedMax = 232448;

// Columns-item stages: as many W tile + E halves stages as fit beside their
// G staging buffer, at most kMaxHStages.
int two_sided_hstages(int KP)
{
    const size_t h = (size_t)two_sided::kBN * KP * 2 + 2 * (size_t)two_sided::kEBytes;
    const size_t room = kTwoSidedMax - kTwoSidedExtra - two_sided::kStgBytes;
    return (int)std::min<size_t>(room / h, two_sided::kMaxHStages);
}

size_t two_sided_bars_off(int KP, int stages)
{
    const size_t h = (size_t)two_sided::kBN * KP * 2 + 2 * (size_t)two_sided::kEBytes;
    return std::max(two_sided_rows_layout(KP, stages), (size_t)two_sided_hstages(KP) * h + two_sided::kStgBytes);
}

size_t two_sided_bytes(int KP, int stages)
{
    return two_sided_bars_off(KP, stages) + kTwoSidedExtra;
}

// At least half of an SM's shared memory, so that one CTA (and one 512-column
// TMEM allocation) runs per SM.
size_t two_sided_smem(int KP, int stages)
{
    return std::max<size_t>(two_sided_bytes(KP, stages), 120 * 1024);
}

// Walked-tile ring depth: as many slots as fit beside the owned tile and the
// E buffers (2 .. kMaxStages).
int two_sided_stages(int KP)
{
    int s = two_sided::kMaxStages;
    while (s > 2 && two_sided_rows_layout(KP, s) + kTwoSidedExtra > kTwoSidedMax) --s;
    return s;
}



}  // namespace

psgld_status prepare_dense(psgld_ctx *c, cudaStream_t st)
{
    const int mode = c->opt.dense_path;
    const bool vb = c->opt.dense_v_bf16 != 0;
    if (!dense_supported(c->K)) return fail(c, PSGLD_ERR_ARG, "dense tensor-core path supports K <= 256");
    c->mtiles = dense_mtiles(c);
    const bool f8 = c->opt.dense_fp8 != 0;
    bool two = mode == 2 || (mode == 1 && !f8 && (vb || c->K > 128 || c->mtiles > 1));
    if ((mode == 3 || f8) && (vb || c->K > 128 || mode == 2))
        return fail(c, PSGLD_ERR_ARG, "single-pass dense kernel (and its E4M3 GEMM1): K <= 128, FP32 V");
    if (!two) {
        c->dense_kind = 1;
        const int kp = dense_kp(c->K);
        const bool f8 = c->opt.dense_fp8 != 0;
        PSGLD_CK(c, cudaFuncSetAttribute(pick_dense(kp, f8), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dense_smem(kp, f8)));
        c->dense_fp8 = f8 ? 1 : 0;
        return PSGLD_OK;
    }
    c->dense_kind = 2;
    c->v_bf16 = vb ? 1 : 0;
    c->KP = 64 * cdiv(c->K, 64);
    const int64_t maxI = (c->I + c->B - 1) / c->B, maxJ = (c->J + c->B - 1) / c->B;
    c->mt_max = cdiv(maxI, 128);
    c->nt_max = cdiv(maxJ, 128);
    c->nt2_max = cdiv(maxJ, 256);
    c->ni_max = cdiv(maxI, 64);
    c->nj_max = cdiv(maxJ, 64);
    const int vs = vb ? 2 : 4;
    // the limit is an attribute of the kernel, shared by every context that
    // launches it (any K width): the largest size any of them asks for
    for (int pm = 0; pm < 4; ++pm) {
        PSGLD_CK(c, cudaFuncSetAttribute(pick_chain(vb, pm), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTwoSidedMax));
        PSGLD_CK(c, cudaFuncSetAttribute(pick_chain_rc(vb, pm), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTwoSidedMax));
    }
    int sms = 0;
    PSGLD_CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    c->share_e = two_sided_share(c->opt.dense_share_e, maxI, c->B, c->mt_max, c->nt_max, sms);
    const int64_t B = c->B;
    const int64_t nA = B * B * c->mt_max * c->nj_max * 8192;
    const int64_t nB = c->share_e ? 0 : B * B * c->nt_max * c->ni_max * 8192;   // V tiles, other orientation
    const int64_t nW = B * 2 * c->mt_max * 64 * c->KP, nH = B * 2 * c->nt_max * 64 * c->KP;
    const int64_t nE = c->share_e ? B * c->mt_max * 4 * c->nt2_max * 8192 : 0;   // one part's E tiles
    auto al = [&](void **p, size_t bytes) -> psgld_status {
        *p = dev_alloc(c, bytes, st);
        if (!*p) return fail(c, PSGLD_ERR_OOM, "device allocation failed");
        // padding stays zero; so do E slots no rows item writes, and the
        // launch counters between launches
        PSGLD_CK(c, cudaMemsetAsync(*p, 0, bytes, st));
        return PSGLD_OK;
    };
    psgld_status s = al(&c->VA, (size_t)nA * vs);
    if (s == PSGLD_OK && nB) s = al(&c->VB, (size_t)nB * vs);
    if (s == PSGLD_OK) s = al((void **)&c->Wsh, (size_t)nW * 2);
    if (s == PSGLD_OK) s = al((void **)&c->Hsh, (size_t)nH * 2);
    if (s == PSGLD_OK && nE) s = al((void **)&c->Et, (size_t)nE * 2);
    if (s == PSGLD_OK) s = al((void **)&c->tsync, sizeof(int) * (size_t)(2 + B));
    return s;
}

psgld_status build_dense_tiles(psgld_ctx *c, cudaStream_t st)
{
    if (c->dense_kind != 2) return PSGLD_OK;
    // V for the rows items; and in the other orientation for columns items
    // that form their own mu (with shared E they take E from the rows items)
    const int64_t n = c->I * c->J;
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 32);
    for (int side = 0; side < (c->share_e ? 1 : 2); ++side) {
        const int own_tiles = side == 0 ? c->mt_max : c->nt_max;
        const int walk_tiles = side == 0 ? c->nj_max : c->ni_max;
        void *out = side == 0 ? c->VA : c->VB;
        if (c->v_bf16)
            build_vtiles_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(c->Vd, c->I, c->J, c->B, side, own_tiles,
                                                                      walk_tiles, (__nv_bfloat16 *)out);
        else
            build_vtiles_kernel<float><<<grid, 256, 0, st>>>(c->Vd, c->I, c->J, c->B, side, own_tiles,
                                                              walk_tiles, (float *)out);
        PSGLD_CK(c, cudaGetLastError());
    }
    return PSGLD_OK;
}

psgld_status build_dense_shadows(psgld_ctx *c, cudaStream_t st)
{
    if (!c->dense || c->dense_kind != 2 || !c->has_factors) return PSGLD_OK;
    for (int side = 0; side < 2; ++side) {
        const int64_t n = side == 0 ? c->I : c->J;
        const float *X = side == 0 ? c->W[c->wcur] : c->Ht[c->hcur];
        const unsigned grid = (unsigned)std::min<int64_t>((n * c->ngroups + 255) / 256, 152 * 16);
        build_shadow_kernel<<<grid, 256, 0, st>>>(X, n, c->ngroups, c->ldk, c->B,
                                                  2 * (side == 0 ? c->mt_max : c->nt_max), c->KP,
                                                  side == 0 ? c->Wsh : c->Hsh);
        PSGLD_CK(c, cudaGetLastError());
    }
    return PSGLD_OK;
}

// Blocks whose columns items cover 256 rows (two accumulators sharing each W
// tile: a third fewer bytes per MAC); the last blocks' columns items, which
// end the launch, keep 128 rows so that its CTAs finish together.  The
// option overrides the rule; the results do not depend on it.
// Columns items take E from the rows items (three contractions per block,
// but a wait for the block's rows items and E through L2 / HBM) when the
// row pieces are long (each columns item walks at least 512 W rows) and the
// part's items fill more than one wave of CTAs; short pieces or a single
// wave favour columns items that form their own mu, all items at once.
// The option overrides the rule (-1 = the rule).
int two_sided_share(int opt, int64_t max_rows, int B, int mt, int nt, int sms)
{
    if (opt >= 0) return opt;
    return max_rows >= 512 && (int64_t)B * (mt + nt) > sms ? 1 : 0;
}

static int two_sided_hwide(const psgld_ctx *c)
{
    if (c->opt.wide_col_blocks >= 0) return std::min(c->opt.wide_col_blocks, c->B);
    return c->B / 2;
}

static void fill_two_sided(const psgld_ctx *c, int part, two_sided::Params &P)
{
    P = two_sided::Params{};
    const int64_t I = c->I, J = c->J;
    two_sided::Side &A = P.side[0], &Bs = P.side[1];
    A.own_sh = c->Wsh; A.walk_sh = c->Hsh; A.Vt = (const unsigned char *)c->VA; A.G = c->G;
    A.n_own = I; A.n_walk = J; A.own_tiles = c->mt_max; A.walk_tiles = c->nj_max;
    A.own_sh64 = 2 * c->mt_max; A.walk_sh64 = 2 * c->nt_max;
    Bs.own_sh = nullptr; Bs.walk_sh = c->Wsh; Bs.Vt = nullptr; Bs.G = c->G + I * c->ldk;
    Bs.n_own = J; Bs.n_walk = I; Bs.own_tiles = c->nt2_max; Bs.walk_tiles = c->ni_max;
    Bs.own_sh64 = 2 * c->nt_max; Bs.walk_sh64 = 2 * c->mt_max;
    P.Et = c->Et;
    P.sync = c->tsync;
    P.et_cols = 4 * c->nt2_max;
    P.ht1 = c->nt_max;
    P.ht2 = c->nt2_max;
    P.hwide = two_sided_hwide(c);
    P.B = c->B;
    P.part = part;
    P.KP = c->KP;
    P.ldk = c->ldk;
    P.stages = two_sided_stages(c->KP);
    P.hstages = two_sided_hstages(c->KP);
    P.bars_off = (int)two_sided_bars_off(c->KP, P.stages);
    P.items_a = c->B * c->mt_max;
    P.items = P.items_a + P.hwide * c->nt2_max + (c->B - P.hwide) * c->nt_max;
    P.phi_inv = (float)(1.0 / c->phi);
    P.p = (float)c->p;
    P.mu_min = (float)c->opt.mu_min;
    P.p_mode = c->p == 0.0 ? 0 : c->p == 1.0 ? 1 : c->p == 2.0 ? 2 : 3;
    P.err = c->kflag;
}

// Every item forming its own mu (the two_sided_rc kernel).
static void fill_rc(const psgld_ctx *c, int part, two_sided_rc::Params &P)
{
    P = two_sided_rc::Params{};
    const int64_t I = c->I, J = c->J;
    two_sided_rc::Side &A = P.side[0], &Bs = P.side[1];
    A.own_sh = c->Wsh; A.walk_sh = c->Hsh; A.Vt = (const unsigned char *)c->VA; A.G = c->G;
    A.n_own = I; A.n_walk = J; A.own_tiles = c->mt_max; A.walk_tiles = c->nj_max;
    A.own_sh64 = 2 * c->mt_max; A.walk_sh64 = 2 * c->nt_max;
    Bs.own_sh = c->Hsh; Bs.walk_sh = c->Wsh; Bs.Vt = (const unsigned char *)c->VB; Bs.G = c->G + I * c->ldk;
    Bs.n_own = J; Bs.n_walk = I; Bs.own_tiles = c->nt_max; Bs.walk_tiles = c->ni_max;
    Bs.own_sh64 = 2 * c->nt_max; Bs.walk_sh64 = 2 * c->mt_max;
    P.B = c->B;
    P.part = part;
    P.KP = c->KP;
    P.ldk = c->ldk;
    const int vs = c->v_bf16 ? 2 : 4;
    rc_stages(c->KP, vs, &P.stages, &P.vstages);
    P.items_a = c->B * c->mt_max;
    P.items = P.items_a + c->B * c->nt_max;
    P.phi_inv = (float)(1.0 / c->phi);
    P.p = (float)c->p;
    P.mu_min = (float)c->opt.mu_min;
    P.p_mode = c->p == 0.0 ? 0 : c->p == 1.0 ? 1 : c->p == 2.0 ? 2 : 3;
    P.err = c->kflag;
}

static psgld_status launch_rc(psgld_ctx *c, int part, cudaStream_t st)
{
    two_sided_rc::Params P;
    fill_rc(c, part, P);
    const int vs = c->v_bf16 ? 2 : 4;
    int sms = 0;
    PSGLD_CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    int grid = std::min(P.items, sms);
    if (c->opt.max_sms > 0) grid = std::min(grid, c->opt.max_sms);   // leave SMs to other work
    const size_t smem = rc_smem(c->KP, vs, P.stages, P.vstages);
    pick_chain_rc(c->v_bf16 != 0, P.p_mode)<<<grid, two_sided_rc::kThreads, smem, st>>>(P);
    PSGLD_CK(c, cudaGetLastError());
    return PSGLD_OK;
}

static psgld_status launch_two_sided(psgld_ctx *c, int part, cudaStream_t st)
{
    if (!c->share_e) return launch_rc(c, part, st);
    two_sided::Params P;
    fill_two_sided(c, part, P);
    int sms = 0;
    PSGLD_CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    int grid = std::min(P.items, sms);
    if (c->opt.max_sms > 0) grid = std::min(grid, c->opt.max_sms);   // leave SMs to other work
    const size_t smem = two_sided_smem(c->KP, P.stages);
    pick_chain(c->v_bf16 != 0, P.p_mode)<<<grid, two_sided::kThreads, smem, st>>>(P);
    PSGLD_CK(c, cudaGetLastError());
    return PSGLD_OK;
}

static void fill_dense_params(const psgld_ctx *c, int part, DenseParams &P)
{
    P = DenseParams{};
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
    P.mtiles = c->mtiles;
    P.phi_inv = (float)(1.0 / c->phi);
    P.p = (float)c->p;
    P.mu_min = (float)c->opt.mu_min;
    P.p_mode = c->p == 0.0 ? 0 : c->p == 1.0 ? 1 : c->p == 2.0 ? 2 : 3;
    P.err = c->kflag;
}

psgld_status launch_dense_grad(psgld_ctx *c, int part, cudaStream_t st)
{
    if (c->dense_kind == 2) return launch_two_sided(c, part, st);
    const int kp = dense_kp(c->K);
    const bool f8 = c->dense_fp8 != 0;
    DenseFn fn = pick_dense(kp, f8);
    if (!fn) return fail(c, PSGLD_ERR_ARG, "single-pass dense kernel supports K <= 128");
    DenseParams P;
    fill_dense_params(c, part, P);
    fn<<<c->B * P.mtiles, kDenseThreads, dense_smem(kp, f8), st>>>(P);
    PSGLD_CK(c, cudaGetLastError());
    return PSGLD_OK;
}

// Batch keys: single-pass 2 KP + fp8 (< 4096); two-sided 4096 + 8 KP +
// 4 v_bf16 + power mode (the chain kernel's template arguments), plus 8192
// for the shared-E kernel.
int dense_batch_key(const psgld_ctx *c)
{
    if (c->dense_kind == 1) return 2 * dense_kp(c->K) + c->dense_fp8;
    if (c->dense_kind == 2) {
        const int pm = c->p == 0.0 ? 0 : c->p == 1.0 ? 1 : c->p == 2.0 ? 2 : 3;
        return 4096 + 8 * c->KP + 4 * c->v_bf16 + pm + (c->share_e ? 8192 : 0);
    }
    return 0;
}

size_t dense_param_bytes()
{
    const size_t m = std::max({sizeof(DenseParams), sizeof(two_sided::Params), sizeof(two_sided_rc::Params)});
    return (m + 15) & ~size_t(15);
}

int fill_dense_param(const psgld_ctx *c, int part, void *dst, int *first_items)
{
    if (c->dense_kind == 2 && !c->share_e) {
        two_sided_rc::Params P;
        fill_rc(c, part, P);
        std::memcpy(dst, &P, sizeof P);
        *first_items = P.items;
        return P.items;
    }
    if (c->dense_kind == 2) {
        two_sided::Params P;
        fill_two_sided(c, part, P);
        std::memcpy(dst, &P, sizeof P);
        *first_items = P.items_a;   // the rows items, then the columns items
        return P.items;
    }
    DenseParams P;
    fill_dense_params(c, part, P);
    std::memcpy(dst, &P, sizeof P);
    *first_items = c->B * P.mtiles;
    return c->B * P.mtiles;
}

psgld_status launch_dense_batch(psgld_ctx *c0, int key, const void *params, const int *cta_start, int n,
                                int total, cudaStream_t st)
{
    const unsigned char *tab = static_cast<const unsigned char *>(params);
    const size_t stride = dense_param_bytes();
    if (key >= 4096 && key < 8192) {
        // two-sided contexts whose items form their own mu: one persistent
        // launch over all their items, round robin (cta_start: their prefix)
        const int KP = (key - 4096) / 8;
        const bool vb = ((key >> 2) & 1) != 0;
        const int pm = key & 3;
        const int vs = vb ? 2 : 4;
        int stages = 0, vstages = 0;
        rc_stages(KP, vs, &stages, &vstages);
        const size_t smem = rc_smem(KP, vs, stages, vstages);
        ChainRcBatchFn fn = pick_chain_batch_rc(vb, pm);
        PSGLD_CK(c0, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTwoSidedMax));
        int sms = 0;
        PSGLD_CK(c0, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c0->device));
        int grid = std::min(total, sms);
        if (c0->opt.batch_ctas > 0) grid = std::min(grid, (int)c0->opt.batch_ctas);
        if (grid > 0) fn<<<grid, two_sided_rc::kThreads, smem, st>>>(tab, stride, cta_start, n);
        PSGLD_CK(c0, cudaGetLastError());
        return PSGLD_OK;
    }
    if (key >= 8192) {
        // two-sided contexts with shared E: one persistent launch over all
        // their items, claimed in order (rows items of every context first)
        const int KP = (key - 8192 - 4096) / 8;
        const bool vb = ((key >> 2) & 1) != 0;
        const int pm = key & 3;
        const size_t smem = two_sided_smem(KP, two_sided_stages(KP));
        ChainBatchFn fn = pick_chain_batch(vb, pm);
        PSGLD_CK(c0, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTwoSidedMax));
        int sms = 0;
        PSGLD_CK(c0, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c0->device));
        int grid = std::min(total, sms);
        if (c0->opt.batch_ctas > 0) grid = std::min(grid, (int)c0->opt.batch_ctas);
        if (grid > 0) fn<<<grid, two_sided::kThreads, smem, st>>>(tab, stride, cta_start, cta_start + n + 1, n);
        PSGLD_CK(c0, cudaGetLastError());
        return PSGLD_OK;
    }
    const int kp = key / 2;
    const bool f8 = (key & 1) != 0;
    DenseBatchFn fn = pick_dense_batch(kp, f8);
    if (!fn) return fail(c0, PSGLD_ERR_ARG, "single-pass dense kernel supports K <= 128");
    const size_t smem = dense_smem(kp, f8);
    PSGLD_CK(c0, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (total > 0) fn<<<total, kDenseThreads, smem, st>>>(tab, stride, cta_start, n);
    PSGLD_CK(c0, cudaGetLastError());
    return PSGLD_OK;
}

}  // namespace psgld
