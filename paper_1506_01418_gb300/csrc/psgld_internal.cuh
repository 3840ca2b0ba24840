// psgld_internal.cuh -- shared declarations of the CUDA PSGLD library.
//
// Device layout (all in HBM, owned by the context):
//   W[2]  : I x ldk fp32, row-major, ping-pong pair (ldk = 4*ceil(K/4); the
//           padding columns are kept at zero so every row is float4-aligned)
//   Ht[2] : J x ldk fp32, H transposed, same rules
//   G     : (I + J) x ldk fp32, the likelihood gradient of the current
//           part-step (rows 0..I-1 for W, I..I+J-1 for H^T)
//   A-side layout (part-major CSR): entries ordered by (part s, row i, col j)
//           ptrA[s*I + i] .. ptrA[s*I + i + 1] -> idxA (col j), valA (v)
//   B-side layout (part-major CSC): entries ordered by (part s, col j, row i)
//           ptrB[s*J + j] .. -> idxB (row i), valB (v)
//   segA/segB : per part, the chunk records of the fused part-step kernel:
//           one per (heavy row, run of at most chunk_len entries)
//   posterior sums: fp64 copies of W, W^2, Ht, Ht^2 (padded like the factors)
//   dense tensor-core path instead of the two layouts:
//   Vd    : I x J fp32, row-major (ldv = J)
//   hpart : mtiles x J x ldk fp32, the per-M-tile partial G_H rows when a
//           block has more than one 128-row tile (single-pass kernel)
//   two-sided kernel: VA, V in 128 x 64 tiles per block (128 rows x 64
//           columns); Wsh / Hsh, BF16 shadows of W and H^T in 64-row
//           swizzled MMA tiles per piece (dev::shadow_store4); Et, one part's
//           E in 128 x 64 BF16 tiles (written by the rows items, read by the
//           columns items); tsync, the kernel's claim and block counters
//   sparse path with gather_bf16: W16 / H16, BF16 copies of W and H^T, rows
//           of ldk rounded up to 8, rewritten by every update
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/psgld.h"

namespace psgld {

constexpr int kMaxK = 512;

struct SideLayout {
    int32_t *ptr = nullptr;    // B*n_rows + 1 entry offsets (absolute)
    int32_t *idx = nullptr;    // other index of each entry
    float *val = nullptr;      // value of each entry
    int32_t *own = nullptr;    // own row of each entry
    std::vector<int64_t> part_first;   // B+1: first entry of each part
    int64_t max_units = 0;     // most units (unit_entries consecutive entries) in one part
    float *partial = nullptr;  // 2 x max_units x ldk: head / tail partial
                               // sums of rows that cross a unit boundary
};

struct Sums {
    double *s = nullptr, *s2 = nullptr;
};

// psgld_batch_sweep's captured sweeps, kept by the list's first context: one
// graph per parity of the ping-pong buffers and per accumulation flag, valid
// while the batch's launch structure (key) is unchanged.
struct BatchGraphs {
    std::vector<int64_t> key;
    int64_t calls = 0;           // consecutive calls with this key
    cudaGraphExec_t exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
};

}  // namespace psgld

struct psgld_ctx {
    int64_t I = 0, J = 0;
    int32_t K = 0, B = 0, ldk = 0, ngroups = 0;
    double p = 0.0, phi = 1.0;
    psgld_prior prior{};
    psgld_options opt{};
    int device = 0;
    std::string err;

    // data
    bool has_data = false;
    int64_t N = 0;
    std::vector<int64_t> part_n;     // observed entries of each part
    psgld::SideLayout side[2];       // 0: rows of W (CSR), 1: rows of Ht (CSC)
    bool dense = false;              // data kept dense for the tensor-core path
    float *Vd = nullptr;             // I x ldv fp32 (dense path)
    int64_t ldv = 0;
    float *hpart = nullptr;          // mtiles x J x ldk partial G_H rows (mtiles > 1)
    int mtiles = 0;                  // 128-row tiles of the largest row piece
    int dense_kind = 0;              // 1: single-pass kernel, 2: two-sided kernel
    int dense_fp8 = 0;               // single-pass kernel with the E4M3 GEMM1
    int KP = 0;                      // K rounded up to 64 (two-sided kernel)
    int v_bf16 = 0;                  // V tiles in BF16
    void *VA = nullptr;                         // V tiles (rows of V owned)
    void *VB = nullptr;                         // ... columns owned (columns items forming their own mu)
    int share_e = 0;                            // columns items take E from the rows items
    uint16_t *Et = nullptr;                     // E tiles of one part (BF16)
    int *tsync = nullptr;                       // two-sided kernel counters: 2 + B ints
    uint16_t *Wsh = nullptr, *Hsh = nullptr;    // BF16 shadows of W, H^T
    uint16_t *W16 = nullptr, *H16 = nullptr;    // sparse path, gather_bf16: BF16 copies of W, H^T
    int mt_max = 0, nt_max = 0;      // 128-row tiles per row piece / column piece
    int nt2_max = 0;                 // 256-row column tiles per column piece (columns items)
    int ni_max = 0, nj_max = 0;      // 64-row tiles per row piece / column piece

    // factors
    float *W[2] = {nullptr, nullptr};
    float *Ht[2] = {nullptr, nullptr};
    float *G = nullptr;              // (I + J) x ldk likelihood gradients of one part-step
    int wcur = 0, hcur = 0;
    bool has_factors = false;

    // posterior
    psgld::Sums sW, sH;
    int64_t n_samples = 0;
    int64_t sweeps_done = 0;
    int64_t t_done = 0;

    // device memory: the caller's allocator, if one was set at create
    psgld_allocator allocator{};
    bool has_allocator = false;

    // reductions
    double *red = nullptr;                 // per-CTA partial sums
    std::vector<double> red_host;          // host copy
    int *flag = nullptr;         // device error flag of the layout build and input checks
    int *kflag = nullptr;        // device error flag of the sampling kernels (16: wait ran out)
    cudaStream_t last_stream = nullptr;   // stream of the latest enqueued work
    cudaEvent_t last_ev = nullptr;         // recorded after it (when last_ev_set)
    bool last_ev_set = false;

    // CUDA graphs of one sweep, per parity of the ping-pong buffers, without
    // and with the posterior accumulation
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    cudaGraphExec_t graph_acc[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t capture_stream = nullptr;
    int64_t *t_dev = nullptr;    // iteration counter read by graph replays
    // sparse part-steps: the rows of H^T on a second stream, forked from and
    // joined back into the launch stream
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    psgld::BatchGraphs bgraphs;  // captured batch sweeps while this context leads a batch

    // psgld_batch_sweep's parameter tables while this context leads a batch
    // (is first in the list): device copy, its size, an event recorded after
    // the last launch that read it, and the host staging buffer
    void *bscratch = nullptr;
    size_t bscratch_bytes = 0;
    cudaEvent_t bdone = nullptr;
    std::vector<unsigned char> btab;

    // profiling: one event pair per part (start, end), and which are unread
    std::vector<cudaEvent_t> ev_start, ev_mid, ev_end;   // mid: after the gradient kernel
    std::vector<char> ev_pending;
};

namespace psgld {

// ---- device memory ---------------------------------------------------------
// Through the context's allocator, or cudaMalloc / cudaFree.  dev_alloc
// returns nullptr on failure; dev_free(nullptr) does nothing.
void *dev_alloc(psgld_ctx *c, size_t bytes, cudaStream_t st);
void dev_free(psgld_ctx *c, void *p, cudaStream_t st = nullptr);

// ---- ordering ----------------------------------------------------------------
// After enqueueing work of c on st: remember the stream and record an event
// behind the work.  wait_enqueued blocks until that work has run (not the
// rest of the stream), or syncs the last stream if no event was recorded.
void mark_enqueued(psgld_ctx *c, cudaStream_t st);
cudaError_t wait_enqueued(psgld_ctx *c);

// ---- error plumbing ------------------------------------------------------
psgld_status fail(psgld_ctx *c, psgld_status s, const std::string &msg);
psgld_status cuda_fail(psgld_ctx *c, cudaError_t e, const char *what);

#define PSGLD_CK(ctx, call)                                        \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return psgld::cuda_fail((ctx), e_, #call); \
    } while (0)

// ---- layout (psgld_layout.cu) ---------------------------------------------
psgld_status build_layout(psgld_ctx *c, int64_t nnz, const int32_t *i_dev,
                          const int32_t *j_dev, const float *v_dev,
                          cudaStream_t st);
void free_layout(psgld_ctx *c);

// ---- part schedule (psgld_api.cu) ------------------------------------------
// Index s of the part used at iteration t (blocks (r, (r + s) mod B)):
// cyclic, or the size-proportional draw of part_mode 1.
int part_of_iteration(const psgld_ctx *c, int64_t t);

// ---- part-step (psgld_step.cu) --------------------------------------------
// Enqueue iteration t.  When t_dev is non-null the kernels read t from
// *t_dev + t_add instead (used inside captured graphs); `t` then only
// selects the part and must satisfy (t-1) % B == part.
// Sparse path with gather_bf16: the gradient kernel gathers BF16 copies of
// the factors (rows of ldk rounded up to 8), kept by the update kernel and
// built from the current factors by build_gather_shadows (allocating them).
bool gather_bf16(const psgld_ctx *c);
psgld_status build_gather_shadows(psgld_ctx *c, cudaStream_t st);

psgld_status launch_part_step(psgld_ctx *c, int64_t t, const int64_t *t_dev,
                              int64_t t_add, cudaStream_t st);

// One-time kernel attributes (dynamic shared memory) for this context's K.
psgld_status prepare_kernels(psgld_ctx *c);
// Entries per work unit of the gradient kernel for a factor width of
// ngroups float4 groups.
int unit_entries(int ngroups);
// After a synchronisation point: PSGLD_ERR_TIMEOUT (and the flag cleared) if
// a sampling kernel reported a bounded wait that ran out, else PSGLD_OK.
psgld_status check_kernel_flag(psgld_ctx *c);

// ---- dense tensor-core path (psgld_dense.cu) --------------------------------
bool dense_supported(int K);
// 128-row tiles of the largest row piece (CTAs per block).
int dense_mtiles(const psgld_ctx *c);
// Chooses the kernel (options dense_path, dense_v_bf16; K; block sizes),
// sets its attributes and allocates the two-sided kernel's tiles.
psgld_status prepare_dense(psgld_ctx *c, cudaStream_t st);
// Whether the two-sided kernel's columns items take E from the rows items
// (opt >= 0: as given; -1: long row pieces and more than one wave of items).
int two_sided_share(int opt, int64_t max_rows, int B, int mt, int nt, int sms);
// V tiles of the two-sided kernel from c->Vd (no-op for the single-pass one).
psgld_status build_dense_tiles(psgld_ctx *c, cudaStream_t st);
// BF16 shadows of the current factors (two-sided kernel with factors set).
psgld_status build_dense_shadows(psgld_ctx *c, cudaStream_t st);
// Enqueue the gradient kernel of part `part`: G rows of W (and of Ht when
// mtiles == 1) or hpart rows of Ht.
psgld_status launch_dense_grad(psgld_ctx *c, int part, cudaStream_t st);

// ---- many contexts in shared launches (psgld_batch_sweep) -----------------
// Each launch reads a device table of per-context kernel parameters; the
// fill_* functions write one context's entry into host memory (with the
// context's current ping-pong buffers) and return its share of the grid:
// CTAs, update items or float4 accumulation units.  The *_start arrays are
// exclusive prefix sums of those shares (n + 1 entries, device memory).
// Dense: contexts of one batch key (> 0): single-pass ones of one K class
// and GEMM1 precision (one CTA range each), or two-sided ones of one K
// width, V type and power (one persistent launch over all their items).
// Every table slot is dense_param_bytes() long.  fill_dense_param returns
// the context's items and sets *first_items to those of the first kind
// (two-sided: the rows items; single-pass: all).  A two-sided group's
// cta_start holds two prefix arrays of n + 1 entries: rows items, then
// columns items.
int dense_batch_key(const psgld_ctx *c);
size_t dense_param_bytes();
int fill_dense_param(const psgld_ctx *c, int part, void *dst, int *first_items);
psgld_status launch_dense_batch(psgld_ctx *c0, int key, const void *params, const int *cta_start, int n,
                                int total, cudaStream_t st);
// Update of part `part` at iteration *t_dev + t_add (t_dev: the context's
// device counter); does not flip the context's buffers.
size_t upd_param_bytes();
int64_t fill_upd_param(psgld_ctx *c, int part, const int64_t *t_dev, int64_t t_add, void *dst);
psgld_status launch_update_batch(psgld_ctx *c0, const void *params, const int64_t *item_start, int n,
                                 int64_t total_items, cudaStream_t st);
// Posterior sums: a context takes the sample when (*t_dev - t0) / B >= acc_from.
size_t acc_param_bytes();
int64_t fill_acc_param(psgld_ctx *c, int64_t t0, int64_t acc_from, void *dst);
psgld_status launch_accumulate_batch(psgld_ctx *c0, const void *params, const int64_t *unit_start, int n,
                                     int64_t total_units, cudaStream_t st);
// mode 0: every context's *t_dev = t0; mode 1: *t_dev += B.
psgld_status launch_t_batch(psgld_ctx *c0, const void *params, int n, int mode, cudaStream_t st);

// ---- reductions (psgld_reduce.cu) -----------------------------------------
psgld_status launch_accumulate(psgld_ctx *c, cudaStream_t st);
psgld_status launch_advance_t(psgld_ctx *c, int64_t by, cudaStream_t st);
psgld_status reduce_loglik_rmse(psgld_ctx *c, int mode, int use_mean,
                                cudaStream_t st, double *out);

// ---- scans and sorts (psgld_layout.cu) ------------------------------------
int bits_for(uint64_t n_values);

}  // namespace psgld

// ---- device helpers -------------------------------------------------------
namespace psgld {
namespace dev {

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64-bit
// multiplies whose high halves are mixed into the other two words with the
// round key; the key advances by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Uniform on (0, 1): the top 23 bits plus one half, times 2^-23 (exact in
// fp32).  Then Box-Muller on (u0, u1) and (u2, u3): cos first, then sin.
__device__ __forceinline__ float4 box_muller4(uint4 x)
{
    const float s = 1.0f / 8388608.0f;
    const float u0 = (__uint2float_rn(x.x >> 9) + 0.5f) * s;
    const float u1 = (__uint2float_rn(x.y >> 9) + 0.5f) * s;
    const float u2 = (__uint2float_rn(x.z >> 9) + 0.5f) * s;
    const float u3 = (__uint2float_rn(x.w >> 9) + 0.5f) * s;
    const float r0 = sqrtf(-2.0f * logf(u0));
    const float r1 = sqrtf(-2.0f * logf(u2));
    float s0, c0, s1, c1;
    sincospif(2.0f * u1, &s0, &c0);
    sincospif(2.0f * u3, &s1, &c1);
    return make_float4(r0 * c0, r0 * s0, r1 * c1, r1 * s1);
}

// BF16 copy of 4 factor entries (row, k0 .. k0+3, k0 % 4 == 0) into the MMA
// tiles of the two-sided dense kernel.  Rows of piece r (Definition 1) fill
// `tiles` 64-row tiles starting at tile r * tiles.  A tile holds KP / 64
// atoms of 64 rows x 128 bytes (64 entries of k), one after the other; in
// row rho of an atom, the 16-byte chunk of entries 8c .. 8c+7 sits at chunk
// position c ^ (rho % 8) -- the 128-byte swizzle that the tensor core's
// operand reads expect (the pattern repeats every 8 rows = 1024 bytes).
__device__ __forceinline__ void shadow_store4(uint16_t *sh, int64_t row, int k0, float4 v, int64_t n,
                                              int B, int tiles, int KP)
{
    // 32-bit arithmetic: rows and B * n are below 2^31 (checked at create)
    const uint32_t piece = ((uint32_t)(row + 1) * (uint32_t)B - 1u) / (uint32_t)n;
    const int64_t rr = row - (int64_t)((piece * (uint32_t)n) / (uint32_t)B);
    const int rho = (int)(rr & 63);
    const int kk = k0 & 63, c = kk >> 3;
    const int64_t off = (piece * tiles + (rr >> 6)) * 64 * KP + (int64_t)(k0 >> 6) * 4096 +
                        rho * 64 + ((c ^ (rho & 7)) << 3) + (kk & 7);
    __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
    *reinterpret_cast<uint2 *>(sh + off) =
        make_uint2(*reinterpret_cast<uint32_t *>(&lo), *reinterpret_cast<uint32_t *>(&hi));
}

}  // namespace dev
}  // namespace psgld
