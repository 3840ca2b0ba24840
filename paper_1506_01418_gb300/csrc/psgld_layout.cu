// psgld_layout.cu -- device construction of the part-major layouts.
//
// Blocks and parts (Definitions 1 and 2 of the paper): row piece r of [I] is
// [floor(r I / B), floor((r+1) I / B)); at iteration t the part pairs row
// piece r with column piece (r + s) mod B, s = (t-1) mod B.  So an observed
// entry (i, j) belongs to the part s = (piece(j) - piece(i)) mod B, and the
// layouts group entries by part:
//   A side: key (s*I + i, j)  -> CSR of every part over all I rows
//   B side: key (s*J + j, i)  -> CSC of every part over all J columns
// Both are produced by a stable LSD radix sort written here (8-bit digits,
// per-tile histograms, a global exclusive scan and a stable scatter whose
// in-tile ranks come from warp match/ballot), so the order is exact and
// repeatable.  Every entry also records its own row (the row of W for the
// A side, the row of H^T for the B side), so that the part-step kernel can
// take any 32 consecutive entries of a part as one unit of work.
#include <algorithm>

#include "psgld_internal.cuh"

namespace psgld {

int bits_for(uint64_t n_values)
{
    int b = 0;
    while (b < 64 && (n_values > (1ull << b))) ++b;
    return b;
}

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan of one tile held in shared memory (n <= kScanTile valid
// values, the rest zero); returns the tile total to thread 0.
__device__ uint32_t block_exclusive_scan(uint32_t *sm, int n)
{
    __shared__ uint32_t warp_tot[kScanThreads / 32];
    const int tid = threadIdx.x;
    uint32_t v[kScanItems];
    uint32_t run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int a = tid * kScanItems + k;
        v[k] = a < n ? sm[a] : 0u;
        run += v[k];
    }
    // inclusive warp scan of the per-thread totals
    const int lane = tid & 31, warp = tid >> 5;
    uint32_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;  // exclusive
    }
    __syncthreads();
    uint32_t base = warp_tot[warp] + inc - run;
    uint32_t total = 0;
    if (tid == kScanThreads - 1) total = base + run;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int a = tid * kScanItems + k;
        if (a < n) sm[a] = base;
        base += v[k];
    }
    __syncthreads();
    return total;
}

__global__ void scan_tile_sums(const uint32_t *__restrict__ in, int64_t n,
                               uint32_t *__restrict__ sums)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t s = 0;
    for (int k = threadIdx.x; k < kScanTile; k += kScanThreads)
        if (base + k < n) s += in[base + k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ uint32_t ws[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

// One CTA scans the tile sums in place (exclusive), tile by tile with a carry.
__global__ void scan_sums_single(uint32_t *sums, int64_t n, uint32_t *total)
{
    __shared__ uint32_t sm[kScanTile];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += kScanTile) {
        const int m = (int)(n - base < kScanTile ? n - base : kScanTile);
        for (int k = threadIdx.x; k < kScanTile; k += kScanThreads)
            sm[k] = k < m ? sums[base + k] : 0u;
        __syncthreads();
        uint32_t t = block_exclusive_scan(sm, m);
        const uint32_t cbase = carry;
        for (int k = threadIdx.x; k < m; k += kScanThreads) sums[base + k] = sm[k] + cbase;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry = cbase + t;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void scan_tiles(const uint32_t *__restrict__ in, int64_t n,
                           const uint32_t *__restrict__ sums, uint32_t *__restrict__ out)
{
    __shared__ uint32_t sm[kScanTile];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    const int m = (int)(n - base < kScanTile ? n - base : kScanTile);
    for (int k = threadIdx.x; k < kScanTile; k += kScanThreads)
        sm[k] = k < m ? in[base + k] : 0u;
    __syncthreads();
    block_exclusive_scan(sm, m);
    const uint32_t off = sums[blockIdx.x];
    for (int k = threadIdx.x; k < m; k += kScanThreads) out[base + k] = sm[k] + off;
}

// ---- radix sort -----------------------------------------------------------

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048 keys per CTA
constexpr int kSortWarps = kSortThreads / 32;

__global__ void radix_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                           uint32_t *__restrict__ hist, int64_t ntiles)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int k = threadIdx.x; k < kSortTile; k += kSortThreads)
        if (base + k < n) atomicAdd(&h[(keys[base + k] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter.  Warp w of the tile owns positions [w*256, (w+1)*256);
// item m of lane l is position w*256 + m*32 + l, so (w, m, l) order is
// position order.  Ranks among equal digits come from __match_any_sync.
__global__ void radix_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                              int64_t n, int shift, const uint32_t *__restrict__ offs,
                              int64_t ntiles, uint64_t *__restrict__ kout,
                              uint32_t *__restrict__ vout)
{
    __shared__ uint32_t wcnt[kSortWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kSortWarps * 256; d += kSortThreads) (&wcnt[0][0])[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile + warp * 256;
    const uint32_t lt = (1u << lane) - 1u;
    uint64_t key[kSortItems];
    uint32_t val[kSortItems], rank[kSortItems];
    int dig[kSortItems];
#pragma unroll
    for (int m = 0; m < kSortItems; ++m) {
        const int64_t pos = base + m * 32 + lane;
        const bool ok = pos < n;
        key[m] = ok ? kin[pos] : 0ull;
        val[m] = ok ? vin[pos] : 0u;
        dig[m] = ok ? (int)((key[m] >> shift) & 255u) : 256 + lane;  // invalid: unique
        const unsigned peers = __match_any_sync(0xffffffffu, dig[m]);
        const uint32_t before = ok ? wcnt[warp][dig[m]] : 0u;
        rank[m] = before + __popc(peers & lt);
        __syncwarp();
        if (ok && (peers & lt) == 0) wcnt[warp][dig[m]] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {   // exclusive prefix over warps, one digit per thread
        const int d = threadIdx.x;
        uint32_t run = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < kSortItems; ++m) {
        if (dig[m] < 256) {
            const uint32_t dst = offs[(int64_t)dig[m] * ntiles + blockIdx.x] + wcnt[warp][dig[m]] + rank[m];
            kout[dst] = key[m];
            vout[dst] = val[m];
        }
    }
}

// ---- layout kernels ---------------------------------------------------------

__device__ __forceinline__ int64_t piece_of(int64_t x, int64_t n, int B)
{
    // largest r with floor(r n / B) <= x
    return ((x + 1) * B - 1) / n;
}

__global__ void validate_and_key(int64_t nnz, const int32_t *__restrict__ ii,
                                 const int32_t *__restrict__ jj, const float *__restrict__ vv,
                                 int64_t I, int64_t J, int B, int nonneg, int bitsI, int bitsJ,
                                 uint64_t *__restrict__ keyA, uint64_t *__restrict__ keyB,
                                 uint32_t *__restrict__ valA, uint32_t *__restrict__ valB,
                                 int *flag)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = ii[e], j = jj[e];
        const float v = vv[e];
        if (i < 0 || i >= I || j < 0 || j >= J) { atomicOr(flag, 1); continue; }
        if (!isfinite(v) || (nonneg && v < 0.0f)) atomicOr(flag, 2);
        const int64_t rp = piece_of(i, I, B), cp = piece_of(j, J, B);
        const int64_t s = (cp - rp + B) % B;
        keyA[e] = ((uint64_t)(s * I + i) << bitsJ) | (uint64_t)j;
        keyB[e] = ((uint64_t)(s * J + j) << bitsI) | (uint64_t)i;
        valA[e] = (uint32_t)e;
        valB[e] = (uint32_t)e;
    }
}

// Gather sorted entries; flag duplicates; fill the slot pointer array.
__global__ void finish_side(int64_t nnz, const uint64_t *__restrict__ key,
                            const uint32_t *__restrict__ perm, const int32_t *__restrict__ other,
                            const float *__restrict__ vv, int bits_other, int64_t nslots,
                            int64_t n_rows, int32_t *__restrict__ idx, float *__restrict__ val,
                            int32_t *__restrict__ own, int32_t *__restrict__ ptr, int *flag)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slot = p < nnz ? (int64_t)(key[p] >> bits_other) : nslots;
        const int64_t prev = p > 0 ? (int64_t)(key[p - 1] >> bits_other) : -1;
        for (int64_t s = prev + 1; s <= slot; ++s) ptr[s] = (int32_t)p;
        if (p < nnz) {
            const uint32_t e = perm[p];
            idx[p] = other[e];
            val[p] = vv[e];
            own[p] = (int32_t)(slot % n_rows);
            if (p > 0 && key[p] == key[p - 1]) atomicOr(flag, 4);
        }
    }
}

__global__ void gather_ptr(const int32_t *__restrict__ ptr, int64_t n_rows, int B,
                           int64_t *__restrict__ out)
{
    const int s = threadIdx.x;
    if (s <= B) out[s] = ptr[(int64_t)s * n_rows];
}

int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

template <typename T>
psgld_status dmalloc(psgld_ctx *c, T **p, int64_t n)
{
    if (n <= 0) n = 1;
    // whole 256-byte granules, so that 16-byte-rounded bulk prefetches of any
    // sub-range stay inside the allocation
    const size_t bytes = (sizeof(T) * (size_t)n + 255) & ~size_t(255);
    *p = static_cast<T *>(dev_alloc(c, bytes, nullptr));
    if (!*p) return fail(c, PSGLD_ERR_OOM, "device allocation of " + std::to_string(sizeof(T) * n) + " bytes failed");
    return PSGLD_OK;
}

// Exclusive scan of n uint32 values (in -> out, out has n+1 entries; out[n]
// is the total).  tmp needs ceil(n / kScanTile) + 1 entries.
psgld_status exclusive_scan(psgld_ctx *c, const uint32_t *in, uint32_t *out, int64_t n,
                            uint32_t *tmp, cudaStream_t st)
{
    const int64_t tiles = std::max<int64_t>(1, (n + kScanTile - 1) / kScanTile);
    scan_tile_sums<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, tmp);
    scan_sums_single<<<1, kScanThreads, 0, st>>>(tmp, tiles, out + n);
    scan_tiles<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, tmp, out);
    PSGLD_CK(c, cudaGetLastError());
    return PSGLD_OK;
}

psgld_status radix_sort(psgld_ctx *c, uint64_t *&k0, uint32_t *&v0, uint64_t *&k1,
                        uint32_t *&v1, int64_t n, int bits, uint32_t *hist, uint32_t *hist_scan,
                        uint32_t *tmp, cudaStream_t st)
{
    const int64_t ntiles = std::max<int64_t>(1, (n + kSortTile - 1) / kSortTile);
    for (int shift = 0; shift < bits; shift += 8) {
        radix_hist<<<(unsigned)ntiles, kSortThreads, 0, st>>>(k0, n, shift, hist, ntiles);
        psgld_status s = exclusive_scan(c, hist, hist_scan, 256 * ntiles, tmp, st);
        if (s != PSGLD_OK) return s;
        radix_scatter<<<(unsigned)ntiles, kSortThreads, 0, st>>>(k0, v0, n, shift, hist_scan,
                                                                 ntiles, k1, v1);
        PSGLD_CK(c, cudaGetLastError());
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    return PSGLD_OK;
}

}  // namespace

void free_layout(psgld_ctx *c)
{
    // work that reads the layouts must be finished before they are handed back
    wait_enqueued(c);
    if (c->capture_stream) cudaStreamSynchronize(c->capture_stream);
    for (auto &sd : c->side) {
        dev_free(c, sd.ptr); dev_free(c, sd.idx); dev_free(c, sd.val); dev_free(c, sd.own);
        dev_free(c, sd.partial);
        sd = SideLayout{};
    }
    dev_free(c, c->Vd);
    dev_free(c, c->hpart);
    dev_free(c, c->VA);
    dev_free(c, c->VB);
    dev_free(c, c->Et);
    dev_free(c, c->tsync);
    dev_free(c, c->Wsh);
    dev_free(c, c->Hsh);
    c->Vd = nullptr;
    c->hpart = nullptr;
    c->VA = c->VB = nullptr;
    c->Et = nullptr;
    c->tsync = nullptr;
    c->Wsh = c->Hsh = nullptr;
    c->dense_kind = 0;
    c->dense_fp8 = 0;
    c->dense = false;
    c->ldv = 0;
    c->mtiles = 0;
    c->has_data = false;
    c->N = 0;
    c->part_n.clear();
}

psgld_status build_layout(psgld_ctx *c, int64_t nnz, const int32_t *i_dev, const int32_t *j_dev,
                          const float *v_dev, cudaStream_t st)
{
    free_layout(c);
    const int64_t I = c->I, J = c->J;
    const int B = c->B;
    const int bitsI = bits_for((uint64_t)I), bitsJ = bits_for((uint64_t)J);
    const int bitsA = bits_for((uint64_t)(B * I)) + bitsJ;
    const int bitsB = bits_for((uint64_t)(B * J)) + bitsI;
    const int64_t n = nnz;

    uint64_t *kA = nullptr, *kB = nullptr, *kt = nullptr;
    uint32_t *pA = nullptr, *pB = nullptr, *pt = nullptr;
    uint32_t *hist = nullptr, *hscan = nullptr, *tmp = nullptr;
    const int64_t ntiles = std::max<int64_t>(1, (n + kSortTile - 1) / kSortTile);
    const int64_t nslots_max = (int64_t)B * std::max(I, J);
    const int64_t scan_n = std::max<int64_t>(256 * ntiles + 1, nslots_max + 1);
    const int64_t tmp_n = (scan_n + kScanTile - 1) / kScanTile + 2;
    psgld_status s = PSGLD_OK;
    std::vector<void *> scratch;
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);   // the scratch is in use by work on st
        for (void *p : scratch) dev_free(c, p, st);
    };
#define PSGLD_ALLOC(ptr, cnt)                      \
    do {                                           \
        s = dmalloc(c, &(ptr), (cnt));             \
        if (s != PSGLD_OK) { cleanup(); free_layout(c); return s; } \
        scratch.push_back((void *)(ptr));          \
    } while (0)
    PSGLD_ALLOC(kA, n); PSGLD_ALLOC(kB, n); PSGLD_ALLOC(kt, n);
    PSGLD_ALLOC(pA, n); PSGLD_ALLOC(pB, n); PSGLD_ALLOC(pt, n);
    PSGLD_ALLOC(hist, scan_n); PSGLD_ALLOC(hscan, scan_n + 1); PSGLD_ALLOC(tmp, tmp_n);
    int64_t *offs_dev = nullptr;
    PSGLD_ALLOC(offs_dev, B + 1);
#undef PSGLD_ALLOC

    auto ck = [&](cudaError_t e, const char *what) -> psgld_status {
        if (e != cudaSuccess) { cleanup(); free_layout(c); return cuda_fail(c, e, what); }
        return PSGLD_OK;
    };
    if ((s = ck(cudaMemsetAsync(c->flag, 0, sizeof(int), st), "memset flag")) != PSGLD_OK) return s;
    if (n > 0)
        validate_and_key<<<grid_for(n, 256), 256, 0, st>>>(n, i_dev, j_dev, v_dev, I, J, B,
                                                           c->prior.kind == PSGLD_PRIOR_EXPONENTIAL,
                                                           bitsI, bitsJ, kA, kB, pA, pB, c->flag);
    if ((s = ck(cudaGetLastError(), "validate_and_key")) != PSGLD_OK) return s;
    int hflag = 0;
    if ((s = ck(cudaMemcpyAsync(&hflag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st), "flag d2h")) != PSGLD_OK) return s;
    if ((s = ck(cudaStreamSynchronize(st), "sync")) != PSGLD_OK) return s;
    if (hflag & 1) { cleanup(); free_layout(c); return fail(c, PSGLD_ERR_ARG, "entry index out of range"); }
    if (hflag & 2) { cleanup(); free_layout(c); return fail(c, PSGLD_ERR_ARG, "entry value not finite, or negative in a non-negative model"); }

    for (int side = 0; side < 2; ++side) {
        SideLayout &sd = c->side[side];
        const int64_t n_rows = side == 0 ? I : J;
        const int64_t nslots = (int64_t)B * n_rows;
        uint64_t *k0 = side == 0 ? kA : kB;
        uint32_t *v0 = side == 0 ? pA : pB;
        uint64_t *k1 = kt;   // free again: the other side's finish_side ran first
        uint32_t *v1 = pt;
        if (n > 0) {
            s = radix_sort(c, k0, v0, k1, v1, n, side == 0 ? bitsA : bitsB, hist, hscan, tmp, st);
            if (s != PSGLD_OK) { cleanup(); free_layout(c); return s; }
        }
        s = dmalloc(c, &sd.ptr, nslots + 1);
        if (s == PSGLD_OK) s = dmalloc(c, &sd.idx, n);
        if (s == PSGLD_OK) s = dmalloc(c, &sd.val, n);
        if (s == PSGLD_OK) s = dmalloc(c, &sd.own, n);
        if (s != PSGLD_OK) { cleanup(); free_layout(c); return s; }
        finish_side<<<grid_for(n + 1, 256), 256, 0, st>>>(n, k0, v0, side == 0 ? j_dev : i_dev, v_dev,
                                                          side == 0 ? bitsJ : bitsI, nslots, n_rows,
                                                          sd.idx, sd.val, sd.own, sd.ptr, c->flag);
        if ((s = ck(cudaGetLastError(), "finish_side")) != PSGLD_OK) return s;
        gather_ptr<<<1, 128, 0, st>>>(sd.ptr, n_rows, B, offs_dev);
        std::vector<int64_t> h(B + 1);
        if ((s = ck(cudaMemcpyAsync(h.data(), offs_dev, sizeof(int64_t) * h.size(), cudaMemcpyDeviceToHost, st), "offsets d2h")) != PSGLD_OK) return s;
        if ((s = ck(cudaStreamSynchronize(st), "sync")) != PSGLD_OK) return s;
        sd.part_first = h;
        if (side == 0) {
            c->part_n.resize(B);
            for (int p = 0; p < B; ++p) c->part_n[p] = h[p + 1] - h[p];
        }
        const int unit = unit_entries(c->ngroups);
        sd.max_units = 0;
        for (int p = 0; p < B; ++p)
            sd.max_units = std::max<int64_t>(sd.max_units, (h[p + 1] - h[p] + unit - 1) / unit);
        s = dmalloc(c, &sd.partial, 2 * std::max<int64_t>(1, sd.max_units) * c->ldk);
        if (s != PSGLD_OK) { cleanup(); free_layout(c); return s; }
    }
    if ((s = ck(cudaMemcpyAsync(&hflag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st), "flag d2h")) != PSGLD_OK) return s;
    if ((s = ck(cudaStreamSynchronize(st), "sync")) != PSGLD_OK) return s;
    cleanup();
    if (hflag & 4) { free_layout(c); return fail(c, PSGLD_ERR_ARG, "duplicate (i, j) entry"); }
    c->N = n;
    c->has_data = true;
    return PSGLD_OK;
}

}  // namespace psgld
