// psgld_api.cu -- the C ABI declared in include/psgld.h.
//
// The context owns every device buffer (factors, layouts, scratch, FP64
// posterior sums).  Sweeps are either launched kernel by kernel or, with
// use_graphs, replayed from a CUDA graph holding the B part-step launches of
// one sweep (plus the posterior accumulation and the iteration-counter
// advance).  The graph reads the iteration index t from device memory, so
// one captured graph serves every sweep; one graph is kept per parity of the
// ping-pong factor buffers and per accumulate / no-accumulate variant.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

#include "psgld_context.cuh"

namespace psgld {

int reduce_blocks();

namespace {
std::mutex g_alloc_mutex;
psgld_allocator g_allocator{};
bool g_has_allocator = false;
}  // namespace

void *dev_alloc(psgld_ctx *c, size_t bytes, cudaStream_t st)
{
    if (bytes == 0) bytes = 256;
    if (c->has_allocator) return c->allocator.alloc(bytes, (void *)st, c->allocator.user);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(psgld_ctx *c, void *p, cudaStream_t st)
{
    if (!p) return;
    if (c->has_allocator) c->allocator.free(p, (void *)st, c->allocator.user);
    else cudaFree(p);
}

void mark_enqueued(psgld_ctx *c, cudaStream_t st)
{
    c->last_stream = st;
    c->last_ev_set = false;
    if (!c->last_ev && cudaEventCreateWithFlags(&c->last_ev, cudaEventDisableTiming) != cudaSuccess) {
        c->last_ev = nullptr;
        cudaGetLastError();
        return;
    }
    if (cudaEventRecord(c->last_ev, st) == cudaSuccess) c->last_ev_set = true;
    else cudaGetLastError();
}

cudaError_t wait_enqueued(psgld_ctx *c)
{
    if (c->last_ev && c->last_ev_set) return cudaEventSynchronize(c->last_ev);
    return cudaStreamSynchronize(c->last_stream);
}

psgld_status fail(psgld_ctx *c, psgld_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

psgld_status cuda_fail(psgld_ctx *c, cudaError_t e, const char *what)
{
    cudaGetLastError();
    return fail(c, PSGLD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Philox4x32-10 on the host (Salmon et al., SC'11): ten rounds of the two
// 32 x 32 -> 64-bit products, key bumped by the Weyl constants.
static void host_philox(const uint32_t ctr[4], uint64_t seed, uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * x0, p1 = (uint64_t)0xCD9E8D57u * x2;
        const uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0, y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        x0 = y0; x1 = (uint32_t)p1; x2 = y2; x3 = (uint32_t)p0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

int part_of_iteration(const psgld_ctx *c, int64_t t)
{
    const int B = c->B;
    if (c->opt.part_mode == 0 || c->N == 0 || (int)c->part_n.size() != B)
        return (int)((t - 1) % B);
    const uint32_t ctr[4] = {0u, 0xFFFFFFFFu, (uint32_t)(uint64_t)t, (uint32_t)((uint64_t)t >> 32) << 1};
    uint32_t x[4];
    host_philox(ctr, c->opt.seed, x);
    const uint64_t x64 = ((uint64_t)x[1] << 32) | x[0];
    const uint64_t r = (uint64_t)(((unsigned __int128)x64 * (uint64_t)c->N) >> 64);
    uint64_t cum = 0;
    for (int s = 0; s < B; ++s) {
        cum += (uint64_t)c->part_n[s];
        if (r < cum) return s;
    }
    return B - 1;
}

psgld_status check_kernel_flag(psgld_ctx *c)
{
    int h = 0;
    PSGLD_CK(c, cudaMemcpy(&h, c->kflag, sizeof(int), cudaMemcpyDeviceToHost));
    if (h == 0) return PSGLD_OK;
    PSGLD_CK(c, cudaMemset(c->kflag, 0, sizeof(int)));
    std::string where;
    if (h & 16) where += " sparse gradient kernel (wait for the row gathers);";
    if (h & 32) where += " single-pass dense kernel (MMA completion);";
    if (h & 64) where += " two-sided dense kernel";
    if (h & 128) where += " (producer: free slot)";
    if (h & 256) where += " (MMA warp: data or epilogue)";
    if (h & 512) where += " (epilogue: data or MMA)";
    return fail(c, PSGLD_ERR_TIMEOUT, "a bounded wait in a part-step kernel ran out:" + where);
}

namespace {

__global__ void dense_to_coo_kernel(const float *__restrict__ V, int64_t I, int64_t J, int64_t ld,
                                    int32_t *__restrict__ ii, int32_t *__restrict__ jj,
                                    float *__restrict__ vv)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < I * J;
         a += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = a / J, j = a - i * J;
        ii[a] = (int32_t)i;
        jj[a] = (int32_t)j;
        vv[a] = V[i * ld + j];
    }
}

__global__ void check_factors_kernel(const float *__restrict__ x, int64_t n, int nonneg, int *flag)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
         a += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[a];
        if (!isfinite(v) || (nonneg && v < 0.0f)) atomicOr(flag, 8);
    }
}

__global__ void check_values_kernel(const float *__restrict__ x, int64_t n, int nonneg, int *flag)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
         a += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[a];
        if (!isfinite(v) || (nonneg && v < 0.0f)) atomicOr(flag, 2);
    }
}

// Every value finite, and >= 0 for non-negative models; synchronises st.
psgld_status check_values(psgld_ctx *c, const float *x, int64_t n, cudaStream_t st)
{
    PSGLD_CK(c, cudaMemsetAsync(c->flag, 0, sizeof(int), st));
    check_values_kernel<<<152 * 4, 256, 0, st>>>(x, n, c->prior.kind == PSGLD_PRIOR_EXPONENTIAL, c->flag);
    PSGLD_CK(c, cudaGetLastError());
    int h = 0;
    PSGLD_CK(c, cudaMemcpyAsync(&h, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    PSGLD_CK(c, cudaStreamSynchronize(st));
    if (h) return fail(c, PSGLD_ERR_ARG, "V entry not finite, or negative in a non-negative model");
    return PSGLD_OK;
}

__global__ void set_t_kernel(int64_t *t, int64_t v)
{
    if (threadIdx.x == 0) *t = v;
}

void destroy_batch_graphs(psgld_ctx *c)
{
    for (auto &row : c->bgraphs.exec)
        for (auto &g : row)
            if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    c->bgraphs.key.clear();
    c->bgraphs.calls = 0;
}

void destroy_graphs(psgld_ctx *c)
{
    for (auto &row : c->graph)
        for (auto &g : row)
            if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    for (auto &g : c->graph_acc)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    destroy_batch_graphs(c);
}

psgld_status zero_posterior(psgld_ctx *c, cudaStream_t st)
{
    const size_t nW = sizeof(double) * (size_t)(c->I * c->ldk);
    const size_t nH = sizeof(double) * (size_t)(c->J * c->ldk);
    PSGLD_CK(c, cudaMemsetAsync(c->sW.s, 0, nW, st));
    PSGLD_CK(c, cudaMemsetAsync(c->sW.s2, 0, nW, st));
    PSGLD_CK(c, cudaMemsetAsync(c->sH.s, 0, nH, st));
    PSGLD_CK(c, cudaMemsetAsync(c->sH.s2, 0, nH, st));
    c->n_samples = 0;
    c->sweeps_done = 0;
    c->t_done = 0;
    return PSGLD_OK;
}

// Zero-filled (when asked) on `st`, in stream order with the work that uses it.
template <typename T>
psgld_status alloc(psgld_ctx *c, T **p, int64_t n, bool zero = true, cudaStream_t st = nullptr)
{
    if (n <= 0) n = 1;
    *p = static_cast<T *>(dev_alloc(c, sizeof(T) * (size_t)n, st));
    if (!*p) return fail(c, PSGLD_ERR_OOM, "device allocation failed");
    if (zero) PSGLD_CK(c, cudaMemsetAsync(*p, 0, sizeof(T) * (size_t)n, st));
    return PSGLD_OK;
}

bool ready(psgld_ctx *c, psgld_status *s)
{
    if (!c->has_data) { *s = fail(c, PSGLD_ERR_STATE, "no data set"); return false; }
    if (!c->has_factors) { *s = fail(c, PSGLD_ERR_STATE, "no factors set"); return false; }
    if (c->opt.gather_bf16 && !c->dense && !(c->W16 && c->H16)) {
        *s = fail(c, PSGLD_ERR_STATE, "gather_bf16 was enabled after the factors were set: set them again");
        return false;
    }
    return true;
}

// Capture one sweep (B part-steps, optional accumulate, t advance) as a graph.
psgld_status capture_sweep(psgld_ctx *c, bool acc, cudaGraphExec_t *out)
{
    cudaStream_t cs = c->capture_stream;
    const int w0 = c->wcur, h0 = c->hcur;
    PSGLD_CK(c, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    psgld_status s = PSGLD_OK;
    for (int b = 0; b < c->B && s == PSGLD_OK; ++b)
        s = launch_part_step(c, b + 1, c->t_dev, b + 1, cs);
    if (s == PSGLD_OK && acc) s = launch_accumulate(c, cs);
    if (s == PSGLD_OK) s = launch_advance_t(c, c->B, cs);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    c->wcur = w0;
    c->hcur = h0;
    if (s != PSGLD_OK) { if (g) cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(c, e, "cudaStreamEndCapture"); }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    return PSGLD_OK;
}

}  // namespace
}  // namespace psgld

using namespace psgld;

extern "C" {

void psgld_default_options(psgld_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->seed = 0;
    o->eps_mode = PSGLD_EPS_FIXED;
    o->eps = 1e-4;
    o->eps_a = 0.01;
    o->eps_b = 0.51;
    o->scale_mode = PSGLD_SCALE_N_OVER_PART;
    o->mu_min = 1e-10;
    o->freeze_W = 0;
    o->freeze_H = 0;
    o->burn_in_sweeps = 0;
    o->use_graphs = 1;
    o->wide_col_blocks = -1;
    o->dense_share_e = -1;
}

psgld_status psgld_create(int64_t I, int64_t J, int32_t K, int32_t B, double tweedie_p, double phi,
                          const psgld_prior *prior, psgld_ctx **out)
{
    return create_context(I, J, K, B, tweedie_p, phi, prior, nullptr, out);
}

}  // extern "C"

namespace psgld {

psgld_status create_context(int64_t I, int64_t J, int32_t K, int32_t B, double tweedie_p, double phi,
                            const psgld_prior *prior, const psgld_allocator *allocator, psgld_ctx **out)
{
    if (!out) return PSGLD_ERR_ARG;
    *out = nullptr;
    if (!prior) return PSGLD_ERR_ARG;
    if (I < 1 || J < 1 || I >= (1ll << 31) || J >= (1ll << 31)) return PSGLD_ERR_ARG;
    if (K < 1 || K > kMaxK) return PSGLD_ERR_ARG;
    if (B < 1 || B > std::min(I, J)) return PSGLD_ERR_ARG;
    if ((int64_t)B * std::max(I, J) >= (1ll << 31)) return PSGLD_ERR_ARG;
    if (!(phi > 0.0) || !std::isfinite(phi) || !std::isfinite(tweedie_p)) return PSGLD_ERR_ARG;
    if (tweedie_p > 0.0 && tweedie_p < 1.0) return PSGLD_ERR_ARG;
    if (prior->kind == PSGLD_PRIOR_EXPONENTIAL) {
        if (!(prior->lambda_w > 0.0) || !(prior->lambda_h > 0.0)) return PSGLD_ERR_ARG;
    } else if (prior->kind == PSGLD_PRIOR_GAUSSIAN) {
        if (!(prior->sigma_w > 0.0) || !(prior->sigma_h > 0.0)) return PSGLD_ERR_ARG;
    } else {
        return PSGLD_ERR_ARG;
    }
    psgld_ctx *c = new (std::nothrow) psgld_ctx();
    if (!c) return PSGLD_ERR_OOM;
    if (allocator) {
        c->allocator = *allocator;
        c->has_allocator = true;
    } else {
        std::lock_guard<std::mutex> lock(g_alloc_mutex);
        c->allocator = g_allocator;
        c->has_allocator = g_has_allocator;
    }
    c->I = I; c->J = J; c->K = K; c->B = B;
    c->ngroups = (K + 3) / 4;
    c->ldk = 4 * c->ngroups;

    c->p = tweedie_p;
    c->phi = phi;
    c->prior = *prior;
    psgld_default_options(&c->opt);
    cudaGetDevice(&c->device);
    psgld_status s = PSGLD_OK;
    // the context's own stream first: the zero fills run on it, in order, and
    // are waited for below (a caller's non-blocking stream is not ordered
    // after the legacy stream)
    if (cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
        s = fail(c, PSGLD_ERR_CUDA, "stream creation failed");
    if (s == PSGLD_OK && (cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
                          cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                          cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess))
        s = fail(c, PSGLD_ERR_CUDA, "stream or event creation failed");
    cudaStream_t zs = c->capture_stream;
    for (int b = 0; b < 2 && s == PSGLD_OK; ++b) {
        s = alloc(c, &c->W[b], I * c->ldk, true, zs);
        if (s == PSGLD_OK) s = alloc(c, &c->Ht[b], J * c->ldk, true, zs);
    }
    if (s == PSGLD_OK) s = alloc(c, &c->G, (I + J) * c->ldk, true, zs);
    if (s == PSGLD_OK) s = alloc(c, &c->sW.s, I * c->ldk, true, zs);
    if (s == PSGLD_OK) s = alloc(c, &c->sW.s2, I * c->ldk, true, zs);
    if (s == PSGLD_OK) s = alloc(c, &c->sH.s, J * c->ldk, true, zs);
    if (s == PSGLD_OK) s = alloc(c, &c->sH.s2, J * c->ldk, true, zs);
    if (s == PSGLD_OK) s = alloc(c, &c->red, reduce_blocks(), true, zs);
    if (s == PSGLD_OK) s = alloc(c, &c->flag, 1, true, zs);
    if (s == PSGLD_OK) s = alloc(c, &c->kflag, 1, true, zs);
    if (s == PSGLD_OK) s = prepare_kernels(c);
    if (s == PSGLD_OK) s = alloc(c, &c->t_dev, 1, true, zs);
    if (s == PSGLD_OK) c->red_host.assign(reduce_blocks(), 0.0);
    if (s == PSGLD_OK && cudaStreamSynchronize(zs) != cudaSuccess)
        s = fail(c, PSGLD_ERR_CUDA, "zero fill failed");
    if (s != PSGLD_OK) {
        psgld_destroy(c);
        cudaGetLastError();
        return s;
    }
    *out = c;
    return PSGLD_OK;
}

}  // namespace psgld

extern "C" {

static void destroy_events(psgld_ctx *c)
{
    for (auto e : c->ev_start) cudaEventDestroy(e);
    for (auto e : c->ev_mid) cudaEventDestroy(e);
    for (auto e : c->ev_end) cudaEventDestroy(e);
    c->ev_start.clear();
    c->ev_mid.clear();
    c->ev_end.clear();
    c->ev_pending.clear();
}

psgld_status psgld_set_options(psgld_ctx *c, const psgld_options *o)
{
    if (!c || !o) return PSGLD_ERR_ARG;
    if (o->eps_mode == PSGLD_EPS_FIXED) {
        if (!(o->eps > 0.0) || !std::isfinite(o->eps)) return fail(c, PSGLD_ERR_ARG, "eps must be > 0");
    } else if (o->eps_mode == PSGLD_EPS_POLY) {
        if (!(o->eps_a > 0.0) || !(o->eps_b > 0.0)) return fail(c, PSGLD_ERR_ARG, "eps_a, eps_b must be > 0");
    } else {
        return fail(c, PSGLD_ERR_ARG, "unknown eps_mode");
    }
    if (o->scale_mode != PSGLD_SCALE_N_OVER_PART && o->scale_mode != PSGLD_SCALE_B)
        return fail(c, PSGLD_ERR_ARG, "unknown scale_mode");
    if (!(o->mu_min > 0.0)) return fail(c, PSGLD_ERR_ARG, "mu_min must be > 0");
    if (o->burn_in_sweeps < 0) return fail(c, PSGLD_ERR_ARG, "burn_in_sweeps must be >= 0");
    if (o->dense_path < 0 || o->dense_path > 3) return fail(c, PSGLD_ERR_ARG, "dense_path must be 0..3");
    if (o->part_mode != 0 && o->part_mode != 1) return fail(c, PSGLD_ERR_ARG, "part_mode must be 0 or 1");
    if (o->dense_fp8 != 0 && o->dense_fp8 != 1) return fail(c, PSGLD_ERR_ARG, "dense_fp8 must be 0 or 1");
    if (o->gather_bf16 != 0 && o->gather_bf16 != 1) return fail(c, PSGLD_ERR_ARG, "gather_bf16 must be 0 or 1");
    if (o->max_sms < 0) return fail(c, PSGLD_ERR_ARG, "max_sms must be >= 0");
    if (o->batch_ctas < 0 || o->batch_update_blocks < 0)
        return fail(c, PSGLD_ERR_ARG, "batch_ctas and batch_update_blocks must be >= 0");
    if (o->debug_wait_polls < 0) return fail(c, PSGLD_ERR_ARG, "debug_wait_polls must be >= 0");
    if (o->wide_col_blocks < -1) return fail(c, PSGLD_ERR_ARG, "wide_col_blocks must be >= -1");
    if (o->dense_share_e < -1 || o->dense_share_e > 1) return fail(c, PSGLD_ERR_ARG, "dense_share_e must be -1, 0 or 1");
    c->opt = *o;
    destroy_graphs(c);
    destroy_events(c);
    if (o->profile) {
        c->ev_start.resize(c->B);
        c->ev_mid.resize(c->B);
        c->ev_end.resize(c->B);
        c->ev_pending.assign(c->B, 0);
        for (int b = 0; b < c->B; ++b) {
            PSGLD_CK(c, cudaEventCreate(&c->ev_start[b]));
            PSGLD_CK(c, cudaEventCreate(&c->ev_mid[b]));
            PSGLD_CK(c, cudaEventCreate(&c->ev_end[b]));
        }
    }
    return PSGLD_OK;
}

psgld_status psgld_profile_read_split(psgld_ctx *c, double *grad_ms, double *update_ms,
                                      int64_t *launches)
{
    if (!c || !grad_ms || !update_ms || !launches) return PSGLD_ERR_ARG;
    if (!c->opt.profile) return fail(c, PSGLD_ERR_STATE, "profiling is off");
    PSGLD_CK(c, wait_enqueued(c));
    {
        psgld_status fs = check_kernel_flag(c);
        if (fs != PSGLD_OK) return fs;
    }
    double g = 0.0, u = 0.0;
    int64_t n = 0;
    for (int b = 0; b < c->B; ++b) {
        if (!c->ev_pending[b]) continue;
        float e1 = 0.f, e2 = 0.f;
        PSGLD_CK(c, cudaEventElapsedTime(&e1, c->ev_start[b], c->ev_mid[b]));
        PSGLD_CK(c, cudaEventElapsedTime(&e2, c->ev_mid[b], c->ev_end[b]));
        g += e1;
        u += e2;
        n += 1;
        c->ev_pending[b] = 0;
    }
    *grad_ms = g;
    *update_ms = u;
    *launches = n;
    return PSGLD_OK;
}

psgld_status psgld_profile_read(psgld_ctx *c, double *total_ms, int64_t *launches)
{
    if (!c || !total_ms || !launches) return PSGLD_ERR_ARG;
    double g = 0.0, u = 0.0;
    const psgld_status s = psgld_profile_read_split(c, &g, &u, launches);
    if (s != PSGLD_OK) return s;
    *total_ms = g + u;
    return PSGLD_OK;
}

psgld_status psgld_set_data_coo(psgld_ctx *c, int64_t nnz, const int32_t *i, const int32_t *j,
                                const float *v, void *stream)
{
    if (!c) return PSGLD_ERR_ARG;
    if (nnz < 0 || nnz >= (1ll << 31)) return fail(c, PSGLD_ERR_ARG, "nnz out of range");
    if (nnz > 0 && (!i || !j || !v)) return fail(c, PSGLD_ERR_ARG, "null entry array");
    cudaStream_t st = (cudaStream_t)stream;
    destroy_graphs(c);
    int32_t *di = nullptr, *dj = nullptr;
    float *dv = nullptr;
    psgld_status s = alloc(c, &di, nnz, false, st);
    if (s == PSGLD_OK) s = alloc(c, &dj, nnz, false, st);
    if (s == PSGLD_OK) s = alloc(c, &dv, nnz, false, st);
    if (s == PSGLD_OK && nnz > 0) {
        cudaError_t e = cudaMemcpyAsync(di, i, sizeof(int32_t) * nnz, cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dj, j, sizeof(int32_t) * nnz, cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dv, v, sizeof(float) * nnz, cudaMemcpyDefault, st);
        if (e != cudaSuccess) s = cuda_fail(c, e, "copy entries");
    }
    if (s == PSGLD_OK) s = build_layout(c, nnz, di, dj, dv, st);
    if (s == PSGLD_OK) s = zero_posterior(c, st);
    if (s == PSGLD_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(c, e, "sync");
    }
    dev_free(c, di); dev_free(c, dj); dev_free(c, dv);
    return s;
}

psgld_status psgld_set_data_dense(psgld_ctx *c, const float *V, int64_t ld, void *stream)
{
    if (!c || !V) return PSGLD_ERR_ARG;
    if (ld < c->J) return fail(c, PSGLD_ERR_ARG, "ld < J");
    const int64_t n = c->I * c->J;
    cudaStream_t st = (cudaStream_t)stream;
    if (c->opt.dense_path) {
        if (!dense_supported(c->K)) return fail(c, PSGLD_ERR_ARG, "dense tensor-core path supports K <= 256");
        destroy_graphs(c);
        free_layout(c);
        psgld_status s = alloc(c, &c->Vd, n, false, st);
        c->ldv = c->J;
        if (s == PSGLD_OK) {
            cudaError_t e = cudaMemcpy2DAsync(c->Vd, sizeof(float) * c->J, V, sizeof(float) * ld,
                                              sizeof(float) * c->J, c->I, cudaMemcpyDefault, st);
            if (e != cudaSuccess) s = cuda_fail(c, e, "copy V");
        }
        if (s == PSGLD_OK) s = check_values(c, c->Vd, n, st);
        if (s == PSGLD_OK) s = prepare_dense(c, st);
        if (s == PSGLD_OK && c->dense_kind == 1 && c->mtiles > 1)
            s = alloc(c, &c->hpart, (int64_t)c->mtiles * c->J * c->ldk, true, st);
        if (s == PSGLD_OK) s = build_dense_tiles(c, st);
        if (s != PSGLD_OK) { free_layout(c); return s; }
        // every entry observed: N = I J, |Pi_s| = sum_b |R_b| |C_(b+s) mod B|
        c->N = n;
        c->part_n.assign(c->B, 0);
        for (int sp = 0; sp < c->B; ++sp)
            for (int b = 0; b < c->B; ++b) {
                const int cb = (b + sp) % c->B;
                const int64_t rows = ((int64_t)(b + 1) * c->I) / c->B - ((int64_t)b * c->I) / c->B;
                const int64_t cols = ((int64_t)(cb + 1) * c->J) / c->B - ((int64_t)cb * c->J) / c->B;
                c->part_n[sp] += rows * cols;
            }
        c->dense = true;
        c->has_data = true;
        s = build_dense_shadows(c, st);
        if (s == PSGLD_OK) s = zero_posterior(c, st);
        if (s == PSGLD_OK) {
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) s = cuda_fail(c, e, "sync");
        }
        return s;
    }
    if (n >= (1ll << 31)) return fail(c, PSGLD_ERR_ARG, "I*J too large for the entry layout");
    float *dV = nullptr, *dv = nullptr;
    int32_t *di = nullptr, *dj = nullptr;
    psgld_status s = alloc(c, &dV, c->I * c->J, false, st);
    if (s == PSGLD_OK) s = alloc(c, &di, n, false, st);
    if (s == PSGLD_OK) s = alloc(c, &dj, n, false, st);
    if (s == PSGLD_OK) s = alloc(c, &dv, n, false, st);
    if (s == PSGLD_OK) {
        cudaError_t e = cudaMemcpy2DAsync(dV, sizeof(float) * c->J, V, sizeof(float) * ld,
                                          sizeof(float) * c->J, c->I, cudaMemcpyDefault, st);
        if (e != cudaSuccess) s = cuda_fail(c, e, "copy V");
    }
    if (s == PSGLD_OK) {
        dense_to_coo_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 32), 256, 0, st>>>(
            dV, c->I, c->J, c->J, di, dj, dv);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = cuda_fail(c, e, "dense_to_coo");
    }
    if (s == PSGLD_OK) {
        // dV is read by dense_to_coo on st; free it after that work
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(c, e, "sync");
    }
    dev_free(c, dV, st);
    dV = nullptr;
    if (s == PSGLD_OK) {
        // psgld_set_data_coo copies again; build directly instead
        destroy_graphs(c);
        s = build_layout(c, n, di, dj, dv, st);
        if (s == PSGLD_OK) s = zero_posterior(c, st);
        if (s == PSGLD_OK) {
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) s = cuda_fail(c, e, "sync");
        }
    }
    dev_free(c, di); dev_free(c, dj); dev_free(c, dv);
    return s;
}

psgld_status psgld_set_factors(psgld_ctx *c, const float *W, const float *Ht, void *stream)
{
    if (!c || !W || !Ht) return PSGLD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t row = sizeof(float) * c->K, pitch = sizeof(float) * c->ldk;
    PSGLD_CK(c, cudaMemcpy2DAsync(c->W[c->wcur], pitch, W, row, row, c->I, cudaMemcpyDefault, st));
    PSGLD_CK(c, cudaMemcpy2DAsync(c->Ht[c->hcur], pitch, Ht, row, row, c->J, cudaMemcpyDefault, st));
    PSGLD_CK(c, cudaMemsetAsync(c->flag, 0, sizeof(int), st));
    const int nonneg = c->prior.kind == PSGLD_PRIOR_EXPONENTIAL;
    check_factors_kernel<<<152 * 4, 256, 0, st>>>(c->W[c->wcur], c->I * c->ldk, nonneg, c->flag);
    check_factors_kernel<<<152 * 4, 256, 0, st>>>(c->Ht[c->hcur], c->J * c->ldk, nonneg, c->flag);
    PSGLD_CK(c, cudaGetLastError());
    int h = 0;
    PSGLD_CK(c, cudaMemcpyAsync(&h, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    PSGLD_CK(c, cudaStreamSynchronize(st));
    if (h) {
        c->has_factors = false;
        return fail(c, PSGLD_ERR_ARG, "factor entry not finite, or negative in a non-negative model");
    }
    c->has_factors = true;
    psgld_status s = build_dense_shadows(c, st);
    if (s == PSGLD_OK) s = build_gather_shadows(c, st);
    return s;
}

psgld_status psgld_get_factors(psgld_ctx *c, float *W, float *Ht, void *stream)
{
    if (!c) return PSGLD_ERR_ARG;
    if (!c->has_factors) return fail(c, PSGLD_ERR_STATE, "no factors set");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t row = sizeof(float) * c->K, pitch = sizeof(float) * c->ldk;
    if (W) PSGLD_CK(c, cudaMemcpy2DAsync(W, row, c->W[c->wcur], pitch, row, c->I, cudaMemcpyDefault, st));
    if (Ht) PSGLD_CK(c, cudaMemcpy2DAsync(Ht, row, c->Ht[c->hcur], pitch, row, c->J, cudaMemcpyDefault, st));
    mark_enqueued(c, st);
    return PSGLD_OK;
}

psgld_status psgld_part_step(psgld_ctx *c, int64_t t, void *stream)
{
    if (!c) return PSGLD_ERR_ARG;
    psgld_status s;
    if (!ready(c, &s)) return s;
    if (t < 1) return fail(c, PSGLD_ERR_ARG, "t must be >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    s = launch_part_step(c, t, nullptr, 0, st);
    mark_enqueued(c, st);                 // also after a failed launch: waits cover it
    if (s != PSGLD_OK) return s;
    c->t_done = t;
    return PSGLD_OK;
}

psgld_status psgld_sweep(psgld_ctx *c, int32_t n_sweeps, void *stream)
{
    if (!c) return PSGLD_ERR_ARG;
    psgld_status s;
    if (!ready(c, &s)) return s;
    if (n_sweeps < 0) return fail(c, PSGLD_ERR_ARG, "n_sweeps < 0");
    if (c->t_done % c->B != 0) return fail(c, PSGLD_ERR_STATE, "sweep must start at a sweep boundary");
    cudaStream_t st = (cudaStream_t)stream;
    // until the closing mark_enqueued, waits fall back to the whole stream
    // (covers work enqueued before an error return)
    c->last_stream = st;
    c->last_ev_set = false;
    if (n_sweeps == 0) return PSGLD_OK;
    const bool graphs = c->opt.use_graphs && c->opt.part_mode == 0;
    if (graphs) {
        set_t_kernel<<<1, 32, 0, st>>>(c->t_dev, c->t_done);
        PSGLD_CK(c, cudaGetLastError());
    }
    for (int32_t n = 0; n < n_sweeps; ++n) {
        const bool acc = c->sweeps_done >= c->opt.burn_in_sweeps;
        if (graphs) {
            cudaGraphExec_t &g = acc ? c->graph_acc[c->wcur * 2 + c->hcur] : c->graph[c->wcur][c->hcur];
            if (!g) {
                s = capture_sweep(c, acc, &g);
                if (s != PSGLD_OK) return s;
            }
            PSGLD_CK(c, cudaGraphLaunch(g, st));
            if (c->opt.profile)
                for (auto &pnd : c->ev_pending) pnd = 1;
            // the replay leaves the buffers as B part-steps do
            if (!c->opt.freeze_W) c->wcur ^= (c->B & 1);
            if (!c->opt.freeze_H) c->hcur ^= (c->B & 1);
        } else {
            for (int b = 0; b < c->B; ++b) {
                s = launch_part_step(c, c->t_done + b + 1, nullptr, 0, st);
                if (s != PSGLD_OK) return s;
            }
            if (acc) {
                s = launch_accumulate(c, st);
                if (s != PSGLD_OK) return s;
            }
        }
        c->t_done += c->B;
        c->sweeps_done += 1;
        if (acc) c->n_samples += 1;
    }
    mark_enqueued(c, st);
    return PSGLD_OK;
}

psgld_status psgld_posterior_mean(psgld_ctx *c, double *Wm, double *Wv, double *Hm, double *Hv,
                                  int64_t *n_samples)
{
    if (!c) return PSGLD_ERR_ARG;
    PSGLD_CK(c, wait_enqueued(c));
    {
        psgld_status fs = check_kernel_flag(c);
        if (fs != PSGLD_OK) return fs;
    }
    const int64_t ldk = c->ldk, K = c->K;
    const double n = (double)c->n_samples;
    for (int side = 0; side < 2; ++side) {
        double *mean = side == 0 ? Wm : Hm, *var = side == 0 ? Wv : Hv;
        if (!mean && !var) continue;
        const int64_t rows = side == 0 ? c->I : c->J;
        const Sums &S = side == 0 ? c->sW : c->sH;
        std::vector<double> s((size_t)(rows * ldk)), s2((size_t)(rows * ldk));
        PSGLD_CK(c, cudaMemcpy(s.data(), S.s, sizeof(double) * s.size(), cudaMemcpyDeviceToHost));
        PSGLD_CK(c, cudaMemcpy(s2.data(), S.s2, sizeof(double) * s2.size(), cudaMemcpyDeviceToHost));
        for (int64_t r = 0; r < rows; ++r)
            for (int64_t k = 0; k < K; ++k) {
                const double m = n > 0 ? s[r * ldk + k] / n : 0.0;
                if (mean) mean[r * K + k] = m;
                if (var) var[r * K + k] = n > 0 ? s2[r * ldk + k] / n - m * m : 0.0;
            }
    }
    if (n_samples) *n_samples = c->n_samples;
    return PSGLD_OK;
}

// The state of a chain beside its factors: the FP64 sums (rows x ldk on the
// device, rows x K on the host) and the counters t, sweeps, samples.
psgld_status psgld_get_state(psgld_ctx *c, double *sW, double *sW2, double *sH, double *sH2,
                             int64_t *counters)
{
    if (!c) return PSGLD_ERR_ARG;
    PSGLD_CK(c, wait_enqueued(c));
    {
        psgld_status fs = check_kernel_flag(c);
        if (fs != PSGLD_OK) return fs;
    }
    const size_t row = sizeof(double) * (size_t)c->K, pitch = sizeof(double) * (size_t)c->ldk;
    const struct { double *dst; const double *src; int64_t rows; } parts[4] = {
        {sW, c->sW.s, c->I}, {sW2, c->sW.s2, c->I}, {sH, c->sH.s, c->J}, {sH2, c->sH.s2, c->J}};
    for (const auto &q : parts)
        if (q.dst)
            PSGLD_CK(c, cudaMemcpy2D(q.dst, row, q.src, pitch, row, (size_t)q.rows, cudaMemcpyDeviceToHost));
    if (counters) {
        counters[0] = c->t_done;
        counters[1] = c->sweeps_done;
        counters[2] = c->n_samples;
    }
    return PSGLD_OK;
}

psgld_status psgld_set_state(psgld_ctx *c, const double *sW, const double *sW2, const double *sH,
                             const double *sH2, const int64_t *counters)
{
    if (!c || !sW || !sW2 || !sH || !sH2 || !counters) return PSGLD_ERR_ARG;
    const int64_t t = counters[0], sweeps = counters[1], samples = counters[2];
    if (t < 0 || sweeps < 0 || samples < 0 || samples > sweeps)
        return fail(c, PSGLD_ERR_ARG, "inconsistent counters (t, sweeps, samples)");
    if (!c->has_factors) return fail(c, PSGLD_ERR_STATE, "set the data and the factors first");
    PSGLD_CK(c, wait_enqueued(c));
    const size_t row = sizeof(double) * (size_t)c->K, pitch = sizeof(double) * (size_t)c->ldk;
    const struct { double *dst; const double *src; int64_t rows; } parts[4] = {
        {c->sW.s, sW, c->I}, {c->sW.s2, sW2, c->I}, {c->sH.s, sH, c->J}, {c->sH.s2, sH2, c->J}};
    // the padding columns (K .. ldk-1) stay as they are: zero
    for (const auto &q : parts)
        PSGLD_CK(c, cudaMemcpy2D(q.dst, pitch, q.src, row, row, (size_t)q.rows, cudaMemcpyHostToDevice));
    PSGLD_CK(c, cudaMemcpy(c->t_dev, &t, sizeof t, cudaMemcpyHostToDevice));
    c->t_done = t;
    c->sweeps_done = sweeps;
    c->n_samples = samples;
    return PSGLD_OK;
}

psgld_status psgld_log_lik(psgld_ctx *c, double *out, void *stream)
{
    if (!c || !out) return PSGLD_ERR_ARG;
    psgld_status s;
    if (!ready(c, &s)) return s;
    return reduce_loglik_rmse(c, 0, 0, (cudaStream_t)stream, out);
}

psgld_status psgld_rmse(psgld_ctx *c, int32_t use_mean, double *out, void *stream)
{
    if (!c || !out) return PSGLD_ERR_ARG;
    psgld_status s;
    if (!ready(c, &s)) return s;
    if (use_mean && c->n_samples == 0) return fail(c, PSGLD_ERR_STATE, "no posterior samples yet");
    double ss = 0.0;
    s = reduce_loglik_rmse(c, 1, use_mean, (cudaStream_t)stream, &ss);
    if (s != PSGLD_OK) return s;
    *out = c->N > 0 ? std::sqrt(ss / (double)c->N) : 0.0;
    return PSGLD_OK;
}

psgld_status psgld_piece_bounds(const psgld_ctx *c, int64_t *rs, int64_t *cs)
{
    if (!c) return PSGLD_ERR_ARG;
    for (int r = 0; r <= c->B; ++r) {
        if (rs) rs[r] = ((int64_t)r * c->I) / c->B;
        if (cs) cs[r] = ((int64_t)r * c->J) / c->B;
    }
    return PSGLD_OK;
}

psgld_status psgld_part_schedule(const psgld_ctx *c, int64_t t, int32_t *col_piece)
{
    if (!c || !col_piece || t < 1) return PSGLD_ERR_ARG;
    if (c->opt.part_mode == 1 && !c->has_data) return PSGLD_ERR_STATE;
    const int64_t s = part_of_iteration(c, t);
    for (int r = 0; r < c->B; ++r) col_piece[r] = (int32_t)((r + s) % c->B);
    return PSGLD_OK;
}

psgld_status psgld_part_layout(psgld_ctx *c, int32_t s, int32_t *row_ptr, int32_t *cols,
                               int64_t *n_entries)
{
    if (!c || s < 0 || s >= c->B) return PSGLD_ERR_ARG;
    if (!c->has_data) return fail(c, PSGLD_ERR_STATE, "no data set");
    if (c->dense) return fail(c, PSGLD_ERR_STATE, "dense tensor-core data keeps no entry layout");
    std::vector<int32_t> ptr((size_t)c->I + 1);
    PSGLD_CK(c, cudaMemcpy(ptr.data(), c->side[0].ptr + (int64_t)s * c->I,
                           sizeof(int32_t) * ptr.size(), cudaMemcpyDeviceToHost));
    const int64_t n = ptr[c->I] - ptr[0];
    if (n_entries) *n_entries = n;
    if (row_ptr)
        for (int64_t r = 0; r <= c->I; ++r) row_ptr[r] = ptr[r] - ptr[0];
    if (cols && n > 0)
        PSGLD_CK(c, cudaMemcpy(cols, c->side[0].idx + ptr[0], sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    return PSGLD_OK;
}

int64_t psgld_iterations_done(const psgld_ctx *c) { return c ? c->t_done : -1; }

// Batched sweeps.  Everything the launches of the call read is known before
// the first one: per part b and per sweep parity q (the ping-pong buffers a
// context starts the sweep in alternate only when B is odd) the dense and
// update parameter tables, per q the accumulation table, and the grid
// prefixes.  They go to the device in one copy; the iteration counter t is
// each context's device counter (set once, advanced by B after each sweep),
// so a sweep is the same 2B + 2 launches every time.
psgld_status psgld_batch_sweep(psgld_ctx *const *ctxs, int32_t n, int32_t n_sweeps, void *stream)
{
    if (!ctxs || n < 1 || n_sweeps < 0) return PSGLD_ERR_ARG;
    psgld_ctx *c0 = ctxs[0];
    if (!c0) return PSGLD_ERR_ARG;
    const int B = c0->B;
    for (int i = 0; i < n; ++i) {
        psgld_ctx *c = ctxs[i];
        if (!c) return PSGLD_ERR_ARG;
        psgld_status s;
        if (!ready(c, &s)) return s;
        if (!c->dense || dense_batch_key(c) <= 0)
            return fail(c, PSGLD_ERR_STATE, "batched sweeps need dense data on the tensor-core kernels");
        if (c->B != B) return fail(c, PSGLD_ERR_ARG, "batched contexts must share B");
        if (c->opt.part_mode != 0) return fail(c, PSGLD_ERR_STATE, "batched sweeps use cyclic parts");
        if (c->t_done % B != 0) return fail(c, PSGLD_ERR_STATE, "sweep must start at a sweep boundary");
        if (c->device != c0->device) return fail(c, PSGLD_ERR_ARG, "batched contexts must share a device");
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == c) return fail(c, PSGLD_ERR_ARG, "a context appears twice in the batch");
    }
    if (n_sweeps == 0) return PSGLD_OK;
    cudaStream_t st = (cudaStream_t)stream;

    // gradient launches: contexts grouped by batch key (kernel variant), in
    // first-seen order
    std::vector<int> keys, order;                 // order: context indices, group by group
    std::vector<int> gbeg;                        // group g: order[gbeg[g] .. gbeg[g + 1])
    for (int i = 0; i < n; ++i) {
        const int key = dense_batch_key(ctxs[i]);
        if (std::find(keys.begin(), keys.end(), key) == keys.end()) keys.push_back(key);
    }
    for (int key : keys) {
        gbeg.push_back((int)order.size());
        for (int i = 0; i < n; ++i)
            if (dense_batch_key(ctxs[i]) == key) order.push_back(i);
    }
    gbeg.push_back(n);
    const int ng = (int)keys.size();
    const int nq = (B & 1) && n_sweeps > 1 ? 2 : 1;

    auto up256 = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t dp = dense_param_bytes(), upb = upd_param_bytes(), ap = acc_param_bytes();
    // per group g, at 2 (gbeg[g] + g): two prefix arrays of its contexts'
    // items (first kind, then second kind), n_g + 1 entries each
    const size_t off_cta = 0;
    const size_t off_items = up256(off_cta + sizeof(int) * (size_t)(2 * (n + ng)));
    const size_t off_units = up256(off_items + sizeof(int64_t) * (size_t)(n + 1));
    const size_t off_dp = up256(off_units + sizeof(int64_t) * (size_t)(n + 1));
    const size_t off_up = up256(off_dp + dp * (size_t)nq * B * n);
    const size_t off_ap = up256(off_up + upb * (size_t)nq * B * n);
    const size_t total = up256(off_ap + ap * (size_t)nq * n);
    std::vector<unsigned char> &tab = c0->btab;
    tab.assign(total, 0);
    int *cta = reinterpret_cast<int *>(tab.data() + off_cta);
    int64_t *items = reinterpret_cast<int64_t *>(tab.data() + off_items);
    int64_t *units = reinterpret_cast<int64_t *>(tab.data() + off_units);
    std::vector<int> g_ctas((size_t)ng, 0);

    std::vector<int> w0((size_t)n), h0((size_t)n);
    for (int i = 0; i < n; ++i) {
        w0[i] = ctxs[i]->wcur;
        h0[i] = ctxs[i]->hcur;
    }
    // buffers a context reads after `steps` part-steps of this call
    auto set_state = [&](int i, int64_t steps) {
        psgld_ctx *c = ctxs[i];
        c->wcur = c->opt.freeze_W ? w0[i] : w0[i] ^ (int)(steps & 1);
        c->hcur = c->opt.freeze_H ? h0[i] : h0[i] ^ (int)(steps & 1);
    };
    for (int q = 0; q < nq; ++q) {
        for (int b = 0; b < B; ++b) {
            const size_t row = (size_t)(q * B + b) * n;
            for (int g = 0; g < ng; ++g) {
                const int ngc = gbeg[g + 1] - gbeg[g];
                int *pre = cta + 2 * (gbeg[g] + g);
                int acc1 = 0, acc2 = 0;
                for (int k = gbeg[g]; k < gbeg[g + 1]; ++k) {
                    const int i = order[k];
                    set_state(i, (int64_t)q * B + b);
                    if (q == 0 && b == 0) {
                        pre[k - gbeg[g]] = acc1;
                        pre[ngc + 1 + k - gbeg[g]] = acc2;
                    }
                    int first = 0;
                    const int all = fill_dense_param(ctxs[i], b, tab.data() + off_dp + dp * (row + k), &first);
                    acc1 += first;
                    acc2 += all - first;
                }
                if (q == 0 && b == 0) {
                    pre[ngc] = acc1;
                    pre[2 * ngc + 1] = acc2;
                    g_ctas[g] = acc1 + acc2;
                }
            }
            int64_t it = 0;
            for (int i = 0; i < n; ++i) {
                set_state(i, (int64_t)q * B + b);
                if (q == 0 && b == 0) items[i] = it;
                it += fill_upd_param(ctxs[i], b, ctxs[i]->t_dev, b + 1, tab.data() + off_up + upb * (row + i));
            }
            if (q == 0 && b == 0) items[n] = it;
        }
        int64_t un = 0;
        for (int i = 0; i < n; ++i) {
            psgld_ctx *c = ctxs[i];
            set_state(i, (int64_t)(q + 1) * B);
            if (q == 0) units[i] = un;
            un += fill_acc_param(c, c->t_done, (int64_t)c->opt.burn_in_sweeps - c->sweeps_done,
                                 tab.data() + off_ap + ap * ((size_t)q * n + i));
        }
        if (q == 0) units[n] = un;
    }
    for (int i = 0; i < n; ++i) set_state(i, 0);     // back to the state the call found

    // the device tables live in the leading context and are reused by its
    // next batch, ordered after the launches of this one by `bdone`
    cudaError_t e = cudaSuccess;
    if (!c0->bdone) {
        e = cudaEventCreateWithFlags(&c0->bdone, cudaEventDisableTiming);
        if (e != cudaSuccess) { c0->bdone = nullptr; return cuda_fail(c0, e, "cudaEventCreate"); }
        e = cudaEventRecord(c0->bdone, st);
        if (e != cudaSuccess) return cuda_fail(c0, e, "cudaEventRecord");
    }
    if (c0->bscratch_bytes < total) {
        if (c0->bscratch) {
            cudaEventSynchronize(c0->bdone);
            dev_free(c0, c0->bscratch, st);
            c0->bscratch = nullptr;
            c0->bscratch_bytes = 0;
        }
        c0->bscratch = dev_alloc(c0, total, st);
        if (!c0->bscratch) return fail(c0, PSGLD_ERR_OOM, "device allocation failed");
        c0->bscratch_bytes = total;
    } else {
        e = cudaStreamWaitEvent(st, c0->bdone, 0);
        if (e != cudaSuccess) return cuda_fail(c0, e, "cudaStreamWaitEvent");
    }
    unsigned char *d = static_cast<unsigned char *>(c0->bscratch);
    psgld_status s = PSGLD_OK;
    // from pageable memory: the source is consumed before the call returns
    e = cudaMemcpyAsync(d, tab.data(), total, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) s = cuda_fail(c0, e, "copy of the batch tables");
    if (s == PSGLD_OK) s = launch_t_batch(c0, d + off_ap, n, 0, st);
    // profiling (first context's option): events around each part's launches,
    // read back with psgld_profile_read_split on the first context
    const bool prof = c0->opt.profile && (int)c0->ev_start.size() == B;
    auto record = [&](cudaEvent_t ev) {
        const cudaError_t re = cudaEventRecord(ev, st);
        return re == cudaSuccess ? PSGLD_OK : cuda_fail(c0, re, "cudaEventRecord");
    };
    // one sweep's launches on stream `ss`: per part the gradient launches of
    // every kernel variant and one update launch, then the accumulation
    // (when any context is past burn-in) and the iteration counters
    auto enqueue_sweep = [&](int q, bool any, cudaStream_t ss) -> psgld_status {
        psgld_status r = PSGLD_OK;
        for (int b = 0; b < B && r == PSGLD_OK; ++b) {
            const size_t row = (size_t)(q * B + b) * n;
            if (prof) r = record(c0->ev_start[b]);
            for (int g = 0; g < ng && r == PSGLD_OK; ++g)
                r = launch_dense_batch(c0, keys[g], d + off_dp + dp * (row + gbeg[g]),
                                       reinterpret_cast<const int *>(d + off_cta) + 2 * (gbeg[g] + g),
                                       gbeg[g + 1] - gbeg[g], g_ctas[g], ss);
            if (r == PSGLD_OK && prof) r = record(c0->ev_mid[b]);
            if (r == PSGLD_OK)
                r = launch_update_batch(c0, d + off_up + upb * row,
                                        reinterpret_cast<const int64_t *>(d + off_items), n, items[n], ss);
            if (r == PSGLD_OK && prof) {
                r = record(c0->ev_end[b]);
                c0->ev_pending[b] = 1;
            }
        }
        if (r == PSGLD_OK && any)
            r = launch_accumulate_batch(c0, d + off_ap + ap * (size_t)q * n,
                                        reinterpret_cast<const int64_t *>(d + off_units), n, units[n], ss);
        if (r == PSGLD_OK) r = launch_t_batch(c0, d + off_ap, n, 1, ss);
        return r;
    };
    // captured graphs: everything a sweep's launches bake in is in the key.
    // A structure is captured once it repeats (the second consecutive call
    // with the same key) or when the call runs several sweeps: a serving
    // loop whose job list changes between calls launches directly rather
    // than capturing graphs it would use once.
    bool graphs = c0->opt.use_graphs && !prof && c0->capture_stream;
    if (graphs && s == PSGLD_OK) {
        std::vector<int64_t> key = {(int64_t)(uintptr_t)d, (int64_t)total, n, ng, B, nq,
                                    c0->opt.batch_ctas, c0->opt.batch_update_blocks, items[n], units[n]};
        for (int g = 0; g < ng; ++g) {
            key.push_back(keys[g]);
            key.push_back(gbeg[g]);
            key.push_back(g_ctas[g]);
        }
        if (key != c0->bgraphs.key) {
            destroy_batch_graphs(c0);
            c0->bgraphs.key = key;
        }
        c0->bgraphs.calls += 1;
        graphs = c0->bgraphs.calls >= 2 || n_sweeps > 1;
    }
    for (int32_t sw = 0; sw < n_sweeps && s == PSGLD_OK; ++sw) {
        const int q = nq == 2 ? (sw & 1) : 0;
        bool any = false;
        for (int i = 0; i < n; ++i) any |= ctxs[i]->sweeps_done + sw >= ctxs[i]->opt.burn_in_sweeps;
        if (!graphs) {
            s = enqueue_sweep(q, any, st);
            continue;
        }
        cudaGraphExec_t &ex = c0->bgraphs.exec[q][any ? 1 : 0];
        if (!ex) {
            cudaStream_t cs = c0->capture_stream;
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) { s = cuda_fail(c0, e, "cudaStreamBeginCapture"); break; }
            s = enqueue_sweep(q, any, cs);
            cudaGraph_t gr = nullptr;
            e = cudaStreamEndCapture(cs, &gr);
            if (s == PSGLD_OK && e != cudaSuccess) s = cuda_fail(c0, e, "cudaStreamEndCapture");
            if (s == PSGLD_OK) {
                e = cudaGraphInstantiate(&ex, gr, 0);
                if (e != cudaSuccess) {
                    ex = nullptr;
                    s = cuda_fail(c0, e, "cudaGraphInstantiate");
                }
            }
            if (gr) cudaGraphDestroy(gr);
            if (s != PSGLD_OK) break;
        }
        e = cudaGraphLaunch(ex, st);
        if (e != cudaSuccess) s = cuda_fail(c0, e, "cudaGraphLaunch");
    }
    for (int i = 0; i < n; ++i) {
        psgld_ctx *c = ctxs[i];
        if (s == PSGLD_OK) {
            set_state(i, (int64_t)n_sweeps * B);
            for (int32_t sw = 0; sw < n_sweeps; ++sw) {
                if (c->sweeps_done >= c->opt.burn_in_sweeps) c->n_samples += 1;
                c->sweeps_done += 1;
            }
            c->t_done += (int64_t)B * n_sweeps;
        }
        // after a failed launch the factors are unspecified (set them again),
        // but whatever was enqueued is still waited for before the context
        // frees its memory
        mark_enqueued(c, st);
    }
    e = cudaEventRecord(c0->bdone, st);
    if (s == PSGLD_OK && e != cudaSuccess) s = cuda_fail(c0, e, "cudaEventRecord");
    return s;
}

psgld_status psgld_set_allocator(const psgld_allocator *a)
{
    if (a && (!a->alloc || !a->free)) return PSGLD_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    g_has_allocator = a != nullptr;
    g_allocator = a ? *a : psgld_allocator{};
    return PSGLD_OK;
}

int64_t psgld_estimate_device_bytes(int64_t I, int64_t J, int32_t K, int32_t B, int64_t nnz,
                                    int32_t dense_path, int32_t dense_v_bf16)
{
    if (I < 1 || J < 1 || K < 1 || K > kMaxK || B < 1 || B > std::min(I, J) || nnz < 0) return -1;
    const int64_t ldk = 4 * ((K + 3) / 4);
    auto cdiv = [](int64_t a, int64_t b) { return (a + b - 1) / b; };
    int64_t bytes = 0;
    // psgld_create: W, Ht (two buffers each), G, FP64 posterior sums, reduction slots
    bytes += 2 * (I + J) * ldk * 4 + (I + J) * ldk * 4 + 2 * (I + J) * ldk * 8 + reduce_blocks() * 8 + 64;
    if (dense_path == 0) {
        // the two part-major entry layouts and their partial-sum slots
        const int unit = unit_entries((K + 3) / 4);
        for (int side = 0; side < 2; ++side) {
            const int64_t n_rows = side == 0 ? I : J;
            bytes += (B * n_rows + 1) * 4 + nnz * 12 + 2 * (cdiv(nnz, unit) + B) * ldk * 4;
        }
        return bytes;
    }
    bytes += I * J * 4;   // the FP32 copy of V
    const int64_t maxI = cdiv(I, B), maxJ = cdiv(J, B);
    const int64_t mtiles = cdiv(maxI, 128);
    const bool two = dense_path == 2 || (dense_path == 1 && (dense_v_bf16 || K > 128 || mtiles > 1));
    if (!two) {
        if (mtiles > 1) bytes += mtiles * J * ldk * 4;
        return bytes;
    }
    const int64_t KP = 64 * cdiv(K, 64), vs = dense_v_bf16 ? 2 : 4;
    const int64_t mt = cdiv(maxI, 128), nt = cdiv(maxJ, 128), ni = cdiv(maxI, 64), nj = cdiv(maxJ, 64);
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool share = two_sided_share(-1, maxI, B, (int)mt, (int)nt, sms) != 0;
    bytes += (int64_t)B * B * mt * nj * 8192 * vs;                 // V tiles
    if (!share) bytes += (int64_t)B * B * nt * ni * 8192 * vs;     // ... other orientation
    bytes += (int64_t)B * 2 * (mt + nt) * 64 * KP * 2;              // BF16 factor shadows
    if (share) bytes += (int64_t)B * mt * 4 * cdiv(maxJ, 256) * 8192 * 2;   // one part's E
    bytes += 4 * (2 + B);                                            // launch counters
    return bytes;
}

const char *psgld_last_error(const psgld_ctx *c) { return c ? c->err.c_str() : "null context"; }

void psgld_destroy(psgld_ctx *c)
{
    if (!c) return;
    destroy_graphs(c);
    destroy_events(c);
    free_layout(c);
    // the context's work must be finished before its memory is handed back
    wait_enqueued(c);
    if (c->last_ev) cudaEventDestroy(c->last_ev);
    if (c->capture_stream) cudaStreamSynchronize(c->capture_stream);
    if (c->bdone) {
        cudaEventSynchronize(c->bdone);
        cudaEventDestroy(c->bdone);
    }
    dev_free(c, c->bscratch);
    dev_free(c, c->W16);
    dev_free(c, c->H16);
    for (int b = 0; b < 2; ++b) { dev_free(c, c->W[b]); dev_free(c, c->Ht[b]); }
    dev_free(c, c->G);
    dev_free(c, c->sW.s); dev_free(c, c->sW.s2); dev_free(c, c->sH.s); dev_free(c, c->sH.s2);
    dev_free(c, c->red); dev_free(c, c->flag); dev_free(c, c->kflag); dev_free(c, c->t_dev);
    if (c->side_stream) {
        cudaStreamSynchronize(c->side_stream);
        cudaStreamDestroy(c->side_stream);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    delete c;
}

}  // extern "C"
