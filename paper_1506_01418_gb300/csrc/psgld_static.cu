// psgld_static.cu -- psgld_log_lik_static: the Tweedie log-likelihood of
// given factors on given entries, evaluated without allocating memory.
//
// Some callers cannot allocate device memory at the moment they want this
// number: code whose device memory is owned by another allocator that has
// reserved it all, or code running where an allocation would synchronise the
// device or is forbidden (for example a monitoring hook inside a latency-
// sensitive loop).  This entry point takes their entries and factors as they
// are (plain row-major arrays, no context, no layout build) and keeps its
// only scratch -- one FP64 partial sum per block of 4096 entries -- in a
// file-scope __device__ array that exists, at 32 KB, on every GPU that loads
// the library until the process exits.
//
// Set-up: the first call on a device looks up the array's device address
// with cudaGetSymbolAddress (with that device current) and caches it per
// device ordinal; make that first call before any stream capture.  The
// cached address belongs to the device's primary context (the one the CUDA
// runtime and PyTorch use): after cudaDeviceReset, or from a context created
// by hand with the driver API, it is no longer valid.  Every call writes the
// partial slots it reads, so nothing needs clearing between calls, but all
// calls share the array: calls that can overlap on a device (different
// streams, no ordering between them) race and must be serialised by the
// caller.
//
// Entry indices are checked against I and J: an entry outside [0, I) x
// [0, J) is not read, and its block's partial sum becomes NaN, so the result
// is NaN (a caller's indexing mistake never reads outside its arrays).
#include <mutex>

#include "psgld_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int64_t kEntriesPerBlock = 4096;
constexpr int kMaxBlocks = 4096;
constexpr int kMaxDevices = 64;
static_assert(PSGLD_STATIC_MAX_NNZ == kEntriesPerBlock * kMaxBlocks, "static scratch size");

static __device__ __align__(256) double g_partial[kMaxBlocks];

std::mutex g_setup_mutex;
double *g_partial_ptr[kMaxDevices] = {};

__device__ double static_beta_div(double v, double mu, double p)
{
    const double beta = 2.0 - p;
    if (beta == 2.0) return 0.5 * (v - mu) * (v - mu);
    if (beta == 1.0) return (v > 0.0 ? v * log(v / mu) : 0.0) - v + mu;
    if (beta == 0.0) return v / mu - log(v / mu) - 1.0;
    return pow(v, beta) / (beta * (beta - 1.0)) - v * pow(mu, beta - 1.0) / (beta - 1.0) +
           pow(mu, beta) / beta;
}

__device__ double block_sum(double x)
{
    __shared__ double sm[kThreads];
    sm[threadIdx.x] = x;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    return sm[0];
}

// Block b sums entries [4096 b, 4096 (b+1)) into partial[b]; NaN if one of
// them has an index outside [0, I) x [0, J) (that entry is skipped).
__global__ void __launch_bounds__(kThreads)
static_ll_blocks(int64_t nnz, const int32_t *__restrict__ ii, const int32_t *__restrict__ jj,
                 const float *__restrict__ vv, const float *__restrict__ W,
                 const float *__restrict__ Ht, int64_t I, int64_t J, int K, double p, double phi,
                 double mu_min, double *__restrict__ partial)
{
    const int64_t lo = blockIdx.x * kEntriesPerBlock;
    const int64_t hi = lo + kEntriesPerBlock < nnz ? lo + kEntriesPerBlock : nnz;
    double acc = 0.0;
    int bad = 0;
    for (int64_t e = lo + threadIdx.x; e < hi; e += kThreads) {
        const int64_t i = ii[e], j = jj[e];
        if (i < 0 || i >= I || j < 0 || j >= J) {
            bad = 1;
            continue;
        }
        double mu = 0.0;
        for (int k = 0; k < K; ++k) mu += (double)W[i * K + k] * (double)Ht[j * K + k];
        if (p > 0.0 && mu < mu_min) mu = mu_min;
        acc -= static_beta_div((double)vv[e], mu, p) / phi;
    }
    bad = __syncthreads_or(bad);
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = bad ? __longlong_as_double(0x7FF8000000000000ll) : s;
}

// One block adds partial[0 .. nblocks) in a fixed order.
__global__ void __launch_bounds__(kThreads)
static_ll_final(int nblocks, const double *__restrict__ partial, double *__restrict__ out)
{
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kThreads) acc += partial[b];
    const double s = block_sum(acc);
    if (threadIdx.x == 0) *out = s;
}

}  // namespace

extern "C" psgld_status psgld_log_lik_static(int64_t nnz, const int32_t *i_dev,
                                             const int32_t *j_dev, const float *v_dev,
                                             const float *W_dev, const float *Ht_dev, int64_t I,
                                             int64_t J, int32_t K, double tweedie_p, double phi,
                                             double mu_min, double *out_dev, void *stream)
{
    if (nnz < 0 || I < 1 || J < 1 || K < 1 || !out_dev || !W_dev || !Ht_dev) return PSGLD_ERR_ARG;
    if (nnz > 0 && (!i_dev || !j_dev || !v_dev)) return PSGLD_ERR_ARG;
    if (!(phi > 0.0) || (tweedie_p > 0.0 && tweedie_p < 1.0) || !(mu_min > 0.0)) return PSGLD_ERR_ARG;
    if (nnz > PSGLD_STATIC_MAX_NNZ) return PSGLD_ERR_SIZE;   // beyond the static scratch

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return PSGLD_ERR_CUDA;
    }
    double *partial = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partial_ptr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_partial) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return PSGLD_ERR_CUDA;
            }
            g_partial_ptr[dev] = static_cast<double *>(ptr);
        }
        partial = g_partial_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nblocks = nnz > 0 ? (int)((nnz + kEntriesPerBlock - 1) / kEntriesPerBlock) : 0;
    if (nblocks > 0)
        static_ll_blocks<<<nblocks, kThreads, 0, st>>>(nnz, i_dev, j_dev, v_dev, W_dev, Ht_dev, I, J,
                                                       K, tweedie_p, phi, mu_min, partial);
    static_ll_final<<<1, kThreads, 0, st>>>(nblocks, partial, out_dev);
    if (cudaGetLastError() != cudaSuccess) return PSGLD_ERR_CUDA;
    return PSGLD_OK;
}
