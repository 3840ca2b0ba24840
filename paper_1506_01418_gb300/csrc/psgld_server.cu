// psgld_server.cu -- a native serving loop: continuous batching of dense
// factorisation jobs on one GPU (psgld_server_* in include/psgld.h).
//
// Two worker threads.  The admission thread reads back and releases jobs
// whose last sweep has run (posterior means to the caller's buffers), and
// admits waiting jobs in arrival order while their estimated device memory
// fits the budget (context, data and factor copies with their input checks
// on the admission stream).  The batch thread takes set-up jobs into the
// batch (its stream waits for their set-up), hands finished ones back, and
// keeps up to max_inflight batch sweeps queued on the batch stream, each one
// psgld_batch_sweep of one sweep over every job with sweeps left; it never
// waits for a set-up or a read-back.  A context passes from one thread to
// the other through the queues under the mutex.  Submission and polling
// only touch the queues.  Contexts allocate from the device's stream-ordered memory pool
// (cudaMallocAsync / cudaFreeAsync), whose release threshold is raised so
// that freed memory stays cached: releasing a finished job waits for
// nothing but its own work.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <limits>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "psgld_context.cuh"

namespace {

using Clock = std::chrono::steady_clock;

void *pool_alloc(size_t bytes, void *stream, void *)
{
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pool_free(void *p, void *stream, void *)
{
    if (cudaFreeAsync(p, static_cast<cudaStream_t>(stream)) != cudaSuccess) cudaGetLastError();
}

// An event shared by the jobs whose last sweep it follows and by the queue
// of batch sweeps in flight; destroyed with its last holder.
struct Ev {
    cudaEvent_t e = nullptr;
    Ev() { cudaEventCreateWithFlags(&e, cudaEventDisableTiming); }
    ~Ev() { if (e) cudaEventDestroy(e); }
    Ev(const Ev &) = delete;
    Ev &operator=(const Ev &) = delete;
};

struct Job {
    int64_t id = 0;
    psgld_job spec{};
    Clock::time_point t_submit;
    size_t bytes = 0;
    psgld_ctx *ctx = nullptr;
    int left = 0;
    cudaEvent_t ready = nullptr;       // recorded on the admission stream after set-up
    std::shared_ptr<Ev> last;          // follows the job's last sweep
};

}  // namespace

struct psgld_server {
    size_t budget = 0, used = 0, peak = 0;
    int max_inflight = 3;
    int device = 0;
    cudaStream_t batch = nullptr, adm = nullptr;
    psgld_allocator allocator{};

    std::mutex m;
    std::condition_variable cv;
    // guarded by m: submitted jobs waiting for memory, jobs set up and not
    // yet in the batch, jobs whose last sweep has run (to read back)
    std::deque<Job *> waiting, ready, retire;
    std::vector<std::pair<int64_t, double>> done;   // finished since the last poll
    int64_t next_id = 0, submitted = 0, finished = 0;
    bool stop = false;
    std::string err, err_copy;
    int64_t sweeps = 0;
    double jobs_in_sweeps = 0.0;

    // the batch thread's own state
    std::vector<Job *> active;
    std::deque<std::shared_ptr<Ev>> inflight;
    std::thread admit_thread, batch_thread;
};

namespace {

void report(psgld_server *s, Job *j, double latency, const std::string &why)
{
    std::lock_guard<std::mutex> lk(s->m);
    s->done.emplace_back(j->id, latency);
    s->used -= j->bytes;
    s->finished += 1;
    if (!why.empty()) s->err = why;
    s->cv.notify_all();
}

// Context, data and factors of an admitted job; false (job reported
// failed) if any step is refused.
bool setup(psgld_server *s, Job *j)
{
    const psgld_job &q = j->spec;
    psgld_ctx *c = nullptr;
    psgld_status st = psgld::create_context(q.I, q.J, q.K, q.B, q.tweedie_p, q.phi, &q.prior, &s->allocator, &c);
    if (st == PSGLD_OK) st = psgld_set_options(c, &q.options);
    if (st == PSGLD_OK) st = psgld_set_data_dense(c, q.V_dev, q.ldv, s->adm);
    if (st == PSGLD_OK) st = psgld_set_factors(c, q.W0_dev, q.Ht0_dev, s->adm);
    if (st == PSGLD_OK && (cudaEventCreateWithFlags(&j->ready, cudaEventDisableTiming) != cudaSuccess ||
                           cudaEventRecord(j->ready, s->adm) != cudaSuccess)) {
        cudaGetLastError();
        st = PSGLD_ERR_CUDA;
    }
    if (st != PSGLD_OK) {
        const std::string why = c ? std::string("job setup: ") + psgld_last_error(c) : "job setup: context";
        if (c) psgld_destroy(c);
        if (j->ready) cudaEventDestroy(j->ready);
        report(s, j, -1.0, why);
        delete j;
        return false;
    }
    j->ctx = c;
    j->left = q.sweeps;
    return true;
}

void finish(psgld_server *s, Job *j)
{
    std::string why;
    const psgld_status st = psgld_posterior_mean(j->ctx, j->spec.Wmean_host, nullptr, j->spec.Hmean_host,
                                                 nullptr, nullptr);
    if (st != PSGLD_OK) why = std::string("job read-back: ") + psgld_last_error(j->ctx);
    psgld_destroy(j->ctx);
    const double lat = std::chrono::duration<double>(Clock::now() - j->t_submit).count();
    report(s, j, st == PSGLD_OK ? lat : -1.0, why);
    delete j;
}

// Admission thread: reads back and releases finished jobs first (that frees
// memory), then sets up the head of the queue when it fits.
void admit_loop(psgld_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->m);
    for (;;) {
        if (!s->retire.empty()) {
            Job *j = s->retire.front();
            s->retire.pop_front();
            lk.unlock();
            finish(s, j);
            lk.lock();
            continue;
        }
        if (!s->waiting.empty() && s->used + s->waiting.front()->bytes <= s->budget) {
            Job *j = s->waiting.front();
            s->waiting.pop_front();
            s->used += j->bytes;
            s->peak = std::max(s->peak, s->used);
            lk.unlock();
            const bool ok = setup(s, j);
            lk.lock();
            if (ok) {
                s->ready.push_back(j);
                s->cv.notify_all();
            }
            continue;
        }
        if (s->stop && s->finished == s->submitted) break;
        s->cv.wait_for(lk, std::chrono::milliseconds(1));
    }
}

// Batch thread: takes set-up jobs into the batch, hands finished ones to
// the admission thread, and keeps up to max_inflight batch sweeps queued.
void batch_loop(psgld_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        bool did = false;
        std::vector<Job *> joined;
        {
            std::lock_guard<std::mutex> lk(s->m);
            joined.assign(s->ready.begin(), s->ready.end());
            s->ready.clear();
        }
        for (Job *j : joined) {
            cudaStreamWaitEvent(s->batch, j->ready, 0);    // its sweeps start after its set-up
            cudaEventDestroy(j->ready);
            j->ready = nullptr;
            s->active.push_back(j);
            did = true;
        }
        for (size_t k = 0; k < s->active.size();) {
            Job *j = s->active[k];
            if (j->left == 0 && cudaEventQuery(j->last->e) == cudaSuccess) {
                s->active.erase(s->active.begin() + (std::ptrdiff_t)k);
                j->last.reset();
                std::lock_guard<std::mutex> lk(s->m);
                s->retire.push_back(j);
                s->cv.notify_all();
                did = true;
            } else {
                ++k;
            }
        }
        while (!s->inflight.empty() && cudaEventQuery(s->inflight.front()->e) == cudaSuccess)
            s->inflight.pop_front();
        if ((int)s->inflight.size() < s->max_inflight) {
            std::vector<psgld_ctx *> live;
            for (Job *j : s->active)
                if (j->left > 0) live.push_back(j->ctx);
            if (!live.empty()) {
                const psgld_status st = psgld_batch_sweep(live.data(), (int32_t)live.size(), 1, s->batch);
                auto ev = std::make_shared<Ev>();
                cudaEventRecord(ev->e, s->batch);
                if (st != PSGLD_OK) {
                    // the batch was refused or failed: its jobs end failed
                    const std::string why = std::string("batch sweep: ") + psgld_last_error(live[0]);
                    cudaStreamSynchronize(s->batch);
                    for (Job *j : s->active) {
                        psgld_destroy(j->ctx);
                        report(s, j, -1.0, why);
                        delete j;
                    }
                    s->active.clear();
                } else {
                    for (Job *j : s->active) {
                        if (j->left <= 0) continue;
                        j->left -= 1;
                        if (j->left == 0) j->last = ev;
                    }
                    s->inflight.push_back(ev);
                    std::lock_guard<std::mutex> lk(s->m);
                    s->sweeps += 1;
                    s->jobs_in_sweeps += (double)live.size();
                }
                did = true;
            }
        }
        std::unique_lock<std::mutex> lk(s->m);
        if (s->stop && s->finished == s->submitted) break;
        if (!did) s->cv.wait_for(lk, std::chrono::microseconds(50));
    }
    cudaStreamSynchronize(s->batch);
    s->inflight.clear();
}

}  // namespace

extern "C" {

psgld_status psgld_server_create(size_t hbm_budget, int32_t max_inflight, psgld_server **out)
{
    if (!out) return PSGLD_ERR_ARG;
    *out = nullptr;
    if (hbm_budget == 0 || max_inflight < 1) return PSGLD_ERR_ARG;
    psgld_server *s = new (std::nothrow) psgld_server();
    if (!s) return PSGLD_ERR_OOM;
    s->budget = hbm_budget;
    s->max_inflight = max_inflight;
    cudaGetDevice(&s->device);
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);    // hi: the most urgent
    if (cudaStreamCreateWithPriority(&s->batch, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&s->adm, cudaStreamNonBlocking, hi) != cudaSuccess) {
        cudaGetLastError();
        if (s->batch) cudaStreamDestroy(s->batch);
        delete s;
        return PSGLD_ERR_CUDA;
    }
    // keep freed blocks in the pool instead of returning them to the driver
    cudaMemPool_t pool = nullptr;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
        uint64_t keep = std::numeric_limits<uint64_t>::max();
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    s->allocator.alloc = pool_alloc;
    s->allocator.free = pool_free;
    s->allocator.user = nullptr;
    try {
        s->admit_thread = std::thread(admit_loop, s);
        s->batch_thread = std::thread(batch_loop, s);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->m);
            s->stop = true;
        }
        s->cv.notify_all();
        if (s->admit_thread.joinable()) s->admit_thread.join();
        cudaStreamDestroy(s->batch);
        cudaStreamDestroy(s->adm);
        delete s;
        return PSGLD_ERR_OOM;
    }
    *out = s;
    return PSGLD_OK;
}

psgld_status psgld_server_submit(psgld_server *s, const psgld_job *job, int64_t *id)
{
    if (!s || !job || !id) return PSGLD_ERR_ARG;
    if (job->sweeps < 1 || !job->V_dev || !job->W0_dev || !job->Ht0_dev || job->ldv < job->J)
        return PSGLD_ERR_ARG;
    if (job->options.dense_path < 1 || job->options.dense_path > 3) return PSGLD_ERR_ARG;
    const int64_t est = psgld_estimate_device_bytes(job->I, job->J, job->K, job->B, 0, job->options.dense_path,
                                                    job->options.dense_v_bf16);
    if (est <= 0) return PSGLD_ERR_ARG;
    if ((size_t)est > s->budget) return PSGLD_ERR_SIZE;
    Job *j = new (std::nothrow) Job();
    if (!j) return PSGLD_ERR_OOM;
    j->spec = *job;
    j->bytes = (size_t)est;
    j->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->m);
        if (s->stop) {
            delete j;
            return PSGLD_ERR_STATE;
        }
        j->id = s->next_id++;
        s->submitted += 1;
        s->waiting.push_back(j);
        *id = j->id;
    }
    s->cv.notify_all();
    return PSGLD_OK;
}

int32_t psgld_server_poll(psgld_server *s, int64_t *ids, double *lat, int32_t max)
{
    if (!s || max < 1) return 0;
    std::lock_guard<std::mutex> lk(s->m);
    const int32_t n = (int32_t)std::min<size_t>((size_t)max, s->done.size());
    for (int32_t k = 0; k < n; ++k) {
        if (ids) ids[k] = s->done[k].first;
        if (lat) lat[k] = s->done[k].second;
    }
    s->done.erase(s->done.begin(), s->done.begin() + n);
    return n;
}

psgld_status psgld_server_wait_idle(psgld_server *s, double timeout_s)
{
    if (!s) return PSGLD_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->m);
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                          std::chrono::duration<double>(std::max(0.0, timeout_s)));
    const bool ok = s->cv.wait_until(lk, until, [s] { return s->finished == s->submitted; });
    return ok ? PSGLD_OK : PSGLD_ERR_TIMEOUT;
}

psgld_status psgld_server_stats(psgld_server *s, int64_t *sweeps, double *jobs_per_sweep, size_t *peak)
{
    if (!s) return PSGLD_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->m);
    if (sweeps) *sweeps = s->sweeps;
    if (jobs_per_sweep) *jobs_per_sweep = s->sweeps ? s->jobs_in_sweeps / (double)s->sweeps : 0.0;
    if (peak) *peak = s->peak;
    return PSGLD_OK;
}

const char *psgld_server_last_error(psgld_server *s)
{
    if (!s) return "";
    std::lock_guard<std::mutex> lk(s->m);
    s->err_copy = s->err;     // stable until the next call of this function
    return s->err_copy.c_str();
}

void psgld_server_destroy(psgld_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->m);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->admit_thread.joinable()) s->admit_thread.join();
    if (s->batch_thread.joinable()) s->batch_thread.join();
    cudaStreamDestroy(s->batch);
    cudaStreamDestroy(s->adm);
    delete s;
}

}  // extern "C"
