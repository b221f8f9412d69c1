// Serving loop with continuous batching (no counterpart in the paper): jobs
// arrive over time, are admitted by free slots and a device-memory budget,
// join the running batch at the next block boundary, and leave it when their
// steps are done.  Job memory comes from a private stream-ordered pool, so
// creating and destroying jobs does not synchronise the device while the
// batch runs.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <string>
#include <thread>
#include <vector>

#include "handle.h"

using namespace stg::host;

namespace {

thread_local std::string g_serve_error;

int sfail(int code, const std::string &msg)
{
    g_serve_error = msg;
    return code;
}

struct Pool {
    cudaMemPool_t pool = nullptr;
    cudaStream_t s = nullptr;
};

void *pool_alloc(size_t bytes, void *ctx)
{
    Pool *p = static_cast<Pool *>(ctx);
    void *ptr = nullptr;
    if (cudaMallocFromPoolAsync(&ptr, bytes, p->pool, p->s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaStreamSynchronize(p->s) != cudaSuccess) return nullptr;
    return ptr;
}

void pool_free(void *ptr, size_t, void *ctx)
{
    Pool *p = static_cast<Pool *>(ctx);
    cudaFreeAsync(ptr, p->s);
}

enum class Phase { Batched, Draining, Done };

struct Running {
    int job = -1;
    stg_lbm *h = nullptr;
    int64_t remaining = 0;
    int64_t bytes = 0;
    Phase phase = Phase::Batched;
    cudaEvent_t fin = nullptr;
};

double percentile(std::vector<double> v, double q)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    // nearest-rank percentile
    const size_t k = (size_t)std::ceil(q * (double)v.size());
    return v[std::min(v.size() - 1, k > 0 ? k - 1 : 0)];
}

}  // namespace

extern "C" {

const char *stg_serve_last_error(void) { return g_serve_error.c_str(); }

int stg_serve_run(const stg_job *jobs, int32_t n_jobs, const stg_serve_config *cfg, void *stream,
                  stg_job_result *results, stg_serve_report *report)
{
    const Range range("stg_serve_run");
    if (n_jobs < 0 || (n_jobs > 0 && (!jobs || !results)) || !cfg || !(cfg->hbm_budget_bytes > 0.0))
        return sfail(STG_ERR_INVALID, "serve: bad arguments");
    for (int32_t i = 0; i < n_jobs; ++i)
        if (!jobs[i].domain || jobs[i].steps < 1 || !(jobs[i].arrival_s >= 0.0))
            return sfail(STG_ERR_INVALID, "serve: job " + std::to_string(i) + " needs a domain, steps >= 1, arrival >= 0");
    std::vector<int> order(n_jobs);
    for (int32_t i = 0; i < n_jobs; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return jobs[a].arrival_s < jobs[b].arrival_s; });
    std::vector<int64_t> est(n_jobs, 0);
    for (int32_t i = 0; i < n_jobs; ++i) {
        results[i] = stg_job_result{};
        results[i].status = -1;
        if (stg_lbm_estimate_bytes(jobs[i].domain, jobs[i].stg, &est[i]) != STG_OK) est[i] = -1;
        results[i].device_bytes = est[i];
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return sfail(STG_ERR_CUDA, "cudaGetDevice");
    Pool pool;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&pool.pool, &props) != cudaSuccess) return sfail(STG_ERR_CUDA, "cudaMemPoolCreate");
    uint64_t keep = UINT64_MAX;  // keep freed blocks in the pool for the next jobs
    cudaMemPoolSetAttribute(pool.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (cudaStreamCreateWithFlags(&pool.s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaMemPoolDestroy(pool.pool);
        return sfail(STG_ERR_CUDA, "cudaStreamCreate");
    }
    stg_allocator alloc{pool_alloc, pool_free, &pool};
    cudaStream_t bstream = static_cast<cudaStream_t>(stream);
    bool own_bstream = false;
    if (!bstream) {
        if (cudaStreamCreateWithFlags(&bstream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaStreamDestroy(pool.s);
            cudaMemPoolDestroy(pool.pool);
            return sfail(STG_ERR_CUDA, "cudaStreamCreate");
        }
        own_bstream = true;
    }
    stg_batch *b = nullptr;
    if (stg_batch_create(bstream, &b) != STG_OK) {
        if (own_bstream) cudaStreamDestroy(bstream);
        cudaStreamDestroy(pool.s);
        cudaMemPoolDestroy(pool.pool);
        return sfail(STG_ERR_CUDA, "batch create");
    }
    // at most two blocks in flight, so admission and completion decisions track the GPU
    cudaEvent_t ring[2] = {nullptr, nullptr};
    if (cudaEventCreateWithFlags(&ring[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ring[1], cudaEventDisableTiming) != cudaSuccess) {
        if (ring[0]) cudaEventDestroy(ring[0]);
        stg_batch_destroy(b);
        if (own_bstream) cudaStreamDestroy(bstream);
        cudaStreamDestroy(pool.s);
        cudaMemPoolDestroy(pool.pool);
        return sfail(STG_ERR_CUDA, "cudaEventCreate");
    }
    bool ring_used[2] = {false, false};
    int ring_i = 0;

    const auto t_start = std::chrono::steady_clock::now();
    auto now_s = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count(); };
    std::vector<Running> run;
    size_t next = 0;
    int64_t used = 0, peak_used = 0, cell_updates = 0;
    int32_t peak_active = 0;
    int64_t completed = 0, failed = 0;
    int rc_run = STG_OK;
    double last_finish = 0.0;

    auto finish = [&](Running &r, int status) {
        stg_job_result &res = results[r.job];
        const stg_job &jb = jobs[r.job];
        res.status = status;
        if (status == STG_OK) {
            stg_stats st{};
            st.mean_sum = jb.mean_sum;
            st.rey_sum = jb.rey_sum;
            const int rc = stg_lbm_stats(r.h, &st);
            res.status = rc;
            res.n_samples = st.n_samples;
            res.mass = st.mass;
            res.mass0 = st.mass0;
            if (rc == STG_OK)
                cell_updates += (int64_t)jb.domain->nx * jb.domain->ny * jb.domain->nz * jb.steps;
        }
        res.finish_s = now_s();
        res.latency_s = res.finish_s - jb.arrival_s;
        last_finish = std::max(last_finish, res.finish_s);
        if (res.status == STG_OK) ++completed;
        else ++failed;
        if (r.fin) cudaEventDestroy(r.fin);
        r.fin = nullptr;
        stg_lbm_destroy(r.h);  // leaves the batch first if still a member
        r.h = nullptr;
        used -= r.bytes;
        r.phase = Phase::Done;
    };
    // a running job leaves the batch; its remaining steps go to its own stream
    auto drain = [&](Running &r) -> int {
        int rc = STG_OK;
        if (r.h->batch) rc = stg_batch_remove(b, r.h);
        if (rc == STG_OK && r.remaining > 0) rc = stg_lbm_step(r.h, r.remaining);
        r.remaining = 0;
        if (rc == STG_OK && cudaEventCreateWithFlags(&r.fin, cudaEventDisableTiming) != cudaSuccess) rc = STG_ERR_CUDA;
        if (rc == STG_OK && cudaEventRecord(r.fin, r.h->stream) != cudaSuccess) rc = STG_ERR_CUDA;
        r.phase = Phase::Draining;
        return rc;
    };

    while (rc_run == STG_OK && (completed + failed) < n_jobs) {
        const double t = now_s();
        // admissions, in arrival order
        int active = 0;
        for (const Running &r : run) active += r.phase != Phase::Done;
        while (next < order.size() && jobs[order[next]].arrival_s <= t &&
               (cfg->max_active <= 0 || active < cfg->max_active)) {
            const int j = order[next];
            const stg_job &jb = jobs[j];
            if (est[j] < 0 || (double)est[j] > cfg->hbm_budget_bytes) {
                results[j].status = est[j] < 0 ? STG_ERR_INVALID : STG_ERR_NOMEM;
                results[j].finish_s = now_s();
                ++failed;
                ++next;
                continue;
            }
            if ((double)(used + est[j]) > cfg->hbm_budget_bytes) break;  // wait for memory
            Running r;
            r.job = j;
            r.bytes = est[j];
            const int rc = stg_lbm_create(jb.domain, jb.rans, jb.stg, jb.seed, &alloc, nullptr, &r.h);
            results[j].admit_s = now_s();
            ++next;
            if (rc != STG_OK) {
                results[j].status = rc;
                results[j].finish_s = results[j].admit_s;
                ++failed;
                continue;
            }
            used += r.bytes;
            peak_used = std::max(peak_used, used);
            r.remaining = jb.steps;
            if (stg_batch_add(b, r.h) != STG_OK) {
                if (drain(r) != STG_OK) {
                    run.push_back(r);
                    finish(run.back(), STG_ERR_CUDA);
                    continue;
                }
            }
            run.push_back(r);
            ++active;
        }
        peak_active = std::max(peak_active, active);
        // jobs whose remaining steps do not fill a block finish on their own stream
        const int B = stg_batch_block_steps(b);
        for (Running &r : run)
            if (r.phase == Phase::Batched && r.remaining < B && drain(r) != STG_OK) finish(r, STG_ERR_CUDA);
        // one block for the batch
        if (stg_batch_size(b) > 0) {
            if (ring_used[ring_i]) cudaEventSynchronize(ring[ring_i]);
            const int rc = stg_batch_step(b, B);
            if (rc != STG_OK) {
                // a member failed its check: take the failed ones out, keep the rest
                bool any = false;
                for (Running &r : run)
                    if (r.phase == Phase::Batched && r.h->sticky) {
                        finish(r, r.h->sticky);
                        any = true;
                    }
                if (!any) rc_run = rc;
                continue;
            }
            for (Running &r : run)
                if (r.phase == Phase::Batched) r.remaining -= B;
            cudaEventRecord(ring[ring_i], bstream);
            ring_used[ring_i] = true;
            ring_i ^= 1;
        }
        // completions
        bool progressed = false;
        for (Running &r : run) {
            if (r.phase != Phase::Draining) continue;
            const cudaError_t e = cudaEventQuery(r.fin);
            if (e == cudaSuccess) {
                finish(r, STG_OK);
                progressed = true;
            } else if (e != cudaErrorNotReady) {
                finish(r, STG_ERR_CUDA);
            }
        }
        run.erase(std::remove_if(run.begin(), run.end(), [](const Running &r) { return r.phase == Phase::Done; }),
                  run.end());
        if (stg_batch_size(b) == 0 && !progressed) {
            // idle or draining only: wait a little (until the next arrival at most)
            double wait = 2e-4;
            if (run.empty() && next < order.size()) wait = std::max(0.0, jobs[order[next]].arrival_s - now_s());
            std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.05)));
        }
    }

    for (Running &r : run)
        if (r.h) finish(r, rc_run != STG_OK ? rc_run : STG_ERR_CUDA);
    for (int32_t i = 0; i < n_jobs; ++i)  // never admitted because the run stopped
        if (results[i].status == -1) results[i].status = rc_run != STG_OK ? rc_run : STG_ERR_CUDA;
    stg_batch_destroy(b);
    if (own_bstream) cudaStreamDestroy(bstream);
    cudaEventDestroy(ring[0]);
    cudaEventDestroy(ring[1]);
    cudaStreamSynchronize(pool.s);
    cudaStreamDestroy(pool.s);
    cudaMemPoolDestroy(pool.pool);

    if (report) {
        std::vector<double> lat;
        for (int32_t i = 0; i < n_jobs; ++i)
            if (results[i].status == STG_OK) lat.push_back(results[i].latency_s);
        stg_serve_report rp{};
        rp.wall_s = last_finish;
        rp.completed = completed;
        rp.failed = failed;
        rp.cell_updates = cell_updates;
        rp.jobs_per_s = last_finish > 0.0 ? (double)completed / last_finish : 0.0;
        rp.aggregate_mlups = last_finish > 0.0 ? (double)cell_updates / last_finish / 1e6 : 0.0;
        rp.p50_latency_s = percentile(lat, 0.50);
        rp.p99_latency_s = percentile(lat, 0.99);
        double s = 0.0;
        for (double v : lat) s += v;
        rp.mean_latency_s = lat.empty() ? 0.0 : s / (double)lat.size();
        rp.peak_device_bytes = peak_used;
        rp.peak_active = peak_active;
        *report = rp;
    }
    if (rc_run != STG_OK) return sfail(rc_run, "serve: the batch failed");
    return STG_OK;
}

}  // extern "C"
