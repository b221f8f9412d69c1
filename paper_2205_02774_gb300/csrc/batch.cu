// Batch executor: many independent lattices advanced together.  The paper runs
// one channel at a time; this is the GPU-side answer to running an ensemble of
// them.  One CUDA graph per block of B steps holds every member's chain of B
// steps (inlet kernel, then the step pass with its forked boundary branch) as
// its own branch between one fork and one join, so the members' kernels
// overlap on the GPU and no member waits for another between steps; a block is
// one graph launch.  A member runs exactly the kernels and arguments it runs
// alone, so its populations and statistics are bit-identical to a solo run.
// While members come and go, each member's own graph of B steps is launched
// on its branch instead (no capture of the whole batch per change); the
// combined graph is captured once the membership has been stable for a few
// blocks.
#include <algorithm>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include "handle.h"

using namespace stg::host;

struct stg_batch {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<stg_lbm *> m;          // members
    std::vector<cudaStream_t> ms;      // each member's branch stream
    std::vector<cudaEvent_t> join;     // each member's join event
    std::vector<int64_t> t_cap;        // member step counters when the block graph was captured
    std::vector<cudaGraphExec_t> mg;   // each member's own graph of B steps (used while membership changes)
    std::vector<int64_t> mg_t;         // member step counter when its graph was captured
    std::vector<int> mg_B;             // B of that capture
    int stable = 0;                    // blocks run since the membership last changed
    cudaEvent_t fork = nullptr, done = nullptr, e0 = nullptr, e1 = nullptr;
    cudaGraphExec_t g = nullptr;
    int B = 16;  // steps per block graph: a multiple of 2 and of every member's sampling period
    bool dirty = true;
    std::string err;
    double timeout_s = 900.0;
};

namespace {

thread_local std::string g_batch_error;

int bfail(stg_batch *b, int code, const std::string &msg)
{
    if (b) b->err = msg;
    else g_batch_error = msg;
    return code;
}

int bcuda(stg_batch *b, cudaError_t e, const char *what)
{
    return bfail(b, STG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define BCK(call)                                           \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return bcuda(b, e_, #call);  \
    } while (0)

int64_t gcd64(int64_t a, int64_t c)
{
    while (c) {
        const int64_t r = a % c;
        a = c;
        c = r;
    }
    return a;
}

// Smallest multiple of lcm(2, sampling periods) that is >= 16; -1 when the
// common multiple exceeds 256 steps.
int block_len(const std::vector<stg_lbm *> &m, const stg_lbm *extra)
{
    int64_t L = 2;
    auto acc = [&L](const stg_lbm *h) {
        const int k = h->d.stats_every;
        if (k > 0) L = L / gcd64(L, k) * k;
    };
    for (const stg_lbm *h : m) acc(h);
    if (extra) acc(extra);
    if (L > 256) return -1;
    return (int)(L * ((16 + L - 1) / L));
}

void drop_graph(stg_batch *b)
{
    if (b->g) cudaGraphExecDestroy(b->g);
    b->g = nullptr;
}

int index_of(const stg_batch *b, const stg_lbm *h)
{
    for (size_t d = 0; d < b->m.size(); ++d)
        if (b->m[d] == h) return (int)d;
    return -1;
}

// the batch stream waits for whatever each member has queued on its own stream
int order_after_members(stg_batch *b)
{
    for (stg_lbm *h : b->m) {
        BCK(cudaEventRecord(h->ev_done, h->stream));
        BCK(cudaStreamWaitEvent(b->stream, h->ev_done, 0));
    }
    return STG_OK;
}

// each member's own stream waits for the batch's work so far
int order_members_after(stg_batch *b)
{
    BCK(cudaEventRecord(b->done, b->stream));
    for (stg_lbm *h : b->m) BCK(cudaStreamWaitEvent(h->stream, b->done, 0));
    return STG_OK;
}

// Block graph of B steps from the members' current step counters.
int capture_block(stg_batch *b)
{
    const Range range("batch capture");
    drop_graph(b);
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(b->fork, b->stream);
    for (size_t d = 0; d < b->m.size() && e == cudaSuccess; ++d) {
        stg_lbm *h = b->m[d];
        const cudaStream_t own = h->stream;
        h->stream = b->ms[d];  // the member's steps go to its branch
        e = cudaStreamWaitEvent(h->stream, b->fork, 0);
        for (int s = 0; s < b->B && e == cudaSuccess; ++s)
            e = enqueue_step(h, (int)((h->t + s) & 1), is_stats_step(h, h->t + s));
        if (e == cudaSuccess) e = cudaEventRecord(b->join[d], h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join[d], 0);
        h->stream = own;
    }
    const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(b, e, "batch capture");
    }
    if (e2 != cudaSuccess) return bcuda(b, e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->g, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->g = nullptr;
        return bcuda(b, e, "cudaGraphInstantiate");
    }
    b->t_cap.resize(b->m.size());
    for (size_t d = 0; d < b->m.size(); ++d) b->t_cap[d] = b->m[d]->t;
    b->dirty = false;
    return STG_OK;
}

constexpr int STABLE_BLOCKS = 3;

// Graph of B steps of member d alone, on its branch stream.
int capture_member(stg_batch *b, size_t d)
{
    const Range range("member capture");
    stg_lbm *h = b->m[d];
    if (b->mg[d]) cudaGraphExecDestroy(b->mg[d]);
    b->mg[d] = nullptr;
    cudaGraph_t g = nullptr;
    const cudaStream_t own = h->stream;
    h->stream = b->ms[d];
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = cudaSuccess;
        for (int s = 0; s < b->B && e1 == cudaSuccess; ++s)
            e1 = enqueue_step(h, (int)((h->t + s) & 1), is_stats_step(h, h->t + s));
        e = cudaStreamEndCapture(h->stream, &g);
        if (e1 != cudaSuccess) e = e1;
    }
    h->stream = own;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(b, e, "member capture");
    }
    e = cudaGraphInstantiate(&b->mg[d], g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->mg[d] = nullptr;
        return bcuda(b, e, "cudaGraphInstantiate");
    }
    b->mg_t[d] = h->t;
    b->mg_B[d] = b->B;
    return STG_OK;
}

// One block through the members' own graphs, each on its branch.
int launch_member_graphs(stg_batch *b)
{
    BCK(cudaEventRecord(b->fork, b->stream));
    for (size_t d = 0; d < b->m.size(); ++d) {
        stg_lbm *h = b->m[d];
        if (!b->mg[d] || b->mg_B[d] != b->B || (h->t - b->mg_t[d]) % b->B != 0) {
            const int rc = capture_member(b, d);
            if (rc) return rc;
        }
        BCK(cudaStreamWaitEvent(b->ms[d], b->fork, 0));
        BCK(cudaGraphLaunch(b->mg[d], b->ms[d]));
        BCK(cudaEventRecord(b->join[d], b->ms[d]));
        BCK(cudaStreamWaitEvent(b->stream, b->join[d], 0));
    }
    return STG_OK;
}

// The block graph replays the members' step patterns (parity and sampling
// steps) only while every member has advanced a multiple of B since capture.
bool graph_valid(const stg_batch *b)
{
    if (!b->g || b->dirty || b->t_cap.size() != b->m.size()) return false;
    for (size_t d = 0; d < b->m.size(); ++d)
        if ((b->m[d]->t - b->t_cap[d]) % b->B != 0) return false;
    return true;
}

int wait_batch(stg_batch *b)
{
    BCK(cudaEventRecord(b->done, b->stream));
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaEventQuery(b->done);
        if (e == cudaSuccess) return STG_OK;
        if (e != cudaErrorNotReady) return bcuda(b, e, "cudaEventQuery");
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > b->timeout_s) return bfail(b, STG_ERR_TIMEOUT, "timed out waiting for the batch");
        std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 5 : 200));
    }
}

int remove_at(stg_batch *b, int d)
{
    stg_lbm *h = b->m[d];
    // the member's later work on its own stream follows the batch's work
    BCK(cudaEventRecord(b->done, b->stream));
    BCK(cudaStreamWaitEvent(h->stream, b->done, 0));
    cudaStreamDestroy(b->ms[d]);  // released once its queued work completes
    cudaEventDestroy(b->join[d]);
    if (b->mg[d]) cudaGraphExecDestroy(b->mg[d]);
    b->m.erase(b->m.begin() + d);
    b->ms.erase(b->ms.begin() + d);
    b->join.erase(b->join.begin() + d);
    b->mg.erase(b->mg.begin() + d);
    b->mg_t.erase(b->mg_t.begin() + d);
    b->mg_B.erase(b->mg_B.begin() + d);
    b->stable = 0;
    h->batch = nullptr;
    const int B = block_len(b->m, nullptr);
    b->B = B > 0 ? B : 16;
    b->dirty = true;
    drop_graph(b);
    return STG_OK;
}

}  // namespace

namespace stg {
namespace host {

void batch_detach(stg_lbm *h)
{
    if (!h || !h->batch) return;
    stg_batch *b = h->batch;
    const int d = index_of(b, h);
    if (d >= 0) remove_at(b, d);
    h->batch = nullptr;
}

}  // namespace host
}  // namespace stg

extern "C" {

int stg_batch_create(void *stream, stg_batch **out)
{
    if (!out) return bfail(nullptr, STG_ERR_INVALID, "out is NULL");
    *out = nullptr;
    stg_batch *b = new stg_batch();
    cudaError_t e = cudaSuccess;
    if (stream) {
        b->stream = static_cast<cudaStream_t>(stream);
    } else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&b->e0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->e1);
    if (e != cudaSuccess) {
        bcuda(nullptr, e, "batch stream / events");
        stg_batch_destroy(b);
        return STG_ERR_CUDA;
    }
    *out = b;
    return STG_OK;
}

int stg_batch_add(stg_batch *b, stg_lbm *h)
{
    if (!b) return bfail(nullptr, STG_ERR_INVALID, "batch is NULL");
    if (!h) return bfail(b, STG_ERR_INVALID, "lattice is NULL");
    if (h->batch) return bfail(b, STG_ERR_INVALID, "the lattice is already in a batch");
    int dev = -1;
    BCK(cudaGetDevice(&dev));
    if (dev != h->device) return bfail(b, STG_ERR_INVALID, "the lattice lives on another device");
    const int B = block_len(b->m, h);
    if (B < 0) return bfail(b, STG_ERR_INVALID, "sampling periods have no common multiple <= 256");
    cudaStream_t s = nullptr;
    cudaEvent_t j = nullptr;
    BCK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    if (cudaEventCreateWithFlags(&j, cudaEventDisableTiming) != cudaSuccess) {
        cudaStreamDestroy(s);
        return bfail(b, STG_ERR_CUDA, "cudaEventCreate");
    }
    b->m.push_back(h);
    b->ms.push_back(s);
    b->join.push_back(j);
    b->mg.push_back(nullptr);
    b->mg_t.push_back(0);
    b->mg_B.push_back(0);
    b->stable = 0;
    h->batch = b;
    b->B = B;
    b->dirty = true;
    drop_graph(b);
    return STG_OK;
}

int stg_batch_remove(stg_batch *b, stg_lbm *h)
{
    if (!b) return bfail(nullptr, STG_ERR_INVALID, "batch is NULL");
    const int d = h ? index_of(b, h) : -1;
    if (d < 0) return bfail(b, STG_ERR_INVALID, "not a member of this batch");
    return remove_at(b, d);
}

int stg_batch_size(const stg_batch *b) { return b ? (int)b->m.size() : 0; }

int stg_batch_block_steps(const stg_batch *b) { return b ? b->B : 0; }

int stg_batch_step(stg_batch *b, int64_t n)
{
    const Range range("stg_batch_step");
    if (!b) return bfail(nullptr, STG_ERR_INVALID, "batch is NULL");
    if (n < 0) return bfail(b, STG_ERR_INVALID, "negative step count");
    for (size_t d = 0; d < b->m.size(); ++d) {
        stg_lbm *h = b->m[d];
        int rc = poll_check(h);
        if (rc == STG_OK && h->sticky) rc = h->sticky;
        if (rc) return bfail(b, rc, "member " + std::to_string(d) + ": " + h->err);
    }
    if (b->m.empty() || n == 0) return STG_OK;
    std::vector<int64_t> t_before(b->m.size());
    for (size_t d = 0; d < b->m.size(); ++d) t_before[d] = b->m[d]->t;
    int rc = order_after_members(b);
    if (rc) return rc;
    while (n >= b->B) {
        if (!graph_valid(b) && b->stable >= STABLE_BLOCKS) {
            rc = capture_block(b);
            if (rc) return rc;
        }
        if (graph_valid(b)) {
            BCK(cudaGraphLaunch(b->g, b->stream));
        } else {
            rc = launch_member_graphs(b);
            if (rc) return rc;
        }
        for (stg_lbm *h : b->m) h->t += b->B;
        n -= b->B;
        ++b->stable;
    }
    if (n > 0) {
        // the rest: each member's own single-step graphs on its branch
        BCK(cudaEventRecord(b->fork, b->stream));
        for (size_t d = 0; d < b->m.size(); ++d) {
            stg_lbm *h = b->m[d];
            BCK(cudaStreamWaitEvent(b->ms[d], b->fork, 0));
            for (int64_t s = 0; s < n; ++s) {
                BCK(cudaGraphLaunch(h->g_single[h->t & 1][is_stats_step(h, h->t) ? 1 : 0], b->ms[d]));
                h->t += 1;
            }
            BCK(cudaEventRecord(b->join[d], b->ms[d]));
            BCK(cudaStreamWaitEvent(b->stream, b->join[d], 0));
        }
    }
    rc = order_members_after(b);
    if (rc) return rc;
    for (size_t d = 0; d < b->m.size(); ++d) {
        rc = queue_check_readback(b->m[d], t_before[d]);
        if (rc) return bfail(b, rc, "member " + std::to_string(d) + ": " + b->m[d]->err);
    }
    return STG_OK;
}

int stg_batch_sync(stg_batch *b)
{
    if (!b) return bfail(nullptr, STG_ERR_INVALID, "batch is NULL");
    return wait_batch(b);
}

int stg_batch_autotune(stg_batch *b, int32_t trial_passes, stg_tile *chosen)
{
    const Range range("stg_batch_autotune");
    if (!b) return bfail(nullptr, STG_ERR_INVALID, "batch is NULL");
    if (b->m.empty()) return bfail(b, STG_ERR_INVALID, "empty batch");
    if (trial_passes < 1 || trial_passes > 1000) return bfail(b, STG_ERR_INVALID, "trial_passes must be in [1, 1000]");
    for (stg_lbm *h : b->m)
        if (h->sticky) return bfail(b, h->sticky, "a member's earlier check failed");
    int ncand = 0;
    const stg_tile *cand = tile_candidates(&ncand);
    int rc = order_after_members(b);
    if (rc) return rc;
    // in-place members: their trial passes update the lattice, saved first and put back
    std::vector<std::vector<unsigned char>> keep(b->m.size());
    std::vector<stg::StepCtl> keep_ctl(b->m.size());
    for (size_t d = 0; d < b->m.size(); ++d) {
        rc = save_trial_state(b->m[d], keep[d], keep_ctl[d]);
        if (rc) return bfail(b, rc, "member " + std::to_string(d) + ": " + b->m[d]->err);
    }
    stg_tile best = b->m[0]->tile;
    float best_ms = -1.f;
    for (int c = 0; c < ncand; ++c) {
        // all members' plain passes from their current states, concurrently
        // (no state advance; see stg_lbm_autotune)
        for (int k = 0; k <= trial_passes; ++k) {
            if (k == 1) BCK(cudaEventRecord(b->e0, b->stream));
            BCK(cudaEventRecord(b->fork, b->stream));
            for (size_t d = 0; d < b->m.size(); ++d) {
                BCK(cudaStreamWaitEvent(b->ms[d], b->fork, 0));
                BCK(trial_pass(b->m[d], cand[c], b->ms[d], k));
                BCK(cudaEventRecord(b->join[d], b->ms[d]));
                BCK(cudaStreamWaitEvent(b->stream, b->join[d], 0));
            }
        }
        BCK(cudaEventRecord(b->e1, b->stream));
        BCK(cudaEventSynchronize(b->e1));
        float ms = 0.f;
        BCK(cudaEventElapsedTime(&ms, b->e0, b->e1));
        if (best_ms < 0.f || ms < best_ms) {
            best_ms = ms;
            best = cand[c];
        }
    }
    rc = order_members_after(b);
    if (rc) return rc;
    for (size_t d = 0; d < b->m.size(); ++d) {
        rc = restore_trial_state(b->m[d], keep[d], keep_ctl[d]);
        if (rc) return bfail(b, rc, "member " + std::to_string(d) + ": " + b->m[d]->err);
    }
    for (size_t d = 0; d < b->m.size(); ++d) {
        rc = apply_tile(b->m[d], best);
        if (rc) return bfail(b, rc, "member " + std::to_string(d) + ": " + b->m[d]->err);
    }
    b->dirty = true;
    drop_graph(b);
    for (size_t d = 0; d < b->m.size(); ++d) {
        if (b->mg[d]) cudaGraphExecDestroy(b->mg[d]);
        b->mg[d] = nullptr;
    }
    b->stable = 0;
    if (chosen) *chosen = best;
    return STG_OK;
}

void stg_batch_destroy(stg_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    while (!b->m.empty()) remove_at(b, (int)b->m.size() - 1);
    drop_graph(b);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->done) cudaEventDestroy(b->done);
    if (b->e0) cudaEventDestroy(b->e0);
    if (b->e1) cudaEventDestroy(b->e1);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char *stg_batch_last_error(const stg_batch *b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

}  // extern "C"
