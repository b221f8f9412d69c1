// The lattice handle behind the C ABI and the host helpers that the batch
// executor and the serving loop share with the single-lattice entry points.
#pragma once

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "internal.h"
#include "stg_lbm.h"

struct stg_batch;

struct stg_lbm {
    stg_domain d{};
    stg_params p{};
    bool inout = false;
    bool aa = false;  // one lattice updated in place (lat[1] == lat[0])
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    stg_allocator alloc{};
    bool has_alloc = false;
    std::vector<std::pair<void *, size_t>> allocs;
    size_t P = 0, elem = 4;
    void *lat[2] = {nullptr, nullptr};
    float *ubc = nullptr, *uf = nullptr;  // ubc: inlet planes of steps t and t + 1, [2][3][nz][ny] by step parity
    float *spf = nullptr;  // sponge factor per column (nullptr: no sponge)
    int n_probes = 0;                     // velocity probes (stg_lbm_set_probes)
    int *probe_xyz = nullptr;             // device [3 n_probes]
    float *probe_buf = nullptr;           // device samples of one step_probed call
    size_t probe_cap = 0;                 // floats in probe_buf
    float *A = nullptr, *B = nullptr, *SQ = nullptr, *sig = nullptr, *a6 = nullptr, *u_int = nullptr;
    unsigned long long *phq = nullptr, *omq = nullptr;  // phi^n and omega^n as Q0.64 fractions of a turn
    int N = 0;
    float a_filter = 0.f;
    stg::StepCtl *ctl = nullptr;
    double *stat_mean = nullptr, *stat_rey = nullptr;
    float *stat_part = nullptr;  // z-group sums of a sampling step (vector kernels)
    double *mass_partial = nullptr, *mass_out = nullptr;
    unsigned *mass_counter = nullptr;
    double *m_partial = nullptr, *m_out = nullptr;
    unsigned *m_counter = nullptr;
    double *h_pinned = nullptr;  // [0]: last checked mass
    cudaEvent_t ev_check = nullptr, ev_done = nullptr;
    cudaStream_t side = nullptr;                       // branch for the edge kernel
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool check_pending = false;
    int64_t t = 0, t0_stats = 0;
    double mass0 = 0.0;
    int sticky = STG_OK;
    std::string err;
    // single steps by [parity][sampling step]; blocks of block_steps steps that
    // start at a step index divisible by the sampling period, by parity
    cudaGraphExec_t g_single[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    cudaGraphExec_t g_block[2] = {nullptr, nullptr};
    int block_steps = 16;
    stg_info info{};
    double timeout_s = 900.0;
    int interior = 0;  // STG_LBM_INTERIOR=scalar|pair overrides the interior kernel choice
    stg_tile tile{1, 8, 24, 0};
    stg_batch *batch = nullptr;  // the batch this lattice belongs to (its steps run there)
};

namespace stg {
namespace host {

// NVTX range for the host side of an entry point (visible in a profiler's
// timeline; inert without one).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

int fail(stg_lbm *h, int code, const std::string &msg);
int cuda_fail(stg_lbm *h, cudaError_t e, const char *what);
// one step of h with the given parity on h->stream (and h->side); `stats`
// selects the sampling-step kernels
cudaError_t enqueue_step(stg_lbm *h, int parity, bool stats);
bool is_stats_step(const stg_lbm *h, int64_t t);
// evaluate the last completed mass check (non-blocking)
int poll_check(stg_lbm *h);
// after the steps that took h from t_before to h->t were enqueued on
// h->stream: queue the read-back of the last mass check, if one ran
int queue_check_readback(stg_lbm *h, int64_t t_before);
// wait for h->stream (bounded by the handle's timeout)
int wait_stream(stg_lbm *h);
// one plain (non-sampling) step pass from the current state with `tile`, on
// stream s; it does not advance the step counter, the filter or the
// statistics (two lattices: it recomputes what the next real step writes).
// In place the pass updates the lattice: the k-th pass of a trial series
// takes the parity of step t + k (so the arrangement stays valid), and the
// caller brackets the series with save_trial_state / restore_trial_state.
cudaError_t trial_pass(stg_lbm *h, const stg_tile &tile, cudaStream_t s, int k = 0);
// in place only: copy the populations and the device step counters to host
// memory before a trial series, and back afterwards (no-ops for two lattices)
int save_trial_state(stg_lbm *h, std::vector<unsigned char> &pops, stg::StepCtl &ctl);
int restore_trial_state(stg_lbm *h, const std::vector<unsigned char> &pops, const stg::StepCtl &ctl);
// set the tile and re-capture the handle's own graphs
int apply_tile(stg_lbm *h, const stg_tile &tile);
// the autotuner's candidate tiles
const stg_tile *tile_candidates(int *n);
// take h out of its batch (batch.cu)
void batch_detach(stg_lbm *h);

}  // namespace host
}  // namespace stg
